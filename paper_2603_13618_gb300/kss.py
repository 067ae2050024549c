"""Thin Python binding of the C ABI in ``include/kss.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/libkss.so``; this module only
converts arguments: numpy arrays are host memory (``on_device=0``), torch CUDA
tensors are device memory (``on_device=1``).  PyTorch supplies device memory and the
stream.  There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkss.so")

KSS_OK = 0
KSS_WARN_NONPOSITIVE = 1
FP64, FP32, FP16DEV = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16dev": FP16DEV, FP64: FP64, FP32: FP32,
              FP16DEV: FP16DEV}

SENSORS = ("tau_ns", "c", "s", "e", "qh", "kn", "neq", "qe", "hr", "kl", "sigma_h",
           "sigma_kl", "alpha")
SENSOR_ID = {n: k for k, n in enumerate(SENSORS)}
FLAG_REFINE, FLAG_SWITCH, FLAG_NONPOS = 0x01, 0x02, 0x80
KERNELS = {"auto": 0, "vector": 1, "tma": 2}


class KssError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"kss error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("refine_sensor", ctypes.c_int32), ("refine_threshold", ctypes.c_double),
        ("switch_sensor", ctypes.c_int32), ("switch_threshold", ctypes.c_double),
        ("record_mask", ctypes.c_uint32), ("output_every", ctypes.c_int32),
        ("tile", ctypes.c_int32), ("stream", ctypes.c_void_p), ("own_stream", ctypes.c_int32),
        ("kernel", ctypes.c_int32), ("rho0", ctypes.c_double), ("dev_exp", ctypes.c_int32),
        ("dev_unscaled", ctypes.c_int32), ("tau2", ctypes.c_double),
    ]


class BatchTuning(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("ms_per_step", ctypes.c_double),
                ("multi_step", ctypes.c_int32)]


class Box(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("x1", ctypes.c_int32),
                ("y1", ctypes.c_int32)]


class AdjointConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nsteps", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("own_stream", ctypes.c_int32)]


_lib = None

# Every entry point declared in include/kss.h, with its ctypes signature.
_DP = ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "kss_version": (ctypes.c_int, []),
    "kss_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "kss_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "kss_config_default": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32]),
    "kss_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "kss_destroy": (None, [ctypes.c_void_p]),
    "kss_set_fields": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "kss_set_fields_f32": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "kss_set_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "kss_get_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "kss_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "kss_read_moments": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "kss_read_sensor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int]),
    "kss_read_flags": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "kss_read_stats": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "kss_get_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "kss_set_aar_region": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "kss_testing_expire_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "kss_testing_expire_mbarrier": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "kss_testing_fail_after": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "kss_testing_live_allocations": (ctypes.c_int64, []),
    "kss_get_aar_region": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "kss_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "kss_slab_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "kss_slab_edges": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int]),
    "kss_slab_set_halos": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int]),
    "kss_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Config),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "kss_batch_destroy": (None, [ctypes.c_void_p]),
    "kss_batch_member": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int32]),
    "kss_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "kss_batch_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchTuning)]),
    "kss_batch_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchTuning)]),
    "kss_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32,
                                          ctypes.POINTER(BatchTuning)]),
    "kss_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "kss_regrid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.c_int]),
    "kss_regrid_flags": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                        ctypes.c_void_p]),
    "kss_adjoint_create": (ctypes.c_int, [ctypes.POINTER(AdjointConfig),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "kss_adjoint_destroy": (None, [ctypes.c_void_p]),
    "kss_adjoint_forward": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_double, ctypes.c_int,
                                                                    _DP]),
    "kss_adjoint_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _DP, ctypes.c_int]),
    "kss_adjoint_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "kss_adjoint_set_multistep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "kss_step_f32_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                            ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                            ctypes.c_double, ctypes.c_int32, ctypes.c_int32]
                             + [ctypes.c_void_p] * 6),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libkss.so; raise if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, on_device) of a numpy array or torch tensor of the given dtype."""
    if _is_torch(a):
        import torch

        want = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8,
                np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be a C-contiguous numpy {np.dtype(dtype).name} array")
    return ctypes.c_void_p(a.ctypes.data), 0


def _dtype_of(a):
    """numpy dtype of a numpy array or torch tensor (None for anything else)."""
    if _is_torch(a):
        import torch

        return {torch.float32: np.float32, torch.float64: np.float64}.get(a.dtype)
    return a.dtype.type if isinstance(a, np.ndarray) else None


def _sensor(s) -> int:
    return SENSOR_ID[s] if isinstance(s, str) else int(s)


def _torch_stream_handle():
    import torch

    return torch.cuda.current_stream().cuda_stream


def make_config(nx: int, ny: int, precision="fp32", tau: float = 0.8, refine_sensor="kn",
                refine_threshold: float = 1e-3, switch_sensor="neq",
                switch_threshold: float = 1e-4, record=("kl",), output_every: int = 1,
                tile: int = 16, stream="torch", kernel="auto", rho0: float = 1.0,
                dev_exp: int = 12, dev_unscaled: bool = False, tau2: float = 0.0) -> Config:
    """A kss_config (see include/kss.h).  stream: "torch" = torch's current stream
    (handle 0 is the CUDA default stream), "own" = a stream created and owned by the
    lattice, or a raw cudaStream_t handle.  rho0, dev_exp, dev_unscaled: the FP16
    deviation storage of precision "fp16dev".  tau2 > 0: adaptive algorithm refinement,
    the two-relaxation model (tau, tau2) in the switched region."""
    lib = load()
    cfg = Config()
    rc = lib.kss_config_default(ctypes.byref(cfg), nx, ny, PRECISIONS[precision])
    if rc < 0:
        raise KssError(rc, lib.kss_strerror(rc).decode())
    cfg.tau = tau
    cfg.refine_sensor = _sensor(refine_sensor)
    cfg.refine_threshold = refine_threshold
    cfg.switch_sensor = _sensor(switch_sensor)
    cfg.switch_threshold = switch_threshold
    cfg.record_mask = sum(1 << _sensor(s) for s in record)
    cfg.output_every = output_every
    cfg.tile = tile
    cfg.kernel = KERNELS[kernel]
    cfg.rho0 = rho0
    cfg.dev_exp = dev_exp
    cfg.dev_unscaled = int(dev_unscaled)
    cfg.tau2 = tau2
    if stream == "own":
        cfg.own_stream, cfg.stream = 1, None
    else:
        cfg.stream = _torch_stream_handle() if stream == "torch" else stream
    return cfg


# storage element of each precision, as numpy / torch dtypes (the raw rows of the slab
# exchange; FP16 deviations travel as their binary16 codes)
STORAGE_NP = {FP64: np.float64, FP32: np.float32, FP16DEV: np.int16}


class Lattice:
    """A periodic D2Q9 lattice on the current CUDA device (see include/kss.h); with
    slab=True one y-slab of a decomposed lattice, whose halo rows the caller sets before
    each step (kss_slab_create)."""

    def __init__(self, nx: int, ny: int, precision="fp32", tau: float = 0.8,
                 refine_sensor="kn", refine_threshold: float = 1e-3, switch_sensor="neq",
                 switch_threshold: float = 1e-4, record=("kl",), output_every: int = 1,
                 tile: int = 16, stream="torch", kernel="auto", rho0: float = 1.0,
                 dev_exp: int = 12, dev_unscaled: bool = False, tau2: float = 0.0,
                 slab: bool = False):
        self._lib = load()
        self._h = None
        cfg = make_config(nx, ny, precision=precision, tau=tau, refine_sensor=refine_sensor,
                          refine_threshold=refine_threshold, switch_sensor=switch_sensor,
                          switch_threshold=switch_threshold, record=record,
                          output_every=output_every, tile=tile, stream=stream, kernel=kernel,
                          rho0=rho0, dev_exp=dev_exp, dev_unscaled=dev_unscaled, tau2=tau2)
        handle = ctypes.c_void_p()
        create = self._lib.kss_slab_create if slab else self._lib.kss_create
        self._check(create(ctypes.byref(cfg), ctypes.byref(handle)))
        self._adopt(handle, cfg, owned=True)
        self.slab = slab

    def _adopt(self, handle, cfg, owned: bool):
        self.cfg = cfg
        self.nx, self.ny, self.tile = cfg.nx, cfg.ny, cfg.tile
        self.precision = cfg.precision
        self._h = handle
        self._owned = owned
        self.last_status = KSS_OK

    @classmethod
    def _member(cls, lib, handle, cfg, batch):
        """A batch member's handle (owned by the batch, which it keeps alive)."""
        self = cls.__new__(cls)
        self._lib = lib
        self._adopt(ctypes.c_void_p(handle), cfg, owned=False)
        self._batch = batch
        return self

    # -- plumbing --
    def _check(self, rc: int) -> int:
        if rc < 0:
            detail = ""
            if getattr(self, "_h", None):
                detail = (self._lib.kss_last_error(self._h) or b"").decode()
            raise KssError(rc, f"{self._lib.kss_strerror(rc).decode()} {detail}".strip())
        self.last_status = rc
        return rc

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                self._lib.kss_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def ntx(self) -> int:
        return -(-self.nx // self.tile)

    @property
    def nty(self) -> int:
        return -(-self.ny // self.tile)

    def _alloc(self, shape, dtype, device: bool):
        if device:
            import torch

            tdt = {np.float64: torch.float64, np.uint8: torch.uint8, np.int32: torch.int32}[dtype]
            return torch.empty(shape, dtype=tdt, device="cuda")
        return np.empty(shape, dtype=dtype)

    # -- API --
    def set_fields(self, rho, ux, uy) -> None:
        """Equilibrium state of the fields [ny, nx]: float64 (kss_set_fields) or, all three
        float32, kss_set_fields_f32 (half the bytes from the host)."""
        f32 = all(_dtype_of(a) == np.float32 for a in (rho, ux, uy))
        dt = np.float32 if f32 else np.float64
        (pr, d0), (pu, d1), (pv, d2) = (_ptr(a, dt) for a in (rho, ux, uy))
        if not d0 == d1 == d2:
            raise TypeError("fields must all be host or all be device memory")
        fn = self._lib.kss_set_fields_f32 if f32 else self._lib.kss_set_fields
        self._check(fn(self._h, pr, pu, pv, d0))

    def set_populations(self, f) -> None:
        p, d = _ptr(f, np.float64)
        self._check(self._lib.kss_set_populations(self._h, p, d))

    def get_populations(self, device: bool = False):
        out = self._alloc((9, self.ny, self.nx), np.float64, device)
        p, d = _ptr(out, np.float64)
        self._check(self._lib.kss_get_populations(self._h, p, d))
        return out

    def step(self, n: int = 1) -> None:
        self._check(self._lib.kss_step(self._h, int(n)))

    def read_moments(self, device: bool = False):
        outs = [self._alloc((self.ny, self.nx), np.float64, device) for _ in range(3)]
        (p0, d), (p1, _), (p2, _) = (_ptr(a, np.float64) for a in outs)
        self._check(self._lib.kss_read_moments(self._h, p0, p1, p2, d))
        return tuple(outs)

    def read_sensor(self, sensor, device: bool = False, out=None):
        """The sensor field [ny, nx] (FP64) of the last output step; `out` = a buffer to
        fill (host or device, float64, contiguous)."""
        if out is None:
            out = self._alloc((self.ny, self.nx), np.float64, device)
        p, d = _ptr(out, np.float64)
        self._check(self._lib.kss_read_sensor(self._h, _sensor(sensor), p, d))
        return out

    def read_flags(self, device: bool = False, out=None):
        """(flags, tile_counts, counts); `out` = (flags, tiles) buffers to fill."""
        if out is not None:
            flags, tiles = out
        else:
            flags = self._alloc((self.ny, self.nx), np.uint8, device)
            tiles = self._alloc((2, self.nty, self.ntx), np.int32, device)
        counts = (ctypes.c_int64 * 3)()
        pf, d = _ptr(flags, np.uint8)
        pt, _ = _ptr(tiles, np.int32)
        self._check(self._lib.kss_read_flags(self._h, pf, pt, counts, d))
        return flags, tiles, np.array(list(counts), dtype=np.int64)

    def _raw(self, a):
        """(pointer, on_device) of a contiguous [3, nx] buffer of the storage type."""
        want = STORAGE_NP[self.precision]
        if _is_torch(a):
            import torch

            tdt = {np.float64: torch.float64, np.float32: torch.float32,
                   np.int16: torch.int16}[want]
            if a.dtype != tdt or not a.is_contiguous() or a.numel() != 3 * self.nx:
                raise TypeError(f"halo rows must be a contiguous {tdt} tensor of 3 x {self.nx}")
            return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
        if (not isinstance(a, np.ndarray) or a.dtype != want or not a.flags["C_CONTIGUOUS"]
                or a.size != 3 * self.nx):
            raise TypeError(f"halo rows must be a C-contiguous {np.dtype(want).name} array "
                            f"of 3 x {self.nx}")
        return ctypes.c_void_p(a.ctypes.data), 0

    def slab_edges(self, device: bool = True, out=None):
        """(to_below, to_above): the rows leaving the slab, [3, nx] each in the storage
        type (q = 4, 7, 8 of row 0; q = 2, 5, 6 of row ny - 1)."""
        if out is None:
            want = STORAGE_NP[self.precision]
            if device:
                import torch

                tdt = {np.float64: torch.float64, np.float32: torch.float32,
                       np.int16: torch.int16}[want]
                out = tuple(torch.empty((3, self.nx), dtype=tdt, device="cuda")
                            for _ in range(2))
            else:
                out = (np.empty((3, self.nx), dtype=want), np.empty((3, self.nx), dtype=want))
        (pb, d), (pa, _) = self._raw(out[0]), self._raw(out[1])
        self._check(self._lib.kss_slab_edges(self._h, pb, pa, d))
        return out

    def set_halos(self, from_below, from_above) -> None:
        """Halo rows of the next step: from_below = the slab below's to_above (its row
        ny - 1, q = 2, 5, 6), from_above = the slab above's to_below."""
        (pb, d), (pa, _) = self._raw(from_below), self._raw(from_above)
        self._check(self._lib.kss_slab_set_halos(self._h, pb, pa, d))

    def read_stats(self):
        sums = (ctypes.c_double * 3)()
        counts = (ctypes.c_int64 * 3)()
        step = ctypes.c_int64()
        self._check(self._lib.kss_read_stats(self._h, sums, counts, ctypes.byref(step)))
        return np.array(list(sums)), np.array(list(counts), dtype=np.int64), step.value

    def set_aar_region(self, region) -> None:
        """Replace the two-relaxation region (uint8 [ny, nx], nonzero = switched)."""
        p, d = _ptr(region, np.uint8)
        self._check(self._lib.kss_set_aar_region(self._h, p, d))

    def get_aar_region(self, device: bool = False):
        """The two-relaxation region in force for the next step (uint8 [ny, nx], 0 / 1)."""
        out = self._alloc((self.ny, self.nx), np.uint8, device)
        p, d = _ptr(out, np.uint8)
        self._check(self._lib.kss_get_aar_region(self._h, p, d))
        return out

    def regrid(self, buffer: int = 2, efficiency: float = 0.98, max_boxes: int = 1 << 16):
        """(boxes [(x0, y0, x1, y1)] in tile units, tile mask [nty, ntx] uint8) of the
        current step's refine flags (see include/kss.h)."""
        mask = np.empty((self.nty, self.ntx), dtype=np.uint8)
        boxes = (Box * max_boxes)()
        n = ctypes.c_int32()
        self._check(self._lib.kss_regrid(self._h, int(buffer), float(efficiency),
                                         ctypes.c_void_p(mask.ctypes.data), boxes,
                                         int(max_boxes), ctypes.byref(n), 0))
        return [(b.x0, b.y0, b.x1, b.y1) for b in boxes[:min(n.value, max_boxes)]], mask

    @property
    def step_count(self) -> int:
        s = ctypes.c_int64()
        self._check(self._lib.kss_get_step(self._h, ctypes.byref(s)))
        return s.value

    def sync(self) -> None:
        self._check(self._lib.kss_sync(self._h))


class Batch:
    """n independent lattices advanced by one launch per step (see include/kss.h).

    ``specs``: one dict of ``make_config`` keyword arguments per lattice (each with
    ``nx`` and ``ny``); ``common``: keyword arguments shared by all of them.  The
    stream is the first lattice's.  ``members`` are ``Lattice`` objects owned by the
    batch (closing them does nothing; ``close()`` frees the batch and its members).
    """

    def __init__(self, specs, **common):
        self._lib = load()
        self._h = None
        cfgs = [make_config(**{**common, **sp}) for sp in specs]
        arr = (Config * len(cfgs))(*cfgs)
        handle = ctypes.c_void_p()
        rc = self._lib.kss_batch_create(len(cfgs), arr, ctypes.byref(handle))
        if rc < 0:
            raise KssError(rc, self._lib.kss_strerror(rc).decode())
        self._h = handle
        self.members = [Lattice._member(self._lib, self._lib.kss_batch_member(handle, k), c, self)
                        for k, c in enumerate(cfgs)]

    def _check(self, rc: int) -> int:
        if rc < 0:
            detail = ""
            if self._h:
                detail = (self._lib.kss_batch_last_error(self._h) or b"").decode()
            raise KssError(rc, f"{self._lib.kss_strerror(rc).decode()} {detail}".strip())
        return rc

    def __len__(self):
        return len(self.members)

    def __getitem__(self, k) -> Lattice:
        return self.members[k]

    def step(self, n: int = 1) -> None:
        self._check(self._lib.kss_batch_step(self._h, int(n)))

    @property
    def tuning(self) -> dict:
        t = BatchTuning()
        self._check(self._lib.kss_batch_get_tuning(self._h, ctypes.byref(t)))
        return {"rows": t.rows, "ctas_per_sm": t.ctas_per_sm, "graph": t.graph,
                "ms_per_step": t.ms_per_step, "multi_step": t.multi_step}

    def set_tuning(self, rows: int = 0, ctas_per_sm: int = 0, graph: int = 1,
                   multi_step: int = 1) -> None:
        t = BatchTuning(rows, ctas_per_sm, graph, 0.0, multi_step)
        self._check(self._lib.kss_batch_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, cache_path: str | None = None, steps: int = 10) -> dict:
        t = BatchTuning()
        path = cache_path.encode() if cache_path else None
        self._check(self._lib.kss_batch_autotune(self._h, path, int(steps), ctypes.byref(t)))
        return {"rows": t.rows, "ctas_per_sm": t.ctas_per_sm, "graph": t.graph,
                "ms_per_step": t.ms_per_step, "multi_step": t.multi_step}

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m._h = None
            self._lib.kss_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Adjoint:
    """Gradient of J = sum W eps_KL (step nsteps) in rho0 and tau (see include/kss.h)."""

    def __init__(self, nx: int, ny: int, nsteps: int, precision="fp32",
                 checkpoint_every: int = 20, stream="torch"):
        self._lib = load()
        self._h = None
        cfg = AdjointConfig(nx, ny, PRECISIONS[precision], nsteps, checkpoint_every, None, 0)
        if stream == "own":
            cfg.own_stream = 1
        else:
            cfg.stream = _torch_stream_handle() if stream == "torch" else stream
        handle = ctypes.c_void_p()
        rc = self._lib.kss_adjoint_create(ctypes.byref(cfg), ctypes.byref(handle))
        if rc < 0:
            raise KssError(rc, self._lib.kss_strerror(rc).decode())
        self._h = handle
        self.nx, self.ny, self.nsteps = nx, ny, nsteps

    def _check(self, rc: int) -> int:
        if rc < 0:
            detail = (self._lib.kss_adjoint_last_error(self._h) or b"").decode() if self._h else ""
            raise KssError(rc, f"{self._lib.kss_strerror(rc).decode()} {detail}".strip())
        return rc

    def forward(self, rho0, ux0, uy0, tau: float, weight=None) -> float:
        ptrs = [_ptr(a, np.float64) for a in (rho0, ux0, uy0)]
        dev = {d for _, d in ptrs}
        wp = None
        if weight is not None:
            wp, wd = _ptr(weight, np.float64)
            dev.add(wd)
        if len(dev) != 1:
            raise TypeError("fields and weights must all be host or all be device memory")
        J = ctypes.c_double()
        self._check(self._lib.kss_adjoint_forward(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                                  wp, float(tau), dev.pop(), ctypes.byref(J)))
        return J.value

    def set_multistep(self, on: bool) -> None:
        """Reverse sweep in one cooperative launch per segment (True, the default) or one
        launch per reverse step; the gradients are the same bit for bit."""
        self._check(self._lib.kss_adjoint_set_multistep(self._h, int(bool(on))))

    def backward(self, device: bool = False):
        """(dJ/drho0 [ny, nx] float64, dJ/dtau) of the last forward pass."""
        if device:
            import torch

            g = torch.empty((self.ny, self.nx), dtype=torch.float64, device="cuda")
        else:
            g = np.empty((self.ny, self.nx))
        p, d = _ptr(g, np.float64)
        gt = ctypes.c_double()
        self._check(self._lib.kss_adjoint_backward(self._h, p, ctypes.byref(gt), d))
        return g, gt.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.kss_adjoint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def regrid_flags(flags, tile: int = 16, buffer: int = 2, efficiency: float = 0.98,
                 max_boxes: int = 1 << 16, stream="torch"):
    """kss_regrid_flags on host flags [ny, nx] uint8: (boxes, tile mask)."""
    lib = load()
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    ny, nx = f.shape
    ntx, nty = -(-nx // tile), -(-ny // tile)
    mask = np.empty((nty, ntx), dtype=np.uint8)
    boxes = (Box * max_boxes)()
    n = ctypes.c_int32()
    st = _torch_stream_handle() if stream == "torch" else stream
    rc = lib.kss_regrid_flags(ctypes.c_void_p(f.ctypes.data), nx, ny, tile, int(buffer),
                              float(efficiency), ctypes.c_void_p(mask.ctypes.data), boxes,
                              int(max_boxes), ctypes.byref(n), 0, st)
    if rc < 0:
        raise KssError(rc, lib.kss_strerror(rc).decode())
    return [(b.x0, b.y0, b.x1, b.y1) for b in boxes[:min(n.value, max_boxes)]], mask
