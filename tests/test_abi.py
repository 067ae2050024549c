"""The C ABI library loads and exports every entry point that include/kss.h declares
(no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kss_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("kss_create", "kss_destroy", "kss_set_fields", "kss_step", "kss_read_moments",
              "kss_read_sensor", "kss_read_flags", "kss_read_stats"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    for n in _declared():
        assert hasattr(lib, n), n
    so = kss.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True)
    exported = set(re.findall(r"\bT (kss_\w+)", out.stdout))
    assert set(_declared()) <= exported
    assert set(kss._SIGNATURES) == set(_declared())


def test_host_only_calls():
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    assert lib.kss_version() >= 100
    assert lib.kss_strerror(-1) == b"invalid argument"
    cfg = kss.Config()
    assert lib.kss_config_default(cfg, 64, 32, kss.FP32) == 0
    assert (cfg.nx, cfg.ny, cfg.tile, cfg.output_every) == (64, 32, 16, 1)
    assert abs(cfg.tau - 0.8) < 1e-15 and cfg.record_mask == 1 << kss.SENSOR_ID["kl"]
    assert cfg.tau2 == 0.0


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -1), ("tau", 0.5), ("tile", 12),
                                         ("precision", 7), ("refine_sensor", 13),
                                         ("output_every", -2), ("record_mask", 1 << 13),
                                         ("own_stream", 2), ("tau2", 0.5), ("tau2", -1.0),
                                         ("tau2", float("inf"))])
def test_create_rejects_bad_config_before_touching_the_gpu(field, value):
    import ctypes

    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    cfg = kss.Config()
    lib.kss_config_default(cfg, 64, 32, kss.FP32)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    rc = lib.kss_create(cfg, ctypes.byref(h))
    assert rc < 0 and not h.value


def _prototypes():
    src = open(os.path.join(ROOT, "include", "kss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(kss_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_arity_matches_header():
    from paper_2603_13618_gb300 import kss

    protos = _prototypes()
    for name, (_, argtypes) in kss._SIGNATURES.items():
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of kss_config, kss_batch_tuning and kss_adjoint_config have the C
    layout (sizes and field offsets from a C program compiled against include/kss.h)."""
    import ctypes

    from paper_2603_13618_gb300 import kss

    structs = {"kss_config": kss.Config, "kss_batch_tuning": kss.BatchTuning,
               "kss_adjoint_config": kss.AdjointConfig, "kss_box": kss.Box}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kss.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, got):
        cname, what, val = line.split()
        cls = structs[cname]
        want = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert int(val) == want, line


@pytest.mark.parametrize("field,value", [("rho0", 0.0), ("rho0", float("nan")), ("dev_exp", 41),
                                         ("dev_exp", -25), ("dev_unscaled", 2)])
def test_create_rejects_bad_fp16_deviation_config(field, value):
    import ctypes

    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    cfg = kss.Config()
    lib.kss_config_default(cfg, 64, 32, kss.FP16DEV)
    assert (cfg.rho0, cfg.dev_exp, cfg.dev_unscaled) == (1.0, 12, 0)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    rc = lib.kss_create(cfg, ctypes.byref(h))
    assert rc == -1 and not h.value


# kss_step_f32_noalloc validates every argument, and the capacity of its static scratch,
# before its first CUDA call.  The pointers below are 16-byte aligned stand-ins that the
# call never dereferences: it returns before any memory access.
_A = 0x10000
_B = 0x1000000  # beyond f_in's 9 x 64 x 64 floats: a distinct output range
_NOALLOC_OK = dict(f_in=_A, f_out=_B, nx=64, ny=64, pitch=64, tau=0.8, refine_sensor=5,
                   refine_threshold=1e-3, switch_sensor=6, switch_threshold=1e-4, tile=16,
                   record_sensor=9, sensor_out=_A, flags=_A, tile_counts=_A, sums=_A,
                   counts=_A, stream=None)


@pytest.mark.parametrize("change,code", [
    (dict(f_in=None), "arg"), (dict(sums=None), "arg"), (dict(nx=0), "arg"),
    (dict(pitch=48), "arg"), (dict(pitch=32), "arg"), (dict(tau=0.5), "arg"),
    (dict(tile=12), "arg"), (dict(refine_sensor=0), "arg"), (dict(switch_sensor=12), "arg"),
    (dict(record_sensor=0), "arg"), (dict(f_out=_B + 8), "arg"), (dict(flags=_A + 2), "arg"),
    (dict(f_out=_A), "arg"), (dict(f_out=_A + 9 * 64 * 64 * 4 - 16), "arg"),
    (dict(f_in=_B + 16), "arg"),
    (dict(nx=16384, ny=16384, pitch=16384, f_out=_A + 9 * 16384 * 16384 * 4), "capacity"),
])
def test_noalloc_rejects_bad_arguments_before_touching_the_gpu(change, code):
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    a = dict(_NOALLOC_OK, **change)
    rc = lib.kss_step_f32_noalloc(*a.values())
    assert rc == {"arg": -1, "capacity": -7}[code], (change, rc)


@pytest.mark.parametrize("field,value,code", [
    ("nx", 0, -1), ("ny", -3, -1), ("nsteps", 0, -1), ("checkpoint_every", 0, -1),
    ("own_stream", 2, -1), ("precision", 2, -6), ("nx", 1 << 16, -1),
])
def test_adjoint_create_rejects_bad_config_before_touching_the_gpu(field, value, code):
    """kss_adjoint_create checks its configuration before its first CUDA call (FP16
    deviations have no adjoint: KSS_ERR_UNSUPPORTED)."""
    import ctypes

    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    cfg = kss.AdjointConfig(nx=64, ny=48, precision=kss.FP32, nsteps=20, checkpoint_every=5,
                            stream=None, own_stream=0)
    setattr(cfg, field, value)
    if field == "nx" and value == 1 << 16:
        cfg.ny = 1 << 16  # 2^32 cells: beyond the 32-bit cell index
    out = ctypes.c_void_p(1)
    assert lib.kss_adjoint_create(ctypes.byref(cfg), ctypes.byref(out)) == code
    assert out.value is None


@pytest.mark.parametrize("case,code", [("empty", -1), ("mixed_precision", -1),
                                       ("aar_cadences", -6)])
def test_batch_create_rejects_before_touching_the_gpu(case, code):
    """kss_batch_create: no members, members of different storage precisions, or members with
    the two-relaxation model (tau2 > 0) and different output cadences are refused before the
    first CUDA call."""
    import ctypes

    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    cfgs = (kss.Config * 2)()
    for k in range(2):
        assert lib.kss_config_default(cfgs[k], 64 + 32 * k, 48, kss.FP32) == 0
    n = 2
    if case == "empty":
        n = 0
    elif case == "mixed_precision":
        cfgs[1].precision = kss.FP64
    else:
        cfgs[0].tau2 = cfgs[1].tau2 = 1.3
        cfgs[1].output_every = 3
    out = ctypes.c_void_p(1)
    assert lib.kss_batch_create(n, cfgs, ctypes.byref(out)) == code
    assert out.value is None


def test_fault_injection_arms_and_disarms_without_a_gpu():
    """kss_testing_fail_after takes kind 0 (allocations) or 1 (step launches) and any n;
    arming and disarming touch no device, and nothing is allocated without a lattice."""
    from paper_2603_13618_gb300 import kss

    lib = kss.load()
    assert lib.kss_testing_fail_after(2, 0) == -1
    for kind in (0, 1):
        assert lib.kss_testing_fail_after(kind, 5) == 0
        assert lib.kss_testing_fail_after(kind, -1) == 0
    assert lib.kss_testing_live_allocations() >= 0
