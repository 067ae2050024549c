"""The debug flavour of the library compiles: -DKSS_DEBUG_BOUNDS=1 (every step block and
adjoint block checks its coordinates, rows, deferred-cell slots and tile indices, and
reports KSS_ERR_BOUNDS instead of an access outside its buffers) and -DKSS_NVTX=0 (no
NVTX ranges), for the FP32 kernels and the single-lattice and adjoint runtimes (nvcc
cross-compiles sm_103a without a GPU).  The release build is what every other test loads."""
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2603_13618_gb300 import build


@pytest.mark.parametrize("macro", ["-DKSS_DEBUG_BOUNDS=1", "-DKSS_NVTX=0"])
def test_debug_flavours_compile(macro):
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("no nvcc")
    srcs = ["launch_f32.cu", "kss_runtime.cu", "kss_adjoint.cu"] if "BOUNDS" in macro \
        else ["kss_runtime.cu", "kss_batch.cu"]
    with tempfile.TemporaryDirectory() as d:
        procs = [subprocess.Popen([build.nvcc(), *build.flags([macro]), "-c",
                                   os.path.join(build.CSRC, s), "-o", os.path.join(d, s + ".o")],
                                  stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
                 for s in srcs]
        for s, p in zip(srcs, procs):
            out, err = p.communicate(timeout=600)
            assert p.returncode == 0, f"{s} {macro}:\n{out}\n{err}"
