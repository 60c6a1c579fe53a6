"""Why the contraction of int8 voltages runs in BF16 on GB300: the sm_103a
target has no int8 tensor-core MMA.  ptxas (CUDA 13.0) accepts a one-line
kernel issuing `tcgen05.mma.cta_group::1.kind::i8` for sm_100a and refuses the
same kernel for sm_103a ("Feature '.kind::i8' not supported"), while the
`.kind::f16` form the beam GEMM and the correlator use assembles for sm_103a.
The int8 input format itself is handled at ingest (converted to FP32 inside
the first FFT pass, tests/test_gpu_precision.py)."""
import os
import shutil
import subprocess
import tempfile

import pytest

NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"

KERNEL = r"""
#include <cstdint>
__global__ void k(uint32_t d, uint64_t a, uint64_t b, uint32_t id) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %%4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::%s [%%0], %%1, %%2, %%3, p;\n\t}"
               :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(1) : "memory");
}
"""


def _assemble(kind: str, arch: str):
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "k.cu")
        with open(src, "w") as f:
            f.write(KERNEL % kind)
        r = subprocess.run([NVCC, "-gencode", "arch=compute_%s,code=sm_%s" % (arch, arch), "-c",
                            src, "-o", os.path.join(tmp, "k.o")], capture_output=True, text=True)
        return r.returncode, r.stdout + r.stderr


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not available")
def test_int8_tensor_core_mma_does_not_exist_on_sm_103a():
    rc, msg = _assemble("i8", "103a")
    assert rc != 0 and "kind::i8" in msg and "sm_103a" in msg, msg
    rc, msg = _assemble("i8", "100a")
    assert rc == 0, msg
    rc, msg = _assemble("f16", "103a")
    assert rc == 0, msg
