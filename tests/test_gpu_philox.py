"""The sampler's Philox4x32-10 on the device against an independent
implementation of the same published function: cuRAND's device-side
curand_Philox4x32_10 (counter and key passed as they are), on 2^22
pseudo-random counters and keys. A library's output is compared; nothing is
disassembled."""
import ctypes
import os
import subprocess
import tempfile

import pytest

from paper_2303_16492_gb300 import build as _build
from tests.gpu_helpers import cuda

pytestmark = [pytest.mark.gpu, cuda]

HERE = os.path.dirname(os.path.abspath(__file__))


def test_device_philox_matches_curand():
    src = os.path.join(HERE, "kernels", "philox_check.cu")
    with tempfile.TemporaryDirectory() as tmp:
        so = os.path.join(tmp, "philox_check.so")
        cmd = [_build.nvcc(), *_build.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
               "-I", _build.CSRC, "-o", so, src]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        lib = ctypes.CDLL(so)
        lib.philox_mismatches.restype = ctypes.c_longlong
        lib.philox_mismatches.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong]
        for seed in (0, 0x2303_16492, 0xFFFF_FFFF_FFFF_FFFF):
            assert lib.philox_mismatches(1 << 22, seed) == 0
