"""Known-answer check of Philox4x32-10 (Salmon et al., SC'11) against a generator neither side
wrote: the CUDA toolkit's device routine curand_Philox4x32_10 (curand_kernel.h), compiled into a
test-only library from tests/kat/curand_philox_kat.cu. The library's Philox (flr_debug_philox) and
the oracle's must both return its blocks bit for bit, for every counter word and both key words,
so a transposed output word, a swapped multiplier or a wrong Weyl constant on either side fails
here even though the two sides would still agree with each other if they shared the mistake."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest
import torch

import oracle
from paper_1706_03024_gb300 import native as N
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kat", "curand_philox_kat.cu")
OUT = os.path.join(HERE, "kat", "_build", "libcurand_philox_kat.so")


def _kat_lib():
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        tmp = OUT + f".{os.getpid()}.tmp"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-Xcompiler",
                        "-fPIC", "-shared", "-o", tmp, SRC], check=True, capture_output=True)
        os.replace(tmp, OUT)
    lib = C.CDLL(OUT)
    lib.kat_philox.argtypes = [C.c_uint32, C.c_uint32, C.c_void_p, C.c_longlong, C.c_void_p]
    lib.kat_philox.restype = C.c_int
    return lib


def _counters():
    rng = np.random.default_rng(2024)
    ctr = rng.integers(0, 2 ** 32, size=(200_000, 4), dtype=np.uint64).astype(np.uint32)
    special = []
    for w in range(4):            # one bit set in each word, and all-ones words
        for b in (0, 1, 31):
            c = np.zeros(4, np.uint32)
            c[w] = np.uint32(1 << b)
            special.append(c)
        c = np.zeros(4, np.uint32)
        c[w] = 0xFFFFFFFF
        special.append(c)
    special.append(np.zeros(4, np.uint32))
    special.append(np.full(4, 0xFFFFFFFF, np.uint32))
    # the library's own counter layout: (path lo, step, slot, path hi)
    pid = np.array([0, 1, 12345, 2 ** 32 - 1, 2 ** 32, 2 ** 40 + 7], np.uint64)
    for p in pid:
        for step in (0, 1, 0xFFFFFFFF):
            for slot in (0, 1, 2, 9):
                special.append(np.array([p & 0xFFFFFFFF, step, slot, p >> 32], np.uint32))
    return np.ascontiguousarray(np.concatenate([np.stack(special), ctr]))


@pytest.mark.parametrize("seed,medium", [(0, 0), (1, 0), (0, 1), (12345, 77),
                                         (0xFFFFFFFF, 0xFFFFFFFF), (0x9E3779B9, 0xBB67AE85)])
def test_philox_blocks_equal_the_toolkit_routine(seed, medium):
    require_gpu()
    lib = _kat_lib()
    ctr = _counters()
    n = ctr.shape[0]
    want = np.zeros_like(ctr)
    assert lib.kat_philox(seed, medium, ctr.ctypes.data, n, want.ctypes.data) == 0
    # the library's Philox
    c = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = torch.empty_like(c)
    assert N.flr_debug_philox(seed, medium, c.data_ptr(), n, out.data_ptr(), 0) == N.FLR_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)
    # the oracle's
    assert np.array_equal(oracle.philox(seed, medium, ctr), want)
    # and not a constant or the identity
    assert len(np.unique(want[:, 0])) > n // 2 and not np.array_equal(want, ctr)
