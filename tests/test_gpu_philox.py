"""The GPU's Philox4x32-10 words against cuRAND's device generator.

Every random draw of the method (start points, directions, the Bernoulli
trials of Eq. 3) is a Philox4x32-10 word.  The oracle's generator is pinned
on the host (known-answer vectors, cuRAND's host generator); here the
library's device generator (rms_philox4x32_10, the function the walk kernels
call) is compared, word for word, with cuRAND's curand_Philox4x32_10 called
from a test kernel built for this GPU, and with the oracle, on 1e6 random
(counter, key) pairs plus the counters the walk actually uses."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CURAND_KERNEL = r"""
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_words_kernel(const uint4 *ctr, const uint2 *key, long long n, uint4 *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_words(const void *ctr, const void *key, long long n, void *out)
{
    curand_words_kernel<<<(unsigned)((n + 255) / 256), 256>>>((const uint4 *)ctr, (const uint2 *)key, n,
                                                             (uint4 *)out);
    return (int)cudaDeviceSynchronize();
}
"""


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("curand_pin")
    src = d / "curand_words.cu"
    src.write_text(CURAND_KERNEL)
    so = d / "libcurand_words.so"
    nvcc = os.environ.get("NVCC", "nvcc")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler",
                           "-fPIC", str(src), "-o", str(so)])
    lib = C.CDLL(str(so))
    lib.curand_words.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
    lib.curand_words.restype = C.c_int
    return lib


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # the counters the walk uses: (walker_lo, walker_hi, step, tag << 16 | call)
    m = n // 4
    w = rng.integers(0, 2 ** 40, size=m, dtype=np.uint64)
    ctr[:m, 0] = (w & 0xFFFFFFFF).astype(np.uint32)
    ctr[:m, 1] = (w >> 32).astype(np.uint32)
    ctr[:m, 2] = rng.integers(0, 300_000, size=m).astype(np.uint32)
    ctr[:m, 3] = ((rng.integers(1, 5, size=m) << 16) | rng.integers(0, 64, size=m)).astype(np.uint32)
    # extremes of every word
    ctr[m:m + 8] = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4] * 4, np.uint32)
    key[m:m + 8] = np.array([[0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0, 0xFFFFFFFF], [0xFFFFFFFF, 0]] * 2, np.uint32)
    return ctr, key


def test_library_philox_equals_curand_and_oracle(curand_lib):
    import torch
    import oracle
    import paper_2012_06478_gb300 as rms
    oracle.build()
    n = 1_000_000
    ctr, key = _inputs(n, 20240)
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    dk = torch.from_numpy(key.view(np.int32)).cuda()
    ours = rms.rms_philox4x32_10(dc, dk)
    torch.cuda.synchronize()
    ref = torch.empty_like(dc)
    assert curand_lib.curand_words(dc.data_ptr(), dk.data_ptr(), n, ref.data_ptr()) == 0
    ours_h = ours.cpu().numpy().view(np.uint32)
    ref_h = ref.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(ours_h, ref_h)
    # the oracle's generator on the same pairs (a sample: it runs on the host)
    sl = slice(0, 200_000)
    np.testing.assert_array_equal(oracle.philox4x32_10(ctr[sl], key[sl]), ours_h[sl])
    # the words are not degenerate
    assert len(np.unique(ours_h[:, 0])) > 0.99 * n


def test_library_philox_argument_checks():
    from paper_2012_06478_gb300 import _lib
    assert _lib.lib.rms_philox4x32_10(None, None, -1, None, None) == _lib.RMS_E_INVALID_ARG
    assert _lib.lib.rms_philox4x32_10(None, None, 5, None, None) == _lib.RMS_E_INVALID_ARG
    assert _lib.lib.rms_philox4x32_10(None, None, 0, None, None) == _lib.RMS_OK
