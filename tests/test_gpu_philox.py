"""The device Philox4x32-10 against the oracle's and against cuRAND's."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_CURAND_REF = r"""
#include <curand_kernel.h>
#include <stdint.h>
__global__ void k(const uint4 *c, unsigned long long n, uint2 key, uint4 *o) {
    unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i < n) o[i] = curand_Philox4x32_10(c[i], key);
}
extern "C" int curand_ref(const void *c, unsigned long long n, unsigned long long seed, void *o) {
    uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    k<<<(unsigned)((n + 127) / 128), 128>>>((const uint4 *)c, n, key, (uint4 *)o);
    return (int)cudaDeviceSynchronize();
}
"""


def _counters(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    c[0] = 0
    c[1] = 0xFFFFFFFF
    c[2] = [7, 0, 3, 0]
    return c


@pytest.mark.parametrize("seed", [1, 2026, 0xDEADBEEFCAFEF00D])
def test_device_philox_matches_oracle(gpu, oracle_mod, seed):
    import torch
    c = _counters(100_003, seed & 0xFFFF)
    out = gpu.philox(torch.from_numpy(c.view(np.int32)).cuda(), seed).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(out, oracle_mod.philox4x32_10(c, seed))


def test_device_philox_matches_curand(gpu, tmp_path):
    import torch
    src = os.path.join(tmp_path, "ref.cu")
    so = os.path.join(tmp_path, "libref.so")
    open(src, "w").write(_CURAND_REF)
    subprocess.run(["nvcc", "-gencode=arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler",
                    "-fPIC", "-o", so, src], check=True)
    ref = C.CDLL(so)
    ref.curand_ref.argtypes = [C.c_void_p, C.c_ulonglong, C.c_ulonglong, C.c_void_p]
    c = _counters(65_537, 5)
    for seed in (1, 42, 0x123456789ABCDEF0):
        ct = torch.from_numpy(c.view(np.int32)).cuda()
        want = torch.empty_like(ct)
        torch.cuda.synchronize()
        assert ref.curand_ref(ct.data_ptr(), c.shape[0], seed, want.data_ptr()) == 0
        got = gpu.philox(ct, seed)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())
