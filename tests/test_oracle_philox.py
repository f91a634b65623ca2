"""Pins for the oracle's Philox4x32-10 and its uniform mapping.

The generator is compared bit for bit with the Philox4x32 of an independent
library (Triton's `philox`, run by its CPU interpreter in a child process).
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

_TRITON_CHILD = textwrap.dedent(r"""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl
    from triton.language.random import philox

    @triton.jit
    def k(c_ptr, out_ptr, seed, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m)
        o0, o1, o2, o3 = philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, o0, mask=m)
        tl.store(out_ptr + 4 * i + 1, o1, mask=m)
        tl.store(out_ptr + 4 * i + 2, o2, mask=m)
        tl.store(out_ptr + 4 * i + 3, o3, mask=m)

    req = json.load(sys.stdin)
    res = {}
    for seed in req["seeds"]:
        c = np.array(req["ctr"], dtype=np.uint32).view(np.int32)
        ct = torch.from_numpy(c.copy())
        out = torch.zeros_like(ct)
        n = ct.numel() // 4
        k[(1,)](ct, out, seed, n, BLOCK=triton.next_power_of_2(n))
        res[str(seed)] = out.numpy().view(np.uint32).tolist()
    json.dump(res, sys.stdout)
""")


def test_philox_matches_library_philox(oracle_mod):
    pytest.importorskip("triton")
    rng = np.random.default_rng(20260101)
    ctr = rng.integers(0, 2 ** 32, size=(200, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [5, 0, 31, 0]  # the engine's (photon_lo, photon_hi, event, 0) shape
    seeds = [0, 1, 2026, 0x123456789ABCDEF0, 2 ** 64 - 1]
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_CHILD], input=json.dumps(
        {"ctr": ctr.reshape(-1).tolist(), "seeds": seeds}), capture_output=True, text=True,
        env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    ref = json.loads(p.stdout)
    for seed in seeds:
        got = oracle_mod.philox4x32_10(ctr, seed)
        want = np.array(ref[str(seed)], dtype=np.uint32).reshape(-1, 4)
        np.testing.assert_array_equal(got, want)


def test_uniform_mapping(oracle_mod):
    lo = oracle_mod.uniform(0)
    hi = oracle_mod.uniform(0xFFFFFFFF)
    assert lo == 2.0 ** -24
    assert hi == 1.0 - 2.0 ** -24
    # every value is exact in single precision, so both precisions draw the same u
    for r in (0, 1, 255, 256, 12345678, 0x80000000, 0xFFFFFF00, 0xFFFFFFFF):
        u = oracle_mod.uniform(r)
        assert float(np.float32(u)) == u
        assert 0.0 < u < 1.0


def test_uniform_moments(oracle_mod):
    n = 1 << 18
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    out = oracle_mod.philox4x32_10(ctr, 1).reshape(-1)
    u = (out >> 9).astype(np.float64) * 2.0 ** -23 + 2.0 ** -24
    m = u.size
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / m)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / m)
    # lanes are uncorrelated with each other
    uu = u.reshape(n, 4)
    c = np.corrcoef(uu.T)
    assert np.max(np.abs(c - np.eye(4))) < 5 / np.sqrt(n)
