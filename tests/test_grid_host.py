"""Host side of the heterogeneous-medium path (no GPU): the engine's mixture
table against the oracle's, and the grid argument checks of the C ABI."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def eng():
    from paper_2507_23189_gb300 import build
    build.build()
    import paper_2507_23189_gb300 as E
    return E


def test_mixture_table_matches_oracle(eng, oracle_mod):
    from paper_2507_23189_gb300 import workloads as W
    d, f = W.size_bins(5.0, 0.3, 16)
    t = eng.MixtureTable(d, f)
    comps, sig_s, sig_e = [], [], []
    m = complex(1.59 / 1.33, 0.0)
    for di in d:
        x = oracle_mod.size_parameter(di, 1.33, 532.0)
        qe, qs, _ = oracle_mod.mie_efficiencies(m, x)
        geo = np.pi * (di * 1e-3) ** 2 / 4
        comps.append(("mie", m, x))
        sig_s.append(qs * geo)
        sig_e.append(qe * geo)
    w = np.array(f) * np.array(sig_s)
    o = oracle_mod.phase_table_mixture(comps, w, n_bins=4096, n_fine=1 << 18)
    np.testing.assert_allclose(t.omu64, o["omu"], rtol=2e-7, atol=2e-10)
    assert t.info["sigma_sca_mm2"] == pytest.approx(float(np.dot(f, sig_s)), rel=1e-10)
    assert t.info["sigma_ext_mm2"] == pytest.approx(float(np.dot(f, sig_e)), rel=1e-10)
    assert t.info["g_table"] == pytest.approx(o["mean"], abs=1e-7)


def test_single_component_mixture_is_the_plain_table(eng):
    a = eng.MixtureTable([5.0], [1.0])
    b = eng.PhaseTable(5.0)
    np.testing.assert_array_equal(a.blob, b.blob)


def test_grid_workspace_validation(eng):
    from paper_2507_23189_gb300 import _native as N
    L = eng.lib()

    def nbytes(**kw):
        g = dict(d_density=None, gx=64, gy=32, gz=32, k_ext=1e-5, k_sca=1e-5, mu_a=0.0, bx=8, by=8, bz=8)
        g.update(kw)
        return L.mc_grid_workspace_bytes(C.byref(N.Grid(**g)))

    assert nbytes() == 8 * 64 * 32 * 32 + 16 * ((4 * 8 * 4 * 4 + 15) // 16)
    assert nbytes(gx=0) == 0
    assert nbytes(k_sca=2e-5) == 0             # more scattering than extinction
    assert nbytes(k_ext=0.0, k_sca=0.0) == 0
    assert nbytes(mu_a=-1.0) == 0
    assert nbytes(bx=1, by=1, bz=1) == 0       # 65536 cells > 16384
    assert nbytes(gx=4097) == 0
