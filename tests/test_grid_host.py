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


def test_new_entry_points_reject_bad_arguments_without_gpu(eng):
    """Invalid arguments come back as MC_ERR_ARG before any CUDA call."""
    from paper_2507_23189_gb300 import _native as N
    L = eng.lib()
    vp = C.c_void_p
    fake = vp(1 << 20)                       # aligned, never dereferenced
    geo = N.Geometry(45.0, 10.0, 10.0, 0.0)
    cam = N.Camera(32, 32, 16, 7.0)
    run = N.RunParams(10, 0, 1, 1e-4, 0.1, 1000, 0, 32, 0, 0, 0, 0)
    tal = N.Tallies(fake, fake, fake, fake, fake, 4096)
    hg = N.Medium(1.0, 0.0, N.PHASE_HG, 0.5, None, 0)
    good = dict(d_density=fake, gx=32, gy=16, gz=16, k_ext=1e-5, k_sca=1e-5, mu_a=0.0, bx=8, by=8, bz=8)

    def grid(**kw):
        g = dict(good)
        g.update(kw)
        return N.Grid(**g)

    # mc_run_grid
    assert L.mc_run_grid(C.byref(grid(gx=0)), fake, C.byref(hg), C.byref(geo), C.byref(cam), C.byref(run),
                         C.byref(tal), None, 0, 0, None) == -1
    assert L.mc_run_grid(C.byref(grid()), None, C.byref(hg), C.byref(geo), C.byref(cam), C.byref(run),
                         C.byref(tal), None, 0, 0, None) == -1
    table_no_blob = N.Medium(1.0, 0.0, N.PHASE_TABLE, 0.0, None, 4096)
    assert L.mc_run_grid(C.byref(grid()), fake, C.byref(table_no_blob), C.byref(geo), C.byref(cam),
                         C.byref(run), C.byref(tal), None, 0, 0, None) == -1
    assert L.mc_run_grid(C.byref(grid()), fake, C.byref(hg), C.byref(geo), C.byref(cam), C.byref(run),
                         C.byref(tal), fake, 0, 32, None) == -1          # trace without photons to trace
    # mc_grid_prepare / mc_grid_adjoint
    assert L.mc_grid_prepare(C.byref(grid(d_density=None)), C.byref(geo), fake, 1 << 30, None) == -1
    assert L.mc_grid_prepare(C.byref(grid()), C.byref(N.Geometry(-1.0, 10.0, 10.0, 0.0)), fake, 1 << 30,
                             None) == -1
    assert L.mc_grid_adjoint(C.byref(grid()), fake, C.byref(hg), C.byref(geo), C.byref(cam), C.byref(run),
                             None, fake, fake, fake, fake, 1 << 30, None) == -1
    # image metrics
    assert L.mc_metrics_out_len(0) == 0 and L.mc_metrics_out_len(4097) == 0
    assert L.mc_metrics_out_len(32) == 13 + 96
    assert L.mc_metrics_workspace_bytes(0) == 0
    assert L.mc_image_metrics(fake, fake, None, 0, 16, 8, fake, fake, 1 << 20, None) == -1
    assert L.mc_image_metrics(fake, None, None, 16, 16, 8, fake, fake, 1 << 20, None) == -1
    assert L.mc_image_metrics(fake, fake, None, 16, 16, 0, fake, fake, 1 << 20, None) == -1
    assert L.mc_image_metrics(fake, fake, None, 16, 16, 8, fake, fake, 8, None) == -3   # workspace too small


def test_paper_and_mixture_builders_reject_bad_arguments(eng):
    from paper_2507_23189_gb300 import _native as N
    L = eng.lib()
    p = N.MieParams(5.0, 1.59, 0.0, 1.33, 532.0, 4096)
    assert L.mc_paper_table_bytes(3000) > 0 and L.mc_paper_table_bytes(15) == 0
    assert L.mie_paper_table_build(C.byref(p), 10, None, None, None) == -1
    bad = N.MieParams(-5.0, 1.59, 0.0, 1.33, 532.0, 4096)
    assert L.mie_paper_table_build(C.byref(bad), 3000, None, None, None) == -1
    ps = (N.MieParams * 2)(N.MieParams(5.0, 1.59, 0.0, 1.33, 532.0, 4096),
                           N.MieParams(3.0, 1.59, 0.0, 1.33, 532.0, 2048))
    f = (C.c_double * 2)(0.5, 0.5)
    assert L.mie_mixture_table_build(ps, f, 2, None, None, None, None) == -1        # mixed n_bins
    ps[1].n_bins = 4096
    f[1] = -0.1
    assert L.mie_mixture_table_build(ps, f, 2, None, None, None, None) == -1        # negative fraction
    assert L.mie_mixture_table_build(ps, f, 0, None, None, None, None) == -1
