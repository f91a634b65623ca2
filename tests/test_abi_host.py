"""Host-side checks of the engine library: it loads, exports every symbol the
C header declares, rejects bad arguments, and its double-precision table
builder agrees with the independent oracle (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def eng():
    from paper_2507_23189_gb300 import build
    build.build()
    import paper_2507_23189_gb300 as E
    return E


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mcmie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("mc_", "mie_"))))


def test_library_exports_every_declared_symbol(eng):
    from paper_2507_23189_gb300 import _native as N
    L = N.lib()
    declared = _declared_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(L, name), name
    assert set(N.EXPORTS) <= set(declared)
    assert set(declared) <= set(N.EXPORTS)


def test_checked_build_compiles_and_exports_every_declared_symbol(eng):
    # the index-checked variant (MC_CHECKED) is the same entry points with
    # bounds checks compiled into the kernels
    from paper_2507_23189_gb300 import build
    L = C.CDLL(build.build_checked())
    for name in _declared_functions():
        assert hasattr(L, name), name
    L.mc_status_string.restype = C.c_char_p
    assert b"checked" in L.mc_status_string(-9)


def test_status_strings(eng):
    L = eng.lib()
    for s in range(-9, 2):
        assert L.mc_status_string(s) and L.mc_status_string(s) != b"unknown status"
    assert L.mc_status_string(-10) == b"unknown status"


def test_table_bytes(eng):
    L = eng.lib()
    assert L.mc_table_bytes(4096) % 16 == 0 and L.mc_table_bytes(4096) > 4096 * 8
    for bad in (0, 3, 100, 32, 1 << 15):
        assert L.mc_table_bytes(bad) == 0


@pytest.mark.parametrize("kw", [dict(diameter_um=-1.0), dict(n_medium=0.0), dict(wavelength_nm=0.0),
                                dict(n_particle=complex(1.5, -0.1)), dict(n_bins=1000),
                                dict(diameter_um=float("nan"))])
def test_table_rejects_bad_arguments(eng, kw):
    from paper_2507_23189_gb300 import _native as N
    with pytest.raises(N.McError) as e:
        eng.PhaseTable(**kw)
    assert e.value.status == -1


@pytest.mark.parametrize("d_um,m", [(5.0, complex(1.59, 0.0)), (1.0, complex(1.59, 0.0)),
                                   (10.0, complex(1.59, 0.0)), (2.0, complex(1.5, 0.01))])
def test_table_builder_matches_oracle(eng, oracle_mod, d_um, m):
    """Two independent double-precision routes to the same table."""
    t = eng.PhaseTable(diameter_um=d_um, n_particle=m, n_medium=1.33, wavelength_nm=532.0)
    x = oracle_mod.size_parameter(d_um, 1.33, 532.0)
    mr = m / 1.33
    qe, qs, g = oracle_mod.mie_efficiencies(mr, x)
    info = t.info
    assert info["x"] == pytest.approx(x, rel=1e-14)
    assert info["qext"] == pytest.approx(qe, rel=1e-11)
    assert info["qsca"] == pytest.approx(qs, rel=1e-11)
    assert info["g"] == pytest.approx(g, abs=1e-11)
    assert info["sigma_ext_mm2"] == pytest.approx(oracle_mod.cross_section_mm2(qe, d_um), rel=1e-11)
    ot = oracle_mod.phase_table(oracle_mod.PHASE_MIE, mr, x)
    np.testing.assert_allclose(t.omu64, ot["omu"], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(t.pdf64, ot["pdf"], rtol=1e-8)
    assert info["g_table"] == pytest.approx(ot["mean"], abs=1e-12)


@pytest.mark.parametrize("d_um,m,n_med,lam,n_bins,rtol", [(0.05, complex(1.59, 0.0), 1.33, 532.0, 4096, 1e-9),
                                                          (3.0, complex(1.5, 0.5), 1.33, 532.0, 1024, 1e-9),
                                                          (5.0, complex(1.59, 0.0), 1.0, 633.0, 64, 1e-9),
                                                          (5.0, complex(1.59, 0.0), 1.33, 532.0, 16384, 1e-9),
                                                          (2.0, complex(2.5, 0.001), 1.33, 532.0, 4096, 1e-9),
                                                          (30.0, complex(1.59, 0.0), 1.33, 532.0, 4096, 1e-8)])
def test_table_builder_matches_oracle_across_sizes_media_and_bins(eng, oracle_mod, d_um, m, n_med, lam, n_bins,
                                                                    rtol):
    """The same two routes for a Rayleigh-sized sphere, a strongly absorbing
    one, a sphere in air at 633 nm, the smallest and largest tables, a
    high-index sphere and a 30 um one (x = 236, where the forward peak is
    1/x wide and the two quadratures differ by a few 1e-9)."""
    t = eng.PhaseTable(diameter_um=d_um, n_particle=m, n_medium=n_med, wavelength_nm=lam, n_bins=n_bins)
    x = oracle_mod.size_parameter(d_um, n_med, lam)
    mr = m / n_med
    qe, qs, g = oracle_mod.mie_efficiencies(mr, x)
    assert t.info["x"] == pytest.approx(x, rel=1e-14)
    assert t.info["qext"] == pytest.approx(qe, rel=1e-10)
    assert t.info["qsca"] == pytest.approx(qs, rel=1e-10)
    assert t.info["g"] == pytest.approx(g, abs=1e-10)
    ot = oracle_mod.phase_table(oracle_mod.PHASE_MIE, mr, x, n_bins=n_bins)
    np.testing.assert_allclose(t.omu64, ot["omu"], rtol=rtol, atol=1e-15)
    np.testing.assert_allclose(t.pdf64, ot["pdf"], rtol=10 * rtol)


def test_packed_table_layout(eng):
    t = eng.PhaseTable()
    b = t.blob
    hdr = np.frombuffer(b[:64].tobytes(), dtype=np.uint32)
    assert hdr[0] == 0x544D434D and hdr[1] == 1
    n = int(hdr[2])
    off_omu, off_pdf, off_guide, total = (int(v) for v in hdr[4:8])
    assert total == b.size and off_omu % 16 == 0 and off_pdf % 16 == 0 and off_guide % 16 == 0
    omu = np.frombuffer(b[off_omu:off_omu + 4 * (n + 1)].tobytes(), dtype=np.float32)
    pdf = np.frombuffer(b[off_pdf:off_pdf + 4 * n].tobytes(), dtype=np.float32)
    guide = np.frombuffer(b[off_guide:off_guide + 2 * (n + 1)].tobytes(), dtype=np.uint16)
    np.testing.assert_array_equal(omu, t.omu64.astype(np.float32))
    np.testing.assert_array_equal(pdf, t.pdf64.astype(np.float32))
    # guide brackets the kernel's single-precision lookup: for a direction
    # cosine m in cell c = floor(fl(m + 1) n/2), the largest j with
    # omu[j] >= fl(1 - m) lies in [guide[c], guide[c + 1]]
    rng = np.random.default_rng(3)
    m = np.concatenate([rng.uniform(-1, 1, 20000), 1 - rng.uniform(0, 1e-3, 5000),
                        np.linspace(-1, 1, 8193)]).astype(np.float32)
    m = np.clip(m, np.float32(-1), np.float32(1))
    cell = np.minimum(np.floor((m + np.float32(1)) * np.float32(n / 2)).astype(np.int64), n - 1)
    om = np.float32(1) - m
    j = np.searchsorted(-omu, -om, side="right") - 1
    j = np.clip(j, 0, n - 1)
    assert np.all(guide[cell] <= j) and np.all(j <= guide[cell + 1])
    # and brackets are tight: most cells hold a single candidate bin
    assert np.mean(guide[1:] == guide[:-1]) > 0.5


def test_medium_from_density_eq17(eng):
    t = eng.PhaseTable(n_particle=complex(1.59, 0.001))
    med = eng.Medium.from_optical_depth(t, 5.0, 45.0, mu_a_medium=0.002)
    mu_ext = med.mu_s + med.mu_a - 0.002
    assert mu_ext * 45.0 == pytest.approx(5.0, rel=1e-12)
    assert med.mu_a - 0.002 == pytest.approx(mu_ext * t.info["qabs"] / t.info["qext"], rel=1e-10)


def test_workspace_and_argument_checks_without_gpu(eng):
    from paper_2507_23189_gb300 import _native as N
    L = N.lib()
    cam = N.Camera(64, 64, 128, 7.0)
    assert L.mc_workspace_bytes(C.byref(cam)) >= 8
    assert L.mc_workspace_bytes(C.byref(N.Camera(0, 64, 128, 7.0))) == 0
    # invalid arguments are rejected before any CUDA call
    med = N.Medium(-1.0, 0.0, N.PHASE_HG, 0.5, None, 0)
    geo = N.Geometry(45.0, 10.0, 10.0, 0.0)
    run = N.RunParams(10, 0, 1, 1e-4, 0.1, 1000, 0, 32, 0, 0, 0, 0)
    tal = N.Tallies(None, None, None, None, None, 0)
    assert L.mc_run(C.byref(med), C.byref(geo), C.byref(cam), C.byref(run), C.byref(tal), None) == -1
    med = N.Medium(0.1, 0.0, N.PHASE_HG, 1.0, None, 0)
    assert L.mc_run(C.byref(med), C.byref(geo), C.byref(cam), C.byref(run), C.byref(tal), None) == -1
    med = N.Medium(0.1, 0.0, N.PHASE_TABLE, 0.0, None, 4096)
    assert L.mc_run(C.byref(med), C.byref(geo), C.byref(cam), C.byref(run), C.byref(tal), None) == -1
    assert L.mc_check(None, None) == -1


def test_peaks_library_exports(eng):
    from paper_2507_23189_gb300 import build
    L = C.CDLL(build.PEAKS_LIB)
    assert hasattr(L, "mc_peak_run")
    L.mc_peak_run.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    assert L.mc_peak_run(0, 0, 256, 10, None, None, None) == -1   # rejected before any launch


def test_static_entry_rejects_an_invalid_camera_before_any_device_call(eng):
    """mc_run_static sizes its scratch from the camera; an invalid camera has
    no workspace size and is MC_ERR_ARG, decided on the host."""
    from paper_2507_23189_gb300 import _native as N
    import paper_2507_23189_gb300 as E
    L = N.lib()
    med = N.Medium()
    med.mu_s, med.phase_kind, med.hg_g = 0.1, N.PHASE_HG, 0.5
    geo = E.Geometry().as_c()
    rp = E.run_params(100)
    for cam in (N.Camera(0, 64, 128, 7.0), N.Camera(64, 64, 0, 7.0), N.Camera(64, 64, 128, -1.0)):
        assert L.mc_workspace_bytes(C.byref(cam)) == 0
        st = L.mc_run_static(C.byref(med), C.byref(geo), C.byref(cam), C.byref(rp),
                             None, None, None, None, None)
        assert st == -1, N.STATUS.get(st)
    # every valid camera's workspace fits the static array with room to spare
    for nx, nz, nr in ((1, 1, 1), (8192, 8192, 65536)):
        assert 0 < L.mc_workspace_bytes(C.byref(N.Camera(nx, nz, nr, 7.0))) <= 4096


def test_eq17_solved_for_the_number_density_in_c(eng):
    """mc_medium_from_optical_depth: OD = n sigma_e L (Eq. 17) with the
    paper's sigma_e = 4.42e-5 mm^2 for the 5 um spheres at 532 nm."""
    from paper_2507_23189_gb300 import _native as N
    L = N.lib()
    info = N.MieInfo(sigma_ext_mm2=4.42e-5, sigma_sca_mm2=4.0e-5, sigma_abs_mm2=0.42e-5)
    out, nd = N.Medium(), C.c_double(0.0)
    assert L.mc_medium_from_optical_depth(C.byref(info), 5.0, 45.0, 0.001, C.byref(out), C.byref(nd)) == 0
    assert nd.value == pytest.approx(5.0 / (4.42e-5 * 45.0), rel=1e-15)
    assert nd.value == pytest.approx(2513.8260432378, rel=1e-12)
    assert out.mu_s == pytest.approx(nd.value * 4.0e-5, rel=1e-15)
    assert out.mu_a == pytest.approx(nd.value * 0.42e-5 + 0.001, rel=1e-15)
    assert (out.mu_s + out.mu_a - 0.001) * 45.0 == pytest.approx(5.0, rel=1e-14)
    assert L.mc_medium_from_optical_depth(C.byref(info), 5.0, 45.0, 0.0, C.byref(out), None) == 0
    for tau, length, sig in ((-1.0, 45.0, 4.42e-5), (5.0, 0.0, 4.42e-5), (float("nan"), 45.0, 4.42e-5),
                             (5.0, float("inf"), 4.42e-5), (5.0, 45.0, 0.0)):
        bad = N.MieInfo(sigma_ext_mm2=sig, sigma_sca_mm2=sig)
        assert L.mc_medium_from_optical_depth(C.byref(bad), tau, length, 0.0, C.byref(out), None) == -1
    assert L.mc_medium_from_optical_depth(None, 5.0, 45.0, 0.0, C.byref(out), None) == -1


def test_auto_image_fraction_bits(eng):
    """F = min(32, 54 - ceil(log2 n)), at least 8: 24 at 1e9 photons."""
    L = eng.lib()
    want = {0: 32, 1: 32, 1 << 22: 32, (1 << 22) + 1: 31, 10 ** 8: 27, 10 ** 9: 24, 1 << 31: 23,
            1 << 46: 8, 1 << 63: 8}
    for n, f in want.items():
        assert L.mc_auto_frac_bits(n) == f, n
        assert eng.auto_frac_bits(n) == f
    for n in (3, 1000, 10 ** 6, 5 * 10 ** 7, 3 * 10 ** 9):
        f = L.mc_auto_frac_bits(n)
        # n photons at one weight unit each in one pixel stay 2^9 below 2^63
        assert f == 32 or (n * 2.0 ** f <= 2.0 ** 54 < n * 2.0 ** (f + 1))


def test_photon_cap_and_automatic_fraction_bits_are_checked_on_the_host(eng):
    """More than 2^31 photons in one call (the 2^-32-unit totals could pass
    2^63), or an automatic F while accumulating (the image being added to
    has its own F), is MC_ERR_ARG; the controls pass every argument check and
    stop at the too-small workspace (MC_ERR_NOMEM), before any CUDA call."""
    from paper_2507_23189_gb300 import _native as N
    L = N.lib()
    buf = (C.c_uint64 * 64)()
    p = C.addressof(buf) + (-C.addressof(buf)) % 16
    med = N.Medium(0.1, 0.0, N.PHASE_HG, 0.5, None, 0)
    geo = N.Geometry(45.0, 10.0, 10.0, 0.0)
    cam = N.Camera(64, 64, 128, 7.0)
    tal = N.Tallies(p, p, p, p, p, 0)

    def run(n, frac, acc):
        rp = N.RunParams(n, 0, 1, 1e-4, 0.1, 1000, 0, frac, acc, 0, 0, 0)
        return L.mc_run(C.byref(med), C.byref(geo), C.byref(cam), C.byref(rp), C.byref(tal), None)

    assert run(1 << 31, 32, 0) == -3
    assert run((1 << 31) + 1, 32, 0) == -1
    assert run(1000, 0, 0) == -3
    assert run(1000, 0, 1) == -1
    assert run(1000, 32, 1) == -3
    assert run(1000, 7, 0) == -1 and run(1000, 49, 0) == -1


def test_weighted_table_rejects_bad_arguments_on_the_host(eng):
    """mc_phase_table_weighted: a table medium, 2..256 weights, an aligned
    output of at least mc_table_bytes and not the input blob; all decided
    before any CUDA call."""
    from paper_2507_23189_gb300 import _native as N
    L = N.lib()
    buf = (C.c_uint64 * 64)()
    p = C.addressof(buf) + (-C.addressof(buf)) % 16
    tb = L.mc_table_bytes(4096)
    base = N.Medium(0.1, 0.0, N.PHASE_TABLE, 0.0, p, 4096)
    q = p + 256
    for args in ((base, 1, p, q, tb, p), (base, 257, p, q, tb, p), (base, 8, None, q, tb, p),
                 (base, 8, p, None, tb, p), (base, 8, p, q + 4, tb, p), (base, 8, p, p, tb, p),
                 (base, 8, p, q, tb, None)):
        m, nw, w, out, nb, err = args
        assert L.mc_phase_table_weighted(C.byref(m), nw, w, out, nb, err, None) == -1, args
    hg = N.Medium(0.1, 0.0, N.PHASE_HG, 0.5, None, 0)
    assert L.mc_phase_table_weighted(C.byref(hg), 8, p, q, tb, p, None) == -1
    assert L.mc_phase_table_weighted(C.byref(base), 8, p, q, tb - 16, p, None) == -3


def test_null_score_gradient_checks_its_majorant_scale(eng):
    """mc_grid_adjoint_nulls wants 1 < majorant_scale <= 16 (finite), decided
    before anything else is looked at."""
    from paper_2507_23189_gb300 import _native as N
    L = N.lib()
    for bad in (1.0, 0.5, 17.0, float("nan"), float("inf")):
        assert L.mc_grid_adjoint_nulls(None, None, None, None, None, None, None, bad, None, None, None, None, 0,
                                       None) == -1
