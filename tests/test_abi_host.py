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


@pytest.mark.parametrize("d_um,m,n_med,lam,n_bins", [(0.05, complex(1.59, 0.0), 1.33, 532.0, 4096),
                                                     (3.0, complex(1.5, 0.5), 1.33, 532.0, 1024),
                                                     (5.0, complex(1.59, 0.0), 1.0, 633.0, 64),
                                                     (5.0, complex(1.59, 0.0), 1.33, 532.0, 16384)])
def test_table_builder_matches_oracle_across_sizes_media_and_bins(eng, oracle_mod, d_um, m, n_med, lam, n_bins):
    """The same two routes for a Rayleigh-sized sphere, a strongly absorbing
    one, a sphere in air at 633 nm and the smallest and largest tables."""
    t = eng.PhaseTable(diameter_um=d_um, n_particle=m, n_medium=n_med, wavelength_nm=lam, n_bins=n_bins)
    x = oracle_mod.size_parameter(d_um, n_med, lam)
    mr = m / n_med
    qe, qs, g = oracle_mod.mie_efficiencies(mr, x)
    assert t.info["x"] == pytest.approx(x, rel=1e-14)
    assert t.info["qext"] == pytest.approx(qe, rel=1e-10)
    assert t.info["qsca"] == pytest.approx(qs, rel=1e-10)
    assert t.info["g"] == pytest.approx(g, abs=1e-10)
    ot = oracle_mod.phase_table(oracle_mod.PHASE_MIE, mr, x, n_bins=n_bins)
    np.testing.assert_allclose(t.omu64, ot["omu"], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(t.pdf64, ot["pdf"], rtol=1e-8)


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
