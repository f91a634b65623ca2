"""The engine's paper-faithful table (mie_paper_table_build, host code; no
GPU needed): its cumulative distribution against the oracle's, the integer
search thresholds against a double-precision search, and the guides that
narrow the kernel's two bisections (the answer must be the same as over the
whole table)."""
import numpy as np
import pytest

M_PS = complex(1.59 / 1.33, 0.0)


@pytest.fixture(scope="module")
def eng_paper():
    from paper_2507_23189_gb300 import build
    build.build()
    import paper_2507_23189_gb300 as g
    return g.PaperTable(n_theta=3000)


GUIDE = 4096


def _header(blob):
    h = np.frombuffer(blob[:64].tobytes(), dtype=np.uint32)
    return dict(magic=int(h[0]), version=int(h[1]), n_theta=int(h[2]), n_int=int(h[3]), off_k=int(h[4]),
                off_dl=int(h[5]), off_ri=int(h[6]), off_omu=int(h[7]), off_pth=int(h[8]), total=int(h[9]),
                top=int(np.frombuffer(blob[44:48].tobytes(), dtype=np.int32)[0]), off_gq=int(h[13]),
                off_go=int(h[14]))


def _guide(blob, off):
    return np.frombuffer(blob[off:off + 2 * (GUIDE + 1)].tobytes(), dtype=np.uint16).astype(np.int64)


def _guided_bisection(a, g, cell, v):
    """The kernel's search: largest i in [g[cell], g[cell + 1]] with a[i] <= v."""
    lo, hi = g[cell].copy(), g[cell + 1].copy()
    while np.any(lo < hi):
        act = lo < hi
        mid = (lo + hi + 1) >> 1
        le = np.zeros_like(act)
        le[act] = a[mid[act]] <= v[act]
        lo = np.where(act & le, mid, lo)
        hi = np.where(act & ~le, mid - 1, hi)
    return lo


def test_cdf_matches_oracle(eng_paper, oracle_mod):
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    o = oracle_mod.paper_cdf(oracle_mod.PHASE_MIE, M_PS, x, n_theta=3000)
    np.testing.assert_allclose(eng_paper.cdf64, o["cdf"], rtol=0, atol=1e-12)
    assert eng_paper.info["g_table"] == pytest.approx(
        np.sum(np.diff(o["cdf"]) * np.diff(np.sin(o["theta"])) / (np.pi / 2999)), abs=1e-12)


def test_integer_thresholds_reproduce_the_double_search(eng_paper):
    h = _header(eng_paper.blob)
    assert h["n_theta"] == 3000 and h["top"] == 2048
    _check_thresholds(eng_paper)


@pytest.mark.parametrize("n_theta", [16, 181, 2049, 8000, 16384])
def test_integer_thresholds_for_other_grids(eng_paper, n_theta):
    import paper_2507_23189_gb300 as g
    t = g.PaperTable(n_theta=n_theta)
    h = _header(t.blob)
    assert h["n_theta"] == n_theta and h["n_int"] == n_theta - 1
    # binary lifting over intervals 0 .. n_int - 1 starts at the largest power
    # of two below n_int, whose steps reach index 2 top - 1 >= n_int - 1
    top = h["top"]
    assert top & (top - 1) == 0 and top < h["n_int"] <= 2 * top
    _check_thresholds(t)


def _check_thresholds(table):
    b = table.blob
    h = _header(b)
    n = h["n_int"]
    assert h["magic"] == 0x504D434D and h["total"] == b.size
    K = np.frombuffer(b[h["off_k"]:h["off_k"] + 4 * (n + 1)].tobytes(), dtype=np.uint32).astype(np.int64)
    dl = np.frombuffer(b[h["off_dl"]:h["off_dl"] + 4 * n].tobytes(), dtype=np.float32).astype(np.float64)
    ri = np.frombuffer(b[h["off_ri"]:h["off_ri"] + 4 * n].tobytes(), dtype=np.float32).astype(np.float64)
    cdf = table.cdf64
    assert K[0] == 0 and K[n] == 1 << 23 and np.all(np.diff(K) >= 0)
    q = np.concatenate([np.arange(0, 1 << 23, 997), [0, (1 << 23) - 1], K[:n], np.maximum(K[:n] - 1, 0)])
    u = (q + 0.5) * 2.0 ** -23
    want = np.searchsorted(cdf[:n], u, side="right") - 1      # largest i with cdf[i] <= u
    got = np.searchsorted(K[:n], q, side="right") - 1         # largest i with K[i] <= q
    np.testing.assert_array_equal(got, want)
    # the kernel's bisection inside the guide's bracket finds the same interval,
    # for every one of the 2^23 uniform indices
    assert h["version"] == 2
    gq = _guide(b, h["off_gq"])
    qa = np.arange(1 << 23, dtype=np.int64)
    want_all = np.searchsorted(K[:n], qa, side="right") - 1
    cell = qa // ((1 << 23) // GUIDE)
    assert np.all(gq[cell] <= want_all) and np.all(want_all <= gq[cell + 1])
    np.testing.assert_array_equal(_guided_bisection(K, gq, cell, qa), want_all)
    # the interpolation aids give the fraction (u - cdf_i) / (cdf_{i+1} - cdf_i)
    i = got
    frac = ((q - K[i]) * 2.0 ** -23 + dl[i]) * ri[i]
    exact = (u - cdf[i]) / (cdf[i + 1] - cdf[i])
    np.testing.assert_allclose(frac, exact, rtol=0, atol=2e-6)


def test_bad_sizes_rejected(eng_paper):
    import paper_2507_23189_gb300 as g
    for n in (0, 15, 16385):
        with pytest.raises(Exception):
            g.PaperTable(n_theta=n)


@pytest.mark.parametrize("n_theta,d_um,m", [(181, 5.0, complex(1.59, 0.0)), (3000, 1.0, complex(1.59, 0.0)),
                                            (1001, 2.0, complex(1.5, 0.05)), (8000, 10.0, complex(1.59, 0.0)),
                                            (3000, 30.0, complex(1.59, 0.0)), (3000, 2.0, complex(2.5, 0.001))])
def test_cdf_matches_oracle_across_grids_and_particles(eng_paper, oracle_mod, n_theta, d_um, m):
    import paper_2507_23189_gb300 as g
    t = g.PaperTable(diameter_um=d_um, n_particle=m, n_theta=n_theta)
    x = oracle_mod.size_parameter(d_um, 1.33, 532.0)
    o = oracle_mod.paper_cdf(oracle_mod.PHASE_MIE, m / 1.33, x, n_theta=n_theta)
    np.testing.assert_allclose(t.cdf64, o["cdf"], rtol=0, atol=1e-12)
    assert t.cdf64[0] == 0.0 and t.cdf64[-1] == 1.0 and np.all(np.diff(t.cdf64) >= 0)


@pytest.mark.parametrize("n_theta", [16, 2049, 3000, 16384])
def test_camera_interval_search_by_guided_bisection(eng_paper, n_theta):
    """The camera density's interval: the largest i < n_int with omu[i] <=
    1 - cos(theta_c), found by the kernel's bisection inside the guide's
    bracket over the blob's omu (1 - cos(i pi / n_int) in single precision)."""
    import paper_2507_23189_gb300 as g
    t = eng_paper if n_theta == 3000 else g.PaperTable(n_theta=n_theta)
    b = t.blob
    h = _header(b)
    n = h["n_int"]
    omu = np.frombuffer(b[h["off_omu"]:h["off_omu"] + 4 * n_theta].tobytes(), dtype=np.float32)
    th = np.arange(n_theta) * np.pi / n
    np.testing.assert_allclose(omu, 2 * np.sin(th / 2) ** 2, rtol=1e-6, atol=1e-12)
    rng = np.random.default_rng(n_theta)
    om = np.concatenate([rng.uniform(0, 2, 20000), omu[:n], np.nextafter(omu[:n], np.float32(-1)), [0.0, 2.0]])
    om = np.clip(om.astype(np.float32), 0, 2)
    edges = (np.arange(GUIDE + 1) * (2.0 / GUIDE)).astype(np.float32)
    om = np.concatenate([om, edges, np.nextafter(edges, np.float32(-1)), np.nextafter(edges, np.float32(3))])
    om = np.clip(om, 0, 2).astype(np.float32)
    want = np.maximum(np.searchsorted(omu[:n], om, side="right") - 1, 0)
    go = _guide(b, h["off_go"])
    cell = np.minimum(np.floor(om * np.float32(GUIDE / 2)).astype(np.int64), GUIDE - 1)   # exact product
    assert np.all(go[cell] <= want) and np.all(want <= go[cell + 1])
    np.testing.assert_array_equal(_guided_bisection(omu, go, cell, om), want)
