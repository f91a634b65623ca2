"""The comparison rules the GPU parity tests apply (tests/parity.py), checked
on the CPU: a single-precision copy of an oracle trace matches itself; a
deviation beyond the 1e-5 tolerance fails the photon unless the oracle's
branch margin says the decision was a near tie; and the tally statistics
(z scores, pooled chi-square, the oracle's per-bin variance) are the textbook
ones."""
import numpy as np
import pytest

from parity import NEE_FLOOR, TOL, compare_traces, oracle_var, report_unmatched, tally_agreement

LX = 45.0


@pytest.fixture(scope="module")
def traced(oracle_mod):
    n, ev = 200, 16
    r = oracle_mod.walk(mu_s=5.0 / LX, mu_a=0.01, phase="hg", hg_g=0.8, n_photons=n, nx=32, nz=32, n_trace=n,
                        n_trace_events=ev, seed=11)
    return np.array(r["trace"], dtype=np.float64), 5.0 / LX + 0.01


def _as_engine(o):
    """What decode_trace() returns for a float32 engine trace of the same events."""
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    return dict(status=o[..., 0].astype(np.int32), r=f32(o[..., 1:4]), d=f32(o[..., 4:7]), w=f32(o[..., 7]),
                nee=f32(o[..., 8]), pix=o[..., 9].astype(np.int32), nee_bin=o[..., 10].astype(np.int32),
                rad_bin=o[..., 11].astype(np.int32))


def _collision(o, p0=0):
    """A photon from p0 on whose event 1 is a collision with a clear margin."""
    for p in range(p0, o.shape[0]):
        if o[p, 0, 0] == 0 and o[p, 1, 0] == 0 and o[p, 1, 12] > 10 * TOL:
            return p
    raise AssertionError("no photon with two clear collisions")


def test_single_precision_copy_matches(traced):
    o, mu_ext = traced
    c = compare_traces(_as_engine(o), o, mu_ext)
    assert c["matched"] == c["n"] and c["flips"] == 0 and c["events"] > 2 * c["n"]
    assert c["worst"]["pos"] < 1e-7 and c["worst"]["w"] < 1e-7


@pytest.mark.parametrize("field,index,scale", [("r", (1, 0), LX), ("d", (1, 1), 1.0), ("w", (1,), None),
                                               ("nee", (1,), None)])
def test_deviation_beyond_tolerance_fails_the_photon(traced, field, index, scale):
    o, mu_ext = traced
    p = _collision(o)
    for factor, ok in ((0.3, True), (3.0, False)):
        g = _as_engine(o)
        ref = g[field][p][index]
        step = factor * TOL * (scale if scale is not None else abs(ref))
        g[field][p][index] = ref + step
        c = compare_traces(g, o, mu_ext)
        assert (p not in c["bad"]) == ok, (field, factor)
        assert c["matched"] == c["n"] - (0 if ok else 1)


def test_discrete_decision_flip_needs_a_near_tie(traced):
    o, mu_ext = traced
    p = _collision(o)
    g = _as_engine(o)
    g["pix"][p, 1] += 1                       # another pixel, clear margin: a mismatch
    c = compare_traces(g, o, mu_ext)
    assert p in c["bad"] and c["flips"] == 0
    o2 = o.copy()
    o2[p, 1, 12] = 0.1 * TOL                  # the oracle's pixel coordinate sat on an edge: a tie
    c = compare_traces(g, o2, mu_ext)
    assert p not in c["bad"] and c["flips"] == 1


def test_events_after_a_tie_are_not_compared(traced):
    o, mu_ext = traced
    p = _collision(o)
    g = _as_engine(o)
    o2 = o.copy()
    o2[p, 1, 12] = 0.1 * TOL
    g["nee_bin"][p, 1] += 1                   # the tie at event 1 ...
    g["r"][p, 2:] += 1.0                      # ... and wildly different events after it
    c = compare_traces(g, o2, mu_ext)
    assert p not in c["bad"] and c["flips"] == 1


def test_tally_agreement_is_the_textbook_z_and_chi2():
    rng = np.random.default_rng(5)
    sig = rng.uniform(0.5, 2.0, 400)
    z = rng.standard_normal(400)
    b = rng.uniform(10, 20, 400)
    a = b + sig * z
    hits = np.where(np.arange(400) % 4 == 0, 5, 100)      # a quarter of the bins too thin to pool
    zmax, chi2, dof, p, zz = tally_agreement(a, b, sig ** 2, hits, min_hits=20)
    np.testing.assert_allclose(zz, z, rtol=1e-12)
    assert zmax == pytest.approx(np.max(np.abs(z)), rel=1e-12)
    assert dof == 300 and chi2 == pytest.approx(np.sum(z[hits >= 20] ** 2), rel=1e-12)
    scipy_stats = pytest.importorskip("scipy.stats")
    assert p == pytest.approx(scipy_stats.chi2.sf(chi2, 300), rel=1e-12)


def test_oracle_var_is_n_times_the_sample_variance():
    rng = np.random.default_rng(8)
    n = 1000
    x = rng.exponential(1.0, (n, 3, 4)) * (rng.uniform(size=(n, 3, 4)) < 0.3)   # per-photon contributions
    res = dict(n_photons=n, image=x.sum(axis=0), image_sq=(x * x).sum(axis=0))
    np.testing.assert_allclose(oracle_var(res), n * x.var(axis=0, ddof=1), rtol=1e-10)


def test_every_unmatched_photon_is_reported_with_its_cause(traced, capsys):
    o, mu_ext = traced
    p = _collision(o)
    g = _as_engine(o)
    g["d"][p][1, 1] += 3.0 * TOL
    c = compare_traces(g, o, mu_ext)
    report_unmatched(c, "case")
    out = capsys.readouterr().out.strip().splitlines()
    assert c["matched"] == c["n"] - 1 and len(out) == 1
    assert out[0].startswith("unmatched case: photon %d event 1: position" % p) and "direction" in out[0]


def test_camera_terms_below_any_tally_unit_are_compared_absolutely(traced):
    """A camera term that single precision flushes to zero (the oracle's 1e-98
    against the engine's 0) matches; one that a tally could register does
    not (the floor is far below the finest image unit over a whole run:
    2.1e15 terms of 1e-31 add to 2.1e-16 < 2^-48)."""
    o, mu_ext = traced
    assert 2.0 ** 31 * 1e6 * NEE_FLOOR < 2.0 ** -48
    p = _collision(o)
    for oracle_value, ok in ((1e-98, True), (1e-33, True), (1e-20, False)):
        oo = o.copy()
        oo[p, 1, 8] = oracle_value
        g = _as_engine(oo)
        g["nee"][p][1] = 0.0
        c = compare_traces(g, oo, mu_ext)
        assert (p not in c["bad"]) == ok, oracle_value


def test_camera_allowance_for_a_deep_transmittance(traced):
    """With the half-height given, a camera term may also differ by 2^-22 times
    the bound mu_ext (hy - r_y) on its transmittance's optical depth: a 3e-5
    difference passes where that bound is 200, and fails without it."""
    o, mu_ext = traced
    p = _collision(o)
    hy = o[p, 1, 2] + 200.0 / mu_ext
    g = _as_engine(o)
    g["nee"][p][1] = o[p, 1, 8] * (1.0 + 3e-5)
    assert p in compare_traces(g, o, mu_ext)["bad"]
    assert p not in compare_traces(g, o, mu_ext, hy=hy)["bad"]
    g["nee"][p][1] = o[p, 1, 8] * (1.0 + 1e-4)
    assert p in compare_traces(g, o, mu_ext, hy=hy)["bad"]
