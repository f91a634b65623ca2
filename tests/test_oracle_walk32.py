"""Pins for the oracle's single-precision mode (oracle/walk32.c, explicit
fused multiply-adds): the walk of Sec. 3.1.3 restated in IEEE single
precision. It is pinned by
  * the double-precision oracle (itself pinned by closed forms): every
    photon's first 32 events agree within single-precision accuracy under
    the trace rule of tests/parity.py, for the Mie table and H-G (the Mie
    table's g, strong back-scattering g = -0.9 and strong forward
    scattering g = 0.99), with absorption and roulette, with a finite beam;
  * Beer-Lambert: the share of photons whose first flight leaves through
    the far face is exp(-tau);
  * implicit capture (Eq. 16): after k collisions the weight is the albedo
    to the k-th power;
  * the H-G polar angle: the angle between successive directions against
    the double-precision inverse of Eq. 11's distribution at the event's
    own uniform.
"""
import math

import numpy as np
import pytest

from parity import compare_traces

LX = 45.0


def _as_engine(t32):
    """The FP32 trace in the layout compare_traces expects of a device trace."""
    return dict(status=t32[..., 0].astype(int), r=t32[..., 1:4], d=t32[..., 4:7], w=t32[..., 7],
                nee=t32[..., 8], pix=t32[..., 9].astype(int), nee_bin=t32[..., 10].astype(int),
                rad_bin=t32[..., 11].astype(int))


def _g(oracle_mod):
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    return oracle_mod.mie_efficiencies(complex(1.59 / 1.33, 0.0), x)[2]


CASES = [("mie", 5.0, 0.0, {}), ("mie", 20.0, 0.08, dict(rr_threshold=0.02)), ("hg", 5.0, 0.0, {}),
         ("hg", 1.0, 0.005, dict(beam_radius=1.25)), ("mie", 2.0, 0.0, dict(beam_radius=1.25)),
         ("hg", 5.0, 0.0, dict(hg_g=-0.9)), ("hg", 5.0, 0.0, dict(hg_g=0.99))]


@pytest.mark.parametrize("phase,tau,mu_a,kw", CASES)
def test_single_precision_walk_follows_the_double_precision_walk(oracle_mod, ps_oracle_table, phase, tau,
                                                                  mu_a, kw):
    n = 1024
    kw = dict(kw)
    g = kw.pop("hg_g", None)
    if phase == "hg" and g is None:
        g = _g(oracle_mod)
    om = dict(phase="mie", table=ps_oracle_table) if phase == "mie" else dict(phase="hg", hg_g=g)
    args = dict(mu_s=tau / LX - mu_a, mu_a=mu_a, nx=64, nz=64, seed=11, **om, **kw)
    t64 = oracle_mod.walk(n_photons=n, n_trace=n, n_trace_events=32, **args)["trace"]
    t32 = oracle_mod.walk32_trace(n_trace=n, n_trace_events=32, **args)
    slope = None
    if phase == "hg":
        slope = lambda mu: 3.0 * abs(g) / (1.0 + g * g - 2.0 * g * mu)
    cmp = compare_traces(_as_engine(t32), t64, mu_ext=tau / LX, nee_slope=slope)
    print(phase, tau, mu_a, kw, "matched %d/%d flips %d events %d worst %s" %
          (cmp["matched"], cmp["n"], cmp["flips"], cmp["events"], {k: "%.2e" % v for k, v in cmp["worst"].items()}))
    assert cmp["matched"] == n, cmp["causes"][:5]
    assert cmp["events"] > 1.2 * n
    assert cmp["worst"]["pos"] < 5e-6 and cmp["worst"]["dir"] < 5e-6 and cmp["worst"]["w"] < 5e-7


def test_ballistic_share_is_beer_lambert(oracle_mod, ps_oracle_table):
    n, tau = 20_000, 1.0
    t32 = oracle_mod.walk32_trace(mu_s=tau / LX, phase="mie", table=ps_oracle_table, n_trace=n, n_trace_events=1)
    share = float(np.mean(t32[:, 0, 0] == 2))
    p = math.exp(-tau)
    assert abs(share - p) < 4 * math.sqrt(p * (1 - p) / n), (share, p)


def test_weight_is_the_albedo_power(oracle_mod, ps_oracle_table):
    mu_s, mu_a = 10.0 / LX, 0.05
    t32 = oracle_mod.walk32_trace(mu_s=mu_s, mu_a=mu_a, phase="mie", table=ps_oracle_table, n_trace=256,
                                  n_trace_events=32, rr_threshold=0.0)
    a = np.float32(mu_s / (mu_s + mu_a))
    for p in range(256):
        w = np.float32(1.0)
        for e in range(32):
            st = t32[p, e, 0]
            if st != 0:
                break
            w = np.float32(w * a)
            assert t32[p, e, 7] == pytest.approx(float(a) ** (e + 1), rel=1e-5)
            assert t32[p, e, 7] == float(w)


def test_hg_polar_angle_is_the_inverse_distribution(oracle_mod):
    g = 0.87
    n = 512
    t32 = oracle_mod.walk32_trace(mu_s=10.0 / LX, phase="hg", hg_g=g, n_trace=n, n_trace_events=32, seed=5)
    checked = 0
    for p in range(n):
        d_prev = np.array([1.0, 0.0, 0.0])
        for e in range(32):
            if t32[p, e, 0] != 0:
                break
            u1 = oracle_mod.uniform(oracle_mod.philox4x32_10([[p, 0, e, 0]], 5)[0, 1])
            q = (1 - g * g) / (1 - g + 2 * g * u1)
            mu = (1 + g * g - q * q) / (2 * g)
            d = t32[p, e, 4:7]
            assert float(np.dot(d, d_prev)) == pytest.approx(mu, abs=2e-6), (p, e)
            d_prev = d
            checked += 1
    assert checked > 2 * n


def _random_configs(seed=7, n=8):
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for k in range(n):
        lx, ly, lz = (float(v) for v in np.exp(rng.uniform(np.log(0.5), np.log(100.0), 3)))
        tau = float(np.exp(rng.uniform(np.log(0.05), np.log(30.0))))
        g = float(rng.uniform(-0.95, 0.99))
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(15.0))))
        mu_a = float(tau / lx * rng.uniform(0.0, 0.5)) if k % 2 else 0.0
        beam = float(rng.uniform(0.0, 0.5) * min(ly, lz)) if k % 4 == 1 else 0.0
        out.append(dict(lx=lx, ly=ly, lz=lz, tau=tau, phase="hg" if k % 3 == 2 else "mie", g=g, d=d, mu_a=mu_a,
                        beam=beam, nx=int(rng.integers(1, 200)), nz=int(rng.integers(1, 200)),
                        rr=(float(rng.uniform(1e-4, 0.05)), float(rng.uniform(0.0, 0.5)))))
    return out


@pytest.mark.parametrize("k", range(8))
def test_single_precision_walk_follows_the_double_precision_walk_in_random_set_ups(oracle_mod, k):
    """The FP32 mode against the FP64 walk over seeded random cuvettes, optical
    depths, particles (Mie tables) or H-G anisotropies, absorption, roulette,
    beams and cameras: the precision the engine's strict build is compared
    with holds outside the hand-picked cases too (the trace rule, with the
    camera transmittance's rounding allowance)."""
    c = _random_configs()[k]
    n = 1024
    mu_ext = c["tau"] / c["lx"]
    if c["phase"] == "mie":
        x = oracle_mod.size_parameter(c["d"], 1.33, 532.0)
        om = dict(phase="mie", table=oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x))
        slope = None
    else:
        g = c["g"]
        om = dict(phase="hg", hg_g=g)
        slope = lambda mu: 3.0 * abs(g) / (1.0 + g * g - 2.0 * g * mu)
    args = dict(mu_s=mu_ext - c["mu_a"], mu_a=c["mu_a"], lx=c["lx"], ly=c["ly"], lz=c["lz"], beam_radius=c["beam"],
                nx=c["nx"], nz=c["nz"], r_max=0.5 * math.hypot(c["ly"], c["lz"]), seed=23,
                rr_threshold=c["rr"][0], rr_survival=c["rr"][1], **om)
    t64 = oracle_mod.walk(n_photons=n, n_trace=n, n_trace_events=32, **args)["trace"]
    t32 = oracle_mod.walk32_trace(n_trace=n, n_trace_events=32, **args)
    cmp = compare_traces(_as_engine(t32), t64, mu_ext=mu_ext, lx=c["lx"], nee_slope=slope, hy=0.5 * c["ly"])
    print(k, c["phase"], round(c["tau"], 3), "matched %d/%d flips %d worst %s" %
          (cmp["matched"], n, cmp["flips"], {q: "%.2e" % v for q, v in cmp["worst"].items()}))
    for p, e, why in cmp["causes"]:
        print("  unmatched photon %d event %d: %s" % (p, e, why))
    assert cmp["matched"] >= 0.998 * n, cmp["causes"][:5]
    assert cmp["flips"] <= 0.01 * n      # no systematic tie decided differently


@pytest.mark.parametrize("lz,nz", [(21.034007022851252, 42), (5.6997014, 24), (10.0, 64)])
def test_first_collisions_on_the_axis_fall_in_row_nz_over_2(oracle_mod, lz, nz):
    """The pixel-tie reading in single precision: a pencil beam's first
    collision lies on z = 0 and belongs to row nz/2 for any cuvette height."""
    t32 = oracle_mod.walk32_trace(mu_s=0.1, phase="hg", hg_g=0.3, lx=20.0, ly=8.0, lz=lz, nx=8, nz=nz, n_trace=500,
                                  n_trace_events=2, seed=3)
    first = t32[:, 0, :]
    coll = first[:, 0] == 0
    assert coll.sum() > 100
    assert np.all(first[coll, 3] == 0.0)
    assert np.all(first[coll, 9].astype(int) // 8 == nz // 2)
