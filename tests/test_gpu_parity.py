"""CUDA walk vs the double-precision oracle on the same seeds and inputs.

Traces: the first 32 events of 4096 photons (rule in tests/parity.py).
Tallies: the 10x10x45 mm cuvette at tau = 1 with 1e6 photons, 64x64 image,
Mie and H-G (g from the Mie series), every bin within 3 sigma and pooled
chi-square p > 0.01, both on the same seed and on independent seeds.
"""
import math

import numpy as np
import pytest

from parity import compare_traces, gpu_batches, oracle_var, tally_agreement, report_unmatched

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _media(gpu, oracle_mod, ps_table, tau, phase, mu_a=0.0):
    mu_ext = tau / LX
    mu_s = mu_ext - mu_a
    g_eng = ps_table.info["g"]
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    g_or = oracle_mod.mie_efficiencies(complex(1.59 / 1.33, 0.0), x)[2]
    med = gpu.Medium(mu_s, mu_a, "table" if phase == "mie" else "hg", g_eng, ps_table)
    return med, dict(mu_s=mu_s, mu_a=mu_a, phase=phase if phase == "hg" else "mie", hg_g=g_or)


def _gpu_run(gpu, med, n, nx, nz, seed=1, trace=0, ev=32, **kw):
    eng = gpu.Engine(gpu.Camera(nx, nz, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    tr = None
    if trace:
        tr = gpu.decode_trace(eng.trace(med, n, trace, ev, seed=seed, **kw))
    else:
        eng.run(med, n, seed=seed, **kw)
    eng.check()
    return eng.result(), tr


TRACE_CASES = [
    ("mie", 5.0, 0.0, {}),
    ("hg", 5.0, 0.0, {}),
    ("mie", 20.0, 0.08, dict(rr_threshold=0.02)),   # absorption + roulette inside 32 events
    ("hg", 20.0, 0.08, dict(rr_threshold=0.02)),
    ("mie", 1.0, 0.0, {}),
]


@pytest.mark.parametrize("phase,tau,mu_a,kw", TRACE_CASES)
def test_trace_parity_first_32_events(gpu, oracle_mod, ps_table, ps_oracle_table, phase, tau, mu_a, kw):
    n = 4096
    med, om = _media(gpu, oracle_mod, ps_table, tau, phase, mu_a)
    res, tr = _gpu_run(gpu, med, n, 64, 64, seed=11, trace=n, ev=32, **kw)
    ores = oracle_mod.walk(table=ps_oracle_table, n_photons=n, nx=64, nz=64, seed=11, n_trace=n,
                           n_trace_events=32, **om, **kw)
    cmp = compare_traces(tr, ores["trace"], mu_ext=tau / LX)
    print(phase, tau, mu_a, cmp["matched"], "/", cmp["n"], "flips", cmp["flips"], "worst", cmp["worst"],
          "events", cmp["events"])
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp["bad"]
    assert cmp["events"] > 1.5 * n
    if kw:
        assert np.any(ores["trace"][..., 0] == 4), "roulette never fired"


def _tally_case(gpu, oracle_mod, ps_table, ps_oracle_table, phase, seed_gpu, seed_or, n=1_000_000,
                tau=1.0):
    med, om = _media(gpu, oracle_mod, ps_table, tau, phase)
    res = gpu_batches(gpu, med, n, 32, gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ),
                      seed=seed_gpu)
    ores = oracle_mod.walk(table=ps_oracle_table, n_photons=n, nx=64, nz=64, seed=seed_or, **om)
    return res, ores


@pytest.mark.parametrize("phase", ["mie", "hg"])
def test_tally_parity_same_seed(gpu, oracle_mod, ps_table, ps_oracle_table, phase):
    res, ores = _tally_case(gpu, oracle_mod, ps_table, ps_oracle_table, phase, 1, 1)
    var = oracle_var(ores) + res["var"]
    zmax, chi2, dof, p, z = tally_agreement(res["image"], ores["image"], var, ores["image_hits"])
    pop = ores["image_hits"] >= 20
    rel = np.abs(res["image"] - ores["image"])[pop] / ores["image"][pop]
    print(phase, "zmax", zmax, "chi2", chi2, "dof", dof, "p", p,
          "fp32-vs-fp64 per-bin rel err: median %.2e max %.2e" % (np.median(rel), rel.max()))
    assert zmax < 3.0 and p > 0.01 and dof > 500
    # exact photon-by-photon bookkeeping: escapes are integers in 2^-32 units
    n = ores["n_photons"]
    raw = res["raw_totals"]
    assert raw[0] + raw[1] + raw[2] == n << 32
    w = raw[:7].astype(np.float64) * 2.0 ** -32
    for k in range(3):
        sig = math.sqrt(max(ores["totals_sq"][k] - ores["totals"][k] ** 2 / n, 0.0))
        assert abs(w[k] - ores["totals"][k]) <= 3 * math.sqrt(2) * sig + 1e-9
    assert abs(res["steps"] - ores["steps"]) <= 1e-4 * ores["steps"]
    # ballistic photons are decided by u0 alone, identically on both sides
    assert w[6] == ores["totals"][6]


@pytest.mark.parametrize("phase", ["mie", "hg"])
def test_tally_agreement_independent_seeds(gpu, oracle_mod, ps_table, ps_oracle_table, phase):
    res, ores = _tally_case(gpu, oracle_mod, ps_table, ps_oracle_table, phase, 2, 1)
    var = oracle_var(ores) + res["var"]
    zmax, chi2, dof, p, z = tally_agreement(res["image"], ores["image"], var, ores["image_hits"])
    frac3 = float(np.mean(np.abs(z[var.ravel() > 0]) > 3.0))
    print(phase, "zmax", zmax, "chi2", chi2, "dof", dof, "p", p, "frac>3sigma", frac3)
    assert p > 0.01 and dof > 500
    # independent estimates: about 0.3 % of bins beyond 3 sigma by chance
    assert frac3 < 0.01 and zmax < 6.0
