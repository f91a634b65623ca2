"""The CUDA walk against the oracle over seeded random configurations, so that
regimes no hand-picked case covers are checked as well: cuvette sides from
0.5 to 100 mm, optical depths from 0.05 to 50, Mie tables of spheres from
0.5 to 20 um (from nearly isotropic to strongly forward) or H-G with
g in (-0.95, 0.99), absorption up to half the extinction, roulette
thresholds and survival chances (the plain cut included), finite beams and
cameras of 1 to 300 pixels a side. Each configuration compares the first 32
events of 2048 photons under the trace rule (tests/parity.py) and prints
every photon it did not match with its cause. Random grids check delta
tracking the same way, and random media and cameras check the adjoint's
gradient against the oracle's on the same photons.
"""
import math

import numpy as np
import pytest

from parity import compare_traces, report_unmatched

pytestmark = pytest.mark.gpu

N_CONFIGS = 12


def _configs(seed=7, n=N_CONFIGS):
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for k in range(n):
        lx, ly, lz = (float(v) for v in np.exp(rng.uniform(np.log(0.5), np.log(100.0), 3)))
        tau = float(np.exp(rng.uniform(np.log(0.05), np.log(50.0))))
        phase = "hg" if k % 3 == 2 else "mie"
        g = float(rng.uniform(-0.95, 0.99))
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(20.0))))
        mu_ext = tau / lx
        mu_a = float(mu_ext * rng.uniform(0.0, 0.5)) if k % 2 else 0.0
        beam = float(rng.uniform(0.0, 0.5) * min(ly, lz)) if k % 4 == 1 else 0.0
        nx, nz = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        rr = (float(rng.uniform(1e-4, 0.05)), float(rng.uniform(0.0, 0.5)))
        out.append(dict(lx=lx, ly=ly, lz=lz, tau=tau, phase=phase, g=g, d=d, mu_a=mu_a, beam=beam, nx=nx, nz=nz,
                        rr=rr))
    return out


@pytest.mark.parametrize("k", range(N_CONFIGS))
def test_random_configuration_traces_match_oracle(gpu, oracle_mod, k):
    c = _configs()[k]
    n = 2048
    mu_ext = c["tau"] / c["lx"]
    mu_s = mu_ext - c["mu_a"]
    r_max = 0.5 * math.hypot(c["ly"], c["lz"])
    kw = dict(rr_threshold=c["rr"][0], rr_survival=c["rr"][1])
    if c["phase"] == "mie":
        med = gpu.Medium(mu_s, c["mu_a"], "table", 0.0, gpu.PhaseTable(diameter_um=c["d"]))
        x = oracle_mod.size_parameter(c["d"], 1.33, 532.0)
        om = dict(phase="mie", table=oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x))
        slope = None
    else:
        g = c["g"]
        med = gpu.Medium(mu_s, c["mu_a"], "hg", g)
        om = dict(phase="hg", hg_g=g)
        slope = lambda mu: 3.0 * abs(g) / (1.0 + g * g - 2.0 * g * mu)
    e = gpu.Engine(gpu.Camera(c["nx"], c["nz"], 128, r_max), gpu.Geometry(c["lx"], c["ly"], c["lz"], c["beam"]))
    tr = gpu.decode_trace(e.trace(med, n, n, 32, seed=31, **kw))
    e.check()
    o = oracle_mod.walk(mu_s=mu_s, mu_a=c["mu_a"], lx=c["lx"], ly=c["ly"], lz=c["lz"], beam_radius=c["beam"],
                        nx=c["nx"], nz=c["nz"], r_max=r_max, n_photons=n, seed=31, n_trace=n, n_trace_events=32,
                        **om, **kw)
    cmp = compare_traces(tr, o["trace"], mu_ext, lx=c["lx"], nee_slope=slope, hy=0.5 * c["ly"])
    print("config %d %s: matched %d/%d flips %d events %d worst %s" %
          (k, {q: (round(v, 3) if isinstance(v, float) else v) for q, v in c.items()}, cmp["matched"], n,
           cmp["flips"], cmp["events"], {q: "%.2e" % v for q, v in cmp["worst"].items()}))
    report_unmatched(cmp, "config %d" % k)
    assert cmp["matched"] >= 0.998 * n, cmp["causes"][:5]
    # near-tie flips end a photon's comparison; a systematic tie (every photon
    # deciding the same boundary differently) would show up as many of them
    assert cmp["flips"] <= 0.01 * n
    assert cmp["events"] >= n


N_GRID_CONFIGS = 8


def _grid_configs(seed=11, n=N_GRID_CONFIGS):
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for k in range(n):
        lx, ly, lz = (float(v) for v in np.exp(rng.uniform(np.log(1.0), np.log(60.0), 3)))
        gx, gy, gz = (int(v) for v in rng.integers(4, 41, 3))
        bx, by, bz = (int(rng.integers(1, v + 1)) for v in (gx, gy, gz))
        while ((gx + bx - 1) // bx) * ((gy + by - 1) // by) * ((gz + bz - 1) // bz) > 16384:
            bx += 1
        tau = float(np.exp(rng.uniform(np.log(0.1), np.log(20.0))))   # mean extinction times lx
        phase = "hg" if k % 2 else "mie"
        g = float(rng.uniform(-0.9, 0.95))
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(15.0))))
        k_ext = 4e-5
        albedo = float(rng.uniform(0.6, 1.0))
        mu_a = float(tau / lx * rng.uniform(0.0, 0.2)) if k % 3 == 0 else 0.0
        spread = float(rng.uniform(0.0, 1.2))
        out.append(dict(lx=lx, ly=ly, lz=lz, shape=(gz, gy, gx), block=(bx, by, bz), tau=tau, phase=phase, g=g, d=d,
                        k_ext=k_ext, k_sca=k_ext * albedo, mu_a=mu_a, spread=spread, seed=100 + k,
                        rr=(float(rng.uniform(1e-4, 0.05)), float(rng.uniform(0.0, 0.5)))))
    return out


@pytest.mark.parametrize("k", range(N_GRID_CONFIGS))
def test_random_grid_configuration_traces_match_oracle(gpu, oracle_mod, k):
    """Delta tracking over seeded random grids: 4 to 40 voxels a side, majorant
    cells from one voxel to the whole grid, log-normal densities of random
    spread scaled to optical depths 0.1 to 20 along lx, particle albedo 0.6 to
    1 and background absorption, the Mie table or H-G."""
    import torch
    from paper_2507_23189_gb300 import workloads as W
    c = _grid_configs()[k]
    n = 2048
    rough = W.rough_grid(c["shape"], c["seed"], mean=1.0, spread=c["spread"])
    dens = (rough * (c["tau"] / (c["k_ext"] * c["lx"] * float(rough.mean())))).astype(np.float32)
    geo = gpu.Geometry(c["lx"], c["ly"], c["lz"])
    grid = gpu.Grid(torch.from_numpy(dens).cuda(), c["k_ext"], c["k_sca"], c["mu_a"], c["block"]).prepare(geo)
    kw = dict(rr_threshold=c["rr"][0], rr_survival=c["rr"][1])
    if c["phase"] == "mie":
        med = gpu.Medium(1.0, 0.0, "table", 0.0, gpu.PhaseTable(diameter_um=c["d"]))
        x = oracle_mod.size_parameter(c["d"], 1.33, 532.0)
        om = dict(phase="mie", table=oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x))
        slope = None
    else:
        g = c["g"]
        med = gpu.Medium(1.0, 0.0, "hg", g)
        om = dict(phase="hg", hg_g=g)
        slope = lambda mu: 3.0 * abs(g) / (1.0 + g * g - 2.0 * g * mu)
    r_max = 0.5 * math.hypot(c["ly"], c["lz"])
    e = gpu.Engine(gpu.Camera(64, 64, 128, r_max), geo)
    tr = gpu.decode_trace(e.run_grid(grid, med, n, seed=37, n_trace=n, n_events=32, **kw))
    e.check()
    o = oracle_mod.walk(mu_s=0.0, mu_a=c["mu_a"], lx=c["lx"], ly=c["ly"], lz=c["lz"], nx=64, nz=64, r_max=r_max,
                        n_photons=n, seed=37, n_trace=n, n_trace_events=32,
                        grid=dict(density=dens.astype(np.float64), k_ext=c["k_ext"], k_sca=c["k_sca"],
                                  block=c["block"]), **om, **kw)
    cmp = compare_traces(tr, o["trace"], c["k_ext"] * float(dens.max()) + c["mu_a"], lx=c["lx"], nee_slope=slope,
                         hy=0.5 * c["ly"])
    print("grid config %d %s: matched %d/%d flips %d events %d worst %s" %
          (k, {q: (round(v, 3) if isinstance(v, float) else v) for q, v in c.items()}, cmp["matched"], n,
           cmp["flips"], cmp["events"], {q: "%.2e" % v for q, v in cmp["worst"].items()}))
    report_unmatched(cmp, "grid config %d" % k)
    assert cmp["matched"] >= 0.998 * n, cmp["causes"][:5]
    assert cmp["flips"] <= 0.01 * n
    assert cmp["events"] >= 0.5 * n     # thin media: many photons leave before any real event


N_ADJ_CONFIGS = 6


def _adjoint_configs(seed=13, n=N_ADJ_CONFIGS):
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for k in range(n):
        lx, ly, lz = (float(v) for v in np.exp(rng.uniform(np.log(2.0), np.log(60.0), 3)))
        tau = float(np.exp(rng.uniform(np.log(0.3), np.log(15.0))))
        phase = "hg" if k % 3 == 2 else "mie"
        g = float(rng.uniform(-0.8, 0.95))
        d = float(np.exp(rng.uniform(np.log(0.5), np.log(15.0))))
        mu_a = float(tau / lx * rng.uniform(0.0, 0.3)) if k % 2 else 0.0
        nx, nz = int(rng.integers(4, 96)), int(rng.integers(4, 96))
        out.append(dict(lx=lx, ly=ly, lz=lz, tau=tau, phase=phase, g=g, d=d, mu_a=mu_a, nx=nx, nz=nz,
                        rr=(float(rng.uniform(1e-4, 0.05)), float(rng.uniform(0.05, 0.5)))))
    return out


@pytest.mark.parametrize("k", range(N_ADJ_CONFIGS))
def test_random_configuration_adjoint_matches_oracle(gpu, oracle_mod, k):
    """The adjoint (mc_adjoint: d/d(mu_s, mu_a) and, with the Mie table, 64
    phase weights) on seeded random cuvettes, media and cameras against the
    oracle's gradient on the same photons: the value to 1e-4 and every
    component within 0.05 sigma + 1e-4 relative, as in the adjoint's own
    parity test."""
    import torch
    c = _adjoint_configs()[k]
    n = 30_000
    mu_ext = c["tau"] / c["lx"]
    mu_s = mu_ext - c["mu_a"]
    r_max = 0.5 * math.hypot(c["ly"], c["lz"])
    kw = dict(rr_threshold=c["rr"][0], rr_survival=c["rr"][1])
    adj = np.random.default_rng(100 + k).uniform(0.0, 1.0, (c["nz"], c["nx"])).astype(np.float32)
    e = gpu.Engine(gpu.Camera(c["nx"], c["nz"], 128, r_max), gpu.Geometry(c["lx"], c["ly"], c["lz"]))
    if c["phase"] == "mie":
        n_w = 64
        med = gpu.Medium(mu_s, c["mu_a"], "table", 0.0, gpu.PhaseTable(diameter_um=c["d"]))
        x = oracle_mod.size_parameter(c["d"], 1.33, 532.0)
        om = dict(phase="mie", table=oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x))
    else:
        n_w = 0
        med = gpu.Medium(mu_s, c["mu_a"], "hg", c["g"])
        om = dict(phase="hg", hg_g=c["g"])
    out = e.adjoint(med, torch.from_numpy(adj), n, n_w=n_w, seed=9, **kw).cpu().numpy()
    e.check()
    o = oracle_mod.adjoint(adj.astype(np.float64), n_w, mu_s=mu_s, mu_a=c["mu_a"], lx=c["lx"], ly=c["ly"],
                           lz=c["lz"], nx=c["nx"], nz=c["nz"], r_max=r_max, n_photons=n, seed=9, **om, **kw)
    g, g2 = o["grad"], o["grad_sq"]
    sig = np.sqrt(np.maximum(g2 - g ** 2 / n, 0))
    d = np.abs(out[1:] - g)
    print("adjoint config %d %s: value %.6g vs %.6g, max |diff|/sigma %.3g" %
          (k, {q: (round(v, 3) if isinstance(v, float) else v) for q, v in c.items()}, out[0], o["value"],
           float(np.max(d / np.maximum(sig, 1e-300)))))
    assert out[0] == pytest.approx(o["value"], rel=1e-4, abs=1e-9)
    assert np.all(d <= 0.05 * sig + 1e-4 * np.abs(g) + 1e-9)


N_GRAD_CONFIGS = 4


def _gradient_configs(seed=17, n=N_GRAD_CONFIGS):
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for k in range(n):
        lx, ly, lz = (float(v) for v in np.exp(rng.uniform(np.log(2.0), np.log(50.0), 3)))
        gx, gy, gz = (2 * int(v) for v in rng.integers(2, 13, 3))          # even sides: 2 x 2 x 2 blocks
        bx, by, bz = (int(rng.integers(1, v + 1)) for v in (gx, gy, gz))
        tau = float(np.exp(rng.uniform(np.log(0.3), np.log(8.0))))
        phase = "hg" if k % 2 else "mie"
        g = float(rng.uniform(-0.5, 0.9))
        d = float(np.exp(rng.uniform(np.log(1.0), np.log(10.0))))
        albedo = float(rng.uniform(0.7, 1.0))
        mu_a = float(tau / lx * rng.uniform(0.0, 0.1)) if k % 2 == 0 else 0.0
        out.append(dict(lx=lx, ly=ly, lz=lz, shape=(gz, gy, gx), block=(bx, by, bz), tau=tau, phase=phase, g=g, d=d,
                        albedo=albedo, mu_a=mu_a, spread=float(rng.uniform(0.0, 0.8)), seed=200 + k))
    return out


@pytest.mark.parametrize("nulls", [None, 1.25])
@pytest.mark.parametrize("k", range(N_GRAD_CONFIGS))
def test_random_grid_density_gradient_matches_oracle(gpu, oracle_mod, k, nulls):
    """The density gradient (mc_grid_adjoint, and with null-collision scores
    mc_grid_adjoint_nulls) on seeded random grids against the oracle's on the
    same photons: projections on smooth fields and the sums over the grid's
    eight octant blocks. The value equals the engine's own forward functional
    on those photons to 1e-5, and the oracle's to 5e-3: at 5e4 photons one
    photon whose path took another turn at a near-tie can move a camera term
    worth ~1e-3 of the image (the terms are heavy-tailed), as the homogeneous
    walk shows on the same table."""
    import torch
    from paper_2507_23189_gb300 import workloads as W
    c = _gradient_configs()[k]
    n = 50_000
    k_ext = 4e-5
    rough = W.rough_grid(c["shape"], c["seed"], mean=1.0, spread=c["spread"])
    dens = (rough * (c["tau"] / (k_ext * c["lx"] * float(rough.mean())))).astype(np.float32)
    geo = gpu.Geometry(c["lx"], c["ly"], c["lz"])
    grid = gpu.Grid(torch.from_numpy(dens).cuda(), k_ext, k_ext * c["albedo"], c["mu_a"], c["block"]).prepare(geo)
    nx = nz = 24
    adj = np.random.default_rng(300 + k).uniform(0, 1, (nz, nx)).astype(np.float32)
    r_max = 0.5 * math.hypot(c["ly"], c["lz"])
    if c["phase"] == "mie":
        med = gpu.Medium(1.0, 0.0, "table", 0.0, gpu.PhaseTable(diameter_um=c["d"]))
        x = oracle_mod.size_parameter(c["d"], 1.33, 532.0)
        om = dict(phase="mie", table=oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x))
    else:
        med = gpu.Medium(1.0, 0.0, "hg", c["g"])
        om = dict(phase="hg", hg_g=c["g"])
    e = gpu.Engine(gpu.Camera(nx, nz, 64, r_max), geo)
    val, grad = e.grid_adjoint(grid, med, torch.from_numpy(adj), n, seed=9, rr_threshold=1e-2, nulls=nulls)
    e.check()
    forward = None
    if not nulls:        # the null-score gradient walks against raised majorants: other paths
        e.run_grid(grid, med, n, seed=9, rr_threshold=1e-2)
        e.check()
        forward = float(np.sum(adj.astype(np.float64) * e.result()["image"]))
    gspec = dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_ext * c["albedo"], block=c["block"])
    if nulls:
        gspec["majorant_scale"] = nulls
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), nulls=bool(nulls), mu_s=0.0, mu_a=c["mu_a"], lx=c["lx"],
                                ly=c["ly"], lz=c["lz"], nx=nx, nz=nz, n_radial=64, r_max=r_max, n_photons=n, seed=9,
                                rr_threshold=1e-2, grid=gspec, **om)
    gg_ = grad.cpu().numpy().astype(np.float64)
    gz, gy, gx = c["shape"]
    z, y, xx = np.meshgrid(np.arange(gz) / gz, np.arange(gy) / gy, np.arange(gx) / gx, indexing="ij")
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(6):
        a = rng.uniform(0, 2, 3)
        f = np.cos(2 * np.pi * (a[0] * xx + a[1] * y + a[2] * z) + rng.uniform(0, 6.3))
        pg, po = float(np.sum(f * gg_)), float(np.sum(f * o["grad"]))
        worst = max(worst, abs(pg - po) / max(float(np.sum(np.abs(f * o["grad"]))), 1e-300))
    bg = gg_.reshape(2, gz // 2, 2, gy // 2, 2, gx // 2).sum(axis=(1, 3, 5))
    bo = o["grad"].reshape(2, gz // 2, 2, gy // 2, 2, gx // 2).sum(axis=(1, 3, 5))
    blk = float(np.max(np.abs(bg - bo)) / max(float(np.max(np.abs(bo))), 1e-300))
    print("gradient config %d nulls %s %s: value %.6g vs %.6g, projections %.2e, octants %.2e" %
          (k, nulls, {q: (round(v, 3) if isinstance(v, float) else v) for q, v in c.items()}, val.item(),
           o["value"], worst, blk))
    if forward is not None:
        assert val.item() == pytest.approx(forward, rel=1e-5)
    assert val.item() == pytest.approx(o["value"], rel=5e-3)
    assert worst <= 3e-3 and blk <= 1e-2
