"""Parity at the sizes the benchmark runs, in its launch configurations.

Batched media: all 64 media of the batched workload (d log-uniform in
1-10 um, tau uniform in 0.5-20, budgets log-uniform in 1e6-1e8, 128x128
images) in one mc_run_batch, as the benchmark launches it. Eight of them --
the smallest and largest particles, the thinnest and thickest media, the
largest and smallest budgets -- are run on the oracle with the oracle's own
table for that diameter, on all of the same photons: every image bin within
3 sigma, pooled chi-square p > 0.01, exact escape bookkeeping, radial
profile and step count; plus first-32-event traces for the smallest and
largest particle.

Heterogeneous plume: the 256^3 Gaussian plume with the 16-bin log-normal
mixture, the production majorant cells (32 x 256 x 256 voxels) and the
512x512 image, 1e6 photons in one mc_run_grid against the oracle's delta
tracking on the same photons; then mc_grid_adjoint at 256^3 against the
oracle's density gradient (value, smooth projections, block sums).
"""
import math

import numpy as np
import pytest

from parity import compare_traces, oracle_var, tally_agreement, report_unmatched

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


# ------------------------------------------------------------ batched media


def _pick(cases):
    """Indices: smallest and largest diameter, thinnest and thickest medium,
    largest and smallest budget, and two more from the middle of the list."""
    d = np.array([c.diameter_um for c in cases])
    t = np.array([c.tau for c in cases])
    n = np.array([c.n_photons for c in cases])
    idx = [int(np.argmin(d)), int(np.argmax(d)), int(np.argmin(t)), int(np.argmax(t)), int(np.argmax(n)),
           int(np.argmin(n)), 12, 33]
    out = []
    for i in idx:
        if i not in out:
            out.append(i)
    return out


@pytest.fixture(scope="module")
def batched_run(gpu):
    from concurrent.futures import ThreadPoolExecutor
    from paper_2507_23189_gb300 import workloads as W
    cases = W.batched()
    with ThreadPoolExecutor(8) as ex:
        tables = list(ex.map(lambda c: gpu.PhaseTable(diameter_um=c.diameter_um), cases))
    media = [gpu.Medium.from_optical_depth(t, c.tau, LX) for t, c in zip(tables, cases)]
    cam, geo = gpu.Camera(128, 128, 128, R_MAX), gpu.Geometry(LX, LY, LZ)
    b = gpu.Batch(len(media), cam, geo)
    b.run(media, [c.n_photons for c in cases], 1, 0)
    b.check()
    return cases, tables, media, b


def test_batched_media_against_oracle(gpu, oracle_mod, batched_run):
    cases, tables, media, b = batched_run
    pick = _pick(cases)
    d = [cases[i].diameter_um for i in pick]
    t = [cases[i].tau for i in pick]
    assert min(d) < 1.05 and max(d) > 9.0 and min(t) < 1.0 and max(t) > 19.5
    scale = 2.0 ** -b.image_frac_bits
    m = complex(1.59 / 1.33, 0.0)
    for i in pick:
        c = cases[i]
        x = oracle_mod.size_parameter(c.diameter_um, 1.33, 532.0)
        ot = oracle_mod.phase_table(oracle_mod.PHASE_MIE, m, x)
        o = oracle_mod.walk(mu_s=c.tau / LX, table=ot, n_photons=c.n_photons, nx=128, nz=128, n_radial=128,
                            r_max=R_MAX, seed=1)
        img = b.image[i].cpu().numpy().astype(np.float64) * scale
        raw_tot = b.totals[i].cpu().numpy()
        # the engine's per-photon spread is the oracle's (one estimator, same
        # photons): both sides' variances are the oracle's
        var = 2.0 * oracle_var(o)
        zmax, chi2, dof, p, z = tally_agreement(img, o["image"], var, o["image_hits"])
        print("medium %d d=%.3f um tau=%.2f N=%d: zmax %.2f chi2/dof %.1f/%d p %.3g steps %d vs %d" %
              (i, c.diameter_um, c.tau, c.n_photons, zmax, chi2, dof, p, raw_tot[7], o["steps"]))
        assert zmax < 3.0 and p > 0.01 and dof > 200, i
        # non-absorbing: every photon leaves with weight 1, exactly
        assert int(raw_tot[0]) + int(raw_tot[1]) + int(raw_tot[2]) == c.n_photons << 32, i
        w = raw_tot[:3].astype(np.float64) * 2.0 ** -32
        for k in range(3):
            sig = math.sqrt(max(o["totals_sq"][k] - o["totals"][k] ** 2 / c.n_photons, 0.0))
            assert abs(w[k] - o["totals"][k]) <= 3 * math.sqrt(2) * sig + 1e-9, (i, k)
        assert abs(int(raw_tot[7]) - o["steps"]) <= 1e-4 * o["steps"], i
        rad = b.radial[i].cpu().numpy().astype(np.float64) * 2.0 ** -32
        rsig = np.sqrt(np.maximum(o["radial_sq"] - o["radial"] ** 2 / c.n_photons, 0))
        assert np.all(np.abs(rad - o["radial"]) <= 3 * np.sqrt(2) * rsig + 1e-6), i


def test_batched_smallest_and_largest_particle_traces(gpu, oracle_mod, batched_run):
    cases, tables, media, _ = batched_run
    d = np.array([c.diameter_um for c in cases])
    m = complex(1.59 / 1.33, 0.0)
    n = 4096
    for i in (int(np.argmin(d)), int(np.argmax(d))):
        c = cases[i]
        e = gpu.Engine(gpu.Camera(128, 128, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
        tr = gpu.decode_trace(e.trace(media[i], n, n, 32, seed=1))
        e.check()
        x = oracle_mod.size_parameter(c.diameter_um, 1.33, 532.0)
        ot = oracle_mod.phase_table(oracle_mod.PHASE_MIE, m, x)
        o = oracle_mod.walk(mu_s=c.tau / LX, table=ot, n_photons=n, nx=128, nz=128, seed=1, n_trace=n,
                            n_trace_events=32)
        cmp = compare_traces(tr, o["trace"], mu_ext=c.tau / LX)
        print("medium %d d=%.3f um tau=%.2f: %d/%d matched, flips %d, worst %s, events %d" %
              (i, c.diameter_um, c.tau, cmp["matched"], n, cmp["flips"], cmp["worst"], cmp["events"]))
        report_unmatched(cmp)
        assert cmp["matched"] >= 0.999 * n, cmp["bad"]
        assert cmp["events"] > 1.2 * n


# ---------------------------------------------------------- the full plume


@pytest.fixture(scope="module")
def plume(gpu, oracle_mod):
    import torch
    from paper_2507_23189_gb300 import workloads as W
    P = W.plume()
    d, f = W.size_bins(P.median_um, P.sigma_ln, P.n_size_bins)
    tab = gpu.MixtureTable(d, f)
    k_ext, k_sca = tab.info["sigma_ext_mm2"], tab.info["sigma_sca_mm2"]
    shape = W.plume_shape(P.shape, (LX, LY, LZ), P.sigma_mm, P.center_x_mm)
    gz, gy, gx = P.shape
    rho0 = P.tau_peak / (k_ext * float(np.sum(shape[gz // 2, gy // 2, :].astype(np.float64))) * LX / gx)
    dens32 = (shape * np.float32(rho0)).astype(np.float32)
    geo = gpu.Geometry(LX, LY, LZ, 0.0)
    grid = gpu.Grid(torch.from_numpy(dens32).cuda(), k_ext, k_sca, 0.0, P.block).prepare(geo)
    m = complex(1.59 / 1.33, 0.0)
    comps, w = [], []
    for di, fi in zip(d, f):
        x = oracle_mod.size_parameter(di, 1.33, 532.0)
        qe, qs, _ = oracle_mod.mie_efficiencies(m, x)
        comps.append(("mie", m, x))
        w.append(fi * qs * np.pi * (di * 1e-3) ** 2 / 4)
    ot = oracle_mod.phase_table_mixture(comps, w)
    ogrid = dict(density=dens32.astype(np.float64), k_ext=k_ext, k_sca=k_sca, block=P.block)
    return P, tab, grid, geo, ot, ogrid


def test_plume_full_size_against_oracle(gpu, oracle_mod, plume):
    P, tab, grid, geo, ot, ogrid = plume
    assert P.shape == (256, 256, 256) and P.block == (32, 256, 256) and (P.nx, P.nz) == (512, 512)
    n = 1_000_000
    cam = gpu.Camera(P.nx, P.nz, 128, R_MAX)
    med = gpu.Medium(1.0, 0.0, "table", 0.0, tab)
    e = gpu.Engine(cam, geo)
    e.run_grid(grid, med, n, seed=1)           # one launch, as the benchmark runs it
    e.check()
    full = e.result()
    # the same photons in 16 launches: bit-identical sums and a batch variance
    f = e.image_frac_bits
    parts, raw_img = [], None
    for k in range(16):
        ek = gpu.Engine(cam, geo)
        ek.run_grid(grid, med, n // 16, seed=1, photon_offset=k * (n // 16), image_frac_bits=f)
        ek.check()
        r = ek.result()
        parts.append(r["image"])
        raw_img = r["raw_image"] if raw_img is None else raw_img + r["raw_image"]
    np.testing.assert_array_equal(raw_img, full["raw_image"])
    parts = np.stack(parts)
    o = oracle_mod.walk(mu_s=0.0, phase="mie", table=ot, n_photons=n, nx=P.nx, nz=P.nz, n_radial=128,
                        r_max=R_MAX, seed=1, grid=ogrid)
    var = oracle_var(o) + 16 * parts.var(axis=0, ddof=1)
    zmax, chi2, dof, p, z = tally_agreement(full["image"], o["image"], var, o["image_hits"])
    t = full["raw_totals"]
    print("plume 256^3, 512^2, 1e6 photons: zmax %.2f chi2/dof %.1f/%d p %.3g; tentative steps %d vs %d; "
          "ballistic %g vs %g" % (zmax, chi2, dof, p, t[7], o["steps"], full["totals"][6], o["totals"][6]))
    assert zmax < 3.0 and p > 0.01 and dof > 2000
    # weight bookkeeping: non-absorbing, every photon leaves with weight 1
    assert int(t[0]) + int(t[1]) + int(t[2]) == n << 32
    # peak optical depth 30 on the beam: no photon crosses unscattered (exp(-30) n ~ 1e-7) on either side
    assert full["totals"][6] == o["totals"][6] == 0.0
    assert abs(int(t[7]) - o["steps"]) <= 2e-4 * o["steps"]
    for k in range(3):
        sig = math.sqrt(max(o["totals_sq"][k] - o["totals"][k] ** 2 / n, 0.0))
        assert abs(full["totals"][k] - o["totals"][k]) <= 3 * math.sqrt(2) * sig + 1e-9, k


def test_plume_full_size_density_gradient_against_oracle(gpu, oracle_mod, plume):
    import torch
    P, tab, grid, geo, ot, ogrid = plume
    n = 200_000
    cam = gpu.Camera(P.nx, P.nz, 128, R_MAX)
    adj = np.random.default_rng(8).uniform(0.0, 1.0, (P.nz, P.nx)).astype(np.float32)
    e = gpu.Engine(cam, geo)
    cap = dict(max_scatter=1500)        # both sides stop a photon at its 1500th collision
    val, grad = e.grid_adjoint(grid, gpu.Medium(1.0, 0.0, "table", 0.0, tab), torch.from_numpy(adj), n, seed=5,
                               **cap)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), max_events=2048, phase="mie", table=ot, mu_s=0.0,
                                n_photons=n, nx=P.nx, nz=P.nz, seed=5, grid=ogrid, **cap)
    gg = grad.cpu().numpy().astype(np.float64)
    go = o["grad"]
    print("plume gradient: value %.8g vs %.8g; sum %.6g vs %.6g" % (val.item(), o["value"], gg.sum(), go.sum()))
    assert val.item() == pytest.approx(o["value"], rel=2e-4)
    # smooth projections (a photon whose single-precision path took another
    # discrete turn moves single voxels, not these)
    gz, gy, gx = P.shape
    z, y, x = np.meshgrid(np.arange(gz) / gz, np.arange(gy) / gy, np.arange(gx) / gx, indexing="ij")
    rng = np.random.default_rng(2)
    for _ in range(4):
        a = rng.uniform(0, 3, 3)
        f = np.cos(2 * np.pi * (a[0] * x + a[1] * y + a[2] * z) + rng.uniform(0, 6.3))
        pg, po = float(np.sum(f * gg)), float(np.sum(f * go))
        assert abs(pg - po) <= 3e-3 * float(np.sum(np.abs(f * go))), (pg, po)
    blk = lambda t: t.reshape(8, 32, 8, 32, 8, 32).sum(axis=(1, 3, 5))
    bg, bo = blk(gg), blk(go)
    worst = np.max(np.abs(bg - bo)) / np.max(np.abs(bo))
    print("plume gradient: worst 32^3 block %.2e of the largest" % worst)
    assert worst <= 1e-2
