"""Delta tracking through a voxel density grid on the GPU (mc_grid_prepare,
mc_run_grid) against the oracle's delta-tracking walk on the same seeds:
the prepared per-voxel data against numpy, traces of real events, tallies,
Beer-Lambert transmission, and the polydisperse plume with the mixture
table."""
import math

import numpy as np
import pytest

from parity import compare_traces, gpu_batches, oracle_var, tally_agreement, report_unmatched

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _grid(gpu, dens, k_ext, k_sca, mu_a=0.0, block=(8, 4, 4)):
    import torch
    g = gpu.Grid(torch.from_numpy(np.ascontiguousarray(dens, dtype=np.float32)).cuda(), k_ext, k_sca, mu_a,
                 block)
    return g.prepare(gpu.Geometry(LX, LY, LZ))


def _rough(shape, seed=4, mean=2000.0):
    from paper_2507_23189_gb300 import workloads as W
    return W.rough_grid(shape, seed, mean=mean)


def test_prepared_grid_matches_numpy(gpu):
    import torch
    dens = _rough((24, 20, 50))
    k_ext, mu_a, block = 4e-5, 0.003, (8, 4, 4)
    g = _grid(gpu, dens, k_ext, 3e-5, mu_a, block)
    torch.cuda.synchronize()
    n = dens.size
    raw = g.work.cpu().numpy()
    cells = raw[:8 * n].view(np.float32).reshape(24, 20, 50, 2)
    mu = k_ext * dens.astype(np.float64) + mu_a
    np.testing.assert_allclose(cells[..., 0], mu, rtol=2e-7)
    vy = LY / 20
    above = np.cumsum(mu[:, ::-1, :], axis=1)[:, ::-1, :] * vy - mu * vy    # voxels strictly above
    np.testing.assert_allclose(cells[..., 1], above, rtol=1e-6, atol=1e-7)
    mx, my, mz = 7, 5, 6
    maj = raw[8 * n:8 * n + 4 * mx * my * mz].view(np.float32).reshape(mz, my, mx)
    for cz in range(mz):
        for cy in range(my):
            for cx in range(mx):
                blk = cells[cz * 4:(cz + 1) * 4, cy * 4:(cy + 1) * 4, cx * 8:(cx + 1) * 8, 0]
                assert maj[cz, cy, cx] == blk.max()


CASES = [("hg", (8, 4, 4), 0.0, {}), ("table", (4, 4, 4), 0.002, dict(rr_threshold=0.02)),
         ("table", (64, 16, 16), 0.0, {})]


@pytest.mark.parametrize("phase,block,mu_a,kw", CASES)
def test_trace_parity_grid(gpu, oracle_mod, ps_table, ps_oracle_table, phase, block, mu_a, kw):
    dens = _rough((16, 16, 64))
    k_ext, k_sca = 4e-5, 3.6e-5
    g = _grid(gpu, dens, k_ext, k_sca, mu_a, block)
    n = 4096
    gg = ps_table.info["g"]
    med = gpu.Medium(1.0, 0.0, "table" if phase == "table" else "hg", gg, ps_table)
    e = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    tr = gpu.decode_trace(e.run_grid(g, med, n, seed=13, n_trace=n, n_events=32, **kw))
    e.check()
    om = dict(phase="mie", table=ps_oracle_table) if phase == "table" else dict(phase="hg", hg_g=gg)
    o = oracle_mod.walk(mu_s=0.0, mu_a=mu_a, n_photons=n, nx=64, nz=64, seed=13, n_trace=n, n_trace_events=32,
                        grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca, block=block),
                        **om, **kw)
    mu_max = k_ext * float(dens.max())
    cmp = compare_traces(tr, o["trace"], mu_ext=mu_max)
    print(phase, block, cmp["matched"], "/", n, "flips", cmp["flips"], "worst", cmp["worst"], "events",
          cmp["events"])
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp["bad"]
    assert cmp["events"] > 2 * n


@pytest.mark.parametrize("seed_or", [1, 2])
def test_tally_parity_grid(gpu, oracle_mod, ps_table, ps_oracle_table, seed_or):
    dens = _rough((16, 16, 64), seed=6)
    k_ext, k_sca = 4e-5, 3.8e-5
    g = _grid(gpu, dens, k_ext, k_sca, 0.0, (8, 4, 4))
    n = 1_000_000
    med = gpu.Medium(1.0, 0.0, "table", 0.0, ps_table)
    cam, geo = gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ)
    imgs = []
    raw_tot = None
    for b in range(32):
        e = gpu.Engine(cam, geo)
        e.run_grid(g, med, n // 32, seed=1, photon_offset=b * (n // 32))
        e.check()
        r = e.result()
        imgs.append(r["image"])
        raw_tot = r["raw_totals"] if raw_tot is None else raw_tot + r["raw_totals"]
    imgs = np.stack(imgs)
    img, var_g = imgs.sum(axis=0), 32 * imgs.var(axis=0, ddof=1)
    o = oracle_mod.walk(mu_s=0.0, phase="mie", table=ps_oracle_table, n_photons=n, nx=64, nz=64, seed=seed_or,
                        grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca, block=(8, 4, 4)))
    zmax, chi2, dof, p, z = tally_agreement(img, o["image"], oracle_var(o) + var_g, o["image_hits"])
    frac3 = float(np.mean(np.abs(z[(oracle_var(o) + var_g).ravel() > 0]) > 3))
    print("seed", seed_or, "zmax %.2f chi2/dof %.1f/%d p %.3g >3sigma %.4f" % (zmax, chi2, dof, p, frac3))
    assert p > 0.01 and dof > 500
    if seed_or == 1:
        assert zmax < 3.0
    else:
        assert frac3 < 0.01
    assert int(raw_tot[0]) + int(raw_tot[1]) + int(raw_tot[2]) + int(raw_tot[3]) + int(raw_tot[4]) == \
        pytest.approx(n * 2 ** 32, rel=1e-6)


def test_ballistic_transmission(gpu, ps_table):
    dens = _rough((16, 16, 64), seed=8)
    k = 4e-5
    g = _grid(gpu, dens, k, k, 0.0, (16, 8, 8))
    n = 10_000_000
    e = gpu.Engine(gpu.Camera(16, 16, 16, R_MAX), gpu.Geometry(LX, LY, LZ))
    e.run_grid(g, gpu.Medium(1.0, 0.0, "hg", 0.5, None), n, seed=5, max_scatter=1)
    e.check()
    tau = float(np.sum(k * dens[8, 8, :].astype(np.float64))) * LX / 64
    p = math.exp(-tau)
    got = e.result()["totals"][6] / n
    assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_plume_with_mixture_table(gpu, oracle_mod):
    """The polydisperse plume (Gaussian, 16 log-normal size bins) on a 64^3
    grid: GPU vs oracle on the same photons, mixture tables built by each
    side's own code."""
    from paper_2507_23189_gb300 import workloads as W
    d, f = W.size_bins(5.0, 0.3, 16)
    t = gpu.MixtureTable(d, f)
    k_ext, k_sca = t.info["sigma_ext_mm2"], t.info["sigma_sca_mm2"]
    shape = W.plume_shape((64, 64, 64))
    rho0 = 12.0 / (k_ext * float(np.sum(shape[32, 32, :].astype(np.float64))) * LX / 64)
    dens = (rho0 * shape).astype(np.float32)
    g = _grid(gpu, dens, k_ext, k_sca, 0.0, (8, 16, 16))
    m = complex(1.59 / 1.33, 0.0)
    comps, w = [], []
    for di, fi in zip(d, f):
        x = oracle_mod.size_parameter(di, 1.33, 532.0)
        qe, qs, _ = oracle_mod.mie_efficiencies(m, x)
        comps.append(("mie", m, x))
        w.append(fi * qs * np.pi * (di * 1e-3) ** 2 / 4)
    ot = oracle_mod.phase_table_mixture(comps, w)
    n = 1_000_000
    res = []
    e = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    for b in range(16):
        e.run_grid(g, gpu.Medium(1.0, 0.0, "table", 0.0, t), n // 16, seed=3, photon_offset=b * (n // 16))
        e.check()
        res.append(e.result()["image"])
    res = np.stack(res)
    img, var_g = res.sum(axis=0), 16 * res.var(axis=0, ddof=1)
    o = oracle_mod.walk(mu_s=0.0, phase="mie", table=ot, n_photons=n, nx=64, nz=64, seed=3,
                        grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca, block=(8, 16, 16)))
    zmax, chi2, dof, p, z = tally_agreement(img, o["image"], oracle_var(o) + var_g, o["image_hits"])
    print("plume zmax %.2f chi2/dof %.1f/%d p %.3g" % (zmax, chi2, dof, p))
    assert zmax < 3.0 and p > 0.01 and dof > 500
