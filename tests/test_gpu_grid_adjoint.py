"""Gradient with respect to the voxel densities on the GPU (mc_grid_adjoint):
the scaling identity against the GPU's own homogeneous adjoint, the oracle's
gradient on the same photons (single scattering voxel by voxel, multiple
scattering through projections and block sums), and an Adam fit of the
density scale of a plume from a target image."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _grid(gpu, dens, k_ext, k_sca, mu_a=0.0, block=(8, 4, 4)):
    import torch
    g = gpu.Grid(torch.from_numpy(np.ascontiguousarray(dens, dtype=np.float32)).cuda(), k_ext, k_sca, mu_a,
                 block)
    return g.prepare(gpu.Geometry(LX, LY, LZ))


def _rough(shape, seed, mean):
    from paper_2507_23189_gb300 import workloads as W
    return W.rough_grid(shape, seed, mean=mean)


@pytest.mark.parametrize("absorb", [False, True])
def test_scaling_identity_against_homogeneous_adjoint(gpu, ps_table, absorb):
    import torch
    k_ext = 2e-5
    k_sca = 0.85 * k_ext if absorb else k_ext
    rho = 4.0 / LX / k_ext
    dens = np.full((8, 16, 32), rho, dtype=np.float32)
    g = _grid(gpu, dens, k_ext, k_sca, 0.0, (4, 4, 4))
    n = 1_000_000
    adj = torch.rand((64, 64), generator=torch.Generator().manual_seed(3))
    e = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    med = gpu.Medium(1.0, 0.0, "table", 0.0, ps_table)
    val, grad = e.grid_adjoint(g, med, adj, n, seed=7, rr_threshold=1e-2)
    e.check()
    mu_s, mu_ap = k_sca * float(np.float32(rho)), (k_ext - k_sca) * float(np.float32(rho))
    h = e.adjoint(gpu.Medium(mu_s, mu_ap, "table", 0.0, ps_table), adj, n, n_w=0, seed=7,
                  rr_threshold=1e-2).cpu().numpy()
    e.check()
    lhs = float(np.float32(rho)) * float(grad.double().sum())
    rhs = mu_s * h[1] + mu_ap * h[2]
    print("value %.6g vs %.6g; sum rho grad %.6g vs %.6g" % (val.item(), h[0], lhs, rhs))
    assert val.item() == pytest.approx(h[0], rel=2e-4)
    assert lhs == pytest.approx(rhs, rel=2e-3)


def test_single_scatter_matches_oracle_voxel_by_voxel(gpu, oracle_mod):
    import torch
    dens = _rough((16, 16, 32), 11, 2000.0)
    k_ext, k_sca, gg = 4e-5, 3e-5, 0.6
    nx, nz = 32, 16
    rng = np.random.default_rng(5)
    adj = np.zeros((nz, nx), dtype=np.float32)
    adj[nz // 2] = rng.uniform(0.2, 1.0, nx)
    g = _grid(gpu, dens, k_ext, k_sca, 0.0, (8, 4, 4))
    n = 200_000
    e = gpu.Engine(gpu.Camera(nx, nz, 64, R_MAX), gpu.Geometry(LX, LY, LZ))
    val, grad = e.grid_adjoint(g, gpu.Medium(1.0, 0.0, "hg", gg, None), torch.from_numpy(adj), n, seed=3,
                               max_scatter=1)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), phase="hg", hg_g=gg, mu_s=0.0, n_photons=n, nx=nx,
                                nz=nz, max_scatter=1, seed=3,
                                grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca,
                                          block=(8, 4, 4)))
    gg_ = grad.cpu().numpy().astype(np.float64)
    mask = np.zeros(dens.shape, bool)
    mask[8, 8:, :] = True
    assert np.all(gg_[~mask] == 0.0)
    assert val.item() == pytest.approx(o["value"], rel=1e-5)
    scale = np.max(np.abs(o["grad"]))
    ok = np.abs(gg_ - o["grad"]) <= 1e-4 * np.abs(o["grad"]) + 1e-5 * scale
    print("voxels within tolerance: %d / %d" % (ok[mask].sum(), mask.sum()))
    assert ok[mask].mean() >= 0.995


def test_multiple_scattering_matches_oracle(gpu, oracle_mod, ps_table, ps_oracle_table):
    import torch
    dens = _rough((16, 16, 64), 12, 1500.0)
    k_ext, k_sca, mu_a = 4e-5, 3.6e-5, 0.002
    nx = nz = 32
    adj = np.random.default_rng(4).uniform(0, 1, (nz, nx)).astype(np.float32)
    g = _grid(gpu, dens, k_ext, k_sca, mu_a, (8, 4, 4))
    n = 200_000
    e = gpu.Engine(gpu.Camera(nx, nz, 64, R_MAX), gpu.Geometry(LX, LY, LZ))
    val, grad = e.grid_adjoint(g, gpu.Medium(1.0, 0.0, "table", 0.0, ps_table), torch.from_numpy(adj), n,
                               seed=9, rr_threshold=1e-2)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), phase="mie", table=ps_oracle_table, mu_s=0.0, mu_a=mu_a,
                                n_photons=n, nx=nx, nz=nz, seed=9, rr_threshold=1e-2,
                                grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca,
                                          block=(8, 4, 4)))
    gg_ = grad.cpu().numpy().astype(np.float64)
    assert val.item() == pytest.approx(o["value"], rel=2e-4)
    # projections on smooth fields: a few photons whose single-precision path
    # took another discrete turn move single voxels, not these
    z, y, x = np.meshgrid(np.arange(16) / 16, np.arange(16) / 16, np.arange(64) / 64, indexing="ij")
    rng = np.random.default_rng(1)
    for _ in range(6):
        a = rng.uniform(0, 3, 3)
        f = np.cos(2 * np.pi * (a[0] * x + a[1] * y + a[2] * z) + rng.uniform(0, 6.3))
        pg, po = float(np.sum(f * gg_)), float(np.sum(f * o["grad"]))
        assert abs(pg - po) <= 3e-3 * float(np.sum(np.abs(f * o["grad"]))), (pg, po)
    blk = lambda t: t.reshape(4, 4, 4, 4, 8, 8).sum(axis=(1, 3, 5))
    bg, bo = blk(gg_), blk(o["grad"])
    assert np.max(np.abs(bg - bo)) <= 1e-2 * np.max(np.abs(bo))


def test_fit_plume_scale_with_adam(gpu):
    """Target image at 0.8 x the plume density; 25 Adam steps on log(scale)
    from 1.3 with gradients from mc_grid_adjoint (independent photons for the
    gradient, the loss being quadratic in the image)."""
    import torch
    from paper_2507_23189_gb300 import workloads as W
    shape = W.plume_shape((32, 32, 64))
    k_ext = 5e-5
    rho0 = 10.0 / (k_ext * float(np.sum(shape[16, 16, :].astype(np.float64))) * LX / 64)
    base = torch.from_numpy(shape).cuda() * rho0
    cam, geo = gpu.Camera(64, 64, 64, R_MAX), gpu.Geometry(LX, LY, LZ)
    tab = gpu.PhaseTable()
    med = gpu.Medium(1.0, 0.0, "table", 0.0, tab)
    e = gpu.Engine(cam, geo)
    g = gpu.Grid(base * 0.8, k_ext, k_ext, 0.0, (8, 8, 8)).prepare(geo)
    nt = 50_000_000
    e.run_grid(g, med, nt, seed=100)
    e.check()
    target = torch.tensor(e.result()["image"] / nt, device="cuda")
    log_s = torch.tensor(math.log(1.3), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([log_s], lr=0.08)
    n = 4_000_000
    scale = 1.0 / float((target ** 2).sum())
    for it in range(25):
        s = math.exp(log_s.item())
        g = gpu.Grid(base * s, k_ext, k_ext, 0.0, (8, 8, 8)).prepare(geo)
        e.run_grid(g, med, n, seed=1 + 2 * it)
        e.check()
        img = torch.tensor(e.result()["image"] / n, device="cuda")
        resid = img - target
        adj = (2.0 * scale / n) * resid                  # d loss / d (image sum)
        _, grad = e.grid_adjoint(g, med, adj, n, seed=2 + 2 * it)
        e.check()
        dl_ds = float((grad.double() * base.double()).sum())   # chain rule through n = s * base
        opt.zero_grad()
        log_s.grad = torch.tensor(dl_ds * s, dtype=torch.float64)
        opt.step()
    s = math.exp(log_s.item())
    print("recovered scale %.4f (true 0.8)" % s)
    assert abs(s / 0.8 - 1) < 0.03


def test_disc_beam_gradient_matches_oracle(gpu, oracle_mod, ps_table, ps_oracle_table):
    """A 2.5 mm disc beam: first flights start in many voxel rows (each one
    entry of the row-suffix sums), single and multiple scattering against the
    oracle on the same photons."""
    import torch
    dens = _rough((16, 16, 32), 13, 2000.0)
    k_ext, k_sca = 4e-5, 3.2e-5
    nx = nz = 32
    adj = np.random.default_rng(6).uniform(0.2, 1.0, (nz, nx)).astype(np.float32)
    geo = gpu.Geometry(LX, LY, LZ, beam_radius=1.25)
    g = gpu.Grid(torch.from_numpy(np.ascontiguousarray(dens, dtype=np.float32)).cuda(), k_ext, k_sca, 0.0,
                 (8, 4, 4)).prepare(geo)
    e = gpu.Engine(gpu.Camera(nx, nz, 64, R_MAX), geo)
    n = 200_000
    grid = dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca, block=(8, 4, 4))
    val, grad = e.grid_adjoint(g, gpu.Medium(1.0, 0.0, "hg", 0.7, None), torch.from_numpy(adj), n, seed=8,
                               max_scatter=1)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), phase="hg", hg_g=0.7, mu_s=0.0, n_photons=n, nx=nx, nz=nz,
                                max_scatter=1, seed=8, beam_radius=1.25, grid=grid)
    gg_ = grad.cpu().numpy().astype(np.float64)
    rows = np.any(o["grad"] != 0.0, axis=2)
    assert rows.sum() >= 12                       # first flights in many rows
    assert val.item() == pytest.approx(o["value"], rel=1e-5)
    scale = np.max(np.abs(o["grad"]))
    ok = np.abs(gg_ - o["grad"]) <= 1e-4 * np.abs(o["grad"]) + 1e-5 * scale
    print("disc beam, single scattering: voxels within tolerance %d / %d" % (ok.sum(), ok.size))
    assert ok.mean() >= 0.995
    val, grad = e.grid_adjoint(g, gpu.Medium(1.0, 0.0, "table", 0.0, ps_table), torch.from_numpy(adj), n, seed=9,
                               rr_threshold=1e-2)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), phase="mie", table=ps_oracle_table, mu_s=0.0, n_photons=n,
                                nx=nx, nz=nz, seed=9, rr_threshold=1e-2, beam_radius=1.25, grid=grid)
    gg_ = grad.cpu().numpy().astype(np.float64)
    assert val.item() == pytest.approx(o["value"], rel=2e-4)
    blk = lambda t: t.reshape(4, 4, 4, 4, 4, 8).sum(axis=(1, 3, 5))
    bg, bo = blk(gg_), blk(o["grad"])
    print("disc beam, multiple scattering: worst block %.2e of max" % (np.max(np.abs(bg - bo)) / np.max(np.abs(bo))))
    assert np.max(np.abs(bg - bo)) <= 1e-2 * np.max(np.abs(bo))


# ------------------------------------------- null-collision scores (nulls=)


def test_null_scores_match_oracle_single_scatter(gpu, oracle_mod):
    """Null-collision scores, single scattering: the GPU and the oracle on the
    same photons with majorants 1.5 times the cell maxima, voxel by voxel."""
    import torch
    dens = _rough((16, 16, 32), 11, 2000.0)
    k_ext, k_sca, gg = 4e-5, 3e-5, 0.6
    nx, nz = 32, 16
    rng = np.random.default_rng(5)
    adj = np.zeros((nz, nx), dtype=np.float32)
    adj[nz // 2] = rng.uniform(0.2, 1.0, nx)
    g = _grid(gpu, dens, k_ext, k_sca, 0.0, (8, 4, 4))
    n = 200_000
    e = gpu.Engine(gpu.Camera(nx, nz, 64, R_MAX), gpu.Geometry(LX, LY, LZ))
    val, grad = e.grid_adjoint(g, gpu.Medium(1.0, 0.0, "hg", gg, None), torch.from_numpy(adj), n, seed=3,
                               max_scatter=1, nulls=1.5)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), nulls=True, max_events=256, phase="hg", hg_g=gg, mu_s=0.0,
                                n_photons=n, nx=nx, nz=nz, max_scatter=1, seed=3,
                                grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca,
                                          block=(8, 4, 4), majorant_scale=1.5))
    gg_ = grad.cpu().numpy().astype(np.float64)
    mask = np.zeros(dens.shape, bool)
    mask[8, 8:, :] = True
    assert np.all(gg_[~mask] == 0.0)
    assert val.item() == pytest.approx(o["value"], rel=1e-5)
    scale = np.max(np.abs(o["grad"]))
    ok = np.abs(gg_ - o["grad"]) <= 1e-4 * np.abs(o["grad"]) + 1e-5 * scale
    print("nulls, single scattering: voxels within tolerance %d / %d" % (ok[mask].sum(), mask.sum()))
    # a null collision's voxel is a discrete decision: a few photons whose
    # single-precision null landed across a voxel face move single voxels
    assert ok[mask].mean() >= 0.98
    rows = lambda t: t[8, 8:, :].sum(axis=1)
    np.testing.assert_allclose(rows(gg_), rows(o["grad"]), rtol=1e-3, atol=1e-4 * np.abs(rows(o["grad"])).max())


def test_null_scores_match_oracle_multiple_scattering(gpu, oracle_mod, ps_table, ps_oracle_table):
    import torch
    dens = _rough((16, 16, 64), 12, 1500.0)
    k_ext, k_sca, mu_a = 4e-5, 3.6e-5, 0.002
    nx = nz = 32
    adj = np.random.default_rng(4).uniform(0, 1, (nz, nx)).astype(np.float32)
    g = _grid(gpu, dens, k_ext, k_sca, mu_a, (8, 4, 4))
    n = 200_000
    e = gpu.Engine(gpu.Camera(nx, nz, 64, R_MAX), gpu.Geometry(LX, LY, LZ))
    val, grad = e.grid_adjoint(g, gpu.Medium(1.0, 0.0, "table", 0.0, ps_table), torch.from_numpy(adj), n,
                               seed=9, rr_threshold=1e-2, nulls=1.25)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), nulls=True, max_events=4096, phase="mie",
                                table=ps_oracle_table, mu_s=0.0, mu_a=mu_a, n_photons=n, nx=nx, nz=nz, seed=9,
                                rr_threshold=1e-2,
                                grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca,
                                          block=(8, 4, 4), majorant_scale=1.25))
    gg_ = grad.cpu().numpy().astype(np.float64)
    assert val.item() == pytest.approx(o["value"], rel=2e-4)
    z, y, x = np.meshgrid(np.arange(16) / 16, np.arange(16) / 16, np.arange(64) / 64, indexing="ij")
    rng = np.random.default_rng(1)
    for _ in range(6):
        a = rng.uniform(0, 3, 3)
        f = np.cos(2 * np.pi * (a[0] * x + a[1] * y + a[2] * z) + rng.uniform(0, 6.3))
        pg, po = float(np.sum(f * gg_)), float(np.sum(f * o["grad"]))
        assert abs(pg - po) <= 3e-3 * float(np.sum(np.abs(f * o["grad"]))), (pg, po)
    blk = lambda t: t.reshape(4, 4, 4, 4, 8, 8).sum(axis=(1, 3, 5))
    bg, bo = blk(gg_), blk(o["grad"])
    assert np.max(np.abs(bg - bo)) <= 1e-2 * np.max(np.abs(bo))


def test_null_scores_match_oracle_with_a_partial_beam_box(gpu, oracle_mod, ps_table, ps_oracle_table):
    """A grid wider than the null-score kernel's box of copies around the beam
    axis (64 x 64 voxels across, the box the central 32 x 32): the voxels
    summed through the copies and those summed directly, against the oracle on
    the same photons, through block sums inside and outside the box."""
    import torch
    dens = _rough((64, 64, 32), 15, 1500.0)
    k_ext, k_sca = 4e-5, 3.8e-5
    nx = nz = 32
    adj = np.random.default_rng(8).uniform(0, 1, (nz, nx)).astype(np.float32)
    g = _grid(gpu, dens, k_ext, k_sca, 0.0, (8, 8, 8))
    n = 100_000
    e = gpu.Engine(gpu.Camera(nx, nz, 64, R_MAX), gpu.Geometry(LX, LY, LZ))
    val, grad = e.grid_adjoint(g, gpu.Medium(1.0, 0.0, "table", 0.0, ps_table), torch.from_numpy(adj), n,
                               seed=13, rr_threshold=1e-2, nulls=1.25)
    e.check()
    o = oracle_mod.grid_adjoint(adj.astype(np.float64), nulls=True, max_events=4096, phase="mie",
                                table=ps_oracle_table, mu_s=0.0, n_photons=n, nx=nx, nz=nz, seed=13,
                                rr_threshold=1e-2,
                                grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca,
                                          block=(8, 8, 8), majorant_scale=1.25))
    gg_ = grad.cpu().numpy().astype(np.float64)
    assert val.item() == pytest.approx(o["value"], rel=2e-4)
    # 8^3-voxel blocks; the box covers blocks 2..5 along y and z
    blk = lambda t: t.reshape(8, 8, 8, 8, 4, 8).sum(axis=(1, 3, 5))
    bg, bo = blk(gg_), blk(o["grad"])
    inside = np.zeros(bg.shape, bool)
    inside[2:6, 2:6, :] = True
    scale = np.max(np.abs(bo))
    print("partial box: worst block inside %.2e, outside %.2e of max" %
          (np.max(np.abs(bg - bo)[inside]) / scale, np.max(np.abs(bg - bo)[~inside]) / scale))
    assert np.max(np.abs(bo[inside])) > 0 and np.max(np.abs(bo[~inside])) > 0
    assert np.max(np.abs(bg - bo)) <= 1e-3 * scale


def test_null_scores_and_exact_lengths_agree_in_expectation(gpu, ps_table):
    """The two estimators on independent photons (their majorants differ):
    block sums agree within the combined batch errors."""
    import torch
    dens = _rough((16, 16, 64), 14, 1500.0)
    k_ext, k_sca = 4e-5, 3.8e-5
    nx = nz = 32
    adj = torch.from_numpy(np.random.default_rng(6).uniform(0, 1, (nz, nx)).astype(np.float32))
    g = _grid(gpu, dens, k_ext, k_sca, 0.0, (8, 4, 4))
    e = gpu.Engine(gpu.Camera(nx, nz, 64, R_MAX), gpu.Geometry(LX, LY, LZ))
    med = gpu.Medium(1.0, 0.0, "table", 0.0, ps_table)
    blk = lambda t: t.reshape(4, 4, 4, 4, 8, 8).sum(axis=(1, 3, 5))
    out = {}
    for name, nulls in (("exact", None), ("nulls", 1.25)):
        bs = []
        for b in range(12):
            _, grad = e.grid_adjoint(g, med, adj, 400_000, seed=31, photon_offset=b * 400_000, rr_threshold=1e-2,
                                     nulls=nulls)
            e.check()
            bs.append(blk(grad.cpu().numpy().astype(np.float64)))
        bs = np.stack(bs)
        out[name] = (bs.mean(axis=0), bs.std(axis=0, ddof=1) / np.sqrt(len(bs)))
    (m0, s0), (m1, s1) = out["exact"], out["nulls"]
    z = (m1 - m0) / np.sqrt(s0 ** 2 + s1 ** 2)
    print("block sums: max |z| %.2f chi2/dof %.1f/%d; null/exact error ratio median %.2f" %
          (np.max(np.abs(z)), np.sum(z ** 2), z.size, np.median(s1 / s0)))
    assert np.max(np.abs(z)) < 4.5
    assert np.sum(z ** 2) < z.size + 6 * np.sqrt(2 * z.size)
