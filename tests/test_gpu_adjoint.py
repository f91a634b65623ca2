"""Adjoint (mc_adjoint) on the GPU: against the oracle's gradient on the same
photons, against the single-scatter closed form, against central
differences with common random numbers, through torch.autograd, and in a
50-step Adam fit recovering mu_s and mu_a from a synthetic target image."""
import math

import numpy as np
import pytest

from parity import oracle_var

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _eng(gpu, nx=64, nz=64):
    return gpu.Engine(gpu.Camera(nx, nz, 128, R_MAX), gpu.Geometry(LX, LY, LZ))


@pytest.mark.parametrize("mu_a,kw", [(0.0, {}), (0.02, dict(rr_threshold=0.05))])
def test_adjoint_matches_oracle_gradient(gpu, oracle_mod, ps_table, ps_oracle_table, mu_a, kw):
    import torch
    n, nx, nz = 200_000, 64, 64
    mu_s = 5.0 / LX - mu_a
    adj = np.random.default_rng(8).uniform(0, 1, (nz, nx))
    e = _eng(gpu, nx, nz)
    med = gpu.Medium(mu_s, mu_a, "table", 0.0, ps_table)
    out = e.adjoint(med, torch.tensor(adj, dtype=torch.float32), n, n_w=64, seed=5, **kw)
    e.check()
    out = out.cpu().numpy()
    ores = oracle_mod.adjoint(adj.astype(np.float32).astype(np.float64), 64, mu_s=mu_s, mu_a=mu_a,
                              table=ps_oracle_table, n_photons=n, nx=nx, nz=nz, seed=5, **kw)
    g, g2 = ores["grad"], ores["grad_sq"]
    sig = np.sqrt(np.maximum(g2 - g ** 2 / n, 0))
    assert out[0] == pytest.approx(ores["value"], rel=1e-4)
    # same photons: differences come only from single-precision rounding and
    # the rare precision flip of a discrete decision
    d = np.abs(out[1:] - g)
    print("rel to sigma: max %.3g, median %.3g" % (np.max(d / sig), np.median(d / sig)))
    assert np.all(d <= 0.05 * sig + 1e-4 * np.abs(g) + 1e-9)


def test_adjoint_value_equals_forward_functional(gpu, ps_table):
    import torch
    n = 500_000
    adj = torch.rand((128, 128), generator=torch.Generator().manual_seed(3))
    e = _eng(gpu, 128, 128)
    med = gpu.Medium(5 / LX, 0.003, "table", 0.0, ps_table)
    e.run(med, n, seed=2)
    e.check()
    img = e.result()["image"]
    out = e.adjoint(med, adj, n, n_w=0, seed=2).cpu().numpy()
    assert out[0] == pytest.approx(float(np.sum(adj.numpy().astype(np.float64) * img)), rel=1e-5)


def test_adjoint_single_scatter_closed_form(gpu, ps_table):
    import torch
    nx, nz, n = 32, 16, 10_000_000
    mu_s, mu_a = 2.0 / LX, 0.01
    mu_ext = mu_s + mu_a
    rng = np.random.default_rng(5)
    adj = rng.uniform(-1, 1, (nz, nx)).astype(np.float32)
    e = _eng(gpu, nx, nz)
    med = gpu.Medium(mu_s, mu_a, "table", 0.0, ps_table)
    # batches for the spread
    outs = np.stack([e.adjoint(med, torch.tensor(adj), n // 10, n_w=64, seed=1, photon_offset=b * (n // 10),
                               max_scatter=1).cpu().numpy() for b in range(10)])
    g = outs.sum(axis=0)
    sig = outs.std(axis=0, ddof=1) * math.sqrt(10)
    icdf = ps_table.icdf64
    j0 = int(np.searchsorted(icdf, 0.0, side="right")) - 1
    psr0 = float(np.float32(ps_table.pdf64[j0])) / (2 * math.pi)
    row = adj[nz // 2].astype(np.float64)
    edges = np.arange(nx + 1) * LX / nx

    def f(ms, ma):
        me = ms + ma
        prob = np.exp(-me * edges[:-1]) - np.exp(-me * edges[1:])
        return n * float(np.sum(row * (ms / me) * psr0 * math.exp(-me * LY / 2) * prob))

    h = 1e-7
    assert abs(g[1] - (f(mu_s + h, mu_a) - f(mu_s - h, mu_a)) / (2 * h)) < 4 * sig[1]
    assert abs(g[2] - (f(mu_s, mu_a + h) - f(mu_s, mu_a - h)) / (2 * h)) < 4 * sig[2]
    # phase weights: d p_w(0)/dw_k = p(0) (phi_k(0) - Z_k); Z from the table
    nodes = -1 + 2 * np.arange(64) / 63
    omu = ps_table.omu64
    z = np.zeros(64)
    for k in range(64):
        c, hh = nodes[k], 2 / 63
        xs = np.linspace(max(c - hh, -1), min(c + hh, 1), 20001)
        idx = np.clip(np.searchsorted(1 - omu, xs, side="right") - 1, 0, 4095)
        z[k] = np.trapezoid(ps_table.pdf64[idx] * np.maximum(0, 1 - np.abs(xs - c) / hh), xs)
    base = f(mu_s, mu_a)
    phi0 = np.maximum(0, 1 - np.abs(nodes) / (2 / 63))
    want = base * (phi0 - z)
    assert np.all(np.abs(g[3:] - want) < 4 * sig[3:] + 2e-3 * abs(base))


def test_adjoint_matches_common_random_number_difference(gpu, ps_table):
    import torch
    n, nx = 2_000_000, 64
    mu_s, mu_a = 5.0 / LX - 0.01, 0.01
    adj = torch.rand((nx, nx), generator=torch.Generator().manual_seed(11))
    e = _eng(gpu, nx, nx)
    batches = 8
    outs, fds = [], []
    for b in range(batches):
        off = b * n // batches
        outs.append(e.adjoint(gpu.Medium(mu_s, mu_a, "table", 0.0, ps_table), adj, n // batches, n_w=0,
                              seed=4, photon_offset=off).cpu().numpy())

        def L(ms, ma):
            e.run(gpu.Medium(ms, ma, "table", 0.0, ps_table), n // batches, seed=4, photon_offset=off)
            e.check()
            return float(np.sum(adj.numpy().astype(np.float64) * e.result()["image"]))

        hs, ha = 1e-3 * mu_s, 1e-3 * mu_a
        fds.append([(L(mu_s + hs, mu_a) - L(mu_s - hs, mu_a)) / (2 * hs),
                    (L(mu_s, mu_a + ha) - L(mu_s, mu_a - ha)) / (2 * ha)])
    outs, fds = np.array(outs), np.array(fds)
    g, fd = outs[:, 1:3].sum(axis=0), fds.sum(axis=0)
    sg = outs[:, 1:3].std(axis=0, ddof=1) * math.sqrt(batches)
    sf = fds.std(axis=0, ddof=1) * math.sqrt(batches)
    print("adjoint", g, "+-", sg, " central difference", fd, "+-", sf)
    assert np.all(np.abs(g - fd) < 4 * np.hypot(sg, sf))


def test_autograd_and_adam_recover_mu_s_mu_a(gpu):
    """Target rendered at mu_s = 0.9 mu_s0, mu_a = 0.01 (independent seed,
    1e8 photons); 50 Adam steps on log(mu) from (mu_s0, 0.003) with 1e7
    photons per step, a decaying step size and gradients from photons
    independent of the forward sample."""
    import torch
    t = gpu.PhaseTable()
    tau = 5.0
    mu_s0 = tau / LX
    cam = gpu.Camera(128, 128, 128, R_MAX)
    eng = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    n_t, n = 100_000_000, 10_000_000
    eng.run(gpu.Medium(0.9 * mu_s0, 0.01, "table", 0.0, t), n_t, seed=99)
    eng.check()
    target = torch.tensor(eng.result()["image"] / n_t, device="cuda")
    log_s = torch.tensor(math.log(mu_s0), dtype=torch.float64, requires_grad=True)
    log_a = torch.tensor(math.log(0.003), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([log_s, log_a], lr=0.1)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=0.93)
    scale = 1.0 / float((target ** 2).sum())
    for it in range(50):
        opt.zero_grad()
        # the loss is quadratic in the image: take the gradient from an
        # independent photon set so it is not correlated with the residual
        img = gpu.camera_image(eng, t, torch.exp(log_s), torch.exp(log_a), n_photons=n, seed=1 + 2 * it,
                               grad_seed=2 + 2 * it)
        loss = scale * ((img / n - target) ** 2).sum()
        loss.backward()
        opt.step()
        sched.step()
        if it % 10 == 9:
            print("step %d loss %.3e mu_s %.5f mu_a %.5f" % (it + 1, loss.item(), math.exp(log_s.item()),
                                                         math.exp(log_a.item())))
    ms, ma = math.exp(log_s.item()), math.exp(log_a.item())
    print("recovered mu_s %.5f (true %.5f)  mu_a %.5f (true 0.01)" % (ms, 0.9 * mu_s0, ma))
    assert abs(ms / (0.9 * mu_s0) - 1) < 0.03
    assert abs(ma / 0.01 - 1) < 0.25
