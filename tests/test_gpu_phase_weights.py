"""Phase weights w != 1 on the GPU. The phase function p_w = p h_w / Z(w)
(p the unweighted table's density, h_w the hat functions' interpolant of the
weights) is tabulated on the device by mc_phase_table_weighted; the walk
samples it and uses it as the camera density, and mc_adjoint evaluates the
gradient at w. Against the oracle's reweighted table and its walk and
gradient on the same photons, and in an Adam fit of hat weights to a target
image rendered at perturbed weights."""
import math

import numpy as np
import pytest

from parity import compare_traces, oracle_var, tally_agreement

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _decode(blob):
    b = blob.cpu().numpy() if hasattr(blob, "cpu") else blob
    hdr = np.frombuffer(b[:64].tobytes(), dtype=np.uint32)
    n = int(hdr[2])
    off_omu, off_pdf, off_guide, total = (int(v) for v in hdr[4:8])
    omu = np.frombuffer(b[off_omu:off_omu + 4 * (n + 1)].tobytes(), dtype=np.float32)
    pdf = np.frombuffer(b[off_pdf:off_pdf + 4 * n].tobytes(), dtype=np.float32)
    guide = np.frombuffer(b[off_guide:off_guide + 2 * (n + 1)].tobytes(), dtype=np.uint16)
    g_table = float(np.frombuffer(b[32:36].tobytes(), dtype=np.float32)[0])
    return dict(magic=int(hdr[0]), n=n, omu=omu, pdf=pdf, guide=guide, g_table=g_table, total=total)


def _weights(n_w, seed, lo=0.5, hi=1.6):
    return np.random.default_rng(seed).uniform(lo, hi, n_w).astype(np.float32)


def _wt(gpu, base, w):
    import torch
    wt = gpu.WeightedTable(base, torch.tensor(w, device="cuda"))
    wt.check()
    return wt


def _guide_brackets(d):
    """For a direction cosine m in cell c = floor(fl(m + 1) n/2), the largest
    j with omu[j] >= fl(1 - m) lies in [guide[c], guide[c + 1]] (the walk's
    single-precision lookup)."""
    n, omu, guide = d["n"], d["omu"], d["guide"]
    rng = np.random.default_rng(3)
    m = np.concatenate([rng.uniform(-1, 1, 20000), 1 - rng.uniform(0, 1e-3, 5000),
                        np.linspace(-1, 1, 8193)]).astype(np.float32)
    m = np.clip(m, np.float32(-1), np.float32(1))
    cell = np.minimum(np.floor((m + np.float32(1)) * np.float32(n / 2)).astype(np.int64), n - 1)
    om = np.float32(1) - m
    j = np.clip(np.searchsorted(-omu, -om, side="right") - 1, 0, n - 1)
    return bool(np.all(guide[cell] <= j) and np.all(j <= guide[cell + 1]))


@pytest.mark.parametrize("n_w,seed", [(5, 1), (64, 2), (256, 3)])
def test_weighted_table_matches_oracle(gpu, oracle_mod, ps_table, ps_oracle_table, n_w, seed):
    w = _weights(n_w, seed)
    d = _decode(_wt(gpu, ps_table, w).device_blob())
    o = oracle_mod.phase_table_reweighted(ps_oracle_table, w.astype(np.float64))
    assert d["magic"] == 0x544D434D and d["n"] == 4096
    assert np.all(np.diff(d["omu"]) < 0)
    np.testing.assert_allclose(d["omu"], o["omu"], rtol=3e-7, atol=1e-12)
    np.testing.assert_allclose(d["pdf"], o["pdf"], rtol=3e-6)
    assert d["g_table"] == pytest.approx(o["mean"], abs=2e-6)
    assert _guide_brackets(d)


def test_unit_weights_give_back_the_table(gpu, ps_table):
    d = _decode(_wt(gpu, ps_table, np.ones(16, np.float32)).device_blob())
    b = _decode(ps_table.blob)
    # the levels are found again from the table's bin densities: the same
    # floats up to one unit in the last place, the same densities
    ulp = np.abs(d["omu"].view(np.int32).astype(np.int64) - b["omu"].view(np.int32).astype(np.int64))
    assert ulp.max() <= 1
    np.testing.assert_allclose(d["pdf"], b["pdf"], rtol=1e-7)
    assert _guide_brackets(d)


def test_non_positive_weights_are_flagged(gpu, ps_table):
    import torch
    from paper_2507_23189_gb300 import _native as N
    for bad in (0.0, -0.5, float("nan")):
        w = np.ones(8, np.float32)
        w[3] = bad
        wt = gpu.WeightedTable(ps_table, torch.tensor(w, device="cuda"))
        with pytest.raises(N.McError) as err:
            wt.check()
        assert err.value.status == -6
        # a walk on that blob stops at its header check
        e = gpu.Engine(gpu.Camera(32, 32, 16, R_MAX), gpu.Geometry(LX, LY, LZ))
        e.run(gpu.Medium(5 / LX, 0.0, "table", 0.0, wt), 10_000, seed=1)
        with pytest.raises(N.McError) as err:
            e.check()
        assert err.value.status == -8


@pytest.mark.parametrize("n_w", [6, 64])
def test_trace_parity_at_weights(gpu, oracle_mod, ps_table, ps_oracle_table, n_w):
    n, tau = 4096, 5.0
    w = _weights(n_w, 10 + n_w)
    wt = _wt(gpu, ps_table, w)
    e = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    tr = gpu.decode_trace(e.trace(gpu.Medium(tau / LX, 0.0, "table", 0.0, wt), n, n, 32, seed=11))
    e.check()
    ot = oracle_mod.phase_table_reweighted(ps_oracle_table, w.astype(np.float64))
    o = oracle_mod.walk(mu_s=tau / LX, table=ot, n_photons=n, nx=64, nz=64, seed=11, n_trace=n,
                        n_trace_events=32)
    cmp = compare_traces(tr, o["trace"], mu_ext=tau / LX)
    print("n_w %d: %d/%d matched, flips %d, worst %s" % (n_w, cmp["matched"], n, cmp["flips"], cmp["worst"]))
    assert cmp["matched"] == n, cmp["causes"][:10]
    assert cmp["events"] > 1.5 * n


def test_tally_parity_at_weights(gpu, oracle_mod, ps_table, ps_oracle_table):
    n, tau, n_w = 1_000_000, 2.0, 8
    w = _weights(n_w, 21)
    wt = _wt(gpu, ps_table, w)
    cam, geo = gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ)
    med = gpu.Medium(tau / LX, 0.0, "table", 0.0, wt)
    imgs = []
    for b in range(16):
        e = gpu.Engine(cam, geo)
        e.run(med, n // 16, seed=1, photon_offset=b * (n // 16))
        e.check()
        imgs.append(e.result()["image"])
    imgs = np.stack(imgs)
    img, var_g = imgs.sum(axis=0), 16 * imgs.var(axis=0, ddof=1)
    ot = oracle_mod.phase_table_reweighted(ps_oracle_table, w.astype(np.float64))
    o = oracle_mod.walk(mu_s=tau / LX, table=ot, n_photons=n, nx=64, nz=64, seed=1)
    zmax, chi2, dof, p, z = tally_agreement(img, o["image"], oracle_var(o) + var_g, o["image_hits"])
    print("zmax %.2f chi2/dof %.1f/%d p %.3g" % (zmax, chi2, dof, p))
    assert zmax < 3.0 and p > 0.01 and dof > 500


@pytest.mark.parametrize("n_w,mu_a,kw", [(8, 0.0, {}), (64, 0.02, dict(rr_threshold=0.05))])
def test_adjoint_at_weights_matches_oracle(gpu, oracle_mod, ps_table, ps_oracle_table, n_w, mu_a, kw):
    import torch
    n, nx, nz = 200_000, 64, 64
    mu_s = 5.0 / LX - mu_a
    w = _weights(n_w, 30 + n_w)
    adj = np.random.default_rng(8).uniform(0, 1, (nz, nx))
    e = gpu.Engine(gpu.Camera(nx, nz, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    med = gpu.Medium(mu_s, mu_a, "table", 0.0, ps_table)
    out = e.adjoint(med, torch.tensor(adj, dtype=torch.float32), n, n_w=n_w, seed=5,
                    phase_w=torch.tensor(w, device="cuda"), **kw)
    e.check()
    out = out.cpu().numpy()
    ot = oracle_mod.phase_table_reweighted(ps_oracle_table, w.astype(np.float64))
    ores = oracle_mod.adjoint(adj.astype(np.float32).astype(np.float64), n_w, w=w.astype(np.float64),
                              base_table=ps_oracle_table, mu_s=mu_s, mu_a=mu_a, table=ot, n_photons=n, nx=nx,
                              nz=nz, seed=5, **kw)
    g, g2 = ores["grad"], ores["grad_sq"]
    sig = np.sqrt(np.maximum(g2 - g ** 2 / n, 0))
    assert out[0] == pytest.approx(ores["value"], rel=1e-4)
    d = np.abs(out[1:] - g)
    print("n_w %d: rel to sigma max %.3g median %.3g" % (n_w, np.max(d / sig), np.median(d / sig)))
    assert np.all(d <= 0.05 * sig + 1e-4 * np.abs(g) + 1e-9)
    # the forward walk on the device-reweighted table gives the same functional
    e.run(gpu.Medium(mu_s, mu_a, "table", 0.0, _wt(gpu, ps_table, w)), n, seed=5, **kw)
    e.check()
    assert out[0] == pytest.approx(float(np.sum(adj.astype(np.float32).astype(np.float64) *
                                                e.result()["image"])), rel=1e-5)


def test_adam_fits_hat_weights(gpu):
    """Target image rendered at perturbed weights of 6 hats (four of them
    moved by 15-30 %); Adam on log w from w = 1 through torch.autograd
    (camera_image with phase_w), gradients from photons independent of the
    forward sample. The phase function does not change under w -> c w, so
    weights are compared as h_w / Z(w), the density relative to the table's.

    The side camera sees every collision's next-event estimate at the
    direction cosine toward it, which for a beam along x is near 0 (90 deg),
    and the spread of the paths, which the forward peak sets: the image
    determines the density at 90 deg and in the forward peak well, while
    other combinations of the weights move it by far less than its noise (a
    finite-difference Jacobian of the 32x32 image has one dominant singular
    direction, forward peak against side weights). So the fit must bring
    the loss down to its noise floor (the loss of an independent image at the
    true weights) and recover the relative densities at mu = 0 and mu = 1."""
    import torch
    t = gpu.PhaseTable()
    n_w, tau = 6, 5.0
    w_true = np.array([1.0, 1.0, 0.75, 1.3, 0.85, 1.15])
    cam = gpu.Camera(32, 32, 128, R_MAX)
    eng = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    mu_s = torch.tensor(tau / LX, dtype=torch.float64)
    mu_a = torch.tensor(0.0, dtype=torch.float64)
    n_t, n = 1_000_000_000, 100_000_000
    wt_dev = torch.tensor(w_true, device="cuda")
    with torch.no_grad():
        target = gpu.camera_image(eng, t, mu_s, mu_a, phase_w=wt_dev, n_photons=n_t, seed=99) / n_t
        scale = 1.0 / float((target ** 2).sum())
        floor = np.mean([scale * float(((gpu.camera_image(eng, t, mu_s, mu_a, phase_w=wt_dev, n_photons=n,
                                                          seed=500 + k) / n - target) ** 2).sum())
                         for k in range(4)])
    theta = torch.zeros(n_w, dtype=torch.float64, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([theta], lr=0.05)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=0.95)
    losses = []
    for it in range(60):
        opt.zero_grad()
        img = gpu.camera_image(eng, t, mu_s, mu_a, phase_w=torch.exp(theta), n_photons=n, seed=1 + 2 * it,
                               grad_seed=2 + 2 * it)
        loss = scale * ((img / n - target) ** 2).sum()
        loss.backward()
        opt.step()
        sched.step()
        losses.append(loss.item())
        if it % 10 == 9:
            print("step %d loss %.3e w %s" % (it + 1, loss.item(), np.round(np.exp(theta.detach().cpu().numpy()), 4)))
    # hat integrals of the table, for Z(w)
    nodes = -1 + 2 * np.arange(n_w) / (n_w - 1)
    xs = np.linspace(-1, 1, 400_001)
    idx = np.clip(np.searchsorted(t.icdf64, xs, side="right") - 1, 0, t.n_bins - 1)
    pd = t.pdf64[idx]
    zk = np.array([np.trapezoid(pd * np.maximum(0, 1 - np.abs(xs - c) * (n_w - 1) / 2), xs) for c in nodes])
    w_fit = np.exp(theta.detach().cpu().numpy())
    a, b = w_fit / float(w_fit @ zk), w_true / float(w_true @ zk)
    rel90 = abs(np.interp(0.0, nodes, a) / np.interp(0.0, nodes, b) - 1)
    rel0 = abs(a[-1] / b[-1] - 1)
    start = losses[0]
    end = float(np.mean(losses[-5:]))
    print("relative densities h_w/Z at the nodes: fit %s true %s; at 90 deg off by %.4f, forward by %.4f; "
          "loss %.3e -> %.3e (noise floor %.3e)" % (np.round(a, 4), np.round(b, 4), rel90, rel0, start, end, floor))
    assert start > 5 * floor                 # the perturbed start is well above the noise
    assert end < 1.5 * floor
    assert rel90 < 0.03 and rel0 < 0.03
