"""Many media in one persistent launch (mc_run_batch) against one mc_run per
medium: the same photons must give bit-identical integer tallies, whatever
the work-item size, the launch shape or a CUDA-graph capture."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _media(gpu, spec, phase="table"):
    tables = {}
    out = []
    for d, tau, _ in spec:
        if d not in tables:
            tables[d] = gpu.PaperTable(diameter_um=d) if phase == "paper" else gpu.PhaseTable(diameter_um=d)
        t = tables[d]
        out.append(gpu.Medium.from_optical_depth(t, tau, LX, phase=phase))
    return out


def _plain(gpu, cam, med, n, seed, offset=0):
    e = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    e.run(med, n, seed=seed, photon_offset=offset)
    e.check()
    r = e.result()
    return r["raw_image"], e.radial.cpu().numpy(), r["raw_totals"]


SPEC = [(5.0, 5.0, 300_000), (1.0, 0.5, 40_000), (10.0, 20.0, 120_000), (2.5, 2.0, 1),
        (5.0, 12.0, 250_000), (7.0, 8.0, 0), (3.0, 1.0, 77_777)]


@pytest.mark.parametrize("phase", ["table", "hg", "paper"])
@pytest.mark.parametrize("item_photons", [0, 32, 65_536])
def test_batch_equals_plain_runs(gpu, phase, item_photons):
    media = _media(gpu, SPEC, phase)
    cam = gpu.Camera(128, 128, 128, R_MAX)
    b = gpu.Batch(len(media), cam, gpu.Geometry(LX, LY, LZ))
    nph = [n for _, _, n in SPEC]
    seeds = [11 + i for i in range(len(SPEC))]
    offs = [1000 * i for i in range(len(SPEC))]
    b.run(media, nph, seeds, offs, item_photons=item_photons)
    b.check()
    for i, med in enumerate(media):
        img, rad, tot = _plain(gpu, cam, med, nph[i], seeds[i], offs[i])
        np.testing.assert_array_equal(b.image[i].cpu().numpy(), img, err_msg="medium %d" % i)
        np.testing.assert_array_equal(b.radial[i].cpu().numpy(), rad, err_msg="medium %d" % i)
        np.testing.assert_array_equal(b.totals[i].cpu().numpy(), tot, err_msg="medium %d" % i)


def test_batch_launch_shapes_and_band_mode(gpu):
    media = _media(gpu, SPEC[:4])
    nph = [n for _, _, n in SPEC[:4]]
    ref = None
    for cam, kw in ((gpu.Camera(256, 256, 128, R_MAX), {}),
                    (gpu.Camera(256, 256, 128, R_MAX), dict(image_mode=2)),
                    (gpu.Camera(256, 256, 128, R_MAX), dict(block_size=512, image_mode=3))):
        b = gpu.Batch(4, cam, gpu.Geometry(LX, LY, LZ))
        b.run(media, nph, 3, 0, item_photons=8192, **kw)
        b.check()
        got = (b.image.cpu().numpy(), b.totals.cpu().numpy())
        if ref is None:
            ref = got
        else:
            np.testing.assert_array_equal(got[0], ref[0])
            np.testing.assert_array_equal(got[1], ref[1])


def test_batch_in_cuda_graph(gpu):
    import torch
    media = _media(gpu, SPEC[:5])
    nph = [n for _, _, n in SPEC[:5]]
    cam = gpu.Camera(128, 128, 128, R_MAX)
    eager = gpu.Batch(5, cam, gpu.Geometry(LX, LY, LZ))
    eager.run(media, nph, 7, 0)
    eager.check()
    b = gpu.Batch(5, cam, gpu.Geometry(LX, LY, LZ))
    b.run(media, nph, 7, 0)   # warm-up: table uploads, function attributes
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run(media, nph, 7, 0, stream=s)
    for _ in range(2):
        b.image.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        b.check()
        np.testing.assert_array_equal(b.image.cpu().numpy(), eager.image.cpu().numpy())
        np.testing.assert_array_equal(b.totals.cpu().numpy(), eager.totals.cpu().numpy())


def test_batch_rejects_mixed_phase(gpu):
    from paper_2507_23189_gb300 import _native as N
    t = gpu.PhaseTable()
    media = [gpu.Medium(0.1, 0.0, "table", 0.0, t), gpu.Medium(0.1, 0.0, "hg", 0.5)]
    b = gpu.Batch(2, gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    with pytest.raises(N.McError):
        b.run(media, 100)
