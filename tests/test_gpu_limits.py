"""The CUDA path at the edges of the sizes the C ABI accepts, against the
oracle on the same photons:
  * the smallest and largest equal-probability phase tables (64 and 16384
    bins, Sec. 3.1.2), and the paper's bisection table with 16 angles and
    with 10240 (the most that fit shared memory; 16384 are refused), each
    built by the engine and, independently, by the oracle: the first 32
    events of 4096 photons under the trace rule;
  * a single-pixel camera, a 8192-pixel-wide camera four rows high and a
    four-pixel-wide one 8192 rows high (8192 is the largest side), with
    radial profiles of 1, 16384 and 7 bins (16384 bins next to the 4096-bin
    table leave room for one 8192-pixel row in shared memory: the image is
    split between the band and global memory): every event's pixel and
    radial bin under the trace rule, blocks of pixels within 2e-3 of the
    oracle's on the same photons, exact energy bookkeeping, the ballistic
    weight exact, the radial profile summing exactly to the far-face total
    and, in groups of bins, within 3 sigma of the oracle's;
  * a radial profile too large to share the CTA's shared memory with the
    table (one run, a batch, or the host-buffer entry point), and the largest table with the most majorant cells in the
    density gradient's kernel, are refused on the host before anything
    runs (the tallies keep their contents); that table and grid with a
    128-bin profile fit a grid walk, whose traces follow the oracle's.
"""
import numpy as np
import pytest

from parity import compare_traces, report_unmatched

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5
TAU = 5.0


@pytest.mark.parametrize("n_bins", [64, 16384])
def test_table_size_extremes_follow_the_oracle(gpu, oracle_mod, n_bins):
    tab = gpu.PhaseTable(diameter_um=5.0, n_particle=1.59, n_medium=1.33, wavelength_nm=532.0, n_bins=n_bins)
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    otab = oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x, n_bins=n_bins)
    n = 4096
    eng = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    tr = gpu.decode_trace(eng.trace(gpu.Medium(TAU / LX, 0.0, "table", 0.0, tab), n, n, 32, seed=13))
    eng.check()
    o = oracle_mod.walk(mu_s=TAU / LX, table=otab, n_photons=n, nx=64, nz=64, seed=13, n_trace=n,
                        n_trace_events=32)
    cmp = compare_traces(tr, o["trace"], TAU / LX)
    print(n_bins, "matched %d/%d flips %d events %d worst %s" %
          (cmp["matched"], n, cmp["flips"], cmp["events"], {k: "%.2e" % v for k, v in cmp["worst"].items()}))
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp["causes"][:5]
    assert cmp["events"] > 1.5 * n


def _blocks(img, gz, gx):
    nz, nx = img.shape
    return img.reshape(gz, nz // gz, gx, nx // gx).sum(axis=(1, 3))


@pytest.mark.parametrize("nx,nz,n_radial", [(1, 1, 1), (8192, 4, 16384), (4, 8192, 7)])
def test_camera_and_profile_extremes_match_oracle(gpu, oracle_mod, ps_table, ps_oracle_table, nx, nz, n_radial):
    med = gpu.Medium(TAU / LX, 0.0, "table", 0.0, ps_table)
    cam = dict(nx=nx, nz=nz, n_radial=n_radial, r_max=R_MAX)
    eng = gpu.Engine(gpu.Camera(nx, nz, n_radial, R_MAX), gpu.Geometry(LX, LY, LZ))

    # every event's pixel and radial bin (at 8192 pixels a side a pixel is
    # 5.5 or 1.2 um: a decision may differ only within 1e-5 of an edge)
    nt = 2048
    tr = gpu.decode_trace(eng.trace(med, nt, nt, 32, seed=21))
    eng.check()
    ot = oracle_mod.walk(mu_s=TAU / LX, table=ps_oracle_table, n_photons=nt, seed=21, n_trace=nt,
                         n_trace_events=32, **cam)
    cmp = compare_traces(tr, ot["trace"], TAU / LX)
    print(nx, nz, n_radial, "traces matched %d/%d flips %d" % (cmp["matched"], nt, cmp["flips"]))
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * nt, cmp["causes"][:5]

    n = 200_000
    eng.run(med, n, seed=21)
    eng.check()
    r = eng.result()
    o = oracle_mod.walk(mu_s=TAU / LX, table=ps_oracle_table, n_photons=n, seed=21, **cam)
    raw = r["raw_totals"]
    assert raw[0] + raw[1] + raw[2] == n << 32
    assert r["totals"][6] == o["totals"][6]            # ballistic: decided by the first uniform alone
    assert abs(r["steps"] - o["steps"]) <= max(2, 1e-4 * o["steps"])

    # image on the same photons: blocks of pixels (a contribution changes
    # block only through a near-edge flip at a block boundary or a photon
    # whose path diverged), the whole image
    assert r["image"].shape == (nz, nx)
    gz, gx = min(nz, 64), min(nx, 64)
    b, bo, hits = _blocks(r["image"], gz, gx), _blocks(o["image"], gz, gx), _blocks(o["image_hits"], gz, gx)
    well = hits >= 200
    dev = np.abs(b - bo)[well] / bo[well]
    print(nx, nz, n_radial, "blocks %d (well populated %d), worst rel dev %.2e, sum %.6g vs %.6g" %
          (b.size, int(well.sum()), dev.max(), r["image"].sum(), o["image"].sum()))
    assert well.sum() >= min(b.size, 64) // 2
    assert dev.max() < 2e-3
    assert r["image"].sum() == pytest.approx(o["image"].sum(), rel=2e-3)

    # radial profile: the far-face weight, bin by bin
    rad_raw = eng.radial.cpu().numpy()
    assert rad_raw.shape == (n_radial,)
    assert int(rad_raw.sum()) == int(raw[1])          # every transmitted photon lands in one bin
    assert abs(r["radial"].sum() - o["radial"].sum()) <= 2e-3 * o["radial"].sum()
    group = max(1, n_radial // 128)
    ng = n_radial // group
    gr = r["radial"][:ng * group].reshape(ng, group).sum(1)
    go = o["radial"][:ng * group].reshape(ng, group).sum(1)
    gv = o["radial_sq"][:ng * group].reshape(ng, group).sum(1) - go ** 2 / n
    assert np.all(np.abs(gr - go) <= 3 * np.sqrt(2 * np.maximum(gv, 0)) + 1e-6), np.max(np.abs(gr - go))


def test_profile_too_large_for_shared_memory_is_refused(gpu, ps_table):
    from paper_2507_23189_gb300 import _native as N
    eng = gpu.Engine(gpu.Camera(64, 64, 65536, R_MAX), gpu.Geometry(LX, LY, LZ))
    eng.image.fill_(5)
    with pytest.raises(N.McError) as ex:
        eng.run(gpu.Medium(TAU / LX, 0.0, "table", 0.0, ps_table), 1000, seed=1)
    assert ex.value.status == -1                     # MC_ERR_ARG, before anything ran
    eng.check()
    assert int(eng.image[0, 0].item()) == 5 and eng.last_error == 0


def test_largest_table_with_most_majorant_cells(gpu, oracle_mod):
    """A 16384-bin table (164 KB) beside 16384 majorant cells (64 KB, the most
    a grid may have) and a 128-bin profile just fits a grid walk's shared
    memory: its traces follow the oracle's. The density gradient's flight
    queues (12 KB more), or a 1024-bin profile, do not fit: refused before
    anything runs, the tallies keeping their contents."""
    import torch
    from paper_2507_23189_gb300 import _native as N
    from paper_2507_23189_gb300 import workloads as W
    dens = W.rough_grid((64, 64, 64), 4, mean=2000.0)
    k_ext, k_sca, block = 4e-5, 4e-5, (2, 2, 4)          # 32 x 32 x 16 cells
    geo = gpu.Geometry(LX, LY, LZ)
    grid = gpu.Grid(torch.from_numpy(dens).cuda(), k_ext, k_sca, 0.0, block)
    grid.prepare(geo)
    big = gpu.PhaseTable(n_bins=16384)
    med = gpu.Medium(1.0, 0.0, "table", 0.0, big)
    n = 4096
    eng = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), geo)
    tr = gpu.decode_trace(eng.run_grid(grid, med, n, seed=13, n_trace=n, n_events=32))
    eng.check()
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    otab = oracle_mod.phase_table(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x, n_bins=16384)
    o = oracle_mod.walk(mu_s=0.0, phase="mie", table=otab, n_photons=n, nx=64, nz=64, seed=13, n_trace=n,
                        n_trace_events=32,
                        grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca, block=block))
    cmp = compare_traces(tr, o["trace"], mu_ext=k_ext * float(dens.max()))
    print("grid, 16384 bins, 16384 cells: matched %d/%d flips %d events %d" %
          (cmp["matched"], n, cmp["flips"], cmp["events"]))
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp["causes"][:5]
    assert cmp["events"] > 2 * n

    eng.image.fill_(5)
    adj = torch.ones((64, 64), dtype=torch.float32, device="cuda")
    for nulls in (None, 1.25):
        with pytest.raises(N.McError) as ex:
            eng.grid_adjoint(grid, med, adj, 1000, seed=1, nulls=nulls)
        assert ex.value.status == -1
    wide = gpu.Engine(gpu.Camera(64, 64, 1024, R_MAX), geo)
    wide.image.fill_(5)
    with pytest.raises(N.McError) as ex:
        wide.run_grid(grid, med, 1000, seed=1)
    assert ex.value.status == -1
    eng.check()
    wide.check()
    assert int(eng.image[0, 0].item()) == 5 and int(wide.image[0, 0].item()) == 5
    assert eng.last_error == 0 and wide.last_error == 0


def test_batch_with_profile_too_large_for_shared_memory_is_refused(gpu, ps_table):
    from paper_2507_23189_gb300 import _native as N
    b = gpu.Batch(2, gpu.Camera(64, 64, 65536, R_MAX), gpu.Geometry(LX, LY, LZ))
    b.image.fill_(5)
    med = gpu.Medium(TAU / LX, 0.0, "table", 0.0, ps_table)
    with pytest.raises(N.McError) as ex:
        b.run([med, med], [1000, 2000], [1, 2])
    assert ex.value.status == -1
    b.check()
    assert int(b.image.min().item()) == 5 and int(b.image.max().item()) == 5


def test_host_buffer_entry_point_refuses_before_copying(gpu, ps_table):
    import torch
    from paper_2507_23189_gb300 import _native as N
    med = gpu.Medium(TAU / LX, 0.0, "table", 0.0, ps_table)
    cam, geo = gpu.Camera(64, 64, 65536, R_MAX), gpu.Geometry(LX, LY, LZ)
    work = torch.empty(gpu.host_workspace_bytes(med, cam), dtype=torch.uint8, device="cuda")
    image = np.full((64, 64), 5, dtype=np.int64)
    with pytest.raises(N.McError) as ex:
        gpu.run_host(med, geo, cam, 1000, work, image=image)
    assert ex.value.status == -1
    assert np.all(image == 5)


def _paper_slope(mu):
    # the paper table's camera density ~ 1 / sin(theta_c) inside an interval
    return abs(mu) / max(1.0 - mu * mu, 1e-300)


@pytest.mark.parametrize("n_theta", [16, 10240])
def test_paper_table_size_extremes_follow_the_oracle(gpu, oracle_mod, n_theta):
    """The paper's bisection table (Sec. 3.1.2) with the fewest angles and with
    the most that fit shared memory beside the tallies (10240: 221 KB)."""
    t = gpu.PaperTable(n_theta=n_theta)
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    ot = oracle_mod.paper_cdf(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x, n_theta=n_theta)
    n = 4096
    eng = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    tr = gpu.decode_trace(eng.trace(gpu.Medium(TAU / LX, 0.0, "paper", 0.0, t), n, n, 32, seed=17))
    eng.check()
    o = oracle_mod.walk(mu_s=TAU / LX, phase="paper", table=ot, n_photons=n, nx=64, nz=64, seed=17, n_trace=n,
                        n_trace_events=32)
    cmp = compare_traces(tr, o["trace"], TAU / LX, nee_slope=_paper_slope)
    print("paper", n_theta, "matched %d/%d flips %d events %d" % (cmp["matched"], n, cmp["flips"], cmp["events"]))
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp["causes"][:5]
    assert cmp["events"] > 1.5 * n


def test_paper_table_too_large_for_shared_memory_is_refused(gpu):
    from paper_2507_23189_gb300 import _native as N
    t = gpu.PaperTable(n_theta=16384)                 # 344 KB
    eng = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    eng.image.fill_(5)
    with pytest.raises(N.McError) as ex:
        eng.run(gpu.Medium(TAU / LX, 0.0, "paper", 0.0, t), 1000, seed=1)
    assert ex.value.status == -1
    eng.check()
    assert int(eng.image[0, 0].item()) == 5
