"""Edge cases and invariances of the CUDA path: empty and ragged ranges,
64-bit photon indices, launch-shape independence, truncation flags, finite
beams, error reporting, the host-buffer entry point, a pure absorber, H-G at
extreme anisotropy, extreme optical depths and a thin-plate geometry."""
import ctypes as C
import math

import numpy as np
import pytest

from parity import compare_traces, report_unmatched

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _eng(gpu, nx=64, nz=64, geom=None):
    return gpu.Engine(gpu.Camera(nx, nz, 128, R_MAX), geom or gpu.Geometry(LX, LY, LZ))


def _g_or(oracle_mod):
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    return oracle_mod.mie_efficiencies(complex(1.59 / 1.33, 0.0), x)[2]


def test_zero_photons_zeroes_tallies(gpu, ps_table):
    e = _eng(gpu)
    med = gpu.Medium(0.1, 0.0, "table", 0.0, ps_table)
    e.run(med, 1000)
    e.run(med, 0)
    e.check()
    r = e.result()
    assert not r["raw_image"].any() and not r["raw_totals"].any()


@pytest.mark.parametrize("n", [1, 37, 1000, 100_003])
def test_ragged_counts_match_oracle(gpu, oracle_mod, ps_table, ps_oracle_table, n):
    e = _eng(gpu, 16, 16)
    e.run(gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table), n, seed=9)
    e.check()
    r = e.result()
    o = oracle_mod.walk(mu_s=5 / LX, table=ps_oracle_table, n_photons=n, nx=16, nz=16, seed=9)
    assert r["raw_totals"][0] + r["raw_totals"][1] + r["raw_totals"][2] == n << 32
    assert abs(r["steps"] - o["steps"]) <= max(2, 1e-4 * o["steps"])
    # same photons on both sides: only rare precision flips can move weight
    assert r["image"].sum() == pytest.approx(o["image"].sum(), rel=2e-3)
    assert r["totals"][6] == o["totals"][6]


def test_photon_index_crosses_32_bits(gpu, oracle_mod, ps_table, ps_oracle_table):
    off = (1 << 32) - 100
    n = 256
    e = _eng(gpu)
    tr = gpu.decode_trace(e.trace(gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table), n, n, 32, seed=4,
                                  photon_offset=off))
    e.check()
    o = oracle_mod.walk(mu_s=5 / LX, table=ps_oracle_table, n_photons=n, photon_offset=off, nx=64, nz=64,
                        seed=4, n_trace=n, n_trace_events=32)
    cmp = compare_traces(tr, o["trace"], 5 / LX)
    assert cmp["matched"] == n, cmp


@pytest.mark.parametrize("phase", ["table", "hg"])
def test_launch_shape_does_not_change_results(gpu, ps_table, phase):
    med = gpu.Medium(5 / LX, 0.002, phase, ps_table.info["g"], ps_table)
    ref = None
    for kw in (dict(), dict(block_size=64), dict(block_size=128, blocks_per_sm=1),
               dict(image_mode=1), dict(image_mode=2), dict(block_size=32, image_mode=2),
               dict(image_mode=3), dict(image_mode=3, block_size=512)):
        e = _eng(gpu)
        e.run(med, 300_000, seed=2, **kw)
        e.check()
        r = e.result()
        if ref is None:
            ref = r
        else:
            np.testing.assert_array_equal(r["raw_image"], ref["raw_image"])
            np.testing.assert_array_equal(r["raw_totals"], ref["raw_totals"])


@pytest.mark.parametrize("nx,nz", [(256, 256), (512, 512), (300, 97)])
def test_band_and_global_images_identical(gpu, ps_table, nx, nz):
    """Rows routed to the shared-memory band or to L2 atomics sum identically."""
    med = gpu.Medium(10 / LX, 0.0, "table", 0.0, ps_table)
    out = []
    for mode in (2, 3):
        e = _eng(gpu, nx, nz)
        e.run(med, 1_000_000, seed=5, image_mode=mode)
        e.check()
        out.append(e.result())
    np.testing.assert_array_equal(out[0]["raw_image"], out[1]["raw_image"])
    np.testing.assert_array_equal(out[0]["raw_totals"], out[1]["raw_totals"])


def test_repeat_runs_bit_identical(gpu, ps_table):
    med = gpu.Medium(10 / LX, 0.0, "table", 0.0, ps_table)
    out = []
    for _ in range(2):
        e = _eng(gpu, 256, 256)
        e.run(med, 2_000_000, seed=1)
        e.check()
        out.append(e.result())
    np.testing.assert_array_equal(out[0]["raw_image"], out[1]["raw_image"])
    np.testing.assert_array_equal(out[0]["raw_totals"], out[1]["raw_totals"])


def test_event_cap_truncates_and_flags(gpu, oracle_mod, ps_table, ps_oracle_table):
    from paper_2507_23189_gb300 import _native as N
    med = gpu.Medium(20 / LX, 0.0, "table", 0.0, ps_table)
    e = _eng(gpu)
    tr = gpu.decode_trace(e.trace(med, 5000, 64, 8, seed=1, max_events=3))
    with pytest.raises(N.McError) as err:
        e.check()
    assert err.value.status == -7
    r = e.result()
    o = oracle_mod.walk(mu_s=20 / LX, table=ps_oracle_table, n_photons=5000, nx=64, nz=64, seed=1,
                        max_events=3)
    assert r["totals"][5] == pytest.approx(o["totals"][5], rel=1e-6)
    assert r["steps"] == o["steps"]
    assert np.any(tr["status"][:, 3] == 6) and np.all(tr["status"][:, 4:] == -1)


def test_max_scatter_one(gpu, ps_table):
    e = _eng(gpu)
    e.run(gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table), 100_000, max_scatter=1)
    e.check()
    r = e.result()
    t = r["raw_totals"]
    assert t[1] + t[2] + t[0] + t[5] == 100_000 << 32
    img = r["image"]
    assert np.count_nonzero(np.delete(img, 32, axis=0)) == 0


def test_finite_beam_matches_oracle(gpu, oracle_mod, ps_table, ps_oracle_table):
    geom = gpu.Geometry(LX, LY, LZ, 1.25)   # the paper's 2.5 mm beam
    n = 2048
    e = _eng(gpu, geom=geom)
    tr = gpu.decode_trace(e.trace(gpu.Medium(5 / LX, 0.0, "table", 0.0, ps_table), n, n, 32, seed=8))
    e.check()
    o = oracle_mod.walk(mu_s=5 / LX, table=ps_oracle_table, n_photons=n, nx=64, nz=64, seed=8,
                        beam_radius=1.25, n_trace=n, n_trace_events=32)
    cmp = compare_traces(tr, o["trace"], 5 / LX)
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp


def test_bad_arguments_raise(gpu, ps_table):
    from paper_2507_23189_gb300 import _native as N
    e = _eng(gpu)
    with pytest.raises(N.McError):
        e.run(gpu.Medium(-0.1, 0.0, "table", 0.0, ps_table), 10)
    with pytest.raises(N.McError):
        e.run(gpu.Medium(0.1, 0.0, "hg", 1.5), 10)
    with pytest.raises(N.McError):
        e.run(gpu.Medium(0.1, 0.0, "table", 0.0, ps_table), 10, rr_survival=2.0)
    with pytest.raises(N.McError):
        e.run(gpu.Medium(0.1, 0.0, "table", 0.0, ps_table), 10, block_size=48)
    big = _eng(gpu, 512, 512)
    with pytest.raises(N.McError):   # a 2 MB image tile cannot live in shared memory
        big.run(gpu.Medium(0.1, 0.0, "table", 0.0, ps_table), 10, image_mode=1)


def test_corrupt_table_is_reported(gpu, ps_table):
    import torch
    from paper_2507_23189_gb300 import _native as N
    bad = ps_table.device_blob().clone()
    bad[0] ^= 0xFF
    m = N.Medium(0.1, 0.0, N.PHASE_TABLE, 0.0, bad.data_ptr(), 4096)
    e = _eng(gpu)
    rp = gpu.run_params(1000)
    g, c, t = e.geometry.as_c(), e.camera.as_c(), e._tallies()
    st = N.lib().mc_run(C.byref(m), C.byref(g), C.byref(c), C.byref(rp), C.byref(t),
                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    with pytest.raises(N.McError) as err:
        e.check()
    assert err.value.status == -8


@pytest.mark.parametrize("phase", ["table", "hg"])
def test_host_entry_point_equals_device_entry_point(gpu, ps_table, phase):
    import torch
    med = gpu.Medium(5 / LX, 0.001, phase, ps_table.info["g"], ps_table)
    cam = gpu.Camera(128, 128, 128, R_MAX)
    e = gpu.Engine(cam, gpu.Geometry(LX, LY, LZ))
    e.run(med, 500_000, seed=3)
    e.check()
    r = e.result()
    work = torch.empty(gpu.host_workspace_bytes(med, cam), dtype=torch.uint8, device="cuda")
    img, rad, tot = gpu.run_host(med, gpu.Geometry(LX, LY, LZ), cam, 500_000, work, seed=3)
    np.testing.assert_array_equal(img, r["raw_image"])
    np.testing.assert_array_equal(tot, r["raw_totals"])
    np.testing.assert_array_equal(rad, e.radial.cpu().numpy())


def test_multi_wall_exits_in_a_cube_match_oracle(gpu, oracle_mod):
    """A 10 mm cube with isotropic scattering: many last flights cross two or
    three walls, so the exit face comes from comparing wall distances
    (reflected / far / side) on every such photon. Traces against the oracle
    and the exit tallies on the same photons."""
    geom = gpu.Geometry(10.0, 10.0, 10.0)
    med = gpu.Medium(0.2, 0.0, "hg", 0.0, None)
    n = 4096
    e = gpu.Engine(gpu.Camera(32, 32, 128, R_MAX), geom)
    tr = gpu.decode_trace(e.trace(med, n, n, 32, seed=12))
    e.check()
    o = oracle_mod.walk(mu_s=0.2, phase="hg", hg_g=0.0, lx=10.0, ly=10.0, lz=10.0, n_photons=n, nx=32, nz=32,
                        seed=12, n_trace=n, n_trace_events=32)
    cmp = compare_traces(tr, o["trace"], 0.2, lx=10.0)
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp
    n = 1_000_000
    e = gpu.Engine(gpu.Camera(32, 32, 128, R_MAX), geom)
    e.run(med, n, seed=3)
    e.check()
    g = e.result()["totals"]
    o = oracle_mod.walk(mu_s=0.2, phase="hg", hg_g=0.0, lx=10.0, ly=10.0, lz=10.0, n_photons=n, nx=32, nz=32,
                        seed=3)["totals"]
    # same photons: only near-tie decisions may differ
    for k in range(3):                     # reflected, far face, side faces
        assert g[k] == pytest.approx(o[k], rel=1e-4, abs=2.0)
    assert g[1] > 0.1 * n and g[2] > 0.3 * n and g[0] > 0.1 * n


@pytest.mark.parametrize("phase", ["table", "hg"])
def test_pure_absorber_matches_oracle(gpu, oracle_mod, ps_table, ps_oracle_table, phase):
    """mu_s = 0 (albedo 0): every collision captures the whole weight (Eq. 16),
    so the far face sees only ballistic photons, the other faces and the
    camera nothing, and absorption takes the rest; a zero-weight photon goes
    on until roulette ends it, step for step as in the oracle."""
    n, tau = 100_000, 2.0
    e = _eng(gpu, 16, 16)
    e.run(gpu.Medium(0.0, tau / LX, phase, 0.5, ps_table), n, seed=4)
    e.check()
    r = e.result()
    om = dict(phase="mie", table=ps_oracle_table) if phase == "table" else dict(phase="hg", hg_g=0.5)
    o = oracle_mod.walk(mu_s=0.0, mu_a=tau / LX, n_photons=n, nx=16, nz=16, seed=4, **om)
    raw = r["raw_totals"]
    assert raw[0] == 0 and raw[2] == 0 and raw[1] == raw[6]
    assert raw[1] + raw[3] == n << 32                  # exact: ballistic exits plus whole captures
    assert not r["raw_image"].any() and o["image"].sum() == 0.0
    assert abs(raw[1] / 2 ** 32 - o["totals"][6]) <= 1
    assert abs(r["steps"] - o["steps"]) <= 2
    p = math.exp(-tau)
    assert abs(raw[1] / 2 ** 32 / n - p) < 5 * math.sqrt(p * (1 - p) / n)


@pytest.mark.parametrize("g", [-0.9, 0.0, 0.99])
def test_hg_extreme_anisotropy_traces_match_oracle(gpu, oracle_mod, g):
    """Eq. 11 sampled and scored at strong back-scattering, isotropy and
    strong forward scattering (where 1 - g = 0.01 sets the scale of both the
    sampled 1 - cos(theta) and the camera density's peak)."""
    n, tau = 4096, 5.0
    e = _eng(gpu)
    tr = gpu.decode_trace(e.trace(gpu.Medium(tau / LX, 0.0, "hg", g), n, n, 32, seed=6))
    e.check()
    o = oracle_mod.walk(mu_s=tau / LX, phase="hg", hg_g=g, n_photons=n, nx=64, nz=64, seed=6, n_trace=n,
                        n_trace_events=32)
    slope = lambda mu: 3.0 * abs(g) / (1.0 + g * g - 2.0 * g * mu)
    cmp = compare_traces(tr, o["trace"], tau / LX, nee_slope=slope)
    print("g", g, "matched %d/%d flips %d events %d worst %s" %
          (cmp["matched"], n, cmp["flips"], cmp["events"], {k: "%.2e" % v for k, v in cmp["worst"].items()}))
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp["causes"][:5]
    assert cmp["events"] > 1.5 * n


@pytest.mark.parametrize("tau,geom,beam", [(0.01, (45.0, 10.0, 10.0), 0.0), (100.0, (45.0, 10.0, 10.0), 0.0),
                                           (5.0, (2.0, 50.0, 0.5), 0.2)])
def test_extreme_depth_and_geometry_traces_match_oracle(gpu, oracle_mod, ps_table, ps_oracle_table, tau, geom, beam):
    """A nearly transparent cuvette (tau = 0.01: almost every photon ballistic),
    a very thick one (tau = 100: steps of 0.45 mm, positions summed over many
    of them) and a thin plate 2 x 50 x 0.5 mm crossed by a 0.2 mm beam (most
    photons leave through the nearby z faces)."""
    n = 4096
    lx, ly, lz = geom
    e = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(lx, ly, lz, beam))
    tr = gpu.decode_trace(e.trace(gpu.Medium(tau / lx, 0.0, "table", 0.0, ps_table), n, n, 32, seed=12))
    e.check()
    o = oracle_mod.walk(mu_s=tau / lx, table=ps_oracle_table, lx=lx, ly=ly, lz=lz, beam_radius=beam, n_photons=n,
                        nx=64, nz=64, seed=12, n_trace=n, n_trace_events=32)
    cmp = compare_traces(tr, o["trace"], tau / lx, lx=lx)
    print("tau", tau, geom, "matched %d/%d flips %d events %d worst %s" %
          (cmp["matched"], n, cmp["flips"], cmp["events"], {k: "%.2e" % v for k, v in cmp["worst"].items()}))
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n, cmp["causes"][:5]
    assert cmp["events"] >= n


@pytest.mark.parametrize("lz,nz", [(5.6997014, 24), (10.0, 64), (4.2667066, 30), (0.964, 2)])
def test_first_collisions_on_the_axis_fall_in_row_nz_over_2(gpu, lz, nz):
    """A pencil beam's first collisions lie on z = 0, the edge between rows
    nz/2 - 1 and nz/2, and belong to row nz/2 whatever the cuvette height
    (5.6997 mm with 24 rows once sent them to row 11); with max_scatter = 1
    only first collisions add camera terms."""
    e = gpu.Engine(gpu.Camera(8, nz, 16, R_MAX), gpu.Geometry(20.0, 8.0, lz))
    e.run(gpu.Medium(0.1, 0.0, "hg", 0.3), 2000, seed=3, max_scatter=1)
    e.check()
    rows = e.result()["raw_image"].sum(axis=1)
    assert rows[nz // 2] > 0 and rows.sum() == rows[nz // 2]
