"""Edge cases of the delta-tracking path on the GPU: no photons, a one-voxel
grid against the oracle's homogeneous walk (traces), a disc beam with the
paper's sampling table, and the event cap."""
import math

import numpy as np
import pytest

from parity import compare_traces, report_unmatched

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
R_MAX = 5.0 * 2 ** 0.5


def _grid(gpu, dens, k_ext, k_sca, mu_a=0.0, block=(1, 1, 1)):
    import torch
    g = gpu.Grid(torch.from_numpy(np.ascontiguousarray(dens, dtype=np.float32)).cuda(), k_ext, k_sca, mu_a,
                 block)
    return g.prepare(gpu.Geometry(LX, LY, LZ))


def test_zero_photons_leave_zero_tallies(gpu, ps_table):
    g = _grid(gpu, np.full((4, 4, 4), 1000.0), 4e-5, 4e-5)
    e = gpu.Engine(gpu.Camera(16, 16, 16, R_MAX), gpu.Geometry(LX, LY, LZ))
    e.run_grid(g, gpu.Medium(1.0, 0.0, "table", 0.0, ps_table), 0, seed=1)
    e.check()
    r = e.result()
    assert not np.any(r["raw_image"]) and not np.any(r["raw_totals"])


def test_one_voxel_grid_traces_match_homogeneous_oracle(gpu, oracle_mod, ps_table, ps_oracle_table):
    """One voxel, majorant = mu_ext: no null collisions, and the delta-tracking
    walk makes the homogeneous walk's decisions with the same numbers."""
    k_ext = 4e-5
    rho = 5.0 / LX / k_ext
    g = _grid(gpu, np.full((1, 1, 1), rho, dtype=np.float32), k_ext, 0.7 * k_ext)
    rho32 = float(np.float32(rho))
    n = 4096
    e = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), gpu.Geometry(LX, LY, LZ))
    tr = gpu.decode_trace(e.run_grid(g, gpu.Medium(1.0, 0.0, "table", 0.0, ps_table), n, seed=17, n_trace=n,
                                     n_events=32, rr_threshold=0.02))
    e.check()
    o = oracle_mod.walk(mu_s=0.7 * k_ext * rho32, mu_a=0.3 * k_ext * rho32, table=ps_oracle_table, n_photons=n,
                        nx=64, nz=64, seed=17, n_trace=n, n_trace_events=32, rr_threshold=0.02)
    cmp = compare_traces(tr, o["trace"], mu_ext=k_ext * rho32)
    print(cmp["matched"], "/", n, "flips", cmp["flips"], "worst", cmp["worst"])
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n
    assert np.any(o["trace"][..., 0] == 4)        # roulette fired


def test_disc_beam_with_paper_table_in_a_grid(gpu, oracle_mod):
    from paper_2507_23189_gb300 import workloads as W
    t = gpu.PaperTable(n_theta=3000)
    x = oracle_mod.size_parameter(5.0, 1.33, 532.0)
    ot = oracle_mod.paper_cdf(oracle_mod.PHASE_MIE, complex(1.59 / 1.33, 0.0), x, n_theta=3000)
    dens = W.rough_grid((8, 16, 32), 21, mean=1500.0)
    k_ext, k_sca = 4e-5, 3.6e-5
    import torch
    geo = gpu.Geometry(LX, LY, LZ, 1.25)
    g = gpu.Grid(torch.from_numpy(dens).cuda(), k_ext, k_sca, 0.0, (8, 4, 4)).prepare(geo)
    n = 4096
    e = gpu.Engine(gpu.Camera(64, 64, 128, R_MAX), geo)
    tr = gpu.decode_trace(e.run_grid(g, gpu.Medium(1.0, 0.0, "paper", 0.0, t), n, seed=23, n_trace=n,
                                     n_events=32))
    e.check()
    o = oracle_mod.walk(mu_s=0.0, phase="paper", table=ot, beam_radius=1.25, n_photons=n, nx=64, nz=64, seed=23,
                        n_trace=n, n_trace_events=32,
                        grid=dict(density=dens.astype(np.float64), k_ext=k_ext, k_sca=k_sca, block=(8, 4, 4)))
    slope = lambda mu: abs(mu) / max(1.0 - mu * mu, 1e-300)
    cmp = compare_traces(tr, o["trace"], mu_ext=k_ext * float(dens.max()), nee_slope=slope)
    print(cmp["matched"], "/", n, "flips", cmp["flips"], "worst", cmp["worst"])
    report_unmatched(cmp)
    assert cmp["matched"] >= 0.999 * n
    assert cmp["events"] > 2 * n


def test_event_cap_is_reported(gpu, ps_table):
    g = _grid(gpu, np.full((4, 4, 8), 40000.0), 4e-5, 4e-5, block=(8, 4, 4))
    e = gpu.Engine(gpu.Camera(16, 16, 16, R_MAX), gpu.Geometry(LX, LY, LZ))
    e.run_grid(g, gpu.Medium(1.0, 0.0, "hg", 0.5, None), 1000, seed=1, max_events=3)
    with pytest.raises(Exception, match="MC_ERR_EVENTS"):
        e.check()
    r = e.result()
    assert r["totals"][5] > 0           # truncated weight
