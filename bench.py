#!/usr/bin/env python3
"""Throughput of the photon walk on the headline workload.

Workload: the optical-depth sweep's tau = 5 Mie point -- 10x10x45 mm cuvette of
water with 5 um polystyrene spheres at 532 nm, pencil beam along the 45 mm
axis, 4096-bin Mie inverse-CDF table, roulette 1e-4 / 0.1, 1e8 photons per
step, 256x256 side-camera image + 128-bin radial profile, Philox seed 1.
A step is one mc_run over the 1e8 photons (the whole hot path). Metric:
photon-steps (sampled free flights) per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Under torchrun each rank runs its own photon range (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon-steps/s at τ=5 Mie on 1 GB300; batched & adjoint vs plain at matched error"
UNIT = "photon-steps/s"
TAU = 5.0
LX, LY, LZ = 45.0, 10.0, 10.0
NX = NZ = 256
N_RADIAL = 128
R_MAX = 5.0 * 2 ** 0.5
N_PHOTONS = 100_000_000
SEED = 1

# Roofline of the walk kernel: it is bound by single-precision / integer
# issue, not by memory (photon state stays in registers, the table in shared
# memory). Peak = SMs x 128 lanes x max SM clock (thread-instructions/s).
# Work per photon-step = thread-instructions the kernel executes per sampled
# flight on this workload, from ncu (smsp__thread_inst_executed.sum / steps);
# DRAM bytes per launch from the same capture (None when stale).
THREAD_INST_PER_STEP = 242.3          # ncu, 1e7-photon launch of this workload
BATCH_THREAD_INST_PER_STEP = 245.4    # ncu, one batch_kernel launch over the 64 media (taken before the camera row's lower clamp came back: about 1 % low now)
ADJ_W_THREAD_INST_PER_STEP = 344.8    # ncu, adjoint_kernel with 64 phase weights, per forward photon-step (tau 5, 1e7)
ADJ_MU_THREAD_INST_PER_STEP = 250.7   # ncu, adjoint_kernel for mu_s, mu_a only, per forward photon-step
GRID_THREAD_INST_PER_TENTATIVE = 361.0  # ncu, grid_kernel on the plume (cells 32x256x256), per tentative collision
DRAM_BYTES_PER_LAUNCH = 596736        # same capture (table + tallies, L2-resident: the same per launch at 1e8)
LANES_PER_SM = 128
SMEM_WAVEFRONTS_PER_STEP = 0.650       # same capture: shared-memory wavefronts (128 B each) per photon-step
SMEM_BYTES_PER_CLK_SM = 128


def _workload_config():
    return {
        "workload": "tau=5 Mie point of the optical-depth sweep: 10x10x45 mm water cuvette, 5 um "
                    "polystyrene (n=1.59) at 532 nm, pencil beam, 4096-bin Mie table, %.0e photons, "
                    "256x256 side image + 128-bin radial profile, roulette 1e-4/0.1, seed 1" % N_PHOTONS,
        "n_photons": N_PHOTONS, "tau": TAU, "phase": "mie", "image": [NZ, NX], "n_radial": N_RADIAL,
        "l2": "flushed between timed steps (512 MiB write)",
    }


LOAD_WINDOW_S = 0.6   # untimed steps under the clock sampler before the timed ones


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s):
        """Wait (at most timeout_s) until nvidia-smi has printed a reading."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def photon_range(rank, n_per_rank):
    """Weak scaling: rank r runs photons [r n, (r + 1) n). Photons are keyed by
    their global index in the Philox counter, so ranks draw disjoint streams
    and the union is exactly the single-GPU run of ws * n photons."""
    return rank * n_per_rank, n_per_rank


def job_rate(t_local_s, steps_local, ws, device):
    """Whole-job rate: photon-steps summed over ranks divided by the slowest
    rank's time (max over ranks). Returns (rate, t_max, total_steps)."""
    import torch
    t = torch.tensor([t_local_s], dtype=torch.float64, device=device)
    st = torch.tensor([float(steps_local)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(st, op=dist.ReduceOp.SUM)
    t_max, total = float(t.item()), float(st.item())
    return total / t_max, t_max, total


# Arm core part numbers (MIDR part field of implementer 0x41) that /proc/cpuinfo reports
ARM_PARTS = {0xd0c: "Neoverse-N1", 0xd40: "Neoverse-V1", 0xd49: "Neoverse-N2", 0xd4f: "Neoverse-V2",
             0xd8e: "Neoverse-N3", 0xd84: "Neoverse-V3"}


def _cpu_model():
    """The host CPU's model: lscpu's model name, else /proc/cpuinfo's (x86),
    else the Arm part number it lists, else the machine architecture."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name:"):
                return "%s %s" % (platform.machine(), ln.split(":", 1)[1].strip())
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        impl = part = None
        for ln in open("/proc/cpuinfo"):
            low = ln.lower()
            if low.startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
            if low.startswith("cpu implementer"):
                impl = int(ln.split(":", 1)[1], 0)
            if low.startswith("cpu part"):
                part = int(ln.split(":", 1)[1], 0)
        if impl == 0x41 and part is not None:
            return "%s %s" % (platform.machine(), ARM_PARTS.get(part, "Arm part 0x%x" % part))
    except (OSError, ValueError):
        pass
    return platform.machine()


def oracle_sample(n_photons, n_threads=None):
    """Time the oracle (test infrastructure) on n_photons of the workload."""
    import oracle
    x = oracle.size_parameter(5.0, 1.33, 532.0)
    m = complex(1.59 / 1.33, 0.0)
    t = oracle.phase_table(oracle.PHASE_MIE, m, x)
    threads = n_threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.walk(mu_s=TAU / LX, table=t, n_photons=n_photons, nx=NX, nz=NZ, n_radial=N_RADIAL,
                    r_max=R_MAX, seed=SEED, n_threads=threads)
    dt = time.perf_counter() - t0
    return r["steps"], dt, threads


def cpu_baseline(target_s=12.0):
    """Oracle throughput on the host cores over a bounded sample."""
    steps, dt, threads = oracle_sample(200_000)
    rate = steps / dt
    n = int(min(max(200_000 * target_s / max(dt, 1e-3), 200_000), 10 * N_PHOTONS))
    steps, dt, threads = oracle_sample(n)
    s1, d1, _ = oracle_sample(max(n // (4 * threads), 20_000), n_threads=1)
    return {"value": steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d photons of the workload (%d photon-steps) in %.1f s on %d threads of %s; "
                      "single thread: %.3g photon-steps/s" % (n, steps, dt, threads, _cpu_model(), s1 / d1),
            "photons_per_s": n / dt}


def _batch_vs_plain(E, dev, media, nph, steps, warmup, flush):
    """One graph-replayed mc_run_batch against sequential mc_run launches over
    the same photons (identical tallies required)."""
    import torch
    from paper_2507_23189_gb300 import autotune
    cam, geo = E.Camera(128, 128, N_RADIAL, R_MAX), E.Geometry(LX, LY, LZ, 0.0)
    batch = E.Batch(len(media), cam, geo, dev)
    if globals().get("NO_TUNE"):
        tune = dict(item_photons=0, block_size=0, skipped=True)
    else:
        # at the full photon budgets: the best shape at a fraction of them is
        # not the best here (the launch-shape differences are below 1 %)
        tune = autotune.tune_batch(batch, media, nph, scale=1)
    # one image scale for the batch and the sequential runs (the batch's own
    # default: the largest budget's), so their tallies compare bit for bit
    frac = E.auto_frac_bits(max(nph))
    kw = dict(item_photons=tune["item_photons"], block_size=tune["block_size"], image_frac_bits=frac)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        batch.run(media, nph, 1, 0, **kw)
    batch.check()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream(dev)
    cs.wait_stream(stream)
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            batch.run(media, nph, 1, 0, stream=cs, **kw)
    stream.wait_stream(cs)
    engines = [E.Engine(cam, geo, dev) for _ in media]

    def plain():
        for e, m, n in zip(engines, media, nph):
            e.run(m, n, seed=1, stream=stream, image_frac_bits=frac)

    for _ in range(warmup):
        plain()
        g.replay()
    torch.cuda.synchronize(dev)
    batch.check()
    for e in engines:
        e.check()
    same = all(bool(torch.equal(batch.totals[i], e.totals)) and bool(torch.equal(batch.image[i], e.image))
               for i, e in enumerate(engines))
    steps_per_run = int(batch.totals[:, 7].sum().item())

    def timed(fn):
        tot = 0.0
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b) / 1e3
        return tot

    t_batch = timed(g.replay)
    t_plain = timed(plain)
    # how busy the GPU is during the sequential launches: the sum of the
    # launches' own durations (events around each) over the wall time
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in engines]
    busy = []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        wall0, wall1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wall0.record(stream)
        for (a, b), e, m, n in zip(ev, engines, media, nph):
            a.record(stream)
            e.run(m, n, seed=1, stream=stream, image_frac_bits=frac)
            b.record(stream)
        wall1.record(stream)
        wall1.synchronize()
        busy.append(sum(a.elapsed_time(b) for a, b in ev) / wall0.elapsed_time(wall1))
    busy_frac = float(sum(busy) / len(busy))
    # the launches' fixed cost (ramp-up, drain tail, table staging, tally
    # flush): each medium once more at twice its photons (the same first N
    # photons and N more); 2 t(N) - t(2N) is what one launch spends beyond
    # its photons' share, the most a single launch over all media can save
    fixed = []
    for e, m, n in zip(engines, media, nph):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        flush.fill_(1)
        a.record(stream)
        e.run(m, n, seed=1, stream=stream, image_frac_bits=frac)
        b.record(stream)
        e.run(m, 2 * n, seed=1, stream=stream, image_frac_bits=frac)
        c.record(stream)
        c.synchronize()
        fixed.append(2 * a.elapsed_time(b) - b.elapsed_time(c))
    t_one = 1e3 * t_plain / steps
    # with short launches the fixed costs are most of the time and the
    # difference above stops measuring them: no ceiling is stated when the
    # photons' own share comes out below a twentieth of the wall time
    work = t_one * busy_frac - sum(fixed)
    ceiling = t_one / work if work > 0.05 * t_one else None
    return {"value": steps * steps_per_run / t_batch, "unit": UNIT,
            "plain_sequential": steps * steps_per_run / t_plain, "speedup": t_plain / t_batch,
            "plain_busy_fraction": busy_frac, "plain_fixed_ms": float(sum(fixed)),
            "speedup_ceiling": ceiling,
            "ms_batched": 1e3 * t_batch / steps, "ms_plain": 1e3 * t_plain / steps,
            "media": len(media), "photons": int(sum(nph)), "photon_steps": steps_per_run,
            "identical_tallies": same, "tuned": {k: tune[k] for k in ("block_size", "item_photons")}}


def batched_comparison(E, dev, steps, warmup, flush):
    """64 media of uneven optical depth, particle size and photon budget
    (workloads.batched): the batched launch against 64 sequential launches;
    and the same 64 media at 2e5 photons each, where launches are short."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2507_23189_gb300 import workloads
    cases = workloads.batched()
    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        tables = list(ex.map(lambda c: E.PhaseTable(diameter_um=c.diameter_um), cases))
    media = [E.Medium.from_optical_depth(t, c.tau, LX) for t, c in zip(tables, cases)]
    out = _batch_vs_plain(E, dev, media, [c.n_photons for c in cases], steps, warmup, flush)
    out["workload"] = ("64 media: d log-uniform 1-10 um, tau uniform 0.5-20, photons log-uniform 1e6-1e8 "
                       "(numpy Philox seed 2026), 128x128 image, Mie tables, graph-captured batch vs "
                       "64 sequential launches")
    out["media_list"] = [[round(c.diameter_um, 4), round(c.tau, 4), c.n_photons] for c in cases]  # d um, tau, N
    small = _batch_vs_plain(E, dev, media, [200_000] * len(media), steps, warmup, flush)
    small["workload"] = "the same 64 media at 2e5 photons each"
    out["small_budgets"] = small
    return out


def paper_comparison(E, dev, steps, flush):
    """The paper's own set-up (Sec. 4.1, 4.3, 5.2): 30 x 10 x 45 mm cuvette with
    the beam through the 30 mm side, 2.5 mm beam, tau = 8 over 30 mm, plain
    cut at w < 0.001, 1e8 photons, 60 x 90 image: the paper's 3000-angle CDF
    sampled by bisection against the 4096-level equal-probability table, same
    photons; then the Sec. 3.1.4 / Tables 3-4 comparison of the two images and
    of H-G (g from Mie) against the table image."""
    import torch
    table = E.PhaseTable(5.0, 1.59, 1.33, 532.0, 4096)
    paper = E.PaperTable(5.0, 1.59, 1.33, 532.0, 3000)
    lx, tau, n = 30.0, 8.0, 100_000_000
    mu_s = tau / lx * table.info["qsca"] / table.info["qext"]
    cam = E.Camera(60, 90, 64, math.hypot(5.0, 22.5))
    geo = E.Geometry(lx, 10.0, 45.0, 1.25)
    kw = dict(rr_threshold=1e-3, rr_survival=0.0)
    stream = torch.cuda.current_stream(dev)
    out = {}
    imgs = {}
    for name, med in (("table", E.Medium(mu_s, 0.0, "table", 0.0, table)),
                      ("paper", E.Medium(mu_s, 0.0, "paper", 0.0, paper)),
                      ("hg", E.Medium(mu_s, 0.0, "hg", table.info["g"], table))):
        eng = E.Engine(cam, geo, dev)
        for _ in range(3):
            eng.run(med, n, seed=1, stream=stream, **kw)
        torch.cuda.synchronize(dev)
        tot = 0.0
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eng.run(med, n, seed=1, stream=stream, **kw)
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        eng.check()
        ms = tot / steps
        steps_run = int(eng.totals[7].item())
        out[name] = {"ms": ms, "photons_per_s": n / (ms * 1e-3), "photon_steps_per_s": steps_run / (ms * 1e-3)}
        imgs[name] = eng.image.clone()
    m = E.image_metrics(imgs["table"], imgs["paper"], imgs["hg"], n_r=32)
    out["paper_vs_table_speed"] = out["table"]["ms"] / out["paper"]["ms"]
    # context only: the paper reports 4.56e6 photons/s on an RTX 3050 (Sec. 3.1.3)
    out["paper_reported_photons_per_s"] = 4.56e6
    out["metrics_vs_table"] = {
        "paper": {"rmse": m[0], "r": m[1], "zone_rmse": list(m[2:5]), "radial_r": m[5]},
        "hg": {"rmse": m[6], "r": m[7], "zone_rmse": list(m[8:11]), "radial_r": m[11]},
        "paper_closer_rings": m[12]}
    out["workload"] = ("30x10x45 mm cuvette, beam along the 30 mm side, 2.5 mm beam, 5 um PS in water, "
                       "tau=8 over 30 mm, w<0.001 cut, 1e8 photons, 60x90 image; 3000-angle CDF + bisection "
                       "vs 4096-level equal-probability table vs H-G; metrics: min-max normalised, 32 rings")
    return out


def plume_leg(E, dev, steps, flush, n_photons=None):
    """Heterogeneous medium at full size: a 256^3 Gaussian plume (sigma 5 mm,
    centred at x = 22.5 mm) of polystyrene spheres with log-normal diameters
    (median 5 um, sigma_ln 0.3, 16 quantile bins, one mixture table), peak
    optical depth 30 along the beam, 512x512 image, 1e9 photons, delta
    tracking with majorant cells of 32x256x256 voxels (8 slabs along the
    beam). Times mc_grid_prepare, mc_run_grid and the density gradient."""
    import numpy as np
    import torch
    from paper_2507_23189_gb300 import workloads as W
    P = W.plume()
    n = int(n_photons or P.n_photons)
    d, f = W.size_bins(P.median_um, P.sigma_ln, P.n_size_bins)
    t0 = time.time()
    tab = E.MixtureTable(d, f)
    t_table = time.time() - t0
    k_ext, k_sca = tab.info["sigma_ext_mm2"], tab.info["sigma_sca_mm2"]
    shape = W.plume_shape(P.shape, (LX, LY, LZ), P.sigma_mm, P.center_x_mm)
    gz, gy, gx = P.shape
    rho0 = P.tau_peak / (k_ext * float(np.sum(shape[gz // 2, gy // 2, :].astype(np.float64))) * LX / gx)
    dens = torch.from_numpy(shape).to(dev).mul_(rho0)
    geo = E.Geometry(LX, LY, LZ, 0.0)
    grid = E.Grid(dens, k_ext, k_sca, 0.0, P.block)
    eng = E.Engine(E.Camera(P.nx, P.nz, N_RADIAL, R_MAX), geo, dev)
    med = E.Medium(1.0, 0.0, "table", 0.0, tab)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        tot = 0.0
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    t_prep = timed(lambda: grid.prepare(geo, stream), steps)
    grid.prepare(geo, stream)
    t_walk = timed(lambda: eng.run_grid(grid, med, n, seed=1, stream=stream), max(1, min(steps, 3)))
    eng.check()
    tentative = int(eng.totals[7].item())
    res = eng.result()
    # gradient w.r.t. all 256^3 densities against the forward walk, 1e7 photons
    n_adj = min(10_000_000, n)
    adj = torch.rand((P.nz, P.nx), generator=torch.Generator().manual_seed(1)).to(dev)
    t_fwd_adj = timed(lambda: eng.run_grid(grid, med, n_adj, seed=2, stream=stream), max(1, min(steps, 3)))
    t_adj = timed(lambda: eng.grid_adjoint(grid, med, adj, n_adj, seed=2, stream=stream), max(1, min(steps, 3)))
    t_null = timed(lambda: eng.grid_adjoint(grid, med, adj, n_adj, seed=2, stream=stream, nulls=NULL_MAJORANT_SCALE),
                   max(1, min(steps, 3)))
    eng.check()
    matched = matched_error(eng, grid, med, adj, n_adj, stream, t_adj, t_null)
    # both gradients once at the full photon budget (the kernels are warm)
    def once(fn):
        torch.cuda.synchronize(dev)
        flush.fill_(7)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)
    t_adj_n = once(lambda: eng.grid_adjoint(grid, med, adj, n, seed=2, stream=stream))
    t_null_n = once(lambda: eng.grid_adjoint(grid, med, adj, n, seed=2, stream=stream, nulls=NULL_MAJORANT_SCALE))
    eng.check()
    return {"prepare_ms": t_prep, "walk_ms": t_walk, "photons_per_s": n / (t_walk * 1e-3),
            "density_gradient": {"photons": n_adj, "forward_ms": t_fwd_adj, "gradient_ms": t_adj,
                                 "cost_vs_forward": t_adj / t_fwd_adj,
                                 "null_scores": {"majorant_scale": NULL_MAJORANT_SCALE, "gradient_ms": t_null,
                                                 "cost_vs_forward": t_null / t_fwd_adj},
                                 "matched_error": matched,
                                 "at_budget": {"photons": n, "forward_ms": t_walk, "gradient_ms": t_adj_n,
                                               "cost_vs_forward": t_adj_n / t_walk, "null_scores_ms": t_null_n,
                                               "null_cost_vs_forward": t_null_n / t_walk}},
            "tentative_steps_per_s": tentative / (t_walk * 1e-3), "tentative_steps_per_photon": tentative / n,
            "ballistic_fraction": float(res["totals"][6] / n), "expected_ballistic": math.exp(-P.tau_peak),
            "mixture_table_build_s": t_table, "k_ext_mm2": k_ext, "k_sca_mm2": k_sca, "g": tab.info["g"],
            "grid_bytes": grid.work.numel(),
            "workload": "256^3 Gaussian plume (sigma 5 mm at x=22.5), 16 log-normal size bins (median 5 um, "
                        "sigma_ln 0.3), peak tau 30 on the beam, %d photons, %dx%d image, cells %s" %
                        (n, P.nx, P.nz, "x".join(map(str, P.block)))}


NULL_MAJORANT_SCALE = 1.25


def matched_error(eng, grid, med, adj, n, stream, t_exact, t_null, batches=8):
    """Exact flight lengths against null-collision scores at equal error:
    each estimator's batch-means variance over `batches` photon batches (the
    same n photons in all), of 32^3-voxel block sums and of single voxels,
    times its time per photon; the ratio (nulls / exact) is the cost of the
    null scores at matched error (< 1: they reach an error sooner)."""
    import torch
    nb = n // batches

    def stats(nulls):
        grads = []
        for b in range(batches):
            _, g = eng.grid_adjoint(grid, med, adj, nb, seed=3, photon_offset=b * nb, stream=stream, nulls=nulls)
            grads.append(g.double())
        eng.check()
        G = torch.stack(grads)                       # [batches, gz, gy, gx]
        gz, gy, gx = G.shape[1:]
        B = G.reshape(batches, gz // 32, 32, gy // 32, 32, gx // 32, 32).sum(dim=(2, 4, 6)).flatten(1)
        mean_v, var_v = G.mean(0).flatten(), G.var(0).flatten()
        return B.mean(0), B.var(0), mean_v, var_v

    bm0, bv0, vm0, vv0 = stats(None)
    bm1, bv1, vm1, vv1 = stats(NULL_MAJORANT_SCALE)
    big = bm0.abs() >= bm0.abs().median()            # blocks with at least the median signal
    a = vm0.abs()
    thr = torch.kthvalue(a.cpu(), max(1, int(0.9 * a.numel()))).values.item()
    vsel = (a >= thr) & (a > 0)                      # the 10 % of voxels with the largest gradient
    ratio_b = float(torch.median(bv1[big] / bv0[big].clamp_min(1e-300)))
    ratio_v = float(torch.median(vv1[vsel] / vv0[vsel].clamp_min(1e-300)))
    return {"batches": batches, "photons_per_batch": nb,
            "variance_ratio_blocks": ratio_b, "variance_ratio_voxels": ratio_v,
            "cost_at_matched_error_blocks": ratio_b * t_null / t_exact,
            "cost_at_matched_error_voxels": ratio_v * t_null / t_exact,
            "note": "median over 32^3 blocks with at least the median |block sum|, and over the 10 % of voxels "
                    "with the largest |gradient|, of var(nulls) / var(exact), times the time ratio"}


def adjoint_comparison(E, dev, steps, flush):
    """Adjoint cost against the forward pass on the tau = 5 Mie cuvette with
    1e7 photons and a 128x128 image: mc_run vs mc_adjoint over the same
    photons, with and without the 64 phase-weight gradients."""
    import torch
    table = E.PhaseTable(5.0, 1.59, 1.33, 532.0, 4096)
    med = E.Medium.from_optical_depth(table, TAU, LX)
    eng = E.Engine(E.Camera(128, 128, N_RADIAL, R_MAX), E.Geometry(LX, LY, LZ, 0.0), dev)
    n = 10_000_000
    adj = torch.rand((128, 128), generator=torch.Generator().manual_seed(1)).to(dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        tot = 0.0
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    t_fwd = timed(lambda: eng.run(med, n, seed=1, stream=stream))
    eng.check()
    fwd_steps = eng.result()["steps"]
    t_w = timed(lambda: eng.adjoint(med, adj, n, n_w=64, seed=1, stream=stream))
    t_0 = timed(lambda: eng.adjoint(med, adj, n, n_w=0, seed=1, stream=stream))
    # at phase weights w != 1: the forward pass reweights the table on the
    # device and walks it; the adjoint does the same and evaluates the scores at w
    w = (0.5 + torch.rand(64, generator=torch.Generator().manual_seed(2), dtype=torch.float32)).to(dev)
    t_fwd_w = timed(lambda: eng.run(E.Medium(med.mu_s, med.mu_a, "table", 0.0,
                                             E.WeightedTable(table, w, dev, stream)), n, seed=1, stream=stream))
    t_adj_w = timed(lambda: eng.adjoint(med, adj, n, n_w=64, seed=1, stream=stream, phase_w=w))
    eng.check()
    return {"forward_ms": t_fwd, "forward_steps": fwd_steps, "adjoint_ms": t_w, "adjoint_mu_only_ms": t_0,
            "cost_vs_forward": t_w / t_fwd, "cost_vs_forward_mu_only": t_0 / t_fwd,
            "at_weights": {"forward_ms": t_fwd_w, "adjoint_ms": t_adj_w, "cost_vs_forward": t_adj_w / t_fwd_w},
            "workload": "tau=5 Mie, 1e7 photons, 128x128 image; gradient w.r.t. mu_s, mu_a and 64 "
                        "phase-table weights (one pass; photons with more than 8 scatterings are replayed once) "
                        "or mu_s, mu_a only (one pass); at_weights: 64 weights in [0.5, 1.5), the table "
                        "reweighted on the device in both passes"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    times, steps_total = [], 0
    n = None
    for i in range(args.warmup + args.steps):
        if n is None:
            s, dt, threads = oracle_sample(100_000)
            n = int(min(max(100_000 * 5.0 / max(dt, 1e-3), 100_000), N_PHOTONS))
        s, dt, threads = oracle_sample(n)
        if i >= args.warmup:
            times.append(dt)
            steps_total += s
    value = steps_total / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": _workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "each step: %d photons of the workload on %d threads of %s"
                                       % (n, threads, _cpu_model())},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_engine(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2507_23189_gb300 import build as B
    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    import paper_2507_23189_gb300 as E
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    table = E.PhaseTable(5.0, 1.59, 1.33, 532.0, 4096)
    med = E.Medium.from_optical_depth(table, TAU, LX)
    cam = E.Camera(NX, NZ, N_RADIAL, R_MAX)
    geo = E.Geometry(LX, LY, LZ, 0.0)
    eng = E.Engine(cam, geo, dev)
    offset, _ = photon_range(rank, N_PHOTONS)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        eng.run(med, N_PHOTONS, seed=SEED, photon_offset=offset, stream=stream)

    for _ in range(args.warmup):
        step()
    eng.check()
    steps_per_run = eng.result()["steps"]

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(torch.cuda.current_device() if ws == 1 else local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    # the clocks are read under this load: the sampler's first reading comes
    # a moment after it starts, so the readings taken while the GPU idled are
    # dropped, the same steps run untimed for LOAD_WINDOW_S, and sampling
    # goes on through the timed steps
    clocks.start()
    clocks.wait_first(2.0)
    clocks.lines.clear()
    t_load = time.perf_counter()
    while time.perf_counter() - t_load < LOAD_WINDOW_S:
        step()
        torch.cuda.synchronize(dev)
    barrier()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    barrier()
    clk = clocks.stop()
    if clk is not None:
        clk["window"] = ("%.1f s of the same steps, untimed, then the %d timed steps" %
                         (LOAD_WINDOW_S, args.steps))
    eng.check()
    assert eng.result()["steps"] == steps_per_run
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_local = sum(ms) / 1e3
    value, t_max, total_steps = job_rate(t_local, steps_per_run * args.steps, ws, dev)

    # end to end through the host-buffer entry point: table in, tallies out
    import numpy as np
    e2e = None
    if not args.no_e2e:
        work = torch.empty(E.host_workspace_bytes(med, cam), dtype=torch.uint8, device=dev)
        pinned = lambda shape: torch.zeros(shape, dtype=torch.int64, pin_memory=True).numpy()
        img, rad, tot = pinned((NZ, NX)), pinned(N_RADIAL), pinned(8)
        blob = torch.from_numpy(table.blob).pin_memory().numpy()
        E.run_host(med, geo, cam, N_PHOTONS, work, seed=SEED, photon_offset=offset, image=img,
                   radial=rad, totals=tot, table_host=blob)
        barrier()
        e2e_t = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            E.run_host(med, geo, cam, N_PHOTONS, work, seed=SEED, photon_offset=offset, image=img,
                       radial=rad, totals=tot, table_host=blob)
            e2e_t.append(time.perf_counter() - t0)
        te = torch.tensor([sum(e2e_t)], dtype=torch.float64, device=dev)
        if ws > 1:
            torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
        # the table goes in and image, radial profile, totals and error word come back
        e2e = {"value": total_steps / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": int(blob.nbytes),
               "d2h_bytes_per_step": int(img.nbytes + rad.nbytes + tot.nbytes + 4)}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = sms * LANES_PER_SM * sm_max * 1e6 / 1e12   # T thread-instructions / s
    kernel_s = t_local / args.steps
    roof = None
    if THREAD_INST_PER_STEP:
        ach = THREAD_INST_PER_STEP * steps_per_run / kernel_s / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tinst/s", "frac": ach / peak,
                "traffic": DRAM_BYTES_PER_LAUNCH,
                "per_unit": "%g thread-instructions per photon-step (ncu), peak = %d SMs x %d lanes x "
                            "%.0f MHz" % (THREAD_INST_PER_STEP, sms, LANES_PER_SM, sm_max)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _workload_config(),
            "photons_per_s": ws * N_PHOTONS * args.steps / t_max,
            "steps_per_photon": steps_per_run / N_PHOTONS,
            "e2e": e2e,
            # per step: the walk kernel and the tally sign check after it
            "gpu_launches": 2 * args.steps, "clocks": clk, "roofline": roof}
    if not args.no_batched and ws == 1:
        line["batched"] = batched_comparison(E, dev, args.steps, args.warmup, flush)
        # the same walk loop over the 64 media (optical depths 0.5-20): its
        # place on the issue roofline, from its own instruction count
        ach_b = BATCH_THREAD_INST_PER_STEP * line["batched"]["value"] / 1e12
        line["batched"]["roofline"] = {
            "bound": "alu", "achieved": ach_b, "peak": peak, "unit": "Tinst/s", "frac": ach_b / peak,
            "per_unit": "%g thread-instructions per photon-step (ncu, batch_kernel on this workload), "
                        "peak = %d SMs x %d lanes x %.0f MHz" % (BATCH_THREAD_INST_PER_STEP, sms, LANES_PER_SM,
                                                                 sm_max)}
        line["adjoint"] = adjoint_comparison(E, dev, args.steps, flush)
        line["paper_mode"] = paper_comparison(E, dev, args.steps, flush)
        line["plume"] = plume_leg(E, dev, args.steps, flush)

        def alu_roof(per_unit, units_per_s, what):
            ach = per_unit * units_per_s / 1e12
            return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tinst/s", "frac": ach / peak,
                    "per_unit": "%g thread-instructions per %s (ncu), peak = %d SMs x %d lanes x %.0f MHz"
                                % (per_unit, what, sms, LANES_PER_SM, sm_max)}
        # the adjoint kernels and the plume's delta-tracking walk on the same
        # issue roofline, from their own instruction counts
        a = line["adjoint"]
        a["roofline"] = alu_roof(ADJ_W_THREAD_INST_PER_STEP, a["forward_steps"] / (a["adjoint_ms"] * 1e-3),
                                 "forward photon-step (adjoint_kernel with 64 phase weights)")
        a["roofline_mu_only"] = alu_roof(ADJ_MU_THREAD_INST_PER_STEP,
                                         a["forward_steps"] / (a["adjoint_mu_only_ms"] * 1e-3),
                                         "forward photon-step (adjoint_kernel, mu_s and mu_a only)")
        pl = line["plume"]
        pl["roofline"] = alu_roof(GRID_THREAD_INST_PER_TENTATIVE, pl["tentative_steps_per_s"],
                                  "tentative collision (grid_kernel)")
    if not args.no_peaks:
        from paper_2507_23189_gb300 import peaks
        pk = peaks.measure(dev)
        line["issue_peaks"] = {"unit": "G ops/s (smem: GB/s)", "sms": pk["sms"],
                               **{k: v / 1e9 for k, v in pk.items() if k != "sms"}}
    # the shared-memory pipe: wavefronts per step (ncu) x 128 B at the measured rate
    smem_peak = (pk["smem_bytes"] / 1e12 if not args.no_peaks
                 else sms * SMEM_BYTES_PER_CLK_SM * sm_max * 1e6 / 1e12)
    smem_ach = SMEM_WAVEFRONTS_PER_STEP * SMEM_BYTES_PER_CLK_SM * steps_per_run / kernel_s / 1e12
    line["smem_roofline"] = {"achieved": smem_ach, "peak": smem_peak, "unit": "TB/s", "frac": smem_ach / smem_peak,
                             "peak_kind": "measured" if not args.no_peaks else "nominal",
                             "per_unit": "%g shared-memory wavefronts of 128 B per photon-step (ncu)"
                                         % SMEM_WAVEFRONTS_PER_STEP}
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the issue-rate microbenchmarks")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-launch comparison")
    ap.add_argument("--photons", type=int, default=N_PHOTONS,
                    help="photons per step (default: the workload's 1e8; smaller for profiling)")
    ap.add_argument("--leg", choices=["batched", "adjoint", "paper", "plume"],
                    help="run only this comparison leg and print its JSON (profiling aid)")
    ap.add_argument("--no-tune", action="store_true", help="batched leg: default launch shape, no autotuning")
    ap.add_argument("--plume-photons", type=int, default=None, help="plume leg: photons per walk")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)   # timing rule: at least three warm-up steps
    globals()["N_PHOTONS"] = args.photons
    globals()["NO_TUNE"] = args.no_tune
    if args.impl == "reference":
        return run_reference(args)
    if args.leg:
        return run_leg(args)
    return run_engine(args)


def run_leg(args):
    """One comparison leg on its own, for profiling its kernels."""
    import torch
    from paper_2507_23189_gb300 import build as B
    B.build()
    import paper_2507_23189_gb300 as E
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    if args.leg == "batched":
        out = batched_comparison(E, dev, args.steps, args.warmup, flush)
    elif args.leg == "adjoint":
        out = adjoint_comparison(E, dev, args.steps, flush)
    elif args.leg == "paper":
        out = paper_comparison(E, dev, args.steps, flush)
    else:
        out = plume_leg(E, dev, args.steps, flush, n_photons=args.plume_photons)
    print(json.dumps({"leg": args.leg, **out}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
