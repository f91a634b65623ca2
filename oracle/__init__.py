"""ctypes wrapper of the C oracle.

TEST INFRASTRUCTURE: a plain, slow, double-precision CPU restatement of the
paper's method (arXiv 2507.23189) used to check the CUDA engine. Only the tests,
the smoke check and the benchmark's CPU-baseline leg may import it; the engine
never does. It shares no code with the engine.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.oracle_mie_nmax.restype = C.c_int
        L.oracle_mie_nmax.argtypes = [C.c_double]
        L.oracle_size_parameter.restype = C.c_double
        L.oracle_size_parameter.argtypes = [C.c_double] * 3
        L.oracle_mie_ab.restype = C.c_int
        L.oracle_mie_ab.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, dp, dp]
        L.oracle_mie_efficiencies.restype = C.c_int
        L.oracle_mie_efficiencies.argtypes = [C.c_double] * 3 + [dp] * 3
        L.oracle_mie_s12.restype = C.c_int
        L.oracle_mie_s12.argtypes = [C.c_double] * 3 + [dp, C.c_int, dp, dp]
        L.oracle_mie_phase_raw.restype = C.c_int
        L.oracle_mie_phase_raw.argtypes = [C.c_double] * 3 + [dp, C.c_int, dp]
        L.oracle_cross_section_mm2.restype = C.c_double
        L.oracle_cross_section_mm2.argtypes = [C.c_double] * 2
        L.oracle_optical_depth.restype = C.c_double
        L.oracle_optical_depth.argtypes = [C.c_double] * 3
        L.oracle_phase_table.restype = C.c_int
        L.oracle_phase_table.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_int, C.c_int, dp, dp, dp, dp]
        L.oracle_phase_table_weighted.restype = C.c_int
        L.oracle_phase_table_weighted.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                                                  C.c_double, C.c_int, dp, C.c_int, C.c_int, dp, dp,
                                                  dp, dp]
        L.oracle_phase_table_mixture.restype = C.c_int
        L.oracle_phase_table_mixture.argtypes = [C.c_int, C.POINTER(C.c_int), dp, dp, dp, dp, dp, C.c_int,
                                                 C.c_int, dp, dp, dp, dp]
        L.oracle_grid_adjoint.restype = C.c_int
        L.oracle_grid_adjoint.argtypes = [C.POINTER(WalkCfg), dp, C.c_int, dp, dp]
        L.oracle_grid_adjoint_nulls.restype = C.c_int
        L.oracle_grid_adjoint_nulls.argtypes = [C.POINTER(WalkCfg), dp, C.c_int, dp, dp]
        L.oracle_paper_cdf.restype = C.c_int
        L.oracle_paper_cdf.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                       C.c_int, dp]
        L.oracle_philox4x32_10_n.restype = None
        L.oracle_philox4x32_10_n.argtypes = [C.POINTER(C.c_uint32), C.c_uint64,
                                             C.c_uint64, C.POINTER(C.c_uint32)]
        L.oracle_uniform.restype = C.c_double
        L.oracle_uniform.argtypes = [C.c_uint32]
        L.oracle_walk.restype = C.c_int
        L.oracle_walk.argtypes = [C.POINTER(WalkCfg), C.POINTER(WalkOut),
                                  C.POINTER(TraceRec), C.c_int, C.c_int]
        L.oracle_walk32_trace.restype = C.c_int
        L.oracle_walk32_trace.argtypes = [C.POINTER(WalkCfg), C.POINTER(TraceRec), C.c_int, C.c_int]
        L.oracle_hat.restype = C.c_double
        L.oracle_hat.argtypes = [C.c_int, C.c_int, C.c_double]
        L.oracle_hat_integrals.restype = None
        L.oracle_hat_integrals.argtypes = [dp, C.c_int, C.c_int, dp]
        L.oracle_adjoint.restype = C.c_int
        L.oracle_adjoint.argtypes = [C.POINTER(WalkCfg), dp, C.c_int, dp, dp, dp]
        L.oracle_adjoint_weighted.restype = C.c_int
        L.oracle_adjoint_weighted.argtypes = [C.POINTER(WalkCfg), dp, C.c_int, dp, dp, dp, dp, dp]
        L.oracle_phase_table_reweighted.restype = C.c_int
        L.oracle_phase_table_reweighted.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


PHASE_MIE = 0
PHASE_HG = 1
PHASE_PAPER = 2
N_TOTALS = 8
TOTAL_NAMES = ("reflect", "far", "side", "absorb", "roulette", "trunc", "ballistic", "cone")


class WalkCfg(C.Structure):
    _fields_ = [
        ("mu_s", C.c_double), ("mu_a", C.c_double),
        ("phase_kind", C.c_int), ("hg_g", C.c_double),
        ("icdf", C.POINTER(C.c_double)), ("omu", C.POINTER(C.c_double)),
        ("n_bins", C.c_int),
        ("cdf", C.POINTER(C.c_double)), ("n_theta", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
        ("beam_radius", C.c_double),
        ("nx", C.c_int), ("nz", C.c_int), ("n_radial", C.c_int), ("r_max", C.c_double),
        ("n_photons", C.c_uint64), ("photon_offset", C.c_uint64), ("seed", C.c_uint64),
        ("rr_threshold", C.c_double), ("rr_survival", C.c_double),
        ("max_events", C.c_uint32), ("max_scatter", C.c_uint32),
        ("cone_cos", C.c_double),
        ("n_threads", C.c_int),
        ("density", C.POINTER(C.c_double)),
        ("gx", C.c_int), ("gy", C.c_int), ("gz", C.c_int),
        ("k_ext", C.c_double), ("k_sca", C.c_double),
        ("bx", C.c_int), ("by", C.c_int), ("bz", C.c_int),
        ("majorant_scale", C.c_double), ("trace_nulls", C.c_int),
    ]


class WalkOut(C.Structure):
    _fields_ = [
        ("image", C.POINTER(C.c_double)), ("image_sq", C.POINTER(C.c_double)),
        ("image_hits", C.POINTER(C.c_double)),
        ("radial", C.POINTER(C.c_double)), ("radial_sq", C.POINTER(C.c_double)),
        ("totals", C.c_double * N_TOTALS), ("totals_sq", C.c_double * N_TOTALS),
        ("steps", C.c_uint64), ("capped", C.c_uint64),
    ]


class TraceRec(C.Structure):
    _fields_ = [("status", C.c_double), ("r", C.c_double * 3), ("d", C.c_double * 3),
                ("w", C.c_double), ("nee", C.c_double), ("pix", C.c_double),
                ("nee_bin", C.c_double), ("rad_bin", C.c_double), ("margin", C.c_double)]


TRACE_FIELDS = ["status", "r0", "r1", "r2", "d0", "d1", "d2", "w", "nee", "pix",
                "nee_bin", "rad_bin", "margin"]

# ------------------------------------------------------------------ Mie


def size_parameter(d_um, n_medium, lambda0_nm):
    """Eq. 3 with the in-medium wavelength."""
    return lib().oracle_size_parameter(d_um, n_medium, lambda0_nm)


def nmax(x):
    return lib().oracle_mie_nmax(x)


def mie_ab(m, x, n=None):
    """a_n, b_n (n = 1..N) of Eq. 7-8 as complex arrays."""
    n = nmax(x) if n is None else n
    a = np.zeros(2 * n)
    b = np.zeros(2 * n)
    if lib().oracle_mie_ab(m.real, m.imag, x, n, _dp(a), _dp(b)):
        raise ValueError("oracle_mie_ab: bad arguments")
    return a[0::2] + 1j * a[1::2], b[0::2] + 1j * b[1::2]


def mie_efficiencies(m, x):
    """(Q_ext, Q_sca, g) from the series (Eq. 13 and its companions)."""
    qe, qs, g = C.c_double(), C.c_double(), C.c_double()
    if lib().oracle_mie_efficiencies(m.real, m.imag, x, C.byref(qe), C.byref(qs), C.byref(g)):
        raise ValueError("oracle_mie_efficiencies: bad arguments")
    return qe.value, qs.value, g.value


def mie_s12(m, x, mu):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    s1 = np.zeros(2 * mu.size)
    s2 = np.zeros(2 * mu.size)
    if lib().oracle_mie_s12(m.real, m.imag, x, _dp(mu), mu.size, _dp(s1), _dp(s2)):
        raise ValueError("oracle_mie_s12: bad arguments")
    return s1[0::2] + 1j * s1[1::2], s2[0::2] + 1j * s2[1::2]


def mie_phase_raw(m, x, mu):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    p = np.zeros(mu.size)
    if lib().oracle_mie_phase_raw(m.real, m.imag, x, _dp(mu), mu.size, _dp(p)):
        raise ValueError("oracle_mie_phase_raw: bad arguments")
    return p


def cross_section_mm2(q, d_um):
    return lib().oracle_cross_section_mm2(q, d_um)


def optical_depth(n_per_mm3, sigma_mm2, l_mm):
    return lib().oracle_optical_depth(n_per_mm3, sigma_mm2, l_mm)


# ------------------------------------------------------------------ table


def phase_table(kind, m=1.0 + 0j, x=1.0, hg_g=0.0, n_bins=4096, n_fine=1 << 18):
    """Equal-probability inverse CDF of a phase function.

    Returns dict(icdf, omu, pdf, norm, g_quad, mean, n_fine)."""
    icdf = np.zeros(n_bins + 1)
    omu = np.zeros(n_bins + 1)
    pdf = np.zeros(n_bins)
    diag = np.zeros(4)
    rc = lib().oracle_phase_table(kind, m.real, m.imag, x, hg_g, n_bins, n_fine,
                                  _dp(icdf), _dp(omu), _dp(pdf), _dp(diag))
    if rc:
        raise ValueError("oracle_phase_table: bad arguments")
    return dict(icdf=icdf, omu=omu, pdf=pdf, norm=diag[0], g_quad=diag[1],
                mean=diag[2], n_fine=int(diag[3]))


def phase_table_weighted(m, x, w, n_bins=4096, n_fine=1 << 18):
    """Mie table of p(mu) h_w(mu) / Z(w) with hat weights w (len n_w)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    icdf, omu, pdf, diag = np.zeros(n_bins + 1), np.zeros(n_bins + 1), np.zeros(n_bins), np.zeros(4)
    rc = lib().oracle_phase_table_weighted(PHASE_MIE, m.real, m.imag, x, 0.0, w.size, _dp(w), n_bins,
                                           n_fine, _dp(icdf), _dp(omu), _dp(pdf), _dp(diag))
    if rc:
        raise ValueError("oracle_phase_table_weighted: bad arguments")
    return dict(icdf=icdf, omu=omu, pdf=pdf, norm=diag[0], g_quad=diag[1], mean=diag[2],
                n_fine=int(diag[3]))


def phase_table_reweighted(table, w):
    """The table's own (piecewise-constant) density times h_w = sum_k w_k
    phi_k, renormalised and inverted at the same number of equal-probability
    levels: the phase function p_w = p h_w / Z(w) the phase-weight gradients
    refer to. Returns dict(icdf, omu, pdf, z) with z = Z(w)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    base = np.ascontiguousarray(table["omu"], dtype=np.float64)
    n = base.size - 1
    icdf, omu, pdf, z = np.zeros(n + 1), np.zeros(n + 1), np.zeros(n), C.c_double(0.0)
    if lib().oracle_phase_table_reweighted(_dp(base), n, w.size, _dp(w), _dp(icdf), _dp(omu), _dp(pdf),
                                           C.byref(z)):
        raise ValueError("oracle_phase_table_reweighted: bad arguments")
    return dict(icdf=icdf, omu=omu, pdf=pdf, z=z.value, mean=float(np.mean(1.0 - 0.5 * (omu[:-1] + omu[1:]))))


def phase_table_mixture(components, weights, n_bins=4096, n_fine=1 << 18):
    """Table of a phase-function mixture. components: list of ("mie", m, x)
    or ("hg", g); weights: each component's share of the scattering
    coefficient. Returns the dict of phase_table."""
    n = len(components)
    kind = (C.c_int * n)()
    mre, mim, xs, gs, w = (np.zeros(n) for _ in range(5))
    for i, comp in enumerate(components):
        if comp[0] == "mie":
            kind[i] = PHASE_MIE
            mre[i], mim[i], xs[i] = comp[1].real, comp[1].imag, comp[2]
        else:
            kind[i] = PHASE_HG
            gs[i] = comp[1]
        w[i] = weights[i]
    icdf, omu, pdf, diag = np.zeros(n_bins + 1), np.zeros(n_bins + 1), np.zeros(n_bins), np.zeros(4)
    if lib().oracle_phase_table_mixture(n, kind, _dp(mre), _dp(mim), _dp(xs), _dp(gs), _dp(w), n_bins,
                                        n_fine, _dp(icdf), _dp(omu), _dp(pdf), _dp(diag)):
        raise ValueError("oracle_phase_table_mixture: bad arguments")
    return dict(icdf=icdf, omu=omu, pdf=pdf, norm=diag[0], g_quad=diag[1], mean=diag[2],
                n_fine=int(diag[3]))


def paper_cdf(kind, m=1.0 + 0j, x=1.0, hg_g=0.0, n_theta=3000):
    """The paper's sampling table (Sec. 3.1.2): cumulative probability at the
    angles theta_i = i pi / (n_theta - 1). Returns dict(cdf, theta)."""
    cdf = np.zeros(n_theta)
    if lib().oracle_paper_cdf(kind, m.real, m.imag, x, hg_g, n_theta, _dp(cdf)):
        raise ValueError("oracle_paper_cdf: bad arguments")
    return dict(cdf=cdf, theta=np.arange(n_theta) * (np.pi / (n_theta - 1)))


# ------------------------------------------------------------------ philox


def philox4x32_10(ctr, seed):
    """ctr: (n, 4) uint32 counters -> (n, 4) uint32 outputs under key = seed."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    lib().oracle_philox4x32_10_n(ctr.ctypes.data_as(C.POINTER(C.c_uint32)), ctr.shape[0],
                                 seed, out.ctypes.data_as(C.POINTER(C.c_uint32)))
    return out


def uniform(r):
    return lib().oracle_uniform(int(r))


# ------------------------------------------------------------------ walk


def hat_integrals(table, n_w=64):
    """Z_k = int p(mu) phi_k(mu) dmu for the tabulated density."""
    omu = np.ascontiguousarray(table["omu"], dtype=np.float64)
    z = np.zeros(n_w)
    lib().oracle_hat_integrals(_dp(omu), omu.size - 1, n_w, _dp(z))
    return z


def hat(n_w, k, mu):
    return lib().oracle_hat(n_w, k, mu)


def adjoint(adj, n_w=64, w=None, base_table=None, **walk_kw):
    """Gradient of sum(adj * image) w.r.t. (mu_s, mu_a, w_0..w_{n_w-1}):
    dict(grad, grad_sq (per-photon squares), value). Same keywords as walk().
    At w = 1 (w None) the walk's table is the phase function itself; at other
    weights walk_kw["table"] is phase_table_reweighted(base_table, w)."""
    cfg, keep = _walk_cfg(**walk_kw)
    a = np.ascontiguousarray(adj, dtype=np.float64).ravel()
    if a.size != cfg.nx * cfg.nz:
        raise ValueError("adjoint image has the wrong size")
    g = np.zeros(2 + n_w)
    g2 = np.zeros(2 + n_w)
    v = C.c_double(0.0)
    if w is None:
        rc = lib().oracle_adjoint(C.byref(cfg), _dp(a), n_w, _dp(g), _dp(g2), C.byref(v))
    else:
        wv = np.ascontiguousarray(w, dtype=np.float64)
        base = np.ascontiguousarray(base_table["omu"], dtype=np.float64)
        if wv.size != n_w or base.size != cfg.n_bins + 1:
            raise ValueError("weights or base table of the wrong size")
        rc = lib().oracle_adjoint_weighted(C.byref(cfg), _dp(a), n_w, _dp(wv), _dp(base), _dp(g), _dp(g2),
                                           C.byref(v))
    if rc:
        raise ValueError("oracle_adjoint: bad arguments")
    return dict(grad=g, grad_sq=g2, value=v.value, n_photons=cfg.n_photons)


def grid_adjoint(adj, max_events=512, nulls=False, **walk_kw):
    """Gradient of sum(adj * image) w.r.t. the voxel densities of
    walk_kw["grid"]["density"]: dict(grad [gz, gy, gx], value). nulls: score
    the flights' transmission at the null collisions of delta tracking
    against majorants grid["majorant_scale"] (> 1) times the cell maxima."""
    cfg, keep = _walk_cfg(**walk_kw)
    a = np.ascontiguousarray(adj, dtype=np.float64).ravel()
    if a.size != cfg.nx * cfg.nz or not cfg.density:
        raise ValueError("adjoint image size or grid missing")
    g = np.zeros(cfg.gz * cfg.gy * cfg.gx)
    v = C.c_double(0.0)
    fn = lib().oracle_grid_adjoint_nulls if nulls else lib().oracle_grid_adjoint
    if fn(C.byref(cfg), _dp(a), max_events, _dp(g), C.byref(v)):
        raise ValueError("oracle_grid_adjoint failed (arguments, or a photon with more real events than "
                         "max_events)")
    return dict(grad=g.reshape(cfg.gz, cfg.gy, cfg.gx), value=v.value)


def _walk_cfg(mu_s, mu_a=0.0, phase="mie", table=None, hg_g=0.0,
              lx=45.0, ly=10.0, lz=10.0, beam_radius=0.0,
              nx=64, nz=64, n_radial=128, r_max=5.0 * 2 ** 0.5,
              n_photons=1000, photon_offset=0, seed=1,
              rr_threshold=1e-4, rr_survival=0.1, max_events=1_000_000, max_scatter=0,
              cone_cos=0.0, n_threads=None, grid=None):
    cfg = WalkCfg()
    cfg.mu_s, cfg.mu_a = mu_s, mu_a
    keep = []
    if phase == "mie":
        icdf = np.ascontiguousarray(table["icdf"], dtype=np.float64)
        omu = np.ascontiguousarray(table["omu"], dtype=np.float64)
        keep += [icdf, omu]
        cfg.phase_kind = PHASE_MIE
        cfg.icdf, cfg.omu = _dp(icdf), _dp(omu)
        cfg.n_bins = icdf.size - 1
    elif phase == "hg":
        cfg.phase_kind = PHASE_HG
        cfg.hg_g = hg_g
    elif phase == "paper":
        cdf = np.ascontiguousarray(table["cdf"], dtype=np.float64)
        keep += [cdf]
        cfg.phase_kind = PHASE_PAPER
        cfg.cdf, cfg.n_theta = _dp(cdf), cdf.size
    else:
        raise ValueError(phase)
    cfg.lx, cfg.ly, cfg.lz, cfg.beam_radius = lx, ly, lz, beam_radius
    cfg.nx, cfg.nz, cfg.n_radial, cfg.r_max = nx, nz, n_radial, r_max
    cfg.n_photons, cfg.photon_offset, cfg.seed = n_photons, photon_offset, seed
    cfg.rr_threshold, cfg.rr_survival = rr_threshold, rr_survival
    cfg.max_events, cfg.max_scatter = max_events, max_scatter
    cfg.cone_cos = cone_cos
    cfg.n_threads = n_threads if n_threads else (os.cpu_count() or 1)
    if grid is not None:
        # dict(density [gz, gy, gx] per mm^3, k_ext, k_sca, block=(bx, by, bz));
        # mu_a is then a uniform background absorption and mu_s is unused
        dens = np.ascontiguousarray(grid["density"], dtype=np.float64)
        keep.append(dens)
        cfg.density = _dp(dens)
        cfg.gz, cfg.gy, cfg.gx = dens.shape
        cfg.k_ext, cfg.k_sca = grid["k_ext"], grid["k_sca"]
        cfg.bx, cfg.by, cfg.bz = grid.get("block", (1, 1, 1))
        cfg.majorant_scale = float(grid.get("majorant_scale", 1.0))
    cfg._keep = keep
    return cfg, keep


def walk32_trace(mu_s, mu_a=0.0, phase="mie", table=None, hg_g=0.0,
                 lx=45.0, ly=10.0, lz=10.0, beam_radius=0.0,
                 nx=64, nz=64, n_radial=128, r_max=5.0 * 2 ** 0.5,
                 n_trace=1000, photon_offset=0, seed=1,
                 rr_threshold=1e-4, rr_survival=0.1, max_events=1_000_000, max_scatter=0,
                 n_trace_events=32):
    """The walk in single precision with explicit fused multiply-adds (the
    oracle's FP32 mode): traces of the first n_trace_events events of photons
    photon_offset .. + n_trace - 1, in the record layout of walk()'s trace.
    Homogeneous medium; phase "mie" (equal-probability table) or "hg"."""
    cfg, keep = _walk_cfg(mu_s, mu_a, phase, table, hg_g, lx, ly, lz, beam_radius, nx, nz, n_radial,
                          r_max, n_trace, photon_offset, seed, rr_threshold, rr_survival, max_events,
                          max_scatter, 0.0, 1, None)
    trace = (TraceRec * (n_trace * n_trace_events))()
    rc = lib().oracle_walk32_trace(C.byref(cfg), C.cast(trace, C.POINTER(TraceRec)), n_trace, n_trace_events)
    if rc:
        raise ValueError("oracle_walk32_trace: bad arguments")
    return np.frombuffer(trace, dtype=np.float64).reshape(n_trace, n_trace_events, 13).copy()


def walk(mu_s, mu_a=0.0, phase="mie", table=None, hg_g=0.0,
         lx=45.0, ly=10.0, lz=10.0, beam_radius=0.0,
         nx=64, nz=64, n_radial=128, r_max=5.0 * 2 ** 0.5,
         n_photons=1000, photon_offset=0, seed=1,
         rr_threshold=1e-4, rr_survival=0.1, max_events=1_000_000, max_scatter=0,
         cone_cos=0.0, n_threads=None, n_trace=0, n_trace_events=32, grid=None):
    """Run the double-precision walk; returns a dict of tallies (and trace).
    phase: "mie" (equal-probability table), "hg" or "paper" (the table of
    paper_cdf, sampled by binary search)."""
    cfg, keep = _walk_cfg(mu_s, mu_a, phase, table, hg_g, lx, ly, lz, beam_radius, nx, nz, n_radial,
                          r_max, n_photons, photon_offset, seed, rr_threshold, rr_survival, max_events,
                          max_scatter, cone_cos, n_threads, grid)
    image = np.zeros(nz * nx)
    image_sq = np.zeros(nz * nx)
    image_hits = np.zeros(nz * nx)
    radial = np.zeros(n_radial)
    radial_sq = np.zeros(n_radial)
    out = WalkOut()
    out.image, out.image_sq, out.image_hits = _dp(image), _dp(image_sq), _dp(image_hits)
    out.radial, out.radial_sq = _dp(radial), _dp(radial_sq)
    trace = None
    tptr = None
    if n_trace:
        trace = (TraceRec * (n_trace * n_trace_events))()
        tptr = C.cast(trace, C.POINTER(TraceRec))
    rc = lib().oracle_walk(C.byref(cfg), C.byref(out), tptr, n_trace, n_trace_events)
    if rc:
        raise ValueError("oracle_walk: bad arguments")
    res = dict(image=image.reshape(nz, nx), image_sq=image_sq.reshape(nz, nx),
               image_hits=image_hits.reshape(nz, nx),
               radial=radial, radial_sq=radial_sq,
               totals=np.array(out.totals[:]), totals_sq=np.array(out.totals_sq[:]),
               steps=int(out.steps), capped=int(out.capped), n_photons=n_photons)
    if n_trace:
        arr = np.frombuffer(trace, dtype=np.float64).reshape(n_trace, n_trace_events, 13).copy()
        res["trace"] = arr
    return res
