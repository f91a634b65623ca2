"""ctypes declarations of the engine's C ABI (include/mcmie.h).

Argument marshalling only: every computation happens in libmcmie.so. Loading
fails loudly if the library has not been built; there is no fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmcmie.so")

MC_OK, MC_NOT_READY = 0, 1
STATUS = {1: "MC_NOT_READY", 0: "MC_OK", -1: "MC_ERR_ARG", -2: "MC_ERR_CUDA", -3: "MC_ERR_NOMEM", -4: "MC_ERR_TIMEOUT",
          -5: "MC_ERR_OVERFLOW", -6: "MC_ERR_NUMERIC", -7: "MC_ERR_EVENTS", -8: "MC_ERR_TABLE",
          -9: "MC_ERR_BOUNDS"}
EFLAG_EVENTS, EFLAG_TIMEOUT, EFLAG_NUMERIC, EFLAG_OVERFLOW, EFLAG_TABLE, EFLAG_BOUNDS = 1, 2, 4, 8, 16, 32
PHASE_TABLE, PHASE_HG, PHASE_PAPER = 0, 1, 2
TOT_REFLECT, TOT_FAR, TOT_SIDE, TOT_ABSORB, TOT_ROULETTE, TOT_TRUNC, TOT_BALLISTIC, TOT_STEPS = range(8)
N_TOTALS = 8
WEIGHT_FRAC_BITS = 32
TRACE_WORDS = 12

# every symbol include/mcmie.h declares
EXPORTS = ("mc_table_bytes", "mie_table_build", "mc_medium_from_density", "mc_workspace_bytes",
           "mc_run", "mc_host_workspace_bytes", "mc_run_host", "mc_trace", "mc_check", "mc_philox",
           "mc_status_string", "mc_run_static", "mc_batch_workspace_bytes", "mc_run_batch",
           "mc_adjoint_workspace_bytes", "mc_adjoint", "mc_paper_table_bytes", "mie_paper_table_build",
           "mc_metrics_out_len", "mc_metrics_workspace_bytes", "mc_image_metrics", "mie_mixture_table_build",
           "mc_grid_workspace_bytes", "mc_grid_prepare", "mc_run_grid", "mc_grid_adjoint_workspace_bytes",
           "mc_grid_adjoint_nulls_workspace_bytes",
           "mc_grid_adjoint", "mc_check_within", "mc_wait_selftest", "mc_medium_from_optical_depth",
           "mc_auto_frac_bits", "mc_phase_table_weighted", "mc_grid_adjoint_nulls")


class McError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (fn, STATUS.get(status, "?"), status))


class MieParams(C.Structure):
    _fields_ = [("diameter_um", C.c_double), ("n_particle_re", C.c_double),
                ("n_particle_im", C.c_double), ("n_medium", C.c_double),
                ("wavelength_nm", C.c_double), ("n_bins", C.c_int)]


class MieInfo(C.Structure):
    _fields_ = [("x", C.c_double), ("m_re", C.c_double), ("m_im", C.c_double),
                ("qext", C.c_double), ("qsca", C.c_double), ("qabs", C.c_double),
                ("g", C.c_double), ("g_table", C.c_double), ("sigma_ext_mm2", C.c_double),
                ("sigma_sca_mm2", C.c_double), ("sigma_abs_mm2", C.c_double), ("nmax", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Grid(C.Structure):
    _fields_ = [("d_density", C.c_void_p), ("gx", C.c_int), ("gy", C.c_int), ("gz", C.c_int),
                ("k_ext", C.c_double), ("k_sca", C.c_double), ("mu_a", C.c_double),
                ("bx", C.c_int), ("by", C.c_int), ("bz", C.c_int)]


class Medium(C.Structure):
    _fields_ = [("mu_s", C.c_double), ("mu_a", C.c_double), ("phase_kind", C.c_int),
                ("hg_g", C.c_double), ("d_table", C.c_void_p), ("n_bins", C.c_int)]


class Geometry(C.Structure):
    _fields_ = [("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("beam_radius", C.c_double)]


class Camera(C.Structure):
    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("n_radial", C.c_int), ("r_max", C.c_double)]


class RunParams(C.Structure):
    _fields_ = [("n_photons", C.c_uint64), ("photon_offset", C.c_uint64), ("seed", C.c_uint64),
                ("rr_threshold", C.c_double), ("rr_survival", C.c_double),
                ("max_events", C.c_uint32), ("max_scatter", C.c_uint32),
                ("image_frac_bits", C.c_int), ("accumulate", C.c_int),
                ("block_size", C.c_int), ("blocks_per_sm", C.c_int), ("image_mode", C.c_int)]


class Instance(C.Structure):
    _fields_ = [("medium", Medium), ("n_photons", C.c_uint64), ("photon_offset", C.c_uint64),
                ("seed", C.c_uint64), ("d_image", C.c_void_p), ("d_radial", C.c_void_p),
                ("d_totals", C.c_void_p)]


class Tallies(C.Structure):
    _fields_ = [("d_image", C.c_void_p), ("d_radial", C.c_void_p), ("d_totals", C.c_void_p),
                ("d_error", C.c_void_p), ("d_work", C.c_void_p), ("work_bytes", C.c_size_t)]


_lib = None


def lib():
    """The loaded engine library. Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = LIB_PATH
    if os.environ.get("MC_CHECKED") == "1":
        # the index-checked build (paper_2507_23189_gb300.build.build_checked())
        path = os.path.join(HERE, "_build", "libmcmie_checked.so")
    elif os.environ.get("MC_STRICT") == "1":
        # the IEEE-strict build (paper_2507_23189_gb300.build.build_strict())
        path = os.path.join(HERE, "_build", "libmcmie_strict.so")
    if not os.path.exists(path):
        raise RuntimeError("engine library %s is missing: run paper_2507_23189_gb300.build.build() "
                           "(or __graft_entry__.build()) first" % path)
    L = C.CDLL(path)
    P = C.POINTER
    vp = C.c_void_p
    L.mc_table_bytes.restype = C.c_size_t
    L.mc_table_bytes.argtypes = [C.c_int]
    L.mie_table_build.restype = C.c_int
    L.mie_table_build.argtypes = [P(MieParams), P(MieInfo), vp, P(C.c_double), P(C.c_double)]
    L.mc_medium_from_density.restype = C.c_int
    L.mc_medium_from_density.argtypes = [P(MieInfo), C.c_double, C.c_double, P(Medium)]
    L.mc_medium_from_optical_depth.restype = C.c_int
    L.mc_medium_from_optical_depth.argtypes = [P(MieInfo), C.c_double, C.c_double, C.c_double, P(Medium),
                                               P(C.c_double)]
    L.mc_auto_frac_bits.restype = C.c_int
    L.mc_auto_frac_bits.argtypes = [C.c_uint64]
    L.mc_workspace_bytes.restype = C.c_size_t
    L.mc_workspace_bytes.argtypes = [P(Camera)]
    L.mc_run.restype = C.c_int
    L.mc_run.argtypes = [P(Medium), P(Geometry), P(Camera), P(RunParams), P(Tallies), vp]
    L.mc_host_workspace_bytes.restype = C.c_size_t
    L.mc_host_workspace_bytes.argtypes = [P(Medium), P(Camera)]
    L.mc_run_host.restype = C.c_int
    L.mc_run_host.argtypes = [P(Medium), vp, P(Geometry), P(Camera), P(RunParams), vp, vp, vp, vp,
                              vp, C.c_size_t, vp]
    L.mc_trace.restype = C.c_int
    L.mc_trace.argtypes = [P(Medium), P(Geometry), P(Camera), P(RunParams), P(Tallies), vp, C.c_int,
                           C.c_int, vp]
    L.mc_check.restype = C.c_int
    L.mc_check.argtypes = [vp, vp]
    L.mc_check_within.restype = C.c_int
    L.mc_check_within.argtypes = [vp, vp, C.c_double]
    L.mc_wait_selftest.restype = C.c_int
    L.mc_wait_selftest.argtypes = [vp, C.c_uint32, vp]
    L.mc_philox.restype = C.c_int
    L.mc_philox.argtypes = [vp, C.c_uint64, C.c_uint64, vp, vp]
    L.mc_run_static.restype = C.c_int
    L.mc_run_static.argtypes = [P(Medium), P(Geometry), P(Camera), P(RunParams), vp, vp, vp, vp, vp]
    L.mc_batch_workspace_bytes.restype = C.c_size_t
    L.mc_batch_workspace_bytes.argtypes = [C.c_int]
    L.mc_run_batch.restype = C.c_int
    L.mc_run_batch.argtypes = [C.c_int, P(Instance), P(Geometry), P(Camera), P(RunParams), C.c_uint64,
                               vp, vp, C.c_size_t, vp]
    L.mc_adjoint_workspace_bytes.restype = C.c_size_t
    L.mc_adjoint_workspace_bytes.argtypes = [C.c_int]
    L.mc_adjoint.restype = C.c_int
    L.mc_adjoint.argtypes = [P(Medium), P(Geometry), P(Camera), P(RunParams), vp, C.c_int, vp, vp, vp, vp,
                             C.c_size_t, vp]
    L.mc_grid_adjoint_nulls.restype = C.c_int
    L.mc_grid_adjoint_nulls.argtypes = [P(Grid), vp, P(Medium), P(Geometry), P(Camera), P(RunParams), vp,
                                        C.c_double, vp, vp, vp, vp, C.c_size_t, vp]
    L.mc_phase_table_weighted.restype = C.c_int
    L.mc_phase_table_weighted.argtypes = [P(Medium), C.c_int, vp, vp, C.c_size_t, vp, vp]
    L.mc_paper_table_bytes.restype = C.c_size_t
    L.mc_paper_table_bytes.argtypes = [C.c_int]
    L.mie_paper_table_build.restype = C.c_int
    L.mie_paper_table_build.argtypes = [P(MieParams), C.c_int, P(MieInfo), vp, P(C.c_double)]
    L.mc_metrics_out_len.restype = C.c_int
    L.mc_metrics_out_len.argtypes = [C.c_int]
    L.mc_metrics_workspace_bytes.restype = C.c_size_t
    L.mc_metrics_workspace_bytes.argtypes = [C.c_int]
    L.mc_image_metrics.restype = C.c_int
    L.mc_image_metrics.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, vp, vp, C.c_size_t, vp]
    L.mie_mixture_table_build.restype = C.c_int
    L.mie_mixture_table_build.argtypes = [P(MieParams), P(C.c_double), C.c_int, P(MieInfo), vp, P(C.c_double),
                                          P(C.c_double)]
    L.mc_grid_workspace_bytes.restype = C.c_size_t
    L.mc_grid_workspace_bytes.argtypes = [P(Grid)]
    L.mc_grid_prepare.restype = C.c_int
    L.mc_grid_prepare.argtypes = [P(Grid), P(Geometry), vp, C.c_size_t, vp]
    L.mc_run_grid.restype = C.c_int
    L.mc_run_grid.argtypes = [P(Grid), vp, P(Medium), P(Geometry), P(Camera), P(RunParams), P(Tallies), vp,
                              C.c_int, C.c_int, vp]
    L.mc_grid_adjoint_workspace_bytes.restype = C.c_size_t
    L.mc_grid_adjoint_workspace_bytes.argtypes = [P(Grid)]
    L.mc_grid_adjoint_nulls_workspace_bytes.restype = C.c_size_t
    L.mc_grid_adjoint_nulls_workspace_bytes.argtypes = [P(Grid)]
    L.mc_grid_adjoint.restype = C.c_int
    L.mc_grid_adjoint.argtypes = [P(Grid), vp, P(Medium), P(Geometry), P(Camera), P(RunParams), vp, vp, vp, vp,
                                  vp, C.c_size_t, vp]
    L.mc_status_string.restype = C.c_char_p
    L.mc_status_string.argtypes = [C.c_int]
    _lib = L
    return L


def check(fn, status):
    if status != MC_OK:
        raise McError(fn, status)
    return status
