"""Python face of the engine: PyTorch holds the device memory and streams;
every step of the walk runs in libmcmie.so through the C ABI.

    table = PhaseTable(diameter_um=5.0, n_particle=1.59, n_medium=1.33, wavelength_nm=532.0)
    med = Medium.from_optical_depth(table, tau=5.0, length_mm=45.0)
    eng = Engine(Camera(256, 256), Geometry())
    eng.run(med, n_photons=10**8, seed=1)
    out = eng.result()          # image/radial/totals as float64 weight units
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _native as N


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _clear_error(error, stream):
    """The error word holds the flags raised since the previous check: a
    check reads it once the stream has finished and then clears it on that
    stream, so the runs themselves add no device work for it."""
    torch = _torch()
    with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream(error.device)):
        error.zero_()


# --------------------------------------------------------------------- table


class PhaseTable:
    """Lorenz-Mie phase table built on the host in double precision
    (mie_table_build), with a cached device copy of the packed blob."""

    def __init__(self, diameter_um=5.0, n_particle=1.59 + 0j, n_medium=1.33, wavelength_nm=532.0,
                 n_bins=4096):
        L = N.lib()
        n_particle = complex(n_particle)
        p = N.MieParams(diameter_um, n_particle.real, n_particle.imag, n_medium, wavelength_nm, n_bins)
        info = N.MieInfo()
        nbytes = L.mc_table_bytes(n_bins)
        if nbytes == 0:
            raise N.McError("mc_table_bytes", -1)
        self.blob = np.zeros(nbytes, dtype=np.uint8)
        self.omu64 = np.zeros(n_bins + 1)
        self.pdf64 = np.zeros(n_bins)
        dp = C.POINTER(C.c_double)
        N.check("mie_table_build", L.mie_table_build(
            C.byref(p), C.byref(info), self.blob.ctypes.data_as(C.c_void_p),
            self.omu64.ctypes.data_as(dp), self.pdf64.ctypes.data_as(dp)))
        self.params = dict(diameter_um=diameter_um, n_particle=n_particle, n_medium=n_medium,
                           wavelength_nm=wavelength_nm, n_bins=n_bins)
        self.info = info.as_dict()
        self.n_bins = n_bins
        self._dev = {}

    @property
    def icdf64(self):
        return 1.0 - self.omu64

    def device_blob(self, device=None):
        torch = _torch()
        dev = torch.device(device if device is not None else "cuda")
        key = str(dev)
        if key not in self._dev:
            self._dev[key] = torch.from_numpy(self.blob).to(dev)
        return self._dev[key]


class MixtureTable(PhaseTable):
    """Phase table of a particle mixture (mie_mixture_table_build), e.g. the
    size bins of a polydisperse sample with number fractions; info holds the
    number-averaged cross sections (sigma_ext_mm2, ...) of one particle."""

    def __init__(self, diameters_um, number_frac, n_particle=1.59 + 0j, n_medium=1.33, wavelength_nm=532.0,
                 n_bins=4096):
        L = N.lib()
        n_particle = complex(n_particle)
        d = [float(v) for v in diameters_um]
        k = len(d)
        ps = (N.MieParams * k)(*[N.MieParams(di, n_particle.real, n_particle.imag, n_medium, wavelength_nm,
                                             n_bins) for di in d])
        f = np.ascontiguousarray(number_frac, dtype=np.float64)
        if f.size != k:
            raise ValueError("one number fraction per diameter")
        info = N.MieInfo()
        nbytes = L.mc_table_bytes(n_bins)
        if nbytes == 0:
            raise N.McError("mc_table_bytes", -1)
        self.blob = np.zeros(nbytes, dtype=np.uint8)
        self.omu64 = np.zeros(n_bins + 1)
        self.pdf64 = np.zeros(n_bins)
        dp = C.POINTER(C.c_double)
        N.check("mie_mixture_table_build", L.mie_mixture_table_build(
            ps, f.ctypes.data_as(dp), k, C.byref(info), self.blob.ctypes.data_as(C.c_void_p),
            self.omu64.ctypes.data_as(dp), self.pdf64.ctypes.data_as(dp)))
        self.params = dict(diameters_um=d, number_frac=list(f), n_particle=n_particle, n_medium=n_medium,
                           wavelength_nm=wavelength_nm, n_bins=n_bins, diameter_um=d[0])
        self.info = info.as_dict()
        self.n_bins = n_bins
        self._dev = {}


class WeightedTable:
    """A phase table reweighted by positive hat-function weights,
    p_w = p h_w / Z(w), built on the device by mc_phase_table_weighted from
    `base` (a PhaseTable) and the weights (a CUDA tensor of n_w values,
    kept as float32; nothing is copied to the host). Use it as a Medium's
    table: the walk then samples p_w and uses it as the camera density."""

    def __init__(self, base, phase_w, device=None, stream=None):
        torch = _torch()
        dev = torch.device(device if device is not None else "cuda")
        self.base = base
        self.n_bins = base.n_bins
        self.info = base.info
        self.phase_w = phase_w.detach().to(device=dev, dtype=torch.float32).contiguous()
        L = N.lib()
        nbytes = L.mc_table_bytes(base.n_bins)
        self._blob = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.error = torch.zeros(1, dtype=torch.int32, device=dev)
        m = N.Medium()
        m.mu_s, m.phase_kind, m.n_bins = 1.0, N.PHASE_TABLE, base.n_bins
        base_blob = base.device_blob(dev)
        m.d_table = base_blob.data_ptr()
        N.check("mc_phase_table_weighted", L.mc_phase_table_weighted(
            C.byref(m), int(self.phase_w.numel()), C.c_void_p(self.phase_w.data_ptr()),
            C.c_void_p(self._blob.data_ptr()), nbytes, C.c_void_p(self.error.data_ptr()),
            _stream_handle(stream)))
        self._keep = base_blob

    def device_blob(self, device=None):
        return self._blob

    def check(self, stream=None):
        """Raise if the weights were rejected (mc_check of the build's word)."""
        N.check("mc_phase_table_weighted", N.lib().mc_check(C.c_void_p(self.error.data_ptr()),
                                                            _stream_handle(stream)))


class PaperTable:
    """The paper's own sampling table (Sec. 3.1.2, mie_paper_table_build):
    the Mie phase function at n_theta equally spaced angles, its cumulative
    distribution, sampled by bisection; with a cached device copy."""

    def __init__(self, diameter_um=5.0, n_particle=1.59 + 0j, n_medium=1.33, wavelength_nm=532.0,
                 n_theta=3000):
        L = N.lib()
        n_particle = complex(n_particle)
        p = N.MieParams(diameter_um, n_particle.real, n_particle.imag, n_medium, wavelength_nm, 0)
        info = N.MieInfo()
        nbytes = L.mc_paper_table_bytes(n_theta)
        if nbytes == 0:
            raise N.McError("mc_paper_table_bytes", -1)
        self.blob = np.zeros(nbytes, dtype=np.uint8)
        self.cdf64 = np.zeros(n_theta)
        N.check("mie_paper_table_build", L.mie_paper_table_build(
            C.byref(p), n_theta, C.byref(info), self.blob.ctypes.data_as(C.c_void_p),
            self.cdf64.ctypes.data_as(C.POINTER(C.c_double))))
        self.params = dict(diameter_um=diameter_um, n_particle=n_particle, n_medium=n_medium,
                           wavelength_nm=wavelength_nm, n_theta=n_theta)
        self.info = info.as_dict()
        self.n_bins = n_theta        # the medium's n_bins field carries n_theta
        self._dev = {}

    device_blob = PhaseTable.device_blob


# -------------------------------------------------------------------- medium


@dataclass
class Medium:
    mu_s: float
    mu_a: float = 0.0
    phase: str = "table"   # "table" (Mie inverse CDF), "hg" or "paper" (PaperTable)
    hg_g: float = 0.0
    table: PhaseTable = None

    @classmethod
    def from_density(cls, table, number_density_per_mm3, mu_a_medium=0.0, phase="table", hg_g=None):
        """Eq. 17: coefficients from number density and the Mie cross sections."""
        info = N.MieInfo(**{k: table.info[k] for k, _ in N.MieInfo._fields_})
        m = N.Medium()
        N.check("mc_medium_from_density", N.lib().mc_medium_from_density(
            C.byref(info), number_density_per_mm3, mu_a_medium, C.byref(m)))
        g = table.info["g"] if hg_g is None else hg_g
        return cls(m.mu_s, m.mu_a, phase, g, table)

    @classmethod
    def from_optical_depth(cls, table, tau, length_mm=45.0, mu_a_medium=0.0, phase="table", hg_g=None):
        """Number density giving optical depth tau over length_mm (Eq. 17,
        mc_medium_from_optical_depth)."""
        info = N.MieInfo(**{k: table.info[k] for k, _ in N.MieInfo._fields_})
        m = N.Medium()
        nd = C.c_double(0.0)
        N.check("mc_medium_from_optical_depth", N.lib().mc_medium_from_optical_depth(
            C.byref(info), float(tau), float(length_mm), float(mu_a_medium), C.byref(m), C.byref(nd)))
        g = table.info["g"] if hg_g is None else hg_g
        med = cls(m.mu_s, m.mu_a, phase, g, table)
        med.number_density = nd.value
        return med

    def as_c(self, device=None):
        m = N.Medium()
        m.mu_s, m.mu_a = self.mu_s, self.mu_a
        if self.phase == "table":
            m.phase_kind = N.PHASE_TABLE
            blob = self.table.device_blob(device)
            m.d_table = blob.data_ptr()
            m.n_bins = self.table.n_bins
            return m, blob
        if self.phase == "hg":
            m.phase_kind = N.PHASE_HG
            m.hg_g = self.hg_g
            return m, None
        if self.phase == "paper":
            if not isinstance(self.table, PaperTable):
                raise ValueError("phase 'paper' needs a PaperTable")
            m.phase_kind = N.PHASE_PAPER
            blob = self.table.device_blob(device)
            m.d_table = blob.data_ptr()
            m.n_bins = self.table.n_bins
            return m, blob
        raise ValueError("phase must be 'table', 'hg' or 'paper'")


@dataclass
class Geometry:
    lx: float = 45.0
    ly: float = 10.0
    lz: float = 10.0
    beam_radius: float = 0.0

    def as_c(self):
        return N.Geometry(self.lx, self.ly, self.lz, self.beam_radius)


@dataclass
class Camera:
    nx: int = 64
    nz: int = 64
    n_radial: int = 128
    r_max: float = 5.0 * 2 ** 0.5

    def as_c(self):
        return N.Camera(self.nx, self.nz, self.n_radial, self.r_max)


def wait_selftest(tries=4096, device=None, stream=None):
    """The kernels' bounded wait on an mbarrier phase that cannot complete
    (mc_wait_selftest); returns mc_check's status afterwards, which is
    MC_ERR_TIMEOUT (-4) when the wait gave up as it must."""
    torch = _torch()
    err = torch.zeros(1, dtype=torch.int32, device=device if device is not None else "cuda")
    N.check("mc_wait_selftest", N.lib().mc_wait_selftest(C.c_void_p(err.data_ptr()), int(tries),
                                                         _stream_handle(stream)))
    return N.lib().mc_check(C.c_void_p(err.data_ptr()), _stream_handle(stream))


def auto_frac_bits(n_photons):
    """Image fraction bits the library picks for a photon budget
    (mc_auto_frac_bits): 32 up to 2^22 photons, 27 at 1e8, 24 at 1e9."""
    return int(N.lib().mc_auto_frac_bits(int(n_photons)))


def run_params(n_photons, seed=1, photon_offset=0, rr_threshold=1e-4, rr_survival=0.1,
               max_events=1_000_000, max_scatter=0, image_frac_bits=0, accumulate=False,
               block_size=0, blocks_per_sm=0, image_mode=0):
    return N.RunParams(int(n_photons), int(photon_offset), int(seed), rr_threshold, rr_survival,
                       int(max_events), int(max_scatter), int(image_frac_bits), int(bool(accumulate)),
                       int(block_size), int(blocks_per_sm), int(image_mode))


class Grid:
    """A heterogeneous medium: particle number density per voxel (float32
    CUDA tensor [gz, gy, gx], per mm^3) with per-particle cross sections
    k_ext, k_sca (mm^2), a uniform background absorption mu_a and majorant
    cells of block = (bx, by, bz) voxels. prepare() builds the device
    workspace mc_run_grid reads (redo it after changing the density)."""

    def __init__(self, density, k_ext, k_sca, mu_a=0.0, block=(8, 16, 16)):
        torch = _torch()
        if density.dtype != torch.float32 or not density.is_cuda or density.dim() != 3:
            raise ValueError("density must be a 3-d float32 CUDA tensor [gz, gy, gx]")
        self.density = density.contiguous()
        self.k_ext, self.k_sca, self.mu_a = float(k_ext), float(k_sca), float(mu_a)
        self.block = tuple(int(b) for b in block)
        g = self.as_c()
        nbytes = N.lib().mc_grid_workspace_bytes(C.byref(g))
        if nbytes == 0:
            raise ValueError("invalid grid (sizes, cross sections or more than 16384 majorant cells)")
        self.work = torch.empty(nbytes, dtype=torch.uint8, device=self.density.device)

    def as_c(self):
        gz, gy, gx = self.density.shape
        return N.Grid(self.density.data_ptr(), gx, gy, gz, self.k_ext, self.k_sca, self.mu_a, *self.block)

    def prepare(self, geometry, stream=None):
        g, geo = self.as_c(), geometry.as_c()
        N.check("mc_grid_prepare", N.lib().mc_grid_prepare(C.byref(g), C.byref(geo),
                                                           C.c_void_p(self.work.data_ptr()), self.work.numel(),
                                                           _stream_handle(stream)))
        return self


# -------------------------------------------------------------------- engine


class Engine:
    """Device tallies for one camera/geometry; runs photon batches into them."""

    def __init__(self, camera=None, geometry=None, device=None):
        torch = _torch()
        self.camera = camera or Camera()
        self.geometry = geometry or Geometry()
        self.device = torch.device(device if device is not None else "cuda")
        cam = self.camera
        L = N.lib()
        wb = L.mc_workspace_bytes(C.byref(cam.as_c()))
        if wb == 0:
            raise N.McError("mc_workspace_bytes", -1)
        dev = self.device
        self.image = torch.zeros((cam.nz, cam.nx), dtype=torch.int64, device=dev)
        self.radial = torch.zeros(cam.n_radial, dtype=torch.int64, device=dev)
        self.totals = torch.zeros(N.N_TOTALS, dtype=torch.int64, device=dev)
        self.error = torch.zeros(1, dtype=torch.int32, device=dev)
        self.work = torch.zeros(wb, dtype=torch.uint8, device=dev)
        self.image_frac_bits = 32
        self.last_error = 0

    def _frac_bits(self, n_photons, kw):
        """kw with an explicit image_frac_bits: the caller's, else the one of
        the tallies being added to (accumulate), else the budget's own."""
        f = kw.get("image_frac_bits")
        if not f:
            f = self.image_frac_bits if kw.get("accumulate") else auto_frac_bits(n_photons)
        self.image_frac_bits = int(f)
        return dict(kw, image_frac_bits=int(f))

    def _tallies(self):
        return N.Tallies(self.image.data_ptr(), self.radial.data_ptr(), self.totals.data_ptr(),
                         self.error.data_ptr(), self.work.data_ptr(), self.work.numel())

    def run(self, medium, n_photons, seed=1, stream=None, **kw):
        """Queue photons on the stream (asynchronous). Without accumulate=True
        the tallies start afresh; check() reports the device flags raised
        since the previous check."""
        rp = run_params(n_photons, seed, **self._frac_bits(n_photons, kw))
        m, keep = medium.as_c(self.device)
        g, c, t = self.geometry.as_c(), self.camera.as_c(), self._tallies()
        N.check("mc_run", N.lib().mc_run(C.byref(m), C.byref(g), C.byref(c), C.byref(rp), C.byref(t),
                                         _stream_handle(stream)))
        self._keep = keep
        return self

    def trace(self, medium, n_photons, n_trace, n_events=32, seed=1, stream=None, **kw):
        """Run with a per-event trace of the first n_trace photons; returns
        an int32 tensor [n_trace, n_events, 12] (float fields bit-cast)."""
        torch = _torch()
        rp = run_params(n_photons, seed, **self._frac_bits(n_photons, kw))
        m, keep = medium.as_c(self.device)
        buf = torch.empty((n_trace, n_events, N.TRACE_WORDS), dtype=torch.int32, device=self.device)
        g, c, t = self.geometry.as_c(), self.camera.as_c(), self._tallies()
        N.check("mc_trace", N.lib().mc_trace(C.byref(m), C.byref(g), C.byref(c), C.byref(rp),
                                             C.byref(t), C.c_void_p(buf.data_ptr()), n_trace, n_events,
                                             _stream_handle(stream)))
        self._keep = keep
        return buf

    def adjoint(self, medium, adj_image, n_photons, n_w=64, seed=1, stream=None, phase_w=None, **kw):
        """(L, dL/dmu_s, dL/dmu_a, dL/dw_0..) for L = sum(adj_image * image)
        as a float64 device tensor (mc_adjoint). medium: the unweighted
        table; phase_w (a tensor of n_w positive weights, or None for w = 1):
        the gradient at those weights, on the photons run() simulates with
        WeightedTable(medium.table, phase_w). adj_image: [nz, nx] in weight
        units per image unit."""
        torch = _torch()
        rp = run_params(n_photons, seed, **kw)
        m, keep = medium.as_c(self.device)
        wdev = None
        if phase_w is not None:
            wdev = phase_w.detach().to(device=self.device, dtype=torch.float32).contiguous()
            if wdev.numel() != n_w:
                raise ValueError("phase_w must hold n_w weights")
        adj = adj_image.to(device=self.device, dtype=torch.float32).contiguous()
        if tuple(adj.shape) != (self.camera.nz, self.camera.nx):
            raise ValueError("adjoint image must be [nz, nx]")
        wb = N.lib().mc_adjoint_workspace_bytes(n_w)
        if wb == 0:
            raise N.McError("mc_adjoint_workspace_bytes", -1)
        if getattr(self, "_adj_work", None) is None or self._adj_work.numel() < wb:
            self._adj_work = torch.empty(wb, dtype=torch.uint8, device=self.device)
        out = torch.empty(3 + n_w, dtype=torch.float64, device=self.device)
        g, c = self.geometry.as_c(), self.camera.as_c()
        N.check("mc_adjoint", N.lib().mc_adjoint(
            C.byref(m), C.byref(g), C.byref(c), C.byref(rp), C.c_void_p(adj.data_ptr()), n_w,
            C.c_void_p(wdev.data_ptr()) if wdev is not None else None,
            C.c_void_p(out.data_ptr()), C.c_void_p(self.error.data_ptr()),
            C.c_void_p(self._adj_work.data_ptr()), self._adj_work.numel(), _stream_handle(stream)))
        self._keep = (keep, adj, wdev)
        return out

    def run_grid(self, grid, phase, n_photons, seed=1, stream=None, n_trace=0, n_events=32, **kw):
        """Delta-tracking walk through a prepared Grid; `phase` is a Medium
        whose phase function is used (its mu_s, mu_a are ignored). With
        n_trace > 0 returns the raw trace of real events (decode_trace)."""
        torch = _torch()
        rp = run_params(n_photons, seed, **self._frac_bits(n_photons, kw))
        m, keep = phase.as_c(self.device)
        m.mu_s, m.mu_a = 1.0, 0.0
        g, geo, c, t = grid.as_c(), self.geometry.as_c(), self.camera.as_c(), self._tallies()
        tr = None
        if n_trace:
            tr = torch.empty(n_trace * n_events * N.TRACE_WORDS, dtype=torch.int32, device=self.device)
        N.check("mc_run_grid", N.lib().mc_run_grid(
            C.byref(g), C.c_void_p(grid.work.data_ptr()), C.byref(m), C.byref(geo), C.byref(c), C.byref(rp),
            C.byref(t), C.c_void_p(tr.data_ptr()) if tr is not None else None, n_trace, n_events,
            _stream_handle(stream)))
        self._keep = (keep, grid)
        if tr is not None:
            return tr.view(n_trace, n_events, N.TRACE_WORDS)
        return self

    def grid_adjoint(self, grid, phase, adj_image, n_photons, seed=1, stream=None, nulls=None, **kw):
        """Gradient of sum(adj_image * image) w.r.t. the voxel densities of a
        prepared Grid (mc_grid_adjoint) on the photons run_grid would use.
        nulls: a majorant scale > 1 to score the flights' transmission at
        null collisions instead (mc_grid_adjoint_nulls). Returns (value
        tensor [1] float64, grad tensor [gz, gy, gx] float32), both on the
        device; check() afterwards for device errors."""
        torch = _torch()
        rp = run_params(n_photons, seed, **kw)
        m, keep = phase.as_c(self.device)
        m.mu_s, m.mu_a = 1.0, 0.0
        adj = adj_image.to(device=self.device, dtype=torch.float32).contiguous()
        if tuple(adj.shape) != (self.camera.nz, self.camera.nx):
            raise ValueError("adjoint image must be [nz, nx]")
        g, geo, c = grid.as_c(), self.geometry.as_c(), self.camera.as_c()
        size_fn = "mc_grid_adjoint_workspace_bytes" if nulls is None else "mc_grid_adjoint_nulls_workspace_bytes"
        nbytes = getattr(N.lib(), size_fn)(C.byref(g))
        if nbytes == 0:
            raise N.McError(size_fn, -1)
        work = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = torch.empty(tuple(grid.density.shape), dtype=torch.float32, device=self.device)
        value = torch.empty(1, dtype=torch.float64, device=self.device)
        vp = C.c_void_p
        if nulls is None:
            N.check("mc_grid_adjoint", N.lib().mc_grid_adjoint(
                C.byref(g), vp(grid.work.data_ptr()), C.byref(m), C.byref(geo), C.byref(c), C.byref(rp),
                vp(adj.data_ptr()), vp(grad.data_ptr()), vp(value.data_ptr()), vp(self.error.data_ptr()),
                vp(work.data_ptr()), work.numel(), _stream_handle(stream)))
        else:
            N.check("mc_grid_adjoint_nulls", N.lib().mc_grid_adjoint_nulls(
                C.byref(g), vp(grid.work.data_ptr()), C.byref(m), C.byref(geo), C.byref(c), C.byref(rp),
                vp(adj.data_ptr()), float(nulls), vp(grad.data_ptr()), vp(value.data_ptr()),
                vp(self.error.data_ptr()), vp(work.data_ptr()), work.numel(), _stream_handle(stream)))
        self._keep = (keep, grid, adj, work)
        return value, grad

    def check(self, stream=None):
        """Wait for the stream and raise if a kernel flagged an error since
        the previous check; the flags are cleared either way. The word read
        is kept as last_error (0 when nothing was flagged)."""
        st = N.lib().mc_check(C.c_void_p(self.error.data_ptr()), _stream_handle(stream))
        self.last_error = int(self.error.cpu().numpy()[0]) & 0xFFFFFFFF
        _clear_error(self.error, stream)
        N.check("mc_check", st)

    def check_within(self, timeout_ms, stream=None):
        """check() with a host-side watchdog: True when the stream finished
        within timeout_ms (raises on a flagged error), False when it is still
        running (it goes on; call again or check())."""
        st = N.lib().mc_check_within(C.c_void_p(self.error.data_ptr()), _stream_handle(stream),
                                     float(timeout_ms))
        if st == N.MC_NOT_READY:
            return False
        self.last_error = int(self.error.cpu().numpy()[0]) & 0xFFFFFFFF
        _clear_error(self.error, stream)
        N.check("mc_check_within", st)
        return True

    def result(self):
        """Tallies as float64 numpy arrays in weight units (one photon = 1),
        the raw integer image and totals, and the error word (the flags
        raised since the previous check)."""
        img = self.image.cpu().numpy().astype(np.float64) * 2.0 ** -self.image_frac_bits
        rad = self.radial.cpu().numpy().astype(np.float64) * 2.0 ** -N.WEIGHT_FRAC_BITS
        tot = self.totals.cpu().numpy()
        w = tot[:7].astype(np.float64) * 2.0 ** -N.WEIGHT_FRAC_BITS
        return dict(image=img, radial=rad, totals=w, steps=int(tot[N.TOT_STEPS]),
                    raw_image=self.image.cpu().numpy(), raw_totals=tot,
                    error=int(self.error.cpu().numpy()[0]))


class Batch:
    """Device tallies for several media sharing camera and geometry, run in
    one persistent launch (mc_run_batch)."""

    def __init__(self, n, camera=None, geometry=None, device=None):
        torch = _torch()
        self.camera = camera or Camera()
        self.geometry = geometry or Geometry()
        self.device = torch.device(device if device is not None else "cuda")
        cam, dev = self.camera, self.device
        self.n = n
        self.image = torch.zeros((n, cam.nz, cam.nx), dtype=torch.int64, device=dev)
        self.radial = torch.zeros((n, cam.n_radial), dtype=torch.int64, device=dev)
        self.totals = torch.zeros((n, N.N_TOTALS), dtype=torch.int64, device=dev)
        self.error = torch.zeros(1, dtype=torch.int32, device=dev)
        wb = N.lib().mc_batch_workspace_bytes(n)
        if wb == 0:
            raise N.McError("mc_batch_workspace_bytes", -1)
        self.work = torch.zeros(wb, dtype=torch.uint8, device=dev)
        self.image_frac_bits = 32

    def run(self, media, n_photons, seeds=1, offsets=0, item_photons=0, stream=None, **kw):
        """media: list of Medium; n_photons, seeds, offsets: scalars or lists."""
        n = len(media)
        if n != self.n:
            raise ValueError("batch holds %d media, got %d" % (self.n, n))
        as_list = lambda v: list(v) if isinstance(v, (list, tuple)) else [v] * n
        nph, sd, off = as_list(n_photons), as_list(seeds), as_list(offsets)
        f = kw.get("image_frac_bits")
        if not f:
            f = self.image_frac_bits if kw.get("accumulate") else auto_frac_bits(max(int(v) for v in nph))
        self.image_frac_bits = int(f)
        rp = run_params(0, 0, **dict(kw, image_frac_bits=int(f)))
        arr = (N.Instance * n)()
        keep = []
        for i, med in enumerate(media):
            m, k = med.as_c(self.device)
            keep.append(k)
            arr[i].medium = m
            arr[i].n_photons, arr[i].photon_offset, arr[i].seed = int(nph[i]), int(off[i]), int(sd[i])
            arr[i].d_image = self.image[i].data_ptr()
            arr[i].d_radial = self.radial[i].data_ptr()
            arr[i].d_totals = self.totals[i].data_ptr()
        g, c = self.geometry.as_c(), self.camera.as_c()
        N.check("mc_run_batch", N.lib().mc_run_batch(
            n, arr, C.byref(g), C.byref(c), C.byref(rp), int(item_photons),
            C.c_void_p(self.error.data_ptr()), C.c_void_p(self.work.data_ptr()), self.work.numel(),
            _stream_handle(stream)))
        self._keep = keep
        return self

    def check(self, stream=None):
        """As Engine.check, for the batch's error word."""
        st = N.lib().mc_check(C.c_void_p(self.error.data_ptr()), _stream_handle(stream))
        _clear_error(self.error, stream)
        N.check("mc_check", st)


def camera_image(engine, table, mu_s, mu_a, phase_w=None, n_photons=10**6, seed=1, grad_seed=None, **kw):
    """Differentiable side-camera image (float64 [nz, nx], weight units).

    mu_s, mu_a: 0-d float64 tensors; phase_w: optional tensor of positive
    hat-function phase weights (the phase function p h_w / Z(w) of
    mc_phase_table_weighted; None: the table itself). Forward runs mc_run
    (with the table reweighted on the device when phase_w is given);
    backward runs mc_adjoint at the same weights with grad_output as the
    adjoint image, on the same photons (grad_seed None: the exact derivative
    of the sampled image) or on an independent photon set drawn with
    grad_seed (an unbiased estimate of the derivative of the expected image,
    uncorrelated with the forward sample; what a loss that is nonlinear in
    the image needs)."""
    torch = _torch()
    if phase_w is None:
        phase_w = torch.ones(0, dtype=torch.float64, device=engine.device)
    gs = seed if grad_seed is None else grad_seed
    return _CameraImage.apply(mu_s, mu_a, phase_w, engine, table, n_photons, (seed, gs), kw)


def _make_camera_image():
    torch = _torch()

    class CameraImageFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, mu_s, mu_a, phase_w, engine, table, n_photons, seed, kw):
            seed, grad_seed = seed
            med = Medium(float(mu_s), float(mu_a), "table", 0.0, table)
            walk_med, wt = med, None
            if phase_w.numel():
                wt = WeightedTable(table, phase_w, engine.device)
                walk_med = Medium(float(mu_s), float(mu_a), "table", 0.0, wt)
            engine.run(walk_med, n_photons, seed=seed, **kw)
            engine.check()
            if wt is not None:
                wt.check()
            img = engine.image.to(torch.float64) * 2.0 ** -engine.image_frac_bits
            ctx.engine, ctx.med, ctx.n, ctx.seed, ctx.kw = engine, med, n_photons, grad_seed, kw
            ctx.n_w = phase_w.numel()
            ctx.w = wt.phase_w if wt is not None else None
            ctx.devs = (mu_s.device, mu_a.device, phase_w.device)
            return img

        @staticmethod
        def backward(ctx, grad_img):
            out = ctx.engine.adjoint(ctx.med, grad_img, ctx.n, n_w=ctx.n_w, seed=ctx.seed, phase_w=ctx.w,
                                     **ctx.kw)
            ctx.engine.check()
            ds, da, dw = ctx.devs
            gw = out[3:].to(dw) if ctx.n_w else None
            return out[1].to(ds), out[2].to(da), gw, None, None, None, None, None

    return CameraImageFn


class _Lazy:
    fn = None

    def apply(self, *a):
        if _Lazy.fn is None:
            _Lazy.fn = _make_camera_image()
        return _Lazy.fn.apply(*a)


_CameraImage = _Lazy()


def decode_trace(buf):
    """int32 [.., 12] trace -> dict of numpy arrays."""
    a = buf.cpu().numpy() if hasattr(buf, "cpu") else np.asarray(buf)
    f = a.view(np.float32)
    return dict(status=a[..., 0], r=f[..., 1:4].astype(np.float64), d=f[..., 4:7].astype(np.float64),
                w=f[..., 7].astype(np.float64), nee=f[..., 8].astype(np.float64), pix=a[..., 9],
                nee_bin=a[..., 10], rad_bin=a[..., 11])


def run_host(medium, geometry, camera, n_photons, d_work, seed=1, stream=None, image=None,
             radial=None, totals=None, table_host=None, **kw):
    """End-to-end call with host buffers (mc_run_host): table in, tallies out.
    `d_work` is a device uint8 tensor of host_workspace_bytes() bytes; the
    host outputs (numpy int64, pinned for speed) are allocated if not given;
    `table_host` replaces the table's own host blob (e.g. a pinned copy)."""
    L = N.lib()
    m = N.Medium()
    m.mu_s, m.mu_a = medium.mu_s, medium.mu_a
    table_ptr = None
    if medium.phase in ("table", "paper"):
        m.phase_kind = N.PHASE_TABLE if medium.phase == "table" else N.PHASE_PAPER
        m.n_bins = medium.table.n_bins
        blob = medium.table.blob if table_host is None else table_host
        if blob.nbytes != medium.table.blob.nbytes:
            raise ValueError("table_host has the wrong size")
        table_ptr = blob.ctypes.data_as(C.c_void_p)
    else:
        m.phase_kind, m.hg_g = N.PHASE_HG, medium.hg_g
    image = image if image is not None else np.zeros((camera.nz, camera.nx), dtype=np.int64)
    radial = radial if radial is not None else np.zeros(camera.n_radial, dtype=np.int64)
    totals = totals if totals is not None else np.zeros(N.N_TOTALS, dtype=np.int64)
    err = np.zeros(1, dtype=np.uint32)
    rp = run_params(n_photons, seed, **kw)
    g, c = geometry.as_c(), camera.as_c()
    vp = C.c_void_p
    st = L.mc_run_host(C.byref(m), table_ptr, C.byref(g), C.byref(c), C.byref(rp),
                       image.ctypes.data_as(vp), radial.ctypes.data_as(vp), totals.ctypes.data_as(vp),
                       err.ctypes.data_as(vp), vp(d_work.data_ptr()), d_work.numel(), _stream_handle(stream))
    N.check("mc_run_host", st)
    return image, radial, totals


def host_workspace_bytes(medium, camera):
    m = N.Medium()
    m.phase_kind = {"table": N.PHASE_TABLE, "hg": N.PHASE_HG, "paper": N.PHASE_PAPER}[medium.phase]
    m.n_bins = medium.table.n_bins if medium.phase != "hg" else 0
    return N.lib().mc_host_workspace_bytes(C.byref(m), C.byref(camera.as_c()))


def image_metrics(ref, a, b=None, n_r=32, stream=None):
    """Sec. 3.1.4 / Tables 3-4 comparison of device int64 images [nz, nx]
    (mc_image_metrics). Returns a float64 numpy array: a vs ref (RMSE, r,
    zone RMSE x3, profile r), the same for b, the share of rings where a is
    closer than b, then the radial profiles of ref, a, b."""
    torch = _torch()
    L = N.lib()
    nz, nx = ref.shape
    for t in (a, b):
        if t is not None and tuple(t.shape) != (nz, nx):
            raise ValueError("images differ in shape")
    imgs = [t.contiguous() if t is not None else None for t in (ref, a, b)]
    for t in imgs:
        if t is not None and (t.dtype != torch.int64 or not t.is_cuda):
            raise ValueError("images must be int64 CUDA tensors")
    n_out = L.mc_metrics_out_len(n_r)
    if n_out == 0:
        raise ValueError("n_r out of range")
    out = torch.empty(n_out, dtype=torch.float64, device=ref.device)
    work = torch.empty(L.mc_metrics_workspace_bytes(n_r), dtype=torch.uint8, device=ref.device)
    vp = C.c_void_p
    N.check("mc_image_metrics", L.mc_image_metrics(
        vp(imgs[0].data_ptr()), vp(imgs[1].data_ptr()), vp(imgs[2].data_ptr()) if b is not None else None,
        nx, nz, n_r, vp(out.data_ptr()), vp(work.data_ptr()), work.numel(), _stream_handle(stream)))
    return out.cpu().numpy()


def philox(ctr, seed, stream=None):
    """Device Philox4x32-10 of a uint32-valued int64/int32 tensor [n, 4]."""
    torch = _torch()
    c = ctr.to(torch.int32).contiguous()
    out = torch.empty_like(c)
    N.check("mc_philox", N.lib().mc_philox(C.c_void_p(c.data_ptr()), c.shape[0], int(seed),
                                           C.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out
