// C ABI entry points of the engine (declared in include/mcmie.h): argument
// validation, conversion to the kernels' single-precision parameters, and the
// host-buffer path. No entry point here allocates device memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "engine.h"
#include "table_format.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kAlign = 256;

size_t up(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }
bool fin(double v) { return std::isfinite(v); }
bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

mc_status check_medium(const mc_medium *m)
{
    if (!m || !fin(m->mu_s) || !fin(m->mu_a) || m->mu_s < 0.0 || m->mu_a < 0.0 ||
        !(m->mu_s + m->mu_a > 0.0))
        return MC_ERR_ARG;
    if (m->phase_kind == MC_PHASE_HG) {
        if (!(m->hg_g > -1.0 && m->hg_g < 1.0)) return MC_ERR_ARG;
    } else if (m->phase_kind == MC_PHASE_TABLE) {
        if (!m->d_table || !aligned(m->d_table, 16) || !mc_table_layout(m->n_bins, nullptr))
            return MC_ERR_ARG;
    } else {
        return MC_ERR_ARG;
    }
    return MC_OK;
}

mc_status check_geom(const mc_geometry *g)
{
    if (!g || !fin(g->lx) || !fin(g->ly) || !fin(g->lz) || !(g->lx > 0) || !(g->ly > 0) ||
        !(g->lz > 0) || !fin(g->beam_radius) || g->beam_radius < 0 ||
        g->beam_radius > 0.5 * std::fmin(g->ly, g->lz))
        return MC_ERR_ARG;
    return MC_OK;
}

mc_status check_camera(const mc_camera *c)
{
    if (!c || c->nx < 1 || c->nz < 1 || c->nx > 8192 || c->nz > 8192 || c->n_radial < 1 ||
        c->n_radial > 65536 || !fin(c->r_max) || !(c->r_max > 0))
        return MC_ERR_ARG;
    return MC_OK;
}

mc_status check_run(const mc_run_params *r)
{
    if (!r || !fin(r->rr_threshold) || r->rr_threshold < 0 || !fin(r->rr_survival) ||
        r->rr_survival < 0 || r->rr_survival > 1 || r->max_events < 1 || r->image_frac_bits < 8 ||
        r->image_frac_bits > 48 || (r->accumulate != 0 && r->accumulate != 1) ||
        r->photon_offset + r->n_photons < r->photon_offset || r->block_size < 0 ||
        r->block_size > 1024 || (r->block_size % 32) != 0 || r->blocks_per_sm < 0 ||
        r->blocks_per_sm > 64 || r->image_mode < 0 || r->image_mode > 3)
        return MC_ERR_ARG;
    return MC_OK;
}

mc_status check_tallies(const mc_tallies *t, const mc_camera *c)
{
    if (!t || !t->d_image || !t->d_radial || !t->d_totals || !t->d_error || !t->d_work ||
        !aligned(t->d_image, 8) || !aligned(t->d_radial, 8) || !aligned(t->d_totals, 8) ||
        !aligned(t->d_error, 4) || !aligned(t->d_work, 16))
        return MC_ERR_ARG;
    if (t->work_bytes < mc_workspace_bytes(c)) return MC_ERR_NOMEM;
    return MC_OK;
}

mcx::WalkArgs make_args(const mc_medium *m, const mc_geometry *g, const mc_camera *c,
                        const mc_run_params *r, const mc_tallies *t)
{
    mcx::WalkArgs a;
    std::memset(&a, 0, sizeof a);
    const double mu_ext = m->mu_s + m->mu_a;
    a.mu_ext = (float)mu_ext;
    a.inv_mu_ext = (float)(1.0 / mu_ext);
    a.absorb_frac = (float)(m->mu_a / mu_ext);
    a.albedo = (float)(1.0 - m->mu_a / mu_ext);
    a.phase_kind = m->phase_kind;
    const double gg = (m->phase_kind == MC_PHASE_HG) ? m->hg_g : 0.0;
    a.hg_g = (float)gg;
    a.hg_one_m_g = (float)(1.0 - gg);
    a.hg_two_g = (float)(2.0 * gg);
    a.hg_A = (float)(2.0 * (1.0 - gg) * (1.0 - gg));
    a.hg_a2 = (float)((1.0 - gg) * (1.0 - gg));
    a.hg_K = (float)((1.0 - gg * gg) / (4.0 * kPi));
    if (m->phase_kind == MC_PHASE_TABLE) {
        a.table = static_cast<const unsigned char *>(m->d_table);
        a.table_bytes = (uint32_t)mc_table_layout(m->n_bins, nullptr);
        a.n_bins = m->n_bins;
    }
    a.lx = (float)g->lx;
    a.hy = (float)(0.5 * g->ly);
    a.hz = (float)(0.5 * g->lz);
    a.beam_r = (float)g->beam_radius;
    a.nx = c->nx;
    a.nz = c->nz;
    a.n_radial = c->n_radial;
    a.sx = (float)(c->nx / g->lx);
    a.sz = (float)(c->nz / g->lz);
    a.sr = (float)(c->n_radial / c->r_max);
    a.n_photons = r->n_photons;
    a.photon_offset = r->photon_offset;
    a.key0 = (uint32_t)r->seed;
    a.key1 = (uint32_t)(r->seed >> 32);
    a.rr_thr = (float)r->rr_threshold;
    a.rr_surv = (float)r->rr_survival;
    a.inv_rr_surv = r->rr_survival > 0 ? (float)(1.0 / r->rr_survival) : 0.0f;
    a.max_events = r->max_events;
    a.max_scatter = r->max_scatter;
    a.img_scale = std::ldexp(1.0f, r->image_frac_bits);
    a.image = reinterpret_cast<unsigned long long *>(t->d_image);
    a.radial = reinterpret_cast<unsigned long long *>(t->d_radial);
    a.totals = reinterpret_cast<unsigned long long *>(t->d_totals);
    a.error = t->d_error;
    a.counter = reinterpret_cast<unsigned long long *>(t->d_work);
    return a;
}

mc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MC_OK : MC_ERR_CUDA; }

mc_status validate_all(const mc_medium *m, const mc_geometry *g, const mc_camera *c,
                       const mc_run_params *r)
{
    mc_status s;
    if ((s = check_medium(m)) != MC_OK) return s;
    if ((s = check_geom(g)) != MC_OK) return s;
    if ((s = check_camera(c)) != MC_OK) return s;
    if ((s = check_run(r)) != MC_OK) return s;
    return MC_OK;
}

mc_status run_common(const mc_medium *m, const mc_geometry *g, const mc_camera *c,
                     const mc_run_params *r, const mc_tallies *t, int32_t *trace, int n_trace,
                     int n_events, cudaStream_t st)
{
    mc_status s;
    if ((s = validate_all(m, g, c, r)) != MC_OK) return s;
    if ((s = check_tallies(t, c)) != MC_OK) return s;
    cudaError_t e;
    if (!r->accumulate) {
        if ((e = cudaMemsetAsync(t->d_image, 0, sizeof(int64_t) * (size_t)c->nx * c->nz, st)))
            return cuda_status(e);
        if ((e = cudaMemsetAsync(t->d_radial, 0, sizeof(int64_t) * (size_t)c->n_radial, st)))
            return cuda_status(e);
        if ((e = cudaMemsetAsync(t->d_totals, 0, sizeof(int64_t) * MC_N_TOTALS, st)))
            return cuda_status(e);
    }
    if ((e = cudaMemsetAsync(t->d_work, 0, sizeof(unsigned long long), st))) return cuda_status(e);
    if (r->n_photons == 0) return MC_OK;
    mcx::WalkArgs a = make_args(m, g, c, r, t);
    a.trace = trace;
    a.n_trace = n_trace;
    a.n_trace_events = n_events;
    mcx::LaunchCfg cfg;
    cfg.block = r->block_size;
    cfg.blocks_per_sm = r->blocks_per_sm;
    cfg.image_mode = r->image_mode;
    e = mcx::launch_walk(a, trace != nullptr, cfg, st);
    if (e == cudaErrorInvalidValue) return MC_ERR_ARG;  // requested image tile does not fit
    return cuda_status(e);
}

}  // namespace

extern "C" {

size_t mc_workspace_bytes(const mc_camera *camera)
{
    if (check_camera(camera) != MC_OK) return 0;
    return kAlign;  // the photon counter
}

mc_status mc_run(const mc_medium *medium, const mc_geometry *geom, const mc_camera *camera,
                 const mc_run_params *run, const mc_tallies *tallies, void *stream)
{
    return run_common(medium, geom, camera, run, tallies, nullptr, 0, 0,
                      static_cast<cudaStream_t>(stream));
}

mc_status mc_trace(const mc_medium *medium, const mc_geometry *geom, const mc_camera *camera,
                   const mc_run_params *run, const mc_tallies *tallies, void *d_trace, int n_trace,
                   int n_events, void *stream)
{
    if (!d_trace || !aligned(d_trace, 4) || n_trace < 1 || n_events < 1 || n_events > 1 << 20 ||
        (uint64_t)n_trace > (run ? run->n_photons : 0))
        return MC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(d_trace, 0xFF, sizeof(int32_t) * 12 * (size_t)n_trace * n_events, st);
    if (e != cudaSuccess) return MC_ERR_CUDA;
    return run_common(medium, geom, camera, run, tallies, static_cast<int32_t *>(d_trace), n_trace,
                      n_events, st);
}

size_t mc_host_workspace_bytes(const mc_medium *medium, const mc_camera *camera)
{
    if (check_camera(camera) != MC_OK || !medium) return 0;
    size_t tb = 0;
    if (medium->phase_kind == MC_PHASE_TABLE) {
        tb = mc_table_layout(medium->n_bins, nullptr);
        if (!tb) return 0;
    }
    return up(tb) + up(sizeof(int64_t) * (size_t)camera->nx * camera->nz) +
           up(sizeof(int64_t) * (size_t)camera->n_radial) + up(sizeof(int64_t) * MC_N_TOTALS) +
           up(sizeof(uint32_t)) + up(mc_workspace_bytes(camera));
}

mc_status mc_run_host(const mc_medium *medium, const void *table, const mc_geometry *geom,
                      const mc_camera *camera, const mc_run_params *run, int64_t *image,
                      int64_t *radial, int64_t *totals, uint32_t *error, void *d_work,
                      size_t work_bytes, void *stream)
{
    if (!medium || !image || !radial || !totals || !error || !d_work || !aligned(d_work, 256))
        return MC_ERR_ARG;
    if (medium->phase_kind == MC_PHASE_TABLE && !table) return MC_ERR_ARG;
    mc_medium m = *medium;
    if (m.phase_kind == MC_PHASE_TABLE) m.d_table = d_work;  // placeholder for validation
    mc_status s;
    if ((s = validate_all(&m, geom, camera, run)) != MC_OK) return s;
    const size_t need = mc_host_workspace_bytes(medium, camera);
    if (!need) return MC_ERR_ARG;
    if (work_bytes < need) return MC_ERR_NOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *p = static_cast<unsigned char *>(d_work);
    size_t tb = m.phase_kind == MC_PHASE_TABLE ? mc_table_layout(m.n_bins, nullptr) : 0;
    const size_t npix = (size_t)camera->nx * camera->nz;
    mc_tallies t;
    unsigned char *d_table = p;
    p += up(tb);
    t.d_image = reinterpret_cast<int64_t *>(p);
    p += up(sizeof(int64_t) * npix);
    t.d_radial = reinterpret_cast<int64_t *>(p);
    p += up(sizeof(int64_t) * (size_t)camera->n_radial);
    t.d_totals = reinterpret_cast<int64_t *>(p);
    p += up(sizeof(int64_t) * MC_N_TOTALS);
    t.d_error = reinterpret_cast<uint32_t *>(p);
    p += up(sizeof(uint32_t));
    t.d_work = p;
    t.work_bytes = mc_workspace_bytes(camera);
    auto fail = [](cudaError_t x) { return x != cudaSuccess; };
    if (tb && fail(cudaMemcpyAsync(d_table, table, tb, cudaMemcpyHostToDevice, st))) return MC_ERR_CUDA;
    if (fail(cudaMemsetAsync(t.d_error, 0, sizeof(uint32_t), st))) return MC_ERR_CUDA;
    mc_run_params r = *run;
    if (r.accumulate) {
        // carry the caller's running tallies in
        if (fail(cudaMemcpyAsync(t.d_image, image, sizeof(int64_t) * npix, cudaMemcpyHostToDevice, st)) ||
            fail(cudaMemcpyAsync(t.d_radial, radial, sizeof(int64_t) * camera->n_radial,
                                 cudaMemcpyHostToDevice, st)) ||
            fail(cudaMemcpyAsync(t.d_totals, totals, sizeof(int64_t) * MC_N_TOTALS,
                                 cudaMemcpyHostToDevice, st)))
            return MC_ERR_CUDA;
    }
    if (tb) m.d_table = d_table;
    if ((s = run_common(&m, geom, camera, &r, &t, nullptr, 0, 0, st)) != MC_OK) return s;
    if (fail(cudaMemcpyAsync(image, t.d_image, sizeof(int64_t) * npix, cudaMemcpyDeviceToHost, st)) ||
        fail(cudaMemcpyAsync(radial, t.d_radial, sizeof(int64_t) * camera->n_radial,
                             cudaMemcpyDeviceToHost, st)) ||
        fail(cudaMemcpyAsync(totals, t.d_totals, sizeof(int64_t) * MC_N_TOTALS, cudaMemcpyDeviceToHost,
                             st)) ||
        fail(cudaMemcpyAsync(error, t.d_error, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)))
        return MC_ERR_CUDA;
    if (fail(cudaStreamSynchronize(st))) return MC_ERR_CUDA;
    if (*error & MC_EFLAG_TIMEOUT) return MC_ERR_TIMEOUT;
    if (*error & MC_EFLAG_TABLE) return MC_ERR_TABLE;
    if (*error & MC_EFLAG_NUMERIC) return MC_ERR_NUMERIC;
    if (*error & MC_EFLAG_OVERFLOW) return MC_ERR_OVERFLOW;
    if (*error & MC_EFLAG_EVENTS) return MC_ERR_EVENTS;
    return MC_OK;
}

mc_status mc_check(const uint32_t *d_error, void *stream)
{
    if (!d_error) return MC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MC_ERR_CUDA;
    uint32_t h = 0;
    if (cudaMemcpy(&h, d_error, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return MC_ERR_CUDA;
    if (h & MC_EFLAG_TIMEOUT) return MC_ERR_TIMEOUT;
    if (h & MC_EFLAG_TABLE) return MC_ERR_TABLE;
    if (h & MC_EFLAG_NUMERIC) return MC_ERR_NUMERIC;
    if (h & MC_EFLAG_OVERFLOW) return MC_ERR_OVERFLOW;
    if (h & MC_EFLAG_EVENTS) return MC_ERR_EVENTS;
    return MC_OK;
}

mc_status mc_philox(const uint32_t *d_ctr, uint64_t n, uint64_t seed, uint32_t *d_out, void *stream)
{
    if ((n && (!d_ctr || !d_out)) || (d_ctr && !aligned(d_ctr, 16)) || (d_out && !aligned(d_out, 16)))
        return MC_ERR_ARG;
    return cuda_status(mcx::launch_philox(d_ctr, n, seed, d_out, static_cast<cudaStream_t>(stream)));
}

const char *mc_status_string(mc_status s)
{
    switch (s) {
    case MC_OK: return "ok";
    case MC_ERR_ARG: return "invalid argument";
    case MC_ERR_CUDA: return "CUDA runtime error";
    case MC_ERR_NOMEM: return "workspace too small";
    case MC_ERR_TIMEOUT: return "device wait timed out";
    case MC_ERR_OVERFLOW: return "fixed-point overflow";
    case MC_ERR_NUMERIC: return "non-finite value";
    case MC_ERR_EVENTS: return "photon reached max_events";
    case MC_ERR_TABLE: return "phase table header mismatch";
    }
    return "unknown status";
}

}  // extern "C"
