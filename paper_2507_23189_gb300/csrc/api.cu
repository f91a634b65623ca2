// C ABI entry points of the engine (declared in include/mcmie.h): argument
// validation, conversion to the kernels' single-precision parameters, and the
// host-buffer path. No entry point here allocates device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <chrono>
#include <cstring>
#include <thread>
#include <new>

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
    } else if (m->phase_kind == MC_PHASE_PAPER) {
        if (!m->d_table || !aligned(m->d_table, 16) || !mc_paper_layout(m->n_bins, nullptr))
            return MC_ERR_ARG;
    } else {
        return MC_ERR_ARG;
    }
    return MC_OK;
}

// Bytes of the medium's table blob (0 for H-G).
size_t table_bytes_of(const mc_medium *m)
{
    if (m->phase_kind == MC_PHASE_TABLE) return mc_table_layout(m->n_bins, nullptr);
    if (m->phase_kind == MC_PHASE_PAPER) return mc_paper_layout(m->n_bins, nullptr);
    return 0;
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

// Photons one call may run: the weight totals are in 2^-32 units and a
// photon's exits, absorption and truncation add up to about its unit weight,
// so 2^31 photons keep every total below 2^63.
constexpr uint64_t kMaxPhotons = 1ull << 31;

// image_frac_bits 0 (fresh tallies only): the fraction bits for a budget of
// n photons, min(32, 54 - ceil(log2 n)), at least 8. 54 = 63 - 9 leaves a
// factor 2^9 between 2^63 and n times one weight unit per photon in one
// pixel (a pixel's expected sum per photon is far below one weight unit).
int auto_frac_bits(uint64_t n)
{
    int lg = 0;
    while (lg < 64 && (1ull << lg) < n) ++lg;   // ceil(log2 n) for n >= 1
    int f = 54 - lg;
    if (f > 32) f = 32;
    if (f < 8) f = 8;
    return f;
}

int frac_bits_of(const mc_run_params *r, uint64_t n_photons)
{
    return r->image_frac_bits ? r->image_frac_bits : auto_frac_bits(n_photons);
}

mc_status check_run(const mc_run_params *r)
{
    if (!r || !fin(r->rr_threshold) || r->rr_threshold < 0 || !fin(r->rr_survival) ||
        r->rr_survival < 0 || r->rr_survival > 1 || r->max_events < 1 ||
        !((r->image_frac_bits >= 8 && r->image_frac_bits <= 48) ||
          (r->image_frac_bits == 0 && r->accumulate == 0)) ||
        r->n_photons > kMaxPhotons || (r->accumulate != 0 && r->accumulate != 1) ||
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

void fill_medium(mcx::MediumArgs &m, const mc_medium *med, uint64_t n_photons, uint64_t offset,
                 uint64_t seed, int64_t *image, int64_t *radial, int64_t *totals)
{
    const double mu_ext = med->mu_s + med->mu_a;
    m.mu_ext = (float)mu_ext;
    m.inv_mu_ext = (float)(1.0 / mu_ext);
    m.absorb_frac = (float)(med->mu_a / mu_ext);
    m.albedo = (float)(1.0 - med->mu_a / mu_ext);
    const double gg = (med->phase_kind == MC_PHASE_HG) ? med->hg_g : 0.0;
    m.hg_g = (float)gg;
    m.hg_one_m_g = (float)(1.0 - gg);
    m.hg_two_g = (float)(2.0 * gg);
    m.hg_A = (float)(2.0 * (1.0 - gg) * (1.0 - gg));
    m.hg_B = (float)(2.0 * (1.0 + gg) * (1.0 + gg));
    m.hg_a2 = (float)((1.0 - gg) * (1.0 - gg));
    m.hg_K = (float)((1.0 - gg * gg) / (4.0 * kPi));
    m.table = (med->phase_kind != MC_PHASE_HG) ? static_cast<const unsigned char *>(med->d_table) : nullptr;
    m.key0 = (uint32_t)seed;
    m.key1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        m.rk[2 * i] = m.key0 + (uint32_t)i * 0x9E3779B9u;
        m.rk[2 * i + 1] = m.key1 + (uint32_t)i * 0xBB67AE85u;
    }
    m.n_photons = n_photons;
    m.photon_offset = offset;
    m.image = reinterpret_cast<unsigned long long *>(image);
    m.radial = reinterpret_cast<unsigned long long *>(radial);
    m.totals = reinterpret_cast<unsigned long long *>(totals);
}

// n_photons: the budget an automatic image_frac_bits is chosen for.
void fill_common(mcx::CommonArgs &c, const mc_medium *m, const mc_geometry *g, const mc_camera *cam,
                 const mc_run_params *r, uint32_t *error, uint64_t n_photons)
{
    c.phase_kind = m->phase_kind;
    c.table_bytes = (uint32_t)table_bytes_of(m);
    c.n_bins = (m->phase_kind != MC_PHASE_HG) ? m->n_bins : 0;
    c.lx = (float)g->lx;
    c.hy = (float)(0.5 * g->ly);
    c.hz = (float)(0.5 * g->lz);
    c.beam_r = (float)g->beam_radius;
    c.nx = cam->nx;
    c.nz = cam->nz;
    c.n_radial = cam->n_radial;
    c.sx = (float)(cam->nx / g->lx);
    c.sz = (float)(cam->nz / g->lz);
    c.sr = (float)(cam->n_radial / cam->r_max);
    c.rr_thr = (float)r->rr_threshold;
    c.rr_surv = (float)r->rr_survival;
    c.inv_rr_surv = r->rr_survival > 0 ? (float)(1.0 / r->rr_survival) : 0.0f;
    c.max_events = r->max_events;
    c.max_scatter = r->max_scatter;
    c.img_scale = std::ldexp(1.0f, frac_bits_of(r, n_photons));
    c.error = error;
    c.extra_bytes = 0;
}

mcx::WalkArgs make_args(const mc_medium *m, const mc_geometry *g, const mc_camera *c,
                        const mc_run_params *r, const mc_tallies *t)
{
    mcx::WalkArgs a;
    std::memset(&a, 0, sizeof a);
    fill_common(a.c, m, g, c, r, t->d_error, r->n_photons);
    fill_medium(a.m, m, r->n_photons, r->photon_offset, r->seed, t->d_image, t->d_radial, t->d_totals);
    a.counter = reinterpret_cast<unsigned long long *>(t->d_work);
    return a;
}

mcx::LaunchCfg launch_cfg(const mc_run_params *r)
{
    mcx::LaunchCfg cfg;
    cfg.block = r->block_size;
    cfg.blocks_per_sm = r->blocks_per_sm;
    cfg.image_mode = r->image_mode;
    return cfg;
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
    mcx::WalkArgs a = make_args(m, g, c, r, t);
    a.c.trace = trace;
    a.c.n_trace = n_trace;
    a.c.n_trace_events = n_events;
    // refused before anything is queued when the shared-memory plan does not fit
    cudaError_t e = mcx::check_plan(a.c, launch_cfg(r));
    if (e != cudaSuccess) return e == cudaErrorInvalidValue ? MC_ERR_ARG : MC_ERR_CUDA;
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
    e = mcx::launch_walk(a, trace != nullptr, launch_cfg(r), st);
    return cuda_status(e);
}

}  // namespace

extern "C" {

int mc_auto_frac_bits(uint64_t n_photons) { return auto_frac_bits(n_photons); }

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
    const size_t tb = table_bytes_of(medium);
    if (medium->phase_kind != MC_PHASE_HG && !tb) return 0;
    return up(tb) + up(sizeof(int64_t) * (size_t)camera->nx * camera->nz) +
           up(sizeof(int64_t) * (size_t)camera->n_radial) + up(sizeof(int64_t) * MC_N_TOTALS) +
           up(sizeof(uint32_t)) + up(mc_workspace_bytes(camera));
}

static mc_status flags_status(uint32_t h)
{
    if (h & MC_EFLAG_TIMEOUT) return MC_ERR_TIMEOUT;
    if (h & MC_EFLAG_TABLE) return MC_ERR_TABLE;
    if (h & MC_EFLAG_BOUNDS) return MC_ERR_BOUNDS;
    if (h & MC_EFLAG_NUMERIC) return MC_ERR_NUMERIC;
    if (h & MC_EFLAG_OVERFLOW) return MC_ERR_OVERFLOW;
    if (h & MC_EFLAG_EVENTS) return MC_ERR_EVENTS;
    return MC_OK;
}

mc_status mc_run_host(const mc_medium *medium, const void *table, const mc_geometry *geom,
                      const mc_camera *camera, const mc_run_params *run, int64_t *image,
                      int64_t *radial, int64_t *totals, uint32_t *error, void *d_work,
                      size_t work_bytes, void *stream)
{
    if (!medium || !image || !radial || !totals || !error || !d_work || !aligned(d_work, 256))
        return MC_ERR_ARG;
    if (medium->phase_kind != MC_PHASE_HG && !table) return MC_ERR_ARG;
    mc_medium m = *medium;
    if (m.phase_kind != MC_PHASE_HG) m.d_table = d_work;  // placeholder for validation
    mc_status s;
    if ((s = validate_all(&m, geom, camera, run)) != MC_OK) return s;
    const size_t need = mc_host_workspace_bytes(medium, camera);
    if (!need) return MC_ERR_ARG;
    if (work_bytes < need) return MC_ERR_NOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *p = static_cast<unsigned char *>(d_work);
    const size_t tb = table_bytes_of(&m);
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
    {   // refused before any copy is queued when the shared-memory plan does not fit
        const mcx::WalkArgs a = make_args(&m, geom, camera, run, &t);
        const cudaError_t pe = mcx::check_plan(a.c, launch_cfg(run));
        if (pe != cudaSuccess) return pe == cudaErrorInvalidValue ? MC_ERR_ARG : MC_ERR_CUDA;
    }
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
    return flags_status(*error);
}

size_t mc_batch_workspace_bytes(int n_instances)
{
    if (n_instances < 1 || n_instances > mcx::kMaxBatch) return 0;
    return up(sizeof(unsigned long long) * (size_t)n_instances);  // one photon counter per medium
}

mc_status mc_run_batch(int n, const mc_instance *inst, const mc_geometry *geom, const mc_camera *camera,
                       const mc_run_params *run, uint64_t item_photons, uint32_t *d_error, void *d_work,
                       size_t work_bytes, void *stream)
{
    if (n < 1 || n > mcx::kMaxBatch || !inst || !d_error || !d_work || !aligned(d_work, 16) ||
        !aligned(d_error, 4) || (item_photons != 0 && (item_photons < 32 || item_photons > (1ull << 20))))
        return MC_ERR_ARG;
    if (work_bytes < mc_batch_workspace_bytes(n)) return MC_ERR_NOMEM;
    mc_status s;
    if ((s = check_geom(geom)) != MC_OK || (s = check_camera(camera)) != MC_OK ||
        (s = check_run(run)) != MC_OK)
        return s;
    for (int i = 0; i < n; ++i) {
        const mc_instance &I = inst[i];
        if ((s = check_medium(&I.medium)) != MC_OK) return s;
        if (I.medium.phase_kind != inst[0].medium.phase_kind ||
            (I.medium.phase_kind != MC_PHASE_HG && I.medium.n_bins != inst[0].medium.n_bins))
            return MC_ERR_ARG;   // one phase kind and table size per batch
        if (!I.d_image || !I.d_radial || !I.d_totals || !aligned(I.d_image, 8) || !aligned(I.d_radial, 8) ||
            !aligned(I.d_totals, 8) || I.photon_offset + I.n_photons < I.photon_offset ||
            I.n_photons > kMaxPhotons)
            return MC_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    {   // refused before anything is queued when the shared-memory plan does not fit
        mcx::CommonArgs c;
        std::memset(&c, 0, sizeof c);
        fill_common(c, &inst[0].medium, geom, camera, run, d_error, 1);
        if ((e = mcx::check_plan(c, launch_cfg(run))) != cudaSuccess)
            return e == cudaErrorInvalidValue ? MC_ERR_ARG : MC_ERR_CUDA;
    }
    if (!run->accumulate)
        for (int i = 0; i < n; ++i) {
            if ((e = cudaMemsetAsync(inst[i].d_image, 0, sizeof(int64_t) * (size_t)camera->nx * camera->nz, st)) ||
                (e = cudaMemsetAsync(inst[i].d_radial, 0, sizeof(int64_t) * (size_t)camera->n_radial, st)) ||
                (e = cudaMemsetAsync(inst[i].d_totals, 0, sizeof(int64_t) * MC_N_TOTALS, st)))
                return MC_ERR_CUDA;
        }
    if ((e = cudaMemsetAsync(d_work, 0, sizeof(unsigned long long) * (size_t)n, st))) return MC_ERR_CUDA;

    // largest estimated cost first: photons x (1 + optical depth along the beam)
    int order[mcx::kMaxBatch];
    double cost[mcx::kMaxBatch];
    for (int i = 0; i < n; ++i) {
        order[i] = i;
        cost[i] = (double)inst[i].n_photons * (1.0 + (inst[i].medium.mu_s + inst[i].medium.mu_a) * geom->lx);
    }
    for (int i = 1; i < n; ++i)   // stable insertion sort, descending
        for (int j = i; j > 0 && cost[order[j]] > cost[order[j - 1]]; --j) {
            int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t;
        }
    mcx::BatchArgs *a = new (std::nothrow) mcx::BatchArgs;
    if (!a) return MC_ERR_NOMEM;
    std::memset(a, 0, sizeof *a);
    uint64_t n_max = 0, n_all = 0;
    for (int i = 0; i < n; ++i) {
        n_max = inst[i].n_photons > n_max ? inst[i].n_photons : n_max;
        n_all += inst[i].n_photons;
    }
    fill_common(a->c, &inst[0].medium, geom, camera, run, d_error, n_max);
    a->n_media = n;
    a->chunk = item_photons ? (unsigned)item_photons : 128u;
    a->counters = static_cast<unsigned long long *>(d_work);
    for (int k = 0; k < n; ++k) {
        const mc_instance &I = inst[order[k]];
        fill_medium(a->m[k], &I.medium, I.n_photons, I.photon_offset, I.seed, I.d_image, I.d_radial, I.d_totals);
    }
    if (n_all == 0) {
        delete a;
        return MC_OK;
    }
    e = mcx::launch_batch(*a, launch_cfg(run), st);
    delete a;
    return cuda_status(e);
}

size_t mc_adjoint_workspace_bytes(int n_phase_w)
{
    if (n_phase_w < 0 || n_phase_w == 1 || n_phase_w > 256) return 0;
    const int rows = mcx::adjoint_max_grid();
    if (rows < 1) return 0;
    // counter, hat integrals, per-CTA partials, and room for the largest
    // reweighted table when there are phase weights
    return kAlign + up(sizeof(double) * 256) + up(sizeof(double) * (size_t)rows * (3 + n_phase_w)) +
           (n_phase_w > 0 ? up(mc_table_layout(mcx::kMaxWeightedBins, nullptr)) : 0);
}

mc_status mc_phase_table_weighted(const mc_medium *base, int n_phase_w, const float *d_phase_w, void *d_table,
                                  size_t table_bytes, uint32_t *d_error, void *stream)
{
    if (!base || base->phase_kind != MC_PHASE_TABLE || check_medium(base) != MC_OK ||
        base->n_bins > mcx::kMaxWeightedBins || n_phase_w < 2 ||
        n_phase_w > 256 || !d_phase_w || !aligned(d_phase_w, 4) || !d_table || !aligned(d_table, 16) ||
        !d_error || !aligned(d_error, 4) || d_table == base->d_table)
        return MC_ERR_ARG;
    if (table_bytes < mc_table_layout(base->n_bins, nullptr)) return MC_ERR_NOMEM;
    return cuda_status(mcx::launch_weighted_table(static_cast<const unsigned char *>(base->d_table), base->n_bins,
                                                  n_phase_w, d_phase_w, static_cast<unsigned char *>(d_table),
                                                  d_error, static_cast<cudaStream_t>(stream)));
}

mc_status mc_adjoint(const mc_medium *medium, const mc_geometry *geom, const mc_camera *camera,
                     const mc_run_params *run, const float *d_adj_image, int n_phase_w,
                     const float *d_phase_w, double *d_out, uint32_t *d_error, void *d_work,
                     size_t work_bytes, void *stream)
{
    mc_status s;
    if ((s = validate_all(medium, geom, camera, run)) != MC_OK) return s;
    if (!d_adj_image || !d_out || !d_error || !d_work || !aligned(d_adj_image, 4) || !aligned(d_out, 8) ||
        !aligned(d_work, 16) || !(medium->mu_s > 0.0) || n_phase_w < 0 || n_phase_w == 1 || n_phase_w > 256 ||
        (n_phase_w > 0 && medium->phase_kind != MC_PHASE_TABLE) || medium->phase_kind == MC_PHASE_PAPER ||
        (d_phase_w && (n_phase_w == 0 || !aligned(d_phase_w, 4) || medium->n_bins > mcx::kMaxWeightedBins)))
        return MC_ERR_ARG;
    const size_t need = mc_adjoint_workspace_bytes(n_phase_w);
    if (!need) return MC_ERR_CUDA;
    if (work_bytes < need) return MC_ERR_NOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_out, 0, sizeof(double) * (3 + n_phase_w), st))) return MC_ERR_CUDA;
    if ((e = cudaMemsetAsync(d_work, 0, sizeof(unsigned long long), st))) return MC_ERR_CUDA;
    if (run->n_photons == 0) return MC_OK;
    mcx::AdjArgs a;
    std::memset(&a, 0, sizeof a);
    fill_common(a.c, medium, geom, camera, run, d_error, run->n_photons);
    fill_medium(a.m, medium, run->n_photons, run->photon_offset, run->seed, nullptr, nullptr, nullptr);
    a.adj = d_adj_image;
    a.n_w = n_phase_w;
    a.w = d_phase_w;
    a.base_table = a.m.table;
    a.c_s = (float)(1.0 / medium->mu_s - 1.0 / (medium->mu_s + medium->mu_a));
    unsigned char *wk = static_cast<unsigned char *>(d_work);
    const int rows = mcx::adjoint_max_grid();
    a.counter = reinterpret_cast<unsigned long long *>(wk);
    a.z = reinterpret_cast<double *>(wk + kAlign);
    a.partials = reinterpret_cast<double *>(wk + kAlign + up(sizeof(double) * 256));
    if (d_phase_w) {
        // the walk samples p h_w / Z(w): the table reweighted on the device
        unsigned char *wt = wk + kAlign + up(sizeof(double) * 256) +
                            up(sizeof(double) * (size_t)rows * (3 + n_phase_w));
        if ((e = mcx::launch_weighted_table(a.base_table, medium->n_bins, n_phase_w, d_phase_w, wt, d_error,
                                            st)) != cudaSuccess)
            return cuda_status(e);
        a.m.table = wt;
    }
    e = mcx::launch_adjoint(a, rows, d_out, st);
    return cuda_status(e);
}

mc_status mc_check(const uint32_t *d_error, void *stream)
{
    if (!d_error) return MC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MC_ERR_CUDA;
    uint32_t h = 0;
    if (cudaMemcpy(&h, d_error, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return MC_ERR_CUDA;
    return flags_status(h);
}

mc_status mc_check_within(const uint32_t *d_error, void *stream, double timeout_ms)
{
    if (!d_error || !(timeout_ms >= 0.0)) return MC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const cudaError_t q = cudaStreamQuery(st);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return MC_ERR_CUDA;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms >= timeout_ms) return MC_NOT_READY;   // the work goes on; check again later
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    uint32_t h = 0;
    if (cudaMemcpy(&h, d_error, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return MC_ERR_CUDA;
    return flags_status(h);
}

mc_status mc_wait_selftest(uint32_t *d_error, uint32_t tries, void *stream)
{
    if (!d_error || tries == 0 || tries > (1u << 22)) return MC_ERR_ARG;
    return cuda_status(mcx::launch_wait_selftest(d_error, tries, static_cast<cudaStream_t>(stream)));
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
    case MC_NOT_READY: return "work still running";
    case MC_OK: return "ok";
    case MC_ERR_ARG: return "invalid argument";
    case MC_ERR_CUDA: return "CUDA runtime error";
    case MC_ERR_NOMEM: return "workspace too small";
    case MC_ERR_TIMEOUT: return "device wait timed out";
    case MC_ERR_OVERFLOW: return "fixed-point overflow";
    case MC_ERR_NUMERIC: return "non-finite value";
    case MC_ERR_EVENTS: return "photon reached max_events";
    case MC_ERR_TABLE: return "phase table header mismatch";
    case MC_ERR_BOUNDS: return "index check failed (checked build)";
    }
    return "unknown status";
}

}  // extern "C"

// ------------------------------------------------------------ voxel grids

namespace {

constexpr int kMaxCells = 16384;

size_t pad16(size_t b) { return (b + 15) & ~(size_t)15; }

bool grid_dims(const mc_grid *g, int *mx, int *my, int *mz)
{
    if (!g || g->gx < 1 || g->gy < 1 || g->gz < 1 || g->gx > 4096 || g->gy > 4096 || g->gz > 4096 ||
        (long long)g->gx * g->gy * g->gz > (1ll << 28) || g->bx < 1 || g->by < 1 || g->bz < 1 ||
        !fin(g->k_ext) || !fin(g->k_sca) || !fin(g->mu_a) || !(g->k_ext > 0.0) || g->k_sca < 0.0 ||
        g->k_sca > g->k_ext || g->mu_a < 0.0)
        return false;
    *mx = (g->gx + g->bx - 1) / g->bx;
    *my = (g->gy + g->by - 1) / g->by;
    *mz = (g->gz + g->bz - 1) / g->bz;
    return (long long)*mx * *my * *mz <= kMaxCells;
}

void fill_grid(mcx::GridArgs &a, const mc_grid *g, int mx, int my, int mz, const void *d_grid_work,
               const mc_medium *m, const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
               uint32_t *d_error, int64_t *image, int64_t *radial, int64_t *totals)
{
    std::memset(&a, 0, sizeof a);
    fill_common(a.c, m, geom, camera, run, d_error, run->n_photons);
    fill_medium(a.m, m, run->n_photons, run->photon_offset, run->seed, image, radial, totals);
    const unsigned char *w = static_cast<const unsigned char *>(d_grid_work);
    a.cells = reinterpret_cast<const float2 *>(w);
    a.maj = reinterpret_cast<const float *>(w + pad16(sizeof(float) * 2 * (size_t)g->gx * g->gy * g->gz));
    a.c.extra_bytes = (uint32_t)pad16(sizeof(float) * (size_t)mx * my * mz);
    a.gx = g->gx; a.gy = g->gy; a.gz = g->gz;
    a.mx = mx; a.my = my; a.mz = mz;
    a.inv_vx = (float)(g->gx / geom->lx);
    a.inv_vy = (float)(g->gy / geom->ly);
    a.inv_vz = (float)(g->gz / geom->lz);
    a.vx = (float)(geom->lx / g->gx);
    a.vy = (float)(geom->ly / g->gy);
    a.vz = (float)(geom->lz / g->gz);
    a.csx = (float)(g->bx * geom->lx / g->gx);
    a.csy = (float)(g->by * geom->ly / g->gy);
    a.csz = (float)(g->bz * geom->lz / g->gz);
    a.inv_csx = (float)(g->gx / (g->bx * geom->lx));
    a.hcy = (float)(0.5 * g->gy / g->by);
    a.hcz = (float)(0.5 * g->gz / g->bz);
    a.inv_csy = (float)(g->gy / (g->by * geom->ly));
    a.inv_csz = (float)(g->gz / (g->bz * geom->lz));
    a.ks_over_ke = (float)(g->k_sca / g->k_ext);
    a.mu_a = (float)g->mu_a;
}

}  // namespace

size_t mc_grid_workspace_bytes(const mc_grid *g)
{
    int mx, my, mz;
    if (!grid_dims(g, &mx, &my, &mz)) return 0;
    return pad16(sizeof(float) * 2 * (size_t)g->gx * g->gy * g->gz) + pad16(sizeof(float) * (size_t)mx * my * mz);
}

mc_status mc_grid_prepare(const mc_grid *g, const mc_geometry *geom, void *d_work, size_t work_bytes,
                          void *stream)
{
    int mx, my, mz;
    mc_status s;
    if (!grid_dims(g, &mx, &my, &mz) || !g->d_density || !aligned(g->d_density, 4) || !d_work ||
        !aligned(d_work, 16))
        return MC_ERR_ARG;
    if ((s = check_geom(geom)) != MC_OK) return s;
    if (work_bytes < mc_grid_workspace_bytes(g)) return MC_ERR_NOMEM;
    unsigned char *w = static_cast<unsigned char *>(d_work);
    float2 *cells = reinterpret_cast<float2 *>(w);
    float *maj = reinterpret_cast<float *>(w + pad16(sizeof(float) * 2 * (size_t)g->gx * g->gy * g->gz));
    const cudaError_t e = mcx::launch_grid_prepare(g->d_density, g->gx, g->gy, g->gz, g->bx, g->by, g->bz,
                                                   (float)g->k_ext, (float)g->mu_a, geom->ly / g->gy, cells,
                                                   maj, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}

mc_status mc_run_grid(const mc_grid *g, const void *d_grid_work, const mc_medium *phase,
                      const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                      const mc_tallies *tallies, void *d_trace, int n_trace, int n_events, void *stream)
{
    int mx, my, mz;
    mc_status s;
    if (!grid_dims(g, &mx, &my, &mz) || !d_grid_work || !aligned(d_grid_work, 16) || !phase) return MC_ERR_ARG;
    // the phase part of the medium; its coefficients are placeholders
    mc_medium m = *phase;
    m.mu_s = 1.0;
    m.mu_a = 0.0;
    if ((s = validate_all(&m, geom, camera, run)) != MC_OK) return s;
    if ((s = check_tallies(tallies, camera)) != MC_OK) return s;
    if (d_trace && (n_trace < 1 || n_events < 1 || n_events > 1 << 20 || !aligned(d_trace, 4) ||
                    (uint64_t)n_trace > run->n_photons))
        return MC_ERR_ARG;
    mcx::GridArgs a;
    fill_grid(a, g, mx, my, mz, d_grid_work, &m, geom, camera, run, tallies->d_error, tallies->d_image,
              tallies->d_radial, tallies->d_totals);
    a.counter = reinterpret_cast<unsigned long long *>(tallies->d_work);
    a.c.trace = static_cast<int32_t *>(d_trace);
    a.c.n_trace = d_trace ? n_trace : 0;
    a.c.n_trace_events = d_trace ? n_events : 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t npix = (size_t)camera->nx * camera->nz;
    auto fail = [](cudaError_t x) { return x != cudaSuccess; };
    // refused before anything is queued when the shared-memory plan does not fit
    const cudaError_t pe = mcx::check_plan(a.c, launch_cfg(run));
    if (pe != cudaSuccess) return pe == cudaErrorInvalidValue ? MC_ERR_ARG : MC_ERR_CUDA;
    if (fail(cudaMemsetAsync(tallies->d_work, 0, sizeof(unsigned long long), st))) return MC_ERR_CUDA;
    if (!run->accumulate) {
        if (fail(cudaMemsetAsync(tallies->d_image, 0, sizeof(int64_t) * npix, st)) ||
            fail(cudaMemsetAsync(tallies->d_radial, 0, sizeof(int64_t) * camera->n_radial, st)) ||
            fail(cudaMemsetAsync(tallies->d_totals, 0, sizeof(int64_t) * MC_N_TOTALS, st)))
            return MC_ERR_CUDA;
    }
    if (d_trace && fail(cudaMemsetAsync(d_trace, 0xFF, sizeof(int32_t) * 12 * (size_t)n_trace * n_events, st)))
        return MC_ERR_CUDA;
    if (run->n_photons == 0) return MC_OK;
    return cuda_status(mcx::launch_grid(a, d_trace != nullptr, launch_cfg(run), st));
}

size_t mc_grid_adjoint_workspace_bytes(const mc_grid *g)
{
    int mx, my, mz;
    if (!grid_dims(g, &mx, &my, &mz)) return 0;
    const int rows = mcx::grid_adjoint_max_grid();
    if (rows < 1) return 0;
    const size_t n = (size_t)g->gx * g->gy * g->gz;
    // voxel sum, column sources, first-flight row entries
    return kAlign + 3 * up(sizeof(double) * n) + up(sizeof(double) * (size_t)rows);
}

// Voxels in the null-score gradient's box around the beam axis: all x, the
// central min(kNullBox, gy, gz) voxels along y and z.
static size_t null_box(const mc_grid *g)
{
    const size_t bw = (size_t)std::min(mcx::kNullBox, std::min(g->gy, g->gz));
    return (size_t)g->gx * bw * bw;
}

size_t mc_grid_adjoint_nulls_workspace_bytes(const mc_grid *g)
{
    int mx, my, mz;
    if (!grid_dims(g, &mx, &my, &mz)) return 0;
    const int rows = mcx::grid_adjoint_max_grid();
    if (rows < 1) return 0;
    const size_t n = (size_t)g->gx * g->gy * g->gz;
    // the voxel sum and the column sources, and kNullCopies copies of each
    // over the box around the beam axis
    return kAlign + 2 * up(sizeof(double) * n) + 2 * (size_t)mcx::kNullCopies * up(sizeof(double) * null_box(g)) +
           up(sizeof(double) * (size_t)rows);
}

namespace {
mc_status grid_adjoint_common(const mc_grid *g, const void *d_grid_work, const mc_medium *phase,
                              const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                              const float *d_adj_image, float *d_grad, double *d_value, uint32_t *d_error,
                              void *d_work, size_t work_bytes, void *stream, int nulls, double maj_scale);
}  // namespace

mc_status mc_grid_adjoint(const mc_grid *g, const void *d_grid_work, const mc_medium *phase,
                          const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                          const float *d_adj_image, float *d_grad, double *d_value, uint32_t *d_error,
                          void *d_work, size_t work_bytes, void *stream)
{
    return grid_adjoint_common(g, d_grid_work, phase, geom, camera, run, d_adj_image, d_grad, d_value, d_error,
                               d_work, work_bytes, stream, 0, 1.0);
}

mc_status mc_grid_adjoint_nulls(const mc_grid *g, const void *d_grid_work, const mc_medium *phase,
                                const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                                const float *d_adj_image, double majorant_scale, float *d_grad, double *d_value,
                                uint32_t *d_error, void *d_work, size_t work_bytes, void *stream)
{
    if (!fin(majorant_scale) || !(majorant_scale > 1.0) || majorant_scale > 16.0) return MC_ERR_ARG;
    return grid_adjoint_common(g, d_grid_work, phase, geom, camera, run, d_adj_image, d_grad, d_value, d_error,
                               d_work, work_bytes, stream, 1, majorant_scale);
}

namespace {
mc_status grid_adjoint_common(const mc_grid *g, const void *d_grid_work, const mc_medium *phase,
                              const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                              const float *d_adj_image, float *d_grad, double *d_value, uint32_t *d_error,
                              void *d_work, size_t work_bytes, void *stream, int nulls, double maj_scale)
{
    int mx, my, mz;
    mc_status s;
    if (!grid_dims(g, &mx, &my, &mz) || !d_grid_work || !aligned(d_grid_work, 16) || !phase || !d_adj_image ||
        !d_grad || !d_value || !d_error || !d_work || !aligned(d_adj_image, 4) || !aligned(d_grad, 4) ||
        !aligned(d_value, 8) || !aligned(d_work, 16))
        return MC_ERR_ARG;
    mc_medium m = *phase;
    m.mu_s = 1.0;
    m.mu_a = 0.0;
    if ((s = validate_all(&m, geom, camera, run)) != MC_OK) return s;
    const size_t need = nulls ? mc_grid_adjoint_nulls_workspace_bytes(g) : mc_grid_adjoint_workspace_bytes(g);
    if (!need) return MC_ERR_CUDA;
    if (work_bytes < need) return MC_ERR_NOMEM;
    const size_t n = (size_t)g->gx * g->gy * g->gz;
    unsigned char *w = static_cast<unsigned char *>(d_work);
    mcx::GridAdjArgs a;
    std::memset(&a, 0, sizeof a);
    fill_grid(a.g, g, mx, my, mz, d_grid_work, &m, geom, camera, run, d_error, nullptr, nullptr, nullptr);
    const size_t nb = up(sizeof(double) * n);
    // exact: s1, ex, gsum; null scores: s1, gsum, then the box copies of s1
    // and of gsum
    const int bw = std::min(mcx::kNullBox, std::min(g->gy, g->gz));
    const size_t bb = up(sizeof(double) * null_box(g));
    const size_t region = nulls ? 2 * nb + 2 * (size_t)mcx::kNullCopies * bb : 3 * nb;
    a.g.counter = reinterpret_cast<unsigned long long *>(w);
    a.s1 = reinterpret_cast<double *>(w + kAlign);
    a.ex = nulls ? nullptr : reinterpret_cast<double *>(w + kAlign + nb);
    a.gsum = reinterpret_cast<double *>(w + kAlign + (nulls ? 1 : 2) * nb);
    a.bs1 = nulls ? reinterpret_cast<double *>(w + kAlign + 2 * nb) : nullptr;
    a.bgs = nulls ? reinterpret_cast<double *>(w + kAlign + 2 * nb + mcx::kNullCopies * bb) : nullptr;
    a.copies = nulls ? mcx::kNullCopies : 1;
    a.bw = nulls ? bw : 0;
    a.by0 = g->gy / 2 - bw / 2;   // centred on the beam axis (y = z = 0)
    a.bz0 = g->gz / 2 - bw / 2;
    a.nbox = null_box(g);
    a.bstride = bb / sizeof(double);
    a.partials = reinterpret_cast<double *>(w + kAlign + region);
    a.adj = d_adj_image;
    a.grad = d_grad;
    a.k_ext = (float)g->k_ext;
    a.nulls = nulls;
    a.maj_scale = (float)maj_scale;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto fail = [](cudaError_t x) { return x != cudaSuccess; };
    // refused before anything is queued when the table and cells do not fit
    const cudaError_t pe = mcx::grid_adjoint_check(a);
    if (pe != cudaSuccess) return pe == cudaErrorInvalidValue ? MC_ERR_ARG : MC_ERR_CUDA;
    if (fail(cudaMemsetAsync(w, 0, kAlign + region, st)) ||
        fail(cudaMemsetAsync(d_grad, 0, sizeof(float) * n, st)) ||
        fail(cudaMemsetAsync(d_value, 0, sizeof(double), st)))
        return MC_ERR_CUDA;
    if (run->n_photons == 0) return MC_OK;
    return cuda_status(mcx::launch_grid_adjoint(a, mcx::grid_adjoint_max_grid(), d_value, st));
}
}  // namespace
