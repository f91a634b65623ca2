// Photon random-walk kernels for sm_103a.
//
// One thread carries one photon at a time (Sec. 2.7); a warp refills lanes
// whose photon ended from a per-warp pool of photon indices, taken in chunks
// from a global counter, so lanes stay busy until the whole range is done.
// Each event draws four uniforms from Philox4x32-10 keyed by
// (seed; photon, event), so results do not depend on which thread ran which
// photon. Per event (Sec. 2.6, Sec. 3.1.3):
//   free path s = -ln(u0)/mu_ext (Eq. 15); a flight that reaches a wall
//   leaves the index-matched cuvette there; otherwise the photon collides:
//   implicit capture w <- w (1 - mu_a/mu_ext) (Eq. 16), a next-event estimate
//   for the side camera (Sec. 4.3), a polar angle from the inverse-CDF table
//   (Sec. 2.6, Sec. 3.1.2) or from H-G (Eq. 11), an azimuth uniform in
//   [0, 2 pi), the direction update, and the weight threshold with roulette.
// Tallies are 64-bit fixed point: each contribution is rounded once, and
// integer sums do not depend on order, so images are bit-reproducible.
// The table is staged into shared memory once per CTA by a bulk async copy
// (cp.async.bulk + mbarrier, bounded wait).
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "table_format.h"

namespace mcx {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int CHUNK = 128;            // photons a warp takes from the counter at once
constexpr float INV_2PI = 0.159154943091895335768883763372514f;
constexpr float W_SCALE = 4294967296.0f;   // 2^32, weight tallies
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // mbarrier polls before giving up

// Index check of the checked build (compiled with MC_CHECKED): an index
// outside [0, n) sets MC_EFLAG_BOUNDS and is clamped into range, so a wrong
// index is reported instead of read or written. The normal build returns
// the index unchanged (n and err unused, their computation dropped).
__device__ __forceinline__ int chk(int i, int n, uint32_t *err)
{
#ifdef MC_CHECKED
    if ((unsigned)i >= (unsigned)n) {
        atomicOr(err, MC_EFLAG_BOUNDS);
        return i < 0 ? 0 : n - 1;
    }
#else
    (void)n;
    (void)err;
#endif
    return i;
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): per round
//   (c0,c1,c2,c3) <- (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// then k += (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same with the round keys precomputed (rk[2i], rk[2i+1]); when rk lives
// in the kernel's parameter space the key XORs take it as an operand.
__device__ __forceinline__ uint4 philox10(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk[2 * i], lo1, hi0 ^ c.w ^ rk[2 * i + 1], lo0);
    }
    return c;
}

// Transcendentals, reciprocals and square roots of the walk. The production
// build calls the hardware approximations (log2 / ex2 / sin / cos / rsqrt /
// reciprocal units, errors of a few units in the last place); the IEEE-strict
// build (MC_STRICT) calls CUDA's accurate logf / expf / exp2f / sincosf and the
// correctly rounded division and square root instead, so that traces can be
// compared with a double-precision reference at the tightest tolerance.
__device__ __forceinline__ float mc_log(float x)
{
#ifdef MC_STRICT
    return logf(x);
#else
    return __logf(x);
#endif
}
__device__ __forceinline__ float mc_exp(float x)
{
#ifdef MC_STRICT
    return expf(x);
#else
    return __expf(x);
#endif
}
__device__ __forceinline__ float mc_exp2(float x)
{
#ifdef MC_STRICT
    return exp2f(x);
#else
    float y;   // the hardware approximation, relative error a few 1e-7
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#endif
}
__device__ __forceinline__ void mc_sincos(float x, float *s, float *c)
{
#ifdef MC_STRICT
    sincosf(x, s, c);
#else
    __sincosf(x, s, c);
#endif
}
__device__ __forceinline__ float mc_div(float a, float b)
{
#ifdef MC_STRICT
    return a / b;
#else
    return __fdividef(a, b);
#endif
}
__device__ __forceinline__ float mc_rsqrt(float x)
{
#ifdef MC_STRICT
    return 1.0f / sqrtf(x);
#else
    return rsqrtf(x);
#endif
}
// sqrt(x) for x >= 0 (0 for x <= 0)
__device__ __forceinline__ float mc_sqrt0(float x)
{
#ifdef MC_STRICT
    return x > 0.0f ? sqrtf(x) : 0.0f;
#else
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
#endif
}

// (r >> 9) 2^-23 + 2^-24, exact: the float 1 + (r>>9) 2^-23 minus (1 - 2^-24).
__device__ __forceinline__ float u01(uint32_t r)
{
    return __int_as_float(0x3F800000u | (r >> 9)) - 0.999999940395355224609375f;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ long long fix32(float w) { return __float2ll_rn(w * W_SCALE); }

// 64-bit add into shared memory as two native 32-bit atomics: the low word's
// returned old value gives the carry, which joins the high word. Exact and
// independent of the order of concurrent adds (integer addition mod 2^64).
__device__ __forceinline__ void sadd64(unsigned long long *p, long long v)
{
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)((unsigned long long)v >> 32);
    uint32_t *w = reinterpret_cast<uint32_t *>(p);
    const uint32_t old = atomicAdd(w, lo);
    const uint32_t up = hi + ((uint32_t)(old + lo) < lo ? 1u : 0u);
    if (up) atomicAdd(w + 1, up);
}

// Image pixel add: the shared-memory band keeps only the low 32 bits of each
// pixel; the contribution's high word and any wrap of the low word go to the
// pixel in global memory at once, the low words at the flush. Exact and
// order-independent (integer addition mod 2^64).
__device__ __forceinline__ void band_add(uint32_t *cell, unsigned long long *gpix, long long v)
{
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)((unsigned long long)v >> 32);
    const uint32_t old = atomicAdd(cell, lo);
    const uint32_t up = hi + ((uint32_t)(old + lo) < lo ? 1u : 0u);
    if (up) atomicAdd(gpix, (unsigned long long)up << 32);
}

// mbarrier for the table copies; initialised once per CTA by thread 0.
__device__ __forceinline__ void mbar_init(unsigned long long *mbar)
{
    const uint32_t bar = smem_u32(mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for mbarrier phase `parity` to complete, giving up after `tries`
// polls (each may suspend the thread for a bounded, hardware-defined time).
// Returns 1 when the phase completed.
__device__ __forceinline__ uint32_t mbar_wait(uint32_t bar, uint32_t parity, uint32_t tries)
{
    uint32_t done = 0;
    for (uint32_t it = 0; it < tries && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
    }
    return done;
}

// Bulk-copy `bytes` (multiple of 16) from global to shared memory and wait
// (bounded) for the mbarrier phase `parity` to complete. Every thread of the
// CTA must call it; the previous contents of dst must no longer be in use.
__device__ bool stage_bulk(void *dst, const void *src, uint32_t bytes, unsigned long long *mbar,
                           uint32_t parity, uint32_t *err)
{
    const uint32_t bar = smem_u32(mbar);
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(bar)
            : "memory");
    }
    const uint32_t done = mbar_wait(bar, parity, WAIT_LIMIT);
    if (!done && threadIdx.x == 0) atomicOr(err, MC_EFLAG_TIMEOUT);
    return __syncthreads_and(done) != 0;
}

// Table bin j with omu[j] >= omu_c > omu[j+1], i.e. icdf[j] <= mu_c < icdf[j+1].
__device__ __forceinline__ int table_bin(const float *omu, const uint16_t *guide, int n, float muc)
{
    muc = fminf(fmaxf(muc, -1.0f), 1.0f);
    const int cell = min(__float2int_rd((muc + 1.0f) * (0.5f * n)), n - 1);
    int lo = guide[cell], hi = guide[cell + 1];   // exact bracket (host-built)
    const float om = 1.0f - muc;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (omu[mid] >= om) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool TRACE>
__device__ __forceinline__ void trace_write(const CommonArgs &C, unsigned long long rel, uint32_t ev,
                                            int status, float rx, float ry, float rz, float dx,
                                            float dy, float dz, float w, float nee, int pix, int nb,
                                            int rb)
{
    if (!TRACE) return;
    if (rel >= (unsigned long long)C.n_trace || ev >= (uint32_t)C.n_trace_events) return;
    int32_t *t = C.trace + (rel * C.n_trace_events + ev) * 12;
    t[0] = status;
    t[1] = __float_as_int(rx); t[2] = __float_as_int(ry); t[3] = __float_as_int(rz);
    t[4] = __float_as_int(dx); t[5] = __float_as_int(dy); t[6] = __float_as_int(dz);
    t[7] = __float_as_int(w);
    t[8] = __float_as_int(nee);
    t[9] = pix; t[10] = nb; t[11] = rb;
}

// Shared memory of a walk CTA:
//   [table blob][image band][radial][totals][mbarrier][item][pool]
// and the views of the staged table: omu / pdf / guide of the inverse-CDF
// table, or, for the paper's table, omu (node 1 - cos theta), pdf (density
// per radian), pk / pdl / pri (search thresholds and interpolation aids).
struct Smem {
    unsigned char *table;
    uint32_t *img;            // low 32 bits of the privatised image pixels
    unsigned long long *rad, *tot, *bar, *item, *pool;
    int npix;                 // privatised image pixels (band rows x nx)
    const float *omu, *pdf;
    const uint16_t *guide;
    const uint32_t *pk;
    const float *pdl, *pri;
    const uint16_t *pgq, *pgo; // guides of the paper table's two searches
    int pn;                   // intervals of the paper table
    float pinv;               // 1 / intervals
};

// ---------------------------------------------------------------- physics
// Shared by the forward walk and the adjoint replay so both compute the very
// same single-precision values.

// Largest i in [g[cell], g[cell + 1]] with a[i] <= v, for nondecreasing a
// and a guide whose bracket is known to hold the answer: the bisection of
// the whole table narrowed to that bracket (most brackets hold one entry).
template <class T>
__device__ __forceinline__ int guided_search(const T *a, const uint16_t *g, int cell, T v)
{
    int lo = g[cell], hi = g[cell + 1];
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Phase density per steradian for the camera direction cosine d_y.
template <int PHASE>
__device__ __forceinline__ float camera_psr(const MediumArgs &M, const CommonArgs &C, const Smem &S,
                                            float dy, int &nb)
{
    if (PHASE == MC_PHASE_HG) {
        // Eq. 11 per steradian, K t^(-3/2) with t = (1-g)^2 + 2g(1 - mu)
        const float t = fmaf(M.hg_two_g, 1.0f - dy, M.hg_a2);
        const float r = mc_rsqrt(t);
        nb = -1;
        return M.hg_K * (r * r * r);
    }
    if (PHASE == MC_PHASE_PAPER) {
        // uniform in theta on each interval: density per radian / sin(theta)
        const float om = 1.0f - fminf(fmaxf(dy, -1.0f), 1.0f);
        const int cell = min(__float2int_rd(om * (0.5f * MC_PAPER_GUIDE)), MC_PAPER_GUIDE - 1);   // exact product
        nb = chk(guided_search(S.omu, S.pgo, cell, om), S.pn, C.error);
        const float st2 = om * (2.0f - om);
        return st2 > 0.0f ? S.pdf[nb] * mc_rsqrt(st2) * INV_2PI : 0.0f;
    }
    nb = chk(table_bin(S.omu, S.guide, C.n_bins, dy), C.n_bins, C.error);
    return S.pdf[nb] * INV_2PI;
}

// Index of the cell of size 1/inv holding coordinate r on an axis centred at
// 0 that `half` cells cover on either side: floor(r inv + half) with one
// rounding. A point on the axis lands in cell `half` whatever the axis length
// (half = n/2 is exact), as the reading of ties on the centre plane fixes; the
// form (r + l/2) inv would round both l/2 and inv first and could give
// half - 1 there, where a pencil beam puts every first collision.
__device__ __forceinline__ int centred_cell(float r, float inv, float half, int n)
{
    return min(max(__float2int_rd(fmaf(r, inv, half)), 0), n - 1);
}

// Camera pixel of a collision at (rx, rz).
__device__ __forceinline__ int camera_pixel(const CommonArgs &C, float rx, float rz, int &ix, int &iz)
{
    ix = min(max(__float2int_rd(rx * C.sx), 0), C.nx - 1);
    iz = centred_cell(rz, C.sz, 0.5f * (float)C.nz, C.nz);
    return chk(iz * C.nx + ix, C.nx * C.nz, C.error);
}

// The same for a collision the caller has tested to lie inside: 0 < rx, so
// the column's product is >= 0 and only its upper clamp (rounding at the far
// edge) can act.
__device__ __forceinline__ int camera_pixel_inside(const CommonArgs &C, float rx, float rz, int &ix, int &iz)
{
    ix = min(__float2int_rd(rx * C.sx), C.nx - 1);
    iz = centred_cell(rz, C.sz, 0.5f * (float)C.nz, C.nz);
    return chk(iz * C.nx + ix, C.nx * C.nz, C.error);
}

// Polar angle as 1 - cos(theta) (accurate near the forward peak).
template <int PHASE>
__device__ __forceinline__ float sample_omu(const MediumArgs &M, const CommonArgs &C, const Smem &S,
                                            float u1)
{
    if (PHASE == MC_PHASE_HG) {
        const float D = fmaf(M.hg_two_g, u1, M.hg_one_m_g);
        return mc_div(M.hg_A * (1.0f - u1) * fmaf(M.hg_g, u1, 1.0f), D * D);
    }
    if (PHASE == MC_PHASE_PAPER) {
        // bisection of the cumulative distribution on the uniform's integer
        // index q (u1 = (q + 1/2) 2^-23 exactly), then linear interpolation
        // in theta: u1 - cdf_i = (q - k_i) 2^-23 + dl_i, fraction = that / w_i
        const int q = __float2int_rd(u1 * 8388608.0f);
        const int i = chk(guided_search(S.pk, S.pgq, q / (8388608 / MC_PAPER_GUIDE),
                                        (uint32_t)q), S.pn, C.error);
        const float fr = fminf(fmaxf(fmaf((float)(q - (int)S.pk[i]), 1.1920928955078125e-7f, S.pdl[i]) *
                                         S.pri[i], 0.0f), 1.0f);
        const float sh = sinpif(0.5f * ((float)i + fr) * S.pinv);   // sin(theta / 2)
        return 2.0f * sh * sh;
    }
    const float tt = u1 * (float)C.n_bins;
    const int i = chk((int)tt, C.n_bins, C.error);
    const float f = tt - (float)i;
    const float o0 = S.omu[i], o1 = S.omu[i + 1];
    return fmaf(f, o1 - o0, o0);
}

// 1 + cos(theta) of the H-G angle that sample_omu draws from the same u1:
// Eq. 11 inverted as 2 (1+g)^2 u1 (1 - g + g u1) / (1 - g + 2 g u1)^2.
__device__ __forceinline__ float hg_opu(const MediumArgs &M, float u1)
{
    const float D = fmaf(M.hg_two_g, u1, M.hg_one_m_g);
    return mc_div(M.hg_B * u1 * fmaf(M.hg_g, u1, M.hg_one_m_g), D * D);
}

// d <- mu d + sin(theta) (cos phi e1 + sin phi e2), (e1, e2) the orthonormal
// basis of Duff et al. (2017) around d, phi = 2 pi u2; renormalised.
__device__ __forceinline__ void rotate_cs(float &dx, float &dy, float &dz, float mu, float st2, float u2)
{
    const float st = mc_sqrt0(st2);
    // phi = 2 pi u2 through the hardware sine / cosine, evaluated at
    // phi - pi in [-pi, pi) where they are most accurate
    float sp, cp;
    mc_sincos(fmaf(6.28318530717958647692f, u2, -3.14159265358979323846f), &sp, &cp);
    sp = -sp;
    cp = -cp;
    const float sg = copysignf(1.0f, dz);
    const float a = mc_div(-1.0f, sg + dz);
    const float b = dx * dy * a;
    const float e1x = fmaf(sg * dx * dx, a, 1.0f), e1y = sg * b, e1z = -sg * dx;
    const float e2x = b, e2y = fmaf(dy * dy, a, sg), e2z = -dy;
    const float qx = fmaf(cp, e1x, sp * e2x), qy = fmaf(cp, e1y, sp * e2y), qz = fmaf(cp, e1z, sp * e2z);
    const float nx = fmaf(mu, dx, st * qx), ny = fmaf(mu, dy, st * qy), nz = fmaf(mu, dz, st * qz);
    const float inv = mc_rsqrt(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    dx = nx * inv; dy = ny * inv; dz = nz * inv;
}

// New direction at polar angle theta given as om = 1 - cos(theta).
__device__ __forceinline__ void rotate(float &dx, float &dy, float &dz, float om, float u2)
{
    rotate_cs(dx, dy, dz, 1.0f - om, om * (2.0f - om), u2);
}

// The same given om = 1 - cos(theta) and op = 1 + cos(theta), each from its
// own closed form: cos(theta) from the smaller of the two and sin^2 = om op,
// so a direction near theta = pi keeps its accuracy (2 - om, formed from a
// rounded om close to 2, would not).
__device__ __forceinline__ void rotate_hg(float &dx, float &dy, float &dz, float om, float op, float u2)
{
    rotate_cs(dx, dy, dz, om <= op ? 1.0f - om : op - 1.0f, om * op, u2);
}

// Scattering: draw the polar angle with u1 and turn the direction (azimuth
// from u2).
template <int PHASE>
__device__ __forceinline__ void scatter(const MediumArgs &M, const CommonArgs &C, const Smem &S, float u1, float u2,
                                        float &dx, float &dy, float &dz)
{
    const float om = sample_omu<PHASE>(M, C, S, u1);
    if (PHASE == MC_PHASE_HG) rotate_hg(dx, dy, dz, om, hg_opu(M, u1), u2);
    else rotate(dx, dy, dz, om, u2);
}

template <int PHASE, bool SMEM_IMAGE>
__device__ __forceinline__ Smem carve(unsigned char *smem, const CommonArgs &C)
{
    Smem S;
    const uint32_t tb = (PHASE != MC_PHASE_HG) ? C.table_bytes : 0u;
    S.table = smem;
    S.npix = SMEM_IMAGE ? C.nx * C.band_rows : 0;
    S.img = reinterpret_cast<uint32_t *>(smem + tb + C.extra_bytes);
    S.rad = reinterpret_cast<unsigned long long *>(smem + tb + C.extra_bytes +
                                                   ((sizeof(uint32_t) * (size_t)S.npix + 15) & ~(size_t)15));
    S.tot = S.rad + C.n_radial;
    S.bar = S.tot + MC_N_TOTALS;
    S.item = S.bar + 1;
    S.pool = S.item + 1;
    S.omu = S.pdf = S.pdl = S.pri = nullptr;
    S.guide = nullptr;
    S.pk = nullptr;
    S.pgq = S.pgo = nullptr;
    S.pn = 0;
    S.pinv = 0.0f;
    return S;
}

__device__ __forceinline__ void zero_tallies(const Smem &S, const CommonArgs &C)
{
    for (int i = threadIdx.x; i < S.npix; i += blockDim.x) S.img[i] = 0u;
    for (int i = threadIdx.x; i < C.n_radial + MC_N_TOTALS; i += blockDim.x) S.rad[i] = 0ull;
}

// Table pointers into the staged blob; false (and the error flag) if its
// header does not describe the expected table.
template <int PHASE>
__device__ __forceinline__ bool bind_table(Smem &S, const CommonArgs &C)
{
    if (PHASE == MC_PHASE_PAPER) {
        const mc_paper_header *h = reinterpret_cast<const mc_paper_header *>(S.table);
        if (h->magic != MC_PAPER_MAGIC || h->version != MC_PAPER_VERSION || h->n_theta != C.n_bins ||
            h->total_bytes != C.table_bytes) {
            if (threadIdx.x == 0) atomicOr(C.error, MC_EFLAG_TABLE);
            return false;
        }
        S.pk = reinterpret_cast<const uint32_t *>(S.table + h->off_k);
        S.pdl = reinterpret_cast<const float *>(S.table + h->off_dl);
        S.pri = reinterpret_cast<const float *>(S.table + h->off_ri);
        S.omu = reinterpret_cast<const float *>(S.table + h->off_omu);
        S.pdf = reinterpret_cast<const float *>(S.table + h->off_pth);
        S.pgq = reinterpret_cast<const uint16_t *>(S.table + h->off_gq);
        S.pgo = reinterpret_cast<const uint16_t *>(S.table + h->off_go);
        S.pn = h->n_int;
        S.pinv = 1.0f / (float)h->n_int;
        return true;
    }
    const mc_table_header *h = reinterpret_cast<const mc_table_header *>(S.table);
    if (h->magic != MC_TABLE_MAGIC || h->n_bins != C.n_bins || h->total_bytes != C.table_bytes) {
        if (threadIdx.x == 0) atomicOr(C.error, MC_EFLAG_TABLE);
        return false;
    }
    S.omu = reinterpret_cast<const float *>(S.table + h->off_omu);
    S.pdf = reinterpret_cast<const float *>(S.table + h->off_pdf);
    S.guide = reinterpret_cast<const uint16_t *>(S.table + h->off_guide);
    return true;
}

// Per-thread tallies, reduced when a CTA finishes a medium.
struct Tally {
    uint32_t steps;             // flushed per medium; a thread's count per flush fits 32 bits
    long long refl, far, side, ball, abs;
};

// Warp -> shared -> the medium's global tallies (one atomic per nonzero entry).
template <bool SMEM_IMAGE>
__device__ void flush(const CommonArgs &C, const MediumArgs &M, const Smem &S, Tally &T)
{
    unsigned long long steps = T.steps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        steps += __shfl_xor_sync(FULL, steps, o);
        T.refl += __shfl_xor_sync(FULL, T.refl, o);
        T.far += __shfl_xor_sync(FULL, T.far, o);
        T.side += __shfl_xor_sync(FULL, T.side, o);
        T.ball += __shfl_xor_sync(FULL, T.ball, o);
        T.abs += __shfl_xor_sync(FULL, T.abs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sadd64(&S.tot[MC_TOT_STEPS], (long long)steps);
        sadd64(&S.tot[MC_TOT_REFLECT], T.refl);
        sadd64(&S.tot[MC_TOT_FAR], T.far);
        sadd64(&S.tot[MC_TOT_SIDE], T.side);
        sadd64(&S.tot[MC_TOT_BALLISTIC], T.ball);
        sadd64(&S.tot[MC_TOT_ABSORB], T.abs);
    }
    T = Tally{0u, 0ll, 0ll, 0ll, 0ll, 0ll};
    __syncthreads();
    if (SMEM_IMAGE) {
        unsigned long long *g = M.image + (size_t)C.band0 * C.nx;
        for (int i = threadIdx.x; i < S.npix; i += blockDim.x)
            if (S.img[i]) atomicAdd(&g[i], (unsigned long long)S.img[i]);
    }
    for (int i = threadIdx.x; i < C.n_radial; i += blockDim.x)
        if (S.rad[i]) atomicAdd(&M.radial[i], S.rad[i]);
    for (int i = threadIdx.x; i < MC_N_TOTALS; i += blockDim.x)
        if (S.tot[i]) atomicAdd(&M.totals[i], S.tot[i]);
    __syncthreads();
}

// The photon walk over indices [.., limit) of medium M: every warp refills
// lanes whose photon ended from chunks of `chunk` indices obtained by
// grab() (called by lane 0), until the range is exhausted.
// rk: the Philox round keys of M's seed (M.rk, or a copy of them).
template <int PHASE, bool SMEM_IMAGE, bool TRACE, class Grab>
__device__ __forceinline__ void walk_loop(const CommonArgs &C, const MediumArgs &M, const uint32_t (&rk)[20],
                                          const Smem &S, unsigned long long limit, unsigned chunk, Grab grab,
                                          Tally &T)
{
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    unsigned long long pool_next = 0, pool_end = 0;  // warp-uniform
    // camera transmittance exp(-mu_ext (ly/2 - r_y)) = 2^(cam_a r_y + cam_b)
    const float cam_a = M.mu_ext * 1.44269504088896340736f, cam_b = -cam_a * C.hy;
    uint32_t *s_img = S.img;
    unsigned long long *s_rad = S.rad, *s_tot = S.tot;

    // photon state
    bool alive = false, done = false;
    unsigned long long rel = 0;     // index within the medium's range
    uint32_t pk0 = 0, pk1 = 0;      // global photon index, lo/hi words
    uint32_t ev = 0, ncoll = 0;
    float rx = 0, ry = 0, rz = 0, dx = 1, dy = 0, dz = 0, w = 1;

    while (true) {
        // -------- refill lanes whose photon ended
        const unsigned need = __ballot_sync(FULL, !alive && !done);
        if (need) {
            const unsigned n_need = __popc(need);
            const unsigned rank = __popc(need & lanemask_lt);
            const unsigned long long avail = pool_end - pool_next;
            unsigned long long mine;
            if (avail >= n_need) {
                mine = pool_next + rank;
                pool_next += n_need;
            } else {
                unsigned long long base = 0;
                if (lane == 0) base = grab();
                base = __shfl_sync(FULL, base, 0);
                mine = (rank < avail) ? pool_next + rank : base + (rank - avail);
                pool_next = base + (n_need - avail);
                pool_end = base + chunk;
            }
            if (!alive && !done) {
                if (mine < limit) {
                    rel = mine;
                    const unsigned long long p = M.photon_offset + mine;
                    pk0 = (uint32_t)p;
                    pk1 = (uint32_t)(p >> 32);
                    ev = 0;
                    ncoll = 0;
                    rx = 0.f; ry = 0.f; rz = 0.f;
                    dx = 1.f; dy = 0.f; dz = 0.f;
                    w = 1.f;
                    if (C.beam_r > 0.f) {
                        const uint4 b = philox10(make_uint4(pk0, pk1, 0xFFFFFFFFu, 0u), M.key0, M.key1);
                        const float rho = C.beam_r * sqrtf(u01(b.x));
                        float sp, cp;
                        sincospif(2.0f * u01(b.y), &sp, &cp);
                        ry = rho * cp;
                        rz = rho * sp;
                    }
                    alive = true;
                } else {
                    done = true;
                }
            }
        }
        if (!__any_sync(FULL, alive)) break;
        if (!alive) continue;

        // -------- one event
        const uint32_t e_now = ev;
        const uint4 rnd = philox10(make_uint4(pk0, pk1, e_now, 0u), rk);
        ++ev;
        ++T.steps;
        const float u0 = u01(rnd.x), u1 = u01(rnd.y), u2 = u01(rnd.z), u3 = u01(rnd.w);

        const float s = -mc_log(u0) * M.inv_mu_ext;                 // Eq. 15
        const float px = fmaf(s, dx, rx), py = fmaf(s, dy, ry), pz = fmaf(s, dz, rz);
        const bool cx = !((px > 0.f) & (px < C.lx));
        const bool cy = !(fabsf(py) < C.hy);
        const bool cz = !(fabsf(pz) < C.hz);

        if (cx | cy | cz) {
            // the flight reaches a wall: the first one crossed is the exit
            // (ties: lowest axis). Wall a comes before wall b when
            // |n_a / d_a| <= |n_b / d_b| (n: distance to the wall along the
            // axis), tested as |n_a| |d_b| <= |n_b| |d_a| without divisions (a
            // different answer than exact arithmetic needs a near tie); with one
            // wall crossed the test picks it
            const float ax = dx > 0.f ? C.lx - rx : rx, ay = dy > 0.f ? C.hy - ry : C.hy + ry;
            const float az = dz > 0.f ? C.hz - rz : C.hz + rz;
            const float bx = fabsf(dx), by = fabsf(dy), bz = fabsf(dz);
            const bool xf = cx && (!cy || ax * by <= ay * bx) && (!cz || ax * bz <= az * bx);
            const bool yf = !xf && cy && (!cz || ay * bz <= az * by);
            const int face = xf ? 0 : (yf ? 1 : 2);
            const long long wv = fix32(w);
            int status, rb = -1;
            float ex = px, ey = py, ez = pz;
            if (face == 0 && dx < 0.f) {
                T.refl += wv;
                status = 1;
            } else if (face == 0) {
                T.far += wv;
                if (ncoll == 0) T.ball += wv;
                const float t = mc_div(C.lx - rx, dx);
                ex = C.lx; ey = fmaf(t, dy, ry); ez = fmaf(t, dz, rz);
                const float r2 = fmaf(ey, ey, ez * ez);
                const float rho = mc_sqrt0(r2);
                rb = chk(min(__float2int_rd(rho * C.sr), C.n_radial - 1), C.n_radial, C.error);
                sadd64(&s_rad[rb], wv);
                status = 2;
            } else {
                T.side += wv;
                status = 3;
            }
            if (TRACE) {
                if (face != 0 || dx < 0.f) {
                    const float t = face == 0 ? (0.f - rx) / dx
                                  : face == 1 ? (dy > 0.f ? C.hy - ry : -C.hy - ry) / dy
                                              : (dz > 0.f ? C.hz - rz : -C.hz - rz) / dz;
                    ex = fmaf(t, dx, rx); ey = fmaf(t, dy, ry); ez = fmaf(t, dz, rz);
                }
                trace_write<TRACE>(C, rel, e_now, status, ex, ey, ez, dx, dy, dz, w, 0.f, -1, -1, rb);
            }
            alive = false;
            continue;
        }

        // -------- collision
        rx = px; ry = py; rz = pz;
        ++ncoll;
        {   // Eq. 16; the captured part w - w a is exact in single precision
            // for albedo a >= 1/2 (Sterbenz), so weight is conserved per photon
            const float wn = w * M.albedo;
            if (M.absorb_frac > 0.f) T.abs += fix32(w - wn);
            w = wn;
        }

        // camera: next-event estimate toward +y
        int nb, ix, iz;
        const float psr = camera_psr<PHASE>(M, C, S, dy, nb);
        const float nee = w * psr * mc_exp2(fmaf(cam_a, ry, cam_b));
        const int pix = camera_pixel_inside(C, rx, rz, ix, iz);   // 0 < rx < lx, |rz| < hz tested above
        const float vf = nee * C.img_scale;
        if (vf < 4.0e18f) {
            const long long v = __float2ll_rn(vf);
            const unsigned brow = (unsigned)(iz - C.band0);
            if (SMEM_IMAGE && brow < (unsigned)C.band_rows) band_add(&s_img[brow * C.nx + ix], &M.image[pix], v);
            else atomicAdd(&M.image[pix], (unsigned long long)v);
        } else {
            atomicOr(C.error, (vf == vf) ? MC_EFLAG_OVERFLOW : MC_EFLAG_NUMERIC);
        }

        if (TRACE) {
            int status = 0;
            if (C.max_scatter && ncoll >= C.max_scatter) {
                sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
                status = 5;
                alive = false;
            } else {
                scatter<PHASE>(M, C, S, u1, u2, dx, dy, dz);
                // weight threshold / roulette (Sec. 3.1.3)
                if (w < C.rr_thr) {
                    if (u3 < C.rr_surv) {
                        const float wn = w * C.inv_rr_surv;
                        sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w) - fix32(wn));
                        w = wn;
                    } else {
                        sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w));
                        status = 4;
                        alive = false;
                    }
                }
                if (!(w == w)) atomicOr(C.error, MC_EFLAG_NUMERIC);
            }
            trace_write<TRACE>(C, rel, e_now, status, rx, ry, rz, dx, dy, dz, status == 4 ? 0.f : w, nee,
                               pix, nb, -1);
            if (alive && ev >= C.max_events) {
                sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
                atomicOr(C.error, MC_EFLAG_EVENTS);
                trace_write<TRACE>(C, rel, ev, 6, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1, -1, -1);
                alive = false;
            }
        } else {
            // the same decisions with one branch for the rare cases: the new
            // direction is computed for every photon (a photon truncated by
            // max_scatter ends here and never uses it)
            const bool cap = C.max_scatter && ncoll >= C.max_scatter;
            scatter<PHASE>(M, C, S, u1, u2, dx, dy, dz);
            if (cap | (w < C.rr_thr) | (ev >= C.max_events) | !(w == w)) {
                if (cap) {
                    sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
                    alive = false;
                } else {
                    if (w < C.rr_thr) {   // weight threshold / roulette (Sec. 3.1.3)
                        if (u3 < C.rr_surv) {
                            const float wn = w * C.inv_rr_surv;
                            sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w) - fix32(wn));
                            w = wn;
                        } else {
                            sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w));
                            alive = false;
                        }
                    }
                    if (!(w == w)) atomicOr(C.error, MC_EFLAG_NUMERIC);
                    if (alive && ev >= C.max_events) {
                        sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
                        atomicOr(C.error, MC_EFLAG_EVENTS);
                        alive = false;
                    }
                }
            }
        }
    }
}

// One medium: the table staged once, the whole photon range from a global
// counter, tallies flushed once.
template <int PHASE, bool SMEM_IMAGE, bool TRACE>
__global__ void __launch_bounds__(1024) walk_kernel(const __grid_constant__ WalkArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Smem S = carve<PHASE, SMEM_IMAGE>(smem, A.c);
    zero_tallies(S, A.c);
    if (threadIdx.x == 0) mbar_init(S.bar);
    if (PHASE != MC_PHASE_HG) {
        if (!stage_bulk(S.table, A.m.table, A.c.table_bytes, S.bar, 0u, A.c.error)) return;
        if (!bind_table<PHASE>(S, A.c)) return;
    } else {
        __syncthreads();
    }
    Tally T{0u, 0ll, 0ll, 0ll, 0ll, 0ll};
    unsigned long long *counter = A.counter;
    walk_loop<PHASE, SMEM_IMAGE, TRACE>(A.c, A.m, A.m.rk, S, A.m.n_photons, CHUNK,
                                        [counter]() { return atomicAdd(counter, (unsigned long long)CHUNK); },
                                        T);
    flush<SMEM_IMAGE>(A.c, A.m, S, T);
}

// Many media in one launch: every CTA goes through the media in the order
// given (largest estimated cost first). Its warps take chunks of the current
// medium's photons from that medium's global counter, as in the one-medium
// launch; once the counter is exhausted and the CTA's warps have finished
// their photons, the CTA flushes its tallies into the medium's, stages the
// next medium's table and goes on. CTAs flow from one medium into the next
// without launch gaps, every medium's photons spread over all CTAs at warp-
// chunk granularity; a CTA skips a medium whose photons were all taken
// before it arrived.
template <int PHASE, bool SMEM_IMAGE>
__global__ void __launch_bounds__(1024) batch_kernel(const __grid_constant__ BatchArgs B)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Smem S = carve<PHASE, SMEM_IMAGE>(smem, B.c);
    zero_tallies(S, B.c);
    if (threadIdx.x == 0) mbar_init(S.bar);
    __syncthreads();
    Tally T{0u, 0ll, 0ll, 0ll, 0ll, 0ll};
    uint32_t parity = 0;
    const unsigned chunk = B.chunk;
    for (int m = 0; m < B.n_media; ++m) {
        // this medium's arguments, copied once: read through the dynamically
        // indexed kernel parameter, every use in the walk would be a load
        const MediumArgs M = B.m[m];
        unsigned long long *ctr = B.counters + m;
        if (threadIdx.x == 0) *S.item = *reinterpret_cast<volatile unsigned long long *>(ctr);
        __syncthreads();
        const bool taken = *S.item >= M.n_photons;
        __syncthreads();
        if (taken) continue;
        if (PHASE != MC_PHASE_HG) {
            if (!stage_bulk(S.table, M.table, B.c.table_bytes, S.bar, parity, B.c.error)) return;
            parity ^= 1u;
            if (!bind_table<PHASE>(S, B.c)) return;
        }
        // the medium's round keys, read once (warp-uniform values)
        uint32_t rk[20];
#pragma unroll
        for (int i = 0; i < 20; ++i) rk[i] = M.rk[i];
        walk_loop<PHASE, SMEM_IMAGE, false>(
            B.c, M, rk, S, M.n_photons, chunk, [ctr, chunk]() { return atomicAdd(ctr, (unsigned long long)chunk); },
            T);
        flush<SMEM_IMAGE>(B.c, M, S, T);
        zero_tallies(S, B.c);
        __syncthreads();
    }
}


// ------------------------------------------------------- heterogeneous medium
// Delta (Woodcock) tracking through a voxel grid (the complex media of
// Sec. 6's outlook). A tentative flight spends tau = -ln u0 of optical depth
// cell by cell at each cell's majorant (a DDA over the cells, majorants in
// shared memory); where tau runs out, the collision is real with probability
// mu_ext / majorant (u3), else null and the photon goes on with the next
// event's numbers. A real collision reuses u3 / (mu_ext / majorant), uniform
// on [0, 1) given acceptance, for roulette, and weights its camera term with
// the exact column transmittance exp(-(depth above the voxel + mu_ext times
// the distance to the voxel's top face)). One Philox call per tentative
// collision; the voxel's (mu_ext, depth) pair is one 8-byte gather from the
// L2-resident grid. Traces record real events only.

// One tentative flight of delta tracking: spends optical depth tau cell by
// cell at the cells' majorants (a DDA over the majorant cells in s_maj) from
// r along d (id = 1/d per axis). Returns 3 at a tentative collision (r moved
// there, mb = that cell's majorant), 0/1/2 when the flight leaves through an
// x/y/z wall first (r on the wall), -1 if no exit plane exists or more cells
// than the grid has were crossed (a non-finite direction).
__device__ __forceinline__ int grid_flight(const GridArgs &G, const float *s_maj, float tau, float &rx,
                                           float &ry, float &rz, float dx, float dy, float dz, float idx,
                                           float idy, float idz, float &mb)
{
    // Incremental DDA: distances along the flight (from its start r) to the
    // next cell plane on each axis, t0 the distance travelled so far; each
    // crossing recomputes only the crossed axis's next plane, from r. Signs
    // are selects, not branches, so lanes flying different ways stay together.
    const CommonArgs &C = G.c;
    const float INF = __int_as_float(0x7f800000);
    int cx = min(max(__float2int_rd(rx * G.inv_csx), 0), G.mx - 1);
    int cy = centred_cell(ry, G.inv_csy, G.hcy, G.my);
    int cz = centred_cell(rz, G.inv_csz, G.hcz, G.mz);
    const bool px = dx > 0.f, py = dy > 0.f, pz = dz > 0.f;
    // next plane of cell c on an axis of cell size cs, lower wall lo, upper wall hi
    auto plane = [](int c, int m, bool up, float cs, float lo, float hi) {
        return up ? (c == m - 1 ? hi : fmaf((float)(c + 1), cs, lo)) : (c == 0 ? lo : fmaf((float)c, cs, lo));
    };
    float tx = dx != 0.f ? fmaxf((plane(cx, G.mx, px, G.csx, 0.f, C.lx) - rx) * idx, 0.f) : INF;
    float ty = dy != 0.f ? fmaxf((plane(cy, G.my, py, G.csy, -C.hy, C.hy) - ry) * idy, 0.f) : INF;
    float tz = dz != 0.f ? fmaxf((plane(cz, G.mz, pz, G.csz, -C.hz, C.hz) - rz) * idz, 0.f) : INF;
    float t0 = 0.f;
    const int max_cross = G.mx + G.my + G.mz + 4;
    for (int it = 0; it < max_cross; ++it) {
        mb = s_maj[chk((cz * G.my + cy) * G.mx + cx, G.mx * G.my * G.mz, C.error)];
        const int ax = (tx <= ty && tx <= tz) ? 0 : (ty <= tz ? 1 : 2);
        const float t1 = fmaxf(ax == 0 ? tx : (ax == 1 ? ty : tz), t0);
        if (mb * (t1 - t0) > tau) {
            const float sl = t0 + mc_div(tau, mb);
            rx = fmaf(sl, dx, rx); ry = fmaf(sl, dy, ry); rz = fmaf(sl, dz, rz);
            return 3;
        }
        if (!(t1 < INF)) return -1;
        tau = fmaf(-mb, t1 - t0, tau);
        t0 = t1;
        if (ax == 0) {
            cx += px ? 1 : -1;
            if (cx < 0 || cx >= G.mx) {
                ry = fmaf(t1, dy, ry); rz = fmaf(t1, dz, rz); rx = px ? C.lx : 0.f;
                return 0;
            }
            tx = fmaxf((plane(cx, G.mx, px, G.csx, 0.f, C.lx) - rx) * idx, t1);
        } else if (ax == 1) {
            cy += py ? 1 : -1;
            if (cy < 0 || cy >= G.my) {
                rx = fmaf(t1, dx, rx); rz = fmaf(t1, dz, rz); ry = py ? C.hy : -C.hy;
                return 1;
            }
            ty = fmaxf((plane(cy, G.my, py, G.csy, -C.hy, C.hy) - ry) * idy, t1);
        } else {
            cz += pz ? 1 : -1;
            if (cz < 0 || cz >= G.mz) {
                rx = fmaf(t1, dx, rx); ry = fmaf(t1, dy, ry); rz = pz ? C.hz : -C.hz;
                return 2;
            }
            tz = fmaxf((plane(cz, G.mz, pz, G.csz, -C.hz, C.hz) - rz) * idz, t1);
        }
    }
    return -1;
}

template <int PHASE, bool SMEM_IMAGE, bool TRACE>
__device__ __forceinline__ void grid_loop(const GridArgs &G, const Smem &S, const float *s_maj, Tally &T)
{
    const CommonArgs &C = G.c;
    const MediumArgs &M = G.m;
    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    unsigned long long pool_next = 0, pool_end = 0;
    uint32_t *s_img = S.img;
    unsigned long long *s_rad = S.rad, *s_tot = S.tot;
    const float INF = __int_as_float(0x7f800000);

    bool alive = false, done = false;
    unsigned long long rel = 0;
    uint32_t pk0 = 0, pk1 = 0, ev = 0, ncoll = 0;
    float rx = 0, ry = 0, rz = 0, dx = 1, dy = 0, dz = 0, w = 1;
    float idx = 1, idy = INF, idz = INF;   // 1 / d (infinite along an axis d does not move on)

    while (true) {
        const unsigned need = __ballot_sync(FULL, !alive && !done);
        if (need) {
            const unsigned n_need = __popc(need), rank = __popc(need & lanemask_lt);
            const unsigned long long avail = pool_end - pool_next;
            unsigned long long mine;
            if (avail >= n_need) {
                mine = pool_next + rank;
                pool_next += n_need;
            } else {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(G.counter, (unsigned long long)CHUNK);
                base = __shfl_sync(FULL, base, 0);
                mine = (rank < avail) ? pool_next + rank : base + (rank - avail);
                pool_next = base + (n_need - avail);
                pool_end = base + CHUNK;
            }
            if (!alive && !done) {
                if (mine < M.n_photons) {
                    rel = mine;
                    const unsigned long long p = M.photon_offset + mine;
                    pk0 = (uint32_t)p;
                    pk1 = (uint32_t)(p >> 32);
                    ev = 0;
                    ncoll = 0;
                    rx = 0.f; ry = 0.f; rz = 0.f;
                    dx = 1.f; dy = 0.f; dz = 0.f;
                    idx = 1.f; idy = INF; idz = INF;
                    w = 1.f;
                    if (C.beam_r > 0.f) {
                        const uint4 b = philox10(make_uint4(pk0, pk1, 0xFFFFFFFFu, 0u), M.key0, M.key1);
                        const float rho = C.beam_r * sqrtf(u01(b.x));
                        float sp, cp;
                        sincospif(2.0f * u01(b.y), &sp, &cp);
                        ry = rho * cp;
                        rz = rho * sp;
                    }
                    alive = true;
                } else {
                    done = true;
                }
            }
        }
        if (!__any_sync(FULL, alive)) break;
        if (!alive) continue;

        if (ev >= C.max_events) {
            sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
            atomicOr(C.error, MC_EFLAG_EVENTS);
            trace_write<TRACE>(C, rel, ncoll, 6, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1, -1, -1);
            alive = false;
            continue;
        }
        const uint4 rnd = philox10(make_uint4(pk0, pk1, ev, 0u), M.rk);
        ++ev;
        ++T.steps;
        const float u1 = u01(rnd.y), u2 = u01(rnd.z);
        float u3 = u01(rnd.w);

        // -------- one tentative flight
        float mb = 0.f;
        const int face = grid_flight(G, s_maj, -mc_log(u01(rnd.x)), rx, ry, rz, dx, dy, dz, idx, idy, idz, mb);
        const bool hit = face == 3;
        if (face < 0) {
            // a non-finite direction or more crossings than cells: give up on
            // the photon and say so
            atomicOr(C.error, MC_EFLAG_NUMERIC);
            sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
            alive = false;
            continue;
        }
        if (!hit) {
            const long long wv = fix32(w);
            int status, rb = -1;
            if (face == 0 && dx < 0.f) {
                T.refl += wv;
                status = 1;
            } else if (face == 0) {
                T.far += wv;
                if (ncoll == 0) T.ball += wv;
                const float r2 = fmaf(ry, ry, rz * rz);
                const float rho = mc_sqrt0(r2);
                rb = chk(min(__float2int_rd(rho * C.sr), C.n_radial - 1), C.n_radial, C.error);
                sadd64(&s_rad[rb], wv);
                status = 2;
            } else {
                T.side += wv;
                status = 3;
            }
            trace_write<TRACE>(C, rel, ncoll, status, rx, ry, rz, dx, dy, dz, w, 0.f, -1, -1, rb);
            alive = false;
            continue;
        }

        // -------- tentative collision: real with probability mu_ext / majorant
        const int ix = min(max(__float2int_rd(rx * G.inv_vx), 0), G.gx - 1);
        const int iy = centred_cell(ry, G.inv_vy, 0.5f * (float)G.gy, G.gy);
        const int iz = centred_cell(rz, G.inv_vz, 0.5f * (float)G.gz, G.gz);
        const float2 cell = __ldg(&G.cells[chk((iz * G.gy + iy) * G.gx + ix, G.gx * G.gy * G.gz, C.error)]);
        const float acc = mc_div(cell.x, mb);   // hardware reciprocal (a few ulp) unless strict
        if (!(u3 < acc)) continue;   // null collision
        u3 = mc_div(u3, acc);
        ++ncoll;
        {   // Eq. 16 with the voxel's albedo
            const float a = G.mu_a > 0.f ? G.ks_over_ke * (1.0f - mc_div(G.mu_a, cell.x)) : G.ks_over_ke;
            const float wn = w * a;
            if (a < 1.0f) T.abs += fix32(w - wn);
            w = wn;
        }
        int nb, pix_x, pix_z;
        const float psr = camera_psr<PHASE>(M, C, S, dy, nb);
        const float top = (iy == G.gy - 1) ? C.hy : fmaf((float)(iy + 1), G.vy, -C.hy);
        const float nee = w * psr * mc_exp(-fmaf(cell.x, top - ry, cell.y));
        const int pix = camera_pixel(C, rx, rz, pix_x, pix_z);
        const float vf = nee * C.img_scale;
        if (vf < 4.0e18f) {
            const long long v = __float2ll_rn(vf);
            const unsigned brow = (unsigned)(pix_z - C.band0);
            if (SMEM_IMAGE && brow < (unsigned)C.band_rows) band_add(&s_img[brow * C.nx + pix_x], &M.image[pix], v);
            else atomicAdd(&M.image[pix], (unsigned long long)v);
        } else {
            atomicOr(C.error, (vf == vf) ? MC_EFLAG_OVERFLOW : MC_EFLAG_NUMERIC);
        }
        if (TRACE) {
            int status = 0;
            if (C.max_scatter && ncoll >= C.max_scatter) {
                sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
                status = 5;
                alive = false;
            } else {
                scatter<PHASE>(M, C, S, u1, u2, dx, dy, dz);
                idx = mc_div(1.0f, dx); idy = mc_div(1.0f, dy); idz = mc_div(1.0f, dz);
                if (w < C.rr_thr) {
                    if (u3 < C.rr_surv) {
                        const float wn = w * C.inv_rr_surv;
                        sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w) - fix32(wn));
                        w = wn;
                    } else {
                        sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w));
                        status = 4;
                        alive = false;
                    }
                }
                if (!(w == w)) atomicOr(C.error, MC_EFLAG_NUMERIC);
            }
            trace_write<TRACE>(C, rel, ncoll - 1, status, rx, ry, rz, dx, dy, dz, status == 4 ? 0.f : w, nee,
                               pix, nb, -1);
        } else {
            // one branch for the rare cases, as in walk_loop
            const bool cap = C.max_scatter && ncoll >= C.max_scatter;
            scatter<PHASE>(M, C, S, u1, u2, dx, dy, dz);
            idx = mc_div(1.0f, dx); idy = mc_div(1.0f, dy); idz = mc_div(1.0f, dz);
            if (cap | (w < C.rr_thr) | !(w == w)) {
                if (cap) {
                    sadd64(&s_tot[MC_TOT_TRUNC], fix32(w));
                    alive = false;
                } else {
                    if (w < C.rr_thr) {
                        if (u3 < C.rr_surv) {
                            const float wn = w * C.inv_rr_surv;
                            sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w) - fix32(wn));
                            w = wn;
                        } else {
                            sadd64(&s_tot[MC_TOT_ROULETTE], fix32(w));
                            alive = false;
                        }
                    }
                    if (!(w == w)) atomicOr(C.error, MC_EFLAG_NUMERIC);
                }
            }
        }
    }
}

template <int PHASE, bool SMEM_IMAGE, bool TRACE>
__global__ void __launch_bounds__(1024) grid_kernel(const __grid_constant__ GridArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Smem S = carve<PHASE, SMEM_IMAGE>(smem, A.c);
    zero_tallies(S, A.c);
    if (threadIdx.x == 0) mbar_init(S.bar);
    const uint32_t tb = (PHASE != MC_PHASE_HG) ? A.c.table_bytes : 0u;
    float *s_maj = reinterpret_cast<float *>(smem + tb);
    uint32_t parity = 0u;
    if (PHASE != MC_PHASE_HG) {
        if (!stage_bulk(S.table, A.m.table, A.c.table_bytes, S.bar, parity, A.c.error)) return;
        parity ^= 1u;
        if (!bind_table<PHASE>(S, A.c)) return;
    }
    if (!stage_bulk(s_maj, A.maj, A.c.extra_bytes, S.bar, parity, A.c.error)) return;
    Tally T{0u, 0ll, 0ll, 0ll, 0ll, 0ll};
    grid_loop<PHASE, SMEM_IMAGE, TRACE>(A, S, s_maj, T);
    flush<SMEM_IMAGE>(A.c, A.m, S, T);
}


// ------------------------------------------------ gradient w.r.t. densities
// For a photon with real collisions r_1..r_J (entry r_0), camera terms
// A_i = adj[pix_i] c_i and B_i = A_i + .. + A_J (the terms that flight i and
// collision i precede): flight i adds B_i / n(r_i) at r_i's voxel (scattering
// density k_sca n exp(-int mu)) and -B_i k_ext times its length inside every
// voxel it crosses; camera term i adds -A_i k_ext times the length of its
// column inside every voxel above r_i: the part in r_i's own voxel directly,
// the rest gathered as the source s1 and folded by a column scan. The first
// flight runs from the entry point along +x inside one voxel row, so it is
// one entry of a row-suffix array (every voxel before the collision's takes
// the full voxel length). A photon runs twice on its Philox counters: the
// first pass sums its camera terms, the second replays it and scatters the
// terms. Roulette factors are held fixed. Every term is formed in single
// precision and summed by double-precision atomics in L2; the SM's own
// double-precision pipe, a small fraction of the single-precision rate,
// is not used on this path.
constexpr int GADJ_BLOCK = 256;
// per-warp queue of flights to rasterise, one column per lane: for the three
// axes in partition order, the first crossing distance and the spacing of
// the plane crossings, and the count with the axis code; then the length,
// the coefficient and the start voxel
constexpr int GADJ_SEG = 12;

// float -> double by moving the bit fields: exact for normal numbers and
// infinities; subnormals (far below any term summed here) become zero.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t s = u & 0x80000000u;
    const uint32_t ex = e == 0xFFu ? 0x7FFu : e + 896u;     // rebias 127 -> 1023
    const uint32_t hi = e == 0u ? s : (s | (ex << 20) | ((u & 0x7FFFFFu) >> 3));
    const uint32_t lo = e == 0u ? 0u : (u << 29);
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Distance along a flight to its j-th crossing of one axis's voxel planes,
// affine in j (planes are evenly spaced) and 0 for a plane the start lies on
// or past. Every use shares this one formula, so the segments between
// consecutive crossings tile the flight exactly.
__device__ __forceinline__ float cross_at(float t0, float dl, int j)
{
    return fmaxf(fmaf((float)j, dl, t0), 0.f);
}

// One axis of a flight of length len from p along d (1/d = id): start voxel
// i0, first crossing t0, spacing dl, and n, the interior planes crossed at
// distances below len.
struct Cross {
    float t0, dl;
    int i0, n;
    bool up;
};

__device__ __forceinline__ Cross axis_cross(float p, float d, float id, float lo, float v, float iv, int g,
                                            float len)
{
    Cross c;
    c.i0 = min(max(__float2int_rd((p - lo) * iv), 0), g - 1);
    c.up = d > 0.f;
    c.t0 = 0.f;
    c.dl = 1.f;
    c.n = 0;
    if (!(fabsf(id) < __int_as_float(0x7f800000))) return c;   // no motion along this axis
    c.t0 = (fmaf((float)(c.up ? c.i0 + 1 : c.i0), v, lo) - p) * id;
    c.dl = v * fabsf(id);
    const int lim = c.up ? g - 1 - c.i0 : c.i0;
    int n = min(max(__float2int_ru((len - c.t0) * (fabsf(d) * iv)), 0), lim);
    while (n > 0 && !(cross_at(c.t0, c.dl, n - 1) < len)) --n;
    while (n < lim && cross_at(c.t0, c.dl, n) < len) ++n;
    c.n = n;
    return c;
}

// crossings of an axis at distances <= t, and the distance of the next one
__device__ __forceinline__ int count_le(float t0, float dl, int n, float t, float &next)
{
    int c = 0;
    if (n > 0) {
        c = min(max(__float2int_rd((t - t0) * rcp_approx(dl)) + 1, 0), n);
        while (c > 0 && cross_at(t0, dl, c - 1) > t) --c;
        while (c < n && cross_at(t0, dl, c) <= t) ++c;
    }
    next = c < n ? cross_at(t0, dl, c) : __int_as_float(0x7f800000);
    return c;
}

// Unit u of queued flight q: the stretch between crossings u-1 and u of its
// partition axis A (the axis it crosses most; the flight's start and end
// close the first and last stretch), walked across the crossings of the
// other two axes B and C inside it; grad[voxel] += coef * length of each
// piece.
__device__ __forceinline__ void raster_unit(const GridArgs &G, double *grad, const float *s_seg, int q, int u)
{
    const float INF = __int_as_float(0x7f800000);
    const float *f = s_seg + q;
    const int *fi = reinterpret_cast<const int *>(f);
    const int wA = fi[192], wB = fi[224], wC = fi[256];
    const int nA = wA & 0xFFFF, nB = wB & 0xFFFF, nC = wC & 0xFFFF;
    auto stride = [&](int w) {
        const int ax = (w >> 16) & 3;
        const int st = ax == 0 ? 1 : (ax == 1 ? G.gx : G.gx * G.gy);
        return (w >> 18) & 1 ? -st : st;
    };
    const float len = f[288], coef = f[320];
    const float tB0 = f[32], dB = f[128], tC0 = f[64], dC = f[160];
    const float t0 = u == 0 ? 0.f : cross_at(f[0], f[96], u - 1);
    const float t1 = u == nA ? len : cross_at(f[0], f[96], u);
    float nextB, nextC;
    int cB = count_le(tB0, dB, nB, t0, nextB);
    int cC = count_le(tC0, dC, nC, t0, nextC);
    const int sB = stride(wB), sC = stride(wC);
    int v = fi[352] + u * stride(wA) + cB * sB + cC * sC;
    float t = t0;
    for (int it = 0; it <= nB + nC; ++it) {
        const bool bfirst = nextB <= nextC;
        const float m = fminf(nextB, nextC);
        const float e = fminf(m, t1);
        if (e > t) atomicAdd(&grad[chk(v, G.gx * G.gy * G.gz, G.c.error)], widen(coef * (e - t)));
        t = e;
        if (!(m < t1)) break;
        if (bfirst) {
            v += sB;
            ++cB;
            nextB = cB < nB ? cross_at(tB0, dB, cB) : INF;
        } else {
            v += sC;
            ++cC;
            nextC = cC < nC ? cross_at(tC0, dC, cC) : INF;
        }
    }
}

// NULLS: the flights' transmission is scored at the null collisions of
// delta tracking instead of integrated along each flight. Against majorants
// scaled by maj_scale > 1 (so mubar > mu_ext in every voxel) a null
// collision has probability 1 - mu_ext / mubar, whose derivative with
// respect to the voxel's density is the score -k_ext / (mubar - mu_ext); it
// multiplies the camera terms that follow its flight. One atomic per null
// collision replaces the rasterised flight; both are unbiased estimates of
// the same gradient.
template <int PHASE, bool NULLS>
__global__ void __launch_bounds__(GADJ_BLOCK) grid_adjoint_kernel(const __grid_constant__ GridAdjArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const GridArgs &G = A.g;
    const CommonArgs &C = G.c;
    const MediumArgs &M = G.m;
    const uint32_t tb = (PHASE != MC_PHASE_HG) ? C.table_bytes : 0u;
    float *s_maj = reinterpret_cast<float *>(smem + tb);
    unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(smem + tb + C.extra_bytes);
    double *s_red = reinterpret_cast<double *>(s_bar + 2);
    // per-warp queue of flight segments to rasterise: (p, d, 1/d, length, coef)
    float *s_seg = reinterpret_cast<float *>(s_red + GADJ_BLOCK / 32) + (threadIdx.x & ~31u) * GADJ_SEG;
    // (column f of lane q at s_seg[32 f + q])
    Smem S = carve<MC_PHASE_HG, false>(smem, C);
    S.table = smem;
    if (threadIdx.x == 0) mbar_init(s_bar);
    uint32_t parity = 0u;
    if (PHASE != MC_PHASE_HG) {
        if (!stage_bulk(smem, M.table, C.table_bytes, s_bar, parity, C.error)) return;
        parity ^= 1u;
        if (!bind_table<PHASE>(S, C)) return;
    }
    if (!stage_bulk(s_maj, G.maj, C.extra_bytes, s_bar, parity, C.error)) return;
    if (NULLS) {
        for (int i = threadIdx.x; i < G.mx * G.my * G.mz; i += blockDim.x) s_maj[i] *= A.maj_scale;
        __syncthreads();
    }

    const int lane = threadIdx.x & 31;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const float INF = __int_as_float(0x7f800000);
    // null scores: inside the box around the beam axis, this CTA's copy of
    // the voxel sums (many CTAs adding to the same voxels there at once
    // serialise in L2; the copies spread them)
    const size_t cpb = (size_t)(blockIdx.x % (unsigned)A.copies) * A.bstride;
    double *gs = A.gsum, *s1c = A.s1, *bgs = A.bgs + cpb, *bs1 = A.bs1 + cpb;
    auto slot = [&](double *main, double *box, int ix, int iy, int iz, size_t v) -> double * {
        const unsigned by = (unsigned)(iy - A.by0), bz = (unsigned)(iz - A.bz0);
        if (NULLS && by < (unsigned)A.bw && bz < (unsigned)A.bw)
            return box + ((size_t)bz * A.bw + by) * G.gx + ix;
        return main + v;
    };
    unsigned long long pool_next = 0, pool_end = 0;
    bool alive = false, done = false;
    int pass = 0;
    uint32_t pk0 = 0, pk1 = 0, ev = 0, ncoll = 0;
    float rx = 0, ry = 0, rz = 0, dx = 1, dy = 0, dz = 0, w = 1;
    float idx = 1, idy = INF, idz = INF;
    float px = 0, py = 0, pz = 0;          // previous real collision (or the entry point)
    float P = 0.f, Ptot = 0.f;             // running / total camera terms of the photon
    double val = 0.0;

    while (true) {
        const unsigned need = __ballot_sync(FULL, !alive && !done);
        if (need) {
            const unsigned n_need = __popc(need), rank = __popc(need & lanemask_lt);
            const unsigned long long avail = pool_end - pool_next;
            unsigned long long mine;
            if (avail >= n_need) {
                mine = pool_next + rank;
                pool_next += n_need;
            } else {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(G.counter, (unsigned long long)CHUNK);
                base = __shfl_sync(FULL, base, 0);
                mine = (rank < avail) ? pool_next + rank : base + (rank - avail);
                pool_next = base + (n_need - avail);
                pool_end = base + CHUNK;
            }
            if (!alive && !done) {
                if (mine < M.n_photons) {
                    const unsigned long long p = M.photon_offset + mine;
                    pk0 = (uint32_t)p;
                    pk1 = (uint32_t)(p >> 32);
                    pass = 0;
                    alive = true;
                    ev = 0;   // the state itself is set below (start of a pass)
                    ncoll = 0xFFFFFFFFu;
                } else {
                    done = true;
                }
            }
        }
        if (!__any_sync(FULL, alive)) break;
        int nseg = 0;          // stretches of the flight this lane queued this round

        if (alive && ncoll == 0xFFFFFFFFu) {
            // start (or restart) the photon's pass at the entry point
            ev = 0;
            ncoll = 0;
            rx = 0.f; ry = 0.f; rz = 0.f;
            dx = 1.f; dy = 0.f; dz = 0.f;
            idx = 1.f; idy = INF; idz = INF;
            w = 1.f;
            P = 0.f;
            if (C.beam_r > 0.f) {
                const uint4 b = philox10(make_uint4(pk0, pk1, 0xFFFFFFFFu, 0u), M.key0, M.key1);
                const float rho = C.beam_r * sqrtf(u01(b.x));
                float sp, cp;
                sincospif(2.0f * u01(b.y), &sp, &cp);
                ry = rho * cp;
                rz = rho * sp;
            }
            px = rx; py = ry; pz = rz;
        }

        bool end = false;
        if (!alive) {
            // nothing to walk; still takes part in the warp's rasterisation below
        } else if (ev >= C.max_events) {
            if (pass == 0) atomicOr(C.error, MC_EFLAG_EVENTS);
            end = true;
        } else {
            const uint4 rnd = philox10(make_uint4(pk0, pk1, ev, 0u), M.rk);
            ++ev;
            const float u1 = u01(rnd.y), u2 = u01(rnd.z);
            float u3 = u01(rnd.w);
            float mb = 0.f;
            const int face = grid_flight(G, s_maj, -mc_log(u01(rnd.x)), rx, ry, rz, dx, dy, dz, idx, idy, idz, mb);
            if (face < 0) {
                atomicOr(C.error, MC_EFLAG_NUMERIC);
                end = true;
            } else if (face < 3) {
                end = true;   // left the cuvette: no camera term follows
            } else {
                const int ix = min(max(__float2int_rd(rx * G.inv_vx), 0), G.gx - 1);
                const int iy = centred_cell(ry, G.inv_vy, 0.5f * (float)G.gy, G.gy);
                const int iz = centred_cell(rz, G.inv_vz, 0.5f * (float)G.gz, G.gz);
                const size_t v = chk((iz * G.gy + iy) * G.gx + ix, G.gx * G.gy * G.gz, C.error);
                const float2 cell = __ldg(&G.cells[v]);
                const float acc = mc_div(cell.x, mb);   // hardware reciprocal (a few ulp) unless strict
                if (NULLS && !(u3 < acc) && pass == 1) {
                    // null collision: its score times the camera terms after it
                    const float B = Ptot - P;
                    if (B != 0.f) atomicAdd(slot(gs, bgs, ix, iy, iz, v), widen(-B * mc_div(A.k_ext, mb - cell.x)));
                }
                if (u3 < acc) {
                    u3 = mc_div(u3, acc);
                    ++ncoll;
                    const float a = G.mu_a > 0.f ? G.ks_over_ke * (1.0f - mc_div(G.mu_a, cell.x)) : G.ks_over_ke;
                    w = w * a;
                    int nb, pix_x, pix_z;
                    const float psr = camera_psr<PHASE>(M, C, S, dy, nb);
                    const float top = (iy == G.gy - 1) ? C.hy : fmaf((float)(iy + 1), G.vy, -C.hy);
                    const float nee = w * psr * mc_exp(-fmaf(cell.x, top - ry, cell.y));
                    const int pix = camera_pixel(C, rx, rz, pix_x, pix_z);
                    const float Aj = __ldg(&A.adj[pix]) * nee;
                    if (pass == 1) {
                        const float B = Ptot - P;
                        // column source: this voxel's part directly, the rest by the fold
                        float gv = -A.k_ext * Aj * (top - ry);
                        if (B != 0.f) {
                            const float dens = cell.x - G.mu_a;   // k_ext n_v
                            if (dens > 0.f) gv = fmaf(B, mc_div(A.k_ext, dens), gv);
                            const float coef = -B * A.k_ext;
                            if (NULLS) {
                                // the flight's transmission was scored at its null collisions
                            } else if (ncoll == 1) {
                                // first flight, along +x from the entry point in this
                                // voxel row: the voxels before ix by the row suffix
                                gv = fmaf(coef, fmaxf(fmaf(-(float)ix, G.vx, rx), 0.f), gv);
                                atomicAdd(&A.ex[v], widen(coef));
                            } else {
                                const float ex = rx - px, ey = ry - py, ez = rz - pz;
                                const float len = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
                                const Cross X = axis_cross(px, dx, idx, 0.f, G.vx, G.inv_vx, G.gx, len);
                                const Cross Y = axis_cross(py, dy, idy, -C.hy, G.vy, G.inv_vy, G.gy, len);
                                const Cross Z = axis_cross(pz, dz, idz, -C.hz, G.vz, G.inv_vz, G.gz, len);
                                // partition axis: the one crossed most; then the other two
                                const int pa = (X.n >= Y.n && X.n >= Z.n) ? 0 : (Y.n >= Z.n ? 1 : 2);
                                const Cross &A0 = pa == 0 ? X : (pa == 1 ? Y : Z);
                                const Cross &B0 = pa == 0 ? Y : X;
                                const Cross &C0 = pa == 2 ? Y : Z;
                                const int ab = pa == 0 ? 1 : 0, ac = pa == 2 ? 1 : 2;
                                float *q = s_seg + lane;
                                int *qi = reinterpret_cast<int *>(q);
                                q[0] = A0.t0; q[32] = B0.t0; q[64] = C0.t0;
                                q[96] = A0.dl; q[128] = B0.dl; q[160] = C0.dl;
                                qi[192] = A0.n | (pa << 16) | ((A0.up ? 0 : 1) << 18);
                                qi[224] = B0.n | (ab << 16) | ((B0.up ? 0 : 1) << 18);
                                qi[256] = C0.n | (ac << 16) | ((C0.up ? 0 : 1) << 18);
                                q[288] = len; q[320] = coef;
                                qi[352] = (Z.i0 * G.gy + Y.i0) * G.gx + X.i0;
                                nseg = A0.n + 1;
                            }
                        }
                        if (gv != 0.f) atomicAdd(slot(gs, bgs, ix, iy, iz, v), widen(gv));
                        if (Aj != 0.f) atomicAdd(slot(s1c, bs1, ix, iy, iz, v), widen(Aj));
                    }
                    P += Aj;
                    px = rx; py = ry; pz = rz;
                    if (C.max_scatter && ncoll >= C.max_scatter) {
                        end = true;
                    } else {
                        scatter<PHASE>(M, C, S, u1, u2, dx, dy, dz);
                        idx = mc_div(1.0f, dx); idy = mc_div(1.0f, dy); idz = mc_div(1.0f, dz);
                        if (w < C.rr_thr) {
                            if (u3 < C.rr_surv) w = w * C.inv_rr_surv;
                            else end = true;
                        }
                    }
                }
            }
        }
        if (alive && end) {
            if (pass == 0) {
                Ptot = P;
                val += (double)P;
                if (P != 0.f) {
                    pass = 1;
                    ncoll = 0xFFFFFFFFu;   // replay
                } else {
                    alive = false;
                }
            } else {
                alive = false;
            }
        }
        // the warp rasterises its queued flights together, one stretch between
        // partition-axis crossings per lane: the stretches of all flights are
        // numbered in lane order and handed out 32 at a time, each lane
        // finding its flight by a search over the exclusive prefix sums
        if (!NULLS && __any_sync(FULL, nseg != 0)) {
            __syncwarp();
            int incl = nseg;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const int excl = incl - nseg;
            const int total = __shfl_sync(FULL, incl, 31);
            for (int base = 0; base < total; base += 32) {
                const int g = base + lane;
                int q = 0, eq = 0;    // last lane whose flight starts at or before g
                for (int st = 16; st > 0; st >>= 1) {
                    const int e = __shfl_sync(FULL, excl, q + st);
                    if (e <= g) { q += st; eq = e; }
                }
                if (g < total) raster_unit(G, gs, s_seg, q, g - eq);
            }
            __syncwarp();
        }
    }
    // fixed-order block reduction of the value
    val += __shfl_xor_sync(FULL, val, 16);
    val += __shfl_xor_sync(FULL, val, 8);
    val += __shfl_xor_sync(FULL, val, 4);
    val += __shfl_xor_sync(FULL, val, 2);
    val += __shfl_xor_sync(FULL, val, 1);
    if (lane == 0) s_red[threadIdx.x / 32] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += s_red[k];
        A.partials[blockIdx.x] = t;
    }
}

// ------------------------------------------------------------------ adjoint
// Gradient of L = sum_pix adj[pix] image[pix] with respect to (mu_s, mu_a)
// and the hat-function phase weights w_k (p_w = p h_w / Z(w), h_w = sum_k
// w_k phi_k, Z(w) = sum_k w_k Z_k, Z_k = int p phi_k over the unweighted
// table p), by likelihood ratios along replayed paths (the photons, random
// numbers and single-precision arithmetic of the forward walk, which samples
// p_w through its reweighted table). For a camera term A_j = adj[pix_j] c_j
// at collision j of a photon:
//   dL/dmu_s += A_j (S_j + j (1/mu_s - 1/mu_ext) - l_j)
//   dL/dmu_a += A_j (S_j - j/mu_ext - l_j)
//   dL/dw_k  += A_j (phi_k(mu_c,j)/h_w(mu_c,j) - j Z_k/Z(w)
//                    + sum_{i<j} phi_k(mu_i)/h_w(mu_i)),
// S_j = sum over the flights up to j of (1/mu_ext - s_i) (Eq. 15 score),
// l_j the distance to the camera face, mu_i the sampled polar cosines. The
// last sum is rearranged as sum_i phi_k(mu_i)/h_w(mu_i) (P_tot - P_i) with
// P_i = A_1 + .. + A_i, which needs the photon's total P_tot: photons with
// more angles than the kernel keeps are replayed a second time (same
// counters). Roulette factors are held fixed.

// Hat functions: nodes mu_k = -1 + k h, h = 2/(n_w - 1); the two nonzero
// weights at mu.
__device__ __forceinline__ int hat_pair(int nw, float mu, float &f)
{
    const float t = (mu + 1.0f) * (0.5f * (float)(nw - 1));
    int k = __float2int_rd(t);
    k = min(max(k, 0), nw - 2);
    f = fminf(fmaxf(t - (float)k, 0.0f), 1.0f);
    return k;
}

// Z_k = int_{-1}^{1} p(mu) phi_k(mu) dmu over the table (bins of constant
// density), exactly, in double precision: CTA k sums the bins of hat k's
// support, each thread a strided subset in order, then a fixed-order tree.
__global__ void hat_integrals_kernel(const unsigned char *table, int nw, double *z)
{
    __shared__ double part[256];
    const mc_table_header *hd = reinterpret_cast<const mc_table_header *>(table);
    const float *omu = reinterpret_cast<const float *>(table + hd->off_omu);
    const float *pdf = reinterpret_cast<const float *>(table + hd->off_pdf);
    const uint16_t *guide = reinterpret_cast<const uint16_t *>(table + hd->off_guide);
    const int n = hd->n_bins, k = blockIdx.x;
    const double h = 2.0 / (nw - 1), inv_h = (nw - 1) / 2.0, c = -1.0 + k * h;
    const double lo = fmax(c - h, -1.0), hi = fmin(c + h, 1.0);
    const int j0 = max(table_bin(omu, guide, n, (float)lo) - 1, 0);
    const int j1 = min(table_bin(omu, guide, n, (float)hi) + 1, n - 1);
    double acc = 0.0;
    for (int j = j0 + (int)threadIdx.x; j <= j1; j += blockDim.x) {
        const double a = fmax(1.0 - (double)omu[j], lo), b = fmin(1.0 - (double)omu[j + 1], hi);
        if (!(b > a)) continue;
        // phi_k is linear on each side of c: trapezoids are exact per piece
        const double m = fmin(fmax(c, a), b);
        const double pa = 1.0 - fabs(a - c) * inv_h, pm = 1.0 - fabs(m - c) * inv_h,
                     pb = 1.0 - fabs(b - c) * inv_h;
        acc += (double)pdf[j] * 0.5 * ((pa + pm) * (m - a) + (pm + pb) * (b - m));
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) z[k] = part[0];
}

constexpr int ADJ_BLOCK = 256;     // threads per CTA without phase weights
constexpr int ADJ_BLOCK_W = 128;   // with phase weights (private accumulators)
constexpr int ADJ_LIST = 8;        // sampled angles kept per photon before a replay is needed

// Compensated (Kahan) sum in single precision: s + c carries the running
// total to about 2^-46 of the summed magnitudes, on the full-rate float pipe
// (GB300's double-precision pipe runs at a small fraction of it).
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Private single-precision accumulators: hat k of thread t at rows[k*B + t]
// (consecutive threads in consecutive banks; no atomics, fixed order). Adds
// v phi(mu) / h_w(mu) for the two hats around mu (k, fraction f), with the
// weights sw in shared memory.
__device__ __forceinline__ void hat_add(float *rows, int nw_stride, const float *sw, int k, float f, float v)
{
    const float u = mc_div(v, fmaf(f, sw[k + 1] - sw[k], sw[k]));
    rows[k * nw_stride + threadIdx.x] += u * (1.0f - f);
    rows[(k + 1) * nw_stride + threadIdx.x] += u * f;
}

template <int PHASE, bool PHASEW>
__global__ void __launch_bounds__(ADJ_BLOCK) adjoint_kernel(const __grid_constant__ AdjArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const CommonArgs &C = A.c;
    const MediumArgs &M = A.m;
    const uint32_t tb = (PHASE == MC_PHASE_TABLE && !PHASEW) ? C.table_bytes : 0u;
    const int nw = PHASEW ? A.n_w : 0;
    const int B = blockDim.x, warps = B / 32, warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    double *s_z = reinterpret_cast<double *>(smem + tb);   // [nw] Z_k / Z(w)
    double *s_red = s_z + nw;                              // [warps][4]
    unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(s_red + warps * 4);
    float *s_w = reinterpret_cast<float *>(s_bar + 2);     // [nw, padded to 4] weights
    float *rows = s_w + ((nw + 3) & ~3);                   // [nw][B]
    for (int i = threadIdx.x; i < nw * B; i += B) rows[i] = 0.0f;
    if (threadIdx.x == 0) mbar_init(s_bar);
    Smem S = carve<MC_PHASE_HG, false>(smem, C);
    S.table = smem;
    if (PHASE == MC_PHASE_TABLE) {
        if (PHASEW) {
            // shared memory holds the private accumulators; the table is read
            // through L1 (41 KB, resident after the first touches)
            S.table = const_cast<unsigned char *>(M.table);
        } else if (!stage_bulk(smem, M.table, tb, s_bar, 0u, C.error)) {
            return;
        }
        if (!bind_table<PHASE>(S, C)) return;
    }
    if (PHASEW) {
        for (int k = threadIdx.x; k < nw; k += B) s_w[k] = A.w ? A.w[k] : 1.0f;
        __syncthreads();
        if (threadIdx.x == 0) {   // Z(w) = sum_k w_k Z_k, fixed order
            double zw = 0.0;
            for (int k = 0; k < nw; ++k) zw += (double)s_w[k] * A.z[k];
            s_red[0] = zw;
        }
        __syncthreads();
        const double zw = s_red[0];
        for (int k = threadIdx.x; k < nw; k += B) s_z[k] = A.z[k] / zw;
    }
    __syncthreads();
    const float c_s = A.c_s;   // 1/mu_s - 1/mu_ext

    const unsigned lanemask_lt = (1u << lane) - 1u;
    unsigned long long pool_next = 0, pool_end = 0;
    bool alive = false, done = false;
    int pass = 1, cnt = 0;
    unsigned long long rel = 0;
    uint32_t pk0 = 0, pk1 = 0, ev = 0, ncoll = 0;
    float rx = 0, ry = 0, rz = 0, dx = 1, dy = 0, dz = 0, w = 1, Ssc = 0;
    // the photon's running and total camera terms in single precision:
    // P_tot - P_i is then accurate to ~1e-7 of the photon's total, far
    // below the statistical error of any gradient
    float P = 0.0f, Ptot = 0.0f;
    // per-thread sums of A_j, A_j dlog/dmu_s, A_j dlog/dmu_a and j A_j as
    // compensated single-precision pairs
    float gs_val = 0.f, gc_val = 0.f, gs_s = 0.f, gc_s = 0.f, gs_a = 0.f, gc_a = 0.f, gs_z = 0.f, gc_z = 0.f;
    // the photon's first ADJ_LIST sampled angles: hat index, fraction, P_i
    // (indexed with compile-time constants only, so they stay in registers)
    int lk[ADJ_LIST];
    float lf[ADJ_LIST], lp[ADJ_LIST];
#pragma unroll
    for (int q = 0; q < ADJ_LIST; ++q) { lk[q] = 0; lf[q] = 0.0f; lp[q] = 0.0f; }

    while (true) {
        const unsigned need = __ballot_sync(FULL, !alive && !done);
        if (need) {
            const unsigned n_need = __popc(need), rank = __popc(need & lanemask_lt);
            const unsigned long long avail = pool_end - pool_next;
            unsigned long long mine;
            if (avail >= n_need) {
                mine = pool_next + rank;
                pool_next += n_need;
            } else {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(A.counter, (unsigned long long)CHUNK);
                base = __shfl_sync(FULL, base, 0);
                mine = (rank < avail) ? pool_next + rank : base + (rank - avail);
                pool_next = base + (n_need - avail);
                pool_end = base + CHUNK;
            }
            if (!alive && !done) {
                if (mine < M.n_photons) {
                    rel = mine;
                    const unsigned long long p = M.photon_offset + mine;
                    pk0 = (uint32_t)p;
                    pk1 = (uint32_t)(p >> 32);
                    pass = 1;
                    alive = true;
                } else {
                    done = true;
                }
            }
        }
        if (!__any_sync(FULL, alive)) break;
        if (!alive) continue;
        if (ev == 0) {
            // (re)start of a pass: the photon enters as in the forward walk
            rx = 0.f; ry = 0.f; rz = 0.f;
            dx = 1.f; dy = 0.f; dz = 0.f;
            w = 1.f;
            P = 0.0f;
            cnt = 0;
            if (C.beam_r > 0.f) {
                const uint4 b = philox10(make_uint4(pk0, pk1, 0xFFFFFFFFu, 0u), M.key0, M.key1);
                const float rho = C.beam_r * sqrtf(u01(b.x));
                float sp, cp;
                sincospif(2.0f * u01(b.y), &sp, &cp);
                ry = rho * cp;
                rz = rho * sp;
            }
        }

        const uint4 rnd = philox10(make_uint4(pk0, pk1, ev, 0u), M.rk);
        ++ev;
        const float u0 = u01(rnd.x), u1 = u01(rnd.y), u2 = u01(rnd.z), u3 = u01(rnd.w);
        const float s = -mc_log(u0) * M.inv_mu_ext;
        const float px = fmaf(s, dx, rx), py = fmaf(s, dy, ry), pz = fmaf(s, dz, rz);
        bool end = !((px > 0.f) & (px < C.lx) & (fabsf(py) < C.hy) & (fabsf(pz) < C.hz));
        if (!end) {
            rx = px; ry = py; rz = pz;
            ++ncoll;
            Ssc += M.inv_mu_ext - s;
            w = w * M.albedo;
            int nb, ix, iz;
            const float psr = camera_psr<PHASE>(M, C, S, dy, nb);
            const float l = C.hy - ry;
            const float nee = w * psr * mc_exp(-M.mu_ext * l);
            const int pix = camera_pixel(C, rx, rz, ix, iz);
            const float Aj = __ldg(&A.adj[pix]) * nee;
            P += Aj;
            if (pass == 1) {
                const float jj = (float)ncoll;
                kahan_add(gs_val, gc_val, Aj);
                kahan_add(gs_s, gc_s, Aj * (Ssc + jj * c_s - l));
                kahan_add(gs_a, gc_a, Aj * (Ssc - jj * M.inv_mu_ext - l));
                kahan_add(gs_z, gc_z, jj * Aj);
                if (PHASEW && Aj != 0.0f) {
                    float f;
                    const int k = chk(hat_pair(nw, dy, f), nw - 1, C.error);
                    hat_add(rows, B, s_w, k, f, Aj);
                }
            }
            if (C.max_scatter && ncoll >= C.max_scatter) {
                end = true;
            } else {
                const float om = sample_omu<PHASE>(M, C, S, u1);
                if (PHASEW) {
                    float f;
                    const int k = chk(hat_pair(nw, 1.0f - om, f), nw - 1, C.error);
                    if (pass == 1) {
#pragma unroll
                        for (int q = 0; q < ADJ_LIST; ++q)
                            if (q == cnt) { lk[q] = k; lf[q] = f; lp[q] = P; }
                        ++cnt;
                    } else {
                        const float coef = Ptot - P;
                        if (coef != 0.0f) hat_add(rows, B, s_w, k, f, coef);
                    }
                }
                if (PHASE == MC_PHASE_HG) rotate_hg(dx, dy, dz, om, hg_opu(M, u1), u2);
                else rotate(dx, dy, dz, om, u2);
                if (w < C.rr_thr) {
                    if (u3 < C.rr_surv) w = w * C.inv_rr_surv;
                    else end = true;
                }
                if (!end && ev >= C.max_events) end = true;
            }
        }
        if (end) {
            bool replay = false;
            if (PHASEW && pass == 1 && P != 0.0f) {
                if (cnt <= ADJ_LIST) {
                    // every sampled angle is in the list: sum_i phi(mu_i) (P_tot - P_i)
#pragma unroll
                    for (int q = 0; q < ADJ_LIST; ++q) {
                        if (q < cnt) {
                            const float coef = P - lp[q];
                            if (coef != 0.0f) hat_add(rows, B, s_w, lk[q], lf[q], coef);
                        }
                    }
                } else {
                    Ptot = P;   // replay the same photon for its later angles
                    pass = 2;
                    replay = true;
                }
            }
            if (!replay) alive = false;
            ev = 0;
            ncoll = 0;
            Ssc = 0.0f;
        }
    }

    // -------- reduce: lanes -> warp -> CTA row of partials (fixed order)
    double g_val = (double)gs_val - (double)gc_val, g_s = (double)gs_s - (double)gc_s;
    double g_a = (double)gs_a - (double)gc_a, g_z = (double)gs_z - (double)gc_z;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        g_val += __shfl_xor_sync(FULL, g_val, o);
        g_s += __shfl_xor_sync(FULL, g_s, o);
        g_a += __shfl_xor_sync(FULL, g_a, o);
        g_z += __shfl_xor_sync(FULL, g_z, o);
    }
    if (lane == 0) {
        s_red[warp * 4 + 0] = g_val;
        s_red[warp * 4 + 1] = g_s;
        s_red[warp * 4 + 2] = g_a;
        s_red[warp * 4 + 3] = g_z;
    }
    __syncthreads();
    double *row = A.partials + (size_t)blockIdx.x * (3 + A.n_w);
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < warps; ++q) t += s_red[q * 4 + threadIdx.x];
        row[threadIdx.x] = t;
    }
    if (PHASEW) {
        double gzb = 0.0;
        for (int q = 0; q < warps; ++q) gzb += s_red[q * 4 + 3];
        for (int k = threadIdx.x; k < nw; k += B) {
            double t = 0.0;
            for (int q = 0; q < B; ++q) t += (double)rows[k * B + q];
            row[3 + k] = t - s_z[k] * gzb;
        }
    }
}

// out[q] = sum over the grid's rows of partials[row][q]: one CTA per column,
// each thread a fixed stride of rows, then a fixed tree (deterministic).
constexpr int RED_BLOCK = 256;
__global__ void __launch_bounds__(RED_BLOCK) adjoint_reduce(const double *partials, int rows, int width,
                                                            double *out)
{
    __shared__ double part[RED_BLOCK];
    const int q = blockIdx.x;
    double t = 0.0;
    for (int r = threadIdx.x; r < rows; r += RED_BLOCK) t += partials[(size_t)r * width + q];
    part[threadIdx.x] = t;
    __syncthreads();
    for (int h = RED_BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = part[0];
}

// Self-test of the bounded wait: a phase that expects 16 bytes of a copy
// that is never issued, so it cannot complete; the wait must give up after
// `tries` polls and flag MC_EFLAG_TIMEOUT. No copy is in flight at exit.
__global__ void wait_selftest_kernel(uint32_t *err, uint32_t tries)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar)), "r"(16u)
                     : "memory");
    }
    __syncthreads();
    const uint32_t done = mbar_wait(smem_u32(&bar), 0u, tries);
    if (!done && threadIdx.x == 0) atomicOr(err, MC_EFLAG_TIMEOUT);
}

__global__ void philox_kernel(const uint4 *ctr, uint64_t n, uint32_t k0, uint32_t k1, uint4 *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = philox10(ctr[i], k0, k1);
}

// Tallies whose contributions are all non-negative (image pixels, radial
// bins, every total but the signed roulette net) can turn negative only by
// passing 2^63 in fixed point: such a sum has wrapped, and the run is flagged
// MC_EFLAG_OVERFLOW. Blocks of medium blockIdx.y scan its tallies grid-stride.
constexpr int SIGN_BLOCK = 256;
__device__ __forceinline__ void sign_scan(const MediumArgs &M, int npix, int n_radial, uint32_t *err)
{
    const long long *img = reinterpret_cast<const long long *>(M.image);
    bool bad = false;
    for (int i = blockIdx.x * SIGN_BLOCK + threadIdx.x; i < npix; i += gridDim.x * SIGN_BLOCK)
        bad |= img[i] < 0;
    if (blockIdx.x == 0) {
        const long long *rad = reinterpret_cast<const long long *>(M.radial);
        for (int i = threadIdx.x; i < n_radial; i += SIGN_BLOCK) bad |= rad[i] < 0;
        if (threadIdx.x < MC_N_TOTALS && threadIdx.x != MC_TOT_ROULETTE)
            bad |= reinterpret_cast<const long long *>(M.totals)[threadIdx.x] < 0;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, MC_EFLAG_OVERFLOW);
}

__global__ void __launch_bounds__(SIGN_BLOCK) sign_check_kernel(const __grid_constant__ WalkArgs A)
{
    sign_scan(A.m, A.c.nx * A.c.nz, A.c.n_radial, A.c.error);
}

__global__ void __launch_bounds__(SIGN_BLOCK) batch_sign_check_kernel(const __grid_constant__ BatchArgs B)
{
    sign_scan(B.m[blockIdx.y], B.c.nx * B.c.nz, B.c.n_radial, B.c.error);
}

unsigned sign_blocks(const CommonArgs &c)
{
    const int npix = c.nx * c.nz;
    const int b = (npix + 4 * SIGN_BLOCK - 1) / (4 * SIGN_BLOCK);
    return (unsigned)(b < 1 ? 1 : (b > 512 ? 512 : b));
}

cudaError_t launch_sign_check(const WalkArgs &a, cudaStream_t st)
{
    sign_check_kernel<<<sign_blocks(a.c), SIGN_BLOCK, 0, st>>>(a);
    return cudaGetLastError();
}

// Persistent grid: SMs x CTAs per SM (occupancy, or the caller's choice),
// capped at what `work_warps` warps of work can use.
template <class Kern>
cudaError_t launch_persistent(Kern kern, const void *args_unused, const LaunchCfg &cfg, size_t smem,
                              unsigned long long work_warps, unsigned *grid)
{
    (void)args_unused;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, bps = cfg.blocks_per_sm;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (bps <= 0) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, cfg.block, smem)) != cudaSuccess)
            return e;
        if (bps < 1) return cudaErrorInvalidConfiguration;
    }
    unsigned long long blocks = (unsigned long long)sms * bps;
    const unsigned long long per_block = cfg.block / 32;
    const unsigned long long cap = (work_warps + per_block - 1) / per_block;
    if (cap < blocks) blocks = cap;
    *grid = (unsigned)(blocks < 1 ? 1 : blocks);
    return cudaSuccess;
}

// Where the image accumulates and how big the CTA is. Sets c.band0/band_rows.
cudaError_t plan_image(CommonArgs &c, LaunchCfg &cfg, bool *smem_img, size_t *smem)
{
    const size_t tb = ((c.phase_kind != MC_PHASE_HG) ? c.table_bytes : 0) + c.extra_bytes;
    const size_t tail = sizeof(unsigned long long) * (c.n_radial + MC_N_TOTALS + 3) + 16;
    const size_t row = sizeof(uint32_t) * (size_t)c.nx;
    int dev = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    // shared memory per CTA: all of it for one CTA per SM, an equal share
    // (less the per-CTA reservation) when several are requested
    int per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    if (cfg.blocks_per_sm > 1) {
        const int share = per_sm / cfg.blocks_per_sm - 1024;
        if (share < optin) optin = share;
    }
    const size_t room = (size_t)optin > tb + tail + 1024 ? (size_t)optin - tb - tail - 1024 : 0;
    const int fit_rows = (int)(room / row);
    // auto: one 1024-thread CTA per SM (32 warps) holding as many image rows
    // around the beam as fit (the whole image when it fits), the rest going
    // to L2 atomics
    int mode = cfg.image_mode;
    if (mode == 0) mode = fit_rows >= 1 ? 3 : 2;
    *smem_img = false;
    c.band0 = 0;
    c.band_rows = 0;
    if (mode == 1) {
        if (fit_rows < c.nz) return cudaErrorInvalidValue;
        *smem_img = true;
        c.band_rows = c.nz;
    } else if (mode == 3) {
        if (fit_rows < 1) return cudaErrorInvalidValue;
        *smem_img = true;
        c.band_rows = fit_rows < c.nz ? fit_rows : c.nz;
        int b0 = c.nz / 2 - c.band_rows / 2;
        if (b0 > c.nz - c.band_rows) b0 = c.nz - c.band_rows;
        c.band0 = b0 < 0 ? 0 : b0;
    }
    if (cfg.block == 0) cfg.block = (mode == 3) ? 1024 : 256;
    *smem = tb + tail + (*smem_img ? row * c.band_rows : 0);
    if (*smem > (size_t)optin) return cudaErrorInvalidValue;
    return cudaSuccess;
}

template <int PHASE, bool SMEM_IMAGE, bool TRACE>
cudaError_t launch_one(const WalkArgs &a, const LaunchCfg &cfg, size_t smem, cudaStream_t st)
{
    auto kern = walk_kernel<PHASE, SMEM_IMAGE, TRACE>;
    unsigned grid = 0;
    cudaError_t e = launch_persistent(kern, &a, cfg, smem, (a.m.n_photons + CHUNK - 1) / CHUNK, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, cfg.block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int PHASE, bool SMEM_IMAGE>
cudaError_t launch_batch_one(const BatchArgs &a, const LaunchCfg &cfg, size_t smem, cudaStream_t st)
{
    auto kern = batch_kernel<PHASE, SMEM_IMAGE>;
    unsigned grid = 0;
    unsigned long long chunks = 0;   // warp chunks of the largest medium: more warps would idle
    for (int i = 0; i < a.n_media; ++i) {
        const unsigned long long c = (a.m[i].n_photons + a.chunk - 1) / a.chunk;
        if (c > chunks) chunks = c;
    }
    cudaError_t e = launch_persistent(kern, &a, cfg, smem, chunks, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, cfg.block, smem, st>>>(a);
    return cudaGetLastError();
}


template <int PHASE, bool SMEM_IMAGE, bool TRACE>
cudaError_t launch_grid_one(const GridArgs &a, const LaunchCfg &cfg, size_t smem, cudaStream_t st)
{
    auto kern = grid_kernel<PHASE, SMEM_IMAGE, TRACE>;
    unsigned grid = 0;
    cudaError_t e = launch_persistent(kern, &a, cfg, smem, (a.m.n_photons + CHUNK - 1) / CHUNK, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, cfg.block, smem, st>>>(a);
    return cudaGetLastError();
}

size_t grid_adjoint_smem(const GridAdjArgs &a)
{
    const size_t tb = (a.g.c.phase_kind != MC_PHASE_HG) ? a.g.c.table_bytes : 0;
    return tb + a.g.c.extra_bytes + 16 + sizeof(double) * (GADJ_BLOCK / 32) + sizeof(float) * GADJ_BLOCK * GADJ_SEG;
}

template <int PHASE, bool NULLS>
cudaError_t launch_grid_adjoint_one(const GridAdjArgs &a, int rows, double *value, cudaStream_t st)
{
    auto kern = grid_adjoint_kernel<PHASE, NULLS>;
    const size_t smem = grid_adjoint_smem(a);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, bps = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, GADJ_BLOCK, smem)) != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)sms * bps;
    const long long cap = (long long)((a.g.m.n_photons + CHUNK - 1) / CHUNK + GADJ_BLOCK / 32 - 1) / (GADJ_BLOCK / 32);
    if (cap < grid) grid = cap < 1 ? 1 : cap;
    if (grid > rows) grid = rows;
    kern<<<(unsigned)grid, GADJ_BLOCK, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (NULLS) {
        e = launch_box_merge(a.gsum, a.s1, a.bgs, a.bs1, a.copies, a.nbox, a.bstride, a.g.gx, a.g.gy, a.by0, a.bz0,
                             a.bw, st);
        if (e != cudaSuccess) return e;
    }
    e = launch_gradient_fold(a.gsum, a.s1, NULLS ? nullptr : a.ex, a.grad, a.g.gx, a.g.gy, a.g.gz, (double)a.k_ext,
                             (double)a.g.vx, (double)a.g.vy, st);
    if (e != cudaSuccess) return e;
    adjoint_reduce<<<1, RED_BLOCK, 0, st>>>(a.partials, (int)grid, 1, value);
    return cudaGetLastError();
}
}  // namespace

namespace {
cudaError_t launch_walk_kernel(const WalkArgs &a, bool trace, const LaunchCfg &cfg, bool smem_img, size_t smem,
                               cudaStream_t st)
{
    switch (a.c.phase_kind * 4 + (smem_img ? 2 : 0) + (trace ? 1 : 0)) {
    case 0: return launch_one<MC_PHASE_TABLE, false, false>(a, cfg, smem, st);
    case 1: return launch_one<MC_PHASE_TABLE, false, true>(a, cfg, smem, st);
    case 2: return launch_one<MC_PHASE_TABLE, true, false>(a, cfg, smem, st);
    case 3: return launch_one<MC_PHASE_TABLE, true, true>(a, cfg, smem, st);
    case 4: return launch_one<MC_PHASE_HG, false, false>(a, cfg, smem, st);
    case 5: return launch_one<MC_PHASE_HG, false, true>(a, cfg, smem, st);
    case 6: return launch_one<MC_PHASE_HG, true, false>(a, cfg, smem, st);
    case 7: return launch_one<MC_PHASE_HG, true, true>(a, cfg, smem, st);
    case 8: return launch_one<MC_PHASE_PAPER, false, false>(a, cfg, smem, st);
    case 9: return launch_one<MC_PHASE_PAPER, false, true>(a, cfg, smem, st);
    case 10: return launch_one<MC_PHASE_PAPER, true, false>(a, cfg, smem, st);
    case 11: return launch_one<MC_PHASE_PAPER, true, true>(a, cfg, smem, st);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_walk(const WalkArgs &a0, bool trace, const LaunchCfg &cfg0, cudaStream_t st)
{
    WalkArgs a = a0;
    LaunchCfg cfg = cfg0;
    bool smem_img = false;
    size_t smem = 0;
    cudaError_t e = plan_image(a.c, cfg, &smem_img, &smem);
    if (e != cudaSuccess) return e;
    if ((e = launch_walk_kernel(a, trace, cfg, smem_img, smem, st)) != cudaSuccess) return e;
    return launch_sign_check(a, st);
}

cudaError_t check_plan(const CommonArgs &c0, const LaunchCfg &cfg0)
{
    CommonArgs c = c0;
    LaunchCfg cfg = cfg0;
    bool smem_img = false;
    size_t smem = 0;
    return plan_image(c, cfg, &smem_img, &smem);
}

namespace {
cudaError_t launch_grid_kernel(const GridArgs &a, bool trace, const LaunchCfg &cfg, bool smem_img, size_t smem,
                               cudaStream_t st)
{
    switch (a.c.phase_kind * 4 + (smem_img ? 2 : 0) + (trace ? 1 : 0)) {
    case 0: return launch_grid_one<MC_PHASE_TABLE, false, false>(a, cfg, smem, st);
    case 1: return launch_grid_one<MC_PHASE_TABLE, false, true>(a, cfg, smem, st);
    case 2: return launch_grid_one<MC_PHASE_TABLE, true, false>(a, cfg, smem, st);
    case 3: return launch_grid_one<MC_PHASE_TABLE, true, true>(a, cfg, smem, st);
    case 4: return launch_grid_one<MC_PHASE_HG, false, false>(a, cfg, smem, st);
    case 5: return launch_grid_one<MC_PHASE_HG, false, true>(a, cfg, smem, st);
    case 6: return launch_grid_one<MC_PHASE_HG, true, false>(a, cfg, smem, st);
    case 7: return launch_grid_one<MC_PHASE_HG, true, true>(a, cfg, smem, st);
    case 8: return launch_grid_one<MC_PHASE_PAPER, false, false>(a, cfg, smem, st);
    case 9: return launch_grid_one<MC_PHASE_PAPER, false, true>(a, cfg, smem, st);
    case 10: return launch_grid_one<MC_PHASE_PAPER, true, false>(a, cfg, smem, st);
    case 11: return launch_grid_one<MC_PHASE_PAPER, true, true>(a, cfg, smem, st);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_grid(const GridArgs &a0, bool trace, const LaunchCfg &cfg0, cudaStream_t st)
{
    GridArgs a = a0;
    LaunchCfg cfg = cfg0;
    bool smem_img = false;
    size_t smem = 0;
    cudaError_t e = plan_image(a.c, cfg, &smem_img, &smem);
    if (e != cudaSuccess) return e;
    if ((e = launch_grid_kernel(a, trace, cfg, smem_img, smem, st)) != cudaSuccess) return e;
    WalkArgs w;
    w.c = a.c;
    w.m = a.m;
    w.counter = a.counter;
    return launch_sign_check(w, st);
}

cudaError_t grid_adjoint_check(const GridAdjArgs &a)
{
    int dev = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    return grid_adjoint_smem(a) <= (size_t)optin ? cudaSuccess : cudaErrorInvalidValue;
}

int grid_adjoint_max_grid()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms * (2048 / GADJ_BLOCK);
}

cudaError_t launch_grid_adjoint(const GridAdjArgs &a, int rows, double *value, cudaStream_t st)
{
    if (rows < 1) return cudaErrorInvalidValue;
    switch (a.g.c.phase_kind * 2 + (a.nulls ? 1 : 0)) {
    case 0: return launch_grid_adjoint_one<MC_PHASE_TABLE, false>(a, rows, value, st);
    case 1: return launch_grid_adjoint_one<MC_PHASE_TABLE, true>(a, rows, value, st);
    case 2: return launch_grid_adjoint_one<MC_PHASE_HG, false>(a, rows, value, st);
    case 3: return launch_grid_adjoint_one<MC_PHASE_HG, true>(a, rows, value, st);
    case 4: return launch_grid_adjoint_one<MC_PHASE_PAPER, false>(a, rows, value, st);
    case 5: return launch_grid_adjoint_one<MC_PHASE_PAPER, true>(a, rows, value, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch(const BatchArgs &a0, const LaunchCfg &cfg0, cudaStream_t st)
{
    BatchArgs a = a0;
    LaunchCfg cfg = cfg0;
    bool smem_img = false;
    size_t smem = 0;
    cudaError_t e = plan_image(a.c, cfg, &smem_img, &smem);
    if (e != cudaSuccess) return e;
    switch (a.c.phase_kind * 2 + (smem_img ? 1 : 0)) {
    case 0: e = launch_batch_one<MC_PHASE_TABLE, false>(a, cfg, smem, st); break;
    case 1: e = launch_batch_one<MC_PHASE_TABLE, true>(a, cfg, smem, st); break;
    case 2: e = launch_batch_one<MC_PHASE_HG, false>(a, cfg, smem, st); break;
    case 3: e = launch_batch_one<MC_PHASE_HG, true>(a, cfg, smem, st); break;
    case 4: e = launch_batch_one<MC_PHASE_PAPER, false>(a, cfg, smem, st); break;
    case 5: e = launch_batch_one<MC_PHASE_PAPER, true>(a, cfg, smem, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    batch_sign_check_kernel<<<dim3(sign_blocks(a.c), (unsigned)a.n_media), SIGN_BLOCK, 0, st>>>(a);
    return cudaGetLastError();
}

int adjoint_max_grid()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms * (2048 / ADJ_BLOCK_W);
}

namespace {
template <int PHASE, bool PHASEW>
cudaError_t launch_adjoint_one(const AdjArgs &a, int rows, double *out, cudaStream_t st)
{
    auto kern = adjoint_kernel<PHASE, PHASEW>;
    const int nw = PHASEW ? a.n_w : 0;
    const int block = PHASEW ? ADJ_BLOCK_W : ADJ_BLOCK;
    const size_t smem = ((PHASE == MC_PHASE_TABLE && !PHASEW) ? a.c.table_bytes : 0) +
                        sizeof(double) * (nw + (block / 32) * 4) + 16 + sizeof(float) * ((nw + 3) & ~3) +
                        sizeof(float) * nw * block;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, bps = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, block, smem)) != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)sms * bps;
    const long long cap = (long long)((a.m.n_photons + CHUNK - 1) / CHUNK + block / 32 - 1) / (block / 32);
    if (cap < grid) grid = cap < 1 ? 1 : cap;
    if (grid > rows) grid = rows;
    if (PHASEW) {
        hat_integrals_kernel<<<a.n_w, 256, 0, st>>>(a.base_table, a.n_w, a.z);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    kern<<<(unsigned)grid, block, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    adjoint_reduce<<<3 + a.n_w, RED_BLOCK, 0, st>>>(a.partials, (int)grid, 3 + a.n_w, out);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_adjoint(const AdjArgs &a, int rows, double *out, cudaStream_t st)
{
    if (rows < 1 || a.c.phase_kind == MC_PHASE_PAPER) return cudaErrorInvalidValue;
    if (a.c.phase_kind == MC_PHASE_TABLE)
        return a.n_w ? launch_adjoint_one<0, true>(a, rows, out, st) : launch_adjoint_one<0, false>(a, rows, out, st);
    if (a.n_w) return cudaErrorInvalidValue;
    return launch_adjoint_one<1, false>(a, rows, out, st);
}

cudaError_t launch_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    philox_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const uint4 *>(ctr), n, (uint32_t)seed,
                                          (uint32_t)(seed >> 32), reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint32_t *err, uint32_t tries, cudaStream_t st)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(err, tries);
    return cudaGetLastError();
}

}  // namespace mcx
