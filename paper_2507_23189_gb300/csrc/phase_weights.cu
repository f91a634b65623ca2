// Phase table reweighted by hat-function weights, built on the device.
//
// The phase function with weights w is p_w = p h_w / Z(w): p the density of
// the unweighted table (constant (1/n) / (omu_j - omu_{j+1}) per unit cos
// theta on bin j, omu = 1 - cos theta at the levels j / n), h_w the linear
// interpolant of the weights w_k at the hat nodes mu_k = -1 + 2k/(n_w - 1)
// (h_w = sum_k w_k phi_k), Z(w) = int p h_w. One cluster of CTAs writes the
// packed blob of p_w's equal-probability table in the layout of
// table_format.h, so the walk, the camera density and the adjoint use it like
// any table:
//   1. each bin's mass p_j int h_w (h_w is linear between hat nodes, so
//      trapezoids piece by piece are exact), in double precision;
//   2. their running sum (a fixed-order block scan), Z(w) its total;
//   3. each level i: the bin whose running sum brackets i Z / n, and inside it
//      the root of the quadratic partial mass of the piece holding the level;
//   4. per-bin densities of the single-precision levels, the table mean and
//      the camera-density guide, computed with the same single-precision
//      operations as the host table builder's guide.
// Weights must be positive and finite; otherwise (or if single precision
// cannot hold the levels apart) the blob gets an invalid header, so a walk
// using it stops with MC_EFLAG_TABLE, and MC_EFLAG_NUMERIC is set.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "table_format.h"

namespace mcx {
namespace {

namespace cg = cooperative_groups;

constexpr int WT_BLOCK = 1024;
constexpr int WT_CLUSTER = 8;   // CTAs of the one cluster (a portable cluster size)
constexpr unsigned FULL = 0xffffffffu;

// h_w at cos theta = mu: the two hats around mu
__device__ __forceinline__ double hw_at(const float *w, int n_w, double mu)
{
    const double t = (mu + 1.0) * (0.5 * (n_w - 1));
    int k = (int)floor(t);
    k = min(max(k, 0), n_w - 2);
    const double f = fmin(fmax(t - (double)k, 0.0), 1.0);
    return (double)w[k] * (1.0 - f) + (double)w[k + 1] * f;
}

// Pieces of bin [v_hi -> v_lo] in 1 - cos theta (v_hi > v_lo) between the
// hat nodes v_k = 2 - 2k/(n_w - 1) it contains, in order of decreasing v;
// fn(a, b, ha, hb) is called for each piece from a down to b.
template <class Fn>
__device__ __forceinline__ void for_pieces(const float *w, int n_w, double v_hi, double v_lo, Fn fn)
{
    const double step = 2.0 / (n_w - 1);
    // nodes strictly inside (v_lo, v_hi): k with 2 - k step in that range,
    // i.e. k in ((2 - v_hi) / step, (2 - v_lo) / step)
    int k0 = (int)floor((2.0 - v_hi) / step) + 1, k1 = (int)ceil((2.0 - v_lo) / step) - 1;
    k0 = max(k0, 0);
    k1 = min(k1, n_w - 1);
    double a = v_hi, ha = hw_at(w, n_w, 1.0 - v_hi);
    for (int k = k0; k <= k1; ++k) {
        const double vk = 2.0 - k * step;
        if (!(vk < a && vk > v_lo)) continue;
        const double hk = (double)w[k];
        if (!fn(a, vk, ha, hk)) return;
        a = vk;
        ha = hk;
    }
    fn(a, v_lo, ha, hw_at(w, n_w, 1.0 - v_lo));
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];   // fixed order
    return t;
}

// Exclusive prefix, in thread order, of one double per thread (warp scans,
// then the warps' totals); every thread of the CTA calls it. red: 32 doubles.
__device__ __forceinline__ double block_exclusive(double own, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        red[lane] = t;   // inclusive sums of the warps' totals
    }
    __syncthreads();
    return (incl - own) + (warp > 0 ? red[warp - 1] : 0.0);
}

// Level i of p_w (in 1 - cos theta): the bin whose running mass brackets
// i Z / n, then the root of the piece's quadratic partial mass.
__device__ __forceinline__ double level_of(int i, int n, double Z, const double *cum, const double *ve,
                                           const float *bpdf, const float *w, int n_w)
{
    if (i <= 0) return ve[0];
    if (i >= n) return 0.0;
    const double target = Z * ((double)i / n);
    int lo = 0, hi = n - 1;   // largest j with cum[j] <= target
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cum[mid] <= target) lo = mid; else hi = mid - 1;
    }
    const int j = lo;
    double rem = (target - cum[j]) / (double)bpdf[j];   // remaining mass / p_j: an integral of h_w
    double v = ve[j + 1];
    for_pieces(w, n_w, ve[j], ve[j + 1], [&](double a, double b, double ha, double hbv) {
        const double piece = 0.5 * (ha + hbv) * (a - b);
        if (rem <= piece) {
            // h(x) = ha + s x, x = a - v: ha x + s x^2 / 2 = rem
            const double s = (hbv - ha) / (a - b);
            const double x = 2.0 * rem / (ha + sqrt(fmax(ha * ha + 2.0 * s * rem, 0.0)));
            v = fmin(fmax(a - x, b), a);
            return false;
        }
        rem -= piece;
        return true;
    });
    return v;
}

// X: the layout of an n-bin blob (the base blob's header must agree). One
// cluster of WT_CLUSTER CTAs: CTA r owns bins [r c, r c + c), c = ceil(n /
// WT_CLUSTER), and computes their widths, masses and levels, the part that
// costs double-precision arithmetic; the per-bin values are exchanged through
// distributed shared memory, and every CTA runs the same fixed-order scans
// over the whole table (cheap additions), so all see identical edges and
// running masses. Dynamic shared memory: double ve[n + 1], cum[n + 1],
// mine[c + 1], red[32], part[2].
__global__ void __launch_bounds__(WT_BLOCK) weighted_table_kernel(const unsigned char *base, mc_table_header X,
                                                                  int n_w, const float *w, unsigned char *out,
                                                                  uint32_t *err)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), nr = (int)cluster.num_blocks();
    const int n = X.n_bins;
    const int c = (n + nr - 1) / nr;
    const int r0 = min(rank * c, n), r1 = min(r0 + c, n);
    extern __shared__ __align__(16) double sh[];
    const mc_table_header *hb = reinterpret_cast<const mc_table_header *>(base);
    mc_table_header *ho = reinterpret_cast<mc_table_header *>(out);
    double *ve = sh;
    double *cum = ve + n + 1;
    double *mine = cum + n + 1;
    double *red = mine + c + 1;
    double *part = red + 32;   // [0]: this CTA's share of the mean, [1]: its failure flag
    bool bad = false;
    for (int k = threadIdx.x; k < n_w; k += blockDim.x) bad |= !(w[k] > 0.0f) || !isfinite(w[k]);
    if (hb->magic != MC_TABLE_MAGIC || hb->n_bins != n || hb->n_guide != X.n_guide || hb->off_omu != X.off_omu ||
        hb->off_pdf != X.off_pdf || hb->off_guide != X.off_guide || hb->total_bytes != X.total_bytes)
        bad = true;
    if (__syncthreads_or(bad)) {   // the same inputs in every CTA: all leave here together
        if (rank == 0 && threadIdx.x == 0) {
            atomicOr(err, MC_EFLAG_NUMERIC);
            ho->magic = 0u;    // walks using this blob stop with MC_EFLAG_TABLE
        }
        return;
    }
    const float *bpdf = reinterpret_cast<const float *>(base + hb->off_pdf);
    float *oo = reinterpret_cast<float *>(out + hb->off_omu);
    float *op = reinterpret_cast<float *>(out + hb->off_pdf);
    uint16_t *og = reinterpret_cast<uint16_t *>(out + hb->off_guide);
    const double inv_n = 1.0 / n;
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    // every CTA's value of bin j, into a full local array
    auto gather = [&](double *dst, int shift) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double *src = cluster.map_shared_rank(mine, j / c);
            dst[j + shift] = src[j % c];
        }
    };

    // 0. the unweighted table's edges in double precision from its bin
    // densities (each bin holds 1/n): widths (1/n) / pdf_j summed from the
    // forward end, omu = 0, so every edge keeps the densities' relative
    // precision. Thread t owns the t-th run of bins counted from that end.
    for (int j = r0 + threadIdx.x; j < r1; j += blockDim.x) mine[j - r0] = inv_n / (double)bpdf[j];
    cluster.sync();
    gather(ve, 0);
    __syncthreads();
    {
        const int jhi = max(n - (int)threadIdx.x * per, 0), jlo = max(jhi - per, 0);
        double own = 0.0;
        for (int j = jhi - 1; j >= jlo; --j) {
            own += ve[j];
            ve[j] = own;   // local suffix sum for now
        }
        const double before = block_exclusive(own, red);
        for (int j = jlo; j < jhi; ++j) ve[j] += before;
        if (threadIdx.x == 0) ve[n] = 0.0;
    }
    cluster.sync();   // every CTA has read the widths: mine is free again

    // 1-2. bin masses p_j int h_w (this CTA's bins) and their running sum
    // (over the whole table; thread t owns the t-th run of bins from mu = -1)
    for (int j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
        double m = 0.0;
        for_pieces(w, n_w, ve[j], ve[j + 1], [&](double a, double b, double ha, double hbv) {
            m += 0.5 * (ha + hbv) * (a - b);
            return true;
        });
        mine[j - r0] = (double)bpdf[j] * m;
    }
    cluster.sync();
    gather(cum, 1);
    __syncthreads();
    {
        const int j0 = min((int)threadIdx.x * per, n), j1 = min(j0 + per, n);
        double own = 0.0;
        for (int j = j0; j < j1; ++j) {
            own += cum[j + 1];
            cum[j + 1] = own;   // local running sum for now
        }
        const double before = block_exclusive(own, red);
        for (int j = j0; j < j1; ++j) cum[j + 1] += before;
        if (threadIdx.x == 0) cum[0] = 0.0;
    }
    cluster.sync();   // every CTA has read the masses: mine is free again
    const double Z = cum[n];

    // 3-4. this CTA's levels r0 .. r1 (one solve each), the densities of its
    // bins from the double levels (as the host builder does), its share of
    // the mean
    for (int i = r0 + threadIdx.x; i <= r1; i += blockDim.x) mine[i - r0] = level_of(i, n, Z, cum, ve, bpdf, w, n_w);
    __syncthreads();
    double msum = 0.0;
    for (int j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
        const double vj = mine[j - r0], vn = mine[j + 1 - r0];
        oo[j] = j == 0 ? 2.0f : (float)vj;
        const double width = vj - vn;
        if (!(width > 0.0)) bad = true;
        op[j] = (float)(inv_n / width);
        msum += 1.0 - 0.5 * (vj + vn);
    }
    if (r1 == n && threadIdx.x == 0) oo[n] = 0.0f;
    const double share = block_sum(msum, red);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        part[0] = share;
        part[1] = bad ? 1.0 : 0.0;
    }
    __threadfence();   // the levels in global memory, before the guide reads them
    cluster.sync();
    double mean = 0.0;
    bool any_bad = false;
    for (int q = 0; q < nr; ++q) {   // fixed order
        const double *pq = cluster.map_shared_rank(part, q);
        mean += pq[0];
        any_bad |= pq[1] != 0.0;
    }
    mean *= inv_n;
    cluster.sync();   // no CTA leaves while others read its shares
    if (any_bad) {
        if (rank == 0 && threadIdx.x == 0) {
            atomicOr(err, MC_EFLAG_NUMERIC);
            ho->magic = 0u;
        }
        return;
    }

    // guide[c]: bin of the smallest float m with cell(m) >= c, where the
    // walk's lookup takes cell(m) = floor(fl(m + 1) (n_guide / 2)) and bin(m)
    // = the largest j with omu[j] >= fl(1 - m); this CTA's share of the cells
    const int G = hb->n_guide;
    const int gc = (G + 1 + nr - 1) / nr, g0 = min(rank * gc, G + 1), g1 = min(g0 + gc, G + 1);
    const float half_g = 0.5f * (float)G;
    auto cell_of = [&](float m) { return (int)floorf((m + 1.0f) * half_g); };
    auto bin_of = [&](float m) {
        const float om = 1.0f - m;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (oo[mid] >= om) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    auto key_of = [](float f) {
        const uint32_t b = __float_as_uint(f);
        return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    };
    auto float_of = [](uint32_t k) {
        return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
    };
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        float m;
        if (g == 0) {
            m = -1.0f;
        } else if (g == G) {
            m = 1.0f;
        } else {
            uint32_t lo = key_of(-1.0f), hi = key_of(1.0f);
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if (cell_of(float_of(mid)) >= g) hi = mid; else lo = mid + 1;
            }
            m = float_of(lo);
        }
        og[g] = (uint16_t)bin_of(m);
    }
    if (rank == 0 && threadIdx.x == 0) {
        mc_table_header h = *hb;
        h.g_table = (float)mean;
        *ho = h;
    }
}

}  // namespace

size_t weighted_table_smem(int n_bins)
{
    const size_t c = ((size_t)n_bins + WT_CLUSTER - 1) / WT_CLUSTER;
    return sizeof(double) * (2 * ((size_t)n_bins + 1) + (c + 1) + 32 + 2);
}

cudaError_t launch_weighted_table(const unsigned char *base, int n_bins, int n_w, const float *w,
                                  unsigned char *out, uint32_t *err, cudaStream_t st)
{
    mc_table_header X;
    if (!mc_table_layout(n_bins, &X) || n_bins > kMaxWeightedBins) return cudaErrorInvalidValue;
    const size_t smem = weighted_table_smem(n_bins);
    cudaError_t e = cudaFuncSetAttribute(weighted_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(WT_CLUSTER);
    cfg.blockDim = dim3(WT_BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = WT_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, weighted_table_kernel, base, X, n_w, w, out, err);
}

}  // namespace mcx
