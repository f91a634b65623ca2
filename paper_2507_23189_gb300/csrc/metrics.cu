// Image comparison metrics on the device (mc_image_metrics, include/mcmie.h):
// Sec. 3.1.4 normalises every image the same way (min-max to [0, 1] here),
// Table 3 compares images by RMSE and Pearson r, Table 4 compares radial
// profiles (means over rings about the image centre) zone by zone.
//
// Four small launches, all in double precision with fixed-order reductions,
// so the numbers do not depend on scheduling:
//   minmax_kernel  one CTA per image: min and max of the int64 image
//   ring_kernel    one CTA per (ring, image), plus one per image for the
//                  plain sum: sum of normalised values and pixel count
//   pair_kernel    one CTA per compared pair: squared error and the centred
//                  cross / auto products of the normalised images
//   final_kernel   one thread: profiles, zone errors, profile correlation
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/mcmie.h"

namespace {

constexpr int MB = 256;        // threads per CTA, fixed: sums are ordered by it
constexpr int MAX_RINGS = 4096;

struct Imgs {
    const long long *p[3];
};

__device__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = MB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Normalised value of pixel v of an image with extremes mn, mx.
__device__ __forceinline__ double norm_px(long long v, double mn, double mx)
{
    return mx == mn ? 0.0 : ((double)v - mn) / (mx - mn);
}

__global__ void __launch_bounds__(MB) minmax_kernel(Imgs im, long long npix, long long *mm)
{
    __shared__ long long smin[MB], smax[MB];
    const long long *a = im.p[blockIdx.x];
    long long lo = a[0], hi = a[0];
    for (long long i = threadIdx.x; i < npix; i += MB) {
        lo = min(lo, a[i]);
        hi = max(hi, a[i]);
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int s = MB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smin[threadIdx.x] = min(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mm[2 * blockIdx.x] = smin[0];
        mm[2 * blockIdx.x + 1] = smax[0];
    }
}

// Ring of pixel (ix, iz): polar radius about the image centre in pixel units,
// n_r equal rings out to the half-diagonal (the radius itself goes last).
__device__ __forceinline__ int ring_of(int ix, int iz, int nx, int nz, double rho_max, int n_r)
{
    const double dx = ((double)ix + 0.5) - (double)nx / 2.0;
    const double dz = ((double)iz + 0.5) - (double)nz / 2.0;
    const double rho = sqrt(dx * dx + dz * dz);
    const double t = floor(rho / rho_max * (double)n_r);
    return t < (double)(n_r - 1) ? (int)t : n_r - 1;
}

__device__ __forceinline__ double half_diagonal(int nx, int nz)
{
    const double hx = (double)nx / 2.0, hz = (double)nz / 2.0;
    return sqrt(hx * hx + hz * hz);
}

// blockIdx.x < n_r: ring sums; blockIdx.x == n_r: whole-image sum.
__global__ void __launch_bounds__(MB) ring_kernel(Imgs im, int nx, int nz, int n_r, const long long *mm,
                                                  double *ring_sum, long long *ring_cnt, double *tot)
{
    __shared__ double sh[MB];
    const int b = blockIdx.x, k = blockIdx.y;
    const long long *a = im.p[k];
    const double mn = (double)mm[2 * k], mx = (double)mm[2 * k + 1];
    const long long npix = (long long)nx * nz;
    const double rho_max = half_diagonal(nx, nz);
    double s = 0.0;
    long long c = 0;
    for (long long i = threadIdx.x; i < npix; i += MB) {
        const int iz = (int)(i / nx), ix = (int)(i - (long long)iz * nx);
        if (b == n_r || ring_of(ix, iz, nx, nz, rho_max, n_r) == b) {
            s += norm_px(a[i], mn, mx);
            ++c;
        }
    }
    const double S = block_sum(s, sh);
    const double Cn = block_sum((double)c, sh);   // exact: counts < 2^53
    if (threadIdx.x == 0) {
        if (b == n_r) {
            tot[k] = S;
        } else {
            ring_sum[(size_t)k * n_r + b] = S;
            if (k == 0) ring_cnt[b] = (long long)Cn;
        }
    }
}

// Pair p compares image 1 + p with image 0 (the reference).
__global__ void __launch_bounds__(MB) pair_kernel(Imgs im, long long npix, const long long *mm,
                                                  const double *tot, double *pair)
{
    __shared__ double sh[MB];
    const int k = 1 + blockIdx.x;
    const long long *a = im.p[k], *r = im.p[0];
    const double amn = (double)mm[2 * k], amx = (double)mm[2 * k + 1];
    const double rmn = (double)mm[0], rmx = (double)mm[1];
    const double am = tot[k] / (double)npix, rm = tot[0] / (double)npix;
    double se = 0.0, sar = 0.0, saa = 0.0, srr = 0.0;
    for (long long i = threadIdx.x; i < npix; i += MB) {
        const double va = norm_px(a[i], amn, amx), vr = norm_px(r[i], rmn, rmx);
        const double e = va - vr, da = va - am, dr = vr - rm;
        se += e * e;
        sar += da * dr;
        saa += da * da;
        srr += dr * dr;
    }
    se = block_sum(se, sh);
    sar = block_sum(sar, sh);
    saa = block_sum(saa, sh);
    srr = block_sum(srr, sh);
    if (threadIdx.x == 0) {
        double *o = pair + 4 * blockIdx.x;
        o[0] = se; o[1] = sar; o[2] = saa; o[3] = srr;
    }
}

__device__ double pearson_profiles(const double *a, const double *r, const long long *cnt, int n_r)
{
    double sa = 0.0, sr = 0.0;
    int m = 0;
    for (int b = 0; b < n_r; ++b)
        if (cnt[b]) { sa += a[b]; sr += r[b]; ++m; }
    if (m == 0) return 0.0;
    const double ma = sa / m, mr = sr / m;
    double sar = 0.0, saa = 0.0, srr = 0.0;
    for (int b = 0; b < n_r; ++b)
        if (cnt[b]) {
            const double da = a[b] - ma, dr = r[b] - mr;
            sar += da * dr; saa += da * da; srr += dr * dr;
        }
    return (saa == 0.0 || srr == 0.0) ? 0.0 : sar / sqrt(saa * srr);
}

__global__ void final_kernel(int n_img, long long npix, int n_r, const double *ring_sum,
                             const long long *ring_cnt, const double *pair, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double *prof = out + 13;   // [3][n_r]
    for (int k = 0; k < 3; ++k)
        for (int b = 0; b < n_r; ++b)
            prof[k * n_r + b] = (k < n_img && ring_cnt[b]) ? ring_sum[(size_t)k * n_r + b] / (double)ring_cnt[b]
                                                           : 0.0;
    for (int i = 0; i < 13; ++i) out[i] = 0.0;
    int m = 0;
    for (int b = 0; b < n_r; ++b) m += ring_cnt[b] ? 1 : 0;
    for (int p = 0; p + 1 < n_img; ++p) {
        const double *P = pair + 4 * p;
        double *o = out + 6 * p;
        o[0] = sqrt(P[0] / (double)npix);
        o[1] = (P[2] == 0.0 || P[3] == 0.0) ? 0.0 : P[1] / sqrt(P[2] * P[3]);
        const double *pa = prof + (1 + p) * n_r, *pr = prof;
        for (int z = 0; z < 3; ++z) {
            double s = 0.0;
            int c = 0;
            for (int b = 0; b < n_r; ++b) {
                if (!ring_cnt[b]) continue;
                const double ang = 180.0 * ((double)b + 0.5) / (double)n_r;
                const int zb = ang < 30.0 ? 0 : (ang <= 120.0 ? 1 : 2);
                if (zb != z) continue;
                const double d = pa[b] - pr[b];
                s += d * d;
                ++c;
            }
            o[2 + z] = c ? sqrt(s / (double)c) : 0.0;
        }
        o[5] = pearson_profiles(pa, pr, ring_cnt, n_r);
    }
    if (n_img == 3) {
        int closer = 0;
        for (int b = 0; b < n_r; ++b)
            if (ring_cnt[b] && fabs(prof[n_r + b] - prof[b]) < fabs(prof[2 * n_r + b] - prof[b])) ++closer;
        out[12] = m ? (double)closer / (double)m : 0.0;
    }
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int mc_metrics_out_len(int n_r) { return (n_r < 1 || n_r > MAX_RINGS) ? 0 : 13 + 3 * n_r; }

extern "C" size_t mc_metrics_workspace_bytes(int n_r)
{
    if (n_r < 1 || n_r > MAX_RINGS) return 0;
    return up256(sizeof(long long) * 6) + up256(sizeof(double) * 3 * (size_t)n_r) +
           up256(sizeof(long long) * (size_t)n_r) + up256(sizeof(double) * 3) + up256(sizeof(double) * 8);
}

extern "C" mc_status mc_image_metrics(const int64_t *d_ref, const int64_t *d_a, const int64_t *d_b, int nx,
                                      int nz, int n_r, double *d_out, void *d_work, size_t work_bytes,
                                      void *stream)
{
    if (!d_ref || !d_a || !d_out || !d_work || nx < 1 || nz < 1 || (long long)nx * nz > (1ll << 26) ||
        n_r < 1 || n_r > MAX_RINGS || (reinterpret_cast<uintptr_t>(d_work) & 15) ||
        (reinterpret_cast<uintptr_t>(d_out) & 7) || (reinterpret_cast<uintptr_t>(d_ref) & 7) ||
        (reinterpret_cast<uintptr_t>(d_a) & 7) || (d_b && (reinterpret_cast<uintptr_t>(d_b) & 7)))
        return MC_ERR_ARG;
    if (work_bytes < mc_metrics_workspace_bytes(n_r)) return MC_ERR_NOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *w = static_cast<unsigned char *>(d_work);
    long long *mm = reinterpret_cast<long long *>(w);
    w += up256(sizeof(long long) * 6);
    double *ring_sum = reinterpret_cast<double *>(w);
    w += up256(sizeof(double) * 3 * (size_t)n_r);
    long long *ring_cnt = reinterpret_cast<long long *>(w);
    w += up256(sizeof(long long) * (size_t)n_r);
    double *tot = reinterpret_cast<double *>(w);
    w += up256(sizeof(double) * 3);
    double *pair = reinterpret_cast<double *>(w);
    Imgs im;
    im.p[0] = reinterpret_cast<const long long *>(d_ref);
    im.p[1] = reinterpret_cast<const long long *>(d_a);
    im.p[2] = reinterpret_cast<const long long *>(d_b ? d_b : d_a);
    const int n_img = d_b ? 3 : 2;
    const long long npix = (long long)nx * nz;
    minmax_kernel<<<n_img, MB, 0, st>>>(im, npix, mm);
    ring_kernel<<<dim3(n_r + 1, n_img), MB, 0, st>>>(im, nx, nz, n_r, mm, ring_sum, ring_cnt, tot);
    pair_kernel<<<n_img - 1, MB, 0, st>>>(im, npix, mm, tot, pair);
    final_kernel<<<1, 32, 0, st>>>(n_img, npix, n_r, ring_sum, ring_cnt, pair, d_out);
    return cudaGetLastError() == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}
