// Preparation of a heterogeneous medium for the delta-tracking walk
// (mc_grid_prepare): per voxel mu_ext = k_ext n + mu_a (Eq. 17 per voxel)
// and the optical depth from the voxel's top face to the camera face
// y = +ly/2, which makes the camera transmittance of any collision exact
// with one gather; and the majorant of every cell of bx x by x bz voxels.
#include <cuda_runtime.h>

#include "engine.h"

namespace mcx {
namespace {

// One thread per (x, z) column, walking down from the camera face: writes
// (mu_ext, depth above) per voxel; consecutive threads touch consecutive x,
// so every row access is coalesced. The depth is summed in double.
__global__ void column_kernel(const float *__restrict__ density, int gx, int gy, int gz, float k_ext,
                              float mu_a, double vy, float2 *__restrict__ cells)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)gx * gz) return;
    const int iz = (int)(t / gx), ix = (int)(t - (long long)iz * gx);
    double od = 0.0;
    for (int iy = gy - 1; iy >= 0; --iy) {
        const size_t v = ((size_t)iz * gy + iy) * gx + ix;
        const float mu = fmaf(k_ext, density[v], mu_a);
        cells[v] = make_float2(mu, (float)od);
        od += (double)mu * vy;
    }
}

// Majorants: blockIdx.y picks the cell, blockIdx.x a piece of MAJ_CHUNK of
// its voxels; each CTA reduces its piece to the largest mu_ext (the same
// single-precision fmaf as the voxels, so no voxel exceeds its majorant) and
// merges it with atomicMax on the float's bits, which order like the
// non-negative floats they are (maj starts at 0).
constexpr int MAJ_CHUNK = 8192;

__global__ void __launch_bounds__(256) majorant_kernel(const float *__restrict__ density, int gx, int gy,
                                                       int gz, int bx, int by, int bz, int mx, int my,
                                                       float k_ext, float mu_a, float *__restrict__ maj)
{
    __shared__ float red[256];
    const int c = blockIdx.y;
    const int cz = c / (mx * my), cy = (c / mx) % my, cx = c % mx;
    const int x0 = cx * bx, y0 = cy * by, z0 = cz * bz;
    const int nxb = min(bx, gx - x0), nyb = min(by, gy - y0), nzb = min(bz, gz - z0);
    const long long nv = (long long)nxb * nyb * nzb;
    const long long i0 = (long long)blockIdx.x * MAJ_CHUNK;
    const long long i1 = min(nv, i0 + MAJ_CHUNK);
    float m = 0.0f;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int xi = (int)(i % nxb), yi = (int)((i / nxb) % nyb), zi = (int)(i / ((long long)nxb * nyb));
        m = fmaxf(m, fmaf(k_ext, density[((size_t)(z0 + zi) * gy + (y0 + yi)) * gx + (x0 + xi)], mu_a));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<int *>(&maj[c]), __float_as_int(fmaxf(red[0], 0.0f)));
}

// One warp per voxel row along x, from its far end: every voxel before the
// one where a first flight ended takes the full voxel length vx of that
// flight's coefficient, gsum[ix] += vx * sum_{j > ix} ex[j]. Chunks of 32
// voxels with a warp suffix scan; rows with no entries cost their loads.
__global__ void row_suffix_kernel(double *__restrict__ gsum, const double *__restrict__ ex, int gx,
                                  long long rows, double vx)
{
    const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (r >= rows) return;   // whole warps leave together
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)r * gx;
    double carry = 0.0;      // sum of ex beyond the current chunk
    for (int c = ((gx - 1) >> 5) << 5; c >= 0; c -= 32) {
        const int ix = c + lane;
        const double e = ix < gx ? ex[base + ix] : 0.0;
        if (__any_sync(0xFFFFFFFFu, e != 0.0)) {
            double s = e;    // inclusive suffix within the chunk
            for (int o = 1; o < 32; o <<= 1) {
                const double t = __shfl_down_sync(0xFFFFFFFFu, s, o);
                if (lane + o < 32) s += t;
            }
            const double after = __shfl_down_sync(0xFFFFFFFFu, s, 1);
            const double total = __shfl_sync(0xFFFFFFFFu, s, 0);
            const double add = carry + (lane < 31 ? after : 0.0);
            if (ix < gx && add != 0.0) gsum[base + ix] += vx * add;
            carry += total;
        } else if (carry != 0.0 && ix < gx) {
            gsum[base + ix] += vx * carry;
        }
    }
}

// One thread per (x, z) column, upward: a camera term A at a collision in
// voxel iy takes A times a full voxel height in every voxel above it (s1,
// summed below); its part in its own voxel is already in gsum.
__global__ void fold_kernel(const double *__restrict__ gsum, const double *__restrict__ s1,
                            float *__restrict__ grad, int gx, int gy, int gz, double k_vy)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)gx * gz) return;
    const int iz = (int)(t / gx), ix = (int)(t - (long long)iz * gx);
    double run = 0.0;
    for (int iy = 0; iy < gy; ++iy) {
        const size_t v = ((size_t)iz * gy + iy) * gx + ix;
        grad[v] = (float)(gsum[v] - k_vy * run);
        run += s1[v];
    }
}

}  // namespace

namespace {
// One thread per box element (ix fastest): its copies summed in copy order
// into the voxel's own sums.
__global__ void box_merge_kernel(double *__restrict__ gsum, double *__restrict__ s1, const double *__restrict__ bgs,
                                 const double *__restrict__ bs1, int copies, size_t nbox, size_t bstride, int gx,
                                 int gy, int by0, int bz0, int bw)
{
    for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < nbox; b += (size_t)gridDim.x * blockDim.x) {
        double tg = 0.0, ts = 0.0;
        for (int c = 0; c < copies; ++c) {
            tg += bgs[(size_t)c * bstride + b];
            ts += bs1[(size_t)c * bstride + b];
        }
        const int ix = (int)(b % (size_t)gx);
        const size_t r = b / (size_t)gx;
        const int iy = by0 + (int)(r % (size_t)bw), iz = bz0 + (int)(r / (size_t)bw);
        const size_t v = ((size_t)iz * gy + iy) * gx + ix;
        gsum[v] += tg;
        s1[v] += ts;
    }
}
}  // namespace

cudaError_t launch_box_merge(double *gsum, double *s1, const double *bgs, const double *bs1, int copies,
                             size_t nbox, size_t bstride, int gx, int gy, int by0, int bz0, int bw, cudaStream_t st)
{
    box_merge_kernel<<<1024, 256, 0, st>>>(gsum, s1, bgs, bs1, copies, nbox, bstride, gx, gy, by0, bz0, bw);
    return cudaGetLastError();
}

cudaError_t launch_gradient_fold(double *gsum, const double *s1, const double *ex, float *grad, int gx, int gy,
                                 int gz, double k_ext, double vx, double vy, cudaStream_t st)
{
    cudaError_t e;
    if (ex) {
        const long long rows = (long long)gy * gz;
        row_suffix_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(gsum, ex, gx, rows, vx);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const long long cols = (long long)gx * gz;
    fold_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(gsum, s1, grad, gx, gy, gz, k_ext * vy);
    return cudaGetLastError();
}

cudaError_t launch_grid_prepare(const float *density, int gx, int gy, int gz, int bx, int by, int bz,
                                float k_ext, float mu_a, double vy, float2 *cells, float *maj,
                                cudaStream_t st)
{
    const long long cols = (long long)gx * gz;
    column_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(density, gx, gy, gz, k_ext, mu_a,
                                                                  vy, cells);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int mx = (gx + bx - 1) / bx, my = (gy + by - 1) / by, mz = (gz + bz - 1) / bz;
    if ((e = cudaMemsetAsync(maj, 0, sizeof(float) * (size_t)mx * my * mz, st)) != cudaSuccess) return e;
    const long long per_cell = (long long)bx * by * bz;
    const dim3 grid((unsigned)((per_cell + MAJ_CHUNK - 1) / MAJ_CHUNK), (unsigned)(mx * my * mz));
    majorant_kernel<<<grid, 256, 0, st>>>(density, gx, gy, gz, bx, by, bz, mx, my, k_ext, mu_a, maj);
    return cudaGetLastError();
}

}  // namespace mcx
