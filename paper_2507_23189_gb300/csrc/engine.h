// Internal interface between the C ABI layer (api.cu) and the kernels (walk.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mcmie.h"

namespace mcx {

// Per-medium parameters, already validated and in the kernels' precision.
struct MediumArgs {
    float mu_ext, inv_mu_ext;   // mm^-1, mm
    float albedo;               // 1 - mu_a/mu_ext (Eq. 16 factor)
    float absorb_frac;          // mu_a/mu_ext
    float hg_g, hg_one_m_g, hg_two_g;
    float hg_A;                 // 2 (1-g)^2        (sampling 1 - cos)
    float hg_B;                 // 2 (1+g)^2        (sampling 1 + cos)
    float hg_a2;                // (1-g)^2           (density)
    float hg_K;                 // (1-g^2) / (4 pi)  (density per sr)
    const unsigned char *table; // packed blob in global memory (table_format.h)
    uint32_t key0, key1;        // Philox key (seed)
    uint32_t rk[20];            // Philox round keys: rk[2i] = key0 + i W0, rk[2i+1] = key1 + i W1
    unsigned long long n_photons, photon_offset;
    unsigned long long *image, *radial, *totals;  // this medium's tallies
};

// Parameters shared by every medium of a launch.
struct CommonArgs {
    int phase_kind;             // MC_PHASE_TABLE / MC_PHASE_HG (one per launch)
    uint32_t table_bytes;
    int n_bins;
    // geometry
    float lx, hy, hz, beam_r;
    // camera
    int nx, nz, n_radial;
    float sx, sz, sr;           // nx/lx, nz/lz, n_radial/r_max
    // run
    float rr_thr, rr_surv, inv_rr_surv;
    uint32_t max_events, max_scatter;
    float img_scale;            // 2^image_frac_bits
    uint32_t *error;
    // image rows [band0, band0 + band_rows) are privatised in shared memory
    // (set by the launcher; band_rows = nz for a whole-image tile)
    int band0, band_rows;
    // trace (trace kernels only)
    int32_t *trace;
    int n_trace, n_trace_events;
    // bytes staged after the table (the majorant cells of a grid walk)
    uint32_t extra_bytes;
};

// One medium, one photon range. Passed by value as a __grid_constant__.
struct WalkArgs {
    CommonArgs c;
    MediumArgs m;
    unsigned long long *counter;  // photon counter in the caller's workspace
};

// Many media in one launch, processed in the order of m[]: medium i's photons
// are taken in warp chunks of `chunk` from counters[i] (caller's workspace).
constexpr int kMaxBatch = 64;
struct BatchArgs {
    CommonArgs c;
    int n_media;
    unsigned chunk;               // photons a warp takes from a counter at once (>= 32)
    unsigned long long *counters; // [n_media] photon counters
    MediumArgs m[kMaxBatch];
};

// Gradient of L = sum_pix adj[pix] image[pix] for one medium (see adjoint
// kernel); partials holds one row of 3 + n_w doubles per CTA.
struct AdjArgs {
    CommonArgs c;
    MediumArgs m;               // m.table: the table the walk samples (reweighted by w if given)
    const float *adj;           // [nz][nx]
    int n_w;                    // phase-weight hats (0: none)
    const float *w;             // [n_w] phase weights (nullptr: all 1)
    const unsigned char *base_table;  // the unweighted table (hat integrals Z_k)
    float c_s;                  // 1/mu_s - 1/mu_ext
    double *z;                  // [n_w] hat integrals of the unweighted table (workspace)
    double *partials;           // [grid][3 + n_w]
    unsigned long long *counter;
};

// A heterogeneous medium on a voxel grid (mc_run_grid): per voxel
// (mu_ext, optical depth from the voxel's top face to the camera face), the
// majorant of each cell of bx x by x bz voxels, and the geometry of both.
struct GridArgs {
    CommonArgs c;
    MediumArgs m;                 // phase, Philox key, photon range, tallies
    const float2 *cells;          // [gz][gy][gx]
    const float *maj;             // [mz][my][mx], staged into shared memory
    int gx, gy, gz, mx, my, mz;
    float inv_vx, inv_vy, inv_vz; // voxels per mm
    float vx, vy, vz;             // voxel sizes, mm
    float csx, csy, csz;          // cell sizes, mm
    float inv_csx, inv_csy, inv_csz;
    float hcy, hcz;               // cells between the y (z) axis and a side, g / (2 b): exact when whole
    float ks_over_ke, mu_a;       // albedo = ks_over_ke (1 - mu_a / mu_ext)
    unsigned long long *counter;
};

// Gradient of L = sum_pix adj[pix] image[pix] with respect to the voxel
// densities (mc_grid_adjoint): point, flight and own-voxel column terms into
// gsum, the rest of each camera column as the per-voxel source s1 and each
// first flight as one row-suffix entry ex, both folded in afterwards.
struct GridAdjArgs {
    GridArgs g;
    const float *adj;             // [nz][nx]
    // [gz][gy][gx] double-precision atomic sums: point, flight and own-voxel
    // column terms; column sources above a collision; first-flight row suffix.
    // With null scores, the voxels of the box iy in [by0, by0 + bw), iz in
    // [bz0, bz0 + bw) around the beam axis (where many CTAs add at once) are
    // summed instead in `copies` copies of the box, bstride elements apart,
    // CTA b adding into copy b % copies: bgs for gsum, bs1 for s1
    double *gsum, *s1, *ex;
    double *bgs, *bs1;
    int copies, by0, bz0, bw;
    size_t nbox, bstride;
    float *grad;                  // [gz][gy][gx] output (written by the fold)
    float k_ext;
    double *partials;             // [grid] value per CTA
    int nulls;                    // 1: flight transmission scored at null collisions
    float maj_scale;              // majorants x this in the walk (nulls: > 1)
};

struct LaunchCfg {
    int block = 0;          // 0: 256 (whole tile / global) or 1024 (band)
    int blocks_per_sm = 0;  // 0: occupancy maximum
    int image_mode = 0;     // 0 auto, 1 whole image in shared memory, 2 global
                            // atomics only, 3 band of rows around the beam in
                            // shared memory, the rest global
};

// Launch the walk (or its trace variant) on `stream`. Returns cudaSuccess or
// the launch error.
cudaError_t launch_walk(const WalkArgs &a, bool trace, const LaunchCfg &cfg, cudaStream_t stream);
// The shared-memory plan of a walk, batch or grid launch without launching
// anything: cudaErrorInvalidValue when the table, the majorant cells, the
// radial profile and the totals (with the image tile image_mode 1 asks for)
// do not fit in one CTA's shared memory.
cudaError_t check_plan(const CommonArgs &c, const LaunchCfg &cfg);

// Launch the batched walk (phase fixed by c.phase_kind) on `stream`.
cudaError_t launch_batch(const BatchArgs &a, const LaunchCfg &cfg, cudaStream_t stream);

// Launch the adjoint replay and the reduction into out[3 + n_w]
// (value, dL/dmu_s, dL/dmu_a, dL/dw_k). partial_rows: capacity of partials.
cudaError_t launch_adjoint(const AdjArgs &a, int partial_rows, double *out, cudaStream_t stream);

// Launch the delta-tracking walk through a prepared grid (trace: records of
// real events in c.trace).
cudaError_t launch_grid(const GridArgs &a, bool trace, const LaunchCfg &cfg, cudaStream_t stream);

// Per-voxel (mu_ext, optical depth above) and per-cell majorants of a grid.
cudaError_t launch_grid_prepare(const float *density, int gx, int gy, int gz, int bx, int by, int bz,
                                float k_ext, float mu_a, double vy, float2 *cells, float *maj,
                                cudaStream_t stream);

// Launch the density-gradient replay, the column fold and the value reduction.
cudaError_t launch_grid_adjoint(const GridAdjArgs &a, int partial_rows, double *value, cudaStream_t stream);
// cudaErrorInvalidValue when the gradient kernel's table, majorant cells and
// flight queues do not fit in one CTA's shared memory (nothing launched).
cudaError_t grid_adjoint_check(const GridAdjArgs &a);

// grad[v] = gsum[v] + vx * (sum of ex after v in its row along x)
//           - k_ext vy * (sum of s1 below v in its column along y); gsum is
// updated in place by the row sums; ex null: no row terms.
cudaError_t launch_gradient_fold(double *gsum, const double *s1, const double *ex, float *grad, int gx, int gy,
                                 int gz, double k_ext, double vx, double vy, cudaStream_t stream);

// gsum[v] += sum over the copies of bgs at v's box element, s1 likewise
// (copies bstride elements apart, summed in copy order).
cudaError_t launch_box_merge(double *gsum, double *s1, const double *bgs, const double *bs1, int copies,
                             size_t nbox, size_t bstride, int gx, int gy, int by0, int bz0, int bw,
                             cudaStream_t stream);

// The null-score gradient's copies of the voxel sums near the beam axis: how
// many, and the box's width in voxels along y and z (at most the grid's).
constexpr int kNullCopies = 8;
constexpr int kNullBox = 32;

// CTAs the grid adjoint may use on the current device (for workspace sizing).
int grid_adjoint_max_grid();

// CTAs the adjoint launch may use on the current device (for workspace sizing).
int adjoint_max_grid();

cudaError_t launch_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out,
                          cudaStream_t stream);

// Largest table the device reweighting takes (two double arrays of n_bins + 1
// entries in shared memory).
constexpr int kMaxWeightedBins = 8192;

// The equal-probability table of p h_w / Z(w) from the unweighted table blob
// `base` (n_bins bins) and n_w device weights, into `out` (the same layout);
// one CTA. Invalid weights set MC_EFLAG_NUMERIC and an invalid header.
cudaError_t launch_weighted_table(const unsigned char *base, int n_bins, int n_w, const float *w,
                                  unsigned char *out, uint32_t *err, cudaStream_t stream);

// The bounded mbarrier wait on a phase that cannot complete (self-test).
cudaError_t launch_wait_selftest(uint32_t *err, uint32_t tries, cudaStream_t stream);

}  // namespace mcx
