// Packed phase-table blob shared by the host table builder and the kernels.
//
// One contiguous, 16-byte aligned block so a single bulk copy stages it into
// shared memory. Layout (byte offsets from the start of the blob):
//   [0, 64)            mc_table_header
//   off_omu            float omu[n_bins + 1]   1 - cos(theta) at levels i/n_bins
//   off_pdf            float pdf[n_bins]       density per unit cos(theta) of bin j
//   off_guide          uint16 guide[n_guide+1] first candidate bin per cos-cell
// Sections are padded to 16 bytes; total_bytes is a multiple of 16.
#pragma once
#include <stddef.h>
#include <stdint.h>

#define MC_TABLE_MAGIC 0x544D434Du  // "MCMT"
#define MC_TABLE_VERSION 1u

struct mc_table_header {
    uint32_t magic;
    uint32_t version;
    int32_t n_bins;
    int32_t n_guide;
    uint32_t off_omu;
    uint32_t off_pdf;
    uint32_t off_guide;
    uint32_t total_bytes;
    float g_table;
    float pad[7];
};
static_assert(sizeof(mc_table_header) == 64, "header must be 64 bytes");

static inline size_t mc_pad16(size_t b) { return (b + 15) & ~(size_t)15; }

// Fills the offsets for n_bins bins; returns total bytes (0 if n_bins invalid).
static inline size_t mc_table_layout(int n_bins, mc_table_header *h)
{
    if (n_bins < 64 || n_bins > 16384 || (n_bins & (n_bins - 1)))
        return 0;
    size_t off = sizeof(mc_table_header);
    size_t omu = off;
    off += mc_pad16(sizeof(float) * (size_t)(n_bins + 1));
    size_t pdf = off;
    off += mc_pad16(sizeof(float) * (size_t)n_bins);
    size_t guide = off;
    off += mc_pad16(sizeof(uint16_t) * (size_t)(n_bins + 1));
    if (h) {
        h->magic = MC_TABLE_MAGIC;
        h->version = MC_TABLE_VERSION;
        h->n_bins = n_bins;
        h->n_guide = n_bins;
        h->off_omu = (uint32_t)omu;
        h->off_pdf = (uint32_t)pdf;
        h->off_guide = (uint32_t)guide;
        h->total_bytes = (uint32_t)off;
        h->g_table = 0.0f;
        for (int i = 0; i < 7; ++i) h->pad[i] = 0.0f;
    }
    return off;
}

// The paper's own sampling table (Sec. 3.1.2): the cumulative distribution
// of the scattering angle at n_theta equally spaced angles theta_i =
// i pi / n_int (n_int = n_theta - 1), searched by bisection. Layout:
//   [0, 64)   mc_paper_header
//   off_k     uint32 k[n_int + 1]  k[i] = smallest 23-bit uniform index q with
//                                  (q + 1/2) 2^-23 >= cdf_i (k[n_int] = 2^23),
//                                  so the search compares integers exactly
//   off_dl    float dl[n_int]      (k[i] + 1/2) 2^-23 - cdf_i, in [0, 2^-23)
//   off_ri    float ri[n_int]      1 / (cdf_{i+1} - cdf_i)  (0 if empty)
//   off_omu   float omu[n_theta]   1 - cos(theta_i)
//   off_pth   float pth[n_int]     (cdf_{i+1} - cdf_i) / dtheta, per radian
//   off_gq    uint16 gq[G + 1]     gq[b] = largest i < n_int with k[i] <= b 2^23 / G:
//                                  a sample's interval for an index q lies in
//                                  [gq[q / (2^23 / G)], gq[q / (2^23 / G) + 1]]
//   off_go    uint16 go[G + 1]     go[c] = largest i < n_int with omu[i] <= c 2 / G
//                                  (as floats): the interval of 1 - cos(theta) = om
//                                  lies in [go[c], go[c + 1]], c = floor(om G / 2)
// G = MC_PAPER_GUIDE; the guides only narrow the bisection, whose answer is
// the same as over the whole table.
#define MC_PAPER_MAGIC 0x504D434Du  // "MCMP"
#define MC_PAPER_VERSION 2u
#define MC_PAPER_GUIDE 4096

struct mc_paper_header {
    uint32_t magic;
    uint32_t version;
    int32_t n_theta;
    int32_t n_int;
    uint32_t off_k, off_dl, off_ri, off_omu, off_pth;
    uint32_t total_bytes;
    float dtheta;
    int32_t top;            // largest power of two <= n_int - 1
    float g_table;          // mean cosine of the sampled distribution
    uint32_t off_gq, off_go;
    float pad;
};
static_assert(sizeof(mc_paper_header) == 64, "header must be 64 bytes");

static inline size_t mc_paper_layout(int n_theta, mc_paper_header *h)
{
    if (n_theta < 16 || n_theta > 16384) return 0;
    const int n = n_theta - 1;
    size_t off = sizeof(mc_paper_header);
    const size_t k = off;
    off += mc_pad16(sizeof(uint32_t) * (size_t)(n + 1));
    const size_t dl = off;
    off += mc_pad16(sizeof(float) * (size_t)n);
    const size_t ri = off;
    off += mc_pad16(sizeof(float) * (size_t)n);
    const size_t om = off;
    off += mc_pad16(sizeof(float) * (size_t)n_theta);
    const size_t pth = off;
    off += mc_pad16(sizeof(float) * (size_t)n);
    const size_t gq = off;
    off += mc_pad16(sizeof(uint16_t) * (size_t)(MC_PAPER_GUIDE + 1));
    const size_t go = off;
    off += mc_pad16(sizeof(uint16_t) * (size_t)(MC_PAPER_GUIDE + 1));
    if (h) {
        int top = 1;
        while (2 * top <= n - 1) top *= 2;
        h->magic = MC_PAPER_MAGIC;
        h->version = MC_PAPER_VERSION;
        h->n_theta = n_theta;
        h->n_int = n;
        h->off_k = (uint32_t)k;
        h->off_dl = (uint32_t)dl;
        h->off_ri = (uint32_t)ri;
        h->off_omu = (uint32_t)om;
        h->off_pth = (uint32_t)pth;
        h->total_bytes = (uint32_t)off;
        h->dtheta = 0.0f;
        h->top = top;
        h->g_table = 0.0f;
        h->off_gq = (uint32_t)gq;
        h->off_go = (uint32_t)go;
        h->pad = 0.0f;
    }
    return off;
}
