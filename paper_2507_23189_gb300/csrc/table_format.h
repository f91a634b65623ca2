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
