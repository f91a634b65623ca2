// Issue-rate microbenchmarks (declared in include/mcpeaks.h). Each kernel runs
// independent dependency chains so that throughput, not latency, limits it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mcpeaks.h"

namespace {

__global__ void k_ffma(float *sink, int iters)
{
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1e-3f * (threadIdx.x + j);
    const float b = 0.9999f, c = 1e-6f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_imad(float *sink, int iters)
{
    uint32_t a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 7u + j;
    const uint32_t c = 0x9E3779B9u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = a[j] * a[(j + 1) & 7] + c;  // non-linear: no folding
    }
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s ^= a[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void k_imulwide(float *sink, int iters)
{
    uint32_t a[8], h = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 7u + j + 1;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint64_t p = (uint64_t)0xCD9E8D57u * a[j];
                a[j] = (uint32_t)p ^ (uint32_t)(p >> 32);
            }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) h ^= a[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)h;
}

__global__ void k_mufu(float *sink, int iters)
{
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.0f + 1e-3f * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 8; ++j) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[j]));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_smem(float *sink, int iters)
{
    __shared__ float4 buf[2048];  // 32 KB
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        buf[i] = make_float4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    float4 acc = make_float4(0, 0, 0, 0);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float4 v = buf[(idx + r * 256) & 2047];
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        idx = (idx + 32) & 2047;
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

}  // namespace

extern "C" int mc_peak_run(int kind, int blocks, int threads, int iters, float *d_sink, double *ops,
                           void *stream)
{
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads % 32) || iters < 1 || !d_sink || !ops)
        return -1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double nthr = (double)blocks * threads;
    switch (kind) {
    case MC_PEAK_FFMA: k_ffma<<<blocks, threads, 0, st>>>(d_sink, iters); *ops = nthr * iters * 32; break;
    case MC_PEAK_IMAD: k_imad<<<blocks, threads, 0, st>>>(d_sink, iters); *ops = nthr * iters * 32; break;
    case MC_PEAK_MUFU: k_mufu<<<blocks, threads, 0, st>>>(d_sink, iters); *ops = nthr * iters * 32; break;
    case MC_PEAK_SMEM: k_smem<<<blocks, threads, 0, st>>>(d_sink, iters); *ops = nthr * iters * 8 * 16; break;
    case MC_PEAK_IMULWIDE:
        k_imulwide<<<blocks, threads, 0, st>>>(d_sink, iters); *ops = nthr * iters * 32; break;
    default: return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
