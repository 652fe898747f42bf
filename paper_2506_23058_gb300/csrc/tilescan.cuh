// tilescan.cuh - exclusive scan of per-tile packed counts, in place, in two
// launches: each block of TS_G threads scans its group of TS_G tiles and writes
// the group total; then each block adds the sum of the totals of the groups
// before it, and the last block writes the grand total to the header. Shared by
// the partition / FiltPart passes and the filter of get_smallest_pairs.
#pragma once

#include "common.cuh"

namespace ixp {

constexpr int TS_G = 1024;

__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long x, unsigned long long *s_w,
                                                                  unsigned long long *total) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    unsigned long long y = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long o = __shfl_up_sync(FULL, y, d);
        if (l >= d) y += o;
    }
    if (l == 31) s_w[w] = y;
    __syncthreads();
    if (w == 0) {
        const unsigned long long v = l < nw ? s_w[l] : 0ull;
        unsigned long long z = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            unsigned long long o = __shfl_up_sync(FULL, z, d);
            if (l >= d) z += o;
        }
        if (l < nw) s_w[l] = z - v;
        if (l == 31) s_w[32] = z;
    }
    __syncthreads();
    const unsigned long long r = s_w[w] + y - x;
    *total = s_w[32];
    __syncthreads();
    return r;
}

static __global__ void __launch_bounds__(TS_G) group_scan_kernel(unsigned long long *tp, int64_t nt,
                                                          unsigned long long *gtot) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long s_w[33];
    const int64_t t = blockIdx.x * (int64_t)TS_G + threadIdx.x;
    const unsigned long long x = t < nt ? tp[t] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan_u64(x, s_w, &tot);
    if (t < nt) tp[t] = ex;
    if (threadIdx.x == 0) gtot[blockIdx.x] = tot;
}

static __global__ void __launch_bounds__(TS_G) group_add_kernel(unsigned long long *tp, int64_t nt,
                                                         const unsigned long long *__restrict__ gtot, Hdr *h) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long s_w[TS_G / 32];
    __shared__ unsigned long long s_pre;
    unsigned long long v = 0;
    for (int64_t g = threadIdx.x; g < (int64_t)blockIdx.x; g += TS_G) v += gtot[g];
    v = block_sum_u64(v, s_w);
    if (threadIdx.x == 0) s_pre = v;
    __syncthreads();
    const unsigned long long pre = s_pre;
    const int64_t t = blockIdx.x * (int64_t)TS_G + threadIdx.x;
    if (t < nt) tp[t] += pre;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) h->total = pre + gtot[blockIdx.x];
}

// Runs both launches over tp[0 .. nt); gtot has room for one total per group.
static inline void scan_tile_counts(unsigned long long *tp, int64_t nt, unsigned long long *gtot, Hdr *h,
                                    cudaStream_t st) {
    if (nt <= 0) return;
    const unsigned ng = (unsigned)((nt + TS_G - 1) / TS_G);
    group_scan_kernel<<<ng, TS_G, 0, st>>>(tp, nt, gtot);
    group_add_kernel<<<ng, TS_G, 0, st>>>(tp, nt, gtot, h);
}

}  // namespace ixp
