// ceilings.cu - microbenchmarks of the hardware rates that bound the library's
// kernels, so that each kernel's time can be read against the rate it actually
// needs (not only against the HBM copy peak):
//   * L2 atomic OR on a bitmap, with the old value returned (what a plain bitmap
//     Inj / Bij test needs) and fire-and-forget (a reduction);
//   * random 32-byte row reads (the rate that bounds a gather or scatter of
//     32-byte rows by a permutation);
//   * a streaming read (the HBM read rate).
// Each kernel does the minimum work per item and folds what it read into one
// word per block, which it writes, so that nothing is optimised away.
#include <algorithm>

#include "common.cuh"

namespace ixp {


// One bit per item: bit = pos[i] & (bits - 1) (bits a power of two), set with
// atomicOr; with RET the old word is folded into the block's checksum.
template <bool RET>
__global__ void __launch_bounds__(STREAM_THREADS) ceil_atomic_or_kernel(unsigned *__restrict__ bm,
                                                                        unsigned long long bits,
                                                                        const unsigned *__restrict__ pos, int64_t n,
                                                                        unsigned *__restrict__ sink) {
    IXP_KERNEL_ENTRY();
    unsigned acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n / 4;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += stride) {
        const uint4 p = __ldcs(reinterpret_cast<const uint4 *>(pos) + q);
        const unsigned v[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const unsigned long long b = (unsigned long long)v[c] & (bits - 1);
            const unsigned mask = 1u << (b & 31);
            if (RET) acc ^= atomicOr(bm + (b >> 5), mask) & mask;
            else atomicOr(bm + (b >> 5), mask);
        }
    }
    acc = __reduce_xor_sync(FULL, acc);
    if ((threadIdx.x & 31) == 0 && acc == 0xdeadbeefu) sink[blockIdx.x] = acc;  // keeps the returns live
}

// Random 32-byte rows: item i reads row idx[i] & (nrows - 1) (nrows a power of
// two; two 16-byte loads) and folds it.
__global__ void __launch_bounds__(STREAM_THREADS) ceil_random_rows_kernel(const uint4 *__restrict__ rows,
                                                                          unsigned row_mask,
                                                                          const unsigned *__restrict__ idx, int64_t n,
                                                                          unsigned *__restrict__ sink) {
    IXP_KERNEL_ENTRY();
    unsigned acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n / 4;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += stride) {
        const uint4 p = __ldcs(reinterpret_cast<const uint4 *>(idx) + q);
        const unsigned r[4] = {p.x & row_mask, p.y & row_mask, p.z & row_mask, p.w & row_mask};
        uint4 a[4], b[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            a[c] = __ldcs(rows + 2 * (uint64_t)r[c]);
            b[c] = __ldcs(rows + 2 * (uint64_t)r[c] + 1);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) acc ^= a[c].x ^ a[c].y ^ a[c].z ^ a[c].w ^ b[c].x ^ b[c].y ^ b[c].z ^ b[c].w;
    }
    acc = __reduce_xor_sync(FULL, acc);
    if ((threadIdx.x & 31) == 0) sink[blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)] = acc;
}

// Streaming read of `words16` 16-byte words, four in flight per thread.
__global__ void __launch_bounds__(STREAM_THREADS) ceil_stream_read_kernel(const uint4 *__restrict__ src,
                                                                          int64_t words16,
                                                                          unsigned *__restrict__ sink) {
    IXP_KERNEL_ENTRY();
    unsigned acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; q + 3 * stride < words16; q += 4 * stride) {
        uint4 a[4];
#pragma unroll
        for (int u = 0; u < 4; u++) a[u] = __ldcs(src + q + u * stride);
#pragma unroll
        for (int u = 0; u < 4; u++) acc ^= a[u].x ^ a[u].y ^ a[u].z ^ a[u].w;
    }
    for (; q < words16; q += stride) {
        const uint4 a = __ldcs(src + q);
        acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
    acc = __reduce_xor_sync(FULL, acc);
    if ((threadIdx.x & 31) == 0) sink[blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)] = acc;
}

}  // namespace ixp

using namespace ixp;

extern "C" unsigned long long ixp_tu_kernels_ceilings(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}


extern "C" int ixp_sink_words(void) { return num_sms() * 8 * (STREAM_THREADS / 32); }

extern "C" int ixp_ceiling_atomic_or(unsigned *bitmap, int64_t bits, const unsigned *pos, int64_t n, int with_return,
                                     unsigned *d_sink, ixp_stream stream) {
    if (bits <= 0 || (bits & (bits - 1)) || n < 0 || n % 4 || !bitmap || !d_sink ||
        (n > 0 && (!pos || !aligned16(pos))))
        return IXP_E_INVAL;
    if (n == 0) return IXP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int g = num_sms() * 8;
    if (with_return)
        ceil_atomic_or_kernel<true><<<g, STREAM_THREADS, 0, st>>>(bitmap, (unsigned long long)bits, pos, n, d_sink);
    else
        ceil_atomic_or_kernel<false><<<g, STREAM_THREADS, 0, st>>>(bitmap, (unsigned long long)bits, pos, n, d_sink);
    return launch_status();
}

extern "C" int ixp_ceiling_random_rows(const void *rows, int64_t nrows, const unsigned *idx, int64_t n,
                                       unsigned *d_sink, ixp_stream stream) {
    if (nrows <= 0 || (nrows & (nrows - 1)) || nrows > (1ll << 32) || n < 0 || n % 4 || !rows || !aligned16(rows) ||
        !d_sink || (n > 0 && (!idx || !aligned16(idx))))
        return IXP_E_INVAL;
    if (n == 0) return IXP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    ceil_random_rows_kernel<<<num_sms() * 8, STREAM_THREADS, 0, st>>>(reinterpret_cast<const uint4 *>(rows),
                                                                       (unsigned)(nrows - 1), idx, n, d_sink);
    return launch_status();
}

extern "C" int ixp_ceiling_stream_read(const void *src, int64_t bytes, unsigned *d_sink, ixp_stream stream) {
    if (bytes < 0 || bytes % 16 || !d_sink || (bytes > 0 && (!src || !aligned16(src)))) return IXP_E_INVAL;
    if (bytes == 0) return IXP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    ceil_stream_read_kernel<<<num_sms() * 8, STREAM_THREADS, 0, st>>>(reinterpret_cast<const uint4 *>(src),
                                                                       bytes / 16, d_sink);
    return launch_status();
}
