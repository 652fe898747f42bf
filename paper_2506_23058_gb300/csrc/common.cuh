// common.cuh - device helpers shared by the library's kernels (not by the oracle).
//
// Layout rules used throughout:
//  * Streaming kernels read 16-byte vectors (int4 / longlong2) in a grid-stride loop
//    unrolled four deep, so each SM keeps ~128 KB of loads in flight; the elements
//    before the first 16-byte boundary and after the last whole vector are handled
//    one by one.
//  * Reductions go warp shuffle -> shared memory -> one global atomic per block.
//  * Every call zeroes a 256-byte header at the start of its workspace. All header
//    slots start at 0 and are only raised with unsigned 64-bit atomicMax, so minima,
//    maxima and "first index" slots are stored under order-preserving encodings:
//        first index i : ~i          (0 = none; decodes to -1)
//        minimum  x    : ~(x ^ SIGN) (0 decodes to INT64_MAX)
//        maximum  x    :  x ^ SIGN   (0 decodes to INT64_MIN)
//  * Every spin-wait is bounded; giving up sets the header's status to
//    IXP_E_TIMEOUT and the kernel carries on without the missing value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ixp.h"

namespace ixp {

constexpr uint64_t SIGN = 0x8000000000000000ull;
constexpr unsigned FULL = 0xffffffffu;

__host__ __device__ inline uint64_t enc_first(int64_t i) { return ~(uint64_t)i; }
__host__ __device__ inline int64_t dec_first(uint64_t k) { return (int64_t)~k; }
__host__ __device__ inline uint64_t enc_min(int64_t x) { return ~((uint64_t)x ^ SIGN); }
__host__ __device__ inline int64_t dec_min(uint64_t k) { return (int64_t)(~k ^ SIGN); }
__host__ __device__ inline uint64_t enc_max(int64_t x) { return (uint64_t)x ^ SIGN; }
__host__ __device__ inline int64_t dec_max(uint64_t k) { return (int64_t)(k ^ SIGN); }

// Workspace header (256 bytes, zeroed by the host at the start of every call).
struct Hdr {
    unsigned long long k_min;     // enc_min of the minimum
    unsigned long long k_max;     // enc_max of the maximum
    unsigned long long k_first;   // enc_first of the first violating index
    unsigned long long k_first2;  // enc_first of a second candidate (Bij: duplicate)
    unsigned long long k_aux;     // enc_first of a partner / missing value offset
    unsigned long long cnt0;      // counters
    unsigned long long cnt1;
    unsigned long long base;      // bitmap base value (as uint64)
    unsigned long long span;      // bitmap span in bits
    unsigned int tile_ctr;        // dynamic tile ticket
    unsigned int flag;            // "a duplicate was seen"
    int status;                   // IXP_OK or a device-side error
    int pad0;
    unsigned long long total;     // scan / partition total
    unsigned long long spare[20];
};
static_assert(sizeof(Hdr) == 256, "header must be 256 bytes");

constexpr size_t HDR_BYTES = 256;

// ------------------------------------------------------------------ loads

template <typename T> struct Vec;
template <> struct Vec<int32_t> { using type = int4; static constexpr int N = 4; };
template <> struct Vec<int64_t> { using type = longlong2; static constexpr int N = 2; };

__device__ __forceinline__ int4 ldv(const int4 *p) { return __ldcs(p); }
__device__ __forceinline__ longlong2 ldv(const longlong2 *p) { return __ldcs(p); }

__device__ __forceinline__ void unpack(const int4 &v, int64_t (&e)[4]) { e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w; }
__device__ __forceinline__ void unpack(const longlong2 &v, int64_t (&e)[2]) { e[0] = v.x; e[1] = v.y; }

// Split [0, n) of an array at p into a scalar head (up to the first 16-byte
// boundary), a run of whole 16-byte vectors, and a scalar tail.
template <typename T> struct Split {
    int64_t head;   // number of leading scalar elements
    int64_t nvec;   // number of vectors after the head
    int64_t tail0;  // first tail element
    __device__ __forceinline__ Split(const T *p, int64_t n) {
        constexpr int V = Vec<T>::N;
        uintptr_t a = reinterpret_cast<uintptr_t>(p);
        head = (int64_t)(((16 - (a & 15)) & 15) / sizeof(T));
        if (head > n) head = n;
        nvec = (n - head) / V;
        tail0 = head + nvec * V;
    }
};

// ------------------------------------------------------------ reductions

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Block-wide max of `v` (all threads call); result valid in thread 0.
// `sm` must hold blockDim.x / 32 entries.
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long *sm) {
    v = warp_max_u64(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sm[l] : 0ull;
        r = warp_max_u64(r);
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *sm) {
    v = warp_sum_u64(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sm[l] : 0ull;
        r = warp_sum_u64(r);
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ void atomic_max_u64(unsigned long long *p, unsigned long long v) {
    if (v) atomicMax(p, v);
}

// ------------------------------------------------------- memory ordering

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void set_status(Hdr *h, int code) { atomicCAS(&h->status, 0, code); }
// ----------------------------------------------- TMA bulk copies + mbarrier
// One-dimensional bulk copies global -> shared (cp.async.bulk) complete on an
// mbarrier with a transaction-byte count. Sources and sizes must be 16-byte
// multiples / aligned.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    unsigned long long state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("" ::"l"(state));
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `phase` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned phase, long long limit) {
    for (long long i = 0; i < limit; i++)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}


// ------------------------------------------------------------ element load

template <typename T> __device__ __forceinline__ int64_t ld1(const T *p, int64_t i) { return (int64_t)__ldg(p + i); }

__device__ __forceinline__ int64_t load_index(const void *p, int t, int64_t i) {
    return t == IXP_I32 ? (int64_t)__ldg((const int32_t *)p + i) : (int64_t)__ldg((const int64_t *)p + i);
}

// Kernel-execution counter: every kernel's first block bumps its translation
// unit's counter once, so the host can read how many kernels actually ran.
static __device__ unsigned long long tu_kernel_count;
#define IXP_KERNEL_ENTRY()                                                  \
    do {                                                                    \
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&tu_kernel_count, 1ull); \
    } while (0)

// ------------------------------------------------------------ segment offsets

// First k in [0, nseg] with off[k] >= key (nseg + 1 if none).
__device__ __forceinline__ int64_t off_lower_bound(const int64_t *off, int64_t nseg, int64_t key) {
    int64_t lo = 0, hi = nseg + 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Last k in [0, nseg) with off[k] <= i: the segment holding element i.
__device__ __forceinline__ int64_t off_segment_of(const int64_t *off, int64_t nseg, int64_t i) {
    int64_t lo = 0, hi = nseg;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Adjacent pairs inside segments, one chunk of SP_CHUNK elements per call (all
// threads of the block call it). The chunk x[j0 .. j0 + cnt) is staged in shared
// memory with 16-byte loads when aligned; every segment start off[k] inside the
// chunk is marked in a bitmap, and f(j, x[j-1], x[j]) runs for every j > 0 of the
// chunk that is not a segment start, so pairs never cross a segment boundary.
constexpr int SP_CHUNK = 4096;

template <typename T>
struct SegPairsSmem {
    T x[SP_CHUNK];
    unsigned head[SP_CHUNK / 32];
    T prev;
    int64_t k;
};

// lb[c] = first k in [0, nseg] with off[k] >= c * SP_CHUNK, for every chunk c, from
// one pass over the offsets (chunks are filled by the segment whose start first
// reaches them; a chunk nothing reaches keeps the caller's fill).
static inline size_t chunk_lb_bytes(int64_t n) {
    return (size_t)(((n > 0 ? n : 0) + SP_CHUNK - 1) / SP_CHUNK * 8 + 8 + 255) / 256 * 256;
}

template <int CH>
__global__ void chunk_lb_kernel(const int64_t *__restrict__ off, int64_t nseg, int64_t n, int64_t *__restrict__ lb) {
    IXP_KERNEL_ENTRY();
    const int64_t nch = (n + CH - 1) / CH;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= nseg; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = k == 0 ? -1 : __ldg(off + k - 1), hi = __ldg(off + k);
        // chunks c with lo < c * CH <= hi
        int64_t c = lo < 0 ? 0 : lo / CH + 1;
        for (; c < nch && c * CH <= hi; c++) lb[c] = k;
    }
}

template <typename T, typename F>
__device__ __forceinline__ void seg_pairs_chunk(const T *__restrict__ x, int64_t n, const int64_t *__restrict__ off,
                                                int64_t nseg, int64_t j0, SegPairsSmem<T> &S,
                                                const int64_t *__restrict__ lbtab, F &&f) {
    const int cnt = (int)min((int64_t)SP_CHUNK, n - j0);
    for (int w = threadIdx.x; w < SP_CHUNK / 32; w += blockDim.x) S.head[w] = 0u;
    if (threadIdx.x == 0) {
        S.prev = j0 > 0 ? x[j0 - 1] : (T)0;
        int64_t k = lbtab ? __ldg(lbtab + j0 / SP_CHUNK) : off_lower_bound(off, nseg, j0);
        S.k = k < 0 ? 0 : (k > nseg ? nseg : k);
    }
    constexpr int V = 16 / (int)sizeof(T);
    if (cnt == SP_CHUNK && (reinterpret_cast<uintptr_t>(x + j0) & 15u) == 0) {
        for (int v = threadIdx.x; v < SP_CHUNK / V; v += blockDim.x)
            reinterpret_cast<int4 *>(S.x)[v] = __ldcs(reinterpret_cast<const int4 *>(x + j0) + v);
    } else {
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) S.x[e] = x[j0 + e];
    }
    __syncthreads();
    for (int64_t k = S.k + threadIdx.x; k <= nseg; k += blockDim.x) {
        const int64_t o = __ldg(off + k);
        if (o >= j0 + cnt) break;
        if (o >= j0) atomicOr(&S.head[(o - j0) >> 5], 1u << ((o - j0) & 31));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int64_t j = j0 + e;
        if (j == 0 || (S.head[e >> 5] >> (e & 31)) & 1u) continue;
        f(j, e ? S.x[e - 1] : S.prev, S.x[e]);
    }
    __syncthreads();
}


// ------------------------------------------------------------ host helpers

static inline int launch_status() { return cudaGetLastError() == cudaSuccess ? IXP_OK : IXP_E_CUDA; }
static inline bool aligned_to(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
static inline bool aligned16(const void *p) { return aligned_to(p, 16); }
static inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
// A caller workspace: present, 256-byte aligned and at least `need` bytes.
static inline int check_ws(void *ws, size_t have, size_t need) {
    return (!ws || !aligned_to(ws, 256) || have < need) ? IXP_E_WORKSPACE : IXP_OK;
}

// Launch shape for grid-stride streaming kernels: 8 blocks of 256 threads per SM.
constexpr int STREAM_THREADS = 256;
int stream_grid(int64_t work_items, int per_thread = 4);
int num_sms();

}  // namespace ixp
