// checks.cu - runtime checks of the paper's index-array properties (Sec. 2.3,
// Fig. 5): Range, Monotonic, Inj and Bij on int32/int64 arrays.
//
// Range and flat Mono are single streaming passes (4 or 8 bytes per element, HBM
// bound). Inj and Bij set one bit per in-codomain element in a bitmap over the value
// span; a bit found already set is a repeat (rule BijF1 of Sec. 3.2 counts the same
// way: Inj plus |Img| in-image elements). Small inputs set the bits with L2
// atomicOr on one global bitmap. Large inputs (n >= 2^18, span >= 2^21) first sort
// each tile's values by bucket (a range of 2^lw values) into per-bucket pools, then
// give every bucket one block with its part of the bitmap in shared memory, where
// the atomicOr's return value flags the repeat. When a repeat was seen, two more
// passes recover the exact witness (smallest repeated index and its partner),
// reading X in index order only up to about the witness; they exit at once
// otherwise.
#include <algorithm>

#include "common.cuh"
#include <type_traits>

namespace ixp {

// ============================================================== Range
// Bounds are clamped to the element type on the host (lo_t, hi_t), so the loop
// compares in the native width; per 16-byte vector only the vector's min and max
// are tested, and the first bad index is located only inside a failing vector.
template <typename T> struct Lim;
template <> struct Lim<int32_t> { static constexpr int32_t lo = INT32_MIN, hi = INT32_MAX; };
template <> struct Lim<int64_t> { static constexpr int64_t lo = INT64_MIN, hi = INT64_MAX; };

template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS, 4) range_kernel(const T *__restrict__ x, int64_t n, T lo, T hi,
                                                               Hdr *h) {
    IXP_KERNEL_ENTRY();
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::N;
    Split<T> s(x, n);
    T mn = Lim<T>::hi, mx = Lim<T>::lo;
    int64_t bad = INT64_MAX;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto one = [&](int64_t i, T xi) {
        mn = xi < mn ? xi : mn;
        mx = xi > mx ? xi : mx;
        if ((xi < lo) | (xi > hi)) bad = i < bad ? i : bad;
    };
    auto vec = [&](int64_t i0, const VT &a) {
        T e[V];
        if (V == 4) {
            const int4 &q = reinterpret_cast<const int4 &>(a);
            e[0] = (T)q.x;
            e[1 % V] = (T)q.y;
            e[2 % V] = (T)q.z;
            e[3 % V] = (T)q.w;
        } else {
            const longlong2 &q = reinterpret_cast<const longlong2 &>(a);
            e[0] = (T)q.x;
            e[1 % V] = (T)q.y;
        }
        T vmin = e[0], vmax = e[0];
#pragma unroll
        for (int k = 1; k < V; k++) {
            vmin = e[k] < vmin ? e[k] : vmin;
            vmax = e[k] > vmax ? e[k] : vmax;
        }
        mn = vmin < mn ? vmin : mn;
        mx = vmax > mx ? vmax : mx;
        if ((vmin < lo) | (vmax > hi)) {
#pragma unroll
            for (int k = V - 1; k >= 0; k--)
                if ((e[k] < lo) | (e[k] > hi)) bad = (i0 + k) < bad ? (i0 + k) : bad;
        }
    };
    for (int64_t i = tid; i < s.head; i += stride) one(i, x[i]);
    for (int64_t i = s.tail0 + tid; i < n; i += stride) one(i, x[i]);
    const VT *xv = reinterpret_cast<const VT *>(x + s.head);
    int64_t v = tid;
    for (; v + 3 * stride < s.nvec; v += 4 * stride) {
        VT a[4];
#pragma unroll
        for (int u = 0; u < 4; u++) a[u] = ldv(xv + v + u * stride);
#pragma unroll
        for (int u = 0; u < 4; u++) vec(s.head + (v + u * stride) * V, a[u]);
    }
    for (; v < s.nvec; v += stride) vec(s.head + v * V, ldv(xv + v));
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    unsigned long long r;
    r = block_max_u64(enc_min((int64_t)mn), sm);
    if (threadIdx.x == 0 && mn <= mx) atomic_max_u64(&h->k_min, r);
    r = block_max_u64(enc_max((int64_t)mx), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_max, r);
    r = block_max_u64(bad == INT64_MAX ? 0ull : enc_first(bad), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

template <typename T>
__global__ void range_finalize(const T *x, int64_t n, const Hdr *h, ixp_verdict *out, int all_bad) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    int64_t bad = h->k_first ? dec_first(h->k_first) : -1;
    if (all_bad && n > 0) bad = 0;
    v.status = h->status;
    v.ok = v.status ? -1 : (bad < 0 ? 1 : 0);
    v.kind = bad < 0 ? IXP_V_NONE : IXP_V_OUT_OF_RANGE;
    v.index = bad;
    v.value = bad < 0 ? 0 : (int64_t)x[bad];
    v.aux0 = dec_min(h->k_min);
    v.aux1 = dec_max(h->k_max);
    v.reserved = 0;
    *out = v;
}

// ======================================================= Monotonic (flat)
__device__ __forceinline__ bool cmp_ok(int c, int64_t a, int64_t b) {
    switch (c) {
        case IXP_LE: return a <= b;
        case IXP_LT: return a < b;
        case IXP_GE: return a >= b;
        default: return a > b;
    }
}

// Grid-stride over 16-byte vectors with a warp-uniform loop: lane l holds vector
// wbase + l, so the element before its vector is lane l-1's last element (one
// shuffle); lane 0 reads it from memory.
template <typename T, int C>
__device__ __forceinline__ bool cmp_t(T a, T b) {
    if (C == IXP_LE) return a <= b;
    if (C == IXP_LT) return a < b;
    if (C == IXP_GE) return a >= b;
    return a > b;
}

template <typename T, int C>
__global__ void __launch_bounds__(STREAM_THREADS, 4) mono_kernel(const T *__restrict__ x, int64_t n, Hdr *h) {
    IXP_KERNEL_ENTRY();
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::N;
    Split<T> s(x, n);
    int64_t bad = INT64_MAX;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    // scalar head and tail pairs (j >= 1)
    for (int64_t j = tid; j < s.head; j += stride)
        if (j >= 1 && !cmp_t<T, C>(x[j - 1], x[j])) bad = j < bad ? j : bad;
    for (int64_t j = s.tail0 + tid; j < n; j += stride)
        if (j >= 1 && !cmp_t<T, C>(x[j - 1], x[j])) bad = j < bad ? j : bad;
    const VT *xv = reinterpret_cast<const VT *>(x + s.head);
    const int64_t wtid = tid - lane;  // warp's first thread
    for (int64_t wb = wtid; wb < s.nvec; wb += 4 * stride) {
        VT a[4];
        T prevm[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t vv = wb + u * stride + lane;
            if (vv < s.nvec) a[u] = ldv(xv + vv);
            const int64_t p = s.head + (wb + u * stride) * V;  // first element of lane 0's vector
            prevm[u] = (lane == 0 && p >= 1 && wb + u * stride < s.nvec) ? x[p - 1] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t vv = wb + u * stride + lane;
            const bool live = vv < s.nvec;
            T e[V];
            if (V == 4) {
                const int4 &q = reinterpret_cast<const int4 &>(a[u]);
                e[0] = (T)q.x;
                e[1 % V] = (T)q.y;
                e[2 % V] = (T)q.z;
                e[3 % V] = (T)q.w;
            } else {
                const longlong2 &q = reinterpret_cast<const longlong2 &>(a[u]);
                e[0] = (T)q.x;
                e[1 % V] = (T)q.y;
            }
            T prev = __shfl_up_sync(FULL, e[V - 1], 1);
            if (lane == 0) prev = prevm[u];
            if (live) {
                const int64_t j0 = s.head + vv * V;
                bool fail = j0 >= 1 && !cmp_t<T, C>(prev, e[0]);
#pragma unroll
                for (int k = 1; k < V; k++) fail |= !cmp_t<T, C>(e[k - 1], e[k]);
                if (fail) {
                    if (j0 >= 1 && !cmp_t<T, C>(prev, e[0])) bad = j0 < bad ? j0 : bad;
#pragma unroll
                    for (int k = 1; k < V; k++)
                        if (!cmp_t<T, C>(e[k - 1], e[k])) bad = (j0 + k) < bad ? (j0 + k) : bad;
                }
            }
        }
    }
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    unsigned long long r = block_max_u64(bad == INT64_MAX ? 0ull : enc_first(bad), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

// =================================================== Monotonic (segmented)
// One SP_CHUNK-element chunk per block iteration, staged in shared memory; segment
// heads inside the chunk are marked in a bitmap and the pair (j-1, j) is tested
// only when j is not a head.
template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS) mono_seg_kernel(const T *__restrict__ x, int64_t n, int c,
                                                                  const int64_t *__restrict__ off, int64_t nseg,
                                                                  const int64_t *__restrict__ lb, uint8_t *seg_ok,
                                                                  Hdr *h) {
    IXP_KERNEL_ENTRY();
    __shared__ SegPairsSmem<T> S;
    int64_t bad = INT64_MAX;
    const int64_t nchunks = (n + SP_CHUNK - 1) / SP_CHUNK;
    for (int64_t t = blockIdx.x; t < nchunks; t += gridDim.x) {
        seg_pairs_chunk<T>(x, n, off, nseg, t * SP_CHUNK, S, lb, [&](int64_t j, T a, T b) {
            if (!cmp_ok(c, (int64_t)a, (int64_t)b)) {
                bad = j < bad ? j : bad;
                if (seg_ok) seg_ok[off_segment_of(off, nseg, j)] = 0;
            }
        });
    }
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    unsigned long long r = block_max_u64(bad == INT64_MAX ? 0ull : enc_first(bad), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

template <typename T>
__global__ void mono_finalize(const T *x, const Hdr *h, ixp_verdict *out) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    int64_t j = h->k_first ? dec_first(h->k_first) : -1;
    v.status = h->status;
    v.ok = v.status ? -1 : (j < 0 ? 1 : 0);
    v.kind = j < 0 ? IXP_V_NONE : IXP_V_ORDER;
    v.index = j;
    v.value = j < 0 ? 0 : (int64_t)x[j];
    v.aux0 = j < 1 ? 0 : (int64_t)x[j - 1];
    v.aux1 = 0;
    v.reserved = 0;
    *out = v;
}

// ================================================================ Inj / Bij
constexpr int BK_TILE = 8192;
constexpr unsigned BK_MAX = 4096;
// Header slots of the bucketed path: bucket count, pool entries per bucket, log2 of
// the bucket width, and the launch shape the setup kernel chose for the span it
// found (both shapes run the same two passes).
constexpr int BK_NB = 0, BK_CAP = 1, BK_LW = 2, BK_MODE = 3;
constexpr unsigned long long BK_STAGED = 1, BK_WIDE = 2, BK_HASH = 3;
// header slots of the hash-set path: the pair of the value -1, the smallest pair
constexpr int HS_NEG1 = 4, HS_PAIR = 5;
// header slots of the partitioned hash-set path: why it gave up (the single-table
// path then decides), repeated values listed, elements whose hash is all ones
constexpr int HP_FLAGS = 6, HP_NDUP = 7, HP_TOPH = 8;
constexpr unsigned long long HP_F_POOL = 1, HP_F_DUPS = 2;

// Min/max of the in-codomain values (needed when Rcd is unbounded). The bounds
// come clamped to T, so every compare is in T; a vector that lies wholly inside
// [lo, hi] (the common case) folds its own min/max in one step. A thread that saw
// nothing ends with mn > mx and contributes the empty encodings.
template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS, 4) minmax_in_kernel(const T *__restrict__ x, int64_t n, T lo, T hi,
                                                                   Hdr *h) {
    IXP_KERNEL_ENTRY();
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::N;
    Split<T> s(x, n);
    T mn = Lim<T>::hi, mx = Lim<T>::lo;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto one = [&](T xi) {
        if ((xi >= lo) & (xi <= hi)) {
            mn = xi < mn ? xi : mn;
            mx = xi > mx ? xi : mx;
        }
    };
    auto vec = [&](const VT &a) {
        T e[V];
        if (V == 4) {
            const int4 &q = reinterpret_cast<const int4 &>(a);
            e[0] = (T)q.x;
            e[1 % V] = (T)q.y;
            e[2 % V] = (T)q.z;
            e[3 % V] = (T)q.w;
        } else {
            const longlong2 &q = reinterpret_cast<const longlong2 &>(a);
            e[0] = (T)q.x;
            e[1 % V] = (T)q.y;
        }
        T vmin = e[0], vmax = e[0];
#pragma unroll
        for (int k = 1; k < V; k++) {
            vmin = e[k] < vmin ? e[k] : vmin;
            vmax = e[k] > vmax ? e[k] : vmax;
        }
        if ((vmin >= lo) & (vmax <= hi)) {
            mn = vmin < mn ? vmin : mn;
            mx = vmax > mx ? vmax : mx;
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) one(e[k]);
        }
    };
    for (int64_t i = tid; i < s.head; i += stride) one(x[i]);
    for (int64_t i = s.tail0 + tid; i < n; i += stride) one(x[i]);
    const VT *xv = reinterpret_cast<const VT *>(x + s.head);
    int64_t v = tid;
    for (; v + 3 * stride < s.nvec; v += 4 * stride) {
        VT a[4];
#pragma unroll
        for (int u = 0; u < 4; u++) a[u] = ldv(xv + v + u * stride);
#pragma unroll
        for (int u = 0; u < 4; u++) vec(a[u]);
    }
    for (; v < s.nvec; v += stride) vec(ldv(xv + v));
    const bool seen = mn <= mx;
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    unsigned long long r = block_max_u64(seen ? enc_min((int64_t)mn) : enc_min(INT64_MAX), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_min, r);
    r = block_max_u64(seen ? enc_max((int64_t)mx) : enc_max(INT64_MIN), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_max, r);
}

// Fix the bitmap's base and span, check it against the capacity, clear the words
// the call will use. Fixed range: base = lo, span = hi - lo + 1. Otherwise the
// range comes from minmax_in_kernel (span 0 when nothing is in range).
__global__ void bitmap_setup_kernel(Hdr *h, int fixed, int64_t lo, int64_t hi, unsigned long long cap_bits,
                                    unsigned *bm, unsigned *dup, int hash_ok) {
    IXP_KERNEL_ENTRY();
    unsigned long long base, span;
    bool empty = false;  // nothing in range
    if (fixed) {
        base = (unsigned long long)lo;
        span = (unsigned long long)hi - (unsigned long long)lo + 1ull;
    } else {
        int64_t mn = dec_min(h->k_min), mx = dec_max(h->k_max);
        empty = mn > mx;
        base = empty ? 0ull : (unsigned long long)mn;
        span = empty ? 0ull : (unsigned long long)mx - (unsigned long long)mn + 1ull;
    }
    // span == 0 after the +1 means the full 2^64 range
    const bool too_big = !empty && (span == 0 || span > cap_bits);
    if (too_big) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (hash_ok) h->spare[BK_MODE] = BK_HASH;  // decided by the hash-set pass instead
            else set_status(h, IXP_E_SPAN);
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h->base = base;
        h->span = span;
    }
    const unsigned long long words = (span + 31) / 32;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < words;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        bm[w] = 0u;
        dup[w] = 0u;
    }
}

// Mark pass. For each element with a value in [mlo, mhi] (Rcd for Inj, Img for
// Bij): atomicOr its bit; a bit already set means a repeat, which is recorded in
// the second bitmap. For Bij, values in Rcd but outside Img are out of image.
template <typename T, bool BIJ>
__global__ void __launch_bounds__(STREAM_THREADS, 4) mark_kernel(const T *__restrict__ x, int64_t n, int64_t rlo,
                                                              int64_t rhi, int64_t mlo, int64_t mhi, Hdr *h,
                                                              unsigned *__restrict__ bm, unsigned *__restrict__ dup) {
    IXP_KERNEL_ENTRY();
    if (h->status) return;
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::N;
    const unsigned long long base = h->base, span = h->span;
    Split<T> s(x, n);
    unsigned long long cnt = 0;
    unsigned anydup = 0;
    int64_t ooi = INT64_MAX;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto visit = [&](int64_t i, int64_t xi) {
        if (xi < rlo || xi > rhi) return;
        if (BIJ && (xi < mlo || xi > mhi)) {
            ooi = i < ooi ? i : ooi;
            return;
        }
        unsigned long long b = (unsigned long long)xi - base;
        if (b >= span) return;  // cannot happen for a consistent header; keeps writes in bounds
        unsigned bit = 1u << (b & 31);
        unsigned old = atomicOr(bm + (b >> 5), bit);
        if (old & bit) {
            atomicOr(dup + (b >> 5), bit);
            anydup = 1;
        }
        cnt++;
    };
    for (int64_t i = tid; i < s.head; i += stride) visit(i, ld1(x, i));
    for (int64_t i = s.tail0 + tid; i < n; i += stride) visit(i, ld1(x, i));
    const VT *xv = reinterpret_cast<const VT *>(x + s.head);
    int64_t v = tid;
    for (; v + 3 * stride < s.nvec; v += 4 * stride) {
        VT a[4];
#pragma unroll
        for (int u = 0; u < 4; u++) a[u] = ldv(xv + v + u * stride);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int64_t e[V];
            unpack(a[u], e);
#pragma unroll
            for (int k = 0; k < V; k++) visit(s.head + (v + u * stride) * V + k, e[k]);
        }
    }
    for (; v < s.nvec; v += stride) {
        int64_t e[V];
        unpack(ldv(xv + v), e);
#pragma unroll
        for (int k = 0; k < V; k++) visit(s.head + v * V + k, e[k]);
    }
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    unsigned long long r = block_sum_u64(cnt, sm);
    if (threadIdx.x == 0 && r) atomicAdd(&h->cnt0, r);
    if (__syncthreads_or(anydup) && threadIdx.x == 0) atomicOr(&h->flag, 1u);
    if (BIJ) {
        r = block_max_u64(ooi == INT64_MAX ? 0ull : enc_first(ooi), sm);
        if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
    }
}

// Witness passes (run only when a repeat was seen). Both walk X in tiles of
// WT_VECS 16-byte vectors per block iteration, each block taking tiles in
// increasing order (grid stride), and stop at the first tile that starts past the
// best position found so far by any block: a skipped tile holds only larger
// positions, so the result is exact, and on a violating input the passes read X
// only up to about the witness instead of to the end.
constexpr int WT_PER = 4;                          // vectors per thread per tile
constexpr int WT_VECS = STREAM_THREADS * WT_PER;  // vectors per tile

// Smallest index whose value (in [mlo, mhi]) has its bit in the repeat bitmap. With
// bucket_mask (bucketed path), only values whose bucket saw a repeat look the
// bitmap up.
template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS, 4) first_dup_kernel(const T *__restrict__ x, int64_t n, int64_t mlo,
                                                                      int64_t mhi, Hdr *h,
                                                                      const unsigned *__restrict__ dup,
                                                                      const unsigned *__restrict__ bucket_mask,
                                                                      unsigned long long *slot) {
    IXP_KERNEL_ENTRY();
    if (h->status || !h->flag) return;
    const unsigned lw = bucket_mask ? (unsigned)h->spare[BK_LW] : 0u;
    __shared__ unsigned s_mask[BK_MAX / 32];
    __shared__ unsigned s_bfirst, s_blast;
    const unsigned long long base = h->base, span = h->span;
    if (threadIdx.x == 0) {
        s_bfirst = ~0u;
        s_blast = 0u;
    }
    __syncthreads();
    if (bucket_mask)
        for (int w = threadIdx.x; w < (int)(BK_MAX / 32); w += blockDim.x) {
            const unsigned m = bucket_mask[w];
            s_mask[w] = m;
            if (m) {
                atomicMin(&s_bfirst, (unsigned)w * 32u + (unsigned)(__ffs(m) - 1));
                atomicMax(&s_blast, (unsigned)w * 32u + (unsigned)(31 - __clz(m)));
            }
        }
    __syncthreads();
    // values outside the flagged buckets' range [lo_f, lo_f + span_f) hold no repeat
    unsigned long long lo_f = 0, span_f = span;
    if (bucket_mask) {
        if (s_bfirst == ~0u) return;  // no bucket flagged, no repeat to find
        lo_f = (unsigned long long)s_bfirst << lw;
        span_f = ((unsigned long long)(s_blast - s_bfirst) + 1ull) << lw;
    }
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::N;
    Split<T> s(x, n);
    int64_t best = INT64_MAX;
    auto one = [&](int64_t i, T xv) {
        const int64_t xi = (int64_t)xv;
        const unsigned long long rel = (unsigned long long)xi - base;
        if (rel - lo_f >= span_f || rel >= span || xi < mlo || xi > mhi) return;
        if (bucket_mask) {
            const unsigned b = (unsigned)(rel >> lw);
            if (!(s_mask[b >> 5] & (1u << (b & 31)))) return;
        }
        if (__ldg(dup + (rel >> 5)) & (1u << (rel & 31))) best = i < best ? i : best;
    };
    if (blockIdx.x == 0) {
        for (int64_t i = threadIdx.x; i < s.head; i += blockDim.x) one(i, x[i]);
        for (int64_t i = s.tail0 + threadIdx.x; i < n; i += blockDim.x) one(i, x[i]);
        if (best != INT64_MAX) atomic_max_u64(slot, enc_first(best));
    }
    const VT *xv = reinterpret_cast<const VT *>(x + s.head);
    const int64_t ntiles = (s.nvec + WT_VECS - 1) / WT_VECS;
    for (int64_t c = blockIdx.x; c < ntiles; c += gridDim.x) {
        const unsigned long long cur = ld_relaxed_u64(slot);
        if (cur && s.head + c * WT_VECS * V > dec_first(cur)) break;
        VT a[WT_PER];
#pragma unroll
        for (int u = 0; u < WT_PER; u++) {
            const int64_t v = c * WT_VECS + u * STREAM_THREADS + threadIdx.x;
            if (v < s.nvec) a[u] = ldv(xv + v);
        }
#pragma unroll
        for (int u = 0; u < WT_PER; u++) {
            const int64_t v = c * WT_VECS + u * STREAM_THREADS + threadIdx.x;
            if (v >= s.nvec) continue;
            int64_t e[V];
            unpack(a[u], e);
#pragma unroll
            for (int k = 0; k < V; k++) one(s.head + v * V + k, (T)e[k]);
        }
        if (best != INT64_MAX) {
            atomic_max_u64(slot, enc_first(best));
            best = INT64_MAX;
        }
    }
}

// Partner of the first repeated index i*: the smallest j > i* with x[j] = x[i*].
template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS, 4) partner_kernel(const T *__restrict__ x, int64_t n, Hdr *h,
                                                                    const unsigned long long *slot) {
    IXP_KERNEL_ENTRY();
    if (h->status || !h->flag || !*slot) return;
    const int64_t i0 = dec_first(*slot);
    const T v0 = x[i0];
    const int64_t start = i0 + 1;
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::N;
    const T *xs = x + start;
    const int64_t m = n - start;
    Split<T> s(xs, m);
    int64_t best = INT64_MAX;
    if (blockIdx.x == 0) {
        for (int64_t i = threadIdx.x; i < s.head; i += blockDim.x)
            if (xs[i] == v0) best = i < best ? i : best;
        for (int64_t i = s.tail0 + threadIdx.x; i < m; i += blockDim.x)
            if (xs[i] == v0) best = i < best ? i : best;
        if (best != INT64_MAX) atomic_max_u64(&h->k_aux, enc_first(start + best));
        best = INT64_MAX;
    }
    const VT *xv = reinterpret_cast<const VT *>(xs + s.head);
    const int64_t ntiles = (s.nvec + WT_VECS - 1) / WT_VECS;
    for (int64_t c = blockIdx.x; c < ntiles; c += gridDim.x) {
        const unsigned long long cur = ld_relaxed_u64(&h->k_aux);
        if (cur && start + s.head + c * WT_VECS * V > dec_first(cur)) break;
        VT a[WT_PER];
#pragma unroll
        for (int u = 0; u < WT_PER; u++) {
            const int64_t v = c * WT_VECS + u * STREAM_THREADS + threadIdx.x;
            if (v < s.nvec) a[u] = ldv(xv + v);
        }
#pragma unroll
        for (int u = 0; u < WT_PER; u++) {
            const int64_t v = c * WT_VECS + u * STREAM_THREADS + threadIdx.x;
            if (v >= s.nvec) continue;
            int64_t e[V];
            unpack(a[u], e);
#pragma unroll
            for (int k = V - 1; k >= 0; k--)
                if ((T)e[k] == v0) best = min(best, s.head + v * V + k);
        }
        if (best != INT64_MAX) {
            atomic_max_u64(&h->k_aux, enc_first(start + best));
            best = INT64_MAX;
        }
    }
}

template <typename T>
__global__ void inj_finalize(const T *x, const Hdr *h, ixp_verdict *out) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    v.status = h->status;
    int64_t i = (h->flag && h->k_first) ? dec_first(h->k_first) : -1;
    v.ok = v.status ? -1 : (i < 0 ? 1 : 0);
    v.kind = (v.status || i < 0) ? IXP_V_NONE : IXP_V_DUPLICATE;
    v.index = v.status ? -1 : i;
    v.value = (v.status || i < 0) ? 0 : (int64_t)x[i];
    v.aux0 = (v.status || i < 0) ? 0 : (h->k_aux ? dec_first(h->k_aux) : -1);
    v.aux1 = 0;
    v.reserved = 0;
    *out = v;
}

// ====================================================== Inj, any value span
// When the span of the in-range values is wider than the workspace bitmap (int64
// ids, hashes, a range that covers most of the type), Inj is decided with an
// open-addressing hash set in the workspace: 2^k >= 2n slots of {key, first, second}
// (16 bytes, zeroed per call). Element i with value v in Rcd probes from slot
// mix(v) (the SplitMix64 finalizer, Steele, Lea and Flood 2014) and claims the
// first slot that is empty (key 0) or holds v (the key is v + 1, so that 0 marks an
// empty slot; v = -1 keeps its pair in the header instead). In the slot, first
// and second keep the two smallest positions of v, stored as ~i so that the
// atomic maximum keeps the minimum and 0 means none: first takes ~i, and second
// the smaller encoding of the old first and ~i, which leaves second = the second
// smallest position once every copy is in. A value with a second position is a
// repeat; the witness (reading 14) is the pair (first, second) with the smallest
// first, found by one sweep over the slots. n < 2^32 - 1 (32-bit positions).
struct HashSlot {
    unsigned long long key;
    unsigned first, second;
};
static_assert(sizeof(HashSlot) == 16, "hash slot must be 16 bytes");

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void hash_keep(unsigned *first, unsigned *second, unsigned enc) {
    const unsigned o = atomicMax(first, enc);
    if (o) atomicMax(second, min(o, enc));  // o = 0: no earlier copy, min(o, enc) = 0 changes nothing
}

// gate = 1: only as the fallback of the partitioned path (which set HP_FLAGS).
__device__ __forceinline__ bool hash_single_runs(const Hdr *h, int gate) {
    return !h->status && h->spare[BK_MODE] == BK_HASH && (!gate || h->spare[HP_FLAGS]);
}

template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS, 4) hash_insert_kernel(const T *__restrict__ x, int64_t n,
                                                                        int64_t rlo, int64_t rhi, Hdr *h,
                                                                        HashSlot *__restrict__ tab,
                                                                        unsigned long long mask, int gate) {
    IXP_KERNEL_ENTRY();
    if (!hash_single_runs(h, gate)) return;
    unsigned *nfirst = reinterpret_cast<unsigned *>(&h->spare[HS_NEG1]);  // the pair of v = -1
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += stride) {
        const int64_t v = (int64_t)__ldcs(x + i);
        if (v < rlo || v > rhi) continue;
        const unsigned enc = ~(unsigned)i;
        if (v == -1) {
            hash_keep(nfirst, nfirst + 1, enc);
            continue;
        }
        const unsigned long long key = (unsigned long long)v + 1ull;
        unsigned long long s = mix64((unsigned long long)v) & mask;
        for (unsigned long long probe = 0; probe <= mask; probe++) {  // the table is never full: ends
            const unsigned long long old = atomicCAS(&tab[s].key, 0ull, key);
            if (old == 0ull || old == key) {
                hash_keep(&tab[s].first, &tab[s].second, enc);
                break;
            }
            s = (s + 1) & mask;
        }
    }
}

// The hash set starts empty: zeroed only when the setup kernel chose the hash path
// (as a fallback, after the partitioned path's repeat, witness and partner).
__global__ void __launch_bounds__(STREAM_THREADS) hash_clear_kernel(Hdr *h, HashSlot *__restrict__ tab,
                                                                    unsigned long long slots, int gate) {
    IXP_KERNEL_ENTRY();
    if (!hash_single_runs(h, gate)) return;
    if (gate && blockIdx.x == 0 && threadIdx.x == 0) {
        h->flag = 0u;
        h->k_first = 0ull;
        h->k_aux = 0ull;
    }
    ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tab);
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < slots;
         k += (unsigned long long)gridDim.x * blockDim.x)
        __stcs(t2 + k, make_ulonglong2(0ull, 0ull));
}

// The smallest (first, second) pair over the slots with a second position, packed
// as first << 32 | second and kept with one atomic maximum of its encoding.
__global__ void __launch_bounds__(STREAM_THREADS) hash_witness_kernel(Hdr *h, const HashSlot *__restrict__ tab,
                                                                      unsigned long long slots, int gate) {
    IXP_KERNEL_ENTRY();
    if (!hash_single_runs(h, gate)) return;
    unsigned long long best = ~0ull;
    auto take = [&](unsigned f, unsigned sc) {
        if (!sc) return;
        const unsigned long long pk = ((unsigned long long)~f << 32) | (unsigned long long)~sc;
        best = pk < best ? pk : best;
    };
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned *nf = reinterpret_cast<const unsigned *>(&h->spare[HS_NEG1]);
        take(nf[0], nf[1]);
    }
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < slots;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const HashSlot e = tab[k];
        if (e.key) take(e.first, e.second);
    }
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    const unsigned long long r = block_max_u64(best == ~0ull ? 0ull : ~best, sm);
    if (threadIdx.x == 0 && r) atomicMax(&h->spare[HS_PAIR], r);
}

// Hash mode's verdict fields: index = first, aux0 = second (the first repeat).
__global__ void hash_result_kernel(Hdr *h, int gate) {
    IXP_KERNEL_ENTRY();
    if (!hash_single_runs(h, gate) || !h->spare[HS_PAIR]) return;
    const unsigned long long pk = ~h->spare[HS_PAIR];
    h->flag = 1u;
    h->k_first = enc_first((int64_t)(pk >> 32));
    h->k_aux = enc_first((int64_t)(pk & 0xffffffffull));
}

// ---------------------------------------------- Inj, any value span: partitioned
// For 2^21 < n <= 2^29 the hash set is split until each piece fits one SM's shared
// memory. hv = mix64(v) is a bijection of the 64-bit values, so v repeats exactly
// when hv does, and the keys hv + 1 (0 marks an empty slot and a pad) are grouped
// twice by the top bits of hv: into P parts (P a power of two, about 2^21 keys a
// part) and each part into HP_Q sub-parts (about 2^13 keys). Each grouping pass
// (hp_group_kernel) takes tiles of HP_TILE entries, stores each entry at its
// group's slot row at the rank its counting atomic returns (an entry past its row
// reserves a pool pair of its own), then reserves one pool run per group with one
// atomicAdd each and moves the rows there as 16-byte chunks. hp_set_kernel then
// gives each sub-part one block with an open-addressing set of 2^k >= 1.5 x its pool
// capacity in shared memory, probing from the low bits of hv; a key found in the set
// is a repeat, and its hv goes once into a list of repeated values. The witness
// pass scans x for the first element whose hv is listed (a set in shared memory),
// and the partner pass of the bitmap paths finds the smallest later copy. The one
// value whose hv is all ones is counted in the header. A group whose pool fills up
// (one value repeated very often, or values crafted to share a group) or more than
// HP_DUPCAP repeated values set HP_FLAGS, and the single-table path above then
// decides the call from scratch.
constexpr int64_t HP_MIN_N = (int64_t)1 << 21, HP_MAX_N = (int64_t)1 << 29;
constexpr int HP_THREADS = 256, HP_PER = 16, HP_TILE = HP_THREADS * HP_PER;
constexpr unsigned HP_LOGQ = 8, HP_Q = 1u << HP_LOGQ;  // sub-parts per part
constexpr unsigned HP_DUPCAP = 2048, HP_SET = 4096;      // listed repeats; slots of the witness pass's set
constexpr int HP_SET_THREADS = 1024;  // threads of a sub-part's block (one block a SM: its set is up to 128 KB)

// One grouping pass's shape: groups per tile, slot rows, pools.
struct HpLevel {
    unsigned logg;            // log2 of the groups an entry can go to (P, or HP_Q within its part)
    unsigned rcap;            // slot-row capacity per group per tile (even)
    unsigned rstride;         // row stride in entries (twice an odd number: 16-byte rows)
    unsigned long long cap;   // pool entries per group (even)
    unsigned *cursors;        // per group
    unsigned long long *pool; // groups x cap keys
};

struct HpCfg {
    unsigned logp;             // log2 of the part count P
    HpLevel l1, l2;            // P parts; P x HP_Q sub-parts
    unsigned tslots;           // slots of a sub-part's set (a power of two)
    unsigned long long *dups;  // HP_DUPCAP repeated hv
};

// Shared memory of a grouping pass: per group a count and a pool reservation, then
// the rows.
__host__ __device__ inline size_t hp_group_smem(const HpLevel &l) {
    return 2 * (size_t)(((1u << l.logg) * 4u + 15u) & ~15u) + (size_t)(1u << l.logg) * l.rstride * 8u;
}

// Zeroes both levels' pool cursors and the header slots.
__global__ void __launch_bounds__(STREAM_THREADS) hp_setup_kernel(Hdr *h, HpCfg c) {
    IXP_KERNEL_ENTRY();
    if (h->status || h->spare[BK_MODE] != BK_HASH) return;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    if (tid == 0) {
        h->spare[HP_FLAGS] = 0ull;
        h->spare[HP_NDUP] = 0ull;
        h->spare[HP_TOPH] = 0ull;
    }
    for (unsigned long long k = tid; k < (1ull << c.logp); k += stride) c.l1.cursors[k] = 0u;
    for (unsigned long long k = tid; k < ((unsigned long long)HP_Q << c.logp); k += stride) c.l2.cursors[k] = 0u;
}

// A grouping pass. SRC = 0: the entries are the in-Rcd elements of x (T), keyed by
// hv + 1 and grouped into parts by the top logp bits of hv. SRC = 1: the entries are
// the keys of the P part pools (tiles of one part each; pads skipped), grouped into
// the part's sub-parts by the next HP_LOGQ bits. Thread t of a tile holds the
// 16-byte vectors t, t + HP_THREADS, ... of the tile (16 entries).
template <typename T, int SRC>
__global__ void __launch_bounds__(HP_THREADS) hp_group_kernel(const T *__restrict__ x, int64_t n, int64_t rlo,
                                                              int64_t rhi, Hdr *h, HpCfg c, int vec_ok) {
    IXP_KERNEL_ENTRY();
    if (h->status || h->spare[BK_MODE] != BK_HASH) return;
    if (SRC == 1 && h->spare[HP_FLAGS]) return;
    constexpr int V = SRC == 0 ? Vec<T>::N : 2;
    constexpr int NV = HP_PER / V;
    const HpLevel &L = SRC == 0 ? c.l1 : c.l2;
    extern __shared__ __align__(16) unsigned char hp_raw[];
    const unsigned G = 1u << L.logg;
    const unsigned gb = (G * 4u + 15u) & ~15u;
    unsigned *s_cnt = reinterpret_cast<unsigned *>(hp_raw);
    unsigned *s_res = reinterpret_cast<unsigned *>(hp_raw + gb);  // pool slot of each group's run
    unsigned long long *s_row = reinterpret_cast<unsigned long long *>(hp_raw + 2 * gb);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned sh1 = 64u - c.logp, sh2 = 64u - c.logp - HP_LOGQ;
    for (unsigned g = tid; g < G; g += HP_THREADS) s_cnt[g] = 0u;
    __syncthreads();
    // SRC = 0: tiles of x; SRC = 1: tiles (part, j) over each part's pool region
    const int64_t per_part = SRC == 0 ? 0 : (int64_t)((c.l1.cap + HP_TILE - 1) / HP_TILE);
    const int64_t ntiles = SRC == 0 ? (n + HP_TILE - 1) / HP_TILE : per_part << c.logp;
    auto geom = [&](int64_t tile, unsigned &part, int64_t &t0, int64_t &m) {
        part = SRC == 0 ? 0u : (unsigned)(tile / per_part);
        t0 = SRC == 0 ? tile * HP_TILE : (tile - (int64_t)part * per_part) * HP_TILE;
        m = SRC == 0 ? n : (int64_t)min((unsigned long long)c.l1.cursors[part], c.l1.cap);  // part's entries
    };
    // a tile's 16-byte vectors, when the whole tile can be read so (pool tiles always:
    // regions and runs are 16-byte aligned and m is even); the next tile's are loaded
    // while this one is placed
    using RV = typename std::conditional<SRC == 0, typename Vec<T>::type, ulonglong2>::type;
    auto load_vecs = [&](int64_t tile, RV (&r)[NV]) -> bool {
        unsigned part;
        int64_t t0, m;
        geom(tile, part, t0, m);
        if (SRC == 0 && !(vec_ok && t0 + HP_TILE <= m)) return false;
        const RV *src = SRC == 0 ? reinterpret_cast<const RV *>(x)
                                 : reinterpret_cast<const RV *>(c.l1.pool + (unsigned long long)part * c.l1.cap);
#pragma unroll
        for (int j = 0; j < NV; j++) {
            const int64_t p0 = t0 + (int64_t)(j * HP_THREADS + tid) * V;
            if (p0 < m) r[j] = __ldcs(src + p0 / V);
            else r[j] = RV{};
        }
        return true;
    };
    RV nxt[NV];
    bool have = blockIdx.x < ntiles ? load_vecs(blockIdx.x, nxt) : false;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        unsigned part;
        int64_t t0, m;
        geom(tile, part, t0, m);
        RV cur[NV];
#pragma unroll
        for (int j = 0; j < NV; j++) cur[j] = nxt[j];
        const bool cur_vec = have;
        have = tile + gridDim.x < ntiles ? load_vecs(tile + gridDim.x, nxt) : false;
        if (SRC == 1 && t0 >= m) continue;  // an empty tile of the part's region (uniform over the block)
#pragma unroll
        for (int j = 0; j < NV; j++) {
            const int64_t p0 = t0 + (int64_t)(j * HP_THREADS + tid) * V;
            unsigned long long key[V];  // hv + 1 of the entry, 0 for none
            if constexpr (SRC == 0) {
                int64_t e[V];
                if (cur_vec) {
                    unpack(cur[j], e);
                } else {
#pragma unroll
                    for (int q = 0; q < V; q++) e[q] = p0 + q < m ? (int64_t)x[p0 + q] : 0;
                }
#pragma unroll
                for (int q = 0; q < V; q++) {
                    const int64_t v = (int64_t)(T)e[q];
                    key[q] = 0ull;
                    if (p0 + q >= m || v < rlo || v > rhi) continue;
                    const unsigned long long hv = mix64((unsigned long long)v);
                    if (hv == ~0ull) atomicAdd(&h->spare[HP_TOPH], 1ull);
                    else key[q] = hv + 1ull;
                }
            } else {
                key[0] = cur[j].x;  // zero past the part's entries
                key[1 % V] = cur[j].y;
            }
#pragma unroll
            for (int q = 0; q < V; q++) {
                if (!key[q]) continue;
                const unsigned long long hv = key[q] - 1ull;
                const unsigned g = SRC == 0 ? (unsigned)(hv >> sh1) : (unsigned)(hv >> sh2) & (HP_Q - 1u);
                const unsigned rk = atomicAdd(&s_cnt[g], 1u);
                if (rk < L.rcap) {
                    s_row[(size_t)g * L.rstride + rk] = key[q];
                } else {
                    // past the row: a pool pair of its own (key, pad), keeping runs 16-byte aligned
                    const unsigned long long gg = (unsigned long long)part * G + g;
                    const unsigned at = atomicAdd(&L.cursors[gg], 2u);
                    if ((unsigned long long)at + 2ull <= L.cap) {
                        L.pool[gg * L.cap + at] = key[q];
                        L.pool[gg * L.cap + at + 1] = 0ull;
                    } else {
                        atomicOr(&h->spare[HP_FLAGS], HP_F_POOL);
                    }
                }
            }
        }
        __syncthreads();
        // one pool reservation per group, all at once (thread g for group g), rounded up
        // to whole 16-byte chunks (pad key 0)
        for (unsigned g = tid; g < G; g += HP_THREADS) {
            const unsigned cr = (min(s_cnt[g], L.rcap) + 1u) & ~1u;
            const unsigned at = cr ? atomicAdd(&L.cursors[(unsigned long long)part * G + g], cr) : 0u;
            s_res[g] = at;
            if ((unsigned long long)at + cr > L.cap) atomicOr(&h->spare[HP_FLAGS], HP_F_POOL);
        }
        __syncthreads();
        // rows to the pools: warp w moves groups w, w + 8, ...
        for (unsigned g = wid; g < G; g += HP_THREADS / 32) {
            const unsigned cnt = min(s_cnt[g], L.rcap);
            const unsigned cr = (cnt + 1u) & ~1u;
            const unsigned at = s_res[g];
            if ((unsigned long long)at + cr > L.cap) continue;
            const unsigned long long *row = s_row + (size_t)g * L.rstride;
            unsigned long long *dst = L.pool + ((unsigned long long)part * G + g) * L.cap + at;
            for (unsigned k = 2 * lane; k < cr; k += 64) {
                const ulonglong2 d = *reinterpret_cast<const ulonglong2 *>(row + k);
                __stcs(reinterpret_cast<ulonglong2 *>(dst + k), make_ulonglong2(d.x, k + 1 < cnt ? d.y : 0ull));
            }
        }
        __syncthreads();  // rows and counts read
        for (unsigned g = tid; g < G; g += HP_THREADS) s_cnt[g] = 0u;
        __syncthreads();
    }
}

// One block per sub-part: its keys into a set of c.tslots slots in shared memory
// (plus one bit per slot: the slot's key is listed as a repeat). Block 0 also
// lists the all-ones hv when it occurred twice or more.
__global__ void __launch_bounds__(HP_SET_THREADS) hp_set_kernel(Hdr *h, HpCfg c) {
    IXP_KERNEL_ENTRY();
    if (h->status || h->spare[BK_MODE] != BK_HASH || h->spare[HP_FLAGS]) return;
    extern __shared__ __align__(16) unsigned char hs_raw[];
    unsigned long long *s_set = reinterpret_cast<unsigned long long *>(hs_raw);
    unsigned *s_rep = reinterpret_cast<unsigned *>(s_set + c.tslots);
    const unsigned mask = c.tslots - 1u;
    auto list = [&](unsigned long long hv) {
        const unsigned long long k = atomicAdd(&h->spare[HP_NDUP], 1ull);
        if (k < HP_DUPCAP) c.dups[k] = hv;
        else atomicOr(&h->spare[HP_FLAGS], HP_F_DUPS);
        atomicOr(&h->flag, 1u);
    };
    if (blockIdx.x == 0 && threadIdx.x == 0 && h->spare[HP_TOPH] >= 2ull) list(~0ull);
    const unsigned long long sp = blockIdx.x;
    const unsigned npair = (unsigned)min((unsigned long long)c.l2.cursors[sp], c.l2.cap) / 2;
    const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(c.l2.pool + sp * c.l2.cap);
    ulonglong2 *z = reinterpret_cast<ulonglong2 *>(s_set);
    for (unsigned k = threadIdx.x; k < c.tslots / 2; k += blockDim.x) z[k] = make_ulonglong2(0ull, 0ull);
    for (unsigned k = threadIdx.x; k < c.tslots / 32; k += blockDim.x) s_rep[k] = 0u;
    __syncthreads();
    for (unsigned q = threadIdx.x; q < npair; q += blockDim.x) {
        const ulonglong2 d = __ldcs(src + q);
        const unsigned long long kk[2] = {d.x, d.y};
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const unsigned long long key = kk[j];
            if (!key) continue;  // pad
            unsigned s = (unsigned)(key - 1ull) & mask;
            for (unsigned probe = 0; probe <= mask; probe++) {  // fewer keys than slots: ends
                const unsigned long long old = atomicCAS(&s_set[s], 0ull, key);
                if (old == 0ull) break;
                if (old == key) {  // a repeat
                    const unsigned bit = 1u << (s & 31);
                    if (!(atomicOr(&s_rep[s >> 5], bit) & bit)) list(key - 1ull);
                    break;
                }
                s = (s + 1u) & mask;
            }
        }
    }
}

// Witness of the partitioned path: the smallest i whose hv is a listed repeat (the
// first occurrence of the value whose first occurrence comes first), in index
// order with the same early stop as first_dup_kernel.
template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS, 4) hp_first_kernel(const T *__restrict__ x, int64_t n, int64_t rlo,
                                                                     int64_t rhi, Hdr *h, HpCfg c) {
    IXP_KERNEL_ENTRY();
    if (h->status || h->spare[BK_MODE] != BK_HASH || h->spare[HP_FLAGS] || !h->flag) return;
    __shared__ unsigned long long s_set[HP_SET];  // hv + 1 of the listed repeats, 0 = empty
    __shared__ int s_top;                         // hv = all ones is a listed repeat
    for (int k = threadIdx.x; k < (int)HP_SET; k += blockDim.x) s_set[k] = 0ull;
    if (threadIdx.x == 0) s_top = 0;
    __syncthreads();
    const unsigned nd = (unsigned)min(h->spare[HP_NDUP], (unsigned long long)HP_DUPCAP);
    for (unsigned k = threadIdx.x; k < nd; k += blockDim.x) {
        const unsigned long long hv = c.dups[k];
        if (hv == ~0ull) {
            s_top = 1;
            continue;
        }
        unsigned s = (unsigned)hv & (HP_SET - 1u);
        for (unsigned probe = 0; probe < HP_SET; probe++) {  // at most HP_DUPCAP keys in HP_SET slots: ends
            const unsigned long long old = atomicCAS(&s_set[s], 0ull, hv + 1ull);
            if (old == 0ull || old == hv + 1ull) break;
            s = (s + 1u) & (HP_SET - 1u);
        }
    }
    __syncthreads();
    auto listed = [&](int64_t v) -> bool {
        if (v < rlo || v > rhi) return false;
        const unsigned long long hv = mix64((unsigned long long)v);
        if (hv == ~0ull) return s_top != 0;
        unsigned s = (unsigned)hv & (HP_SET - 1u);
        for (unsigned probe = 0; probe < HP_SET; probe++) {
            const unsigned long long k = s_set[s];
            if (k == hv + 1ull) return true;
            if (k == 0ull) return false;
            s = (s + 1u) & (HP_SET - 1u);
        }
        return false;
    };
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::N;
    Split<T> sp(x, n);
    unsigned long long *slot = &h->k_first;
    int64_t best = INT64_MAX;
    if (blockIdx.x == 0) {
        for (int64_t i = threadIdx.x; i < sp.head; i += blockDim.x)
            if (listed((int64_t)x[i])) best = min(best, i);
        for (int64_t i = sp.tail0 + threadIdx.x; i < n; i += blockDim.x)
            if (listed((int64_t)x[i])) best = min(best, i);
        if (best != INT64_MAX) atomic_max_u64(slot, enc_first(best));
        best = INT64_MAX;
    }
    const VT *xv = reinterpret_cast<const VT *>(x + sp.head);
    const int64_t ntiles = (sp.nvec + WT_VECS - 1) / WT_VECS;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const unsigned long long cur = ld_relaxed_u64(slot);
        if (cur && sp.head + t * WT_VECS * V > dec_first(cur)) break;
        VT a[WT_PER];
#pragma unroll
        for (int u = 0; u < WT_PER; u++) {
            const int64_t v = t * WT_VECS + u * STREAM_THREADS + threadIdx.x;
            if (v < sp.nvec) a[u] = ldv(xv + v);
        }
#pragma unroll
        for (int u = 0; u < WT_PER; u++) {
            const int64_t v = t * WT_VECS + u * STREAM_THREADS + threadIdx.x;
            if (v >= sp.nvec) continue;
            int64_t e[V];
            unpack(a[u], e);
#pragma unroll
            for (int k = 0; k < V; k++)
                if (listed((int64_t)(T)e[k])) best = min(best, sp.head + v * V + k);
        }
        if (best != INT64_MAX) {
            atomic_max_u64(slot, enc_first(best));
            best = INT64_MAX;
        }
    }
}

// Bij "missing" value: when nothing is out of image and nothing repeats but fewer
// than |Img| elements hit the image, the smallest clear bit is the first value no
// element takes.
__global__ void __launch_bounds__(STREAM_THREADS) missing_kernel(Hdr *h, const unsigned *__restrict__ bm) {
    IXP_KERNEL_ENTRY();
    if (h->status || h->flag || h->k_first) return;
    const unsigned long long span = h->span;
    if (h->cnt0 >= span) return;
    const unsigned long long words = (span + 31) / 32;
    unsigned long long best = ~0ull;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < words;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned z = ~bm[w];
        if (w == words - 1 && (span & 31)) z &= (1u << (span & 31)) - 1u;
        if (z) {
            best = w * 32 + (__ffs(z) - 1);
            break;
        }
    }
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    unsigned long long r = block_max_u64(best == ~0ull ? 0ull : enc_first((int64_t)best), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_aux, r);
}

template <typename T>
__global__ void bij_finalize(const T *x, const Hdr *h, ixp_verdict *out, int64_t img_lo, int64_t img_size) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    v.status = h->status;
    v.reserved = 0;
    v.aux0 = (int64_t)h->cnt0;
    v.aux1 = img_size;
    int64_t ooi = h->k_first ? dec_first(h->k_first) : -1;
    int64_t dupi = (h->flag && h->k_first2) ? dec_first(h->k_first2) : -1;
    if (v.status) {
        v.ok = -1;
        v.kind = IXP_V_NONE;
        v.index = -1;
        v.value = 0;
    } else if (ooi >= 0 && (dupi < 0 || ooi < dupi)) {
        v.ok = 0;
        v.kind = IXP_V_OUT_OF_IMAGE;
        v.index = ooi;
        v.value = (int64_t)x[ooi];
    } else if (dupi >= 0) {
        v.ok = 0;
        v.kind = IXP_V_DUPLICATE;
        v.index = dupi;
        v.value = (int64_t)x[dupi];
    } else if ((int64_t)h->cnt0 < img_size) {
        v.ok = 0;
        v.kind = IXP_V_MISSING;
        v.index = -1;
        v.value = img_lo + (h->k_aux ? dec_first(h->k_aux) : 0);
    } else {
        v.ok = 1;
        v.kind = IXP_V_NONE;
        v.index = -1;
        v.value = 0;
    }
    *out = v;
}

// ============================================== Inj / Bij, value-bucketed path
// For large spans the bitmap is split into B buckets of W = 2^lw consecutive
// values. Pass 1 reads X once and writes each in-range value's offset (rel mod W)
// into its bucket's region of a pool: a block sorts its tile by bucket in shared
// memory (a counting sort), reserves space with one atomicAdd per bucket, and writes
// contiguous runs. Pass 2 gives each bucket one block with a W-bit shared-memory
// bitmap and sets one bit per stored offset; the atomicOr's return value flags a
// repeat, which is recorded in the global repeat bitmap for the witness passes.
// A bucket that receives more values than its pool region holds sends the excess
// through L2 atomics on the global mark bitmap (pass 1), and pass 2 merges those
// bits before it sets its own, so skewed inputs stay exact.

struct BucketCfg {
    unsigned lw;                // log2 of the bucket width W (values per bucket)
    unsigned bmax;              // bucket count the launch shapes are sized for
    unsigned long long pool;    // pool capacity in entries
};

// Spans up to 2^28 take at most 512 buckets with a width picked on the device from
// the span found ("staged" shape); wider spans, up to the host's bucket shape, the
// host's configuration with up to BK_MAX buckets ("wide" shape).
constexpr unsigned long long ST_MAX_SPAN = 1ull << 28;
constexpr unsigned ST_LOGB = 9;  // at most 512 buckets: about 16 elements per bucket per tile
constexpr unsigned ST_LW_MIN = 10;

__host__ __device__ inline unsigned ceil_log2_u64(unsigned long long v) {
    unsigned l = 0;
    while (l < 64 && (1ull << l) < v) l++;
    return l;
}

// Bucket width of the staged path: the smallest power of two that gives at most
// 2^logb buckets (and at least 2^ST_LW_MIN values per bucket).
__host__ __device__ inline unsigned staged_lw(unsigned long long span, unsigned logb) {
    const unsigned l = ceil_log2_u64(span);
    return l > logb + ST_LW_MIN ? l - logb : ST_LW_MIN;
}

__global__ void bucket_setup_kernel(Hdr *h, int fixed, int64_t lo, int64_t hi, unsigned long long cap_bits,
                                    BucketCfg cfg, unsigned staged_logb, unsigned *cursors, unsigned *marks,
                                    unsigned *dup, unsigned *bucket_mask, int hash_ok) {
    IXP_KERNEL_ENTRY();
    unsigned long long base = 0, span = 0;
    bool too_big = false;
    if (fixed) {
        base = (unsigned long long)lo;
        span = (unsigned long long)hi - (unsigned long long)lo + 1ull;
        too_big = span == 0 || span > cap_bits;
    } else {
        const int64_t mn = dec_min(h->k_min), mx = dec_max(h->k_max);
        if (mn <= mx) {
            const unsigned long long d = (unsigned long long)mx - (unsigned long long)mn;
            too_big = d >= cap_bits;
            base = (unsigned long long)mn;
            span = d + 1ull;
        }
    }
    const bool staged = !too_big && span <= ST_MAX_SPAN;
    const unsigned lw = staged ? staged_lw(span, staged_logb) : cfg.lw;
    const unsigned long long nb = too_big ? 0ull : (span + (1ull << lw) - 1ull) >> lw;
    if (too_big || (!staged && nb > cfg.bmax)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (hash_ok) h->spare[BK_MODE] = BK_HASH;  // decided by the hash-set pass instead
            else set_status(h, IXP_E_SPAN);
        }
        return;
    }
    const unsigned long long cap = nb ? (cfg.pool / nb) & ~3ull : 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h->base = base;
        h->span = span;
        h->spare[BK_NB] = nb;
        h->spare[BK_CAP] = cap;
        h->spare[BK_LW] = lw;
        h->spare[BK_MODE] = staged ? BK_STAGED : BK_WIDE;
    }
    const unsigned long long words = (span + 31) / 32;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long w = tid; w < words; w += stride) {
        marks[w] = 0u;
        dup[w] = 0u;
    }
    for (unsigned long long b = tid; b < nb; b += stride) cursors[b] = 0u;
    for (unsigned long long w = tid; w < BK_MAX / 32; w += stride) bucket_mask[w] = 0u;
}

// Pass 1: each block takes tiles of BK_TILE elements. An element whose value lies
// in [base, base + span) (the bitmap's range: Img for Bij, the fixed Rcd or the
// observed [min, max] for Inj) has rel = value - base, bucket rel >> lw and offset
// rel & (W - 1); its rank among the tile's entries of its bucket is the return
// value of the bucket's counting atomic. Each bucket's entries are written to its
// pool as one contiguous run; entries past a bucket's pool capacity go to the
// global bitmap through L2 atomics instead. For Bij, elements of Rcd outside Img
// give the first such index (k_first).
//
// Two kernels. bucket_slot_kernel (at most BS_SLOT_NB buckets: the staged shape)
// stores each entry straight into a fixed row of BS_CAP slots of its bucket at its
// rank, so a tile needs neither a block-wide scan of the bucket counts nor a lookup
// of its bucket's start; each warp then moves the rows of its 32 buckets to the
// pools. A tile in which some bucket gets more than BS_CAP entries (clustered or
// repeated values) is redone from the registers by the counting sort below. That
// counting sort (scan of the counts, entries placed in bucket order in shared
// memory, runs written out) is all of bucket_scatter_kernel, which serves the wide
// shape (up to BK_MAX buckets).
constexpr int BS_THREADS = 512;
constexpr int BS_PER = BK_TILE / BS_THREADS;  // elements per thread per tile
constexpr unsigned BS_PAD_MAX = 1024;         // most buckets for the padded-run write-out
constexpr unsigned BS_SLOT_NB = 512;          // buckets of the slot kernel: 16 entries per bucket per tile
constexpr unsigned BS_CAP = 40;               // slots per bucket row (a multiple of 4: whole 16-byte chunks)
// Row stride in words: a multiple of 4 (16-byte rows, read back as 16-byte chunks)
// that is an odd multiple of 4, so that rows of random buckets start in 8 different
// bank groups (the ranks stored at the same time are close to one another, and with
// a stride of 48 words the stores fell into two groups and took twice as long). Word
// BS_CAP of a row is a spare that takes the stores of ranks past BS_CAP.
constexpr unsigned BS_STRIDE = BS_CAP + 4;
static_assert(BS_STRIDE % 4 == 0 && (BS_STRIDE / 4) % 2 == 1, "16-byte rows, odd in 16-byte units");
constexpr unsigned BS_SENT = ~0u;             // pad entry (pass 2 skips it)

// Shared memory of the counting sort. Per bucket: pool index of tile slot 0 (8
// bytes), count, start, limit (4 bytes each); the sorted tile (TILE entries, plus up
// to 3 pad entries per bucket when runs are padded to 16-byte chunks); with padding,
// the bucket of each 16-byte chunk (2 bytes).
// Layout: sorted tile (16-byte aligned, rounded to whole chunks) | pool index of
// slot 0 per bucket | count | start | limit | chunk -> bucket.
__host__ __device__ constexpr unsigned bs_sorted_cap(unsigned bmax, bool pad) {
    return pad ? (BK_TILE + 3 * bmax + 3) & ~3u : BK_TILE;
}
__host__ __device__ constexpr size_t bs_smem_bytes(unsigned bmax, bool pad) {
    return (size_t)bs_sorted_cap(bmax, pad) * 4 + (size_t)bmax * (8 + 4 + 4 + 4) +
           (pad ? (size_t)(bs_sorted_cap(bmax, pad) / 4) * 2 : 0);
}
// Shared memory of the slot kernel: the counts (BS_SLOT_NB words), then one region
// that holds either the slot rows or the counting sort's arrays other than the
// counts (a tile that falls back to the counting sort no longer needs its rows).
__host__ __device__ constexpr size_t bs_slot_region_bytes() {
    return (size_t)BS_SLOT_NB * BS_STRIDE * 4 > bs_smem_bytes(BS_SLOT_NB, true) - (size_t)BS_SLOT_NB * 4
               ? (size_t)BS_SLOT_NB * BS_STRIDE * 4
               : bs_smem_bytes(BS_SLOT_NB, true) - (size_t)BS_SLOT_NB * 4;
}
__host__ __device__ constexpr size_t bs_slot_smem_bytes() { return (size_t)BS_SLOT_NB * 4 + bs_slot_region_bytes(); }

// Bucket of an element, or -1 when its value is outside [base, base + span):
// rel = x - base in 64 bits, or in 32 bits when the caller has checked that the
// whole range [base, base + span) lies inside the int32 range (then the unsigned
// 32-bit difference is below span exactly for the values in range).
template <bool R32, typename T>
__device__ __forceinline__ bool bs_rel(T x, unsigned long long base, unsigned long long span, unsigned span_m1,
                                       unsigned &rel) {
    if (R32) {
        rel = (unsigned)(int)x - (unsigned)base;
        return rel <= span_m1;
    } else {
        const unsigned long long r = (unsigned long long)(int64_t)x - base;
        rel = (unsigned)r;
        return r < span;
    }
}

// Pass 1 over one tile's elements already in registers: count each in-range
// element's bucket in shared memory (the atomic's return value is its rank in the
// bucket) and remember which were in range (vm).
template <typename T, bool BIJ, bool R32, bool FULL>
__device__ __forceinline__ void bs_classify(const T (&e)[BS_PER / Vec<T>::N][Vec<T>::N], int64_t t0, int64_t n,
                                            int tid, unsigned long long base, unsigned long long span,
                                            unsigned span_m1, unsigned lw, unsigned *s_cnt, int64_t rlo, int64_t rhi,
                                            unsigned (&rv)[BS_PER], unsigned (&rk)[BS_PER], unsigned &vm,
                                            int64_t &ooi) {
    constexpr int V = Vec<T>::N;
    constexpr int NV = BS_PER / V;
#pragma unroll
    for (int j = 0; j < NV; j++) {
#pragma unroll
        for (int c = 0; c < V; c++) {
            const int q = j * V + c;
            const int64_t i = t0 + (int64_t)(j * BS_THREADS + tid) * V + c;
            unsigned rel;
            const bool in = bs_rel<R32>(e[j][c], base, span, span_m1, rel);
            rv[q] = rel;
            if ((FULL || i < n) && in) {
                rk[q] = atomicAdd(&s_cnt[rel >> lw], 1u);
                vm |= 1u << q;
            } else if (BIJ && (FULL || i < n) && (int64_t)e[j][c] >= rlo && (int64_t)e[j][c] <= rhi) {
                ooi = i < ooi ? i : ooi;
            }
        }
    }
}

// Loads one tile's elements (16-byte vectors when the array is 16-byte aligned,
// zeros past n).
template <typename T>
__device__ __forceinline__ void bs_load(const T *__restrict__ x, int64_t t0, int64_t n, bool full, int vec_ok, int tid,
                                        T (&e)[BS_PER / Vec<T>::N][Vec<T>::N]) {
    constexpr int V = Vec<T>::N;
    constexpr int NV = BS_PER / V;
#pragma unroll
    for (int j = 0; j < NV; j++) {
        const int64_t p0 = t0 + (int64_t)(j * BS_THREADS + tid) * V;
        if (vec_ok && (full || p0 + V <= n)) {
            if (V == 4) {
                int4 v = __ldcs(reinterpret_cast<const int4 *>(x + p0));
                e[j][0] = (T)v.x;
                e[j][1 % V] = (T)v.y;
                e[j][2 % V] = (T)v.z;
                e[j][3 % V] = (T)v.w;
            } else {
                longlong2 v = __ldcs(reinterpret_cast<const longlong2 *>(x + p0));
                e[j][0] = (T)v.x;
                e[j][1 % V] = (T)v.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < V; c++) e[j][c] = (p0 + c < n) ? x[p0 + c] : (T)0;
        }
    }
}

// An entry that does not fit its bucket's pool region: its bit goes straight into
// the global mark bitmap (pass 2 merges it), a bit already set is a repeat.
__device__ __forceinline__ void bs_spill(unsigned v, unsigned b, unsigned *marks, unsigned *dup, unsigned *bucket_mask,
                                         unsigned &anydup) {
    const unsigned bit = 1u << (v & 31);
    const unsigned old = atomicOr(marks + (v >> 5), bit);
    if (old & bit) {
        atomicOr(dup + (v >> 5), bit);
        atomicOr(bucket_mask + (b >> 5), 1u << (b & 31));
        anydup = 1;
    }
}

// Shared arrays of the counting sort.
struct BsSort {
    unsigned *cnt;         // nb: entries per bucket (filled by bs_classify)
    unsigned *sorted;      // the tile in bucket order (+ pads)
    long long *dst;        // pool index of tile slot 0, per bucket
    unsigned *start;       // first tile slot, per bucket
    unsigned *lim;         // tile slots below this fit the pool, per bucket
    unsigned short *cb;    // bucket of each 16-byte chunk (PAD)
    unsigned *wsum;        // BS_THREADS / 32
    unsigned *total;       // 1
};

// The counting sort of one tile whose ranks are counted (s.cnt, rk): exclusive scan
// of the (padded) bucket counts, pool space reserved per bucket with one atomicAdd
// each, entries placed in bucket order, runs written out. PAD: runs padded to whole
// 16-byte chunks written as 16-byte stores (every chunk lies in one bucket's run and
// starts on a 16-byte boundary of the pool: bucket regions, cursors and runs are all
// multiples of four entries); otherwise entries keep their bucket in the sorted tile
// and are stored one by one. Contains two block barriers; returns before the sorted
// tile has been read by every thread.
template <bool PAD>
__device__ __forceinline__ void bs_sort_tile(const BsSort &s, const unsigned (&rv)[BS_PER],
                                             const unsigned (&rk)[BS_PER], unsigned vm, unsigned nb, unsigned lw,
                                             unsigned long long cap, unsigned *__restrict__ cursors,
                                             unsigned *__restrict__ pool, unsigned *__restrict__ marks,
                                             unsigned *__restrict__ dup, unsigned *__restrict__ bucket_mask,
                                             unsigned &anydup) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned wmask = (1u << lw) - 1u;
    const unsigned per = (nb + BS_THREADS - 1) / BS_THREADS;  // bucket-count scan entries per thread
    {
        unsigned loc = 0;
        const unsigned b0 = tid * per;
        for (unsigned k = 0; k < per; k++)
            if (b0 + k < nb) loc += PAD ? (s.cnt[b0 + k] + 3u) & ~3u : s.cnt[b0 + k];
        unsigned y = loc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            unsigned o = __shfl_up_sync(FULL, y, d);
            if (lane >= d) y += o;
        }
        if (lane == 31) s.wsum[wid] = y;
        __syncthreads();
        unsigned wpre = 0, tot = 0;
#pragma unroll
        for (int i = 0; i < BS_THREADS / 32; i++) {
            wpre += i < wid ? s.wsum[i] : 0u;
            tot += s.wsum[i];
        }
        unsigned run = wpre + y - loc;
        for (unsigned k = 0; k < per; k++)
            if (b0 + k < nb) {
                const unsigned b = b0 + k, c = s.cnt[b];
                const unsigned cr = PAD ? (c + 3u) & ~3u : c;  // reserved entries
                const unsigned long long g = cr ? atomicAdd(&cursors[b], cr) : 0ull;
                s.start[b] = run;
                s.dst[b] = (long long)((unsigned long long)b * cap + g) - (long long)run;
                s.lim[b] = g >= cap ? run : run + (unsigned)min((unsigned long long)cr, cap - g);
                if (PAD) {
                    for (unsigned p = c; p < cr; p++) s.sorted[run + p] = BS_SENT;
                    for (unsigned p = 0; p < cr; p += 4) s.cb[(run + p) >> 2] = (unsigned short)b;
                }
                run += cr;
            }
        if (tid == 0) *s.total = tot;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BS_PER; q++)
        if ((vm >> q) & 1u) s.sorted[s.start[rv[q] >> lw] + rk[q]] = PAD ? (rv[q] & wmask) : rv[q];
    __syncthreads();
    const unsigned total = *s.total;
    if (PAD) {
        for (unsigned k = tid; k < total / 4; k += BS_THREADS) {
            const unsigned b = s.cb[k];
            const unsigned p = 4 * k;
            const uint4 d = *reinterpret_cast<const uint4 *>(s.sorted + p);
            const long long dst = s.dst[b] + (long long)p;
            const unsigned lim = s.lim[b];
            if (p + 4 <= lim) {
                __stcs(reinterpret_cast<uint4 *>(pool + dst), d);
            } else {
                const unsigned o[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    if (p + c < lim) pool[dst + c] = o[c];  // pads too: pass 2 reads every reserved slot
                    else if (o[c] != BS_SENT) bs_spill((b << lw) | o[c], b, marks, dup, bucket_mask, anydup);
                }
            }
        }
    } else {
        for (unsigned p = tid; p < total; p += BS_THREADS) {
            const unsigned v = s.sorted[p];
            const unsigned b = v >> lw;
            if (p < s.lim[b]) __stcs(pool + (s.dst[b] + (long long)p), v & wmask);
            else bs_spill(v, b, marks, dup, bucket_mask, anydup);
        }
    }
}

// Per-block results of pass 1: in-range count, whether a spilled entry repeated,
// and (Bij) the first element of Rcd outside Img.
template <bool BIJ>
__device__ __forceinline__ void bs_finish(Hdr *h, unsigned long long valid, unsigned anydup, int64_t ooi) {
    __shared__ unsigned long long sm[BS_THREADS / 32];
    const unsigned long long tv = block_sum_u64(valid, sm);
    if (threadIdx.x == 0 && tv) atomicAdd(&h->cnt0, tv);
    if (__syncthreads_or(anydup) && threadIdx.x == 0) atomicOr(&h->flag, 1u);
    if (BIJ) {
        const unsigned long long r = block_max_u64(ooi == INT64_MAX ? 0ull : enc_first(ooi), sm);
        if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
    }
}

// Whether [base, base + span) lies in the int32 range, so that 32-bit relative
// values are exact.
template <typename T>
__device__ __forceinline__ bool bs_r32(unsigned long long base, unsigned long long span) {
    return sizeof(T) == 4 && span >= 1 && span <= (1ull << 32) && (int64_t)base >= (int64_t)INT32_MIN &&
           (int64_t)base <= (int64_t)INT32_MAX && (int64_t)base + (int64_t)(span - 1) <= (int64_t)INT32_MAX;
}

template <typename T, bool BIJ>
__device__ __forceinline__ void bs_classify_tile(const T (&e)[BS_PER / Vec<T>::N][Vec<T>::N], bool r32, bool full,
                                                 int64_t t0, int64_t n, unsigned long long base,
                                                 unsigned long long span, unsigned span_m1, unsigned lw,
                                                 unsigned *s_cnt, int64_t rlo, int64_t rhi, unsigned (&rv)[BS_PER],
                                                 unsigned (&rk)[BS_PER], unsigned &vm, int64_t &ooi) {
    const int tid = threadIdx.x;
    if (r32 && full)
        bs_classify<T, BIJ, true, true>(e, t0, n, tid, base, span, span_m1, lw, s_cnt, rlo, rhi, rv, rk, vm, ooi);
    else if (full)
        bs_classify<T, BIJ, false, true>(e, t0, n, tid, base, span, span_m1, lw, s_cnt, rlo, rhi, rv, rk, vm, ooi);
    else
        bs_classify<T, BIJ, false, false>(e, t0, n, tid, base, span, span_m1, lw, s_cnt, rlo, rhi, rv, rk, vm, ooi);
}

template <typename T, bool BIJ, bool PAD>
__global__ void __launch_bounds__(BS_THREADS, 2) bucket_scatter_kernel(
    const T *__restrict__ x, int64_t n, int64_t rlo, int64_t rhi, Hdr *h, BucketCfg cfg, unsigned long long mode,
    unsigned *__restrict__ cursors, unsigned *__restrict__ pool, unsigned *__restrict__ marks,
    unsigned *__restrict__ dup, unsigned *__restrict__ bucket_mask, int vec_ok) {
    IXP_KERNEL_ENTRY();
    if (h->status || h->spare[BK_MODE] != mode) return;
    constexpr int V = Vec<T>::N;
    extern __shared__ __align__(16) unsigned char bk_raw[];
    __shared__ unsigned s_wsum[BS_THREADS / 32];
    __shared__ unsigned s_total;
    const unsigned bmax = cfg.bmax;
    BsSort s;
    s.sorted = reinterpret_cast<unsigned *>(bk_raw);
    s.dst = reinterpret_cast<long long *>(s.sorted + bs_sorted_cap(bmax, PAD));
    s.cnt = reinterpret_cast<unsigned *>(s.dst + bmax);
    s.start = s.cnt + bmax;
    s.lim = s.start + bmax;
    s.cb = reinterpret_cast<unsigned short *>(s.lim + bmax);
    s.wsum = s_wsum;
    s.total = &s_total;
    const unsigned long long base = h->base, span = h->span;
    const unsigned nb = (unsigned)h->spare[BK_NB];
    const unsigned long long cap = h->spare[BK_CAP];
    const unsigned lw = (unsigned)h->spare[BK_LW];
    const bool r32 = bs_r32<T>(base, span);
    const unsigned span_m1 = (unsigned)(span - 1);
    const int64_t ntiles = (n + BK_TILE - 1) / BK_TILE;
    const int tid = threadIdx.x;
    unsigned long long valid = 0;
    unsigned anydup = 0;
    int64_t ooi = INT64_MAX;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = tile * BK_TILE;
        const bool full = t0 + BK_TILE <= n;
        for (unsigned b = tid; b < nb; b += BS_THREADS) s.cnt[b] = 0u;
        T e[BS_PER / V][V];
        bs_load<T>(x, t0, n, full, vec_ok, tid, e);
        __syncthreads();  // counts zeroed
        unsigned rv[BS_PER], rk[BS_PER], vm = 0;
        bs_classify_tile<T, BIJ>(e, r32, full, t0, n, base, span, span_m1, lw, s.cnt, rlo, rhi, rv, rk, vm, ooi);
        __syncthreads();
        bs_sort_tile<PAD>(s, rv, rk, vm, nb, lw, cap, cursors, pool, marks, dup, bucket_mask, anydup);
        valid += __popc(vm);
        __syncthreads();
    }
    bs_finish<BIJ>(h, valid, anydup, ooi);
}

// The slot kernel (staged shape, nb <= BS_SLOT_NB, n < 2^31). Per tile: classify
// (ranks from the counting atomics) and store each entry at slot row (bucket) x
// BS_STRIDE + rank. Unless a bucket overflowed its row, warp w moves the rows of buckets 32w ..
// 32w + 31: lane l reserves bucket 32w + l's run (its count rounded up to whole
// 16-byte chunks, the pad entries BS_SENT) with one atomicAdd, a warp scan of the
// chunk counts lays the 32 runs end to end, and lane j of round i moves chunk 32i + j
// of that sequence, finding its bucket from a bitmap of the runs' first chunks and
// the bucket's run from a per-warp table (one entry per non-empty bucket).
constexpr int BS_MAPW = 16;  // map words per warp: at least (32 x BS_CAP / 4) / 32
static_assert(32 * (BS_CAP / 4) <= 32 * BS_MAPW && 32 * (BS_CAP / 4) < 1024 && BS_CAP < 64,
              "run table packing: first chunk in 10 bits, count and limit in 6 and 8 bits");
template <typename T, bool BIJ>
__global__ void __launch_bounds__(BS_THREADS, 2) bucket_slot_kernel(
    const T *__restrict__ x, int64_t n, int64_t rlo, int64_t rhi, Hdr *h, unsigned long long mode,
    unsigned *__restrict__ cursors, unsigned *__restrict__ pool, unsigned *__restrict__ marks,
    unsigned *__restrict__ dup, unsigned *__restrict__ bucket_mask, int vec_ok) {
    IXP_KERNEL_ENTRY();
    if (h->status || h->spare[BK_MODE] != mode) return;
    constexpr int V = Vec<T>::N;
    extern __shared__ __align__(16) unsigned char bk_raw[];
    __shared__ unsigned s_wsum[BS_THREADS / 32];
    __shared__ unsigned s_total;
    __shared__ unsigned s_map[BS_THREADS / 32][BS_MAPW];  // first chunks of the warp's runs
    __shared__ uint2 s_tab[BS_THREADS / 32][32];          // per non-empty bucket: reserved slot, packed run
    unsigned *s_cnt = reinterpret_cast<unsigned *>(bk_raw);
    unsigned *s_slot = s_cnt + BS_SLOT_NB;  // BS_SLOT_NB rows of BS_STRIDE words
    const unsigned long long base = h->base, span = h->span;
    const unsigned nb = (unsigned)h->spare[BK_NB];
    const unsigned cap = (unsigned)h->spare[BK_CAP];  // pool entries (and so positions) are below 2^32
    const unsigned lw = (unsigned)h->spare[BK_LW];
    const unsigned wmask = (1u << lw) - 1u;
    const bool r32 = bs_r32<T>(base, span);
    const unsigned span_m1 = (unsigned)(span - 1);
    const unsigned ntiles = (unsigned)((n + BK_TILE - 1) / BK_TILE);  // n < 2^31
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lane_le = lane == 31 ? FULL : (2u << lane) - 1u;
    unsigned valid = 0;  // in-range entries this thread saw (n < 2^31)
    unsigned anydup = 0;
    int64_t ooi = INT64_MAX;
    for (unsigned b = tid; b < BS_SLOT_NB; b += BS_THREADS) s_cnt[b] = 0u;
    __syncthreads();
    for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = (int64_t)tile * BK_TILE;
        const bool full = t0 + BK_TILE <= n;
        T e[BS_PER / V][V];
        bs_load<T>(x, t0, n, full, vec_ok, tid, e);
        unsigned rv[BS_PER], rk[BS_PER], vm = 0, ovf = 0;
        // the common case, every element of the thread's share in range: no branch
        // per element (a rank past BS_CAP stores into the row's spare word)
        // (int64: the test first, rv after it, so that the 64-bit values die as rv fills)
        constexpr bool KEEP = sizeof(T) == 4;
        // (not for int64 Bij, where both forms inline would spill registers)
        bool all_in = full && !(BIJ && sizeof(T) == 8);
        if (all_in) {
#pragma unroll
            for (int j = 0; j < BS_PER / V; j++)
#pragma unroll
                for (int c = 0; c < V; c++) {
                    unsigned rel;
                    all_in &= r32 ? bs_rel<true>(e[j][c], base, span, span_m1, rel)
                                  : bs_rel<false>(e[j][c], base, span, span_m1, rel);
                    if (KEEP) rv[j * V + c] = rel;
                }
        }
        if (all_in) {
            if (!KEEP)
#pragma unroll
                for (int j = 0; j < BS_PER / V; j++)
#pragma unroll
                    for (int c = 0; c < V; c++) rv[j * V + c] = (unsigned)((unsigned long long)(int64_t)e[j][c] - base);
#pragma unroll
            for (int q = 0; q < BS_PER; q++) rk[q] = atomicAdd(&s_cnt[rv[q] >> lw], 1u);
#pragma unroll
            for (int q = 0; q < BS_PER; q++) {
                s_slot[(rv[q] >> lw) * BS_STRIDE + min(rk[q], BS_CAP)] = rv[q] & wmask;
                ovf |= rk[q] >= BS_CAP;
            }
            vm = (1u << BS_PER) - 1u;
        } else {
            bs_classify_tile<T, BIJ>(e, r32, full, t0, n, base, span, span_m1, lw, s_cnt, rlo, rhi, rv, rk, vm, ooi);
#pragma unroll
            for (int q = 0; q < BS_PER; q++)
                if ((vm >> q) & 1u) {
                    if (rk[q] < BS_CAP) s_slot[(rv[q] >> lw) * BS_STRIDE + rk[q]] = rv[q] & wmask;
                    else ovf = 1;
                }
        }
        valid += __popc(vm);
        if (__syncthreads_or(ovf)) {
            // count again (the ranks were not kept) and sort the tile instead
            for (unsigned b = tid; b < BS_SLOT_NB; b += BS_THREADS) s_cnt[b] = 0u;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < BS_PER; q++)
                if ((vm >> q) & 1u) rk[q] = atomicAdd(&s_cnt[rv[q] >> lw], 1u);
            __syncthreads();
            BsSort s;  // the counting sort's arrays overlay the rows
            s.cnt = s_cnt;
            s.sorted = s_slot;
            s.dst = reinterpret_cast<long long *>(s.sorted + bs_sorted_cap(BS_SLOT_NB, true));
            s.start = reinterpret_cast<unsigned *>(s.dst + BS_SLOT_NB);
            s.lim = s.start + BS_SLOT_NB;
            s.cb = reinterpret_cast<unsigned short *>(s.lim + BS_SLOT_NB);
            s.wsum = s_wsum;
            s.total = &s_total;
            bs_sort_tile<true>(s, rv, rk, vm, nb, lw, cap, cursors, pool, marks, dup, bucket_mask, anydup);
            // every thread is past the scan, the last reader of the counts
            for (unsigned b = tid; b < BS_SLOT_NB; b += BS_THREADS) s_cnt[b] = 0u;
        } else {
            const unsigned bl = wid * 32 + lane;
            unsigned c = 0;
            if (bl < nb) {
                c = s_cnt[bl];
                s_cnt[bl] = 0u;
            }
            const unsigned cr = (c + 3u) & ~3u;  // reserved entries, c <= BS_CAP
            const unsigned g = cr ? atomicAdd(&cursors[bl], cr) : 0u;
            const unsigned lim = g >= cap ? 0u : min(cr, cap - g);
            const unsigned nch = cr >> 2;
            unsigned sc = nch;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned o = __shfl_up_sync(FULL, sc, d);
                if (lane >= d) sc += o;
            }
            const unsigned first = sc - nch, nchunks = __shfl_sync(FULL, sc, 31);
            const unsigned nz = __ballot_sync(FULL, nch != 0);
            if (lane < BS_MAPW) s_map[wid][lane] = 0u;
            __syncwarp();
            if (nch) {
                atomicOr(&s_map[wid][first >> 5], 1u << (first & 31));
                s_tab[wid][__popc(nz & (lane_le >> 1))] =
                    make_uint2(g, first | (c << 10) | (lim << 16) | ((unsigned)lane << 24));
            }
            __syncwarp();
            unsigned before = 0;  // runs that start in earlier map words
#pragma unroll 1
            for (unsigned i = 0; 32 * i < nchunks; i++) {
                const unsigned word = s_map[wid][i];
                const unsigned r = before + __popc(word & lane_le) - 1u;  // this chunk's run
                before += __popc(word);
                const unsigned k = 32 * i + lane;
                if (k >= nchunks) continue;
                const uint2 tv = s_tab[wid][r];
                const unsigned cb = (tv.y >> 10) & 63u, limb = (tv.y >> 16) & 255u;
                const unsigned b = wid * 32 + (tv.y >> 24);
                const unsigned p = 4 * (k - (tv.y & 1023u));
                const uint4 d = *reinterpret_cast<const uint4 *>(s_slot + b * BS_STRIDE + p);
                const unsigned o[4] = {p < cb ? d.x : BS_SENT, p + 1 < cb ? d.y : BS_SENT, p + 2 < cb ? d.z : BS_SENT,
                                       p + 3 < cb ? d.w : BS_SENT};
                const unsigned long long dst = (unsigned long long)b * cap + tv.x + p;
                if (p + 4 <= limb) {
                    __stcs(reinterpret_cast<uint4 *>(pool + dst), make_uint4(o[0], o[1], o[2], o[3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if (p + j < limb) pool[dst + j] = o[j];  // pads too: pass 2 reads every reserved slot
                        else if (o[j] != BS_SENT) bs_spill((b << lw) | o[j], b, marks, dup, bucket_mask, anydup);
                    }
                }
            }
        }
        __syncthreads();  // rows (or the sorted tile) read, counts zeroed
    }
    bs_finish<BIJ>(h, (unsigned long long)valid, anydup, ooi);
}

// Pass 2: one block per bucket, a W-bit bitmap in shared memory. Launched once per
// pass-1 path (its grid and shared memory sized for that path's buckets); only the
// launch whose path the setup kernel chose does the work.
//
// NT threads a block: 256 for bitmaps up to 32 KB; 512 for 64 KB ones (two blocks
// a SM: 512 buckets then take two waves of two buckets per SM instead of two waves
// of three, with the same warps resident); 1024 for 128 KB (one a SM).
template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : (NT == 512 ? 2 : 1)) bucket_check_kernel(Hdr *h, unsigned long long mode,
                                                                  const unsigned *__restrict__ cursors,
                                                                  const unsigned *__restrict__ pool,
                                                                  const unsigned *__restrict__ marks,
                                                                  unsigned *__restrict__ dup,
                                                                  unsigned *__restrict__ bucket_mask, int bij) {
    IXP_KERNEL_ENTRY();
    extern __shared__ unsigned s_bm[];
    const unsigned nb = (unsigned)h->spare[BK_NB];
    const unsigned b = blockIdx.x;
    if (h->status || h->spare[BK_MODE] != mode || b >= nb) return;
    const unsigned long long cap = h->spare[BK_CAP], span = h->span;
    const unsigned lw = (unsigned)h->spare[BK_LW];
    const unsigned words = (1u << lw) / 32;
    const unsigned long long lo_rel = (unsigned long long)b << lw;
    const unsigned long long range = min(1ull << lw, span - lo_rel);  // values this bucket covers
    const unsigned cnt = cursors[b];
    const unsigned long long stored = min((unsigned long long)cnt, cap);
    const bool overflowed = cnt > cap;
    for (unsigned w = threadIdx.x; w < words; w += blockDim.x)
        s_bm[w] = (overflowed && (lo_rel >> 5) + w < (span + 31) / 32) ? marks[(lo_rel >> 5) + w] : 0u;
    __syncthreads();
    unsigned anydup = 0;
    const unsigned *src = pool + (unsigned long long)b * cap;
    const unsigned long long nv = stored / 4;
    constexpr int U = 8;  // 16-byte loads in flight per thread
    for (unsigned long long q0 = threadIdx.x; q0 < nv; q0 += (unsigned long long)U * blockDim.x) {
        uint4 o4[U];
#pragma unroll
        for (int j = 0; j < U; j++) {
            const unsigned long long q = q0 + (unsigned long long)j * blockDim.x;
            o4[j] = q < nv ? __ldcs(reinterpret_cast<const uint4 *>(src) + q) : make_uint4(~0u, ~0u, ~0u, ~0u);
        }
#pragma unroll
        for (int j = 0; j < U; j++) {
            const unsigned o[4] = {o4[j].x, o4[j].y, o4[j].z, o4[j].w};
#pragma unroll
            for (int c = 0; c < 4; c++) {
                if (o[c] == ~0u) continue;  // beyond this thread's share
                const unsigned bit = 1u << (o[c] & 31);
                if (atomicOr(&s_bm[o[c] >> 5], bit) & bit) {
                    atomicOr(dup + ((lo_rel + o[c]) >> 5), 1u << ((lo_rel + o[c]) & 31));
                    anydup = 1;
                }
            }
        }
    }
    for (unsigned long long q = nv * 4 + threadIdx.x; q < stored; q += blockDim.x) {
        const unsigned off = src[q];
        if (off == ~0u) continue;  // pad entry
        const unsigned bit = 1u << (off & 31);
        if (atomicOr(&s_bm[off >> 5], bit) & bit) {
            atomicOr(dup + ((lo_rel + off) >> 5), 1u << ((lo_rel + off) & 31));
            anydup = 1;
        }
    }
    if (__syncthreads_or(anydup) && threadIdx.x == 0) {
        atomicOr(&h->flag, 1u);
        atomicOr(bucket_mask + (b >> 5), 1u << (b & 31));
    }
    if (bij) {
        // smallest value of this bucket that no element takes (the entry count
        // cannot rule a gap out: padded runs reserve more slots than values)
        unsigned long long best = ~0ull;
        for (unsigned w = threadIdx.x; w < (range + 31) / 32; w += blockDim.x) {
            unsigned z = ~s_bm[w];
            if ((unsigned long long)(w + 1) * 32 > range) z &= (1u << (range & 31)) - 1u;
            if (z) {
                best = lo_rel + (unsigned long long)w * 32 + (__ffs(z) - 1);
                break;
            }
        }
        __shared__ unsigned long long sm[NT / 32];
        unsigned long long r = block_max_u64(best == ~0ull ? 0ull : enc_first((int64_t)best), sm);
        if (threadIdx.x == 0) atomic_max_u64(&h->k_aux, r);
    }
}

// ================================================================ host side




static int elem_size(int t) { return t == IXP_I32 ? 4 : 8; }

}  // namespace ixp

using namespace ixp;

extern "C" int ixp_check_range(const void *x, int itype, int64_t n, int64_t lo, int64_t hi, ixp_verdict *d_verdict,
                               void *ws, size_t ws_bytes, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (n < 0 || lo > hi || !d_verdict || (n > 0 && (!x || !aligned_to(x, elem_size(itype))))) return IXP_E_INVAL;
    int rc = check_ws(ws, ws_bytes, ixp_workspace_size(IXP_OP_RANGE, itype, n, 0));
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Hdr *h = (Hdr *)ws;
    if (cudaMemsetAsync(h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    int grid = stream_grid((n + 3) / 4);
    if (itype == IXP_I32) {
        // every int32 value violates when the bounds miss the int32 range entirely
        const int all_bad = lo > (int64_t)INT32_MAX || hi < (int64_t)INT32_MIN;
        const int32_t lo32 = (int32_t)std::max<int64_t>(lo, INT32_MIN), hi32 = (int32_t)std::min<int64_t>(hi, INT32_MAX);
        if (n > 0) range_kernel<int32_t><<<grid, STREAM_THREADS, 0, st>>>((const int32_t *)x, n, lo32, hi32, h);
        range_finalize<int32_t><<<1, 1, 0, st>>>((const int32_t *)x, n, h, d_verdict, all_bad);
    } else {
        if (n > 0) range_kernel<int64_t><<<grid, STREAM_THREADS, 0, st>>>((const int64_t *)x, n, lo, hi, h);
        range_finalize<int64_t><<<1, 1, 0, st>>>((const int64_t *)x, n, h, d_verdict, 0);
    }
    return launch_status();
}

template <typename T>
static void launch_mono(const T *x, int64_t n, int cmp, int grid, Hdr *h, cudaStream_t st) {
    switch (cmp) {
        case IXP_LE: mono_kernel<T, IXP_LE><<<grid, STREAM_THREADS, 0, st>>>(x, n, h); break;
        case IXP_LT: mono_kernel<T, IXP_LT><<<grid, STREAM_THREADS, 0, st>>>(x, n, h); break;
        case IXP_GE: mono_kernel<T, IXP_GE><<<grid, STREAM_THREADS, 0, st>>>(x, n, h); break;
        default: mono_kernel<T, IXP_GT><<<grid, STREAM_THREADS, 0, st>>>(x, n, h); break;
    }
}

extern "C" int ixp_check_mono(const void *x, int itype, int64_t n, int cmp, ixp_segs segs, ixp_verdict *d_verdict,
                              uint8_t *d_seg_ok, void *ws, size_t ws_bytes, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (n < 0 || cmp < 0 || cmp > 3 || !d_verdict || (n > 0 && (!x || !aligned_to(x, elem_size(itype)))))
        return IXP_E_INVAL;
    const bool seg = segs.offsets != nullptr;
    if ((seg && segs.nseg < 1) || (!seg && (segs.nseg != 0 || d_seg_ok))) return IXP_E_INVAL;
    int rc = check_ws(ws, ws_bytes, ixp_workspace_size(IXP_OP_MONO, itype, n, segs.nseg));
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Hdr *h = (Hdr *)ws;
    if (cudaMemsetAsync(h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (seg && d_seg_ok && cudaMemsetAsync(d_seg_ok, 1, (size_t)segs.nseg, st) != cudaSuccess) return IXP_E_CUDA;
    if (n > 1) {
        if (!seg) {
            int grid = stream_grid((n + 3) / 4);
            if (itype == IXP_I32) launch_mono((const int32_t *)x, n, cmp, grid, h, st);
            else launch_mono((const int64_t *)x, n, cmp, grid, h, st);
        } else {
            int64_t tiles = (n + SP_CHUNK - 1) / SP_CHUNK;
            int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * 8);
            int64_t *lb = (int64_t *)((char *)ws + HDR_BYTES);  // first segment at or after each chunk start
            if (cudaMemsetAsync(lb, 0, (size_t)tiles * 8, st) != cudaSuccess) return IXP_E_CUDA;
            chunk_lb_kernel<SP_CHUNK><<<stream_grid(segs.nseg + 1, 4), STREAM_THREADS, 0, st>>>(segs.offsets,
                                                                                               segs.nseg, n, lb);
            if (itype == IXP_I32)
                mono_seg_kernel<int32_t><<<grid, STREAM_THREADS, 0, st>>>((const int32_t *)x, n, cmp, segs.offsets,
                                                                          segs.nseg, lb, d_seg_ok, h);
            else
                mono_seg_kernel<int64_t><<<grid, STREAM_THREADS, 0, st>>>((const int64_t *)x, n, cmp, segs.offsets,
                                                                          segs.nseg, lb, d_seg_ok, h);
        }
    }
    if (itype == IXP_I32) mono_finalize<int32_t><<<1, 1, 0, st>>>((const int32_t *)x, h, d_verdict);
    else mono_finalize<int64_t><<<1, 1, 0, st>>>((const int64_t *)x, h, d_verdict);
    return launch_status();
}

namespace ixp {
// Workspace layouts for Inj/Bij. Small inputs: header | marks | repeats (two bitmaps).
// Large inputs (n >= BK_MIN_N): header | bucket cursors | pool | marks | repeats.
constexpr int64_t BK_MIN_N = 1 << 18;
constexpr unsigned long long BK_MIN_SPAN = 1ull << 21;

// Pool entries of the wide path (per-bucket regions, 32-bit positions).
static unsigned long long bk_pool_entries(int64_t n) {
    return ((unsigned long long)n + (unsigned long long)n / 4 + 4ull * BK_MAX + 3ull) & ~3ull;
}
size_t bk_prefix_bytes(int64_t n) {
    return HDR_BYTES + round256(BK_MAX * 4) + round256(BK_MAX / 8) + round256(bk_pool_entries(n) * 4);
}

struct BitmapWs {
    Hdr *h;
    unsigned *cursors, *bmask, *pool, *bm, *dup;
    unsigned long long cap;  // bits per bitmap
    bool buckets;            // bucketed layout available
    HashSlot *tab;           // hash set for spans wider than the bitmaps (nullptr: none)
    unsigned long long slots;
};

// Hash-set slots for n elements: the power of two at least 2n (at least 2).
unsigned long long inj_hash_slots(int64_t n) {
    unsigned long long c = 2;
    while (c < 2ull * (unsigned long long)(n > 0 ? n : 0)) c <<= 1;
    return c;
}
// Bitmap bits of the any-span workspace: the default span capacity 4n + 4096, at
// least the 2^21 bits every Inj workspace gets (as ixp_workspace_size sizes them).
static unsigned long long inj_default_span(int64_t n) {
    return std::max<unsigned long long>(4ull * (unsigned long long)(n > 0 ? n : 0) + 4096ull, BK_MIN_SPAN);
}

static BitmapWs bitmap_ws(void *ws, size_t ws_bytes, int64_t n, bool allow_hash) {
    BitmapWs w{};
    char *p = (char *)ws;
    w.h = (Hdr *)p;
    // pool positions and bucket cursors are 32-bit
    w.buckets = n >= BK_MIN_N && bk_pool_entries(n) < (1ull << 32) && ws_bytes >= bk_prefix_bytes(n) + 2 * (BK_MIN_SPAN / 8);
    size_t off = HDR_BYTES;
    if (w.buckets) {
        w.cursors = (unsigned *)(p + HDR_BYTES);
        w.bmask = (unsigned *)(p + HDR_BYTES + round256(BK_MAX * 4));
        w.pool = (unsigned *)(p + HDR_BYTES + round256(BK_MAX * 4) + round256(BK_MAX / 8));
        off = bk_prefix_bytes(n);
    }
    // the hash set sits at the end of the workspace when the workspace also leaves
    // the any-span bitmaps (two of inj_default_span bits) before it; a workspace
    // sized for a given span (no hash set) is smaller than that
    size_t end = ws_bytes;
    const size_t hb = round256(inj_hash_slots(n) * sizeof(HashSlot));
    const size_t bmin = 2 * round256((inj_default_span(n) + 31) / 32 * 4);
    if (allow_hash && n < (int64_t)UINT32_MAX && ws_bytes >= off + bmin + hb) {
        end = (ws_bytes - hb) & ~(size_t)255;
        w.tab = (HashSlot *)(p + end);
        w.slots = inj_hash_slots(n);
    }
    w.cap = end > off ? (unsigned long long)((end - off) / 8) * 32ull : 0ull;
    w.bm = (unsigned *)(p + off);
    w.dup = w.bm + w.cap / 32;
    return w;
}

size_t inj_any_span_ws_bytes(int64_t n) {
    const size_t prefix = n >= BK_MIN_N ? bk_prefix_bytes(n) : HDR_BYTES;
    return prefix + 2 * round256((inj_default_span(n) + 31) / 32 * 4) + round256(inj_hash_slots(n) * sizeof(HashSlot)) +
           256;
}

// Layout of the partitioned hash-set path inside the hash-set region (2^k >= 2n
// slots of 16 bytes): part cursors | sub-part cursors | repeat list | part pools |
// sub-part pools. P = 2^logp >= n / 2^21 (4 to 256 parts) and HP_Q sub-parts a
// part; a grouping pass's rows hold (entries per group per tile) + 6 x its square
// root + 8; a pool holds 1.25 x the mean keys of its group + 64; a sub-part's set
// 2^k >= 1.5 x its pool. False (the single table decides) for n <= HP_MIN_N, whose
// table already fits in L2, for n > HP_MAX_N, or when the layout does not fit.
static bool hp_layout(const BitmapWs &w, int64_t n, HpCfg *c) {
    if (!w.tab || n <= HP_MIN_N || n > HP_MAX_N) return false;
    unsigned logp = 2;
    while (logp < 8 && (unsigned long long)n > (1ull << (21 + logp))) logp++;
    const unsigned long long P = 1ull << logp, PQ = P * HP_Q;
    auto level = [](HpLevel &L, unsigned logg, unsigned long long mean) {
        L.logg = logg;
        const unsigned m = (unsigned)HP_TILE >> logg;
        unsigned sq = 1;
        while (sq * sq < m) sq++;
        L.rcap = (m + 6 * sq + 8 + 1) & ~1u;
        L.rstride = ((L.rcap / 2) & 1u) ? L.rcap : L.rcap + 2;
        L.cap = (mean + mean / 4 + 64ull + 1ull) & ~1ull;
    };
    level(c->l1, logp, (unsigned long long)n / P);
    level(c->l2, HP_LOGQ, (unsigned long long)n / PQ);
    unsigned ts = 64;
    while (ts < c->l2.cap + c->l2.cap / 2) ts <<= 1;
    c->logp = logp;
    c->tslots = ts;
    char *base = (char *)w.tab;
    size_t off = 0;
    c->l1.cursors = (unsigned *)(base + off);
    off += round256((size_t)P * 4);
    c->l2.cursors = (unsigned *)(base + off);
    off += round256((size_t)PQ * 4);
    c->dups = (unsigned long long *)(base + off);
    off += round256((size_t)HP_DUPCAP * 8);
    c->l1.pool = (unsigned long long *)(base + off);
    off += round256((size_t)(P * c->l1.cap * 8));
    c->l2.pool = (unsigned long long *)(base + off);
    off += round256((size_t)(PQ * c->l2.cap * 8));
    return off <= (size_t)w.slots * sizeof(HashSlot) && hp_group_smem(c->l1) <= 200 * 1024 &&
           hp_group_smem(c->l2) <= 200 * 1024 && (size_t)ts * 8 + ts / 8 <= 200 * 1024;
}

// Bucket width: about two buckets per SM, between 2^14 and 2^19 values (a 64 KB
// shared bitmap), widened to 2^20 if the bucket count would exceed BK_MAX.
static bool bucket_config(unsigned long long span, unsigned long long pool, BucketCfg *cfg) {
    unsigned long long target = span / (2ull * (unsigned long long)num_sms());
    unsigned lw = 14;
    while (lw < 19 && (1ull << (lw + 1)) <= target) lw++;
    unsigned long long bmax = (span + (1ull << lw) - 1) >> lw;
    if (bmax > BK_MAX) {
        lw = 20;
        bmax = (span + (1ull << lw) - 1) >> lw;
    }
    if (bmax > BK_MAX) return false;
    cfg->lw = lw;
    cfg->bmax = (unsigned)bmax;
    cfg->pool = pool;
    return true;
}

// Pass 1 with the launch shape of one path: `shape` gives the bucket count the
// shared memory is laid out for; the bucket width comes from the setup kernel.
template <typename T, bool BIJ>
static void launch_pass1(const T *x, int64_t n, int64_t rlo, int64_t rhi, const BitmapWs &w, const BucketCfg &shape,
                         unsigned long long mode, int vec, cudaStream_t st) {
    const int64_t ntiles = (n + BK_TILE - 1) / BK_TILE;
    const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms() * 2));
    if (shape.bmax <= BS_SLOT_NB && n < (1ll << 31)) {
        // fixed slot rows per bucket (16 elements per bucket per tile on average)
        cudaFuncSetAttribute(bucket_slot_kernel<T, BIJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bs_slot_smem_bytes());
        bucket_slot_kernel<T, BIJ><<<g1, BS_THREADS, bs_slot_smem_bytes(), st>>>(
            x, n, rlo, rhi, w.h, mode, w.cursors, w.pool, w.bm, w.dup, w.bmask, vec);
    } else if (shape.bmax <= BS_PAD_MAX && n < (1ll << 31)) {
        // runs padded to 16-byte chunks (at least 8 elements per bucket per tile on average)
        cudaFuncSetAttribute(bucket_scatter_kernel<T, BIJ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bs_smem_bytes(BS_PAD_MAX, true));
        bucket_scatter_kernel<T, BIJ, true><<<g1, BS_THREADS, bs_smem_bytes(shape.bmax, true), st>>>(
            x, n, rlo, rhi, w.h, shape, mode, w.cursors, w.pool, w.bm, w.dup, w.bmask, vec);
    } else {
        cudaFuncSetAttribute(bucket_scatter_kernel<T, BIJ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bs_smem_bytes(BK_MAX, false));
        bucket_scatter_kernel<T, BIJ, false><<<g1, BS_THREADS, bs_smem_bytes(shape.bmax, false), st>>>(
            x, n, rlo, rhi, w.h, shape, mode, w.cursors, w.pool, w.bm, w.dup, w.bmask, vec);
    }
    // shape.lw: the widest bucket this launch can be given (the device may choose a narrower one)
    const unsigned bm_bytes = (1u << shape.lw) / 8;
#define IXP_BK_CHECK(NT)                                                                                       \
    cudaFuncSetAttribute(bucket_check_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (1 << 20) / 8);  \
    bucket_check_kernel<NT><<<shape.bmax, NT, bm_bytes, st>>>(w.h, mode, w.cursors, w.pool, w.bm, w.dup, w.bmask, \
                                                              BIJ ? 1 : 0)
    if (bm_bytes <= 32768u) {
        IXP_BK_CHECK(256);
    } else if (bm_bytes <= 65536u) {
        IXP_BK_CHECK(512);
    } else {
        IXP_BK_CHECK(1024);
    }
#undef IXP_BK_CHECK
}

// span_cap: the largest span the setup kernel can find (the fixed range, or the
// bitmap capacity when the range comes from the data). Spans up to 2^28 get at most
// 512 buckets with a width picked on the device from the span found; when span_cap
// is wider, the launch shape of the host's bucket configuration is launched too
// and runs only if the span found is above 2^28.
template <typename T, bool BIJ>
static void launch_buckets(const T *x, int64_t n, int64_t rlo, int64_t rhi, int fixed, int64_t flo, int64_t fhi,
                           unsigned long long span_cap, const BitmapWs &w, const BucketCfg &cfg, cudaStream_t st) {
    const int sgrid = num_sms() * 4;
    bucket_setup_kernel<<<sgrid, STREAM_THREADS, 0, st>>>(w.h, fixed, flo, fhi, w.cap, cfg, ST_LOGB, w.cursors, w.bm,
                                                          w.dup, w.bmask, w.tab != nullptr);
    const int vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    // staged shape: room for 2^ST_LOGB buckets (a narrower span found on the device
    // gives narrower buckets, never more of them), and the widest bucket the span cap
    // allows for the shared bitmap of pass 2
    const unsigned long long scap = std::min<unsigned long long>(span_cap, ST_MAX_SPAN);
    const BucketCfg sshape{staged_lw(scap, ST_LOGB), 1u << ST_LOGB, cfg.pool};
    launch_pass1<T, BIJ>(x, n, rlo, rhi, w, sshape, BK_STAGED, vec, st);
    if (span_cap > ST_MAX_SPAN) launch_pass1<T, BIJ>(x, n, rlo, rhi, w, cfg, BK_WIDE, vec, st);
}

template <typename T>
static void run_bitmap_check(const T *x, int64_t n, int64_t rlo, int64_t rhi, bool bij, int64_t ilo, int64_t ihi,
                             const BitmapWs &w, ixp_verdict *out, cudaStream_t st) {
    Hdr *h = w.h;
    unsigned *bm = w.bm, *dup = w.dup;
    const unsigned long long cap = w.cap;
    const int grid = stream_grid((n + 3) / 4);
    const int sgrid = num_sms() * 4;
    BucketCfg cfg{};
    if (bij) {
        const unsigned long long isize = (unsigned long long)ihi - (unsigned long long)ilo + 1ull;
        if (w.buckets && isize >= BK_MIN_SPAN && bucket_config(isize, bk_pool_entries(n), &cfg)) {
            launch_buckets<T, true>(x, n, rlo, rhi, 1, ilo, ihi, isize, w, cfg, st);
            first_dup_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, ilo, ihi, h, dup, w.bmask, &h->k_first2);
        } else {
            bitmap_setup_kernel<<<sgrid, STREAM_THREADS, 0, st>>>(h, 1, ilo, ihi, cap, bm, dup, 0);
            if (n > 0) {
                mark_kernel<T, true><<<grid, STREAM_THREADS, 0, st>>>(x, n, rlo, rhi, ilo, ihi, h, bm, dup);
                first_dup_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, ilo, ihi, h, dup, nullptr, &h->k_first2);
            }
            missing_kernel<<<sgrid, STREAM_THREADS, 0, st>>>(h, bm);
        }
        bij_finalize<T><<<1, 1, 0, st>>>(x, h, out, ilo, (int64_t)((unsigned long long)ihi - (unsigned long long)ilo + 1));
        return;
    }
    // Inj: a finite Rcd that fits the bitmap is used as is; otherwise find [min, max].
    const unsigned long long rspan = (unsigned long long)rhi - (unsigned long long)rlo + 1ull;
    const bool fixed = rspan != 0 && rspan <= cap && rspan <= 4ull * (unsigned long long)n + 4096ull;
    if (!fixed && n > 0) {
        // Rcd clamped to T's values; an empty clamp leaves lo > hi, so nothing is in range.
        const int64_t clo = std::max<int64_t>(rlo, (int64_t)Lim<T>::lo);
        const int64_t chi = std::min<int64_t>(rhi, (int64_t)Lim<T>::hi);
        const bool none = clo > chi;
        minmax_in_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, none ? Lim<T>::hi : (T)clo,
                                                             none ? Lim<T>::lo : (T)chi, h);
    }
    const unsigned long long span_cap = fixed ? rspan : cap;
    const bool bk = w.buckets && span_cap >= BK_MIN_SPAN && bucket_config(span_cap, bk_pool_entries(n), &cfg);
    if (bk) {
        launch_buckets<T, false>(x, n, rlo, rhi, fixed ? 1 : 0, rlo, rhi, span_cap, w, cfg, st);
    } else {
        bitmap_setup_kernel<<<sgrid, STREAM_THREADS, 0, st>>>(h, fixed ? 1 : 0, rlo, rhi, cap, bm, dup,
                                                              w.tab != nullptr);
        if (n > 0) mark_kernel<T, false><<<grid, STREAM_THREADS, 0, st>>>(x, n, rlo, rhi, rlo, rhi, h, bm, dup);
    }
    if (n > 0) {
        first_dup_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, rlo, rhi, h, dup, bk ? w.bmask : nullptr,
                                                             &h->k_first);
        partner_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, h, &h->k_first);
    }
    if (w.tab && n > 0) {  // spans wider than the bitmaps: the hash set decides (the kernels exit otherwise)
        HpCfg hc{};
        const int gate = hp_layout(w, n, &hc) ? 1 : 0;
        if (gate) {  // partitioned; the single table below runs only if it gives up
            const size_t sm1 = hp_group_smem(hc.l1), sm2 = hp_group_smem(hc.l2);
            const size_t sms = (size_t)hc.tslots * 8 + hc.tslots / 8;
            const int64_t t1 = (n + HP_TILE - 1) / HP_TILE;
            const int64_t t2 = (int64_t)((hc.l1.cap + HP_TILE - 1) / HP_TILE) << hc.logp;
            const int64_t gcap = (int64_t)num_sms() * 4;
            hp_setup_kernel<<<sgrid, STREAM_THREADS, 0, st>>>(h, hc);
            cudaFuncSetAttribute(hp_group_kernel<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
            hp_group_kernel<T, 0><<<(int)std::min(t1, gcap), HP_THREADS, sm1, st>>>(
                x, n, rlo, rhi, h, hc, (reinterpret_cast<uintptr_t>(x) & 15u) == 0);
            cudaFuncSetAttribute(hp_group_kernel<int64_t, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
            hp_group_kernel<int64_t, 1><<<(int)std::min(t2, gcap), HP_THREADS, sm2, st>>>(nullptr, n, rlo, rhi, h,
                                                                                          hc, 1);
            cudaFuncSetAttribute(hp_set_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms);
            hp_set_kernel<<<(unsigned)(HP_Q << hc.logp), HP_SET_THREADS, sms, st>>>(h, hc);
            hp_first_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, rlo, rhi, h, hc);
            partner_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, h, &h->k_first);
        }
        hash_clear_kernel<<<sgrid, STREAM_THREADS, 0, st>>>(h, w.tab, w.slots, gate);
        hash_insert_kernel<T><<<grid, STREAM_THREADS, 0, st>>>(x, n, rlo, rhi, h, w.tab, w.slots - 1, gate);
        hash_witness_kernel<<<sgrid, STREAM_THREADS, 0, st>>>(h, w.tab, w.slots, gate);
        hash_result_kernel<<<1, 1, 0, st>>>(h, gate);
    }
    inj_finalize<T><<<1, 1, 0, st>>>(x, h, out);
}
}  // namespace ixp

extern "C" int ixp_check_inj(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi,
                             ixp_verdict *d_verdict, void *ws, size_t ws_bytes, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (n < 0 || rcd_lo > rcd_hi || !d_verdict || (n > 0 && (!x || !aligned_to(x, elem_size(itype)))))
        return IXP_E_INVAL;
    int rc = check_ws(ws, ws_bytes, HDR_BYTES + 256);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const BitmapWs w = bitmap_ws(ws, ws_bytes, n, true);
    if (cudaMemsetAsync(w.h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (itype == IXP_I32)
        run_bitmap_check((const int32_t *)x, n, rcd_lo, rcd_hi, false, 0, 0, w, d_verdict, st);
    else
        run_bitmap_check((const int64_t *)x, n, rcd_lo, rcd_hi, false, 0, 0, w, d_verdict, st);
    return launch_status();
}

extern "C" int ixp_check_bij(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, int64_t img_lo,
                             int64_t img_hi, ixp_verdict *d_verdict, void *ws, size_t ws_bytes, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (n < 0 || rcd_lo > rcd_hi || img_lo > img_hi || img_lo < rcd_lo || img_hi > rcd_hi || !d_verdict ||
        (n > 0 && (!x || !aligned_to(x, elem_size(itype)))))
        return IXP_E_INVAL;
    const unsigned long long isize = (unsigned long long)img_hi - (unsigned long long)img_lo + 1ull;
    if (isize == 0 || isize > (1ull << 40)) return IXP_E_INVAL;
    int rc = check_ws(ws, ws_bytes, HDR_BYTES + 256);
    if (rc) return rc;
    const BitmapWs w = bitmap_ws(ws, ws_bytes, n, false);
    if (isize > w.cap) return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(w.h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (itype == IXP_I32)
        run_bitmap_check((const int32_t *)x, n, rcd_lo, rcd_hi, true, img_lo, img_hi, w, d_verdict, st);
    else
        run_bitmap_check((const int64_t *)x, n, rcd_lo, rcd_hi, true, img_lo, img_hi, w, d_verdict, st);
    return launch_status();
}

extern "C" unsigned long long ixp_tu_kernels_checks(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}
