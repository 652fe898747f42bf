// classes.cu - InvFiltPart with v classes (Sec. 2.3, FiltPart Y X (e_k, p^f, p^p_1..v)
// and its scatter-index form): per segment k, the elements kept by p^f are placed
// stably by class, class 0 first, after all kept elements of the segments before
// k. Element i's class is min(cls[i], v - 1); the last class collects everything
// the first v - 1 class predicates leave over.
//
// The destination of a kept element i of segment k and class h is
//     F_k + (kept elements of segment k with class < h) + (class-h elements of
//     segment k before i),
// and a dropped element's Z must lie outside [0, N). Flat arrays with v <= 4 use
// tiles of 4096 elements, 16 consecutive ones per thread: the check is one pass
// that records, per tile and class, the constant Z - (rank in the tile), then a
// pass that scans the tile counts and compares each constant with its class
// prefix, and an element-by-element pass over the first failing tile only; the
// partition counts the tiles, scans the counts and writes. Flat arrays with more
// classes use three tiled passes (per-tile class histograms; a scan of each class
// over the tiles with the class bases; the comparison, where an element's rank
// inside its tile comes from the lanes of its warp with the same class and
// per-warp class counters).
// Segmented arrays give each segment to one block (claimed from a counter): its
// class histogram, the class bases, then the comparison chunk by chunk with class
// counters carried from chunk to chunk; F_k comes from a scan of the per-segment
// kept counts. The first wrong element and its expected destination are packed
// into one word (i << 32 | expected + 1) whose smallest value wins, so no
// separate witness pass is needed.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "preds.cuh"

namespace ixp {

constexpr int CL_TILE = 4096;
constexpr int CL_THREADS = 256;
constexpr int CL_WARPS = CL_THREADS / 32;
constexpr int CL_ROUNDS = CL_TILE / CL_THREADS;  // 32-element rounds per warp per tile
constexpr int CL_MAXV = 256;
constexpr int CL_G = 1024;  // group size of the per-segment count scan

// Header slot for the packed first mismatch (complemented, raised with atomicMax).
__device__ __forceinline__ void cl_report(Hdr *h, int64_t i, int64_t ref) {
    const unsigned long long packed = ((unsigned long long)i << 32) | (unsigned long long)(ref + 1);
    atomicMax(&h->k_first, ~packed);
}

template <typename KT>
__device__ __forceinline__ int cl_class(const KT *keys, const uint8_t *cls, const DPred &filt, int v, int64_t i) {
    const int64_t key = keys ? (int64_t)__ldg(keys + i) : 0;
    if (!pred_one(filt, key, i)) return -1;  // dropped
    const int c = (int)__ldg(cls + i);
    return c < v - 1 ? c : v - 1;
}

// ----------------------------------------------------------- flat: pass 1
// VS > 0 (v <= VS): warps count classes with one ballot per class and add the
// warp totals, instead of one shared atomic per element (few classes would
// serialise on a few counters).
template <typename KT, int VS>
__global__ void __launch_bounds__(CL_THREADS) cl_count_kernel(const KT *__restrict__ keys,
                                                              const uint8_t *__restrict__ cls, int64_t n, DPred filt,
                                                              int v, int64_t nt, unsigned *__restrict__ cnt) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned s_h[CL_MAXV];
    for (int c = threadIdx.x; c < v; c += CL_THREADS) s_h[c] = 0u;
    __syncthreads();
    const int64_t t0 = blockIdx.x * (int64_t)CL_TILE;
    if constexpr (VS > 0) {
        unsigned wc[VS];
#pragma unroll
        for (int k = 0; k < VS; k++) wc[k] = 0u;
        for (int e = threadIdx.x; e < CL_TILE; e += CL_THREADS) {  // whole warps stay in the loop
            const int64_t i = t0 + e;
            const int c = i < n ? cl_class(keys, cls, filt, v, i) : -1;
#pragma unroll
            for (int k = 0; k < VS; k++) wc[k] += __popc(__ballot_sync(FULL, c == k));
        }
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < VS; k++)
                if (k < v && wc[k]) atomicAdd(&s_h[k], wc[k]);
    } else {
        for (int e = threadIdx.x; e < CL_TILE; e += CL_THREADS) {
            const int64_t i = t0 + e;
            if (i >= n) break;
            const int c = cl_class(keys, cls, filt, v, i);
            if (c >= 0) atomicAdd(&s_h[c], 1u);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < v; c += CL_THREADS) cnt[(int64_t)c * nt + blockIdx.x] = s_h[c];
}

// ----------------------------------------------------------- flat, v <= 4
// A thread takes the CL_PER consecutive elements of its tile slot (one 16-byte
// class load, 16-byte key and Z loads), so one block scan of the threads' class
// counts gives every element's rank, which then runs as a per-class counter.
//
// The check needs one pass over Z: for a kept element of class k at tile rank r,
// Z - r must be the same constant C_k(t) for every class-k element of tile t, and
// C_k(t) must equal base_k + (class-k elements of the tiles before t). The tile
// pass records C_k(t) (or "several values") and each tile's class counts; a
// decide pass scans the counts and compares; only the first failing tile (which
// holds the first wrong element, since a tile whose constants all match and whose
// dropped elements lie outside [0, N) has no wrong element) is revisited element
// by element. The per-tile counts are also summed per range of tiles (atomic adds
// into one counter pair per range), so the decide pass gets every range's prefix
// without a second kernel.
constexpr int CL_PER = CL_TILE / CL_THREADS;  // consecutive elements per thread
static_assert(CL_PER == 16, "16 four-bit class codes per thread fill one 64-bit word");
constexpr long long CL_NONE = LLONG_MIN;      // no element of the class in the tile
constexpr long long CL_BAD = LLONG_MIN + 1;   // the class's Z - rank is not one constant
constexpr int CL_MAX_RANGES = 1024;

struct ClRec {
    long long c[4];
};

// Tiles per decide thread so that at most CL_MAX_RANGES ranges of
// CL_THREADS * tpt tiles cover the array.
static inline int cl_tpt(int64_t nt) {
    const int64_t per = (int64_t)CL_THREADS * CL_MAX_RANGES;
    return (int)std::max<int64_t>(1, (nt + per - 1) / per);
}

struct Cl16Ws {
    ulonglong2 *rs;               // per range: class counts (c0 | c1 << 32, c2 | c3 << 32)
    unsigned long long *tcnt;     // per tile: class counts, 16 bits each
    ClRec *rec;                   // per tile: C_k(t)
    unsigned long long *dmin;     // per tile: smallest dropped Z, as uint64 (negative: huge)
    ulonglong2 *pre;              // per tile: first destination of each class (32 bits each)
    unsigned long long *codes;    // per thread slot of a tile: its 16 class codes (the partition's pass 1)
    int tpt;
    int64_t nr;                   // ranges
    size_t clear;                 // bytes after the header that must start zeroed (the range counters)
    size_t bytes;                 // bytes after the header
};

// Layout after the header: range counters | tile counts | records | dropped minima |
// first destinations | class codes. With ws null only the sizes are filled in.
static Cl16Ws cl16_ws(void *ws, int64_t n) {
    const int64_t nt = (n + CL_TILE - 1) / CL_TILE;
    Cl16Ws W;
    W.tpt = cl_tpt(nt);
    const int64_t R = (int64_t)W.tpt * CL_THREADS;
    W.nr = (nt + R - 1) / R;
    const size_t o_rs = 0, o_tc = o_rs + round256((size_t)W.nr * 16), o_rec = o_tc + round256((size_t)nt * 8),
                 o_dm = o_rec + round256((size_t)nt * sizeof(ClRec)), o_pre = o_dm + round256((size_t)nt * 8);
    const size_t o_cd = o_pre + round256((size_t)nt * 16);
    W.clear = o_tc;
    W.bytes = o_cd + round256((size_t)nt * CL_THREADS * 8);
    char *p = ws ? (char *)ws + HDR_BYTES : nullptr;
    W.rs = p ? (ulonglong2 *)(p + o_rs) : nullptr;
    W.tcnt = p ? (unsigned long long *)(p + o_tc) : nullptr;
    W.rec = p ? (ClRec *)(p + o_rec) : nullptr;
    W.dmin = p ? (unsigned long long *)(p + o_dm) : nullptr;
    W.pre = p ? (ulonglong2 *)(p + o_pre) : nullptr;
    W.codes = p ? (unsigned long long *)(p + o_cd) : nullptr;
    return W;
}

// Class codes of the thread's CL_PER elements from e0: four bits each, class + 1,
// or 0 for an element that is dropped or past n. `full`: all in range and every
// array 16-byte aligned. Four class bytes are clamped to v - 1 at once: with
// d = (c | 0x80 per byte) - (v - 1 per byte) (no borrow crosses a byte), byte i
// of (d | c) has its top bit set exactly when c_i >= v - 1.
// The filter over the thread's CL_PER keys from e0, as a 16-bit mask (positions
// at or past n are 0): one dispatch on the predicate kind for all of them.
template <typename KT>
__device__ __forceinline__ unsigned cl_kept16(const KT *__restrict__ keys, const DPred &filt, int64_t e0, int64_t n,
                                              bool full) {
    const unsigned valid = full || e0 + CL_PER <= n ? 0xffffu : (e0 >= n ? 0u : (1u << (unsigned)(n - e0)) - 1u);
    if (filt.kind == IXP_P_TRUE) return valid;
    if (filt.kind == IXP_P_FLAGS) {
        unsigned m = 0;
#pragma unroll
        for (int e = 0; e < CL_PER; e++) m |= (unsigned)(((valid >> e) & 1u) && __ldg(filt.flags + e0 + e) != 0) << e;
        return m;
    }
    KT kv[CL_PER];
#pragma unroll
    for (int g = 0; g < CL_PER / 4; g++) {
        KT k4[4];
        load_slot<KT, 4>(keys, e0 + 4 * g, n, full ? 1 : 0, k4);
#pragma unroll
        for (int k = 0; k < 4; k++) kv[4 * g + k] = k4[k];
    }
    unsigned m = 0;
    if (filt.kind == IXP_P_LT) {
        if (sizeof(KT) == 4) {
            if (filt.b > (long long)INT32_MAX) return valid;
            if (filt.b <= (long long)INT32_MIN) return 0u;
            const int32_t b = (int32_t)filt.b;
#pragma unroll
            for (int e = 0; e < CL_PER; e++) m |= (unsigned)((int32_t)kv[e] < b) << e;
        } else {
#pragma unroll
            for (int e = 0; e < CL_PER; e++) m |= (unsigned)((int64_t)kv[e] < filt.b) << e;
        }
        return m & valid;
    }
    // MOD_EQ (floored remainder in [0, a))
    if (filt.b < 0 || filt.b >= (long long)filt.a) return 0u;
#pragma unroll
    for (int e = 0; e < CL_PER; e++) {
        if (sizeof(KT) == 4) {
            int32_t r = (int32_t)kv[e] % filt.a;
            r += r < 0 ? filt.a : 0;
            m |= (unsigned)(r == (int32_t)filt.b) << e;
        } else {
            int64_t r = (int64_t)kv[e] % (int64_t)filt.a;
            r += r < 0 ? (int64_t)filt.a : 0;
            m |= (unsigned)(r == filt.b) << e;
        }
    }
    return m & valid;
}

template <typename KT>
__device__ __forceinline__ unsigned long long cl_codes16(const KT *__restrict__ keys, const uint8_t *__restrict__ cls,
                                                         const DPred &filt, int v, int64_t e0, int64_t n, bool full) {
    unsigned cw[4];
    if (full) {
        const uint4 c4 = __ldcs(reinterpret_cast<const uint4 *>(cls + e0));
        cw[0] = c4.x;
        cw[1] = c4.y;
        cw[2] = c4.z;
        cw[3] = c4.w;
    } else {
#pragma unroll
        for (int g = 0; g < 4; g++) {
            cw[g] = 0u;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (e0 + 4 * g + k < n) cw[g] |= (unsigned)cls[e0 + 4 * g + k] << (8 * k);
        }
    }
    const unsigned kept = cl_kept16<KT>(keys, filt, e0, n, full);
    const unsigned top4 = (unsigned)(v - 1) * 0x01010101u;
    unsigned long long codes = 0;
#pragma unroll
    for (int g = 0; g < 4; g++) {
        const unsigned kept4 = (kept >> (4 * g)) & 15u;
        const unsigned c = cw[g];
        const unsigned ge = (((c | 0x80808080u) - top4) | c) & 0x80808080u;
        const unsigned gm = (ge >> 7) * 0xffu;                              // 0xff where c_i >= v - 1
        const unsigned km = ((kept4 * 0x204081u) & 0x01010101u) * 0xffu;    // 0xff where kept
        const unsigned b = (((c & ~gm) | (top4 & gm)) + 0x01010101u) & km;  // class + 1, or 0
        const unsigned x = b | (b >> 4);
        codes |= (unsigned long long)((x & 0xffu) | ((x >> 8) & 0xff00u)) << (16 * g);
    }
    return codes;
}

// Class counts of 16 codes (four-bit fields equal to k + 1), as lo = c0 | c1 << 16
// and hi = c2 | c3 << 16; eq[k] gets bit 4e set when element e has class k.
__device__ __forceinline__ void cl_count_codes(unsigned long long codes, unsigned &lo, unsigned &hi,
                                               unsigned long long (&eq)[4]) {
    constexpr unsigned long long ONES = 0x1111111111111111ull;
    unsigned c[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const unsigned long long t = codes ^ (ONES * (unsigned long long)(k + 1));  // zero nibble: class k
        unsigned long long u = t | (t >> 1);
        u |= u >> 2;  // bit 0 of each nibble: the OR of its four bits
        eq[k] = ~u & ONES;
        c[k] = (unsigned)__popcll(eq[k]);
    }
    lo = c[0] | (c[1] << 16);
    hi = c[2] | (c[3] << 16);
}
__device__ __forceinline__ void cl_count_codes(unsigned long long codes, unsigned &lo, unsigned &hi) {
    unsigned long long eq[4];
    cl_count_codes(codes, lo, hi, eq);
}

// In-thread class ranks: nibble e of the result is the number of elements before e
// in the thread with e's class (0 for a dropped element). eq[k] * 0x1111...10
// puts in nibble e the count of class-k elements before e (at most 15, so no
// nibble carries), and eq[k] * 15 masks it to the class-k positions.
template <int VS>
__device__ __forceinline__ unsigned long long cl_ranks16(const unsigned long long (&eq)[4]) {
    unsigned long long x = 0;
#pragma unroll
    for (int k = 0; k < VS; k++) x |= (eq[k] * 0x1111111111111110ull) & (eq[k] * 0xfull);
    return x;
}

// Exclusive block scan of the threads' packed class counts (16-bit fields; a tile
// has at most CL_TILE elements of a class); the tile totals go to tlo / thi.
__device__ __forceinline__ void cl_block_scan16(unsigned &lo, unsigned &hi, uint2 *s_w, unsigned &tlo,
                                                unsigned &thi) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned ylo = lo, yhi = hi;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned a = __shfl_up_sync(FULL, ylo, d), b = __shfl_up_sync(FULL, yhi, d);
        if (l >= d) {
            ylo += a;
            yhi += b;
        }
    }
    if (l == 31) s_w[w] = make_uint2(ylo, yhi);
    __syncthreads();
    unsigned plo = 0, phi = 0;
    tlo = 0;
    thi = 0;
#pragma unroll
    for (int i = 0; i < CL_WARPS; i++) {
        const uint2 s = s_w[i];
        plo += i < w ? s.x : 0u;
        phi += i < w ? s.y : 0u;
        tlo += s.x;
        thi += s.y;
    }
    lo = plo + ylo - lo;
    hi = phi + yhi - hi;
}

// Widens 16-bit packed tile counts (c0 | c1 << 16 | c2 << 32 | c3 << 48) to two
// words of 32-bit fields.
__device__ __forceinline__ ulonglong2 cl_widen(unsigned long long c) {
    return make_ulonglong2((c & 0xffffull) | (((c >> 16) & 0xffffull) << 32),
                           ((c >> 32) & 0xffffull) | ((c >> 48) << 32));
}

__device__ __forceinline__ void cl_add_range(ulonglong2 *rs, unsigned long long tc) {
    const ulonglong2 w = cl_widen(tc);
    if (w.x) atomicAdd(&rs->x, w.x);
    if (w.y) atomicAdd(&rs->y, w.y);
}

template <typename ZT>
__device__ __forceinline__ void cl_load_z16(const ZT *__restrict__ z, int64_t e0, int64_t n, bool full,
                                            ZT (&zz)[CL_PER]) {
    if (full) {
        if constexpr (sizeof(ZT) == 4) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int4 q = __ldcs(reinterpret_cast<const int4 *>(z + e0) + u);
                zz[4 * u] = q.x;
                zz[4 * u + 1] = q.y;
                zz[4 * u + 2] = q.z;
                zz[4 * u + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const longlong2 q = __ldcs(reinterpret_cast<const longlong2 *>(z + e0) + u);
                zz[2 * u] = q.x;
                zz[2 * u + 1] = q.y;
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < CL_PER; e++) zz[e] = e0 + e < n ? z[e0 + e] : (ZT)-1;  // -1: never inside [0, N)
    }
}

template <typename T>
__device__ __forceinline__ T cl_warp_min(T x) {
    if constexpr (sizeof(T) == 4) {
        return __reduce_min_sync(FULL, x);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T y = __shfl_xor_sync(FULL, x, o);
            x = y < x ? y : x;
        }
        return x;
    }
}
template <typename T>
__device__ __forceinline__ T cl_warp_max(T x) {
    if constexpr (sizeof(T) == 4) {
        return __reduce_max_sync(FULL, x);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T y = __shfl_xor_sync(FULL, x, o);
            x = y > x ? y : x;
        }
        return x;
    }
}

// Check, tile pass. QT is the type Z - rank is taken in: int32 (modulo 2^32) when Z
// is int32 and n <= INT32_MAX, since then Z and every expected destination lie in
// the int32 range and Z - rank equals a destination's constant modulo 2^32 only
// when Z is that destination; int64 otherwise (modulo 2^64, the same argument).
// VS: classes handled (v <= VS).
//
// The tile's class-k constant C_k is the Z of its first class-k element (tile rank
// 0), read back by the one thread that holds it and shared through shared memory;
// then an element's expected Z is C_k + its tile rank: the thread's first rank
// for the class (block scan), looked up by class in a per-thread row of shared
// memory, plus its in-thread class rank (cl_ranks16). Any mismatch marks the tile
// as failing; otherwise C_k is recorded for the decide pass.
template <typename KT, typename ZT, typename QT, int VS>
__global__ void __launch_bounds__(CL_THREADS, sizeof(ZT) == 4 ? 4 : 3) cl_tile_kernel(const ZT *__restrict__ z, const KT *__restrict__ keys,
                                                             const uint8_t *__restrict__ cls, int64_t n, DPred filt,
                                                             int v, int vec_ok, int64_t R,
                                                             unsigned long long *__restrict__ tcnt,
                                                             ClRec *__restrict__ rec,
                                                             unsigned long long *__restrict__ dmin,
                                                             ulonglong2 *__restrict__ rs) {
    IXP_KERNEL_ENTRY();
    using UQ = typename std::make_unsigned<QT>::type;
    __shared__ uint2 s_w[CL_WARPS];
    __shared__ UQ s_c[VS];
    __shared__ UQ s_dm[CL_WARPS];
    __shared__ unsigned s_bad;
    __shared__ UQ s_e[VS + 1][CL_THREADS];  // row q: expected Z of the thread's first class-(q - 1) element
    const int64_t t = blockIdx.x;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t e0 = t * CL_TILE + (int64_t)threadIdx.x * CL_PER;
    const bool full = vec_ok && e0 + CL_PER <= n;
    if (threadIdx.x == 0) s_bad = 0u;
    const unsigned long long codes = cl_codes16<KT>(keys, cls, filt, v, e0, n, full);
    ZT zz[CL_PER];
    cl_load_z16<ZT>(z, e0, n, full, zz);
    unsigned lo, hi, tlo, thi;
    unsigned long long eq[4];
    cl_count_codes(codes, lo, hi, eq);
    const unsigned has = (lo & 0xffffu ? 1u : 0u) | (lo >> 16 ? 2u : 0u) | (hi & 0xffffu ? 4u : 0u) | (hi >> 16 ? 8u : 0u);
    cl_block_scan16(lo, hi, s_w, tlo, thi);
    const unsigned rk[4] = {lo & 0xffffu, lo >> 16, hi & 0xffffu, hi >> 16};  // tile rank of the first one
#pragma unroll
    for (int k = 0; k < VS; k++)
        if (((has >> k) & 1u) && rk[k] == 0u) {  // this thread holds the tile's first class-k element
            const int f = (__ffsll((long long)eq[k]) - 1) >> 2;
            s_c[k] = (UQ)(QT)z[e0 + f];
        }
    const unsigned long long xr = cl_ranks16<VS>(eq);
    __syncthreads();
    s_e[0][threadIdx.x] = 0;
#pragma unroll
    for (int k = 0; k < VS; k++) s_e[k + 1][threadIdx.x] = s_c[k] + (UQ)rk[k];
    bool bad = false;
    UQ dm = (UQ)~(UQ)0;
#pragma unroll
    for (int e = 0; e < CL_PER; e++) {
        const unsigned q = (unsigned)(codes >> (4 * e)) & 15u;
        const UQ zv = (UQ)(QT)zz[e];
        const UQ want = s_e[q][threadIdx.x] + (UQ)((xr >> (4 * e)) & 15u);
        bad |= q != 0u && want != zv;
        dm = q == 0u && zv < dm ? zv : dm;
    }
    dm = cl_warp_min<UQ>(dm);
    if (__any_sync(FULL, bad) && l == 0) s_bad = 1u;
    if (l == 0) s_dm[w] = dm;
    const unsigned thas = __reduce_or_sync(FULL, has);
    __shared__ unsigned s_has[CL_WARPS];
    if (l == 0) s_has[w] = thas;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned all = 0;
        for (int i = 0; i < CL_WARPS; i++) all |= s_has[i];
        ClRec out;
#pragma unroll
        for (int k = 0; k < 4; k++) out.c[k] = CL_NONE;
#pragma unroll
        for (int k = 0; k < VS; k++) {
            // a negative constant is never a destination
            const QT c = (QT)s_c[k];
            if ((all >> k) & 1u) out.c[k] = c >= 0 && !s_bad ? (long long)c : CL_BAD;
        }
        UQ m = s_dm[0];
        for (int i = 1; i < CL_WARPS; i++) m = s_dm[i] < m ? s_dm[i] : m;
        const unsigned long long tc = (unsigned long long)tlo | ((unsigned long long)thi << 32);
        tcnt[t] = tc;
        rec[t] = out;
        dmin[t] = (unsigned long long)m;
        cl_add_range(rs + t / R, tc);
    }
}

// Forward, pass 1: the tile's class counts (and its range's), and every thread's
// class codes for the write pass (half a byte per element instead of the keys and
// classes again).
template <typename KT>
__global__ void __launch_bounds__(CL_THREADS) cl_tile_count_kernel(const KT *__restrict__ keys,
                                                                   const uint8_t *__restrict__ cls, int64_t n,
                                                                   DPred filt, int v, int vec_ok, int64_t R,
                                                                   unsigned long long *__restrict__ tcnt,
                                                                   ulonglong2 *__restrict__ rs,
                                                                   unsigned long long *__restrict__ codes_out) {
    IXP_KERNEL_ENTRY();
    __shared__ uint2 s_w[CL_WARPS];
    const int64_t t = blockIdx.x;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t e0 = t * CL_TILE + (int64_t)threadIdx.x * CL_PER;
    const unsigned long long codes = cl_codes16<KT>(keys, cls, filt, v, e0, n, vec_ok && e0 + CL_PER <= n);
    __stcs(codes_out + t * CL_THREADS + threadIdx.x, codes);
    unsigned lo, hi;
    cl_count_codes(codes, lo, hi);
    lo = __reduce_add_sync(FULL, lo);  // at most 512 per field
    hi = __reduce_add_sync(FULL, hi);
    if (l == 0) s_w[w] = make_uint2(lo, hi);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned a = 0, b = 0;
        for (int i = 0; i < CL_WARPS; i++) {
            a += s_w[i].x;
            b += s_w[i].y;
        }
        const unsigned long long tc = (unsigned long long)a | ((unsigned long long)b << 32);
        tcnt[t] = tc;
        cl_add_range(rs + t / R, tc);
    }
}

// Block sum of two words (every thread gets it).
__device__ __forceinline__ ulonglong2 cl_block_sum2(ulonglong2 x, ulonglong2 *s) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    x.x = warp_sum_u64(x.x);
    x.y = warp_sum_u64(x.y);
    __syncthreads();
    if (l == 0) s[w] = x;
    __syncthreads();
    ulonglong2 r = make_ulonglong2(0ull, 0ull);
#pragma unroll
    for (int i = 0; i < CL_WARPS; i++) {
        r.x += s[i].x;
        r.y += s[i].y;
    }
    return r;
}

// Class bases (32-bit fields, classes 0 | 1 and 2 | 3) from the class totals, and N.
__device__ __forceinline__ ulonglong2 cl_bases(ulonglong2 tot, unsigned long long &N) {
    const unsigned long long t0 = tot.x & 0xffffffffull, t1 = tot.x >> 32;
    const unsigned long long t2 = tot.y & 0xffffffffull, t3 = tot.y >> 32;
    N = t0 + t1 + t2 + t3;
    return make_ulonglong2(0ull | (t0 << 32), (t0 + t1) | ((t0 + t1 + t2) << 32));
}

// Decide (check) or prefix (forward) pass: block b takes range b of R = tpt *
// CL_THREADS tiles, thread j its tiles b * R + j * tpt .. + tpt - 1. The class
// prefix at the range's start comes from the range counters; each tile's first
// destination per class is base_k + that prefix + the block's exclusive scan. With
// rec, a tile whose constants or dropped Z disagree raises the first-failing-tile
// slot; with pre, the first destinations are stored for the write pass. Block 0
// stores N.
__global__ void __launch_bounds__(CL_THREADS) cl_decide_kernel(const unsigned long long *__restrict__ tcnt,
                                                               const ClRec *__restrict__ rec,
                                                               const unsigned long long *__restrict__ dmin,
                                                               const ulonglong2 *__restrict__ rs, int64_t nt, int tpt,
                                                               int64_t nr, Hdr *h, ulonglong2 *__restrict__ pre) {
    IXP_KERNEL_ENTRY();
    __shared__ ulonglong2 s_a[CL_WARPS], s_t[CL_WARPS], s_x[CL_WARPS];
    const int64_t b = blockIdx.x;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    ulonglong2 a = make_ulonglong2(0ull, 0ull), s = a;
    for (int64_t j = threadIdx.x; j < nr; j += CL_THREADS) {
        const ulonglong2 x = rs[j];
        s.x += x.x;
        s.y += x.y;
        if (j < b) {
            a.x += x.x;
            a.y += x.y;
        }
    }
    a = cl_block_sum2(a, s_a);
    s = cl_block_sum2(s, s_t);
    unsigned long long N;
    const ulonglong2 base = cl_bases(s, N);
    if (b == 0 && threadIdx.x == 0) h->total = N << 32;
    const int64_t t1 = b * (int64_t)tpt * CL_THREADS + (int64_t)threadIdx.x * tpt;
    ulonglong2 mine = make_ulonglong2(0ull, 0ull);
    for (int u = 0; u < tpt; u++)
        if (t1 + u < nt) {
            const ulonglong2 c = cl_widen(tcnt[t1 + u]);
            mine.x += c.x;
            mine.y += c.y;
        }
    // exclusive scan of the threads' sums (fields stay below 2^32: no carries)
    ulonglong2 y = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long p = __shfl_up_sync(FULL, y.x, d), q = __shfl_up_sync(FULL, y.y, d);
        if (l >= d) {
            y.x += p;
            y.y += q;
        }
    }
    if (l == 31) s_x[w] = y;
    __syncthreads();
    ulonglong2 P = make_ulonglong2(base.x + a.x + y.x - mine.x, base.y + a.y + y.y - mine.y);
    for (int i = 0; i < w; i++) {
        P.x += s_x[i].x;
        P.y += s_x[i].y;
    }
    for (int u = 0; u < tpt; u++) {
        const int64_t t = t1 + u;
        if (t >= nt) break;
        if (pre) pre[t] = P;
        if (rec) {
            const ClRec r = rec[t];
            const long long want[4] = {(long long)(P.x & 0xffffffffull), (long long)(P.x >> 32),
                                       (long long)(P.y & 0xffffffffull), (long long)(P.y >> 32)};
            bool bad = dmin[t] < N;
#pragma unroll
            for (int k = 0; k < 4; k++) bad |= r.c[k] != CL_NONE && r.c[k] != want[k];
            if (bad) atomicMax(&h->k_first2, ~(unsigned long long)t);
        }
        const ulonglong2 c = cl_widen(tcnt[t]);
        P.x += c.x;
        P.y += c.y;
    }
}

// Check, exact pass over the first failing tile (one block; nothing to do when no
// tile failed): every element's destination from the class prefix at the tile, and
// the first wrong one reported.
template <typename KT, typename ZT>
__global__ void __launch_bounds__(CL_THREADS) cl_exact_kernel(const ZT *__restrict__ z, const KT *__restrict__ keys,
                                                              const uint8_t *__restrict__ cls, int64_t n, DPred filt,
                                                              int v, int vec_ok,
                                                              const unsigned long long *__restrict__ tcnt,
                                                              const ulonglong2 *__restrict__ rs, int tpt, int64_t nr,
                                                              Hdr *h) {
    IXP_KERNEL_ENTRY();
    __shared__ ulonglong2 s_a[CL_WARPS], s_t[CL_WARPS];
    __shared__ uint2 s_w[CL_WARPS];
    if (h->k_first2 == 0) return;
    const int64_t t = (int64_t)~h->k_first2;
    const int64_t R = (int64_t)tpt * CL_THREADS, rb = t / R;
    ulonglong2 a = make_ulonglong2(0ull, 0ull), s = a;
    for (int64_t j = threadIdx.x; j < nr; j += CL_THREADS) {
        const ulonglong2 x = rs[j];
        s.x += x.x;
        s.y += x.y;
        if (j < rb) {
            a.x += x.x;
            a.y += x.y;
        }
    }
    for (int64_t j = rb * R + threadIdx.x; j < t; j += CL_THREADS) {
        const ulonglong2 c = cl_widen(tcnt[j]);
        a.x += c.x;
        a.y += c.y;
    }
    a = cl_block_sum2(a, s_a);
    s = cl_block_sum2(s, s_t);
    unsigned long long N;
    const ulonglong2 base = cl_bases(s, N);
    const unsigned long long P0 = base.x + a.x, P1 = base.y + a.y;
    const int64_t e0 = t * CL_TILE + (int64_t)threadIdx.x * CL_PER;
    const bool full = vec_ok && e0 + CL_PER <= n;
    const unsigned long long codes = cl_codes16<KT>(keys, cls, filt, v, e0, n, full);
    ZT zz[CL_PER];
    cl_load_z16<ZT>(z, e0, n, full, zz);
    unsigned lo, hi, tlo, thi;
    cl_count_codes(codes, lo, hi);
    cl_block_scan16(lo, hi, s_w, tlo, thi);
    int64_t r[4] = {(int64_t)(P0 & 0xffffffffull) + (lo & 0xffffu), (int64_t)(P0 >> 32) + (lo >> 16),
                    (int64_t)(P1 & 0xffffffffull) + (hi & 0xffffu), (int64_t)(P1 >> 32) + (hi >> 16)};
    for (int e = 0; e < CL_PER; e++) {
        const int64_t i = e0 + e;
        if (i >= n) break;
        const unsigned q = (unsigned)(codes >> (4 * e)) & 15u;
        const int64_t zi = (int64_t)zz[e];
        int64_t ref = -1;
        if (q) ref = r[q - 1]++;
        const bool wrong = q ? zi != ref : (zi >= 0 && zi < (int64_t)N);
        if (wrong) {
            cl_report(h, i, ref);
            break;
        }
    }
}

// Forward, write pass, from the class codes of pass 1: each element's destination
// (-1 for a dropped one) is its class's first destination in the thread (tile
// prefix + block scan, looked up by class in a per-thread row of shared memory)
// plus its in-thread class rank; 16-byte streaming stores.
template <typename OT, int VS>
__global__ void __launch_bounds__(CL_THREADS) cl_write_kernel(const unsigned long long *__restrict__ codes_in, int64_t n,
                                                              int vec_ok, const ulonglong2 *__restrict__ pre,
                                                              OT *__restrict__ dst) {
    IXP_KERNEL_ENTRY();
    using UT = typename std::make_unsigned<OT>::type;
    __shared__ uint2 s_w[CL_WARPS];
    __shared__ UT s_e[VS + 1][CL_THREADS];  // row q: first destination of class q - 1 in the thread; row 0: -1
    const int64_t t = blockIdx.x;
    const int64_t e0 = t * CL_TILE + (int64_t)threadIdx.x * CL_PER;
    const bool full = vec_ok && e0 + CL_PER <= n;
    const unsigned long long codes = __ldcs(codes_in + t * CL_THREADS + threadIdx.x);
    unsigned lo, hi, tlo, thi;
    unsigned long long eq[4];
    cl_count_codes(codes, lo, hi, eq);
    cl_block_scan16(lo, hi, s_w, tlo, thi);
    const ulonglong2 P = pre[t];
    const unsigned first[4] = {(unsigned)P.x + (lo & 0xffffu), (unsigned)(P.x >> 32) + (lo >> 16),
                               (unsigned)P.y + (hi & 0xffffu), (unsigned)(P.y >> 32) + (hi >> 16)};
    s_e[0][threadIdx.x] = (UT)~(UT)0;
#pragma unroll
    for (int k = 0; k < VS; k++) s_e[k + 1][threadIdx.x] = (UT)first[k];
    const unsigned long long xr = cl_ranks16<VS>(eq);
    OT o[CL_PER];
#pragma unroll
    for (int e = 0; e < CL_PER; e++) {
        const unsigned q = (unsigned)(codes >> (4 * e)) & 15u;
        o[e] = (OT)(s_e[q][threadIdx.x] + (UT)((xr >> (4 * e)) & 15u));  // dropped: -1 + 0
    }
    if (full) {
        if constexpr (sizeof(OT) == 4) {
#pragma unroll
            for (int u = 0; u < 4; u++)
                __stcs(reinterpret_cast<int4 *>(dst + e0) + u,
                       make_int4((int)o[4 * u], (int)o[4 * u + 1], (int)o[4 * u + 2], (int)o[4 * u + 3]));
        } else {
#pragma unroll
            for (int u = 0; u < 8; u++)
                __stcs(reinterpret_cast<longlong2 *>(dst + e0) + u,
                       make_longlong2((long long)o[2 * u], (long long)o[2 * u + 1]));
        }
    } else {
#pragma unroll
        for (int e = 0; e < CL_PER; e++)
            if (e0 + e < n) dst[e0 + e] = o[e];
    }
}

// ----------------------------------------------------------- flat: pass 2
// Block c: exclusive scan of class c's tile counts in place, total to tot[c].
__global__ void __launch_bounds__(1024) cl_class_scan_kernel(unsigned *__restrict__ cnt, int64_t nt,
                                                             unsigned long long *__restrict__ tot) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long s_w[32];
    unsigned *row = cnt + (int64_t)blockIdx.x * nt;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned long long carry = 0;
    for (int64_t base = 0; base < nt; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const unsigned long long x = t < nt ? row[t] : 0ull;
        unsigned long long y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        if (l == 31) s_w[w] = y;
        __syncthreads();
        unsigned long long wpre = 0, all = 0;
        for (int i = 0; i < 32; i++) {
            wpre += i < w ? s_w[i] : 0ull;
            all += s_w[i];
        }
        if (t < nt) row[t] = (unsigned)(carry + wpre + y - x);
        carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// Class bases (exclusive scan of the class totals) and N into the header.
__global__ void cl_base_kernel(const unsigned long long *__restrict__ tot, int v, unsigned long long *__restrict__ base,
                               Hdr *h) {
    IXP_KERNEL_ENTRY();
    if (threadIdx.x != 0) return;
    unsigned long long run = 0;
    for (int c = 0; c < v; c++) {
        base[c] = run;
        run += tot[c];
    }
    h->total = run << 32;  // N, where the verdict's finalize reads it
}

// Ranks of one 32-element round of a warp: for each lane, the number of lanes
// below it with the same class, and (through the warp's class counters s_wc) the
// elements of that class earlier in the warp's range.
__device__ __forceinline__ unsigned cl_round_rank(int c, unsigned *s_wc) {
    const int l = threadIdx.x & 31;
    const unsigned m = __match_any_sync(FULL, c);
    const unsigned below = __popc(m & ((1u << l) - 1u));
    unsigned r = 0;
    if (c >= 0) r = s_wc[c] + below;
    __syncwarp();
    if (c >= 0 && below == 0) s_wc[c] += __popc(m);
    __syncwarp();
    return r;
}

// The same with the warp's class counters in registers (v <= VS, uniform across
// the warp): one ballot per class replaces the match.
template <int VS>
__device__ __forceinline__ unsigned cl_round_rank_small(int c, unsigned (&wc)[VS]) {
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    unsigned r = 0;
#pragma unroll
    for (int k = 0; k < VS; k++) {
        const unsigned m = __ballot_sync(FULL, c == k);
        if (c == k) r = wc[k] + __popc(m & lt);
        wc[k] += __popc(m);
    }
    return r;
}

// ----------------------------------------------------------- flat: pass 3
// WRITE: store the destinations (-1 for dropped elements) to `dst` instead of
// comparing them with Z (the v-class filter-partition itself).
template <typename KT, typename ZT, bool WRITE, int VS>
__global__ void __launch_bounds__(CL_THREADS) cl_check_kernel(const ZT *__restrict__ z, const KT *__restrict__ keys,
                                                              const uint8_t *__restrict__ cls, int64_t n, DPred filt,
                                                              int v, int64_t nt, const unsigned *__restrict__ cnt,
                                                              const unsigned long long *__restrict__ base, Hdr *h,
                                                              ZT *__restrict__ dst) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned s_wc[CL_WARPS][CL_MAXV];
    __shared__ unsigned long long s_off[CL_MAXV];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int e = threadIdx.x; e < CL_WARPS * CL_MAXV; e += CL_THREADS) (&s_wc[0][0])[e] = 0u;
    for (int c = threadIdx.x; c < v; c += CL_THREADS) s_off[c] = base[c] + cnt[(int64_t)c * nt + blockIdx.x];
    __syncthreads();
    const int64_t t0 = blockIdx.x * (int64_t)CL_TILE + (int64_t)w * (CL_ROUNDS * 32);
    int cl[CL_ROUNDS];
    unsigned rk[CL_ROUNDS];
    if constexpr (VS > 0) {
        unsigned wc[VS];
#pragma unroll
        for (int k = 0; k < VS; k++) wc[k] = 0u;
#pragma unroll
        for (int r = 0; r < CL_ROUNDS; r++) {
            const int64_t i = t0 + r * 32 + l;
            cl[r] = i < n ? cl_class(keys, cls, filt, v, i) : -2;
            rk[r] = cl_round_rank_small<VS>(cl[r], wc);
        }
        if (l == 0)
#pragma unroll
            for (int k = 0; k < VS; k++)
                if (k < v) s_wc[w][k] = wc[k];
    } else {
#pragma unroll
        for (int r = 0; r < CL_ROUNDS; r++) {
            const int64_t i = t0 + r * 32 + l;
            cl[r] = i < n ? cl_class(keys, cls, filt, v, i) : -2;
            rk[r] = cl_round_rank(cl[r], s_wc[w]);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < v; c += CL_THREADS) {
        unsigned run = 0;
        for (int ww = 0; ww < CL_WARPS; ww++) {
            const unsigned x = s_wc[ww][c];
            s_wc[ww][c] = run;
            run += x;
        }
    }
    __syncthreads();
    const int64_t N = (int64_t)(h->total >> 32);
    int64_t bad = INT64_MAX, bref = 0;
#pragma unroll
    for (int r = 0; r < CL_ROUNDS; r++) {
        const int64_t i = t0 + r * 32 + l;
        if (i >= n) continue;
        const int c = cl[r];
        const int64_t ref = c >= 0 ? (int64_t)(s_off[c] + s_wc[w][c] + rk[r]) : -1;
        if (WRITE) {
            dst[i] = (ZT)ref;
            continue;
        }
        const int64_t zi = (int64_t)z[i];
        const bool wrong = c >= 0 ? zi != ref : (zi >= 0 && zi < N);
        if (wrong && i < bad) {
            bad = i;
            bref = ref;
        }
    }
    if (bad != INT64_MAX) cl_report(h, bad, bref);
}

// ----------------------------------------------------------- segmented
// Kept elements per segment (one block per claimed segment).
template <typename KT>
__global__ void __launch_bounds__(CL_THREADS) cl_seg_count_kernel(const KT *__restrict__ keys,
                                                                  const uint8_t *__restrict__ cls, int64_t n,
                                                                  DPred filt, int v, const int64_t *__restrict__ off,
                                                                  int64_t nseg, unsigned long long *__restrict__ kc) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long sm[CL_WARPS];
    for (int64_t k = blockIdx.x; k < nseg; k += gridDim.x) {
        int64_t a = __ldg(off + k), b = __ldg(off + k + 1);
        a = a < 0 ? 0 : (a > n ? n : a);
        b = b < a ? a : (b > n ? n : b);
        unsigned long long c = 0;
        for (int64_t i = a + threadIdx.x; i < b; i += CL_THREADS) c += cl_class(keys, cls, filt, v, i) >= 0;
        c = block_sum_u64(c, sm);
        if (threadIdx.x == 0) kc[k] = c;
    }
}

__global__ void __launch_bounds__(CL_G) cl_group_scan_kernel(unsigned long long *x, int64_t m,
                                                             unsigned long long *gtot) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long s_w[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t t = blockIdx.x * (int64_t)CL_G + threadIdx.x;
    const unsigned long long v = t < m ? x[t] : 0ull;
    unsigned long long y = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long o = __shfl_up_sync(FULL, y, d);
        if (l >= d) y += o;
    }
    if (l == 31) s_w[w] = y;
    __syncthreads();
    unsigned long long wpre = 0, all = 0;
    for (int i = 0; i < 32; i++) {
        wpre += i < w ? s_w[i] : 0ull;
        all += s_w[i];
    }
    if (t < m) x[t] = wpre + y - v;
    if (threadIdx.x == 0) gtot[blockIdx.x] = all;
}

__global__ void __launch_bounds__(CL_G) cl_group_add_kernel(unsigned long long *x, int64_t m,
                                                            const unsigned long long *__restrict__ gtot, Hdr *h) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long s_w[CL_G / 32];
    __shared__ unsigned long long s_pre;
    unsigned long long v = 0;
    for (int64_t g = threadIdx.x; g < (int64_t)blockIdx.x; g += CL_G) v += gtot[g];
    v = block_sum_u64(v, s_w);
    if (threadIdx.x == 0) s_pre = v;
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)CL_G + threadIdx.x;
    if (t < m) x[t] += s_pre;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) h->total = (s_pre + gtot[blockIdx.x]) << 32;
}

// One block per segment (claimed from h->tile_ctr): class histogram, class bases,
// then the comparison in chunks of CL_TILE with per-class counters carried over.
template <typename KT, typename ZT, bool WRITE>
__global__ void __launch_bounds__(CL_THREADS) cl_seg_check_kernel(const ZT *__restrict__ z,
                                                                  const KT *__restrict__ keys,
                                                                  const uint8_t *__restrict__ cls, int64_t n,
                                                                  DPred filt, int v, const int64_t *__restrict__ off,
                                                                  int64_t nseg,
                                                                  const unsigned long long *__restrict__ Fk, Hdr *h,
                                                                  ZT *__restrict__ dst) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned s_wc[CL_WARPS][CL_MAXV];
    __shared__ unsigned long long s_off[CL_MAXV];  // destination of the next element of each class
    __shared__ unsigned s_tot[CL_MAXV];
    __shared__ int64_t s_k;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t N = (int64_t)(h->total >> 32);
    int64_t bad = INT64_MAX, bref = 0;
    for (;;) {
        if (threadIdx.x == 0) s_k = (int64_t)atomicAdd(&h->tile_ctr, 1u);
        __syncthreads();
        const int64_t k = s_k;
        if (k >= nseg) break;
        int64_t a = __ldg(off + k), b = __ldg(off + k + 1);
        a = a < 0 ? 0 : (a > n ? n : a);
        b = b < a ? a : (b > n ? n : b);
        // class histogram of the segment
        for (int c = threadIdx.x; c < CL_MAXV; c += CL_THREADS) s_wc[0][c] = 0u;
        __syncthreads();
        for (int64_t i = a + threadIdx.x; i < b; i += CL_THREADS) {
            const int c = cl_class(keys, cls, filt, v, i);
            if (c >= 0) atomicAdd(&s_wc[0][c], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long run = Fk[k];
            for (int c = 0; c < v; c++) {
                const unsigned x = s_wc[0][c];
                s_off[c] = run;
                run += x;
            }
        }
        __syncthreads();
        for (int64_t c0 = a; c0 < b; c0 += CL_TILE) {
            for (int e = threadIdx.x; e < CL_WARPS * CL_MAXV; e += CL_THREADS) (&s_wc[0][0])[e] = 0u;
            __syncthreads();
            const int64_t t0 = c0 + (int64_t)w * (CL_ROUNDS * 32);
            int cl[CL_ROUNDS];
            unsigned rk[CL_ROUNDS];
#pragma unroll
            for (int r = 0; r < CL_ROUNDS; r++) {
                const int64_t i = t0 + r * 32 + l;
                cl[r] = i < b ? cl_class(keys, cls, filt, v, i) : -2;
                rk[r] = cl_round_rank(cl[r], s_wc[w]);
            }
            __syncthreads();
            for (int c = threadIdx.x; c < v; c += CL_THREADS) {  // exclusive prefix over the warps
                unsigned run = 0;
                for (int ww = 0; ww < CL_WARPS; ww++) {
                    const unsigned x = s_wc[ww][c];
                    s_wc[ww][c] = run;
                    run += x;
                }
                s_tot[c] = run;  // this chunk's count of class c
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < CL_ROUNDS; r++) {
                const int64_t i = t0 + r * 32 + l;
                if (i >= b) continue;
                const int c = cl[r];
                const int64_t ref = c >= 0 ? (int64_t)(s_off[c] + s_wc[w][c] + rk[r]) : -1;
                if (WRITE) {
                    dst[i] = (ZT)ref;
                    continue;
                }
                const int64_t zi = (int64_t)z[i];
                const bool wrong = c >= 0 ? zi != ref : (zi >= 0 && zi < N);
                if (wrong && i < bad) {
                    bad = i;
                    bref = ref;
                }
            }
            __syncthreads();
            for (int c = threadIdx.x; c < v; c += CL_THREADS) s_off[c] += s_tot[c];
            __syncthreads();
        }
    }
    if (bad != INT64_MAX) cl_report(h, bad, bref);
}

}  // namespace ixp

namespace ixp {

template <typename ZT>
__global__ void cl_finalize(const ZT *z, const Hdr *h, ixp_verdict *out) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    v.status = h->status;
    v.reserved = 0;
    const bool found = h->k_first != 0 && !v.status;
    const unsigned long long packed = ~h->k_first;
    const int64_t i = found ? (int64_t)(packed >> 32) : -1;
    v.ok = v.status ? -1 : (found ? 0 : 1);
    v.kind = found ? IXP_V_WRONG_DEST : IXP_V_NONE;
    v.index = i;
    v.value = found ? (int64_t)z[i] : 0;
    v.aux0 = (int64_t)(h->total >> 32);
    v.aux1 = found ? (int64_t)(packed & 0xffffffffull) - 1 : 0;
    *out = v;
}

__global__ void cl_kept_kernel(const Hdr *h, int64_t *kept) {
    IXP_KERNEL_ENTRY();
    *kept = (int64_t)(h->total >> 32);
}


size_t filtpart_classes_ws_bytes(int v, int64_t n, int64_t nseg) {
    if (v < 1) v = 1;
    if (n < 0) n = 0;
    const size_t nt = (size_t)((n + CL_TILE - 1) / CL_TILE);
    const size_t flat = v <= 4 ? cl16_ws(nullptr, n).bytes : round256(nt * (size_t)v * 4) + 2 * round256((size_t)v * 8);
    const size_t ns = (size_t)(nseg > 0 ? nseg : 0);
    const size_t seg = round256((ns + 1) * 8) + round256(((ns + CL_G - 1) / CL_G + 1) * 8);
    return HDR_BYTES + std::max(flat, seg);
}

// With `write`, stores the destinations to dst instead of checking z (out unused,
// N to *d_kept when given; dst may be null only when n == 0).
template <typename KT, typename ZT>
static int run_classes(const ZT *z, int64_t n, const KT *keys, ixp_pred filt, const uint8_t *cls, int v,
                       ixp_segs segs, ixp_verdict *out, void *ws, cudaStream_t st, bool write = false,
                       ZT *dst = nullptr, int64_t *d_kept = nullptr) {
    Hdr *h = (Hdr *)ws;
    char *p = (char *)ws + HDR_BYTES;
    if (cudaMemsetAsync(h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    const DPred f = dpred(filt);
    if (!segs.offsets) {
        const int64_t nt = (n + CL_TILE - 1) / CL_TILE;
        unsigned *cnt = (unsigned *)p;
        unsigned long long *tot = (unsigned long long *)(p + round256((size_t)nt * v * 4));
        unsigned long long *base = (unsigned long long *)((char *)tot + round256((size_t)v * 8));
        if (nt > 0) {
            const unsigned g = (unsigned)nt;
#define IXP_CL_PASSES(VS)                                                                                       \
    cl_count_kernel<KT, VS><<<g, CL_THREADS, 0, st>>>(keys, cls, n, f, v, nt, cnt);                             \
    cl_class_scan_kernel<<<(unsigned)v, 1024, 0, st>>>(cnt, nt, tot);                                           \
    cl_base_kernel<<<1, 32, 0, st>>>(tot, v, base, h);                                                          \
    if (write)                                                                                                  \
        cl_check_kernel<KT, ZT, true, VS><<<g, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, nt, cnt, base, h, dst); \
    else                                                                                                        \
        cl_check_kernel<KT, ZT, false, VS><<<g, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, nt, cnt, base, h, nullptr)
            const auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
            const int vec = (!keys || al16(keys)) && al16(cls) && (write ? (!dst || al16(dst)) : al16(z));
            if (v <= 4) {
                const Cl16Ws W = cl16_ws(ws, n);
                const int64_t R = (int64_t)W.tpt * CL_THREADS;
                const unsigned gr = (unsigned)W.nr;
                if (cudaMemsetAsync(W.rs, 0, W.clear, st) != cudaSuccess) return IXP_E_CUDA;
                if (write) {
                    cl_tile_count_kernel<KT><<<g, CL_THREADS, 0, st>>>(keys, cls, n, f, v, vec, R, W.tcnt, W.rs,
                                                                       W.codes);
                    cl_decide_kernel<<<gr, CL_THREADS, 0, st>>>(W.tcnt, nullptr, nullptr, W.rs, nt, W.tpt, W.nr, h,
                                                                W.pre);
                    const int dvec = !dst || (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
                    if (v <= 2)
                        cl_write_kernel<ZT, 2><<<g, CL_THREADS, 0, st>>>(W.codes, n, dvec, W.pre, dst);
                    else
                        cl_write_kernel<ZT, 4><<<g, CL_THREADS, 0, st>>>(W.codes, n, dvec, W.pre, dst);
                } else {
#define IXP_CL_TILE(QT, VS)                                                                                    \
    cl_tile_kernel<KT, ZT, QT, VS><<<g, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, vec, R, W.tcnt, W.rec, W.dmin, \
                                                             W.rs)
                    bool narrow = false;
                    if constexpr (sizeof(ZT) == 4) {
                        if (n <= INT32_MAX) {
                            narrow = true;
                            if (v <= 2)
                                IXP_CL_TILE(int32_t, 2);
                            else
                                IXP_CL_TILE(int32_t, 4);
                        }
                    }
                    if (!narrow) {
                        if (v <= 2)
                            IXP_CL_TILE(int64_t, 2);
                        else
                            IXP_CL_TILE(int64_t, 4);
                    }
#undef IXP_CL_TILE
                    cl_decide_kernel<<<gr, CL_THREADS, 0, st>>>(W.tcnt, W.rec, W.dmin, W.rs, nt, W.tpt, W.nr, h,
                                                                nullptr);
                    cl_exact_kernel<KT, ZT><<<1, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, vec, W.tcnt, W.rs,
                                                                      W.tpt, W.nr, h);
                }
            } else if (v <= 8) {
                IXP_CL_PASSES(8);
            } else {
                IXP_CL_PASSES(0);
            }
#undef IXP_CL_PASSES
        }
    } else {
        const int64_t m = segs.nseg;
        unsigned long long *kc = (unsigned long long *)p;
        unsigned long long *gtot = (unsigned long long *)(p + round256((size_t)(m + 1) * 8));
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(m, (int64_t)num_sms() * 8));
        cl_seg_count_kernel<KT><<<g, CL_THREADS, 0, st>>>(keys, cls, n, f, v, segs.offsets, m, kc);
        const unsigned ng = (unsigned)((m + CL_G - 1) / CL_G);
        cl_group_scan_kernel<<<ng, CL_G, 0, st>>>(kc, m, gtot);
        cl_group_add_kernel<<<ng, CL_G, 0, st>>>(kc, m, gtot, h);
        if (write)
            cl_seg_check_kernel<KT, ZT, true><<<g, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, segs.offsets, m, kc, h,
                                                                       dst);
        else
            cl_seg_check_kernel<KT, ZT, false><<<g, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, segs.offsets, m, kc,
                                                                        h, nullptr);
    }
    if (write) {
        if (d_kept) cl_kept_kernel<<<1, 1, 0, st>>>(h, d_kept);
    } else {
        cl_finalize<ZT><<<1, 1, 0, st>>>(z, h, out);
    }
    return launch_status();
}

}  // namespace ixp

using namespace ixp;

extern "C" int ixp_check_filtpart_classes(const void *z, int ztype, int64_t n, const void *keys, int ktype,
                                          ixp_pred filt, const uint8_t *cls, int32_t v, ixp_segs segs,
                                          ixp_verdict *d_verdict, void *ws, size_t ws_bytes, ixp_stream stream) {
    if ((ztype != IXP_I32 && ztype != IXP_I64) || (keys && ktype != IXP_I32 && ktype != IXP_I64)) return IXP_E_DTYPE;
    if (n < 0 || n >= (1ll << 32) || v < 1 || v > CL_MAXV || (n > 0 && (!z || !cls)) || !d_verdict)
        return IXP_E_INVAL;
    if (!pred_ok(filt, keys != nullptr || n == 0)) return IXP_E_INVAL;
    if ((segs.offsets && segs.nseg < 1) || (!segs.offsets && segs.nseg != 0)) return IXP_E_INVAL;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) ||
        ws_bytes < filtpart_classes_ws_bytes(v, n, segs.offsets ? segs.nseg : 0))
        return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const bool k64 = keys && ktype == IXP_I64;
#define IXP_CL(KT, ZT) run_classes<KT, ZT>((const ZT *)z, n, (const KT *)keys, filt, cls, v, segs, d_verdict, ws, st)
    if (!k64) return ztype == IXP_I32 ? IXP_CL(int32_t, int32_t) : IXP_CL(int32_t, int64_t);
    return ztype == IXP_I32 ? IXP_CL(int64_t, int32_t) : IXP_CL(int64_t, int64_t);
#undef IXP_CL
}

extern "C" int ixp_filtpart_classes(const void *keys, int ktype, int64_t n, ixp_pred filt, const uint8_t *cls,
                                    int32_t v, ixp_segs segs, void *out_idx, int out_type, int64_t *d_kept, void *ws,
                                    size_t ws_bytes, ixp_stream stream) {
    if ((out_type != IXP_I32 && out_type != IXP_I64) || (keys && ktype != IXP_I32 && ktype != IXP_I64))
        return IXP_E_DTYPE;
    if (n < 0 || n >= (1ll << 32) || v < 1 || v > CL_MAXV || (n > 0 && (!out_idx || !cls))) return IXP_E_INVAL;
    if (out_type == IXP_I32 && n > INT32_MAX) return IXP_E_INVAL;
    if (!pred_ok(filt, keys != nullptr || n == 0)) return IXP_E_INVAL;
    if ((segs.offsets && segs.nseg < 1) || (!segs.offsets && segs.nseg != 0)) return IXP_E_INVAL;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) ||
        ws_bytes < filtpart_classes_ws_bytes(v, n, segs.offsets ? segs.nseg : 0))
        return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const bool k64 = keys && ktype == IXP_I64;
#define IXP_CLW(KT, OT) \
    run_classes<KT, OT>(nullptr, n, (const KT *)keys, filt, cls, v, segs, nullptr, ws, st, true, (OT *)out_idx, d_kept)
    if (!k64) return out_type == IXP_I32 ? IXP_CLW(int32_t, int32_t) : IXP_CLW(int32_t, int64_t);
    return out_type == IXP_I32 ? IXP_CLW(int64_t, int32_t) : IXP_CLW(int64_t, int64_t);
#undef IXP_CLW
}

extern "C" unsigned long long ixp_tu_kernels_classes(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}
