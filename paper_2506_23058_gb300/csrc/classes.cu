// classes.cu - InvFiltPart with v classes (Sec. 2.3, FiltPart Y X (e_k, p^f, p^p_1..v)
// and its scatter-index form): per segment k, the elements kept by p^f are placed
// stably by class, class 0 first, after all kept elements of the segments before
// k. Element i's class is min(cls[i], v - 1); the last class collects everything
// the first v - 1 class predicates leave over.
//
// The destination of a kept element i of segment k and class h is
//     F_k + (kept elements of segment k with class < h) + (class-h elements of
//     segment k before i),
// and a dropped element's Z must lie outside [0, N). Flat arrays use three tiled
// passes (per-tile class histograms; a scan of each class over the tiles with the
// class bases; the comparison, where an element's rank inside its tile comes from
// the lanes of its warp with the same class and per-warp class counters).
// Segmented arrays give each segment to one block (claimed from a counter): its
// class histogram, the class bases, then the comparison chunk by chunk with class
// counters carried from chunk to chunk; F_k comes from a scan of the per-segment
// kept counts. The first wrong element and its expected destination are packed
// into one word (i << 32 | expected + 1) whose smallest value wins, so no
// separate witness pass is needed.
#include <algorithm>

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

// Classes of 4 consecutive elements at p0 (16-byte key loads, one 4-byte class
// load when aligned and in range), packed one byte each: class + 1, or 0 for an
// element that is dropped or past n.
template <typename KT>
__device__ __forceinline__ unsigned cl_load4(const KT *__restrict__ keys, const uint8_t *__restrict__ cls,
                                             const DPred &filt, int v, int64_t p0, int64_t n, int vec_ok) {
    KT kv[4];
    load_slot<KT, 4>(keys, p0, n, vec_ok, kv);
    const unsigned kept = pred_mask<KT, 4>(filt, kv, p0, n);
    unsigned cw;
    if (vec_ok && p0 + 4 <= n) {
        cw = __ldg(reinterpret_cast<const unsigned *>(cls + p0));
    } else {
        cw = 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (p0 + k < n) cw |= (unsigned)__ldg(cls + p0 + k) << (8 * k);
    }
    unsigned out = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int c = (int)((cw >> (8 * k)) & 0xffu);
        const unsigned cc = (unsigned)(c < v - 1 ? c : v - 1);
        if ((kept >> k) & 1u) out |= (cc + 1u) << (8 * k);
    }
    return out;
}

// Per class k < 4: how many of the 4 packed elements have class k, one byte per
// class (byte k of the result; at most 4 each).
__device__ __forceinline__ unsigned cl_onehot4(unsigned packed) {
    unsigned x = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const unsigned b = (packed >> (8 * e)) & 0xffu;
        x += b ? 1u << (8 * (b - 1u)) : 0u;
    }
    return x;
}

// Small v (v <= VS), pass 1: lanes take 4 consecutive elements; class counts are
// kept per lane and reduced over the warp at the end.
template <typename KT, int VS>
__global__ void __launch_bounds__(CL_THREADS) cl_count4_kernel(const KT *__restrict__ keys,
                                                               const uint8_t *__restrict__ cls, int64_t n,
                                                               DPred filt, int v, int64_t nt, int vec_ok,
                                                               unsigned *__restrict__ cnt) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned s_h[VS];
    if (threadIdx.x < VS) s_h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t t0 = blockIdx.x * (int64_t)CL_TILE;
    static_assert(VS <= 4 && CL_TILE / CL_THREADS <= 252, "byte-packed class counters");
    unsigned acc = 0;  // byte k: class-k elements of this lane (at most CL_TILE / CL_THREADS)
#pragma unroll
    for (int r = 0; r < CL_TILE / (4 * CL_THREADS); r++) {
        const int64_t p0 = t0 + ((int64_t)r * CL_THREADS + threadIdx.x) * 4;
        acc += cl_onehot4(cl_load4<KT>(keys, cls, filt, v, p0, n, vec_ok));
    }
#pragma unroll
    for (int k = 0; k < VS; k++) {
        const unsigned t = __reduce_add_sync(FULL, (acc >> (8 * k)) & 0xffu);
        if ((threadIdx.x & 31) == 0 && t) atomicAdd(&s_h[k], t);
    }
    __syncthreads();
    if (threadIdx.x < v && threadIdx.x < VS) cnt[(int64_t)threadIdx.x * nt + blockIdx.x] = s_h[threadIdx.x];
}

// Small v, pass 3: warp w takes 512 consecutive elements as 4 rounds of 128 (4 per
// lane). In a round, each class's lane counts are scanned across the warp; the
// warp's running class counts stay in registers; the warps' totals are scanned in
// shared memory; then each element's destination is its class offset in the tile
// plus the warp, lane and in-lane ranks.
template <typename KT, typename ZT, bool WRITE, int VS>
__global__ void __launch_bounds__(CL_THREADS, 4) cl_check4_kernel(const ZT *__restrict__ z, const KT *__restrict__ keys,
                                                               const uint8_t *__restrict__ cls, int64_t n,
                                                               DPred filt, int v, int64_t nt, int vec_ok,
                                                               const unsigned *__restrict__ cnt,
                                                               const unsigned long long *__restrict__ base, Hdr *h,
                                                               ZT *__restrict__ dst) {
    IXP_KERNEL_ENTRY();
    constexpr int R = CL_TILE / (4 * CL_THREADS);  // rounds of 4 elements per lane
    static_assert(VS <= 4, "byte-packed class counters");
    __shared__ unsigned s_rt[CL_WARPS][R];                   // byte k: class-k elements of the warp's round
    __shared__ unsigned long long s_base[CL_WARPS][R][VS];   // destination of the round's first class-k element
    __shared__ unsigned long long s_off[VS];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (threadIdx.x < VS) s_off[threadIdx.x] = threadIdx.x < v ? base[threadIdx.x] + cnt[(int64_t)threadIdx.x * nt + blockIdx.x] : 0ull;
    const int64_t wbase = blockIdx.x * (int64_t)CL_TILE + (int64_t)w * (R * 128);
    // per round: the lane's classes, and (one scan of the byte-packed counts, at
    // most 128 per class) the class counts of the lanes below it
    unsigned pk[R], lp[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t p0 = wbase + r * 128 + l * 4;
        pk[r] = cl_load4<KT>(keys, cls, filt, v, p0, n, vec_ok);
        const unsigned x = cl_onehot4(pk[r]);
        unsigned y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        lp[r] = y - x;
        if (l == 31) s_rt[w][r] = y;
    }
    __syncthreads();
    // class k's elements lie in (warp, round) order inside the tile
    if (threadIdx.x < VS) {
        const int k = threadIdx.x;
        unsigned long long run = s_off[k];
        for (int ww = 0; ww < CL_WARPS; ww++)
#pragma unroll
            for (int r = 0; r < R; r++) {
                s_base[ww][r][k] = run;
                run += (s_rt[ww][r] >> (8 * k)) & 0xffu;
            }
    }
    __syncthreads();
    const int64_t N = (int64_t)(h->total >> 32);
    int64_t bad = INT64_MAX, bref = 0;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int64_t p0 = wbase + r * 128 + l * 4;
        ZT zv[4];
        if (!WRITE) load_vec<ZT, 4>(z, p0, n, vec_ok, zv);
        unsigned seen = lp[r];  // byte k: class-k elements before the next one of this lane
        ZT out4[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const unsigned b = (pk[r] >> (8 * e)) & 0xffu;
            int64_t ref = -1;
            if (b) {
                const unsigned sh = 8 * (b - 1u);
                ref = (int64_t)(s_base[w][r][b - 1u] + ((seen >> sh) & 0xffu));
                seen += 1u << sh;
            }
            out4[e] = (ZT)ref;
            const int64_t i = p0 + e;
            if (!WRITE && i < n) {
                const int64_t zi = (int64_t)zv[e];
                const bool wrong = b ? zi != ref : (zi >= 0 && zi < N);
                if (wrong && i < bad) {
                    bad = i;
                    bref = ref;
                }
            }
        }
        if (WRITE) {
            if (vec_ok && p0 + 4 <= n) {
                if (sizeof(ZT) == 4) {
                    int4 q;
                    q.x = (int)out4[0];
                    q.y = (int)out4[1];
                    q.z = (int)out4[2];
                    q.w = (int)out4[3];
                    __stcs(reinterpret_cast<int4 *>(dst + p0), q);
                } else {
                    longlong2 a, c;
                    a.x = (long long)out4[0];
                    a.y = (long long)out4[1];
                    c.x = (long long)out4[2];
                    c.y = (long long)out4[3];
                    __stcs(reinterpret_cast<longlong2 *>(dst + p0), a);
                    __stcs(reinterpret_cast<longlong2 *>(dst + p0) + 1, c);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (p0 + e < n) dst[p0 + e] = out4[e];
            }
        }
    }
    if (bad != INT64_MAX) cl_report(h, bad, bref);
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
    const size_t flat = round256(nt * (size_t)v * 4) + 2 * round256((size_t)v * 8);
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
#define IXP_CL4_PASSES(VS)                                                                                      \
    cl_count4_kernel<KT, VS><<<g, CL_THREADS, 0, st>>>(keys, cls, n, f, v, nt, vec, cnt);                       \
    cl_class_scan_kernel<<<(unsigned)v, 1024, 0, st>>>(cnt, nt, tot);                                           \
    cl_base_kernel<<<1, 32, 0, st>>>(tot, v, base, h);                                                          \
    if (write)                                                                                                  \
        cl_check4_kernel<KT, ZT, true, VS><<<g, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, nt, vec, cnt, base, h, \
                                                                    dst);                                       \
    else                                                                                                        \
        cl_check4_kernel<KT, ZT, false, VS><<<g, CL_THREADS, 0, st>>>(z, keys, cls, n, f, v, nt, vec, cnt, base,  \
                                                                     h, nullptr)
            const auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
            const int vec = (!keys || al16(keys)) && (reinterpret_cast<uintptr_t>(cls) & 3u) == 0 &&
                            (write ? (!dst || al16(dst)) : al16(z));
            if (v <= 4) {
                IXP_CL4_PASSES(4);
            } else if (v <= 8) {
                IXP_CL_PASSES(8);
            } else {
                IXP_CL_PASSES(0);
            }
#undef IXP_CL_PASSES
#undef IXP_CL4_PASSES
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
