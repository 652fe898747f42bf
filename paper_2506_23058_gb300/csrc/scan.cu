// scan.cu - scan (Sec. 2.1), stable two-way partition (partition2, Fig. 2;
// partition2L, Sec. 6), the InvFiltPart check (Sec. 2.3, Fig. 5) and mkSgmDescr
// (Fig. 2, right).
//
// Tiles. A block of 256 threads owns one tile of 1024 16-byte vectors (4096 int32
// or 2048 int64 elements) in a warp-striped layout: warp w, sub-chunk u, lane l
// holds vector q = (4w + u) * 32 + l, so every load and store instruction of a warp
// touches 512 contiguous bytes.
//
// Single-pass scan. Tiles take ids from an atomic ticket (so a tile only waits on
// tiles that are already running), publish their aggregate, and warp 0 looks back
// over up to 32 predecessors at a time (decoupled look-back: Merrill & Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016). Segmented
// sums use the pair operator (f1, v1) + (f2, v2) = (f1 | f2, f2 ? v2 : v1 + v2) of
// the paper's sgmSum; a predecessor whose aggregate holds a segment head ends the
// look-back as an inclusive prefix would. Every wait is bounded.
//
// Partition / InvFiltPart. Pass 1 counts kept and kept-true elements per tile,
// turns the counts into exclusive tile prefixes with the same look-back, and
// records the prefix at every segment start. Pass 2 re-reads the tile, ranks each
// element inside the tile with warp scans, and writes destinations (partition) or
// compares them with Z (check). The design moves 20 bytes per element for a
// partition of int32 keys with a 4-byte payload (16 algorithmic), because the false
// elements' destinations need the total count of trues before anything is written.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "preds.cuh"
#include "lookback.cuh"
#include "tilescan.cuh"

namespace ixp {

constexpr int TB = 256;  // threads per tile
constexpr int SUB = 4;   // vectors per thread per tile

// The bounded-wait configuration every look-back and bulk-copy wait uses (set by
// ixp_debug_set_wait or IXP_DEBUG_SPIN_LIMIT); the protocol is in lookback.cuh.
Wait g_wait = {-1, -1};

Wait wait_config() {
    if (g_wait.spin_limit < 0) {
        const char *e = std::getenv("IXP_DEBUG_SPIN_LIMIT");
        long long v = e ? std::atoll(e) : 0;
        g_wait.spin_limit = v > 0 ? v : (1ll << 20);
    }
    return g_wait;
}

struct SP {
    unsigned f;
    unsigned long long v;
};
__device__ __forceinline__ SP sp_op(SP a, SP b) { return SP{a.f | b.f, b.f ? b.v : a.v + b.v}; }
__device__ __forceinline__ SP shfl_up_sp(SP a, int d) {
    return SP{__shfl_up_sync(FULL, a.f, d), __shfl_up_sync(FULL, a.v, d)};
}
__device__ __forceinline__ SP shfl_down_sp(SP a, int d) {
    return SP{__shfl_down_sync(FULL, a.f, d), __shfl_down_sync(FULL, a.v, d)};
}
__device__ __forceinline__ SP shfl_sp(SP a, int src) { return SP{__shfl_sync(FULL, a.f, src), __shfl_sync(FULL, a.v, src)}; }

// Called by all 32 lanes of one warp. Publishes `agg` for tile t, waits for the
// predecessors and returns the exclusive prefix of tile t (same value in every lane).
// Lane l reads tiles top - 4l - 0..3 (nearest first); the window is combined in
// order with the segmented-sum operator and the walk stops at the nearest tile
// whose inclusive prefix is known or whose aggregate holds a segment head.
__device__ SP lookback(const Lookback L, int64_t t, SP agg, Hdr *h, Wait wt) {
    const int lane = threadIdx.x & 31;
    const bool publish = t != wt.skip_tile;
    if (t == 0) {
        if (lane == 0 && publish) publish_status(L.st, agg.v, 2ull | ((unsigned long long)agg.f << 2));
        return SP{0u, 0ull};
    }
    if (lane == 0 && publish) publish_status(L.st + t, agg.v, 1ull | ((unsigned long long)agg.f << 2));
    SP excl{0u, 0ull};
    int64_t top = t - 1;
    long long spins = 0;
    bool gave_up = false;
    while (true) {
        ulonglong2 w[LB_PER_LANE];
#pragma unroll
        for (int q = 0; q < LB_PER_LANE; q++) {
            const int64_t j = top - (int64_t)lane * LB_PER_LANE - q;
            w[q] = j >= 0 ? read_status(L.st + j) : make_ulonglong2(0ull, 2ull);
        }
        while (true) {
            bool pending = false;
#pragma unroll
            for (int q = 0; q < LB_PER_LANE; q++) pending |= (w[q].y & 3ull) == 0ull;
            if (!__any_sync(FULL, pending)) break;
            if (++spins > wt.spin_limit) {
#pragma unroll
                for (int q = 0; q < LB_PER_LANE; q++)
                    if ((w[q].y & 3ull) == 0ull) {
                        w[q] = make_ulonglong2(0ull, 2ull);
                        gave_up = true;
                    }
                break;
            }
            if (spins > 16) __nanosleep(32);
#pragma unroll
            for (int q = 0; q < LB_PER_LANE; q++) {
                const int64_t j = top - (int64_t)lane * LB_PER_LANE - q;
                if ((w[q].y & 3ull) == 0ull) w[q] = read_status(L.st + j);
            }
        }
        // combine this lane's tiles (farthest first), cutting at the nearest stopper
        SP mine{0u, 0ull};
        bool stop_here = false;
#pragma unroll
        for (int q = 0; q < LB_PER_LANE; q++) {
            if (stop_here) continue;
            const bool stopper = (w[q].y & 3ull) == 2ull || (w[q].y & 4ull);
            SP e{stopper ? 1u : 0u, w[q].x};
            mine = sp_op(e, mine);  // tile q is earlier than tiles 0..q-1
            stop_here = stopper;
        }
        const unsigned stop = __ballot_sync(FULL, stop_here);
        const int L0 = stop ? __ffs(stop) - 1 : 32;
        if (lane > L0) mine = SP{0u, 0ull};
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            SP o = shfl_down_sp(mine, d);
            if (lane + d < 32) mine = sp_op(o, mine);
        }
        excl = sp_op(shfl_sp(mine, 0), excl);
        if (L0 < 32) break;
        top -= 32 * LB_PER_LANE;
    }
    if (gave_up && lane == 0) set_status(h, IXP_E_TIMEOUT);
    if (lane == 0 && publish) publish_status(L.st + t, sp_op(excl, agg).v, 2ull | ((unsigned long long)agg.f << 2));
    return excl;
}

// ------------------------------------------------------------ segment heads

__device__ __forceinline__ int64_t lb_off(const int64_t *off, int64_t nseg, int64_t key) {
    int64_t lo = 0, hi = nseg + 1;  // first k in [0, nseg] with off[k] >= key
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t seg_of(const int64_t *off, int64_t nseg, int64_t i) {
    int64_t lo = 0, hi = nseg;  // last k in [0, nseg) with off[k] <= i
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Mark positions off[k] in [t0, t1) in a shared bitmap of TILE bits.
template <int TILE>
__device__ __forceinline__ void mark_heads(unsigned *heads, const int64_t *off, int64_t nseg, int64_t t0, int64_t t1,
                                           int64_t *s_k) {
    for (int w = threadIdx.x; w < TILE / 32; w += blockDim.x) heads[w] = 0u;
    if (threadIdx.x == 0) *s_k = lb_off(off, nseg, t0);
    __syncthreads();
    for (int64_t k = *s_k + threadIdx.x; k < nseg; k += blockDim.x) {
        int64_t o = __ldg(off + k);
        if (o >= t1) break;
        if (o >= t0) atomicOr(&heads[(o - t0) >> 5], 1u << ((o - t0) & 31));
    }
    __syncthreads();
}

// ============================================================== scan kernel

template <typename TI, typename TO, bool SEG>
// SEG with `flags` set: a segment starts at every i with flags[i] != 0 (the flag
// form of sgmSum, Fig. 2) instead of at the offsets.
__global__ void __launch_bounds__(TB) scan_kernel(const TI *__restrict__ in, TO *__restrict__ out, int64_t n,
                                                  int inclusive, const int64_t *__restrict__ off, int64_t nseg,
                                                  Lookback L, Hdr *h, Wait wt, TO *total_out, int vec_ok,
                                                  const uint8_t *__restrict__ flags = nullptr) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(TI);
    constexpr int TILE = TB * SUB * V;
    __shared__ int64_t s_tile, s_k;
    __shared__ unsigned heads[SEG ? TILE / 32 : 1];
    __shared__ SP s_warp[TB / 32];
    if (threadIdx.x == 0) s_tile = atomicAdd(&h->tile_ctr, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    if (SEG && !flags) mark_heads<TILE>(heads, off, nseg, t0, t1, &s_k);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;

    unsigned long long a[SUB][V];
    unsigned hb[SUB];
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t q = (int64_t)((w * SUB + u) * 32 + l);
        const int64_t p0 = t0 + q * V;
        if (vec_ok && p0 + V <= n) {
            if (V == 4) {
                int4 v = __ldcs(reinterpret_cast<const int4 *>(in + p0));
                a[u][0] = (unsigned long long)(int64_t)v.x;
                a[u][1 % V] = (unsigned long long)(int64_t)v.y;
                a[u][2 % V] = (unsigned long long)(int64_t)v.z;
                a[u][3 % V] = (unsigned long long)(int64_t)v.w;
            } else {
                longlong2 v = __ldcs(reinterpret_cast<const longlong2 *>(in + p0));
                a[u][0] = (unsigned long long)v.x;
                a[u][1 % V] = (unsigned long long)v.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) a[u][k] = (p0 + k < n) ? (unsigned long long)(int64_t)in[p0 + k] : 0ull;
        }
        hb[u] = 0;
        if (SEG && flags) {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (p0 + k < n && __ldg(flags + p0 + k)) hb[u] |= 1u << k;
        } else if (SEG) {
#pragma unroll
            for (int k = 0; k < V; k++) {
                int r = (int)(q * V + k);
                if (heads[r >> 5] & (1u << (r & 31))) hb[u] |= 1u << k;
            }
        }
    }
    // warp-level scan, sub-chunk by sub-chunk
    SP carry{0u, 0ull};
    SP lane_pre[SUB];
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        SP x{0u, 0ull};
#pragma unroll
        for (int k = 0; k < V; k++) x = sp_op(x, SP{(hb[u] >> k) & 1u, a[u][k]});
        SP y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            SP o = shfl_up_sp(y, d);
            if (l >= d) y = sp_op(o, y);
        }
        SP ex = shfl_up_sp(y, 1);
        if (l == 0) ex = SP{0u, 0ull};
        lane_pre[u] = sp_op(carry, ex);
        carry = sp_op(carry, shfl_sp(y, 31));
    }
    if (l == 0) s_warp[w] = carry;
    __syncthreads();
    if (w == 0) {
        SP wt8 = l < TB / 32 ? s_warp[l] : SP{0u, 0ull};
        SP y = wt8;
#pragma unroll
        for (int d = 1; d < TB / 32; d <<= 1) {
            SP o = shfl_up_sp(y, d);
            if (l >= d) y = sp_op(o, y);
        }
        SP ex = shfl_up_sp(y, 1);
        if (l == 0) ex = SP{0u, 0ull};
        SP tile_agg = shfl_sp(y, TB / 32 - 1);
        SP tile_ex = lookback(L, t, tile_agg, h, wt);
        __syncwarp();
        if (l < TB / 32) s_warp[l] = sp_op(tile_ex, ex);
        if (l == 0 && total_out && t1 == n) *total_out = (TO)sp_op(tile_ex, tile_agg).v;
    }
    __syncthreads();
    const SP pre = s_warp[w];
    constexpr int VO = 16 / sizeof(TO);
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
        SP run = sp_op(pre, lane_pre[u]);
        TO o[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            run = sp_op(run, SP{(hb[u] >> k) & 1u, a[u][k]});
            o[k] = (TO)(inclusive ? run.v : run.v - a[u][k]);
        }
        if (vec_ok && p0 + V <= n) {
#pragma unroll
            for (int c = 0; c < V; c += VO) {
                if (VO == 4) {
                    int4 s;
                    s.x = (int)o[c];
                    s.y = (int)o[(c + 1) % V];
                    s.z = (int)o[(c + 2) % V];
                    s.w = (int)o[(c + 3) % V];
                    __stcs(reinterpret_cast<int4 *>(out + p0 + c), s);
                } else {
                    longlong2 s;
                    s.x = (long long)o[c];
                    s.y = (long long)o[(c + 1) % V];
                    __stcs(reinterpret_cast<longlong2 *>(out + p0 + c), s);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (p0 + k < n) out[p0 + k] = o[k];
        }
    }
}

// Flat scan: plain sums in the output width (32-bit accumulators for int32
// outputs), four 16-byte vectors per thread, at least four blocks per SM.
template <typename TI, typename TO, int NT = TB, int S = SUB, int MINB = 1024 / NT>
__global__ void __launch_bounds__(NT, MINB) scan_flat_kernel(const TI *__restrict__ in, TO *__restrict__ out,
                                                                  int64_t n, int inclusive, Lookback L, Hdr *h, Wait wt,
                                                                  TO *total_out, int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(TI);
    constexpr int TILE = NT * S * V;
    using ACC = typename std::conditional<sizeof(TO) == 4, uint32_t, unsigned long long>::type;
    __shared__ int64_t s_tile;
    __shared__ ACC s_warp[NT / 32];
    if (threadIdx.x == 0) s_tile = atomicAdd(&h->tile_ctr, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    const int64_t t0 = t * TILE;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    ACC a[S][V];
#pragma unroll
    for (int u = 0; u < S; u++) {
        const int64_t p0 = t0 + (int64_t)((w * S + u) * 32 + l) * V;
        if (vec_ok && p0 + V <= n) {
            if (V == 4) {
                int4 v = __ldcs(reinterpret_cast<const int4 *>(in + p0));
                a[u][0] = (ACC)(int64_t)v.x;
                a[u][1 % V] = (ACC)(int64_t)v.y;
                a[u][2 % V] = (ACC)(int64_t)v.z;
                a[u][3 % V] = (ACC)(int64_t)v.w;
            } else {
                longlong2 v = __ldcs(reinterpret_cast<const longlong2 *>(in + p0));
                a[u][0] = (ACC)v.x;
                a[u][1 % V] = (ACC)v.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) a[u][k] = (p0 + k < n) ? (ACC)(int64_t)in[p0 + k] : (ACC)0;
        }
    }
    ACC carry = 0, lane_pre[S];
#pragma unroll
    for (int u = 0; u < S; u++) {
        ACC x = 0;
#pragma unroll
        for (int k = 0; k < V; k++) x += a[u][k];
        ACC y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            ACC o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        lane_pre[u] = carry + y - x;
        carry += __shfl_sync(FULL, y, 31);
    }
    if (l == 0) s_warp[w] = carry;
    __syncthreads();
    if (w == 0) {
        const ACC x = l < NT / 32 ? s_warp[l] : (ACC)0;
        ACC y = x;
#pragma unroll
        for (int d = 1; d < NT / 32; d <<= 1) {
            ACC o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        const ACC tile_agg = __shfl_sync(FULL, y, NT / 32 - 1);
        const unsigned long long tile_ex = lookback_sum(L, t, (unsigned long long)tile_agg, h, wt);
        __syncwarp();
        if (l < NT / 32) s_warp[l] = (ACC)tile_ex + (y - x);
        if (l == 0 && total_out && t0 + TILE >= n) *total_out = (TO)(tile_ex + (unsigned long long)tile_agg);
    }
    __syncthreads();
    const ACC pre = s_warp[w];
    constexpr int VO = 16 / sizeof(TO);
#pragma unroll
    for (int u = 0; u < S; u++) {
        const int64_t p0 = t0 + (int64_t)((w * S + u) * 32 + l) * V;
        ACC run = pre + lane_pre[u];
        TO o[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            run += a[u][k];
            o[k] = (TO)(inclusive ? run : run - a[u][k]);
        }
        if (vec_ok && p0 + V <= n) {
#pragma unroll
            for (int c = 0; c < V; c += VO) {
                if (VO == 4) {
                    int4 st4;
                    st4.x = (int)o[c];
                    st4.y = (int)o[(c + 1) % V];
                    st4.z = (int)o[(c + 2) % V];
                    st4.w = (int)o[(c + 3) % V];
                    __stcs(reinterpret_cast<int4 *>(out + p0 + c), st4);
                } else {
                    longlong2 st2;
                    st2.x = (long long)o[c];
                    st2.y = (long long)o[(c + 1) % V];
                    __stcs(reinterpret_cast<longlong2 *>(out + p0 + c), st2);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (p0 + k < n) out[p0 + k] = o[k];
        }
    }
}

// Flat scan with the tile staged in shared memory by TMA bulk copies: thread 0
// takes the tile ticket and issues the copies (64 KB of input per tile), all
// threads wait on the mbarrier, then the tile is read twice from shared memory
// (sums, then outputs) so that few registers are live and three tiles fit per SM.
constexpr int TMA_NT = 256;
constexpr int TMA_TILE_BYTES = 65536;
constexpr int TMA_CHUNK = 16384;  // bytes per bulk copy

// Thread 0 takes the tile ticket and starts bulk copies of the tile's whole 16-byte
// chunks (of a TMA_TILE_BYTES tile) into buf; every thread returns with the tile
// index (cnt = elements in the tile, bulk = elements the copies bring; the rest
// are read from global memory). tma_wait_tile then waits for the copies (thread 0,
// bounded: IXP_E_TIMEOUT, after a second bounded wait for the copies in flight);
// a __syncthreads after it publishes the tile to the block.
template <typename TI, int TILE_BYTES = TMA_TILE_BYTES>
__device__ __forceinline__ int64_t tma_issue_tile(const TI *in, int64_t n, unsigned char *buf,
                                                  unsigned long long *bar, int64_t *s_tile, Hdr *h, int64_t &cnt,
                                                  int64_t &bulk) {
    constexpr int TILE = TILE_BYTES / (int)sizeof(TI);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *s_tile = atomicAdd(&h->tile_ctr, 1u);
    }
    __syncthreads();
    const int64_t t = *s_tile;
    const int64_t t0 = t * TILE;
    cnt = min((int64_t)TILE, n - t0);
    bulk = (cnt * (int64_t)sizeof(TI)) / 16 * 16 / (int64_t)sizeof(TI);
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)(bulk * sizeof(TI));
        mbar_expect_tx(bar, bytes);
        for (unsigned o = 0; o < bytes; o += TMA_CHUNK)
            bulk_g2s(buf + o, (const char *)(in + t0) + o, min((unsigned)TMA_CHUNK, bytes - o), bar);
    }
    return t;
}

__device__ __forceinline__ void tma_wait_tile(unsigned long long *bar, Hdr *h, Wait wt) {
    if (threadIdx.x == 0 && !mbar_wait_bounded(bar, 0, wt.spin_limit)) {
        set_status(h, IXP_E_TIMEOUT);
        mbar_wait_bounded(bar, 0, wt.spin_limit);  // let the copies land before the block moves on
    }
}

template <typename TI, int TILE_BYTES = TMA_TILE_BYTES>
__device__ __forceinline__ int64_t tma_stage_tile(const TI *in, int64_t n, unsigned char *buf,
                                                  unsigned long long *bar, int64_t *s_tile, Hdr *h, Wait wt,
                                                  int64_t &cnt, int64_t &bulk) {
    const int64_t t = tma_issue_tile<TI, TILE_BYTES>(in, n, buf, bar, s_tile, h, cnt, bulk);
    tma_wait_tile(bar, h, wt);
    __syncthreads();
    return t;
}

// The flat scan's tile: 72 KB (three blocks a SM fill 216 KB of shared memory);
// larger tiles amortise each tile's look-back (measured on 2^28 int32: 0.454 ms
// against 0.474 with 64 KB tiles and 0.51-0.58 with 16-32 KB tiles).
constexpr int SCAN_TILE_BYTES = 73728;

template <typename TI, typename TO>
__global__ void __launch_bounds__(TMA_NT, 3) scan_tma_kernel(const TI *__restrict__ in, TO *__restrict__ out,
                                                             int64_t n, int inclusive, Lookback L, Hdr *h, Wait wt,
                                                             TO *total_out) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(TI);
    constexpr int TILE = SCAN_TILE_BYTES / (int)sizeof(TI);
    constexpr int S = TILE / V / TMA_NT;  // vectors per thread
    using ACC = typename std::conditional<sizeof(TO) == 4, uint32_t, unsigned long long>::type;
    extern __shared__ __align__(128) unsigned char tma_buf[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int64_t s_tile;
    __shared__ ACC s_warp[TMA_NT / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int64_t cnt, bulk_elems;
    const int64_t t = tma_stage_tile<TI, SCAN_TILE_BYTES>(in, n, tma_buf, &bar, &s_tile, h, wt, cnt, bulk_elems);
    const int64_t t0 = t * TILE;
    const TI *sv = reinterpret_cast<const TI *>(tma_buf);
    auto elem = [&](int64_t r) -> ACC {  // element r of the tile
        if (r < bulk_elems) return (ACC)(int64_t)sv[r];
        return (r < cnt) ? (ACC)(int64_t)in[t0 + r] : (ACC)0;
    };
    // pass 1: per sub-chunk vector sums, warp scans with carry
    ACC carry = 0, lane_pre[S];
#pragma unroll
    for (int u = 0; u < S; u++) {
        const int64_t r0 = (int64_t)((w * S + u) * 32 + l) * V;
        ACC x = 0;
        if (r0 + V <= bulk_elems) {
            if (V == 4) {
                const int4 q = reinterpret_cast<const int4 *>(tma_buf)[r0 / 4];
                x = (ACC)(int64_t)q.x + (ACC)(int64_t)q.y + (ACC)(int64_t)q.z + (ACC)(int64_t)q.w;
            } else {
                const longlong2 q = reinterpret_cast<const longlong2 *>(tma_buf)[r0 / 2];
                x = (ACC)q.x + (ACC)q.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) x += elem(r0 + k);
        }
        ACC y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            ACC o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        lane_pre[u] = carry + y - x;
        carry += __shfl_sync(FULL, y, 31);
    }
    if (l == 0) s_warp[w] = carry;
    __syncthreads();
    if (w == 0) {
        const ACC x = l < TMA_NT / 32 ? s_warp[l] : (ACC)0;
        ACC y = x;
#pragma unroll
        for (int d = 1; d < TMA_NT / 32; d <<= 1) {
            ACC o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        const ACC tile_agg = __shfl_sync(FULL, y, TMA_NT / 32 - 1);
        const unsigned long long tile_ex = lookback_sum(L, t, (unsigned long long)tile_agg, h, wt);
        __syncwarp();
        if (l < TMA_NT / 32) s_warp[l] = (ACC)tile_ex + (y - x);
        if (l == 0 && total_out && t0 + TILE >= n) *total_out = (TO)(tile_ex + (unsigned long long)tile_agg);
    }
    __syncthreads();
    // pass 2: outputs
    const ACC pre = s_warp[w];
    constexpr int VO = 16 / sizeof(TO);
#pragma unroll
    for (int u = 0; u < S; u++) {
        const int64_t r0 = (int64_t)((w * S + u) * 32 + l) * V;
        ACC a[V];
        if (r0 + V <= bulk_elems) {
            if (V == 4) {
                const int4 q = reinterpret_cast<const int4 *>(tma_buf)[r0 / 4];
                a[0] = (ACC)(int64_t)q.x;
                a[1 % V] = (ACC)(int64_t)q.y;
                a[2 % V] = (ACC)(int64_t)q.z;
                a[3 % V] = (ACC)(int64_t)q.w;
            } else {
                const longlong2 q = reinterpret_cast<const longlong2 *>(tma_buf)[r0 / 2];
                a[0] = (ACC)q.x;
                a[1 % V] = (ACC)q.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) a[k] = elem(r0 + k);
        }
        ACC run = pre + lane_pre[u];
        TO o[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            run += a[k];
            o[k] = (TO)(inclusive ? run : run - a[k]);
        }
        const int64_t p0 = t0 + r0;
        if (p0 + V <= n) {
#pragma unroll
            for (int c = 0; c < V; c += VO) {
                if (VO == 4) {
                    int4 st4;
                    st4.x = (int)o[c];
                    st4.y = (int)o[(c + 1) % V];
                    st4.z = (int)o[(c + 2) % V];
                    st4.w = (int)o[(c + 3) % V];
                    __stcs(reinterpret_cast<int4 *>(out + p0 + c), st4);
                } else {
                    longlong2 st2;
                    st2.x = (long long)o[c];
                    st2.y = (long long)o[(c + 1) % V];
                    __stcs(reinterpret_cast<longlong2 *>(out + p0 + c), st2);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (p0 + k < n) out[p0 + k] = o[k];
        }
    }
}

// Segmented scan (sgmSum) with the tile staged as in scan_tma_kernel. The heads
// come from a uint8 flag array (FLAGS) or from the offsets; either way they are
// first marked in a shared bitmap of the tile. Inside a warp the segmented operator reduces to a plain scan: with x the
// lane's local aggregate (its vector's sum after the vector's last head), y the
// inclusive and e = y - x the exclusive plain scans over the lanes, and s the last
// lane below l whose vector holds a head (a ballot), the values since that head
// sum to e[l] - e[s]; with no such lane the warp's earlier carry applies.
template <typename TI, typename TO, bool FLAGS>
__global__ void __launch_bounds__(TMA_NT, sizeof(TO) == 4 ? 3 : 2) sgm_tma_kernel(const TI *__restrict__ in, TO *__restrict__ out,
                                                            int64_t n, int inclusive, const uint8_t *__restrict__ flags,
                                                            const int64_t *__restrict__ off, int64_t nseg, Lookback L,
                                                            Hdr *h, Wait wt) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(TI);
    constexpr int TILE = TMA_TILE_BYTES / (int)sizeof(TI);
    constexpr int S = TILE / V / TMA_NT;  // vectors per thread
    static_assert(S * V <= 64 && S <= 32, "head bits per thread");
    using ACC = typename std::conditional<sizeof(TO) == 4, uint32_t, unsigned long long>::type;
    extern __shared__ __align__(128) unsigned char tma_buf[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int64_t s_tile, s_k;
    __shared__ unsigned heads[TILE / 32];
    __shared__ ACC s_wv[TMA_NT / 32];
    __shared__ unsigned s_wf[TMA_NT / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int64_t cnt, bulk_elems;
    const int64_t t = tma_issue_tile(in, n, tma_buf, &bar, &s_tile, h, cnt, bulk_elems);
    const int64_t t0 = t * TILE;
    // the heads are read while the tile's copies are in flight
    if (FLAGS) {
        // 16 flags per 16-byte chunk become 16 head bits (a byte compare, then a
        // multiply that gathers the four low bits of a word); lane pairs fill one word
        constexpr int FC = TILE / 16 / TMA_NT;  // chunks per thread
        const bool f16 = (reinterpret_cast<uintptr_t>(flags) & 15) == 0;
        uint4 fq[FC];
#pragma unroll
        for (int i = 0; i < FC; i++) {
            const int64_t p = t0 + 16 * (int64_t)(threadIdx.x + i * TMA_NT);
            fq[i] = (f16 && p + 16 <= n) ? __ldcs(reinterpret_cast<const uint4 *>(flags + p)) : make_uint4(0, 0, 0, 0);
        }
        tma_wait_tile(&bar, h, wt);
#pragma unroll
        for (int i = 0; i < FC; i++) {
            const int c = threadIdx.x + i * TMA_NT;
            const int64_t p = t0 + 16 * (int64_t)c;
            unsigned bits = 0;
            if (f16 && p + 16 <= n) {
                const unsigned wd[4] = {fq[i].x, fq[i].y, fq[i].z, fq[i].w};
#pragma unroll
                for (int j = 0; j < 4; j++)
                    bits |= ((((__vcmpne4(wd[j], 0u) & 0x01010101u) * 0x01020408u) >> 24) & 0xfu) << (4 * j);
            } else {
                for (int k = 0; k < 16; k++)
                    if (p + k < n && flags[p + k]) bits |= 1u << k;
            }
            const unsigned hi = __shfl_down_sync(FULL, bits, 1);
            if ((c & 1) == 0) heads[c >> 1] = bits | (hi << 16);
        }
    } else {
        mark_heads<TILE>(heads, off, nseg, t0, t0 + cnt, &s_k);
        tma_wait_tile(&bar, h, wt);
    }
    __syncthreads();
    const TI *sv = reinterpret_cast<const TI *>(tma_buf);
    auto load = [&](int64_t r0, ACC (&a)[V]) {
        if (r0 + V <= bulk_elems) {
            if (V == 4) {
                const int4 q = reinterpret_cast<const int4 *>(tma_buf)[r0 / 4];
                a[0] = (ACC)(int64_t)q.x;
                a[1 % V] = (ACC)(int64_t)q.y;
                a[2 % V] = (ACC)(int64_t)q.z;
                a[3 % V] = (ACC)(int64_t)q.w;
            } else {
                const longlong2 q = reinterpret_cast<const longlong2 *>(tma_buf)[r0 / 2];
                a[0] = (ACC)q.x;
                a[1 % V] = (ACC)q.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) {
                const int64_t r = r0 + k;
                a[k] = r < bulk_elems ? (ACC)(int64_t)sv[r] : (r < cnt ? (ACC)(int64_t)in[t0 + r] : (ACC)0);
            }
        }
    };
    const unsigned lt_mask = (1u << l) - 1u;
    // pass 1: head bits, local aggregates, warp scans with a segmented carry
    unsigned long long hbits = 0;  // V head bits per vector
    unsigned pstop = 0;            // bit u: the lane prefix of vector u holds a head
    ACC lane_pre[S];
    ACC cv = 0;
    unsigned cf = 0;
#pragma unroll
    for (int u = 0; u < S; u++) {
        const int64_t r0 = (int64_t)((w * S + u) * 32 + l) * V;
        ACC a[V];
        load(r0, a);
        // V head bits of this vector (V divides 32, so they sit in one word)
        const unsigned hb = (heads[(int)r0 >> 5] >> ((int)r0 & 31)) & ((1u << V) - 1u);
        hbits |= (unsigned long long)hb << (u * V);
        ACC x = 0;
#pragma unroll
        for (int k = 0; k < V; k++) x = ((hb >> k) & 1u) ? a[k] : x + a[k];
        ACC y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const ACC o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        const ACC e = y - x;
        const unsigned fm = __ballot_sync(FULL, hb != 0u);
        const unsigned below = fm & lt_mask;
        const ACC e_s = __shfl_sync(FULL, e, below ? 31 - __clz(below) : 0);
        lane_pre[u] = below ? e - e_s : cv + e;
        pstop |= (below || cf) ? (1u << u) : 0u;
        const ACC y_all = __shfl_sync(FULL, y, 31);
        const ACC e_last = __shfl_sync(FULL, e, fm ? 31 - __clz(fm) : 0);
        cv = fm ? y_all - e_last : cv + y_all;
        cf |= fm ? 1u : 0u;
    }
    if (l == 0) {
        s_wv[w] = cv;
        s_wf[w] = cf;
    }
    __syncthreads();
    if (w == 0) {
        const SP x = l < TMA_NT / 32 ? SP{s_wf[l], (unsigned long long)s_wv[l]} : SP{0u, 0ull};
        SP y = x;
#pragma unroll
        for (int d = 1; d < TMA_NT / 32; d <<= 1) {
            const SP o = shfl_up_sp(y, d);
            if (l >= d) y = sp_op(o, y);
        }
        SP ex = shfl_up_sp(y, 1);
        if (l == 0) ex = SP{0u, 0ull};
        const SP tile_agg = shfl_sp(y, TMA_NT / 32 - 1);
        const SP tile_ex = lookback(L, t, tile_agg, h, wt);
        __syncwarp();
        if (l < TMA_NT / 32) s_wv[l] = (ACC)sp_op(tile_ex, ex).v;
    }
    __syncthreads();
    // pass 2: outputs
    const ACC pre = s_wv[w];
    constexpr int VO = 16 / sizeof(TO);
#pragma unroll
    for (int u = 0; u < S; u++) {
        const int64_t r0 = (int64_t)((w * S + u) * 32 + l) * V;
        ACC a[V];
        load(r0, a);
        const unsigned hb = (unsigned)(hbits >> (u * V));
        ACC run = ((pstop >> u) & 1u) ? lane_pre[u] : pre + lane_pre[u];
        TO o[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            run = ((hb >> k) & 1u) ? a[k] : run + a[k];
            o[k] = (TO)(inclusive ? run : run - a[k]);
        }
        const int64_t p0 = t0 + r0;
        if (p0 + V <= n) {
#pragma unroll
            for (int c = 0; c < V; c += VO) {
                if (VO == 4) {
                    int4 st4;
                    st4.x = (int)o[c];
                    st4.y = (int)o[(c + 1) % V];
                    st4.z = (int)o[(c + 2) % V];
                    st4.w = (int)o[(c + 3) % V];
                    __stcs(reinterpret_cast<int4 *>(out + p0 + c), st4);
                } else {
                    longlong2 st2;
                    st2.x = (long long)o[c];
                    st2.y = (long long)o[(c + 1) % V];
                    __stcs(reinterpret_cast<longlong2 *>(out + p0 + c), st2);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (p0 + k < n) out[p0 + k] = o[k];
        }
    }
}

// Segment totals after a segmented scan: tot[k] = inclusive value at the segment's
// last element, 0 for an empty segment.
template <typename TI, typename TO>
__global__ void seg_totals_kernel(const TI *in, const TO *out, const int64_t *off, int64_t nseg, int64_t n,
                                  int inclusive, TO *tot) {
    IXP_KERNEL_ENTRY();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nseg; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = off[k], b = off[k + 1];
        if (b < a || a < 0 || b > n) b = a;  // invalid offsets: keep accesses in bounds
        if (b > a) {
            unsigned long long v = (unsigned long long)(int64_t)out[b - 1];
            if (!inclusive) v += (unsigned long long)(int64_t)in[b - 1];
            tot[k] = (TO)v;
        } else {
            tot[k] = (TO)0;
        }
    }
}

// ========================================================= predicate counts

// In-tile exclusive counts. Inputs: per sub-chunk u, V-bit masks kt (kept and
// true) and kk (kept). Output: per u, the packed exclusive count (kk << 16 | kt)
// of the elements before this thread's vector in the tile, and the tile total.
template <int V>
__device__ __forceinline__ unsigned tile_counts(const unsigned (&kt)[SUB], const unsigned (&kk)[SUB],
                                                unsigned (&pre)[SUB], unsigned *s_warp_u32) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned carry = 0, lp[SUB];
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        unsigned x = (unsigned)__popc(kt[u]) | ((unsigned)__popc(kk[u]) << 16);
        unsigned y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            unsigned o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y += o;
        }
        lp[u] = carry + y - x;
        carry += __shfl_sync(FULL, y, 31);
    }
    if (l == 0) s_warp_u32[w] = carry;
    __syncthreads();
    unsigned wpre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < TB / 32; i++) {
        unsigned c = s_warp_u32[i];
        if (i < w) wpre += c;
        tot += c;
    }
#pragma unroll
    for (int u = 0; u < SUB; u++) pre[u] = wpre + lp[u];
    __syncthreads();
    return tot;
}

__device__ __forceinline__ unsigned long long widen(unsigned packed) {
    return (unsigned long long)(packed & 0xffffu) | ((unsigned long long)(packed >> 16) << 32);
}

// Pass 1a: per-tile counts, streaming (no inter-tile dependency). Tile t writes its
// packed count (kept << 32 | kept_true) to tile_prefix[t]; with segments, every
// segment start off[k] inside the tile gets the in-tile exclusive count before it
// in seg_cnt[k] (the tile's prefix is added by seg_fix_kernel once it is known).
template <typename KT, bool SEG>
__global__ void __launch_bounds__(TB, 6) count_kernel(const KT *__restrict__ keys, int64_t n, DPred filt, DPred part,
                                                   const int64_t *__restrict__ off, int64_t nseg,
                                                   unsigned long long *tile_prefix, unsigned long long *seg_cnt,
                                                   int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int TILE = TB * SUB * V;
    __shared__ int64_t s_k;
    __shared__ unsigned s_w[TB / 32];
    __shared__ unsigned s_cnt[SEG ? TILE : 1];
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned kt[SUB], kk[SUB];
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
        KT kv[V];
        load_slot<KT, V>(keys, p0, n, vec_ok, kv);
        kk[u] = pred_mask<KT, V>(filt, kv, p0, n);
        kt[u] = kk[u] & pred_mask<KT, V>(part, kv, p0, n);
    }
    if (!SEG) {
        unsigned x = 0;
#pragma unroll
        for (int u = 0; u < SUB; u++) x += (unsigned)__popc(kt[u]) | ((unsigned)__popc(kk[u]) << 16);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        if (l == 0) s_w[w] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
#pragma unroll
            for (int i = 0; i < TB / 32; i++) tot += s_w[i];
            tile_prefix[t] = widen(tot);
        }
        return;
    }
    unsigned pre[SUB];
    const unsigned tot = tile_counts<V>(kt, kk, pre, s_w);
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int r0 = ((w * SUB + u) * 32 + l) * V;
#pragma unroll
        for (int k = 0; k < V; k++) {
            unsigned below = (1u << k) - 1u;
            s_cnt[r0 + k] = pre[u] + (unsigned)__popc(kt[u] & below) + ((unsigned)__popc(kk[u] & below) << 16);
        }
    }
    if (threadIdx.x == 0) {
        tile_prefix[t] = widen(tot);
        s_k = lb_off(off, nseg, t0);
    }
    __syncthreads();
    for (int64_t k = s_k + threadIdx.x; k <= nseg; k += blockDim.x) {
        const int64_t o = __ldg(off + k);
        if (o >= t1) break;
        if (o >= t0) seg_cnt[k] = widen(s_cnt[o - t0]);
    }
}

// Pass 1a without segments: each block counts CT consecutive tiles with all their
// loads issued up front (more bytes in flight per thread than one tile gives).
constexpr int CT = 2;

template <typename KT>
__global__ void __launch_bounds__(TB, 4) count_tiles_kernel(const KT *__restrict__ keys, int64_t n, DPred filt,
                                                         DPred part, int64_t nt, unsigned long long *tile_prefix,
                                                         int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int TILE = TB * SUB * V;
    __shared__ unsigned s_w[CT][TB / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    KT kv[CT][SUB][V];
#pragma unroll
    for (int c = 0; c < CT; c++)
#pragma unroll
        for (int u = 0; u < SUB; u++) {
            const int64_t p0 = ((int64_t)blockIdx.x * CT + c) * TILE + (int64_t)((w * SUB + u) * 32 + l) * V;
            load_slot<KT, V>(keys, p0, n, vec_ok, kv[c][u]);
        }
#pragma unroll
    for (int c = 0; c < CT; c++) {
        unsigned x = 0;
#pragma unroll
        for (int u = 0; u < SUB; u++) {
            const int64_t p0 = ((int64_t)blockIdx.x * CT + c) * TILE + (int64_t)((w * SUB + u) * 32 + l) * V;
            const unsigned kk = pred_mask<KT, V>(filt, kv[c][u], p0, n);
            const unsigned kt = kk & pred_mask<KT, V>(part, kv[c][u], p0, n);
            x += (unsigned)__popc(kt) | ((unsigned)__popc(kk) << 16);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        if (l == 0) s_w[c][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < CT) {
        const int64_t t = (int64_t)blockIdx.x * CT + threadIdx.x;
        unsigned tot = 0;
#pragma unroll
        for (int i = 0; i < TB / 32; i++) tot += s_w[threadIdx.x][i];
        if (t < nt) tile_prefix[t] = widen(tot);
    }
}

// Pass 1b: the grouped scan of the packed tile counts (tilescan.cuh).

// Pass 1c: seg_cnt[k] = packed count before off[k] (tile prefix + in-tile part);
// off[k] = n maps to the total. Offsets outside [0, n] leave seg_cnt[k] without
// meaning but in bounds.
template <int TILE>
__global__ void seg_fix_kernel(const int64_t *__restrict__ off, int64_t nseg, int64_t n,
                               const unsigned long long *__restrict__ tp, unsigned long long *seg_cnt, const Hdr *h) {
    IXP_KERNEL_ENTRY();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= nseg; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = __ldg(off + k);
        if (o >= n || o < 0) seg_cnt[k] = h->total;
        else seg_cnt[k] += __ldg(tp + o / TILE);
    }
}

// In-tile segment ids: element position r in the tile belongs to segment
// k0 + rel[r] where k0 is the segment of the tile's first element.
template <int V>
__device__ __forceinline__ void tile_segments(const int64_t *off, int64_t nseg, int64_t t0, int64_t t1, int *s_rel,
                                              int64_t *s_k0, int (&rel)[SUB][V]) {
    constexpr int TILE = TB * SUB * V;
    for (int r = threadIdx.x; r < TILE; r += blockDim.x) s_rel[r] = 0;
    if (threadIdx.x == 0) *s_k0 = seg_of(off, nseg, t0);
    __syncthreads();
    const int64_t k0 = *s_k0;
    for (int64_t k = k0 + 1 + threadIdx.x; k < nseg; k += blockDim.x) {
        int64_t o = __ldg(off + k);
        if (o >= t1) break;
        if (o > t0) atomicMax(&s_rel[o - t0], (int)(k - k0));
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __shared__ int s_wmax[TB / 32];
    int carry = 0;
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int r0 = ((w * SUB + u) * 32 + l) * V;
        int m = 0;
#pragma unroll
        for (int k = 0; k < V; k++) {
            m = max(m, s_rel[r0 + k]);
            rel[u][k] = m;  // running max inside the vector
        }
        int y = m;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(FULL, y, d);
            if (l >= d) y = max(y, o);
        }
        int ex = __shfl_up_sync(FULL, y, 1);
        if (l == 0) ex = 0;
        ex = max(ex, carry);
#pragma unroll
        for (int k = 0; k < V; k++) rel[u][k] = max(rel[u][k], ex);
        carry = max(carry, __shfl_sync(FULL, y, 31));
    }
    if (l == 0) s_wmax[w] = carry;
    __syncthreads();
    int wpre = 0;
    for (int i = 0; i < w; i++) wpre = max(wpre, s_wmax[i]);
#pragma unroll
    for (int u = 0; u < SUB; u++)
#pragma unroll
        for (int k = 0; k < V; k++) rel[u][k] = max(rel[u][k], wpre);
    __syncthreads();
}

// =========================================== segmented tiles, consecutive layout
// The segmented count, partition and InvFiltPart passes with the element layout of
// the flat InvFiltPart kernel: thread j of a tile takes the SUB * V consecutive
// elements t0 + j * SUB * V ..., so one warp scan of the threads' packed counts
// gives every rank and ranks run as counters over the thread's elements. The
// segment starts that fall in the tile are listed in shared memory (positions in
// increasing order; an empty segment repeats its position); a thread finds the
// segment of its first element by a binary search of the list and then walks it,
// loading a segment's counts only when the walk reaches its start. The tile sizes
// and the tile_prefix / seg_cnt layouts are those of the other segmented kernels.
constexpr int SG_MAXS = 4096;  // listed starts per tile; a tile with more walks the offsets in memory

struct SegList {
    int64_t ks;  // segment index of the list's first entry
    int ns;      // entries listed (-1: more than SG_MAXS)
};

// Lists the starts off[k] in [t0, t1) (all threads call it); lb = the first k with
// off[k] >= t0, from the per-tile table.
__device__ __forceinline__ SegList seg_list(const int64_t *__restrict__ off, int64_t nseg, int64_t t0, int64_t t1,
                                            int64_t lb, int *s_start, int64_t *s_ks, int *s_ns) {
    if (threadIdx.x == 0) {
        *s_ks = lb;
        *s_ns = 0;
    }
    __syncthreads();
    const int64_t ks = *s_ks;
    for (int64_t k = ks + threadIdx.x; k < nseg; k += blockDim.x) {
        const int64_t o = __ldg(off + k);
        if (o >= t1) break;
        const int64_t j = k - ks;
        if (j < SG_MAXS) s_start[j] = (int)(o - t0);
        atomicMax(s_ns, j < SG_MAXS ? (int)(j + 1) : SG_MAXS + 1);
    }
    __syncthreads();
    SegList L;
    L.ks = ks;
    L.ns = *s_ns > SG_MAXS ? -1 : *s_ns;
    return L;
}

// Segment walker of one thread: k = the segment of the current element (the last k
// with off[k] <= i), and the counts of segment k.
struct SegWalk {
    int64_t k;      // current segment
    int next;       // index in the tile's list of the next start not yet passed
    int64_t ek;     // off[k]
    int64_t ctk;    // trues before the segment (global, kept and true)
    int64_t ckk;    // kept before the segment
    int64_t tk;     // kept trues in the segment
};

__device__ __forceinline__ void seg_load(SegWalk &W, const int64_t *__restrict__ off, int64_t nseg,
                                         const unsigned long long *__restrict__ seg_cnt) {
    const int64_t k = W.k < 0 ? 0 : (W.k >= nseg ? nseg - 1 : W.k);  // stays in bounds for invalid offsets
    const unsigned long long a0 = __ldg(seg_cnt + k), a1 = __ldg(seg_cnt + k + 1);
    W.ek = __ldg(off + k);
    W.ctk = (int64_t)(a0 & 0xffffffffull);
    W.ckk = (int64_t)(a0 >> 32);
    W.tk = (int64_t)(a1 & 0xffffffffull) - W.ctk;
}

// Starts the walk at in-tile position r0.
__device__ __forceinline__ void seg_begin(SegWalk &W, const SegList &L, const int *s_start, int r0, int64_t t0,
                                          const int64_t *__restrict__ off, int64_t nseg,
                                          const unsigned long long *__restrict__ seg_cnt) {
    if (L.ns >= 0) {
        int lo = 0, hi = L.ns;  // number of listed starts <= r0
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_start[mid] <= r0) lo = mid + 1;
            else hi = mid;
        }
        W.next = lo;
        W.k = L.ks - 1 + lo;
    } else {
        W.next = 0;
        W.k = seg_of(off, nseg, t0 + r0);
    }
    seg_load(W, off, nseg, seg_cnt);
}

// Moves the walk to in-tile position r (increasing).
__device__ __forceinline__ void seg_step(SegWalk &W, const SegList &L, const int *s_start, int r, int64_t t0,
                                         const int64_t *__restrict__ off, int64_t nseg,
                                         const unsigned long long *__restrict__ seg_cnt) {
    bool moved = false;
    if (L.ns >= 0) {
        while (W.next < L.ns && s_start[W.next] <= r) {
            W.next++;
            W.k++;
            moved = true;
        }
    } else {
        while (W.k + 1 < nseg && __ldg(off + W.k + 1) <= t0 + r) {
            W.k++;
            moved = true;
        }
    }
    if (moved) seg_load(W, off, nseg, seg_cnt);
}

// Masks of this thread's PER consecutive elements at e0 (bit j = element e0 + j).
template <typename KT>
__device__ __forceinline__ void seg_masks(const KT *__restrict__ keys, int64_t e0, int64_t n, int vec_ok, DPred filt,
                                          DPred part, unsigned &kk, unsigned &kt, KT (&kv)[SUB][16 / sizeof(KT)]) {
    constexpr int V = 16 / sizeof(KT);
#pragma unroll
    for (int u = 0; u < SUB; u++) load_slot<KT, V>(keys, e0 + u * V, n, vec_ok, kv[u]);
    kk = pred_mask_run<KT, SUB, V>(filt, kv, e0, n);
    kt = kk & pred_mask_run<KT, SUB, V>(part, kv, e0, n);
}

// Packed in-tile exclusive count (kept << 16 | kept true) of this thread's first
// element, and the tile total, from one warp scan and the warp totals.
__device__ __forceinline__ unsigned seg_thread_prefix(unsigned x, unsigned *s_w, unsigned &tot) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned y = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(FULL, y, d);
        if (l >= d) y += o;
    }
    if (l == 31) s_w[w] = y;
    __syncthreads();
    unsigned wpre = 0;
    tot = 0;
#pragma unroll
    for (int i = 0; i < TB / 32; i++) {
        const unsigned c = s_w[i];
        wpre += i < w ? c : 0u;
        tot += c;
    }
    return wpre + y - x;
}

// Pass 1 with segments (consecutive layout): tile counts, and for every segment
// start in the tile its in-tile exclusive count (seg_fix_kernel adds the prefix).
template <typename KT>
__global__ void __launch_bounds__(TB, 4) count_seg_kernel(const KT *__restrict__ keys, int64_t n, DPred filt,
                                                       DPred part, const int64_t *__restrict__ off, int64_t nseg,
                                                       const int64_t *__restrict__ tile_lb,
                                                       unsigned long long *tile_prefix, unsigned long long *seg_cnt,
                                                       int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int PER = SUB * V;
    constexpr int TILE = TB * PER;
    __shared__ unsigned s_w[TB / 32];
    __shared__ unsigned s_pre[TB], s_kt[TB], s_kk[TB];
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int64_t e0 = t0 + (int64_t)threadIdx.x * PER;
    unsigned kk, kt;
    KT kv[SUB][V];
    seg_masks<KT>(keys, e0, n, vec_ok, filt, part, kk, kt, kv);
    unsigned tot;
    const unsigned pre = seg_thread_prefix((unsigned)__popc(kt) | ((unsigned)__popc(kk) << 16), s_w, tot);
    s_pre[threadIdx.x] = pre;
    s_kt[threadIdx.x] = kt;
    s_kk[threadIdx.x] = kk;
    if (threadIdx.x == 0) tile_prefix[t] = widen(tot);
    const int64_t ks = __ldg(tile_lb + t);
    __syncthreads();
    for (int64_t k = ks + threadIdx.x; k <= nseg; k += blockDim.x) {
        const int64_t o = __ldg(off + k);
        if (o >= t1) break;
        if (o >= t0) {
            const int r = (int)(o - t0), j = r / PER;
            const unsigned below = (1u << (r % PER)) - 1u;
            const unsigned c = s_pre[j] + (unsigned)__popc(s_kt[j] & below) + ((unsigned)__popc(s_kk[j] & below) << 16);
            seg_cnt[k] = widen(c);
        }
    }
}

// Per-segment bases of the walk: within segment k, an element's destination is
// bt + (kept trues before it, over the whole array) when it is a kept true, and
// bf + (kept falses before it) when it is a kept false: bt = F_k - C_k and
// bf = F_k + T_k - (F_k - C_k) = T_k + C_k, with F_k the kept elements and C_k
// the kept trues before the segment, T_k the segment's kept trues (partition2L
// keeps everything, so F_k = e_k there).
template <typename AT>
__device__ __forceinline__ void seg_bases(const SegWalk &W, AT &bt, AT &bf) {
    bt = (AT)(W.ckk - W.ctk);
    bf = (AT)(W.tk + W.ctk);
}

// Next listed start position after the walk's current one (INT_MAX: none).
__device__ __forceinline__ int seg_next_pos(const SegWalk &W, const SegList &L, const int *s_start,
                                            const int64_t *__restrict__ off, int64_t nseg, int64_t t0) {
    if (L.ns >= 0) return W.next < L.ns ? s_start[W.next] : INT_MAX;
    if (W.k + 1 >= nseg) return INT_MAX;
    const int64_t o = __ldg(off + W.k + 1) - t0;
    return o > (int64_t)INT_MAX ? INT_MAX : (int)(o < 0 ? 0 : o);
}

// Pass 2 of partition2L (consecutive layout): destinations (index form), and the
// keys / payload rows moved to them. AT: the arithmetic type of the running
// counts and destinations (int32 when n <= INT32_MAX).
template <typename KT, typename OT, typename AT>
__global__ void __launch_bounds__(TB, 4) partition_seg_kernel(
    const KT *__restrict__ keys, int64_t n, DPred pred, const uint32_t *__restrict__ payload, int row_words,
    OT *__restrict__ out_idx, KT *__restrict__ out_keys, uint32_t *__restrict__ out_payload,
    const int64_t *__restrict__ off, int64_t nseg, const int64_t *__restrict__ tile_lb,
    const unsigned long long *__restrict__ tile_prefix, const unsigned long long *__restrict__ seg_cnt, int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int PER = SUB * V;
    constexpr int TILE = TB * PER;
    __shared__ unsigned s_w[TB / 32];
    __shared__ int s_start[SG_MAXS];
    __shared__ int64_t s_ks;
    __shared__ int s_ns;
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int64_t e0 = t0 + (int64_t)threadIdx.x * PER;
    const DPred all{IXP_P_TRUE, 0, 0, nullptr};
    unsigned kk, kt;
    KT kv[SUB][V];
    seg_masks<KT>(keys, e0, n, vec_ok, all, pred, kk, kt, kv);
    unsigned tot;
    const unsigned pre = seg_thread_prefix((unsigned)__popc(kt) | ((unsigned)__popc(kk) << 16), s_w, tot);
    const SegList L = seg_list(off, nseg, t0, t1, __ldg(tile_lb + t), s_start, &s_ks, &s_ns);
    const unsigned long long tp = tile_prefix[t];
    AT ct = (AT)((tp & 0xffffffffull) + (pre & 0xffffu));                                  // trues before
    AT cf = (AT)(((tp >> 32) - (tp & 0xffffffffull)) + ((pre >> 16) - (pre & 0xffffu)));  // falses before
    const int r0 = (int)threadIdx.x * PER;
    SegWalk W;
    AT bt = 0, bf = 0;
    int nxt = INT_MAX;
    if (e0 < n) {
        seg_begin(W, L, s_start, r0, t0, off, nseg, seg_cnt);
        seg_bases<AT>(W, bt, bf);
        nxt = seg_next_pos(W, L, s_start, off, nseg, t0);
    }
    const bool moves = out_keys || out_payload;
    OT dst[PER];
    if (!moves && e0 + PER <= n && nxt >= r0 + PER) {
        // no segment starts inside the run (the common case): every element is kept
        // (partition2L has no filter), so its rank among the run's trues or falses
        // is a popcount of the mask below it
#pragma unroll
        for (int j = 0; j < PER; j++) {
            const unsigned tb = (unsigned)__popc(kt & ((1u << j) - 1u));
            dst[j] = (OT)(((kt >> j) & 1u) ? bt + ct + (AT)tb : bf + cf + (AT)(j - tb));
        }
    } else
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const bool c = (kt >> j) & 1u;
        if (r0 + j >= nxt && e0 + j < n) {  // a segment starts here: move the walk
            seg_step(W, L, s_start, r0 + j, t0, off, nseg, seg_cnt);
            seg_bases<AT>(W, bt, bf);
            nxt = seg_next_pos(W, L, s_start, off, nseg, t0);
        }
        const AT d = c ? bt + ct : bf + cf;
        dst[j] = (OT)d;
        ct += c ? 1 : 0;
        cf += c ? 0 : 1;
        if (moves && e0 + j < n && d >= 0 && (int64_t)d < n) {  // d is outside [0, n) only for invalid offsets
            const int64_t i = e0 + j;
            if (out_keys) out_keys[d] = kv[j / V][j % V];
            if (out_payload)
                for (int c2 = 0; c2 < row_words; c2++) out_payload[(int64_t)d * row_words + c2] = payload[i * row_words + c2];
        }
    }
    if (out_idx) {
        if (vec_ok && e0 + PER <= n) {
            if (sizeof(OT) == 4) {
#pragma unroll
                for (int u = 0; u < PER / 4; u++)
                    __stcs(reinterpret_cast<int4 *>(out_idx + e0) + u,
                           make_int4((int)dst[4 * u], (int)dst[4 * u + 1], (int)dst[4 * u + 2], (int)dst[4 * u + 3]));
            } else {
#pragma unroll
                for (int u = 0; u < PER / 2; u++)
                    __stcs(reinterpret_cast<longlong2 *>(out_idx + e0) + u,
                           make_longlong2((long long)dst[2 * u], (long long)dst[2 * u + 1]));
            }
        } else {
#pragma unroll
            for (int j = 0; j < PER; j++)
                if (e0 + j < n) out_idx[e0 + j] = dst[j];
        }
    }
}

// Segmented InvFiltPart check, pass 2 (consecutive layout): the smallest i whose Z
// is not its expected destination (kept) or lies inside [0, N) (dropped).
template <typename KT, typename ZT, typename AT>
__global__ void __launch_bounds__(TB, 4) filtpart_seg_kernel(
    const ZT *__restrict__ z, int64_t n, const KT *__restrict__ keys, DPred filt, DPred part,
    const int64_t *__restrict__ off, int64_t nseg, const int64_t *__restrict__ tile_lb,
    const unsigned long long *__restrict__ tile_prefix, const unsigned long long *__restrict__ seg_cnt, Hdr *h,
    int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int PER = SUB * V;
    constexpr int TILE = TB * PER;
    __shared__ unsigned s_w[TB / 32];
    __shared__ int s_start[SG_MAXS];
    __shared__ int64_t s_ks;
    __shared__ int s_ns;
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int64_t e0 = t0 + (int64_t)threadIdx.x * PER;
    unsigned kk, kt;
    KT kv[SUB][V];
    seg_masks<KT>(keys, e0, n, vec_ok, filt, part, kk, kt, kv);
    ZT zz[PER];
    const bool zvec = vec_ok && e0 + PER <= n && (reinterpret_cast<uintptr_t>(z + e0) & 15u) == 0;
    if (zvec) {
#pragma unroll
        for (int u = 0; u < PER * (int)sizeof(ZT) / 16; u++) {
            if constexpr (sizeof(ZT) == 4) {
                const int4 q = __ldcs(reinterpret_cast<const int4 *>(z + e0) + u);
                zz[4 * u] = q.x;
                zz[4 * u + 1] = q.y;
                zz[4 * u + 2] = q.z;
                zz[4 * u + 3] = q.w;
            } else {
                const longlong2 q = __ldcs(reinterpret_cast<const longlong2 *>(z + e0) + u);
                zz[2 * u] = q.x;
                zz[2 * u + 1] = q.y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < PER; j++) zz[j] = e0 + j < n ? z[e0 + j] : (ZT)0;
    }
    unsigned tot;
    const unsigned pre = seg_thread_prefix((unsigned)__popc(kt) | ((unsigned)__popc(kk) << 16), s_w, tot);
    const SegList L = seg_list(off, nseg, t0, t1, __ldg(tile_lb + t), s_start, &s_ks, &s_ns);
    const unsigned long long tp = tile_prefix[t];
    AT ct = (AT)((tp & 0xffffffffull) + (pre & 0xffffu));                                  // kept trues before
    AT cf = (AT)(((tp >> 32) - (tp & 0xffffffffull)) + ((pre >> 16) - (pre & 0xffffu)));  // kept falses before
    const int64_t Ntot = (int64_t)(h->total >> 32);
    const int r0 = (int)threadIdx.x * PER;
    SegWalk W;
    AT bt = 0, bf = 0;
    int nxt = INT_MAX;
    if (e0 < n) {
        seg_begin(W, L, s_start, r0, t0, off, nseg, seg_cnt);
        seg_bases<AT>(W, bt, bf);
        nxt = seg_next_pos(W, L, s_start, off, nseg, t0);
    }
    int bad = INT_MAX;  // position in the thread's run
    if (e0 + PER <= n && nxt >= r0 + PER) {
        // no segment starts inside the run: ranks are popcounts of the masks below
        // each element; the wrong elements collect in a mask
        unsigned wm = 0;
        const unsigned kf = kk & ~kt;
#pragma unroll
        for (int j = 0; j < PER; j++) {
            const unsigned below = (1u << j) - 1u;
            const bool c = (kt >> j) & 1u;
            const AT ref = c ? bt + ct + (AT)__popc(kt & below) : bf + cf + (AT)__popc(kf & below);
            const int64_t zi = (int64_t)zz[j];
            const bool wrong = ((kk >> j) & 1u) ? zi != (int64_t)ref : (zi >= 0 && zi < Ntot);
            wm |= (unsigned)wrong << j;
        }
        bad = wm ? __ffs(wm) - 1 : INT_MAX;
    } else
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const bool kept = (kk >> j) & 1u, c = (kt >> j) & 1u;
        if (r0 + j >= nxt && e0 + j < n) {  // a segment starts here: move the walk
            seg_step(W, L, s_start, r0 + j, t0, off, nseg, seg_cnt);
            seg_bases<AT>(W, bt, bf);
            nxt = seg_next_pos(W, L, s_start, off, nseg, t0);
        }
        const AT ref = c ? bt + ct : bf + cf;
        const int64_t zi = (int64_t)zz[j];
        const bool wrong = kept ? zi != (int64_t)ref : (zi >= 0 && zi < Ntot);
        if (wrong && e0 + j < n) bad = min(bad, j);
        ct += c ? 1 : 0;
        cf += (kept && !c) ? 1 : 0;
    }
    __shared__ unsigned long long sm[TB / 32];
    const unsigned long long r = block_max_u64(bad == INT_MAX ? 0ull : enc_first(e0 + bad), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

// Pass 2 of the partition: destinations, and the scattered keys/payload.
template <typename KT, typename OT, bool SEG>
__global__ void __launch_bounds__(TB) partition_write_kernel(
    const KT *__restrict__ keys, int64_t n, DPred pred, const uint32_t *__restrict__ payload, int row_words,
    OT *__restrict__ out_idx, KT *__restrict__ out_keys, uint32_t *__restrict__ out_payload,
    const int64_t *__restrict__ off, int64_t nseg, const unsigned long long *__restrict__ tile_prefix,
    const unsigned long long *__restrict__ seg_cnt, const Hdr *h, int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int TILE = TB * SUB * V;
    __shared__ unsigned s_w[TB / 32];
    __shared__ int s_rel[SEG ? TILE : 1];
    __shared__ int64_t s_k0;
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned kt[SUB], kk[SUB];
    KT kv[SUB][V];
    const DPred all{IXP_P_TRUE, 0, 0, nullptr};
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
        load_slot<KT, V>(keys, p0, n, vec_ok, kv[u]);
        kk[u] = pred_mask<KT, V>(all, kv[u], p0, n);
        kt[u] = pred_mask<KT, V>(pred, kv[u], p0, n);
    }
    unsigned pre[SUB];
    tile_counts<V>(kt, kk, pre, s_w);
    int rel[SUB][V];
    if (SEG) tile_segments<V>(off, nseg, t0, t1, s_rel, &s_k0, rel);
    const unsigned long long tp = tile_prefix[t];
    const int64_t T = (int64_t)(h->total & 0xffffffffull);
    const int64_t tile_ct = (int64_t)(tp & 0xffffffffull);
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
        OT dst[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            const int64_t i = p0 + k;
            const unsigned below = (1u << k) - 1u;
            const int64_t ct = tile_ct + (int64_t)(pre[u] & 0xffffu) + __popc(kt[u] & below);  // trues before i
            const bool c = (kt[u] >> k) & 1u;
            int64_t d;
            if (!SEG) {
                d = c ? ct : T + (i - ct);
            } else {
                const int64_t sk = s_k0 + rel[u][k];
                const int64_t ek = __ldg(off + sk);
                const int64_t ctk = (int64_t)(__ldg(seg_cnt + sk) & 0xffffffffull);
                const int64_t tk = (int64_t)(__ldg(seg_cnt + sk + 1) & 0xffffffffull) - ctk;
                const int64_t tb = ct - ctk;  // trues before i in its segment
                d = c ? ek + tb : ek + tk + (i - ek) - tb;
            }
            dst[k] = (OT)d;
            if (i < n && d >= 0 && d < n) {  // d is outside [0, n) only for invalid offsets
                if (out_keys) out_keys[d] = kv[u][k];
                if (out_payload)
                    for (int c2 = 0; c2 < row_words; c2++) out_payload[d * row_words + c2] = payload[i * row_words + c2];
            }
        }
        if (!out_idx) {
            // keys / payload only
        } else if (vec_ok && p0 + V <= n && sizeof(OT) * V >= 16) {
            if (sizeof(OT) == 4) {
                int4 s;
                s.x = (int)dst[0];
                s.y = (int)dst[1 % V];
                s.z = (int)dst[2 % V];
                s.w = (int)dst[3 % V];
                __stcs(reinterpret_cast<int4 *>(out_idx + p0), s);
            } else {
#pragma unroll
                for (int c = 0; c < V; c += 2) {
                    longlong2 s;
                    s.x = (long long)dst[c];
                    s.y = (long long)dst[(c + 1) % V];
                    __stcs(reinterpret_cast<longlong2 *>(out_idx + p0 + c), s);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (p0 + k < n) out_idx[p0 + k] = dst[k];
        }
    }
}

// Flat partition, pass 2, for payload rows of one 32-bit word. The tile's keys
// and payload are staged in shared memory (one bulk copy each when the tile is
// full and aligned, plain loads otherwise). The tile's trues land in one
// contiguous run [tp, tp + T_tile) of the outputs and its falses in another, so
// the payload (and keys) are placed in run order in shared memory, each run
// shifted by its destination's offset within a 16-byte chunk, and written out as
// aligned 16-byte stores with scalar stores only at the two ends of each run.
template <typename E>
__device__ __forceinline__ void write_run(E *__restrict__ g, const E *s, int64_t d0, int len, int sh) {
    constexpr int C = 16 / (int)sizeof(E);
    const int nch = (sh + len + C - 1) / C;
    E *gb = g + (d0 - sh);  // 16-byte aligned
    for (int k = threadIdx.x; k < nch; k += blockDim.x) {
        const int e0 = k * C;
        if (e0 >= sh && e0 + C <= sh + len) {
            __stcs(reinterpret_cast<int4 *>(gb + e0), *reinterpret_cast<const int4 *>(s + e0));
        } else {
#pragma unroll
            for (int c = 0; c < C; c++)
                if (e0 + c >= sh && e0 + c < sh + len) gb[e0 + c] = s[e0 + c];
        }
    }
}

template <typename KT>
__host__ __device__ constexpr int pf_tile() { return TB * SUB * (16 / (int)sizeof(KT)); }

// Shared layout: keys in | payload in | payload out | keys out. Each output area
// holds both runs, each starting on a 16-byte boundary after a shift of up to one
// chunk, and is read in whole chunks: TILE + 16 entries cover that.
template <typename KT>
__host__ __device__ constexpr size_t pf_smem_bytes(bool out_keys) {
    return (size_t)pf_tile<KT>() * sizeof(KT) + (size_t)pf_tile<KT>() * 4 + (size_t)(pf_tile<KT>() + 16) * 4 +
           (out_keys ? (size_t)(pf_tile<KT>() + 16) * sizeof(KT) : 0);
}

template <typename KT, typename OT, bool OUT_KEYS>
__global__ void __launch_bounds__(TB, 4) partition_flat_kernel(
    const KT *__restrict__ keys, int64_t n, DPred pred, const uint32_t *__restrict__ payload, OT *__restrict__ out_idx,
    KT *__restrict__ out_keys, uint32_t *__restrict__ out_payload, const unsigned long long *__restrict__ tile_prefix,
    Hdr *h, int vec_ok, int bulk_ok, Wait wt) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int TILE = TB * SUB * V;
    constexpr int CK = 16 / (int)sizeof(KT);  // keys per 16-byte chunk
    extern __shared__ __align__(128) unsigned char pf_buf[];
    KT *s_kin = reinterpret_cast<KT *>(pf_buf);
    uint32_t *s_pin = reinterpret_cast<uint32_t *>(s_kin + TILE);
    uint32_t *s_pout = s_pin + TILE;
    KT *s_kout = reinterpret_cast<KT *>(s_pout + TILE + 16);
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned s_w[TB / 32];
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int cnt = (int)(t1 - t0);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (bulk_ok && cnt == TILE) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            const unsigned kb = keys ? (unsigned)(TILE * sizeof(KT)) : 0u, pb = payload ? (unsigned)(TILE * 4) : 0u;
            mbar_expect_tx(&bar, kb + pb);
            for (unsigned o = 0; o < kb; o += 16384u)
                bulk_g2s((char *)s_kin + o, (const char *)(keys + t0) + o, min(16384u, kb - o), &bar);
            for (unsigned o = 0; o < pb; o += 16384u)
                bulk_g2s((char *)s_pin + o, (const char *)(payload + t0) + o, min(16384u, pb - o), &bar);
            if (!mbar_wait_bounded(&bar, 0, wt.spin_limit)) {
                set_status(h, IXP_E_TIMEOUT);
                mbar_wait_bounded(&bar, 0, wt.spin_limit);  // let the copies land before the block moves on
            }
        }
    } else {
        for (int r = threadIdx.x; r < cnt; r += TB) {
            if (keys) s_kin[r] = keys[t0 + r];
            if (payload) s_pin[r] = payload[t0 + r];
        }
    }
    __syncthreads();
    unsigned kt[SUB], kk[SUB];
    const DPred all{IXP_P_TRUE, 0, 0, nullptr};
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int r0 = ((w * SUB + u) * 32 + l) * V;
        const int64_t p0 = t0 + r0;
        KT kv[V];
        if (keys) {
            const int4 q = *reinterpret_cast<const int4 *>(s_kin + r0);
            memcpy(kv, &q, 16);
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) kv[k] = (KT)0;
        }
        kk[u] = pred_mask<KT, V>(all, kv, p0, n);
        kt[u] = pred_mask<KT, V>(pred, kv, p0, n);
    }
    unsigned pre[SUB];
    const unsigned tot = tile_counts<V>(kt, kk, pre, s_w);
    const int tile_T = (int)(tot & 0xffffu);
    const int64_t tp = (int64_t)(tile_prefix[t] & 0xffffffffull);
    const int64_t T = (int64_t)(h->total & 0xffffffffull);
    const int64_t fbase = T + (t0 - tp);  // destination of the tile's first false
    const int sh_t = (int)(tp & 3), sh_f = (int)(fbase & 3);
    const int f_off = (sh_t + tile_T + 3) & ~3;  // start of the false run in s_pout (16-byte aligned)
    const int kh_t = (int)(tp % CK), kh_f = (int)(fbase % CK);
    const int kf_off = (kh_t + tile_T + CK - 1) / CK * CK;
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int r0 = ((w * SUB + u) * 32 + l) * V;
        const int64_t p0 = t0 + r0;
        OT dst[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            const int r = r0 + k;
            const int lt = (int)(pre[u] & 0xffffu) + __popc(kt[u] & ((1u << k) - 1u));
            const bool c = (kt[u] >> k) & 1u;
            dst[k] = (OT)(c ? tp + lt : fbase + (r - lt));
            if (r < cnt) {
                if (out_payload) s_pout[c ? sh_t + lt : f_off + sh_f + (r - lt)] = s_pin[r];
                if (OUT_KEYS) s_kout[c ? kh_t + lt : kf_off + kh_f + (r - lt)] = s_kin[r];
            }
        }
        if (!out_idx) {
            // destinations used for the staged runs only
        } else if (vec_ok && p0 + V <= n && sizeof(OT) * V >= 16) {
            if (sizeof(OT) == 4) {
                int4 s4;
                s4.x = (int)dst[0];
                s4.y = (int)dst[1 % V];
                s4.z = (int)dst[2 % V];
                s4.w = (int)dst[3 % V];
                __stcs(reinterpret_cast<int4 *>(out_idx + p0), s4);
            } else {
#pragma unroll
                for (int c = 0; c < V; c += 2) {
                    longlong2 s2;
                    s2.x = (long long)dst[c];
                    s2.y = (long long)dst[(c + 1) % V];
                    __stcs(reinterpret_cast<longlong2 *>(out_idx + p0 + c), s2);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (p0 + k < n) out_idx[p0 + k] = dst[k];
        }
    }
    if (!out_payload && !OUT_KEYS) return;
    __syncthreads();
    const int tile_F = cnt - tile_T;
    // the runs stay inside [0, n) whenever the header is consistent
    const bool runs_ok = tp >= 0 && tp + tile_T <= n && fbase >= 0 && fbase + tile_F <= n;
    if (!runs_ok) return;
    if (out_payload) {
        write_run<uint32_t>(out_payload, s_pout, tp, tile_T, sh_t);
        write_run<uint32_t>(out_payload, s_pout + f_off, fbase, tile_F, sh_f);
    }
    if (OUT_KEYS) {
        write_run<KT>(out_keys, s_kout, tp, tile_T, kh_t);
        write_run<KT>(out_keys, s_kout + kf_off, fbase, tile_F, kh_f);
    }
}

// Flat InvFiltPart check, streaming pass over Z and the keys (8 bytes per int32
// element). A kept true element at in-tile true rank r must hold P_t + r, where
// P_t is the count of kept trues before the tile; a kept false at in-tile false
// rank r must hold T + F_t + r (T the total of kept trues, F_t the kept falses
// before the tile). Neither P_t, F_t nor T is known yet, so each tile records
// whether Z - r is one constant over its kept trues (and over its kept falses) and
// which: rec[t] = {true constant, false constant}, with FP_NONE for no such element
// and FP_BAD when they differ or a value is below its rank. A dropped element must
// lie outside [0, N), so the smallest non-negative dropped Z goes to h->k_first2.
// The packed tile count goes to tile_prefix[t] for the scan that follows.
constexpr long long FP_NONE = -1, FP_BAD = -2;

// AT: the arithmetic type of the per-element bookkeeping (int32 when Z is int32
// and n <= INT32_MAX, so every rank, Z and Z - rank fits; int64 otherwise).
template <typename AT> struct Lim;
template <> struct Lim<int32_t> { static constexpr int32_t lo = INT32_MIN, hi = INT32_MAX; };
template <> struct Lim<int64_t> { static constexpr int64_t lo = INT64_MIN, hi = INT64_MAX; };

template <typename AT>
__device__ __forceinline__ void fp_fold(AT &mn, AT &mx, AT zi, AT r) {
    const AT q = zi < r ? Lim<AT>::lo : zi - r;
    mn = q < mn ? q : mn;
    mx = q > mx ? q : mx;
}

// Widen a (min, max) pair; the empty pair (AT max, AT min) stays empty.
template <typename AT>
__device__ __forceinline__ int64_t fp_wide_min(AT v) {
    return v == Lim<AT>::hi ? INT64_MAX : (int64_t)v;
}

__device__ __forceinline__ long long fp_rec(int64_t mn, int64_t mx) {
    if (mn > mx) return FP_NONE;
    return (mn == mx && mn >= 0) ? (long long)mn : FP_BAD;
}

template <typename KT, typename ZT, typename AT>
__global__ void __launch_bounds__(TB, sizeof(ZT) > sizeof(KT) ? 3 : 4) filtpart_tile_kernel(const ZT *__restrict__ z, int64_t n,
                                                              const KT *__restrict__ keys, DPred filt, DPred part,
                                                              unsigned long long *tile_prefix, longlong2 *rec, Hdr *h,
                                                              int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int TILE = TB * SUB * V;
    __shared__ unsigned s_w[TB / 32];
    __shared__ unsigned long long s_r[5][TB / 32];
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned kt[SUB], kk[SUB];
    ZT zv[SUB][V];
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
        KT kv[V];
        load_slot<KT, V>(keys, p0, n, vec_ok, kv);
        load_vec<ZT, V>(z, p0, n, vec_ok, zv[u]);
        kk[u] = pred_mask<KT, V>(filt, kv, p0, n);
        kt[u] = kk[u] & pred_mask<KT, V>(part, kv, p0, n);
    }
    unsigned pre[SUB];
    const unsigned tot = tile_counts<V>(kt, kk, pre, s_w);
    constexpr AT AMAX = Lim<AT>::hi, AMIN = Lim<AT>::lo;
    AT tmn = AMAX, tmx = AMIN, fmn = AMAX, fmx = AMIN, dmin = AMAX;
    const bool full = t0 + TILE <= n;
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
#pragma unroll
        for (int k = 0; k < V; k++) {
            if (!full && p0 + k >= n) continue;
            const unsigned below = (1u << k) - 1u;
            const AT rt = (AT)((pre[u] & 0xffffu) + __popc(kt[u] & below));
            const AT rk = (AT)((pre[u] >> 16) + __popc(kk[u] & below));
            const AT zi = (AT)zv[u][k];
            if ((kk[u] >> k) & 1u) {
                if ((kt[u] >> k) & 1u) fp_fold<AT>(tmn, tmx, zi, rt);
                else fp_fold<AT>(fmn, fmx, zi, rk - rt);
            } else if (zi >= 0) {
                dmin = zi < dmin ? zi : dmin;
            }
        }
    }
    if constexpr (sizeof(AT) == 4) {
        // 32-bit bookkeeping: one warp-reduce instruction per value, then the
        // order-preserving 64-bit encodings once per warp
        tmn = __reduce_min_sync(FULL, tmn);
        tmx = __reduce_max_sync(FULL, tmx);
        fmn = __reduce_min_sync(FULL, fmn);
        fmx = __reduce_max_sync(FULL, fmx);
        dmin = __reduce_min_sync(FULL, dmin);
        if (l == 0) {
            s_r[0][w] = enc_min(fp_wide_min(tmn));
            s_r[1][w] = enc_max((int64_t)tmx);
            s_r[2][w] = enc_min(fp_wide_min(fmn));
            s_r[3][w] = enc_max((int64_t)fmx);
            s_r[4][w] = enc_min(fp_wide_min(dmin));
        }
    } else {
        unsigned long long r[5] = {enc_min(fp_wide_min(tmn)), enc_max((int64_t)tmx), enc_min(fp_wide_min(fmn)),
                                   enc_max((int64_t)fmx), enc_min(fp_wide_min(dmin))};
#pragma unroll
        for (int j = 0; j < 5; j++) {
            r[j] = warp_max_u64(r[j]);
            if (l == 0) s_r[j][w] = r[j];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long r[5];
#pragma unroll
        for (int j = 0; j < 5; j++) {
            r[j] = s_r[j][0];
            for (int i = 1; i < TB / 32; i++) r[j] = s_r[j][i] > r[j] ? s_r[j][i] : r[j];
        }
        tile_prefix[t] = widen(tot);
        rec[t] = make_longlong2(fp_rec(dec_min(r[0]), dec_max(r[1])), fp_rec(dec_min(r[2]), dec_max(r[3])));
        atomic_max_u64(&h->k_first2, r[4]);
    }
}

// The same tile pass for the common form (int32 keys and Z, filter TRUE, predicate
// key < b, 16-byte aligned inputs, n <= INT32_MAX), written for few instructions
// per element: a thread takes 16 consecutive elements of the tile (four 16-byte
// loads), so one warp scan of the threads' counts gives every rank, which then runs
// as a counter over the thread's elements; Z - rank is taken modulo 2^32,
// which is exact here because Z and every expected destination lie in the int32
// range (Z - rank equals the tile constant modulo 2^32 only when Z is the expected
// destination), so no element needs a separate negative guard; the folds are
// branch-free min / max updates. Records the same rec[t], tile_prefix[t] and
// dropped-element minimum (none: every element is kept) as filtpart_tile_kernel.
__global__ void __launch_bounds__(TB, 4) filtpart_tile_lt_kernel(const int32_t *__restrict__ z, int64_t n,
                                                                const int32_t *__restrict__ keys, int32_t b,
                                                                unsigned long long *tile_prefix, longlong2 *rec) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 4;
    constexpr int PER = SUB * V;  // consecutive elements per thread
    constexpr int TILE = TB * PER;
    __shared__ unsigned s_w[TB / 32];
    __shared__ int s_r[4][TB / 32];
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t e0 = t0 + (int64_t)threadIdx.x * PER;  // this thread's first element
    int zz[PER];
    unsigned kt = 0, kk;
    if (e0 + PER <= n) {
#pragma unroll
        for (int u = 0; u < SUB; u++) {
            const int4 kv = __ldcs(reinterpret_cast<const int4 *>(keys + e0) + u);
            const int4 zq = __ldcs(reinterpret_cast<const int4 *>(z + e0) + u);
            kt |= ((unsigned)(kv.x < b) | (unsigned)(kv.y < b) << 1 | (unsigned)(kv.z < b) << 2 |
                   (unsigned)(kv.w < b) << 3) << (u * V);
            zz[u * V] = zq.x;
            zz[u * V + 1] = zq.y;
            zz[u * V + 2] = zq.z;
            zz[u * V + 3] = zq.w;
        }
        kk = (1u << PER) - 1u;
    } else {
        const int c = e0 < n ? (int)(n - e0) : 0;
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const bool in = k < c;
            zz[k] = in ? z[e0 + k] : 0;
            kt |= (unsigned)(in && keys[e0 + k] < b) << k;
        }
        kk = (1u << c) - 1u;
    }
    // this thread's trues and kept before it in the tile: one warp scan, then the warps
    const unsigned x = (unsigned)__popc(kt) | ((unsigned)__popc(kk) << 16);
    unsigned y = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(FULL, y, d);
        if (l >= d) y += o;
    }
    if (l == 31) s_w[w] = y;
    __syncthreads();
    unsigned wpre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < TB / 32; i++) {
        const unsigned c = s_w[i];
        wpre += i < w ? c : 0u;
        tot += c;
    }
    const unsigned pre = wpre + y - x;
    unsigned rt = pre & 0xffffu, rk = pre >> 16;
    int tmn = INT32_MAX, tmx = INT32_MIN, fmn = INT32_MAX, fmx = INT32_MIN;
#pragma unroll
    for (int k = 0; k < PER; k++) {
        const bool kept = (kk >> k) & 1u;
        const bool tr = (kt >> k) & 1u;
        const int q = (int)((unsigned)zz[k] - (tr ? rt : rk - rt));
        tmn = (kept && tr) ? min(tmn, q) : tmn;
        tmx = (kept && tr) ? max(tmx, q) : tmx;
        fmn = (kept && !tr) ? min(fmn, q) : fmn;
        fmx = (kept && !tr) ? max(fmx, q) : fmx;
        rt += tr ? 1u : 0u;
        rk += kept ? 1u : 0u;
    }
    tmn = __reduce_min_sync(FULL, tmn);
    tmx = __reduce_max_sync(FULL, tmx);
    fmn = __reduce_min_sync(FULL, fmn);
    fmx = __reduce_max_sync(FULL, fmx);
    if (l == 0) {
        s_r[0][w] = tmn;
        s_r[1][w] = tmx;
        s_r[2][w] = fmn;
        s_r[3][w] = fmx;
    }
    __syncthreads();
    if (w == 0) {
        int a = l < TB / 32 ? s_r[0][l] : INT32_MAX, c = l < TB / 32 ? s_r[1][l] : INT32_MIN;
        int d = l < TB / 32 ? s_r[2][l] : INT32_MAX, e = l < TB / 32 ? s_r[3][l] : INT32_MIN;
        a = __reduce_min_sync(FULL, a);
        c = __reduce_max_sync(FULL, c);
        d = __reduce_min_sync(FULL, d);
        e = __reduce_max_sync(FULL, e);
        if (l == 0) {
            tile_prefix[t] = widen(tot);
            // (INT32_MAX, INT32_MIN): no element of the class
            rec[t] = make_longlong2(a > c ? FP_NONE : (a == c && a >= 0 ? (long long)a : FP_BAD),
                                    d > e ? FP_NONE : (d == e && d >= 0 ? (long long)d : FP_BAD));
        }
    }
}

// After the tile scan: a tile passes when its recorded constants are P_t and
// T + F_t; any failing tile, or a dropped Z inside [0, N), raises the flag that
// enables the exact pass.
__global__ void filtpart_decide_kernel(const unsigned long long *__restrict__ tp, const longlong2 *__restrict__ rec,
                                       int64_t nt, Hdr *h) {
    IXP_KERNEL_ENTRY();
    const int64_t T = (int64_t)(h->total & 0xffffffffull), N = (int64_t)(h->total >> 32);
    bool bad = false;
    if (blockIdx.x == 0 && threadIdx.x == 0) bad = dec_min(h->k_first2) < N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long p = __ldg(tp + t);
        const int64_t ct = (int64_t)(p & 0xffffffffull), cf = (int64_t)(p >> 32) - ct;
        const longlong2 r = rec[t];
        bad |= (r.x != FP_NONE && r.x != ct) || (r.y != FP_NONE && r.y != T + cf);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) h->flag = 1u;
}

__global__ void num_true_kernel(const unsigned long long *seg_cnt, const Hdr *h, int64_t nseg, int64_t *num_true) {
    IXP_KERNEL_ENTRY();
    if (nseg == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) num_true[0] = (int64_t)(h->total & 0xffffffffull);
        return;
    }
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nseg; k += (int64_t)gridDim.x * blockDim.x)
        num_true[k] = (int64_t)(seg_cnt[k + 1] & 0xffffffffull) - (int64_t)(seg_cnt[k] & 0xffffffffull);
}

// Pass 2 of the InvFiltPart check: compare Z with the expected destinations.
// With `witness` set, only the tile holding the first mismatch runs (grid of 1)
// and it stores that element's expected destination (+1, 0 for dropped) in k_aux.
template <typename KT, typename ZT, bool SEG>
__global__ void __launch_bounds__(TB, 4) filtpart_cmp_kernel(
    const ZT *__restrict__ z, int64_t n, const KT *__restrict__ keys, DPred filt, DPred part,
    const int64_t *__restrict__ off, int64_t nseg, const unsigned long long *__restrict__ tile_prefix,
    const unsigned long long *__restrict__ seg_cnt, Hdr *h, int vec_ok, int witness, int need_flag) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int TILE = TB * SUB * V;
    __shared__ unsigned s_w[TB / 32];
    __shared__ int s_rel[SEG ? TILE : 1];
    __shared__ int64_t s_k0;
    if (need_flag && !h->flag) return;
    int64_t t = blockIdx.x;
    int64_t target = -1;
    if (witness) {
        if (!h->k_first || h->status) return;
        target = dec_first(h->k_first);
        t = target / TILE;
    }
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned kt[SUB], kk[SUB];
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
        KT kv[V];
        load_slot<KT, V>(keys, p0, n, vec_ok, kv);
        kk[u] = pred_mask<KT, V>(filt, kv, p0, n);
        kt[u] = kk[u] & pred_mask<KT, V>(part, kv, p0, n);
    }
    unsigned pre[SUB];
    tile_counts<V>(kt, kk, pre, s_w);
    int rel[SUB][V];
    if (SEG) tile_segments<V>(off, nseg, t0, t1, s_rel, &s_k0, rel);
    const unsigned long long tp = tile_prefix[t];
    const int64_t Ntot = (int64_t)(h->total >> 32);
    const int64_t Ttot = (int64_t)(h->total & 0xffffffffull);
    int64_t bad = INT64_MAX;
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
#pragma unroll
        for (int k = 0; k < V; k++) {
            const int64_t i = p0 + k;
            if (i >= n) continue;
            const unsigned below = (1u << k) - 1u;
            const int64_t ct = (int64_t)(tp & 0xffffffffull) + (int64_t)(pre[u] & 0xffffu) + __popc(kt[u] & below);
            const int64_t ck = (int64_t)(tp >> 32) + (int64_t)(pre[u] >> 16) + __popc(kk[u] & below);
            const bool kept = (kk[u] >> k) & 1u, c = (kt[u] >> k) & 1u;
            int64_t ref = -1;
            if (kept) {
                int64_t Fk = 0, ctk = 0, ckk = 0, tk = Ttot;
                if (SEG) {
                    const int64_t sk = s_k0 + rel[u][k];
                    const unsigned long long a0 = __ldg(seg_cnt + sk), a1 = __ldg(seg_cnt + sk + 1);
                    ctk = (int64_t)(a0 & 0xffffffffull);
                    ckk = (int64_t)(a0 >> 32);
                    Fk = ckk;
                    tk = (int64_t)(a1 & 0xffffffffull) - ctk;
                }
                const int64_t tb = ct - ctk, kb = ck - ckk;  // trues / kept before i in its segment
                ref = c ? Fk + tb : Fk + tk + (kb - tb);
            }
            const int64_t zi = (int64_t)z[i];
            const bool wrong = kept ? (zi != ref) : (zi >= 0 && zi < Ntot);
            if (wrong) bad = i < bad ? i : bad;
            if (witness && i == target) h->cnt1 = (unsigned long long)(ref + 1);
        }
    }
    if (witness) return;
    __shared__ unsigned long long sm[TB / 32];
    unsigned long long r = block_max_u64(bad == INT64_MAX ? 0ull : enc_first(bad), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

// FiltPart value form: for every kept element i with expected destination
// ref(i) (as in filtpart_cmp_kernel) and ref(i) < ny, compare row X[i] with row
// Y[ref(i)] word by word; the smallest differing position and its source index are
// kept packed as (ref << 32) | i (n < 2^32), so one atomic max of the encoding
// keeps the lexicographically smallest pair.
template <typename KT, bool SEG>
__global__ void __launch_bounds__(TB, 4) filtpart_val_kernel(
    const uint32_t *__restrict__ y, int64_t ny, const uint32_t *__restrict__ x, int row_words, int64_t n,
    const KT *__restrict__ keys, DPred filt, DPred part, const int64_t *__restrict__ off, int64_t nseg,
    const unsigned long long *__restrict__ tile_prefix, const unsigned long long *__restrict__ seg_cnt, Hdr *h,
    int vec_ok) {
    IXP_KERNEL_ENTRY();
    constexpr int V = 16 / sizeof(KT);
    constexpr int TILE = TB * SUB * V;
    __shared__ unsigned s_w[TB / 32];
    __shared__ int s_rel[SEG ? TILE : 1];
    __shared__ int64_t s_k0;
    const int64_t t = blockIdx.x;
    const int64_t t0 = t * TILE, t1 = min(n, t0 + TILE);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    unsigned kt[SUB], kk[SUB];
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
        KT kv[V];
        load_slot<KT, V>(keys, p0, n, vec_ok, kv);
        kk[u] = pred_mask<KT, V>(filt, kv, p0, n);
        kt[u] = kk[u] & pred_mask<KT, V>(part, kv, p0, n);
    }
    unsigned pre[SUB];
    tile_counts<V>(kt, kk, pre, s_w);
    int rel[SUB][V];
    if (SEG) tile_segments<V>(off, nseg, t0, t1, s_rel, &s_k0, rel);
    const unsigned long long tp = tile_prefix[t];
    const int64_t Ttot = (int64_t)(h->total & 0xffffffffull);
    unsigned long long bad = ~0ull;
#pragma unroll
    for (int u = 0; u < SUB; u++) {
        const int64_t p0 = t0 + (int64_t)((w * SUB + u) * 32 + l) * V;
#pragma unroll
        for (int k = 0; k < V; k++) {
            const int64_t i = p0 + k;
            if (i >= n || !((kk[u] >> k) & 1u)) continue;
            const unsigned below = (1u << k) - 1u;
            const int64_t ct = (int64_t)(tp & 0xffffffffull) + (int64_t)(pre[u] & 0xffffu) + __popc(kt[u] & below);
            const int64_t ck = (int64_t)(tp >> 32) + (int64_t)(pre[u] >> 16) + __popc(kk[u] & below);
            const bool c = (kt[u] >> k) & 1u;
            int64_t Fk = 0, ctk = 0, ckk = 0, tk = Ttot;
            if (SEG) {
                const int64_t sk = s_k0 + rel[u][k];
                const unsigned long long a0 = __ldg(seg_cnt + sk), a1 = __ldg(seg_cnt + sk + 1);
                ctk = (int64_t)(a0 & 0xffffffffull);
                ckk = (int64_t)(a0 >> 32);
                Fk = ckk;
                tk = (int64_t)(a1 & 0xffffffffull) - ctk;
            }
            const int64_t tb = ct - ctk, kb = ck - ckk;  // trues / kept before i in its segment
            const int64_t ref = c ? Fk + tb : Fk + tk + (kb - tb);
            if (ref >= ny) continue;
            bool differ = false;
            for (int j = 0; j < row_words; j++)
                differ |= __ldg(x + i * row_words + j) != __ldg(y + ref * row_words + j);
            if (differ) {
                const unsigned long long pk = ((unsigned long long)ref << 32) | (unsigned long long)i;
                bad = pk < bad ? pk : bad;
            }
        }
    }
    __shared__ unsigned long long sm[TB / 32];
    const unsigned long long r = block_max_u64(bad == ~0ull ? 0ull : enc_first((int64_t)bad), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

// Class form of the value check: the destinations come from the class kernels
// (dest[i] >= 0 for kept i, -1 for dropped ones); compare as above.
__global__ void __launch_bounds__(256) filtpart_val_rows_kernel(const uint32_t *__restrict__ y, int64_t ny,
                                                                const uint32_t *__restrict__ x, int row_words,
                                                                int64_t n, const int64_t *__restrict__ dest, Hdr *h) {
    IXP_KERNEL_ENTRY();
    unsigned long long bad = ~0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ref = __ldg(dest + i);
        if (ref < 0 || ref >= ny) continue;
        bool differ = false;
        for (int j = 0; j < row_words; j++)
            differ |= __ldg(x + i * row_words + j) != __ldg(y + ref * row_words + j);
        if (differ) {
            const unsigned long long pk = ((unsigned long long)ref << 32) | (unsigned long long)i;
            bad = pk < bad ? pk : bad;
        }
    }
    __shared__ unsigned long long sm[256 / 32];
    const unsigned long long r = block_max_u64(bad == ~0ull ? 0ull : enc_first((int64_t)bad), sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

// Verdict of the value form. N = the kept count (the tile totals' upper half, or
// *kept for the class form); a Y whose length is not N is reported as such
// (index -1, value = ny); otherwise the smallest differing position of Y (index)
// and its source element (value).
__global__ void filtpart_val_finalize(const Hdr *h, const int64_t *kept, int64_t ny, ixp_verdict *out) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    v.status = h->status;
    v.reserved = 0;
    const int64_t N = kept ? *kept : (int64_t)(h->total >> 32);
    v.aux0 = N;
    v.aux1 = 0;
    v.ok = 1;
    v.kind = IXP_V_NONE;
    v.index = -1;
    v.value = 0;
    if (v.status) {
        v.ok = -1;
    } else if (ny != N) {
        v.ok = 0;
        v.kind = IXP_V_WRONG_DEST;
        v.value = ny;
    } else if (h->k_first) {
        const unsigned long long pk = (unsigned long long)dec_first(h->k_first);
        v.ok = 0;
        v.kind = IXP_V_WRONG_DEST;
        v.index = (int64_t)(pk >> 32);
        v.value = (int64_t)(pk & 0xffffffffull);
    }
    *out = v;
}

template <typename ZT>
__global__ void filtpart_finalize(const ZT *z, const Hdr *h, ixp_verdict *out) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    v.status = h->status;
    v.reserved = 0;
    const int64_t i = h->k_first ? dec_first(h->k_first) : -1;
    v.ok = v.status ? -1 : (i < 0 ? 1 : 0);
    v.kind = (v.status || i < 0) ? IXP_V_NONE : IXP_V_WRONG_DEST;
    v.index = v.status ? -1 : i;
    v.value = (v.status || i < 0) ? 0 : (int64_t)z[i];
    v.aux0 = (int64_t)(h->total >> 32);
    v.aux1 = (v.status || i < 0) ? 0 : (int64_t)h->cnt1 - 1;
    *out = v;
}

// ============================================================== mkSgmDescr

__global__ void shape_check_kernel(const int64_t *shape, int64_t m, int32_t *status) {
    IXP_KERNEL_ENTRY();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        if (shape[k] < 0) atomicCAS(status, 0, IXP_E_INVAL);
}

template <typename OT>
__global__ void flags_scatter_kernel(const int64_t *shape, const int64_t *xs, const int64_t *offs, int64_t m,
                                     OT *out, int64_t out_len, const int32_t *status) {
    IXP_KERNEL_ENTRY();
    if (*status) return;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = offs[k];
        if (shape[k] > 0 && e >= 0 && e < out_len) out[e] = (OT)(xs ? xs[k] : 1);
    }
}

__global__ void status_copy_kernel(const Hdr *h, int32_t *d_status) {
    IXP_KERNEL_ENTRY();
    if (h->status) atomicCAS(d_status, 0, h->status);
}

// ================================================================ host side



static int64_t ntiles_for(int64_t n, int V) { return (n + (int64_t)TB * SUB * V - 1) / ((int64_t)TB * SUB * V); }

// Workspace layout for the tiled passes (all offsets 256-aligned):
//   header | status {u64, u64}[T] | tile_prefix u64[T] | seg_cnt u64[nseg+1]
struct TileWs {
    Hdr *h;
    Lookback L;
    unsigned long long *tile_prefix;
    unsigned long long *seg_cnt;
    unsigned long long *gtot;  // per group of TS_G tiles
    int64_t *tile_lb;          // per tile: first k with off[k] >= the tile's first element
    size_t bytes;
};


static TileWs tile_ws(void *ws, int64_t ntiles, int64_t nseg) {
    TileWs r;
    char *p = (char *)ws;
    size_t o = HDR_BYTES;
    r.h = (Hdr *)p;
    r.L.st = (ulonglong2 *)(p + o);
    o += round256((size_t)ntiles * 16);
    r.tile_prefix = (unsigned long long *)(p + o);
    o += round256((size_t)ntiles * 8);
    r.seg_cnt = (unsigned long long *)(p + o);
    o += round256((size_t)(nseg + 1) * 8);
    r.gtot = (unsigned long long *)(p + o);
    o += round256((size_t)((ntiles + TS_G - 1) / TS_G + 1) * 8);
    r.tile_lb = (int64_t *)(p + o);
    o += nseg > 0 ? round256((size_t)(ntiles + 1) * 8) : 0;
    r.bytes = o;
    return r;
}

size_t tiled_ws_bytes(int64_t n, int V, int64_t nseg) {
    int64_t nt = ntiles_for(n, V);
    return tile_ws(nullptr, nt, nseg < 0 ? 0 : nseg).bytes;
}



// Segmented scan over TMA-staged tiles (16-byte aligned input and output).
template <typename TI, typename TO, bool FLAGS>
static void launch_sgm_tma(const TI *in, TO *out, int64_t n, int inclusive, const uint8_t *flags, const int64_t *off,
                           int64_t nseg, const TileWs &W, Wait wt, cudaStream_t st) {
    constexpr int64_t tile = TMA_TILE_BYTES / (int64_t)sizeof(TI);
    const int64_t ntma = (n + tile - 1) / tile;
    cudaFuncSetAttribute(sgm_tma_kernel<TI, TO, FLAGS>, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_TILE_BYTES);
    sgm_tma_kernel<TI, TO, FLAGS><<<(unsigned)ntma, TMA_NT, TMA_TILE_BYTES, st>>>(in, out, n, inclusive, flags, off,
                                                                                nseg, W.L, W.h, wt);
}

template <typename TI, typename TO>
static int run_scan(const TI *in, TO *out, int64_t n, int inclusive, ixp_segs segs, TO *tot, int32_t *d_status,
                    void *ws, size_t ws_bytes, cudaStream_t st, bool keep_status = false) {
    constexpr int V = 16 / sizeof(TI);
    const bool seg = segs.offsets != nullptr;
    const int64_t nt = ntiles_for(n, V);
    TileWs W = tile_ws(ws, nt, seg ? segs.nseg : 0);
    int rc = check_ws(ws, ws_bytes, W.bytes);
    if (rc) return rc;
    if (cudaMemsetAsync(ws, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (nt > 0 && cudaMemsetAsync(W.L.st, 0, (size_t)nt * 16, st) != cudaSuccess) return IXP_E_CUDA;
    if (d_status && !keep_status && cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return IXP_E_CUDA;
    if (!seg && tot && n == 0 && cudaMemsetAsync(tot, 0, sizeof(TO), st) != cudaSuccess) return IXP_E_CUDA;
    const int vec = aligned16(in) && aligned16(out);
    const Wait wt = wait_config();
    if (nt > 0) {
        if (seg && vec)
            launch_sgm_tma<TI, TO, false>(in, out, n, inclusive, nullptr, segs.offsets, segs.nseg, W, wt, st);
        else if (seg)
            scan_kernel<TI, TO, true><<<(unsigned)nt, TB, 0, st>>>(in, out, n, inclusive, segs.offsets, segs.nseg,
                                                                  W.L, W.h, wt, nullptr, vec);
        else if (vec) {
            constexpr int64_t tile = SCAN_TILE_BYTES / (int64_t)sizeof(TI);
            const int64_t ntma = (n + tile - 1) / tile;
            cudaFuncSetAttribute(scan_tma_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SCAN_TILE_BYTES);
            scan_tma_kernel<TI, TO><<<(unsigned)ntma, TMA_NT, SCAN_TILE_BYTES, st>>>(in, out, n, inclusive, W.L, W.h,
                                                                                   wt, tot);
        } else
            scan_flat_kernel<TI, TO><<<(unsigned)nt, TB, 0, st>>>(in, out, n, inclusive, W.L, W.h, wt, tot, vec);
    }
    if (seg && tot && segs.nseg > 0) {
        int g = (int)std::min<int64_t>((segs.nseg + 255) / 256, 4096);
        seg_totals_kernel<TI, TO><<<g, 256, 0, st>>>(in, out, segs.offsets, segs.nseg, n, inclusive, tot);
    }
    if (d_status) status_copy_kernel<<<1, 1, 0, st>>>(W.h, d_status);
    return launch_status();
}

// Exclusive scan of the packed tile counts (h->total gets the sum; it stays 0
// from the header reset when there are no tiles).
static void scan_tiles(TileWs &W, int64_t nt, cudaStream_t st) { scan_tile_counts(W.tile_prefix, nt, W.gtot, W.h, st); }

template <typename KT>
static int run_counts(const KT *keys, int64_t n, DPred filt, DPred part, ixp_segs segs, TileWs &W, int64_t nt,
                      int vec, cudaStream_t st) {
    constexpr int V = 16 / sizeof(KT);
    const bool seg = segs.offsets != nullptr;
    if (cudaMemsetAsync(W.h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (nt > 0) {
        if (seg) {
            // first segment index per tile, from one pass over the offsets (0 fills
            // what invalid offsets leave unset)
            if (cudaMemsetAsync(W.tile_lb, 0, (size_t)(nt + 1) * 8, st) != cudaSuccess) return IXP_E_CUDA;
            const int g = (int)std::max<int64_t>(1, std::min<int64_t>((segs.nseg + 256) / 256, 4096));
            chunk_lb_kernel<TB * SUB * V><<<g, 256, 0, st>>>(segs.offsets, segs.nseg, n, W.tile_lb);
            count_seg_kernel<KT><<<(unsigned)nt, TB, 0, st>>>(keys, n, filt, part, segs.offsets, segs.nseg,
                                                             W.tile_lb, W.tile_prefix, W.seg_cnt, vec);
        }
        else
            count_tiles_kernel<KT><<<(unsigned)((nt + CT - 1) / CT), TB, 0, st>>>(keys, n, filt, part, nt,
                                                                                W.tile_prefix, vec);
    }
    scan_tiles(W, nt, st);
    if (seg) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((segs.nseg + 256) / 256, 4096));
        seg_fix_kernel<TB * SUB * V><<<g, 256, 0, st>>>(segs.offsets, segs.nseg, n, W.tile_prefix, W.seg_cnt, W.h);
    }
    return IXP_OK;
}

template <typename KT, typename OT>
static int run_partition(const KT *keys, int64_t n, ixp_pred pred, const void *payload, int row_bytes, OT *out_idx,
                         KT *out_keys, void *out_payload, int64_t *num_true, ixp_segs segs, int32_t *d_status,
                         void *ws, size_t ws_bytes, cudaStream_t st) {
    constexpr int V = 16 / sizeof(KT);
    const bool seg = segs.offsets != nullptr;
    const int64_t nt = ntiles_for(n, V);
    TileWs W = tile_ws(ws, nt, seg ? segs.nseg : 0);
    int rc = check_ws(ws, ws_bytes, W.bytes);
    if (rc) return rc;
    const int vec = (keys == nullptr || aligned16(keys)) && aligned16(out_idx);
    const DPred all{IXP_P_TRUE, 0, 0, nullptr};
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return IXP_E_CUDA;
    rc = run_counts<KT>(keys, n, all, dpred(pred), segs, W, nt, vec, st);
    if (rc) return rc;
    if (nt > 0 && !seg && (!out_payload || row_bytes == 4)) {
        // 16-byte stores of the payload and key runs need 16-byte aligned outputs
        const int vec_ok = vec && (!out_payload || aligned16(out_payload)) && (!out_keys || aligned16(out_keys));
        const int bulk_ok = (!keys || aligned16(keys)) && (!out_payload || aligned16(payload));
        const Wait wt = wait_config();
        if (vec_ok && out_keys) {
            cudaFuncSetAttribute(partition_flat_kernel<KT, OT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pf_smem_bytes<KT>(true));
            partition_flat_kernel<KT, OT, true><<<(unsigned)nt, TB, pf_smem_bytes<KT>(true), st>>>(
                keys, n, dpred(pred), out_payload ? (const uint32_t *)payload : nullptr, out_idx, out_keys,
                (uint32_t *)out_payload, W.tile_prefix, W.h, vec_ok, bulk_ok, wt);
        } else if (vec_ok) {
            cudaFuncSetAttribute(partition_flat_kernel<KT, OT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pf_smem_bytes<KT>(false));
            partition_flat_kernel<KT, OT, false><<<(unsigned)nt, TB, pf_smem_bytes<KT>(false), st>>>(
                keys, n, dpred(pred), out_payload ? (const uint32_t *)payload : nullptr, out_idx, nullptr,
                (uint32_t *)out_payload, W.tile_prefix, W.h, vec_ok, bulk_ok, wt);
        } else {
            partition_write_kernel<KT, OT, false><<<(unsigned)nt, TB, 0, st>>>(
                keys, n, dpred(pred), (const uint32_t *)payload, row_bytes / 4, out_idx, out_keys,
                (uint32_t *)out_payload, nullptr, 0, W.tile_prefix, nullptr, W.h, vec);
        }
    } else if (nt > 0) {
        if (seg)
        {
            const int v2 = vec && (!out_idx || aligned16(out_idx));
            if (n <= INT32_MAX)
                partition_seg_kernel<KT, OT, int32_t><<<(unsigned)nt, TB, 0, st>>>(
                    keys, n, dpred(pred), (const uint32_t *)payload, row_bytes / 4, out_idx, out_keys,
                    (uint32_t *)out_payload, segs.offsets, segs.nseg, W.tile_lb, W.tile_prefix, W.seg_cnt, v2);
            else
                partition_seg_kernel<KT, OT, int64_t><<<(unsigned)nt, TB, 0, st>>>(
                    keys, n, dpred(pred), (const uint32_t *)payload, row_bytes / 4, out_idx, out_keys,
                    (uint32_t *)out_payload, segs.offsets, segs.nseg, W.tile_lb, W.tile_prefix, W.seg_cnt, v2);
        }
        else
            partition_write_kernel<KT, OT, false><<<(unsigned)nt, TB, 0, st>>>(
                keys, n, dpred(pred), (const uint32_t *)payload, row_bytes / 4, out_idx, out_keys,
                (uint32_t *)out_payload, nullptr, 0, W.tile_prefix, nullptr, W.h, vec);
    }
    const int64_t ns = seg ? segs.nseg : 0;
    int g = (int)std::max<int64_t>(1, std::min<int64_t>((ns + 255) / 256, 4096));
    num_true_kernel<<<g, 256, 0, st>>>(W.seg_cnt, W.h, ns, num_true);
    if (d_status) status_copy_kernel<<<1, 1, 0, st>>>(W.h, d_status);
    return launch_status();
}

template <typename KT, typename ZT>
static int run_filtpart(const ZT *z, int64_t n, const KT *keys, ixp_pred filt, ixp_pred part, ixp_segs segs,
                        ixp_verdict *out, void *ws, size_t ws_bytes, cudaStream_t st) {
    constexpr int V = 16 / sizeof(KT);
    const bool seg = segs.offsets != nullptr;
    const int64_t nt = ntiles_for(n, V);
    TileWs W = tile_ws(ws, nt, seg ? segs.nseg : 0);
    int rc = check_ws(ws, ws_bytes, W.bytes);
    if (rc) return rc;
    const int vec = keys == nullptr || aligned16(keys);
    if (!seg) {
        if (cudaMemsetAsync(W.h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
        if (nt > 0) {
            longlong2 *rec = reinterpret_cast<longlong2 *>(W.L.st);
            bool narrow = false;
            if constexpr (sizeof(ZT) == 4 && sizeof(KT) == 4) {
                // the common form: filter TRUE, predicate key < b, aligned int32 arrays
                if (n <= INT32_MAX && filt.kind == IXP_P_TRUE && part.kind == IXP_P_LT && keys && aligned16(keys) &&
                    aligned16(z) && part.b > (long long)INT32_MIN && part.b <= (long long)INT32_MAX) {
                    narrow = true;
                    filtpart_tile_lt_kernel<<<(unsigned)nt, TB, 0, st>>>((const int32_t *)z, n,
                                                                         (const int32_t *)keys, (int32_t)part.b,
                                                                         W.tile_prefix, rec);
                }
            }
            if constexpr (sizeof(ZT) == 4) {
                if (!narrow && n <= INT32_MAX) {
                    narrow = true;
                    filtpart_tile_kernel<KT, ZT, int32_t><<<(unsigned)nt, TB, 0, st>>>(
                        z, n, keys, dpred(filt), dpred(part), W.tile_prefix, rec, W.h, vec);
                }
            }
            if (!narrow)
                filtpart_tile_kernel<KT, ZT, int64_t><<<(unsigned)nt, TB, 0, st>>>(z, n, keys, dpred(filt),
                                                                              dpred(part), W.tile_prefix, rec, W.h,
                                                                              vec);
            scan_tiles(W, nt, st);
            const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nt + 255) / 256, 1024));
            filtpart_decide_kernel<<<g, 256, 0, st>>>(W.tile_prefix, rec, nt, W.h);
            filtpart_cmp_kernel<KT, ZT, false><<<(unsigned)nt, TB, 0, st>>>(
                z, n, keys, dpred(filt), dpred(part), nullptr, 0, W.tile_prefix, nullptr, W.h, vec, 0, 1);
            filtpart_cmp_kernel<KT, ZT, false><<<1, TB, 0, st>>>(z, n, keys, dpred(filt), dpred(part), nullptr, 0,
                                                                W.tile_prefix, nullptr, W.h, vec, 1, 1);
        }
        filtpart_finalize<ZT><<<1, 1, 0, st>>>(z, W.h, out);
        return launch_status();
    }
    rc = run_counts<KT>(keys, n, dpred(filt), dpred(part), segs, W, nt, vec, st);
    if (rc) return rc;
    if (nt > 0) {
        if (n <= INT32_MAX)
            filtpart_seg_kernel<KT, ZT, int32_t><<<(unsigned)nt, TB, 0, st>>>(
                z, n, keys, dpred(filt), dpred(part), segs.offsets, segs.nseg, W.tile_lb, W.tile_prefix, W.seg_cnt,
                W.h, vec);
        else
            filtpart_seg_kernel<KT, ZT, int64_t><<<(unsigned)nt, TB, 0, st>>>(
                z, n, keys, dpred(filt), dpred(part), segs.offsets, segs.nseg, W.tile_lb, W.tile_prefix, W.seg_cnt,
                W.h, vec);
        filtpart_cmp_kernel<KT, ZT, true><<<1, TB, 0, st>>>(z, n, keys, dpred(filt), dpred(part), segs.offsets,
                                                           segs.nseg, W.tile_prefix, W.seg_cnt, W.h, vec, 1, 0);
    }
    filtpart_finalize<ZT><<<1, 1, 0, st>>>(z, W.h, out);
    return launch_status();
}

// Workspace of the value form: the predicate form uses the tiled layout (sized for
// int64 keys, which have the most tiles); the class form adds the destinations
// (int64 per element) and the kept count to the class kernels' workspace.
size_t filtpart_classes_ws_bytes(int v, int64_t n, int64_t nseg);  // classes.cu
size_t filtpart_values_ws_bytes(int v, int64_t n, int64_t nseg) {
    if (v <= 0) return tiled_ws_bytes(n, 2, nseg);
    return filtpart_classes_ws_bytes(v, n, nseg) + round256((size_t)(n > 0 ? n : 0) * 8) + 256;
}

template <typename KT>
static int run_filtpart_values(const uint32_t *y, int64_t ny, const uint32_t *x, int row_words, int64_t n,
                               const KT *keys, ixp_pred filt, ixp_pred part, ixp_segs segs, ixp_verdict *out,
                               void *ws, size_t ws_bytes, cudaStream_t st) {
    constexpr int V = 16 / sizeof(KT);
    const bool seg = segs.offsets != nullptr;
    const int64_t nt = ntiles_for(n, V);
    TileWs W = tile_ws(ws, nt, seg ? segs.nseg : 0);
    int rc = check_ws(ws, ws_bytes, W.bytes);
    if (rc) return rc;
    const int vec = keys == nullptr || aligned16(keys);
    rc = run_counts<KT>(keys, n, dpred(filt), dpred(part), segs, W, nt, vec, st);
    if (rc) return rc;
    if (nt > 0) {
        if (seg)
            filtpart_val_kernel<KT, true><<<(unsigned)nt, TB, 0, st>>>(y, ny, x, row_words, n, keys, dpred(filt),
                                                                      dpred(part), segs.offsets, segs.nseg,
                                                                      W.tile_prefix, W.seg_cnt, W.h, vec);
        else
            filtpart_val_kernel<KT, false><<<(unsigned)nt, TB, 0, st>>>(y, ny, x, row_words, n, keys, dpred(filt),
                                                                       dpred(part), nullptr, 0, W.tile_prefix,
                                                                       nullptr, W.h, vec);
    }
    filtpart_val_finalize<<<1, 1, 0, st>>>(W.h, nullptr, ny, out);
    return launch_status();
}

static int run_filtpart_values_classes(const uint32_t *y, int64_t ny, const uint32_t *x, int row_words, int64_t n,
                                       const void *keys, int ktype, ixp_pred filt, const uint8_t *cls, int v,
                                       ixp_segs segs, ixp_verdict *out, void *ws, size_t ws_bytes, cudaStream_t st) {
    const size_t cb = filtpart_classes_ws_bytes(v, n, segs.offsets ? segs.nseg : 0);
    int rc = check_ws(ws, ws_bytes, filtpart_values_ws_bytes(v, n, segs.offsets ? segs.nseg : 0));
    if (rc) return rc;
    // layout: the class kernels' workspace | destinations (int64 per element) | kept count
    int64_t *dest = (int64_t *)((char *)ws + cb);
    int64_t *kept = (int64_t *)((char *)ws + cb + round256((size_t)(n > 0 ? n : 0) * 8));
    rc = ixp_filtpart_classes(keys, ktype, n, filt, cls, v, segs, n > 0 ? dest : nullptr, IXP_I64, kept, ws, cb,
                              (ixp_stream)st);
    if (rc) return rc;
    // the class kernels are done with their workspace (same stream): its start holds the header now
    Hdr *hh = (Hdr *)ws;
    if (cudaMemsetAsync(hh, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (n > 0) {
        const int g = stream_grid(n, 1);
        filtpart_val_rows_kernel<<<g, 256, 0, st>>>(y, ny, x, row_words, n, dest, hh);
    }
    filtpart_val_finalize<<<1, 1, 0, st>>>(hh, kept, ny, out);
    return launch_status();
}

}  // namespace ixp

using namespace ixp;

extern "C" int ixp_check_filtpart_values(const void *y, int64_t ny, const void *x, int64_t n, int32_t row_bytes,
                                         const void *keys, int ktype, ixp_pred filt, ixp_pred part,
                                         const uint8_t *cls, int32_t v, ixp_segs segs, ixp_verdict *d_verdict,
                                         void *ws, size_t ws_bytes, ixp_stream stream) {
    if (keys && ktype != IXP_I32 && ktype != IXP_I64) return IXP_E_DTYPE;
    if (n < 0 || ny < 0 || row_bytes <= 0 || row_bytes % 4 || !d_verdict || n >= (1ll << 32)) return IXP_E_INVAL;
    if ((n > 0 && !x) || (ny > 0 && !y) || !aligned_to(x, 4) || !aligned_to(y, 4)) return IXP_E_INVAL;
    if ((segs.offsets && segs.nseg < 1) || (!segs.offsets && segs.nseg != 0)) return IXP_E_INVAL;
    // the class form: a class array, or, for an empty input (whose arrays may be
    // NULL), any v other than the predicate form's 2
    const bool classes = cls != nullptr || (n == 0 && v != 2);
    if (classes ? (v < 1 || v > 256) : v != 2) return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {  // N = 0: only the length of Y can be wrong
        const int rc = check_ws(ws, ws_bytes, HDR_BYTES);
        if (rc) return rc;
        if (cudaMemsetAsync(ws, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
        filtpart_val_finalize<<<1, 1, 0, st>>>((const Hdr *)ws, nullptr, ny, d_verdict);
        return launch_status();
    }
    const uint32_t *yw = (const uint32_t *)y, *xw = (const uint32_t *)x;
    const int words = row_bytes / 4;
    if (classes) return run_filtpart_values_classes(yw, ny, xw, words, n, keys, ktype, filt, cls, v, segs, d_verdict, ws,
                                                ws_bytes, st);
    if (!keys || ktype == IXP_I32)
        return run_filtpart_values(yw, ny, xw, words, n, (const int32_t *)keys, filt, part, segs, d_verdict, ws,
                                   ws_bytes, st);
    return run_filtpart_values(yw, ny, xw, words, n, (const int64_t *)keys, filt, part, segs, d_verdict, ws, ws_bytes,
                               st);
}

extern "C" int ixp_scan(const void *in, int in_type, void *out, int out_type, int64_t n, int inclusive, ixp_segs segs,
                        void *d_totals, int32_t *d_status, void *ws, size_t ws_bytes, ixp_stream stream) {
    if ((in_type != IXP_I32 && in_type != IXP_I64) || (out_type != IXP_I32 && out_type != IXP_I64) ||
        (in_type == IXP_I64 && out_type == IXP_I32))
        return IXP_E_DTYPE;
    if (n < 0 || (n > 0 && (!in || !out))) return IXP_E_INVAL;
    if ((segs.offsets && segs.nseg < 1) || (!segs.offsets && segs.nseg != 0)) return IXP_E_INVAL;
    const int es = in_type == IXP_I32 ? 4 : 8, eo = out_type == IXP_I32 ? 4 : 8;
    if ((reinterpret_cast<uintptr_t>(in) % es) || (reinterpret_cast<uintptr_t>(out) % eo)) return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (in_type == IXP_I32 && out_type == IXP_I32)
        return run_scan((const int32_t *)in, (int32_t *)out, n, inclusive, segs, (int32_t *)d_totals, d_status, ws,
                        ws_bytes, st);
    if (in_type == IXP_I32)
        return run_scan((const int32_t *)in, (int64_t *)out, n, inclusive, segs, (int64_t *)d_totals, d_status, ws,
                        ws_bytes, st);
    return run_scan((const int64_t *)in, (int64_t *)out, n, inclusive, segs, (int64_t *)d_totals, d_status, ws,
                    ws_bytes, st);
}

extern "C" int ixp_sgm_scan(const uint8_t *flags, const void *in, int in_type, void *out, int out_type, int64_t n,
                            int inclusive, int32_t *d_status, void *ws, size_t ws_bytes, ixp_stream stream) {
    if ((in_type != IXP_I32 && in_type != IXP_I64) || (out_type != IXP_I32 && out_type != IXP_I64))
        return IXP_E_DTYPE;
    if (in_type == IXP_I64 && out_type == IXP_I32) return IXP_E_DTYPE;
    if (n < 0 || (n > 0 && (!flags || !in || !out))) return IXP_E_INVAL;
    const int es = in_type == IXP_I32 ? 4 : 8, eo = out_type == IXP_I32 ? 4 : 8;
    if ((reinterpret_cast<uintptr_t>(in) % es) || (reinterpret_cast<uintptr_t>(out) % eo)) return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int V = in_type == IXP_I32 ? 4 : 2;
    const int64_t nt = ntiles_for(n, V);
    TileWs W = tile_ws(ws, nt, 0);
    int rc = check_ws(ws, ws_bytes, W.bytes);
    if (rc) return rc;
    if (cudaMemsetAsync(ws, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (nt > 0 && cudaMemsetAsync(W.L.st, 0, (size_t)nt * 16, st) != cudaSuccess) return IXP_E_CUDA;
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return IXP_E_CUDA;
    const Wait wt = wait_config();
    if (nt > 0) {
        const bool vec = aligned16(in) && aligned16(out);
#define IXP_SGM(TI, TO)                                                                                           \
    do {                                                                                                          \
        if (vec)                                                                                                  \
            launch_sgm_tma<TI, TO, true>((const TI *)in, (TO *)out, n, inclusive, flags, nullptr, 0, W, wt, st);  \
        else                                                                                                      \
            scan_kernel<TI, TO, true><<<(unsigned)nt, TB, 0, st>>>((const TI *)in, (TO *)out, n, inclusive,       \
                                                                   nullptr, 0, W.L, W.h, wt, nullptr, 0, flags); \
    } while (0)
        if (in_type == IXP_I32 && out_type == IXP_I32) IXP_SGM(int32_t, int32_t);
        else if (in_type == IXP_I32) IXP_SGM(int32_t, int64_t);
        else IXP_SGM(int64_t, int64_t);
#undef IXP_SGM
    }
    if (d_status) status_copy_kernel<<<1, 1, 0, st>>>(W.h, d_status);
    return launch_status();
}

extern "C" int ixp_partition(const void *keys, int ktype, int64_t n, ixp_pred pred, const void *payload,
                             int32_t row_bytes, void *out_indices, int out_type, void *out_keys, void *out_payload,
                             int64_t *d_num_true, ixp_segs segs, int32_t *d_status, void *ws, size_t ws_bytes,
                             ixp_stream stream) {
    if ((keys && ktype != IXP_I32 && ktype != IXP_I64) || (out_type != IXP_I32 && out_type != IXP_I64))
        return IXP_E_DTYPE;
    if (n < 0 || n >= (1ll << 32) || !d_num_true || !pred_ok(pred, keys != nullptr || n == 0))
        return IXP_E_INVAL;
    if (out_type == IXP_I32 && n > INT32_MAX) return IXP_E_INVAL;
    if ((out_keys && !keys) || (out_payload && (!payload || row_bytes <= 0 || row_bytes % 4 || row_bytes > 64)))
        return IXP_E_INVAL;
    if ((segs.offsets && segs.nseg < 1) || (!segs.offsets && segs.nseg != 0)) return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool k64 = keys && ktype == IXP_I64;
    if (!k64) {
        if (out_type == IXP_I32)
            return run_partition((const int32_t *)keys, n, pred, payload, row_bytes, (int32_t *)out_indices,
                                 (int32_t *)out_keys, out_payload, d_num_true, segs, d_status, ws, ws_bytes, st);
        return run_partition((const int32_t *)keys, n, pred, payload, row_bytes, (int64_t *)out_indices,
                             (int32_t *)out_keys, out_payload, d_num_true, segs, d_status, ws, ws_bytes, st);
    }
    if (out_type == IXP_I32)
        return run_partition((const int64_t *)keys, n, pred, payload, row_bytes, (int32_t *)out_indices,
                             (int64_t *)out_keys, out_payload, d_num_true, segs, d_status, ws, ws_bytes, st);
    return run_partition((const int64_t *)keys, n, pred, payload, row_bytes, (int64_t *)out_indices,
                         (int64_t *)out_keys, out_payload, d_num_true, segs, d_status, ws, ws_bytes, st);
}

extern "C" int ixp_check_filtpart(const void *z, int ztype, int64_t n, const void *keys, int ktype, ixp_pred filt,
                                  ixp_pred part, ixp_segs segs, ixp_verdict *d_verdict, void *ws, size_t ws_bytes,
                                  ixp_stream stream) {
    if ((ztype != IXP_I32 && ztype != IXP_I64) || (keys && ktype != IXP_I32 && ktype != IXP_I64)) return IXP_E_DTYPE;
    if (n < 0 || n >= (1ll << 32) || (n > 0 && !z) || !d_verdict) return IXP_E_INVAL;
    if (!pred_ok(filt, keys != nullptr || n == 0) || !pred_ok(part, keys != nullptr || n == 0)) return IXP_E_INVAL;
    if ((segs.offsets && segs.nseg < 1) || (!segs.offsets && segs.nseg != 0)) return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool k64 = keys && ktype == IXP_I64;
    if (!k64) {
        if (ztype == IXP_I32)
            return run_filtpart((const int32_t *)z, n, (const int32_t *)keys, filt, part, segs, d_verdict, ws, ws_bytes,
                                st);
        return run_filtpart((const int64_t *)z, n, (const int32_t *)keys, filt, part, segs, d_verdict, ws, ws_bytes,
                            st);
    }
    if (ztype == IXP_I32)
        return run_filtpart((const int32_t *)z, n, (const int64_t *)keys, filt, part, segs, d_verdict, ws, ws_bytes,
                            st);
    return run_filtpart((const int64_t *)z, n, (const int64_t *)keys, filt, part, segs, d_verdict, ws, ws_bytes, st);
}

extern "C" int ixp_flags_from_shape(const int64_t *shape, int64_t m, const int64_t *xs, void *out, int out_type,
                                    int64_t out_len, int64_t *d_offsets, int32_t *d_status, void *ws, size_t ws_bytes,
                                    ixp_stream stream) {
    if (out_type != IXP_I32 && out_type != IXP_I64) return IXP_E_DTYPE;
    if (m < 0 || (m > 0 && !shape) || out_len < 0 || (out_len > 0 && !out) || !d_offsets || !d_status)
        return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // scan workspace first, then nothing else is needed (offsets live in d_offsets)
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return IXP_E_CUDA;
    int g = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 4096));
    if (m > 0) shape_check_kernel<<<g, 256, 0, st>>>(shape, m, d_status);
    const ixp_segs flat{nullptr, 0};
    int rc = run_scan(shape, d_offsets, m, 0, flat, d_offsets + m, d_status, ws, ws_bytes, st, true);
    if (rc) return rc;
    if (out_len > 0) {
        const size_t es = out_type == IXP_I32 ? 4 : 8;
        if (cudaMemsetAsync(out, 0, (size_t)out_len * es, st) != cudaSuccess) return IXP_E_CUDA;
        if (m > 0) {
            if (out_type == IXP_I32)
                flags_scatter_kernel<int32_t><<<g, 256, 0, st>>>(shape, xs, d_offsets, m, (int32_t *)out, out_len,
                                                                 d_status);
            else
                flags_scatter_kernel<int64_t><<<g, 256, 0, st>>>(shape, xs, d_offsets, m, (int64_t *)out, out_len,
                                                                 d_status);
        }
    }
    return launch_status();
}

// ---------------------------------------------------------------- no-alloc scan
// A flat scan whose scratch (the call header and one 16-byte look-back status per
// tile) lives in a fixed array in this library's own device memory instead of a
// caller-provided workspace. The array is reached from host code only through the
// address cudaGetSymbolAddress returns for the current device; the symbol itself is
// a host-side stand-in.
constexpr int64_t NOALLOC_MAX_TILES = 16384;
static __device__ __align__(256) unsigned char g_noalloc_scratch[HDR_BYTES + NOALLOC_MAX_TILES * 16];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_addr[256] = {};

// First call on a device: look up the array's device address with that device
// current and remember it. Returns nullptr on failure.
void *noalloc_scratch_for_current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
        g_noalloc_addr[dev] = p;
    }
    return g_noalloc_addr[dev];
}

template <typename TI, typename TO>
int run_scan_noalloc(const TI *in, TO *out, int64_t n, int inclusive, TO *tot, int32_t *d_status, cudaStream_t st) {
    constexpr int V = 16 / sizeof(TI);
    const int64_t nt = ntiles_for(n, V);
    if (nt > NOALLOC_MAX_TILES) return IXP_E_INVAL;
    void *base = noalloc_scratch_for_current_device();
    if (!base) return IXP_E_CUDA;
    Hdr *h = (Hdr *)base;
    Lookback L;
    L.st = (ulonglong2 *)((char *)base + HDR_BYTES);
    // the array keeps the previous call's contents: clear the header and the statuses used
    if (cudaMemsetAsync(h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (nt > 0 && cudaMemsetAsync(L.st, 0, (size_t)nt * 16, st) != cudaSuccess) return IXP_E_CUDA;
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(int32_t), st) != cudaSuccess) return IXP_E_CUDA;
    if (tot && n == 0 && cudaMemsetAsync(tot, 0, sizeof(TO), st) != cudaSuccess) return IXP_E_CUDA;
    const int vec = aligned16(in) && aligned16(out);
    if (nt > 0)
        scan_flat_kernel<TI, TO><<<(unsigned)nt, TB, 0, st>>>(in, out, n, inclusive, L, h, wait_config(), tot, vec);
    if (d_status) status_copy_kernel<<<1, 1, 0, st>>>(h, d_status);
    return launch_status();
}
}  // namespace

extern "C" int64_t ixp_scan_noalloc_max_n(int in_type) {
    const int V = in_type == IXP_I64 ? 2 : 4;
    return NOALLOC_MAX_TILES * (int64_t)TB * SUB * V;
}

extern "C" int ixp_scan_noalloc(const void *in, int in_type, void *out, int out_type, int64_t n, int inclusive,
                                void *d_totals, int32_t *d_status, ixp_stream stream) {
    if ((in_type != IXP_I32 && in_type != IXP_I64) || (out_type != IXP_I32 && out_type != IXP_I64) ||
        (in_type == IXP_I64 && out_type == IXP_I32))
        return IXP_E_DTYPE;
    if (n < 0 || (n > 0 && (!in || !out))) return IXP_E_INVAL;
    if (n > ixp_scan_noalloc_max_n(in_type)) return IXP_E_INVAL;
    const int es = in_type == IXP_I32 ? 4 : 8, eo = out_type == IXP_I32 ? 4 : 8;
    if ((reinterpret_cast<uintptr_t>(in) % es) || (reinterpret_cast<uintptr_t>(out) % eo)) return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // the array's address is per device: the stream must belong to the current one
    // (the legacy and per-thread default stream handles always do)
    if (reinterpret_cast<uintptr_t>(st) > 2) {
        int cur = -1, sdev = -1;
        if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) return IXP_E_CUDA;
        if (sdev != cur) return IXP_E_INVAL;
    }
    if (in_type == IXP_I32 && out_type == IXP_I32)
        return run_scan_noalloc((const int32_t *)in, (int32_t *)out, n, inclusive, (int32_t *)d_totals, d_status, st);
    if (in_type == IXP_I32)
        return run_scan_noalloc((const int32_t *)in, (int64_t *)out, n, inclusive, (int64_t *)d_totals, d_status, st);
    return run_scan_noalloc((const int64_t *)in, (int64_t *)out, n, inclusive, (int64_t *)d_totals, d_status, st);
}

extern "C" int ixp_debug_set_wait(long long spin_limit, long long skip_tile) {
    ixp::g_wait.spin_limit = spin_limit > 0 ? spin_limit : (1ll << 20);
    ixp::g_wait.skip_tile = skip_tile;
    return IXP_OK;
}

extern "C" unsigned long long ixp_tu_kernels_scan(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}
