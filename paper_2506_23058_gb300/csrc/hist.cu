// hist.cu - reduce-by-index with the min operator (Futhark's hist, Sec. 6), the
// dynamic verification of a scatter's injectivity built on it, and
// get_smallest_pairs of maxMatching (Fig. 16).
//
// Reduce-by-index: every in-bounds element issues one atomic min whose result is
// unused, so each is a fire-and-forget reduction at L2. Its rate is that of L2
// atomics while H fits in L2 (129 MB) and that of random HBM sectors when it does
// not (each reduction then reads and writes back one 32-byte sector).
//
// Dynamic Inj check (what the paper's evaluation compares static verification
// against, Sec. 6): H = hist min over [0, m) of iota by x; Inj on [0, m) holds
// iff every in-bounds i has H[x[i]] == i. A violation at j means x[j] repeats an
// earlier element H[x[j]] < j; the smallest such H[x[j]] is the first
// occurrence of the earliest repeated value and the smallest j with that H is its
// next occurrence, which is the verdict ixp_check_inj gives. Both are packed into
// one word (H << 32 | j) whose smallest value wins.
//
// get_smallest_pairs: H = hist min (neutral n_es) over the vertices of the edge
// priorities is by es; a slot is kept when its priority is its vertex's minimum;
// both arrays are filtered by that flag, stably. The filter is two tiled passes:
// the first computes each slot's flag (one bit, stored as a bitmap word per 32
// slots) and each tile's count, a grouped scan of the counts gives each tile's
// output offset, and the second writes the kept pairs with ranks from the bitmap.
// (A single pass with a decoupled look-back measured slower: the tiles hold their
// gathers in registers while they wait.) int64 priorities that all lie in
// [0, 2^32 - 2] are reduced in a 32-bit H, half the L2 footprint of an int64 one;
// a priority outside that range switches the call, on the device, to the 64-bit H.
#include <algorithm>

#include "common.cuh"
#include "tilescan.cuh"

namespace ixp {


// Four consecutive elements 4q .. 4q + 3 with 16-byte loads (p 16-byte aligned).
template <typename T> __device__ __forceinline__ void ld4(const T *p, int64_t q, T (&v)[4]);
template <> __device__ __forceinline__ void ld4<int32_t>(const int32_t *p, int64_t q, int32_t (&v)[4]) {
    const int4 a = __ldcs(reinterpret_cast<const int4 *>(p) + q);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <> __device__ __forceinline__ void ld4<uint32_t>(const uint32_t *p, int64_t q, uint32_t (&v)[4]) {
    const uint4 a = __ldcs(reinterpret_cast<const uint4 *>(p) + q);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <> __device__ __forceinline__ void ld4<int64_t>(const int64_t *p, int64_t q, int64_t (&v)[4]) {
    const longlong2 a = __ldcs(reinterpret_cast<const longlong2 *>(p) + 2 * q);
    const longlong2 b = __ldcs(reinterpret_cast<const longlong2 *>(p) + 2 * q + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Fire-and-forget atomic min (the result is unused, so it compiles to a reduction).
__device__ __forceinline__ void red_min(int32_t *p, int32_t v) { atomicMin(p, v); }
__device__ __forceinline__ void red_min(uint32_t *p, uint32_t v) { atomicMin(p, v); }
__device__ __forceinline__ void red_min(int64_t *p, int64_t v) {
    atomicMin(reinterpret_cast<long long *>(p), (long long)v);
}

// H[idx[i]] = min(H[idx[i]], v_i) for 0 <= idx[i] < m, v_i = vals[i] or i (IOTA).
// Grid-stride over groups of four elements (16-byte loads when `vec`), then the
// elements after the last whole group one by one.
// gate (nullable): the kernel runs only when gate->flag is set.
template <typename IT, typename HT, bool IOTA>
__global__ void __launch_bounds__(STREAM_THREADS) hist_min_kernel(HT *__restrict__ H, int64_t m,
                                                                  const IT *__restrict__ idx,
                                                                  const HT *__restrict__ vals, int64_t n, int vec,
                                                                  const Hdr *gate) {
    IXP_KERNEL_ENTRY();
    if (gate && !gate->flag) return;
    const int64_t n4 = vec ? n / 4 : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t q = t0; q < n4; q += stride) {
        IT k[4];
        HT v[4];
        ld4<IT>(idx, q, k);
        if (!IOTA) ld4<HT>(vals, q, v);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int64_t kk = (int64_t)k[c];
            if ((uint64_t)kk < (uint64_t)m) red_min(H + kk, IOTA ? (HT)(4 * q + c) : v[c]);
        }
    }
    for (int64_t i = n4 * 4 + t0; i < n; i += stride) {
        const int64_t kk = (int64_t)idx[i];
        if ((uint64_t)kk < (uint64_t)m) red_min(H + kk, IOTA ? (HT)i : vals[i]);
    }
}

template <typename T>
__global__ void __launch_bounds__(STREAM_THREADS) fill_kernel(T *__restrict__ p, int64_t m, T v, const Hdr *gate) {
    IXP_KERNEL_ENTRY();
    if (gate && !gate->flag) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

template <typename IT, typename HT>
static void launch_hist(HT *H, int64_t m, const IT *idx, const HT *vals, int64_t n, cudaStream_t st,
                        const Hdr *gate = nullptr) {
    if (n <= 0) return;
    const int vec = aligned16(idx) && (vals == nullptr || aligned16(vals));
    const int g = stream_grid((n + 3) / 4, 1);
    if (vals)
        hist_min_kernel<IT, HT, false><<<g, STREAM_THREADS, 0, st>>>(H, m, idx, vals, n, vec, gate);
    else
        hist_min_kernel<IT, HT, true><<<g, STREAM_THREADS, 0, st>>>(H, m, idx, nullptr, n, vec, gate);
}

// The 32-bit form of the reduce-by-index for int64 priorities: H32[es[i]] =
// min(H32[es[i]], is[i]) while is[i] lies in [0, 2^32 - 2]; a priority of an
// in-bounds slot outside that range sets h->flag instead (the 64-bit H is then
// built and used).
__global__ void __launch_bounds__(STREAM_THREADS) hist_min_narrow_kernel(uint32_t *__restrict__ H, int64_t m,
                                                                         const int64_t *__restrict__ idx,
                                                                         const int64_t *__restrict__ vals, int64_t n,
                                                                         int vec, Hdr *h) {
    IXP_KERNEL_ENTRY();
    const int64_t n4 = vec ? n / 4 : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool wide = false;
    for (int64_t q = t0; q < n4; q += stride) {
        int64_t k[4], v[4];
        ld4<int64_t>(idx, q, k);
        ld4<int64_t>(vals, q, v);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if ((uint64_t)k[c] >= (uint64_t)m) continue;
            if ((uint64_t)v[c] > 0xfffffffeull) wide = true;
            else red_min(H + k[c], (uint32_t)v[c]);
        }
    }
    for (int64_t i = n4 * 4 + t0; i < n; i += stride) {
        const int64_t kk = idx[i];
        if ((uint64_t)kk >= (uint64_t)m) continue;
        const int64_t vv = vals[i];
        if ((uint64_t)vv > 0xfffffffeull) wide = true;
        else red_min(H + kk, (uint32_t)vv);
    }
    if (__syncthreads_or(wide) && threadIdx.x == 0) atomicOr(&h->flag, 1u);
}

// ------------------------------------------------------------ dynamic Inj check

// Every in-bounds i with H[x[i]] != i is a repeat of H[x[i]]; the block's smallest
// (H[x[i]] << 32 | i), complemented, raises h->k_first.
template <typename IT>
__global__ void __launch_bounds__(STREAM_THREADS) inj_hist_check_kernel(const IT *__restrict__ x, int64_t n,
                                                                        int64_t m, const uint32_t *__restrict__ H,
                                                                        Hdr *h, int vec) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long sm[STREAM_THREADS / 32];
    unsigned long long best = ~0ull;
    const int64_t n4 = vec ? n / 4 : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t q = t0; q < n4; q += stride) {
        IT k[4];
        ld4<IT>(x, q, k);
        uint32_t hv[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int64_t kk = (int64_t)k[c];
            hv[c] = (uint64_t)kk < (uint64_t)m ? __ldg(H + kk) : (uint32_t)(4 * q + c);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint64_t i = (uint64_t)(4 * q + c);
            if (hv[c] != (uint32_t)i) {
                const unsigned long long key = ((unsigned long long)hv[c] << 32) | i;
                best = key < best ? key : best;
            }
        }
    }
    for (int64_t i = n4 * 4 + t0; i < n; i += stride) {
        const int64_t kk = (int64_t)x[i];
        if ((uint64_t)kk < (uint64_t)m) {
            const uint32_t hv = __ldg(H + kk);
            if (hv != (uint32_t)i) {
                const unsigned long long key = ((unsigned long long)hv << 32) | (uint64_t)i;
                best = key < best ? key : best;
            }
        }
    }
    const unsigned long long r = block_max_u64(~best, sm);
    if (threadIdx.x == 0) atomic_max_u64(&h->k_first, r);
}

template <typename IT>
__global__ void inj_hist_finalize(const IT *x, const Hdr *h, ixp_verdict *out) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    v.status = h->status;
    const bool bad = h->k_first != 0;
    const unsigned long long key = ~h->k_first;
    const int64_t i = bad ? (int64_t)(key >> 32) : -1;
    v.ok = v.status ? -1 : (bad ? 0 : 1);
    v.kind = bad ? IXP_V_DUPLICATE : IXP_V_NONE;
    v.index = i;
    v.value = bad ? (int64_t)x[i] : 0;
    v.aux0 = bad ? (int64_t)(key & 0xffffffffull) : 0;
    v.aux1 = 0;
    v.reserved = 0;
    *out = v;
}

size_t inj_hist_ws_bytes(int64_t m) { return HDR_BYTES + round256((size_t)(m > 0 ? m : 0) * 4); }

template <typename IT>
static int run_inj_hist(const IT *x, int64_t n, int64_t m, ixp_verdict *out, void *ws, cudaStream_t st) {
    Hdr *h = reinterpret_cast<Hdr *>(ws);
    uint32_t *H = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(ws) + HDR_BYTES);
    if (cudaMemsetAsync(h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (m > 0 && cudaMemsetAsync(H, 0xff, (size_t)m * 4, st) != cudaSuccess) return IXP_E_CUDA;
    if (n > 0 && m > 0) {
        launch_hist<IT, uint32_t>(H, m, x, nullptr, n, st);
        const int vec = aligned16(x);
        inj_hist_check_kernel<IT><<<stream_grid((n + 3) / 4, 1), STREAM_THREADS, 0, st>>>(x, n, m, H, h, vec);
    }
    inj_hist_finalize<IT><<<1, 1, 0, st>>>(x, h, out);
    return launch_status();
}

// ------------------------------------------------------------ get_smallest_pairs

constexpr int SP_THREADS = 256;
constexpr int SP_ROUNDS = 16;                    // 32-slot rounds per warp per tile
constexpr int SP_TILE = SP_THREADS * SP_ROUNDS;  // 4096 slots
constexpr int SP_WARP_SPAN = 32 * SP_ROUNDS;     // 512 consecutive slots per warp

struct SpWs {
    Hdr *h;
    void *H;        // n_verts entries of the index type
    uint32_t *H32;  // n_verts entries (int64 priorities that fit 32 bits)
    unsigned long long *tile_cnt;
    unsigned long long *gtot;
    uint32_t *keep;  // one bit per slot
    size_t bytes;
};

static SpWs sp_ws(void *ws, int64_t n, int64_t n_verts, int es) {
    SpWs w{};
    char *b = reinterpret_cast<char *>(ws);
    const int64_t nt = (n + SP_TILE - 1) / SP_TILE;
    const size_t nv = (size_t)(n_verts > 0 ? n_verts : 0);
    size_t o = HDR_BYTES;
    w.h = reinterpret_cast<Hdr *>(b);
    w.H = b + o;
    o += round256(nv * es);
    w.H32 = reinterpret_cast<uint32_t *>(b + o);
    o += es == 8 ? round256(nv * 4) : 0;
    w.tile_cnt = reinterpret_cast<unsigned long long *>(b + o);
    o += round256((size_t)(nt + 1) * 8);
    w.gtot = reinterpret_cast<unsigned long long *>(b + o);
    o += round256((size_t)((nt + TS_G - 1) / TS_G + 1) * 8);
    w.keep = reinterpret_cast<uint32_t *>(b + o);
    o += round256((size_t)(nt * SP_TILE / 32) * 4);
    w.bytes = o;
    return w;
}

size_t smallest_pairs_ws_bytes(int itype, int64_t n, int64_t n_verts) {
    return sp_ws(nullptr, n < 0 ? 0 : n, n_verts, itype == IXP_I64 ? 8 : 4).bytes;
}

// Pass 1: keep[i] = (0 <= es[i] < n_verts && H[es[i]] == is[i]) as bitmap words
// (word i / 32, bit i % 32) and the tile's count. Lane l of warp w handles slot
// t0 + 512 w + 32 r + l in round r; all rounds' loads and gathers are issued
// before the compares.
template <typename T, typename HT>
__device__ __forceinline__ void sp_flag_tile(const T *__restrict__ es, const T *__restrict__ is, int64_t n,
                                             int64_t n_verts, const HT *__restrict__ H, uint32_t *__restrict__ keep,
                                             unsigned long long *__restrict__ tile_cnt, unsigned *s_w) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * SP_TILE + (int64_t)w * SP_WARP_SPAN;
    T e[SP_ROUNDS];
    HT hv[SP_ROUNDS];
#pragma unroll
    for (int r = 0; r < SP_ROUNDS; r++) {
        const int64_t i = base + r * 32 + l;
        e[r] = i < n ? __ldcs(es + i) : (T)-1;
    }
#pragma unroll
    for (int r = 0; r < SP_ROUNDS; r++)
        hv[r] = (uint64_t)(int64_t)e[r] < (uint64_t)n_verts ? __ldg(H + (int64_t)e[r]) : (HT)0;
    unsigned cnt = 0;
#pragma unroll
    for (int r = 0; r < SP_ROUNDS; r++) {
        const int64_t i = base + r * 32 + l;
        const bool in = (uint64_t)(int64_t)e[r] < (uint64_t)n_verts;  // false past n (e = -1)
        const bool k = in && (int64_t)__ldcs(is + i) == (int64_t)hv[r];
        const unsigned word = __ballot_sync(FULL, k);
        if (l == 0) keep[(base + r * 32) >> 5] = word;
        cnt += __popc(word);
    }
    if (l == 0) s_w[w] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < SP_THREADS / 32; i++) t += s_w[i];
        tile_cnt[blockIdx.x] = t;
    }
}

// wide: compare with H (the index type); otherwise with the 32-bit H32 unless
// the narrow reduce-by-index flagged a priority outside its range (h->flag).
template <typename T>
__global__ void __launch_bounds__(SP_THREADS) sp_flag_kernel(const T *__restrict__ es, const T *__restrict__ is,
                                                             int64_t n, int64_t n_verts, const T *__restrict__ H,
                                                             const uint32_t *__restrict__ H32, int wide, const Hdr *h,
                                                             uint32_t *__restrict__ keep,
                                                             unsigned long long *__restrict__ tile_cnt) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned s_w[SP_THREADS / 32];
    if (wide || h->flag)
        sp_flag_tile<T, T>(es, is, n, n_verts, H, keep, tile_cnt, s_w);
    else
        sp_flag_tile<T, uint32_t>(es, is, n, n_verts, H32, keep, tile_cnt, s_w);
}

// Pass 2: each kept slot goes to (tile offset) + (kept slots before it in its tile).
template <typename T>
__global__ void __launch_bounds__(SP_THREADS) sp_write_kernel(const T *__restrict__ es, const T *__restrict__ is,
                                                              int64_t n, const uint32_t *__restrict__ keep,
                                                              const unsigned long long *__restrict__ tile_pre,
                                                              const Hdr *h, T *__restrict__ out_es,
                                                              T *__restrict__ out_is, int64_t *d_count) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned s_w[SP_THREADS / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * SP_TILE + (int64_t)w * SP_WARP_SPAN;
    // lane r < SP_ROUNDS holds the warp's word for round r
    const uint32_t myword = l < SP_ROUNDS ? keep[(base >> 5) + l] : 0u;
    unsigned c = __popc(myword);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (l == 0) s_w[w] = c;
    __syncthreads();
    unsigned wpre = 0;
    for (int i = 0; i < w; i++) wpre += s_w[i];
    int64_t run = (int64_t)tile_pre[blockIdx.x] + wpre;
#pragma unroll
    for (int r = 0; r < SP_ROUNDS; r++) {
        const uint32_t word = __shfl_sync(FULL, myword, r);
        if ((word >> l) & 1u) {
            const int64_t i = base + r * 32 + l;
            const int64_t d = run + __popc(word & ((1u << l) - 1u));
            out_es[d] = __ldcs(es + i);
            out_is[d] = __ldcs(is + i);
        }
        run += __popc(word);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_count = (int64_t)h->total;
}

template <typename T>
static int run_smallest_pairs(const T *es, const T *is, int64_t n, int64_t n_verts, int64_t n_es, T *out_es,
                              T *out_is, int64_t *d_count, void *ws, size_t ws_bytes, cudaStream_t st) {
    const SpWs w = sp_ws(ws, n, n_verts, (int)sizeof(T));
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < w.bytes) return IXP_E_WORKSPACE;
    if (cudaMemsetAsync(w.h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    if (cudaMemsetAsync(d_count, 0, sizeof(int64_t), st) != cudaSuccess) return IXP_E_CUDA;
    if (n == 0 || n_verts == 0) return launch_status();
    T *H = reinterpret_cast<T *>(w.H);
    const int gf = stream_grid(n_verts, 4);
    int wide = 1;
    if (sizeof(T) == 4 || n_es < 0) {
        // int32 priorities, or a negative neutral element (below every priority a
        // 32-bit H holds): the reduce-by-index in the index type
        fill_kernel<T><<<gf, STREAM_THREADS, 0, st>>>(H, n_verts, (T)n_es, nullptr);
        launch_hist<T, T>(H, n_verts, es, is, n, st);
    } else {
        wide = 0;
        const uint32_t neutral = (uint32_t)std::min<int64_t>(n_es, 0xffffffffll);
        fill_kernel<uint32_t><<<gf, STREAM_THREADS, 0, st>>>(w.H32, n_verts, neutral, nullptr);
        const int vec = aligned16(es) && aligned16(is);
        hist_min_narrow_kernel<<<stream_grid((n + 3) / 4, 1), STREAM_THREADS, 0, st>>>(
            w.H32, n_verts, (const int64_t *)es, (const int64_t *)is, n, vec, w.h);
        // only when a priority did not fit: the 64-bit H
        fill_kernel<T><<<gf, STREAM_THREADS, 0, st>>>(H, n_verts, (T)n_es, w.h);
        launch_hist<T, T>(H, n_verts, es, is, n, st, w.h);
    }
    const int64_t nt = (n + SP_TILE - 1) / SP_TILE;
    sp_flag_kernel<T><<<(unsigned)nt, SP_THREADS, 0, st>>>(es, is, n, n_verts, H, w.H32, wide, w.h, w.keep,
                                                           w.tile_cnt);
    scan_tile_counts(w.tile_cnt, nt, w.gtot, w.h, st);
    sp_write_kernel<T><<<(unsigned)nt, SP_THREADS, 0, st>>>(es, is, n, w.keep, w.tile_cnt, w.h, out_es, out_is,
                                                           d_count);
    return launch_status();
}

}  // namespace ixp

using namespace ixp;

extern "C" unsigned long long ixp_tu_kernels_hist(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}

extern "C" int ixp_hist_min(void *H, int htype, int64_t m, const void *idx, int itype, const void *vals, int64_t n,
                            ixp_stream stream) {
    if ((htype != IXP_I32 && htype != IXP_I64) || (itype != IXP_I32 && itype != IXP_I64)) return IXP_E_DTYPE;
    if (n < 0 || m < 0 || (m > 0 && !H) || (n > 0 && !idx)) return IXP_E_INVAL;
    if (!vals && htype == IXP_I32 && n - 1 > INT32_MAX) return IXP_E_INVAL;  // iota must fit H's type
    const size_t hs = htype == IXP_I64 ? 8 : 4, is = itype == IXP_I64 ? 8 : 4;
    if ((reinterpret_cast<uintptr_t>(H) % hs) || (reinterpret_cast<uintptr_t>(idx) % is) ||
        (vals && reinterpret_cast<uintptr_t>(vals) % hs))
        return IXP_E_INVAL;
    if (n == 0 || m == 0) return IXP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (htype == IXP_I32) {
        if (itype == IXP_I32)
            launch_hist<int32_t, int32_t>((int32_t *)H, m, (const int32_t *)idx, (const int32_t *)vals, n, st);
        else
            launch_hist<int64_t, int32_t>((int32_t *)H, m, (const int64_t *)idx, (const int32_t *)vals, n, st);
    } else {
        if (itype == IXP_I32)
            launch_hist<int32_t, int64_t>((int64_t *)H, m, (const int32_t *)idx, (const int64_t *)vals, n, st);
        else
            launch_hist<int64_t, int64_t>((int64_t *)H, m, (const int64_t *)idx, (const int64_t *)vals, n, st);
    }
    return launch_status();
}

extern "C" int ixp_check_inj_hist(const void *x, int itype, int64_t n, int64_t m, ixp_verdict *d_verdict, void *ws,
                                  size_t ws_bytes, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    const size_t es = itype == IXP_I64 ? 8 : 4;
    if (n < 0 || n >= (1ll << 32) || m < 0 || !d_verdict || (n > 0 && (!x || reinterpret_cast<uintptr_t>(x) % es)))
        return IXP_E_INVAL;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < inj_hist_ws_bytes(m)) return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (itype == IXP_I32) return run_inj_hist((const int32_t *)x, n, m, d_verdict, ws, st);
    return run_inj_hist((const int64_t *)x, n, m, d_verdict, ws, st);
}

extern "C" int ixp_smallest_pairs(const void *es, const void *is, int itype, int64_t n, int64_t n_verts, int64_t n_es,
                                  void *out_es, void *out_is, int64_t *d_count, void *ws, size_t ws_bytes,
                                  ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    const size_t esz = itype == IXP_I64 ? 8 : 4;
    auto misaligned = [esz](const void *p) { return reinterpret_cast<uintptr_t>(p) % esz != 0; };
    if (n < 0 || n >= (1ll << 40) || n_verts < 0 || !d_count ||
        (n > 0 && (!es || !is || !out_es || !out_is || misaligned(es) || misaligned(is) || misaligned(out_es) ||
                   misaligned(out_is))))
        return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (itype == IXP_I64)
        return run_smallest_pairs((const int64_t *)es, (const int64_t *)is, n, n_verts, n_es, (int64_t *)out_es,
                                  (int64_t *)out_is, d_count, ws, ws_bytes, st);
    // int32 priorities: a neutral element above INT32_MAX acts as INT32_MAX (no
    // priority exceeds it); one below INT32_MIN is below every priority, so
    // nothing is kept.
    if (n_es < (int64_t)INT32_MIN) n = 0;
    const int64_t neutral = std::min<int64_t>(n_es, INT32_MAX);
    return run_smallest_pairs((const int32_t *)es, (const int32_t *)is, n, n_verts, neutral, (int32_t *)out_es,
                              (int32_t *)out_is, d_count, ws, ws_bytes, st);
}
