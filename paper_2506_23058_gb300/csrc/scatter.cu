// scatter.cu - scatter and gather of payload rows (Sec. 2.1: scatter ignores
// indices outside the destination), the additive scatter used as the adjoint of
// gather, and the float64 -> float32 rounding of its accumulator.
//
// Rows whose size is a multiple of 16 bytes (with 16-byte aligned bases) move as
// 16-byte chunks, L lanes of a warp per row (L the largest power of two <= the
// chunk count, at most 32), so that one warp instruction touches 32 / L rows and a
// 32-byte row is one full sector written (or read) by a lane pair. Other rows move
// one thread per row in 4-byte words.
#include <algorithm>

#include "common.cuh"

namespace ixp {

// Rows move as 16-byte chunks when the row size is a multiple of 16 (vec16); each
// thread keeps RU rows in flight (indices first, then all row loads, then stores).
constexpr int RU = 4;

template <typename IT>
__global__ void __launch_bounds__(STREAM_THREADS) scatter_rows_kernel(char *__restrict__ dst, int64_t dst_len,
                                                                      const IT *__restrict__ idx,
                                                                      const char *__restrict__ vals, int64_t n,
                                                                      int row_bytes) {
    IXP_KERNEL_ENTRY();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = tid; i < n; i += stride) {
        const int64_t d = (int64_t)__ldg(idx + i);
        if (d < 0 || d >= dst_len) continue;
        const uint32_t *src = reinterpret_cast<const uint32_t *>(vals + i * row_bytes);
        uint32_t *t = reinterpret_cast<uint32_t *>(dst + d * row_bytes);
        for (int c = 0; c < row_bytes / 4; c++) t[c] = src[c];
    }
}

// Read-only 16-byte load whose L2 miss fetches 64 bytes, not a whole 128-byte
// line: rows read at random indices then cost about half the DRAM traffic (the
// random-row rate is the same either way).
__device__ __forceinline__ int4 ld_row_chunk(const int4 *p) {
    int4 v;
    asm("ld.global.nc.L2::64B.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Lane-split row move: lane j of the L lanes serving row r moves chunks j and
// (CPL = 2) j + L of the row's nc 16-byte chunks. SCATTER: dst[idx[r]] = vals[r]
// (indices outside [0, dst_len) ignored); gather: out[r] = src[idx[r]] (zero row
// and an OOB status for indices outside [0, src_len)).
template <typename IT, int L, int CPL, bool SCATTER>
__global__ void __launch_bounds__(STREAM_THREADS, CPL == 1 ? 6 : 4)
    rows_lanes_kernel(int4 *__restrict__ out, int64_t out_len, const IT *__restrict__ idx,
                      const int4 *__restrict__ in, int64_t in_len, int64_t n, int nc, int32_t *status) {
    IXP_KERNEL_ENTRY();
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int j = (int)(gt % L);
    const int64_t r0 = gt / L;
    const int64_t rs = (int64_t)gridDim.x * blockDim.x / L;
    const bool two = CPL == 2 && j + L < nc;
    bool any_oob = false;
    for (int64_t rb = r0; rb < n; rb += RU * rs) {
        int64_t d[RU];
        int4 v[RU][CPL];
#pragma unroll
        for (int u = 0; u < RU; u++) {
            const int64_t r = rb + u * rs;
            d[u] = r < n ? (int64_t)__ldcs(idx + r) : -1;
        }
        if (SCATTER) {
#pragma unroll
            for (int u = 0; u < RU; u++) {
                const int64_t r = rb + u * rs;
                if (r < n) {
                    v[u][0] = __ldcs(in + r * nc + j);
                    if (two) v[u][CPL - 1] = __ldcs(in + r * nc + j + L);
                }
            }
#pragma unroll
            for (int u = 0; u < RU; u++) {
                if (d[u] < 0 || d[u] >= out_len) continue;
                __stcs(out + d[u] * nc + j, v[u][0]);
                if (two) __stcs(out + d[u] * nc + j + L, v[u][CPL - 1]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < RU; u++) {
                const int64_t r = rb + u * rs;
                const bool ok = d[u] >= 0 && d[u] < in_len;
                if (r < n && !ok) any_oob = true;
                v[u][0] = v[u][CPL - 1] = make_int4(0, 0, 0, 0);
                if (r < n && ok) {
                    v[u][0] = ld_row_chunk(in + d[u] * nc + j);
                    if (two) v[u][CPL - 1] = ld_row_chunk(in + d[u] * nc + j + L);
                }
            }
#pragma unroll
            for (int u = 0; u < RU; u++) {
                const int64_t r = rb + u * rs;
                if (r >= n) continue;
                __stcs(out + r * nc + j, v[u][0]);
                if (two) __stcs(out + r * nc + j + L, v[u][CPL - 1]);
            }
        }
    }
    if (!SCATTER && any_oob && status) atomicCAS(status, 0, IXP_E_OOB);
}

template <typename IT, bool SCATTER>
static void launch_rows_lanes(int4 *out, int64_t out_len, const IT *idx, const int4 *in, int64_t in_len, int64_t n,
                              int nc, int32_t *status, cudaStream_t st) {
    int L = 1;
    while (L * 2 <= nc && L < 32) L *= 2;
    const int cpl = (nc + L - 1) / L;  // 1 or 2
    const int64_t per_block = (int64_t)STREAM_THREADS / L * RU;
    const int64_t cap = (int64_t)num_sms() * (cpl == 1 ? 6 : 4);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, cap));
#define IXP_ROWS_CASE(LL)                                                                                       \
    case LL:                                                                                                    \
        if (cpl == 1)                                                                                           \
            rows_lanes_kernel<IT, LL, 1, SCATTER><<<g, STREAM_THREADS, 0, st>>>(out, out_len, idx, in, in_len, n, \
                                                                               nc, status);                    \
        else                                                                                                    \
            rows_lanes_kernel<IT, LL, 2, SCATTER><<<g, STREAM_THREADS, 0, st>>>(out, out_len, idx, in, in_len, n, \
                                                                               nc, status);                    \
        break;
    switch (L) {
        IXP_ROWS_CASE(1)
        IXP_ROWS_CASE(2)
        IXP_ROWS_CASE(4)
        IXP_ROWS_CASE(8)
        IXP_ROWS_CASE(16)
        IXP_ROWS_CASE(32)
    }
#undef IXP_ROWS_CASE
}

template <typename IT, typename FT>
__global__ void __launch_bounds__(STREAM_THREADS) scatter_add_kernel(FT *__restrict__ dst, int64_t dst_len,
                                                                     const IT *__restrict__ idx,
                                                                     const FT *__restrict__ vals, int64_t n,
                                                                     int row_elems) {
    IXP_KERNEL_ENTRY();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t d = (int64_t)__ldg(idx + i);
        if (d < 0 || d >= dst_len) continue;
        for (int c = 0; c < row_elems; c++) atomicAdd(dst + d * row_elems + c, vals[i * row_elems + c]);
    }
}

// Additive scatter of float32 rows into a float64 accumulator. For rows of up to
// HOT_COLS values each block keeps a direct-mapped cache of HOT_SLOTS target rows in
// shared memory, and a warp takes 32 / CP rows per step with CP lanes per row (one
// column each, CP = row width rounded up to a power of two): the values load as
// coalesced column words, a row whose target owns its cache slot (claiming a free
// slot on first use) is added into the cached row, and a row that misses is added
// to the global accumulator with one float64 atomic per lane, the CP lanes of a row
// hitting one contiguous row (the L2 takes such a warp's reductions about three
// times faster than 32 scattered rows). Hot targets (a Zipf head) thus cost
// shared-memory atomics instead of serialised global ones. The cached rows are
// exact 64-bit fixed-point sums held as two 32-bit words (native 32-bit shared
// atomics; the low word's wrap-arounds are carried into the high word by the adder
// that caused them, so the pair stays exact modulo 2^64). The block samples the
// largest biased exponent E of its first rows; with R <= 2^r the most rows the
// block can take, the unit is 2^L, L = (E - 125) + r - 62. A float32 value with
// biased exponent in [E + r - 37, E + 1] is then an integer multiple of 2^L below
// 2^(62 - r) units, so its scaled value is exact and 2^r of them cannot overflow;
// any other value (smaller, larger than the sample, not finite) takes the float64
// path, zeros are skipped. When the block ends each cached sum is rounded to
// float64 once and added globally: at least as accurate as float64 atomics. Wider
// rows combine same-target lanes of a warp first (match_any + a shuffle tree in
// float64) and add the sums globally.
constexpr int HOT_COLS = 8;        // cached row width; wider rows bypass the cache
constexpr int HOT_SLOTS = 1024;    // cached target rows per block (a power of two)
constexpr int HOT_BLOCKS_PER_SM = 3;
constexpr int HOT_THREADS = 512;   // three blocks of 512 threads and their caches fill an SM
// shared bytes of the cache: the tags, then the fixed-point rows (low words, high words)
constexpr size_t hot_smem_bytes(int slots) { return (size_t)slots * (8 + 8 * HOT_COLS); }

// Float32 bits -> biased exponent (0 for zero and denormals).
__device__ __forceinline__ int f32_bexp(float v) { return (int)((__float_as_uint(v) >> 23) & 0xffu); }

template <typename IT>
__global__ void __launch_bounds__(HOT_THREADS, HOT_BLOCKS_PER_SM) scatter_add_f64_kernel(double *__restrict__ acc, int64_t dst_len,
                                                                         const IT *__restrict__ idx,
                                                                         const float *__restrict__ vals, int64_t n,
                                                                         int row_elems, int slots) {
    IXP_KERNEL_ENTRY();
    extern __shared__ __align__(16) unsigned long long hot_raw[];
    unsigned long long *s_tag = hot_raw;  // slots; ~0 = free
    unsigned *s_lo = reinterpret_cast<unsigned *>(hot_raw + slots);  // [slot][HOT_COLS]
    unsigned *s_hi = s_lo + (size_t)slots * HOT_COLS;
    __shared__ int s_emax;
    const bool cache = row_elems <= HOT_COLS && slots > 0;
    for (int sl = threadIdx.x; sl < slots; sl += blockDim.x) {
        s_tag[sl] = ~0ull;
        for (int c = 0; c < HOT_COLS; c++) s_lo[sl * HOT_COLS + c] = s_hi[sl * HOT_COLS + c] = 0u;
    }
    if (threadIdx.x == 0) s_emax = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // the scale: the largest biased exponent among this block's first rows
    if (cache && tid < n) {
        int e = 0;
        for (int c = 0; c < row_elems; c++) e = max(e, f32_bexp(__ldg(vals + tid * row_elems + c)));
        atomicMax(&s_emax, e);
    }
    __syncthreads();
    if (cache) {
        const int lg = row_elems <= 1 ? 0 : row_elems <= 2 ? 1 : row_elems <= 4 ? 2 : 3;  // CP = 2^lg lanes a row
        const int rpw = 32 >> lg;                                                           // rows a warp step
        const int j = lane >> lg, c = lane & ((1 << lg) - 1);
        const bool col = c < row_elems;
        const int64_t wpb = blockDim.x >> 5;
        const int64_t rstride = (int64_t)gridDim.x * wpb * rpw;  // rows per grid step
        const long long rb = ((n + rstride - 1) / rstride) * wpb * rpw;  // rows this block takes at most
        const int r = max(1, 64 - __clzll((unsigned long long)max(rb, 2ll) - 1ull));  // 2^r >= rb
        const int L = (s_emax - 125) + r - 62;  // fixed-point unit 2^L
        const int eb_lo = s_emax + r - 37, eb_hi = s_emax + 1;  // biased exponents kept in the cache
        const bool fix_ok = s_emax > 0 && s_emax < 254 && -L <= 127 && -L >= -126 && eb_lo <= eb_hi;
        const float to_fix = fix_ok ? ldexpf(1.0f, -L) : 0.0f;  // a power of two: the scaling is exact
        // a lane's row target (-1 when out of bounds or past n) and its column value;
        // software-pipelined: the next step's are in flight while this one is added
        const auto load = [&](int64_t rw, int64_t &d, float &x) {
            d = -1;
            x = 0.0f;
            if (rw >= n) return;
            d = (int64_t)__ldg(idx + rw);
            if (d < 0 || d >= dst_len) d = -1;
            if (col) x = __ldcs(vals + rw * row_elems + c);
        };
        int64_t rw = ((int64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * rpw + j;
        int64_t d;
        float x;
        load(rw, d, x);
        for (; rw < n; rw += rstride) {
            int64_t dn;
            float xn;
            load(rw + rstride, dn, xn);
            if (d >= 0 && col) {
                const int sl = (int)(d & (int64_t)(slots - 1));
                unsigned long long tag = s_tag[sl];
                if (tag == ~0ull) {
                    const unsigned long long prev = atomicCAS(&s_tag[sl], ~0ull, (unsigned long long)d);
                    tag = prev == ~0ull ? (unsigned long long)d : prev;
                }
                const int e = f32_bexp(x);
                if (!(e == 0 && x == 0.0f)) {
                    if (fix_ok && tag == (unsigned long long)d && e >= eb_lo && e <= eb_hi) {
                        const long long q = __float2ll_rn(x * to_fix);  // exact: an integer at this scale
                        const unsigned ql = (unsigned)(unsigned long long)q;
                        const unsigned qh = (unsigned)((unsigned long long)q >> 32);
                        const unsigned old = atomicAdd(&s_lo[sl * HOT_COLS + c], ql);
                        const unsigned up = qh + (old + ql < old ? 1u : 0u);
                        if (up) atomicAdd(&s_hi[sl * HOT_COLS + c], up);
                    } else {
                        atomicAdd(acc + d * row_elems + c, (double)x);
                    }
                }
            }
            d = dn;
            x = xn;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < slots * HOT_COLS; e += blockDim.x) {
            const int sl = e / HOT_COLS, cc = e % HOT_COLS;
            const unsigned long long t = s_tag[sl];
            const long long q = (long long)(((unsigned long long)s_hi[e] << 32) | (unsigned long long)s_lo[e]);
            if (t != ~0ull && cc < row_elems && q != 0) atomicAdd(acc + (int64_t)t * row_elems + cc, ldexp((double)q, L));
        }
        return;
    }
    {
        for (int64_t base = tid - lane; base < n; base += stride) {
            const int64_t i = base + lane;
            const bool live = i < n;
            int64_t d = live ? (int64_t)__ldg(idx + i) : -1;
            if (d < 0 || d >= dst_len) d = -1;
            {
            // wide rows: the lanes holding the same target combine their rows across the warp
            // (one column at a time) and one of them adds the sum
            const unsigned peers = __match_any_sync(FULL, (unsigned long long)d);
            const bool single = __popc(peers) == 1;
            unsigned todo = __ballot_sync(FULL, !single && d >= 0);
            if (d >= 0 && single)
                for (int c = 0; c < row_elems; c++) atomicAdd(acc + d * row_elems + c, (double)vals[i * row_elems + c]);
            while (todo) {
                const int src = __ffs(todo) - 1;
                const int64_t key = __shfl_sync(FULL, d, src);
                const unsigned grp = __ballot_sync(FULL, d == key);
                todo &= ~grp;
                for (int c = 0; c < row_elems; c++) {
                    double x = (d == key) ? (double)vals[i * row_elems + c] : 0.0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
                    if (lane == src) atomicAdd(acc + key * row_elems + c, x);
                }
            }
            }
        }
    }
}

__global__ void f32_to_f64_kernel(double *__restrict__ out, const float *__restrict__ in, int64_t count) {
    IXP_KERNEL_ENTRY();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += stride) out[i] = (double)in[i];
}

__global__ void f64_to_f32_kernel(float *__restrict__ out, const double *__restrict__ acc, int64_t count) {
    IXP_KERNEL_ENTRY();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += stride) out[i] = (float)acc[i];
}

template <typename IT>
__global__ void __launch_bounds__(STREAM_THREADS) gather_rows_kernel(char *__restrict__ out,
                                                                     const char *__restrict__ src, int64_t src_len,
                                                                     const IT *__restrict__ idx, int64_t n,
                                                                     int row_bytes, int32_t *status) {
    IXP_KERNEL_ENTRY();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool any_oob = false;
    for (int64_t i = tid; i < n; i += stride) {
        const int64_t s = (int64_t)__ldg(idx + i);
        const bool ok = s >= 0 && s < src_len;
        if (!ok) any_oob = true;
        uint32_t *t = reinterpret_cast<uint32_t *>(out + i * row_bytes);
        const uint32_t *f = reinterpret_cast<const uint32_t *>(src + (ok ? s : 0) * row_bytes);
        for (int c = 0; c < row_bytes / 4; c++) t[c] = ok ? __ldg(f + c) : 0u;
    }
    if (any_oob && status) atomicCAS(status, 0, IXP_E_OOB);
}

// Gather of whole segments: output segment k (out_off[k] .. out_off[k+1]) is a
// copy of source segment seg_src[k] (src_off[s] .. src_off[s+1]). This is the
// gather out[j] = src[src_off[seg_src[II[j]]] + j - out_off[II[j]]] with II the
// segment-id array of the output shape (mkII, Fig. 2), done without materialising
// II or the index array: each block takes GS_CHUNK consecutive output elements,
// marks the starts of the non-empty segments inside them in a shared bitmap, and
// finds an element's segment by counting the starts at or before it. The segment
// holding each chunk's first element comes from a table one pass over the
// segments fills beforehand.
constexpr int GS_CHUNK = 4096;
constexpr int GS_THREADS = 256;
constexpr int GS_WORDS = GS_CHUNK / 32;

size_t gather_segments_ws_bytes(int64_t n_out) {
    const int64_t nch = (n_out + GS_CHUNK - 1) / GS_CHUNK;
    return (size_t)((nch + 1) * 8 + 255) / 256 * 256;
}

// k0[c] = the non-empty segment that holds element c * GS_CHUNK.
__global__ void gs_chunk_table_kernel(const int64_t *__restrict__ out_off, int64_t m, int64_t n,
                                      int64_t *__restrict__ k0) {
    IXP_KERNEL_ENTRY();
    const int64_t nch = (n + GS_CHUNK - 1) / GS_CHUNK;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = __ldg(out_off + k), b = __ldg(out_off + k + 1);
        if (b <= a || a < 0 || b > n) continue;
        for (int64_t c = (a + GS_CHUNK - 1) / GS_CHUNK; c < nch && c * GS_CHUNK < b; c++) k0[c] = k;
    }
}

__device__ __forceinline__ unsigned gs_heads_upto(const unsigned *s_head, const unsigned *s_pre, int e) {
    const int w = e >> 5;
    return s_pre[w] + __popc(s_head[w] & (0xffffffffu >> (31 - (e & 31))));
}

template <typename E, typename ST>
__global__ void __launch_bounds__(GS_THREADS) gather_segments_kernel(E *__restrict__ out,
                                                                     const int64_t *__restrict__ out_off,
                                                                     const E *__restrict__ src,
                                                                     const int64_t *__restrict__ src_off,
                                                                     const ST *__restrict__ seg_src, int64_t m,
                                                                     int64_t n, int64_t src_m, int64_t src_len,
                                                                     const int64_t *__restrict__ k0tab,
                                                                     int32_t *status) {
    IXP_KERNEL_ENTRY();
    __shared__ int64_t s_rel[GS_CHUNK];  // by rank among the chunk's non-empty segments: source - output start
    __shared__ unsigned s_head[GS_WORDS];
    __shared__ unsigned s_pre[GS_WORDS];
    __shared__ int s_bad;
    const int64_t j0 = blockIdx.x * (int64_t)GS_CHUNK;
    if (j0 >= n) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (__ldg(out_off + m) != n || __ldg(out_off) != 0) && status)
        atomicCAS(status, 0, IXP_E_INVAL);
    const int cnt = (int)min((int64_t)GS_CHUNK, n - j0);
    for (int w = threadIdx.x; w < GS_WORDS; w += GS_THREADS) s_head[w] = 0u;
    if (threadIdx.x == 0) s_bad = 0;
    int64_t k0 = __ldg(k0tab + blockIdx.x);
    k0 = k0 < 0 ? 0 : (k0 >= m ? m - 1 : k0);  // only an inconsistent table leaves it out of range
    __syncthreads();
    for (int64_t k = k0 + 1 + threadIdx.x; k < m; k += GS_THREADS) {
        const int64_t a = __ldg(out_off + k);
        if (a >= j0 + cnt) break;
        if (a > j0 && __ldg(out_off + k + 1) > a) atomicOr(&s_head[(a - j0) >> 5], 1u << ((a - j0) & 31));
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the per-word start counts
        constexpr int PW = GS_WORDS / 32;
        unsigned c[PW], run = 0;
#pragma unroll
        for (int i = 0; i < PW; i++) {
            c[i] = __popc(s_head[threadIdx.x * PW + i]);
            run += c[i];
        }
        unsigned y = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(FULL, y, d);
            if ((int)threadIdx.x >= d) y += o;
        }
        unsigned pre = y - run;
#pragma unroll
        for (int i = 0; i < PW; i++) {
            s_pre[threadIdx.x * PW + i] = pre;
            pre += c[i];
        }
    }
    __syncthreads();
    bool bad = false;
    for (int64_t k = k0 + threadIdx.x; k < m; k += GS_THREADS) {
        const int64_t a = __ldg(out_off + k);
        if (a >= j0 + cnt) break;
        const int64_t b = __ldg(out_off + k + 1);
        if (b <= a) continue;  // empty
        const int64_t s = (int64_t)__ldg(seg_src + k);
        int64_t sa = 0;
        if (s < 0 || s >= src_m) {
            bad = true;
        } else {
            sa = __ldg(src_off + s);
            if (__ldg(src_off + s + 1) - sa != b - a || sa < 0 || sa + (b - a) > src_len) bad = true;
        }
        const unsigned r = a <= j0 ? 0u : gs_heads_upto(s_head, s_pre, (int)(a - j0));
        if (r < GS_CHUNK) s_rel[r] = sa - a;
    }
    if (bad) atomicOr(&s_bad, 1);
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0 && status) atomicCAS(status, 0, IXP_E_INVAL);
        return;
    }
    bool oob = false;
    for (int e = threadIdx.x; e < cnt; e += GS_THREADS) {
        const int64_t j = j0 + e;
        const int64_t i = j + s_rel[gs_heads_upto(s_head, s_pre, e)];
        if (i >= 0 && i < src_len) out[j] = __ldg(src + i);
        else oob = true;  // only with inconsistent offsets
    }
    if (oob && status) atomicCAS(status, 0, IXP_E_INVAL);
}

// mkII (Fig. 2): out[j] = k for out_off[k] <= j < out_off[k+1], by chunks like the
// segment gather (the chunk's first segment from the table, the starts of the
// non-empty segments inside it in a bitmap, and the segment of each start by its
// rank among them).
template <typename OT>
__global__ void __launch_bounds__(GS_THREADS) segment_ids_kernel(OT *__restrict__ out,
                                                                 const int64_t *__restrict__ out_off, int64_t m,
                                                                 int64_t n, const int64_t *__restrict__ k0tab,
                                                                 int32_t *status) {
    IXP_KERNEL_ENTRY();
    __shared__ int64_t s_seg[GS_CHUNK];
    __shared__ unsigned s_head[GS_WORDS];
    __shared__ unsigned s_pre[GS_WORDS];
    const int64_t j0 = blockIdx.x * (int64_t)GS_CHUNK;
    if (j0 >= n) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (__ldg(out_off + m) != n || __ldg(out_off) != 0) && status)
        atomicCAS(status, 0, IXP_E_INVAL);
    const int cnt = (int)min((int64_t)GS_CHUNK, n - j0);
    for (int w = threadIdx.x; w < GS_WORDS; w += GS_THREADS) s_head[w] = 0u;
    int64_t k0 = __ldg(k0tab + blockIdx.x);
    k0 = k0 < 0 ? 0 : (k0 >= m ? m - 1 : k0);
    if (threadIdx.x == 0) s_seg[0] = k0;
    __syncthreads();
    for (int64_t k = k0 + 1 + threadIdx.x; k < m; k += GS_THREADS) {
        const int64_t a = __ldg(out_off + k);
        if (a >= j0 + cnt) break;
        if (a > j0 && __ldg(out_off + k + 1) > a) atomicOr(&s_head[(a - j0) >> 5], 1u << ((a - j0) & 31));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int PW = GS_WORDS / 32;
        unsigned c[PW], run = 0;
#pragma unroll
        for (int i = 0; i < PW; i++) {
            c[i] = __popc(s_head[threadIdx.x * PW + i]);
            run += c[i];
        }
        unsigned y = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(FULL, y, d);
            if ((int)threadIdx.x >= d) y += o;
        }
        unsigned pre = y - run;
#pragma unroll
        for (int i = 0; i < PW; i++) {
            s_pre[threadIdx.x * PW + i] = pre;
            pre += c[i];
        }
    }
    __syncthreads();
    for (int64_t k = k0 + 1 + threadIdx.x; k < m; k += GS_THREADS) {
        const int64_t a = __ldg(out_off + k);
        if (a >= j0 + cnt) break;
        if (a > j0 && __ldg(out_off + k + 1) > a) s_seg[gs_heads_upto(s_head, s_pre, (int)(a - j0))] = k;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += GS_THREADS) out[j0 + e] = (OT)s_seg[gs_heads_upto(s_head, s_pre, e)];
}


static int row_grid(int64_t n) { return stream_grid(n, 1); }

}  // namespace ixp

using namespace ixp;

extern "C" int ixp_scatter(void *dst, int64_t dst_len, const void *idx, int itype, const void *vals, int64_t n,
                           int32_t row_elems, int32_t elem_bytes, int32_t mode, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (elem_bytes != 4 && elem_bytes != 8) return IXP_E_DTYPE;
    if (n < 0 || dst_len < 0 || row_elems <= 0 || row_elems > 64 || (n > 0 && (!idx || !vals)) ||
        (dst_len > 0 && !dst) || (mode != IXP_SCATTER_ASSIGN && mode != IXP_SCATTER_ADD))
        return IXP_E_INVAL;
    if (!aligned_to(idx, itype == IXP_I32 ? 4 : 8) || !aligned_to(vals, elem_bytes) || !aligned_to(dst, elem_bytes))
        return IXP_E_INVAL;
    if (n == 0) return IXP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int rb = row_elems * elem_bytes;
    const int g = row_grid(n);
    if (mode == IXP_SCATTER_ASSIGN) {
        const int v16 = (rb % 16 == 0) && aligned_to(dst, 16) && aligned_to(vals, 16);
        if (v16 && itype == IXP_I32)
            launch_rows_lanes<int32_t, true>((int4 *)dst, dst_len, (const int32_t *)idx, (const int4 *)vals, n, n,
                                             rb / 16, nullptr, st);
        else if (v16)
            launch_rows_lanes<int64_t, true>((int4 *)dst, dst_len, (const int64_t *)idx, (const int4 *)vals, n, n,
                                             rb / 16, nullptr, st);
        else if (itype == IXP_I32)
            scatter_rows_kernel<int32_t><<<g, STREAM_THREADS, 0, st>>>((char *)dst, dst_len, (const int32_t *)idx,
                                                                       (const char *)vals, n, rb);
        else
            scatter_rows_kernel<int64_t><<<g, STREAM_THREADS, 0, st>>>((char *)dst, dst_len, (const int64_t *)idx,
                                                                       (const char *)vals, n, rb);
    } else if (elem_bytes == 4) {
        if (itype == IXP_I32)
            scatter_add_kernel<int32_t, float><<<g, STREAM_THREADS, 0, st>>>((float *)dst, dst_len, (const int32_t *)idx,
                                                                             (const float *)vals, n, row_elems);
        else
            scatter_add_kernel<int64_t, float><<<g, STREAM_THREADS, 0, st>>>((float *)dst, dst_len, (const int64_t *)idx,
                                                                             (const float *)vals, n, row_elems);
    } else {
        if (itype == IXP_I32)
            scatter_add_kernel<int32_t, double><<<g, STREAM_THREADS, 0, st>>>(
                (double *)dst, dst_len, (const int32_t *)idx, (const double *)vals, n, row_elems);
        else
            scatter_add_kernel<int64_t, double><<<g, STREAM_THREADS, 0, st>>>(
                (double *)dst, dst_len, (const int64_t *)idx, (const double *)vals, n, row_elems);
    }
    return launch_status();
}

extern "C" int ixp_scatter_add_f32_to_f64(double *acc, int64_t dst_len, const void *idx, int itype, const float *vals,
                                          int64_t n, int32_t row_elems, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (n < 0 || dst_len < 0 || row_elems <= 0 || row_elems > 64 || (n > 0 && (!idx || !vals)) || (dst_len > 0 && !acc))
        return IXP_E_INVAL;
    if (!aligned_to(idx, itype == IXP_I32 ? 4 : 8) || !aligned_to(vals, 4) || !aligned_to(acc, 8)) return IXP_E_INVAL;
    if (n == 0) return IXP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int slots = row_elems <= HOT_COLS ? HOT_SLOTS : 0;
    const size_t smem = hot_smem_bytes(slots);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + HOT_THREADS - 1) / HOT_THREADS,
                                                                (int64_t)num_sms() * HOT_BLOCKS_PER_SM));
    if (itype == IXP_I32) {
        cudaFuncSetAttribute(scatter_add_f64_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        scatter_add_f64_kernel<int32_t><<<g, HOT_THREADS, smem, st>>>(acc, dst_len, (const int32_t *)idx, vals, n,
                                                                      row_elems, slots);
    } else {
        cudaFuncSetAttribute(scatter_add_f64_kernel<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        scatter_add_f64_kernel<int64_t><<<g, HOT_THREADS, smem, st>>>(acc, dst_len, (const int64_t *)idx, vals, n,
                                                                      row_elems, slots);
    }
    return launch_status();
}

extern "C" int ixp_f64_to_f32(float *out, const double *acc, int64_t count, ixp_stream stream) {
    if (count < 0 || (count > 0 && (!out || !acc))) return IXP_E_INVAL;
    if (count == 0) return IXP_OK;
    f64_to_f32_kernel<<<stream_grid(count, 4), STREAM_THREADS, 0, (cudaStream_t)stream>>>(out, acc, count);
    return launch_status();
}

template <typename IT, typename OT>
__global__ void __launch_bounds__(STREAM_THREADS) invert_kernel(const IT *__restrict__ idx, int64_t n,
                                                                OT *__restrict__ inv, int64_t inv_len) {
    IXP_KERNEL_ENTRY();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t j = (int64_t)__ldg(idx + i);
        if (j >= 0 && j < inv_len) inv[j] = (OT)i;
    }
}

extern "C" int ixp_invert(const void *idx, int itype, int64_t n, void *inv, int inv_type, int64_t inv_len,
                          ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (inv_type != IXP_I32 && inv_type != IXP_I64) return IXP_E_DTYPE;
    if (n < 0 || inv_len < 0 || (n > 0 && !idx) || (inv_len > 0 && !inv)) return IXP_E_INVAL;
    if (inv_type == IXP_I32 && n > INT32_MAX) return IXP_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t eb = inv_type == IXP_I32 ? 4 : 8;
    if (inv_len > 0 && cudaMemsetAsync(inv, 0xff, (size_t)inv_len * eb, st) != cudaSuccess) return IXP_E_CUDA;
    if (n == 0) return IXP_OK;
    const int g = row_grid(n);
    if (itype == IXP_I32) {
        if (inv_type == IXP_I32) invert_kernel<int32_t, int32_t><<<g, STREAM_THREADS, 0, st>>>((const int32_t *)idx, n, (int32_t *)inv, inv_len);
        else invert_kernel<int32_t, int64_t><<<g, STREAM_THREADS, 0, st>>>((const int32_t *)idx, n, (int64_t *)inv, inv_len);
    } else {
        if (inv_type == IXP_I32) invert_kernel<int64_t, int32_t><<<g, STREAM_THREADS, 0, st>>>((const int64_t *)idx, n, (int32_t *)inv, inv_len);
        else invert_kernel<int64_t, int64_t><<<g, STREAM_THREADS, 0, st>>>((const int64_t *)idx, n, (int64_t *)inv, inv_len);
    }
    return launch_status();
}

extern "C" int ixp_f32_to_f64(double *out, const float *in, int64_t count, ixp_stream stream) {
    if (count < 0 || (count > 0 && (!out || !in))) return IXP_E_INVAL;
    if (count == 0) return IXP_OK;
    f32_to_f64_kernel<<<stream_grid(count, 4), STREAM_THREADS, 0, (cudaStream_t)stream>>>(out, in, count);
    return launch_status();
}

extern "C" int ixp_gather(void *out, const void *src, int64_t src_len, const void *idx, int itype, int64_t n,
                          int32_t row_elems, int32_t elem_bytes, int32_t *d_status, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    if (elem_bytes != 4 && elem_bytes != 8) return IXP_E_DTYPE;
    if (n < 0 || src_len < 0 || row_elems <= 0 || row_elems > 64 || (n > 0 && (!idx || !out)) ||
        (src_len > 0 && !src))
        return IXP_E_INVAL;
    if (!aligned_to(idx, itype == IXP_I32 ? 4 : 8) || !aligned_to(out, elem_bytes) || !aligned_to(src, elem_bytes))
        return IXP_E_INVAL;
    if (n == 0) return IXP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int rb = row_elems * elem_bytes;
    const int v16 = (rb % 16 == 0) && aligned_to(out, 16) && aligned_to(src, 16);
    const int g = row_grid(n);
    if (v16 && itype == IXP_I32)
        launch_rows_lanes<int32_t, false>((int4 *)out, n, (const int32_t *)idx, (const int4 *)src, src_len, n,
                                          rb / 16, d_status, st);
    else if (v16)
        launch_rows_lanes<int64_t, false>((int4 *)out, n, (const int64_t *)idx, (const int4 *)src, src_len, n,
                                          rb / 16, d_status, st);
    else if (itype == IXP_I32)
        gather_rows_kernel<int32_t><<<g, STREAM_THREADS, 0, st>>>((char *)out, (const char *)src, src_len,
                                                                  (const int32_t *)idx, n, rb, d_status);
    else
        gather_rows_kernel<int64_t><<<g, STREAM_THREADS, 0, st>>>((char *)out, (const char *)src, src_len,
                                                                  (const int64_t *)idx, n, rb, d_status);
    return launch_status();
}

extern "C" int ixp_gather_segments(void *out, int64_t n_out, const int64_t *out_off, int64_t m, const void *src,
                                   int64_t src_len, const int64_t *src_off, int64_t src_m, const void *seg_src,
                                   int seg_type, int32_t elem_bytes, int32_t *d_status, void *ws, size_t ws_bytes,
                                   ixp_stream stream) {
    if (seg_type != IXP_I32 && seg_type != IXP_I64) return IXP_E_DTYPE;
    if (elem_bytes != 4 && elem_bytes != 8) return IXP_E_DTYPE;
    if (m < 0 || src_m < 0 || n_out < 0 || src_len < 0 || !out_off || !src_off ||
        (n_out > 0 && (m == 0 || !seg_src || !out || !src)))
        return IXP_E_INVAL;
    if (!aligned_to(out, elem_bytes) || !aligned_to(src, elem_bytes) || !aligned_to(seg_src, seg_type == IXP_I32 ? 4 : 8)) return IXP_E_INVAL;
    if (n_out == 0) return IXP_OK;
    if (!ws || !aligned_to(ws, 256) || ws_bytes < gather_segments_ws_bytes(n_out)) return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t *k0 = (int64_t *)ws;
    const unsigned g = (unsigned)((n_out + GS_CHUNK - 1) / GS_CHUNK);
    // a chunk whose start no non-empty segment covers (inconsistent offsets) keeps -1 and is clamped
    if (cudaMemsetAsync(k0, 0xff, (size_t)g * 8, st) != cudaSuccess) return IXP_E_CUDA;
    gs_chunk_table_kernel<<<stream_grid(m, 4), STREAM_THREADS, 0, st>>>(out_off, m, n_out, k0);
#define IXP_GS(E, ST)                                                                                          \
    gather_segments_kernel<E, ST><<<g, GS_THREADS, 0, st>>>((E *)out, out_off, (const E *)src, src_off,       \
                                                            (const ST *)seg_src, m, n_out, src_m, src_len, k0, \
                                                            d_status)
    if (elem_bytes == 4 && seg_type == IXP_I32) IXP_GS(uint32_t, int32_t);
    else if (elem_bytes == 4) IXP_GS(uint32_t, int64_t);
    else if (seg_type == IXP_I32) IXP_GS(unsigned long long, int32_t);
    else IXP_GS(unsigned long long, int64_t);
#undef IXP_GS
    return launch_status();
}

extern "C" int ixp_mkii(const int64_t *offsets, int64_t m, void *out, int out_type, int64_t n, int32_t *d_status,
                        void *ws, size_t ws_bytes, ixp_stream stream) {
    if (out_type != IXP_I32 && out_type != IXP_I64) return IXP_E_DTYPE;
    if (m < 0 || n < 0 || !offsets || (n > 0 && (m == 0 || !out))) return IXP_E_INVAL;
    if (out_type == IXP_I32 && m > INT32_MAX) return IXP_E_INVAL;
    if (!aligned_to(out, out_type == IXP_I32 ? 4 : 8)) return IXP_E_INVAL;
    if (n == 0) return IXP_OK;
    if (!ws || !aligned_to(ws, 256) || ws_bytes < gather_segments_ws_bytes(n)) return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t *k0 = (int64_t *)ws;
    const unsigned g = (unsigned)((n + GS_CHUNK - 1) / GS_CHUNK);
    if (cudaMemsetAsync(k0, 0xff, (size_t)g * 8, st) != cudaSuccess) return IXP_E_CUDA;
    gs_chunk_table_kernel<<<stream_grid(m, 4), STREAM_THREADS, 0, st>>>(offsets, m, n, k0);
    if (out_type == IXP_I32)
        segment_ids_kernel<int32_t><<<g, GS_THREADS, 0, st>>>((int32_t *)out, offsets, m, n, k0, d_status);
    else
        segment_ids_kernel<int64_t><<<g, GS_THREADS, 0, st>>>((int64_t *)out, offsets, m, n, k0, d_status);
    return launch_status();
}

extern "C" unsigned long long ixp_tu_kernels_scatter(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}
