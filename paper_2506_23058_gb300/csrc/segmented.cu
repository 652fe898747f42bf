// segmented.cu - per-segment Inj and Bij (Sec. 2.3, Fig. 5: Bij with a segmented
// shape (e^m, k, e_k) and images Img_k = [e_k, e_{k+1}); Inj read as Inj of each
// segment on its own).
//
// Work is split by segment length:
//  * segments of at most 256 elements: one warp each (static striding over the
//    segments). Inj first tests strict increase (which implies Inj, the
//    monotonicity argument of rule InjF1, Sec. 3.2) and otherwise compares all
//    pairs; Bij marks a 256-bit per-warp bitmap.
//  * longer segments: one block each, claimed from a list the warp pass builds.
//    The in-Rcd values of a segment are marked in a shared-memory bitmap of up to
//    2^20 bits whose atomicOr return value flags a repeat.
//  * the rare non-increasing segment whose value span exceeds 2^20 goes to a third
//    pass of 32 blocks, each with a private 2^24-bit bitmap in global memory.
// The first failing segment (smallest k) is then re-examined by one block that
// computes the verdict's witness exactly.
#include <algorithm>

#include "common.cuh"

namespace ixp {

constexpr int SG_THREADS = 256;
constexpr int SG_SMALL = 256;                  // max elements for the warp path
constexpr unsigned long long SG_SMEM_BITS = 1ull << 20;  // shared bitmap capacity (128 KB)
constexpr unsigned long long SG_HUGE_BITS = 1ull << 24;  // private global bitmap per huge-pass block
constexpr int SG_HUGE_BLOCKS = 32;

// header slots used here (Hdr::spare)
enum { SG_NLARGE = 2, SG_NHUGE = 3, SG_KIND = 4, SG_INDEX = 5, SG_VALUE = 6, SG_AUX0 = 7, SG_AUX1 = 8, SG_HCLAIM = 9,
       SG_NSLOW = 10 };

struct SegWs {
    Hdr *h;
    unsigned *slow;   // Inj: segment ids that are not strictly increasing
    unsigned *failbm; // Inj: one bit per segment, set when it enters `slow`
    unsigned *large;  // segment ids with more than SG_SMALL elements
    unsigned *huge;   // segment ids for the global-bitmap pass
    unsigned *hbm;    // SG_HUGE_BLOCKS private bitmaps of SG_HUGE_BITS bits
    unsigned *dbm;    // two detail bitmaps of SG_HUGE_BITS bits
};

__device__ __forceinline__ void seg_bounds(const int64_t *off, int64_t k, int64_t n, int64_t &a, int64_t &b) {
    a = __ldg(off + k);
    b = __ldg(off + k + 1);
    a = a < 0 ? 0 : (a > n ? n : a);
    b = b < a ? a : (b > n ? n : b);
}

__device__ __forceinline__ void seg_fail(Hdr *h, uint8_t *seg_ok, int64_t k) {
    if (seg_ok) seg_ok[k] = 0;
    atomicMax(&h->k_first, enc_first(k));
}

// ------------------------------------------------------------- Inj pre-pass
// A strictly increasing segment is injective (the monotonicity argument of rule
// InjF1, Sec. 3.2), and so is its in-Rcd part. One streaming pass over X tests
// every in-segment adjacent pair; only the segments with a non-increasing pair are
// listed (once each, through a per-segment bit) for the exact passes below.
template <typename T>
__global__ void __launch_bounds__(SG_THREADS) seg_inj_prepass_kernel(const T *__restrict__ x, int64_t n,
                                                                     const int64_t *__restrict__ off, int64_t nseg,
                                                                     const int64_t *__restrict__ lb, SegWs W) {
    IXP_KERNEL_ENTRY();
    __shared__ SegPairsSmem<T> S;
    const int64_t nchunks = (n + SP_CHUNK - 1) / SP_CHUNK;
    for (int64_t t = blockIdx.x; t < nchunks; t += gridDim.x) {
        seg_pairs_chunk<T>(x, n, off, nseg, t * SP_CHUNK, S, lb, [&](int64_t j, T a, T b) {
            if (a < b) return;
            const int64_t k = off_segment_of(off, nseg, j);
            const unsigned bit = 1u << (k & 31);
            if (!(atomicOr(W.failbm + (k >> 5), bit) & bit))
                W.slow[atomicAdd(&W.h->spare[SG_NSLOW], 1ull)] = (unsigned)k;
        });
    }
}

// ------------------------------------------------------------- warp pass
// `listed`: visit only the segments of W.slow (the Inj pre-pass), else all of them.
template <typename T, bool BIJ>
__global__ void __launch_bounds__(SG_THREADS) seg_warp_kernel(const T *__restrict__ x, int64_t n, int64_t rlo,
                                                              int64_t rhi, const int64_t *__restrict__ off,
                                                              int64_t nseg, uint8_t *seg_ok, SegWs W, int listed) {
    IXP_KERNEL_ENTRY();
    __shared__ T s_val[SG_THREADS / 32][SG_SMALL];
    __shared__ unsigned s_bits[SG_THREADS / 32][SG_SMALL / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Hdr *h = W.h;
    unsigned long long cnt_all = 0;
    const int64_t count = listed ? (int64_t)min((unsigned long long)nseg, h->spare[SG_NSLOW]) : nseg;
    for (int64_t it = gw; it < count; it += nw) {
        const int64_t k = listed ? (int64_t)W.slow[it] : it;
        int64_t a, b;
        seg_bounds(off, k, n, a, b);
        const int64_t L = b - a;
        if (L > SG_SMALL) {
            if (lane == 0) W.large[atomicAdd(&h->spare[SG_NLARGE], 1ull)] = (unsigned)k;
            continue;
        }
        bool bad = false;
        if (BIJ) {
            if (lane < SG_SMALL / 32) s_bits[wib][lane] = 0u;
            __syncwarp();
            unsigned cnt = 0;
            for (int64_t i = lane; i < L; i += 32) {
                const int64_t v = (int64_t)x[a + i];
                if (v < rlo || v > rhi) continue;
                if (v < a || v >= b) {
                    bad = true;
                    continue;
                }
                const unsigned r = (unsigned)(v - a), bit = 1u << (r & 31);
                if (atomicOr(&s_bits[wib][r >> 5], bit) & bit) bad = true;
                cnt++;
            }
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
            bad = __any_sync(FULL, bad) || cnt != (unsigned)L;
            cnt_all += lane == 0 ? cnt : 0;
        } else {
            bool ns = false;
            for (int64_t i = lane + 1; i < L; i += 32)
                if (!(x[a + i - 1] < x[a + i])) ns = true;
            if (__any_sync(FULL, ns)) {
                // all pairs of in-Rcd values
                for (int64_t i = lane; i < L; i += 32) s_val[wib][i] = x[a + i];
                __syncwarp();
                for (int64_t i = lane; i < L && !bad; i += 32) {
                    const T v = s_val[wib][i];
                    if ((int64_t)v < rlo || (int64_t)v > rhi) continue;
                    for (int64_t j = 0; j < L; j++)
                        if (j != i && s_val[wib][j] == v) {
                            bad = true;
                            break;
                        }
                }
                bad = __any_sync(FULL, bad);
                __syncwarp();
            }
        }
        if (lane == 0) {
            if (bad) seg_fail(h, seg_ok, k);
            else if (seg_ok) seg_ok[k] = 1;
        }
    }
    if (BIJ && lane == 0 && cnt_all) atomicAdd(&h->cnt0, cnt_all);
}

// ----------------------------------------------------------- block pass
// Examines segment [a, b) with all threads of the block. Returns 1 (holds),
// 0 (fails) or 2 (needs the global-bitmap pass). Adds the Bij in-image count.
template <typename T, bool BIJ>
__device__ int block_check(const T *__restrict__ x, int64_t a, int64_t b, int64_t rlo, int64_t rhi,
                           unsigned *bm, unsigned long long bm_bits, bool global_bm, Hdr *h) {
    __shared__ unsigned long long s_red[SG_THREADS / 32];
    __shared__ int s_flag;
    const int64_t L = b - a;
    int64_t base;
    unsigned long long span;
    if (BIJ) {
        base = a;
        span = (unsigned long long)L;
    } else {
        // strict increase, and the in-Rcd value range
        bool ns = false;
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
            const T v = x[i];
            if (i > a && !(x[i - 1] < v)) ns = true;
            const int64_t vi = (int64_t)v;
            if (vi >= rlo && vi <= rhi) {
                mn = vi < mn ? vi : mn;
                mx = vi > mx ? vi : mx;
            }
        }
        const int any_ns = __syncthreads_or(ns);
        if (!any_ns) return 1;
        const unsigned long long kmn = block_max_u64(enc_min(mn), s_red);
        const unsigned long long kmx = block_max_u64(enc_max(mx), s_red);
        if (threadIdx.x == 0) {
            s_red[0] = kmn;
            s_red[1] = kmx;
        }
        __syncthreads();
        const int64_t gmn = dec_min(s_red[0]), gmx = dec_max(s_red[1]);
        __syncthreads();
        if (gmn > gmx) return 1;  // no value inside Rcd
        base = gmn;
        span = (unsigned long long)gmx - (unsigned long long)gmn + 1ull;
    }
    if (span == 0 || span > bm_bits) return 2;  // span 0: the full 64-bit range
    const unsigned long long words = (span + 31) / 32;
    for (unsigned long long w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    bool bad = false;
    unsigned long long cnt = 0;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const int64_t v = (int64_t)x[i];
        if (v < rlo || v > rhi) continue;
        if (BIJ && (v < a || v >= b)) {
            bad = true;
            continue;
        }
        const unsigned long long r = (unsigned long long)v - (unsigned long long)base;
        const unsigned bit = 1u << (r & 31);
        if (atomicOr(bm + (r >> 5), bit) & bit) bad = true;
        cnt++;
    }
    if (BIJ) {
        const unsigned long long c = block_sum_u64(cnt, s_red);
        if (threadIdx.x == 0) {
            atomicAdd(&h->cnt0, c);
            if (c != (unsigned long long)L) s_flag = 1;
        }
    }
    const int any_bad = __syncthreads_or(bad);
    const int res = (any_bad || s_flag) ? 0 : 1;
    __syncthreads();
    (void)global_bm;
    return res;
}

template <typename T, bool BIJ>
__global__ void __launch_bounds__(SG_THREADS) seg_block_kernel(const T *__restrict__ x, int64_t n, int64_t rlo,
                                                               int64_t rhi, const int64_t *__restrict__ off,
                                                               uint8_t *seg_ok, SegWs W) {
    IXP_KERNEL_ENTRY();
    extern __shared__ unsigned sg_bm[];
    __shared__ unsigned long long s_k;
    Hdr *h = W.h;
    const unsigned long long nl = h->spare[SG_NLARGE];
    while (true) {
        if (threadIdx.x == 0) s_k = atomicAdd(&h->tile_ctr, 1u);
        __syncthreads();
        const unsigned long long c = s_k;
        __syncthreads();
        if (c >= nl) break;
        const int64_t k = W.large[c];
        int64_t a, b;
        seg_bounds(off, k, n, a, b);
        const int r = block_check<T, BIJ>(x, a, b, rlo, rhi, sg_bm, SG_SMEM_BITS, false, h);
        if (threadIdx.x == 0) {
            if (r == 2) W.huge[atomicAdd(&h->spare[SG_NHUGE], 1ull)] = (unsigned)k;
            else if (r == 0) seg_fail(h, seg_ok, k);
            else if (seg_ok) seg_ok[k] = 1;
        }
    }
}

template <typename T, bool BIJ>
__global__ void __launch_bounds__(SG_THREADS) seg_huge_kernel(const T *__restrict__ x, int64_t n, int64_t rlo,
                                                              int64_t rhi, const int64_t *__restrict__ off,
                                                              uint8_t *seg_ok, SegWs W) {
    IXP_KERNEL_ENTRY();
    __shared__ unsigned long long s_k;
    Hdr *h = W.h;
    const unsigned long long nh = h->spare[SG_NHUGE];
    unsigned *bm = W.hbm + (SG_HUGE_BITS / 32) * blockIdx.x;
    while (true) {
        if (threadIdx.x == 0) s_k = atomicAdd(&h->spare[SG_HCLAIM], 1ull);
        __syncthreads();
        const unsigned long long c = s_k;
        __syncthreads();
        if (c >= nh) break;
        const int64_t k = W.huge[c];
        int64_t a, b;
        seg_bounds(off, k, n, a, b);
        const int r = block_check<T, BIJ>(x, a, b, rlo, rhi, bm, SG_HUGE_BITS, true, h);
        if (threadIdx.x == 0) {
            if (r == 2) {
                set_status(h, IXP_E_SPAN);
                seg_fail(h, seg_ok, k);
            } else if (r == 0) {
                seg_fail(h, seg_ok, k);
            } else if (seg_ok) {
                seg_ok[k] = 1;
            }
        }
    }
}

// ---------------------------------------------------------- detail pass
// One block re-examines the first failing segment k* with two global bitmaps
// (marks, repeats) and writes the witness into the header.
template <typename T, bool BIJ>
__global__ void __launch_bounds__(SG_THREADS) seg_detail_kernel(const T *__restrict__ x, int64_t n, int64_t rlo,
                                                                int64_t rhi, const int64_t *__restrict__ off,
                                                                SegWs W) {
    IXP_KERNEL_ENTRY();
    Hdr *h = W.h;
    if (h->status || !h->k_first) return;
    __shared__ unsigned long long s_red[SG_THREADS / 32];
    __shared__ long long s_v[4];
    const int64_t k = dec_first(h->k_first);
    int64_t a, b;
    seg_bounds(off, k, n, a, b);
    int64_t base;
    unsigned long long span;
    if (BIJ) {
        base = a;
        span = (unsigned long long)(b - a);
    } else {
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
            const int64_t v = (int64_t)x[i];
            if (v >= rlo && v <= rhi) {
                mn = v < mn ? v : mn;
                mx = v > mx ? v : mx;
            }
        }
        const unsigned long long kmn = block_max_u64(enc_min(mn), s_red);
        const unsigned long long kmx = block_max_u64(enc_max(mx), s_red);
        if (threadIdx.x == 0) {
            s_v[0] = dec_min(kmn);
            s_v[1] = dec_max(kmx);
        }
        __syncthreads();
        base = s_v[0];
        span = s_v[0] <= s_v[1] ? (unsigned long long)s_v[1] - (unsigned long long)s_v[0] + 1ull : 0ull;
        __syncthreads();
    }
    if ((!BIJ && span == 0) || span > SG_HUGE_BITS) {
        if (threadIdx.x == 0) set_status(h, IXP_E_SPAN);
        return;
    }
    unsigned *mk = W.dbm, *rp = W.dbm + SG_HUGE_BITS / 32;
    const unsigned long long words = (span + 31) / 32;
    for (unsigned long long w = threadIdx.x; w < words; w += blockDim.x) {
        mk[w] = 0u;
        rp[w] = 0u;
    }
    __syncthreads();
    int64_t ooi = INT64_MAX;
    unsigned long long cnt = 0;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const int64_t v = (int64_t)x[i];
        if (v < rlo || v > rhi) continue;
        if (BIJ && (v < a || v >= b)) {
            ooi = i < ooi ? i : ooi;
            continue;
        }
        const unsigned long long r = (unsigned long long)v - (unsigned long long)base;
        const unsigned bit = 1u << (r & 31);
        if (atomicOr(mk + (r >> 5), bit) & bit) atomicOr(rp + (r >> 5), bit);
        cnt++;
    }
    __threadfence_block();
    __syncthreads();
    // smallest index whose value repeats inside the segment
    int64_t di = INT64_MAX;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const int64_t v = (int64_t)x[i];
        if (v < rlo || v > rhi || (BIJ && (v < a || v >= b))) continue;
        const unsigned long long r = (unsigned long long)v - (unsigned long long)base;
        if (atomicOr(rp + (r >> 5), 0u) & (1u << (r & 31))) {
            di = i;
            break;
        }
    }
    const unsigned long long kdi = block_max_u64(di == INT64_MAX ? 0ull : enc_first(di), s_red);
    const unsigned long long kooi = block_max_u64(ooi == INT64_MAX ? 0ull : enc_first(ooi), s_red);
    const unsigned long long ccnt = block_sum_u64(cnt, s_red);
    if (threadIdx.x == 0) {
        s_v[0] = kdi ? dec_first(kdi) : -1;
        s_v[1] = kooi ? dec_first(kooi) : -1;
    }
    __syncthreads();
    const int64_t i0 = s_v[0], o0 = s_v[1];
    if (!BIJ) {
        // partner: the next j > i0 with the same value
        int64_t pj = INT64_MAX;
        if (i0 >= 0) {
            const T v0 = x[i0];
            for (int64_t j = i0 + 1 + threadIdx.x; j < b; j += blockDim.x)
                if (x[j] == v0) {
                    pj = j;
                    break;
                }
        }
        const unsigned long long kpj = block_max_u64(pj == INT64_MAX ? 0ull : enc_first(pj), s_red);
        if (threadIdx.x == 0) {
            h->spare[SG_KIND] = IXP_V_DUPLICATE;
            h->spare[SG_INDEX] = (unsigned long long)i0;
            h->spare[SG_VALUE] = i0 >= 0 ? (unsigned long long)(int64_t)x[i0] : 0ull;
            h->spare[SG_AUX0] = kpj ? (unsigned long long)dec_first(kpj) : ~0ull;
            h->spare[SG_AUX1] = 0ull;
        }
        return;
    }
    // Bij: out of image vs repeat by index, else the smallest missing image value
    int64_t miss = INT64_MAX;
    if (o0 < 0 && i0 < 0) {
        for (unsigned long long w = threadIdx.x; w < words; w += blockDim.x) {
            unsigned z = ~atomicOr(mk + w, 0u);
            if (w == words - 1 && (span & 31)) z &= (1u << (span & 31)) - 1u;
            if (z) {
                miss = (int64_t)(w * 32 + (__ffs(z) - 1));
                break;
            }
        }
    }
    const unsigned long long kms = block_max_u64(miss == INT64_MAX ? 0ull : enc_first(miss), s_red);
    if (threadIdx.x == 0) {
        h->spare[SG_AUX0] = ccnt;
        h->spare[SG_AUX1] = (unsigned long long)(b - a);
        if (o0 >= 0 && (i0 < 0 || o0 < i0)) {
            h->spare[SG_KIND] = IXP_V_OUT_OF_IMAGE;
            h->spare[SG_INDEX] = (unsigned long long)o0;
            h->spare[SG_VALUE] = (unsigned long long)(int64_t)x[o0];
        } else if (i0 >= 0) {
            h->spare[SG_KIND] = IXP_V_DUPLICATE;
            h->spare[SG_INDEX] = (unsigned long long)i0;
            h->spare[SG_VALUE] = (unsigned long long)(int64_t)x[i0];
        } else {
            h->spare[SG_KIND] = IXP_V_MISSING;
            h->spare[SG_INDEX] = ~0ull;
            h->spare[SG_VALUE] = (unsigned long long)(a + (kms ? dec_first(kms) : 0));
        }
    }
}

__global__ void seg_finalize(const Hdr *h, ixp_verdict *out, int bij, int64_t n) {
    IXP_KERNEL_ENTRY();
    ixp_verdict v;
    v.status = h->status;
    v.reserved = 0;
    if (v.status) {
        v.ok = -1;
        v.kind = IXP_V_NONE;
        v.index = -1;
        v.value = 0;
        v.aux0 = 0;
        v.aux1 = 0;
    } else if (!h->k_first) {
        v.ok = 1;
        v.kind = IXP_V_NONE;
        v.index = -1;
        v.value = 0;
        v.aux0 = bij ? (int64_t)h->cnt0 : 0;
        v.aux1 = bij ? n : 0;
    } else {
        v.ok = 0;
        v.kind = (int32_t)h->spare[SG_KIND];
        v.index = (int64_t)h->spare[SG_INDEX];
        v.value = (int64_t)h->spare[SG_VALUE];
        v.aux0 = (int64_t)h->spare[SG_AUX0];
        v.aux1 = (int64_t)h->spare[SG_AUX1];
    }
    *out = v;
}

static size_t rnd(size_t b) { return (b + 255) & ~(size_t)255; }

size_t seg_ws_bytes(int64_t nseg) {
    const size_t ns = (size_t)(nseg > 0 ? nseg : 1);
    return HDR_BYTES + 3 * rnd(ns * 4) + rnd((ns + 31) / 32 * 4) + rnd(SG_HUGE_BLOCKS * (SG_HUGE_BITS / 8)) +
           rnd(2 * (SG_HUGE_BITS / 8));
}

static SegWs seg_ws(void *ws, int64_t nseg) {
    SegWs w;
    char *p = (char *)ws;
    size_t o = HDR_BYTES;
    w.h = (Hdr *)p;
    const size_t ns = (size_t)(nseg > 0 ? nseg : 1);
    w.slow = (unsigned *)(p + o);
    o += rnd(ns * 4);
    w.failbm = (unsigned *)(p + o);
    o += rnd((ns + 31) / 32 * 4);
    w.large = (unsigned *)(p + o);
    o += rnd((size_t)(nseg > 0 ? nseg : 1) * 4);
    w.huge = (unsigned *)(p + o);
    o += rnd((size_t)(nseg > 0 ? nseg : 1) * 4);
    w.hbm = (unsigned *)(p + o);
    o += rnd(SG_HUGE_BLOCKS * (SG_HUGE_BITS / 8));
    w.dbm = (unsigned *)(p + o);
    return w;
}

template <typename T, bool BIJ>
static int run_seg(const T *x, int64_t n, int64_t rlo, int64_t rhi, ixp_segs segs, ixp_verdict *out,
                   uint8_t *seg_ok, void *ws, cudaStream_t st) {
    SegWs W = seg_ws(ws, segs.nseg);
    if (cudaMemsetAsync(W.h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    const int sms = num_sms();
    const int64_t warps_needed = segs.nseg;
    const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>((warps_needed + 7) / 8, (int64_t)sms * 8));
    if (!BIJ) {
        // segments the pre-pass does not list hold; the exact passes settle the listed ones
        if (cudaMemsetAsync(W.failbm, 0, ((size_t)segs.nseg + 31) / 32 * 4, st) != cudaSuccess) return IXP_E_CUDA;
        if (seg_ok && cudaMemsetAsync(seg_ok, 1, (size_t)segs.nseg, st) != cudaSuccess) return IXP_E_CUDA;
        if (n > 0) {
            const int64_t chunks = (n + SP_CHUNK - 1) / SP_CHUNK;
            int64_t *lb = (int64_t *)((char *)ws + seg_ws_bytes(segs.nseg));
            if (cudaMemsetAsync(lb, 0, (size_t)chunks * 8, st) != cudaSuccess) return IXP_E_CUDA;
            chunk_lb_kernel<SP_CHUNK><<<stream_grid(segs.nseg + 1, 4), STREAM_THREADS, 0, st>>>(segs.offsets,
                                                                                               segs.nseg, n, lb);
            const int gp = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)sms * 8));
            seg_inj_prepass_kernel<T><<<gp, SG_THREADS, 0, st>>>(x, n, segs.offsets, segs.nseg, lb, W);
        }
    }
    seg_warp_kernel<T, BIJ><<<g1, SG_THREADS, 0, st>>>(x, n, rlo, rhi, segs.offsets, segs.nseg, seg_ok, W, BIJ ? 0 : 1);
    const size_t smem = SG_SMEM_BITS / 8;
    cudaFuncSetAttribute(seg_block_kernel<T, BIJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    seg_block_kernel<T, BIJ><<<sms, SG_THREADS, smem, st>>>(x, n, rlo, rhi, segs.offsets, seg_ok, W);
    seg_huge_kernel<T, BIJ><<<SG_HUGE_BLOCKS, SG_THREADS, 0, st>>>(x, n, rlo, rhi, segs.offsets, seg_ok, W);
    seg_detail_kernel<T, BIJ><<<1, SG_THREADS, 0, st>>>(x, n, rlo, rhi, segs.offsets, W);
    seg_finalize<<<1, 1, 0, st>>>(W.h, out, BIJ ? 1 : 0, n);
    return cudaGetLastError() == cudaSuccess ? IXP_OK : IXP_E_CUDA;
}

template <bool BIJ>
static int seg_entry(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, ixp_segs segs,
                     ixp_verdict *d_verdict, uint8_t *d_seg_ok, void *ws, size_t ws_bytes, ixp_stream stream) {
    if (itype != IXP_I32 && itype != IXP_I64) return IXP_E_DTYPE;
    const int es = itype == IXP_I32 ? 4 : 8;
    if (n < 0 || rcd_lo > rcd_hi || !d_verdict || (n > 0 && (!x || (reinterpret_cast<uintptr_t>(x) % es))))
        return IXP_E_INVAL;
    if (!segs.offsets || segs.nseg < 1 || segs.nseg >= (1ll << 32)) return IXP_E_INVAL;
    if (BIJ && n > 0 && (rcd_lo > 0 || rcd_hi < n - 1)) return IXP_E_INVAL;  // every Img_k must lie inside Rcd
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < seg_ws_bytes(segs.nseg) + chunk_lb_bytes(n))
        return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (itype == IXP_I32)
        return run_seg<int32_t, BIJ>((const int32_t *)x, n, rcd_lo, rcd_hi, segs, d_verdict, d_seg_ok, ws, st);
    return run_seg<int64_t, BIJ>((const int64_t *)x, n, rcd_lo, rcd_hi, segs, d_verdict, d_seg_ok, ws, st);
}

}  // namespace ixp

extern "C" int ixp_check_inj_seg(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, ixp_segs segs,
                                 ixp_verdict *d_verdict, uint8_t *d_seg_ok, void *ws, size_t ws_bytes,
                                 ixp_stream stream) {
    return ixp::seg_entry<false>(x, itype, n, rcd_lo, rcd_hi, segs, d_verdict, d_seg_ok, ws, ws_bytes, stream);
}

extern "C" int ixp_check_bij_seg(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, ixp_segs segs,
                                 ixp_verdict *d_verdict, uint8_t *d_seg_ok, void *ws, size_t ws_bytes,
                                 ixp_stream stream) {
    return ixp::seg_entry<true>(x, itype, n, rcd_lo, rcd_hi, segs, d_verdict, d_seg_ok, ws, ws_bytes, stream);
}

extern "C" unsigned long long ixp_tu_kernels_segmented(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}
