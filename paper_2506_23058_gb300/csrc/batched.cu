// batched.cu - the batched pipeline over a jagged array in one persistent launch:
// for every segment k of a shape array (Sec. 2.1, mkSgmDescr / partition2L of
// Sec. 6), the flag array from the shape, the stable per-segment partition of the
// keys, and per-segment Mono / Inj / Bij checks of two given index arrays.
//
// Each CTA claims whole segments from a work list (longest first when the caller
// passes that order) and does all work of a segment by itself, so the launch needs
// no grid-wide barrier:
//   e_k      block sum of shape[0..k) (the exclusive scan of Fig. 2's mkSgmDescr)
//   flags    flags[e_k] = 1 for a non-empty segment, 0 elsewhere in it
//   count    sweep 1 over the segment's keys: T_k = number of trues
//   write    sweep 2: block-wide ranks with a carry across chunks;
//            indices[i] = e_k + trues before i, or e_k + T_k + falses before i
//   Mono     adjacent pairs of `iota` inside the segment must increase strictly
//   Inj/Bij  `chk` restricted to the segment: one bitmap pass over [min, max] of its
//            values (shared memory when the span fits, else a CTA-private bitmap in
//            global memory) flags repeats; Bij additionally needs min >= e_k and
//            max < e_{k+1}.
// Launch shape (threads, CTAs per SM, chunk length, shared bitmap size) comes from
// the caller's tuning struct, which the Python autotuner fills.
#include <algorithm>

#include "common.cuh"

namespace ixp {

constexpr unsigned long long BT_GLOBAL_BITS = 1ull << 21;  // CTA-private global bitmap (256 KB)

enum { BT_CLAIM = 10, BT_MONO = 11, BT_INJ = 12, BT_BIJ = 13 };  // header spare slots

struct DPredB {
    int kind;
    int a;
    long long b;
};

__device__ __forceinline__ bool bt_pred(const DPredB &p, int32_t key) {
    switch (p.kind) {
        case IXP_P_TRUE: return true;
        case IXP_P_MOD_EQ: {
            int64_t r = (int64_t)key % (int64_t)p.a;
            if (r < 0) r += p.a;
            return r == p.b;
        }
        default: return (int64_t)key < p.b;
    }
}

template <int NT>
__device__ __forceinline__ unsigned long long bt_block_sum(unsigned long long v, unsigned long long *sm) {
    v = warp_sum_u64(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    unsigned long long r = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; i++) r += sm[i];
    return r;  // same value in every thread
}

template <int NT, int CH>
__global__ void __launch_bounds__(NT) batch_kernel(const int64_t *__restrict__ shape, int64_t m,
                                                   const int32_t *__restrict__ keys, DPredB pred,
                                                   const int32_t *__restrict__ chk, const int32_t *__restrict__ iota,
                                                   int64_t n, const int32_t *__restrict__ order,
                                                   int32_t *__restrict__ flags, int32_t *__restrict__ indices,
                                                   int64_t *__restrict__ num_true, int64_t *__restrict__ offsets,
                                                   uint8_t *__restrict__ seg_ok, Hdr *h, unsigned *gbm,
                                                   unsigned long long smem_bits) {
    IXP_KERNEL_ENTRY();
    extern __shared__ unsigned bt_bm[];
    __shared__ unsigned long long s_red[NT / 32];
    __shared__ unsigned s_cnt[CH][NT / 32];
    __shared__ unsigned long long s_k;
    constexpr int CHUNK = NT * CH;  // elements per sweep step
    unsigned *my_gbm = gbm + (BT_GLOBAL_BITS / 32) * blockIdx.x;
    while (true) {
        if (threadIdx.x == 0) s_k = atomicAdd(&h->spare[BT_CLAIM], 1ull);
        __syncthreads();
        const unsigned long long c = s_k;
        __syncthreads();
        if (c >= (unsigned long long)m) break;
        const int64_t k = order ? (int64_t)order[c] : (int64_t)c;
        if (k < 0 || k >= m) {  // the work list must be a permutation of [0, m)
            if (threadIdx.x == 0) set_status(h, IXP_E_INVAL);
            continue;
        }
        // e_k = sum of shape[0..k); a negative size invalidates the call
        unsigned long long part = 0;
        bool neg = false;
        for (int64_t j = threadIdx.x; j < k; j += NT) {
            const int64_t s = __ldg(shape + j);
            neg |= s < 0;
            part += (unsigned long long)s;
        }
        const int64_t L0 = __ldg(shape + k);
        neg |= L0 < 0;
        const int64_t e = (int64_t)bt_block_sum<NT>(part, s_red);
        if (__syncthreads_or(neg)) {
            if (threadIdx.x == 0) set_status(h, IXP_E_INVAL);
            continue;
        }
        const int64_t a = e < 0 ? 0 : (e > n ? n : e);
        const int64_t b = (e + L0) > n ? n : (e + L0);
        if (threadIdx.x == 0) {
            offsets[k] = e;
            if (k == m - 1) {
                offsets[m] = e + L0;
                if (e + L0 != n) set_status(h, IXP_E_INVAL);
            }
        }
        if (b <= a) {
            if (threadIdx.x == 0) {
                num_true[k] = 0;
                seg_ok[k] = seg_ok[m + k] = seg_ok[2 * m + k] = 1;
            }
            continue;
        }
        // ---- sweep 1: trues, Mono of iota, min/max of chk
        unsigned long long tcount = 0;
        bool mono_bad = false;
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        for (int64_t i0 = a; i0 < b; i0 += CHUNK) {
#pragma unroll
            for (int q = 0; q < CH; q++) {
                const int64_t i = i0 + q * NT + threadIdx.x;
                if (i < b) {
                    tcount += bt_pred(pred, __ldcs(keys + i)) ? 1u : 0u;
                    const int32_t it = __ldg(iota + i);
                    if (i > a && !(__ldg(iota + i - 1) < it)) mono_bad = true;
                    const int64_t v = (int64_t)__ldcs(chk + i);
                    mn = v < mn ? v : mn;
                    mx = v > mx ? v : mx;
                }
            }
        }
        const unsigned long long T = bt_block_sum<NT>(tcount, s_red);
        const int any_mono_bad = __syncthreads_or(mono_bad);
        const unsigned long long kmn = block_max_u64(enc_min(mn), s_red);
        const unsigned long long kmx = block_max_u64(enc_max(mx), s_red);
        __shared__ long long s_mm[2];
        if (threadIdx.x == 0) {
            s_mm[0] = dec_min(kmn);
            s_mm[1] = dec_max(kmx);
        }
        __syncthreads();
        const int64_t gmn = s_mm[0], gmx = s_mm[1];
        // ---- sweep 2: partition destinations and the flag array. Element (q, warp w,
        // lane l) of a chunk sits at i0 + q * NT + 32 w + l; ranks come from ballots.
        unsigned long long carry = 0;
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        const unsigned lt = (1u << l) - 1u;
        for (int64_t i0 = a; i0 < b; i0 += CHUNK) {
            unsigned bal[CH];
#pragma unroll
            for (int q = 0; q < CH; q++) {
                const int64_t i = i0 + q * NT + threadIdx.x;
                const bool t = i < b && bt_pred(pred, __ldg(keys + i));
                bal[q] = __ballot_sync(FULL, t);
                if (l == 0) s_cnt[q][w] = __popc(bal[q]);
            }
            __syncthreads();
            unsigned before = 0, tot = 0;  // trues of this chunk before (q, w); chunk total
#pragma unroll
            for (int q = 0; q < CH; q++) {
                for (int ww = 0; ww < NT / 32; ww++) tot += s_cnt[q][ww];
            }
#pragma unroll
            for (int q = 0; q < CH; q++) {
                unsigned pq = 0;
                for (int qq = 0; qq < q; qq++)
                    for (int ww = 0; ww < NT / 32; ww++) pq += s_cnt[qq][ww];
                for (int ww = 0; ww < w; ww++) pq += s_cnt[q][ww];
                before = pq;
                const int64_t i = i0 + q * NT + threadIdx.x;
                if (i < b) {
                    const unsigned long long tb = carry + before + __popc(bal[q] & lt);
                    const bool t = (bal[q] >> l) & 1u;
                    const int64_t d = t ? a + (int64_t)tb : a + (int64_t)T + (i - a) - (int64_t)tb;
                    __stcs(indices + i, (int32_t)d);
                    __stcs(flags + i, i == a ? 1 : 0);
                }
            }
            carry += tot;
            __syncthreads();
        }
        // ---- Inj / Bij of chk over [gmn, gmx]
        const unsigned long long span = (unsigned long long)gmx - (unsigned long long)gmn + 1ull;
        bool dup = false;
        bool decided = true;
        unsigned *bm = span <= smem_bits ? bt_bm : my_gbm;
        if (span == 0 || span > BT_GLOBAL_BITS) {
            decided = false;
        } else {
            const unsigned long long words = (span + 31) / 32;
            for (unsigned long long w = threadIdx.x; w < words; w += NT) bm[w] = 0u;
            __syncthreads();
            for (int64_t i = a + threadIdx.x; i < b; i += NT) {
                const unsigned long long r = (unsigned long long)(int64_t)__ldg(chk + i) - (unsigned long long)gmn;
                const unsigned bit = 1u << (r & 31);
                if (atomicOr(bm + (r >> 5), bit) & bit) dup = true;
            }
        }
        const int any_dup = __syncthreads_or(dup);
        if (threadIdx.x == 0) {
            num_true[k] = (int64_t)T;
            const bool mono_ok = !any_mono_bad;
            const bool inj_ok = decided && !any_dup;
            const bool bij_ok = inj_ok && gmn >= a && gmx < b;
            if (!decided) set_status(h, IXP_E_SPAN);
            seg_ok[k] = mono_ok;
            seg_ok[m + k] = inj_ok;
            seg_ok[2 * m + k] = bij_ok;
            if (!mono_ok) atomicMax(&h->spare[BT_MONO], enc_first(k));
            if (!inj_ok) atomicMax(&h->spare[BT_INJ], enc_first(k));
            if (!bij_ok) atomicMax(&h->spare[BT_BIJ], enc_first(k));
        }
        __syncthreads();
    }
}

__global__ void batch_finalize(const Hdr *h, int64_t *first_bad, int32_t *status) {
    IXP_KERNEL_ENTRY();
    for (int c = 0; c < 3; c++) {
        const unsigned long long v = h->spare[BT_MONO + c];
        first_bad[c] = v ? dec_first(v) : -1;
    }
    *status = h->status;
}

static size_t rnd(size_t b) { return (b + 255) & ~(size_t)255; }

template <int NT, int CH>
static void launch_batch(int grid, size_t smem, const int64_t *shape, int64_t m, const int32_t *keys, DPredB pred,
                         const int32_t *chk, const int32_t *iota, int64_t n, const int32_t *order, int32_t *flags,
                         int32_t *indices, int64_t *num_true, int64_t *offsets, uint8_t *seg_ok, Hdr *h, unsigned *gbm,
                         unsigned long long smem_bits, cudaStream_t st) {
    cudaFuncSetAttribute(batch_kernel<NT, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_kernel<NT, CH><<<grid, NT, smem, st>>>(shape, m, keys, pred, chk, iota, n, order, flags, indices, num_true,
                                                 offsets, seg_ok, h, gbm, smem_bits);
}

}  // namespace ixp

using namespace ixp;

extern "C" size_t ixp_batch_workspace_size(const ixp_batch_tuning *tuning) {
    const int per_sm = tuning && tuning->ctas_per_sm > 0 ? tuning->ctas_per_sm : 2;
    const size_t ctas = (size_t)num_sms() * (size_t)std::min(per_sm, 8);
    return HDR_BYTES + rnd(ctas * (BT_GLOBAL_BITS / 8));
}

extern "C" int ixp_batch_run(const int64_t *shape, int64_t m, const int32_t *keys, ixp_pred pred, const int32_t *chk,
                             const int32_t *iota, int64_t n, const int32_t *order, int32_t *flags, int32_t *indices,
                             int64_t *d_num_true, int64_t *d_offsets, uint8_t *d_seg_ok, int64_t *d_first_bad,
                             int32_t *d_status, const ixp_batch_tuning *tuning, void *ws, size_t ws_bytes,
                             ixp_stream stream) {
    if (m < 1 || n < 0 || n > INT32_MAX || !shape || !d_num_true || !d_offsets || !d_seg_ok || !d_first_bad ||
        !d_status || (n > 0 && (!keys || !chk || !iota || !flags || !indices)))
        return IXP_E_INVAL;
    if (pred.kind != IXP_P_TRUE && pred.kind != IXP_P_MOD_EQ && pred.kind != IXP_P_LT) return IXP_E_INVAL;
    if (pred.kind == IXP_P_MOD_EQ && pred.a <= 0) return IXP_E_INVAL;
    ixp_batch_tuning t{256, 2, 16, 4};
    if (tuning) t = *tuning;
    if ((t.threads != 256 && t.threads != 512) || t.ctas_per_sm < 1 || t.ctas_per_sm > 8 || t.smem_bits_log2 < 10 ||
        t.smem_bits_log2 > 20 || (t.chunk != 4 && t.chunk != 8))
        return IXP_E_INVAL;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < ixp_batch_workspace_size(&t)) return IXP_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    Hdr *h = (Hdr *)ws;
    unsigned *gbm = (unsigned *)((char *)ws + HDR_BYTES);
    if (cudaMemsetAsync(h, 0, HDR_BYTES, st) != cudaSuccess) return IXP_E_CUDA;
    const DPredB p{pred.kind, pred.a, (long long)pred.b};
    const int grid = num_sms() * t.ctas_per_sm;
    const unsigned long long sbits = 1ull << t.smem_bits_log2;
    const size_t smem = sbits / 8;
    if (t.threads == 256) {
        if (t.chunk == 4)
            launch_batch<256, 4>(grid, smem, shape, m, keys, p, chk, iota, n, order, flags, indices, d_num_true,
                                 d_offsets, d_seg_ok, h, gbm, sbits, st);
        else
            launch_batch<256, 8>(grid, smem, shape, m, keys, p, chk, iota, n, order, flags, indices, d_num_true,
                                 d_offsets, d_seg_ok, h, gbm, sbits, st);
    } else {
        if (t.chunk == 4)
            launch_batch<512, 4>(grid, smem, shape, m, keys, p, chk, iota, n, order, flags, indices, d_num_true,
                                 d_offsets, d_seg_ok, h, gbm, sbits, st);
        else
            launch_batch<512, 8>(grid, smem, shape, m, keys, p, chk, iota, n, order, flags, indices, d_num_true,
                                 d_offsets, d_seg_ok, h, gbm, sbits, st);
    }
    batch_finalize<<<1, 1, 0, st>>>(h, d_first_bad, d_status);
    return cudaGetLastError() == cudaSuccess ? IXP_OK : IXP_E_CUDA;
}

extern "C" unsigned long long ixp_tu_kernels_batched(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}
