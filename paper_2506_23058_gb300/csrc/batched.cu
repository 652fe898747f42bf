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
    __shared__ unsigned long long s_k, s_carry;
    __shared__ long long s_mm[2];
    constexpr int U = 4;  // 16-byte vectors in flight per thread in sweep 1
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    unsigned *my_gbm = gbm + (BT_GLOBAL_BITS / 32) * blockIdx.x;
    while (true) {
        if (tid == 0) s_k = atomicAdd(&h->spare[BT_CLAIM], 1ull);
        __syncthreads();
        const unsigned long long c = s_k;
        __syncthreads();
        if (c >= (unsigned long long)m) break;
        const int64_t k = order ? (int64_t)order[c] : (int64_t)c;
        if (k < 0 || k >= m) {  // the work list must be a permutation of [0, m)
            if (tid == 0) set_status(h, IXP_E_INVAL);
            continue;
        }
        // e_k = sum of shape[0..k); a negative size invalidates the call
        unsigned long long part = 0;
        bool neg = false;
        for (int64_t j = tid; j < k; j += NT) {
            const int64_t sj = __ldg(shape + j);
            neg |= sj < 0;
            part += (unsigned long long)sj;
        }
        const int64_t L0 = __ldg(shape + k);
        neg |= L0 < 0;
        const int64_t e = (int64_t)bt_block_sum<NT>(part, s_red);
        if (__syncthreads_or(neg)) {
            if (tid == 0) set_status(h, IXP_E_INVAL);
            continue;
        }
        const int64_t a = e < 0 ? 0 : (e > n ? n : e);
        const int64_t b = (e + L0) > n ? n : (e + L0);
        if (tid == 0) {
            offsets[k] = e;
            if (k == m - 1) {
                offsets[m] = e + L0;
                if (e + L0 != n) set_status(h, IXP_E_INVAL);
            }
        }
        if (b <= a) {
            if (tid == 0) {
                num_true[k] = 0;
                seg_ok[k] = seg_ok[m + k] = seg_ok[2 * m + k] = 1;
            }
            continue;
        }
        const int64_t L = b - a;
        // head [a, a4), body of whole 16-byte vectors [a4, b4), tail [b4, b)
        const int64_t a4 = min(b, (a + 3) & ~(int64_t)3);
        const int64_t nv = (b - a4) / 4;
        const int64_t b4 = a4 + 4 * nv;
        // bitmap over the segment's image [a, b) for chk
        const bool img_fits = (unsigned long long)L <= BT_GLOBAL_BITS;
        unsigned *bm = (unsigned long long)L <= smem_bits ? bt_bm : my_gbm;
        if (img_fits)
            for (int64_t q = tid; q < (L + 31) / 32; q += NT) bm[q] = 0u;
        __syncthreads();
        // ---- sweep 1: trues, Mono of iota, image marks and min/max of chk
        unsigned long long tcount = 0;
        bool mono_bad = false, dup = false, outside = false;
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        auto visit = [&](int64_t i, int32_t kv, int32_t it, int32_t it_prev, int32_t cv) {
            tcount += bt_pred(pred, kv) ? 1u : 0u;
            if (i > a && !(it_prev < it)) mono_bad = true;
            const int64_t v = cv;
            mn = v < mn ? v : mn;
            mx = v > mx ? v : mx;
            if (v < a || v >= b) {
                outside = true;
            } else if (img_fits) {
                const unsigned r = (unsigned)(v - a), bit = 1u << (r & 31);
                if (atomicOr(bm + (r >> 5), bit) & bit) dup = true;
            }
        };
        if (tid < 3) {
            const int64_t i = a + tid;
            if (i < a4) visit(i, keys[i], iota[i], i > a ? iota[i - 1] : 0, chk[i]);
            const int64_t j = b4 + tid;
            if (j < b) visit(j, keys[j], iota[j], j > a ? iota[j - 1] : 0, chk[j]);
        }
        for (int64_t v0 = tid; v0 < nv; v0 += (int64_t)NT * U) {
            int4 kq[U], iq[U], cq[U];
            int32_t ip[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t v = v0 + (int64_t)u * NT;
                if (v < nv) {
                    const int64_t p = a4 + 4 * v;
                    kq[u] = __ldcs(reinterpret_cast<const int4 *>(keys + p));
                    iq[u] = __ldcs(reinterpret_cast<const int4 *>(iota + p));
                    cq[u] = __ldcs(reinterpret_cast<const int4 *>(chk + p));
                    ip[u] = p > a ? __ldg(iota + p - 1) : 0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t v = v0 + (int64_t)u * NT;
                if (v < nv) {
                    const int64_t p = a4 + 4 * v;
                    visit(p, kq[u].x, iq[u].x, ip[u], cq[u].x);
                    visit(p + 1, kq[u].y, iq[u].y, iq[u].x, cq[u].y);
                    visit(p + 2, kq[u].z, iq[u].z, iq[u].y, cq[u].z);
                    visit(p + 3, kq[u].w, iq[u].w, iq[u].z, cq[u].w);
                }
            }
        }
        const unsigned long long T = bt_block_sum<NT>(tcount, s_red);
        const int any_mono_bad = __syncthreads_or(mono_bad);
        const int any_dup = __syncthreads_or(dup);
        const int any_out = __syncthreads_or(outside);
        const unsigned long long kmn = block_max_u64(enc_min(mn), s_red);
        const unsigned long long kmx = block_max_u64(enc_max(mx), s_red);
        if (tid == 0) {
            s_mm[0] = dec_min(kmn);
            s_mm[1] = dec_max(kmx);
        }
        __syncthreads();
        // ---- sweep 2: partition destinations and the flag array
        auto dest = [&](int64_t i, bool t, unsigned long long tb) -> int32_t {
            return (int32_t)(t ? a + (int64_t)tb : a + (int64_t)T + (i - a) - (int64_t)tb);
        };
        if (tid == 0) {  // head elements, in order
            unsigned long long cc = 0;
            for (int64_t i = a; i < a4; i++) {
                const bool t = bt_pred(pred, keys[i]);
                indices[i] = dest(i, t, cc);
                flags[i] = i == a ? 1 : 0;
                cc += t ? 1u : 0u;
            }
            s_carry = cc;
        }
        __syncthreads();
        unsigned long long carry = s_carry;
        const unsigned ltm = (1u << l) - 1u;
        for (int64_t c0 = 0; c0 < nv; c0 += (int64_t)NT * CH) {
            unsigned msk[CH], lpre[CH];
            int4 kq[CH];
#pragma unroll
            for (int q = 0; q < CH; q++) {
                const int64_t v = c0 + (int64_t)q * NT + tid;
                msk[q] = 0;
                if (v < nv) {
                    kq[q] = __ldg(reinterpret_cast<const int4 *>(keys + a4 + 4 * v));
                    msk[q] = (bt_pred(pred, kq[q].x) ? 1u : 0u) | (bt_pred(pred, kq[q].y) ? 2u : 0u) |
                             (bt_pred(pred, kq[q].z) ? 4u : 0u) | (bt_pred(pred, kq[q].w) ? 8u : 0u);
                }
                const unsigned x = __popc(msk[q]);
                unsigned y = x;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const unsigned o = __shfl_up_sync(FULL, y, d);
                    if (l >= d) y += o;
                }
                lpre[q] = y - x;
                if (l == 31) s_cnt[q][w] = y;
            }
            __syncthreads();
            unsigned tot = 0, run = 0;
#pragma unroll
            for (int q = 0; q < CH; q++) {
                unsigned before = run;  // all of q' < q
                for (int ww = 0; ww < NT / 32; ww++) {
                    const unsigned cq2 = s_cnt[q][ww];
                    if (ww < w) before += cq2;
                    run += cq2;
                }
                const int64_t v = c0 + (int64_t)q * NT + tid;
                if (v < nv) {
                    const int64_t p = a4 + 4 * v;
                    const unsigned long long tb0 = carry + before + lpre[q];
                    int4 o, f;
                    o.x = dest(p, msk[q] & 1u, tb0);
                    o.y = dest(p + 1, (msk[q] >> 1) & 1u, tb0 + __popc(msk[q] & 1u));
                    o.z = dest(p + 2, (msk[q] >> 2) & 1u, tb0 + __popc(msk[q] & 3u));
                    o.w = dest(p + 3, (msk[q] >> 3) & 1u, tb0 + __popc(msk[q] & 7u));
                    f.x = p == a ? 1 : 0;
                    f.y = f.z = f.w = 0;
                    __stcs(reinterpret_cast<int4 *>(indices + p), o);
                    __stcs(reinterpret_cast<int4 *>(flags + p), f);
                }
            }
            tot = run;
            carry += tot;
            __syncthreads();
        }
        if (tid == 0) {  // tail elements, in order
            unsigned long long cc = carry;
            for (int64_t i = b4; i < b; i++) {
                const bool t = bt_pred(pred, keys[i]);
                indices[i] = dest(i, t, cc);
                flags[i] = i == a ? 1 : 0;
                cc += t ? 1u : 0u;
            }
        }
        (void)ltm;
        // ---- Inj when some chk value lies outside the segment's image: one more
        // bitmap pass over [min, max] (rare; decides Inj, Bij has failed already)
        const int64_t gmn = s_mm[0], gmx = s_mm[1];
        bool inj_decided = img_fits && !any_out;
        bool inj_dup = any_dup;
        if (any_out) {
            const unsigned long long span = (unsigned long long)gmx - (unsigned long long)gmn + 1ull;
            if (span != 0 && span <= BT_GLOBAL_BITS) {
                unsigned *bm2 = span <= smem_bits ? bt_bm : my_gbm;
                __syncthreads();
                for (unsigned long long q = tid; q < (span + 31) / 32; q += NT) bm2[q] = 0u;
                __syncthreads();
                bool d2 = false;
                for (int64_t i = a + tid; i < b; i += NT) {
                    const unsigned long long r = (unsigned long long)(int64_t)__ldg(chk + i) - (unsigned long long)gmn;
                    const unsigned bit = 1u << (r & 31);
                    if (atomicOr(bm2 + (r >> 5), bit) & bit) d2 = true;
                }
                inj_dup = __syncthreads_or(d2);
                inj_decided = true;
            } else {
                inj_decided = false;
            }
        }
        if (tid == 0) {
            num_true[k] = (int64_t)T;
            const bool mono_ok = !any_mono_bad;
            const bool inj_ok = inj_decided && !inj_dup;
            const bool bij_ok = img_fits && !any_out && !any_dup;  // L distinct values inside an L-value image
            if (!inj_decided || !img_fits) set_status(h, IXP_E_SPAN);
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
    const uintptr_t al = reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(chk) |
                         reinterpret_cast<uintptr_t>(iota) | reinterpret_cast<uintptr_t>(flags) |
                         reinterpret_cast<uintptr_t>(indices);
    if (al & 15u) return IXP_E_INVAL;  // the five element arrays must be 16-byte aligned
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
    return launch_status();
}

extern "C" unsigned long long ixp_tu_kernels_batched(void) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ixp::tu_kernel_count, sizeof(v)) != cudaSuccess) return 0;
    return v;
}
