// preds.cuh - the partition predicates of the C ABI (TRUE, floored MOD_EQ, LT,
// FLAGS) on the device, evaluated for one 16-byte slot of keys at a time, and the
// slot loads that feed them. Shared by the partition / FiltPart translation units.
#pragma once

#include "common.cuh"

namespace ixp {

struct DPred {
    int kind;
    int a;
    long long b;
    const uint8_t *flags;
};

// Predicate over the V keys of one vector slot at positions p0..p0+V-1, as a
// V-bit mask (positions at or past n are 0). The kind is tested once per slot and
// 32-bit keys are compared in 32-bit arithmetic: a bound outside the int32 range
// makes LT constant, and MOD_EQ (a > 0, result in [0, a)) runs as a 32-bit
// remainder.
// The predicate at one element (key widened to int64, position i).
__device__ __forceinline__ bool pred_one(const DPred &p, int64_t key, int64_t i) {
    switch (p.kind) {
        case IXP_P_TRUE: return true;
        case IXP_P_LT: return key < p.b;
        case IXP_P_MOD_EQ: {
            if (p.b < 0 || p.b >= (long long)p.a) return false;
            int64_t r = key % (int64_t)p.a;
            r += r < 0 ? (int64_t)p.a : 0;
            return r == p.b;
        }
        default: return __ldg(p.flags + i) != 0;
    }
}

template <typename KT, int V>
__device__ __forceinline__ unsigned pred_mask(const DPred &p, const KT (&kv)[V], int64_t p0, int64_t n) {
    const unsigned valid = p0 + V <= n ? (1u << V) - 1u : (p0 >= n ? 0u : (1u << (unsigned)(n - p0)) - 1u);
    unsigned m = 0;
    switch (p.kind) {
        case IXP_P_TRUE: return valid;
        case IXP_P_LT:
            if (sizeof(KT) == 4) {
                if (p.b > (long long)INT32_MAX) return valid;
                if (p.b <= (long long)INT32_MIN) return 0u;
                const int32_t b = (int32_t)p.b;
#pragma unroll
                for (int k = 0; k < V; k++) m |= (unsigned)((int32_t)kv[k] < b) << k;
            } else {
#pragma unroll
                for (int k = 0; k < V; k++) m |= (unsigned)((int64_t)kv[k] < p.b) << k;
            }
            return m & valid;
        case IXP_P_MOD_EQ:
            if (p.b < 0 || p.b >= (long long)p.a) return 0u;
            if (sizeof(KT) == 4) {
                const int32_t a = p.a, b = (int32_t)p.b;
#pragma unroll
                for (int k = 0; k < V; k++) {
                    int32_t r = (int32_t)kv[k] % a;
                    r += r < 0 ? a : 0;
                    m |= (unsigned)(r == b) << k;
                }
            } else {
#pragma unroll
                for (int k = 0; k < V; k++) {
                    int64_t r = (int64_t)kv[k] % (int64_t)p.a;
                    r += r < 0 ? (int64_t)p.a : 0;
                    m |= (unsigned)(r == p.b) << k;
                }
            }
            return m & valid;
        default:
#pragma unroll
            for (int k = 0; k < V; k++) m |= (unsigned)(p0 + k < n && __ldg(p.flags + p0 + k) != 0) << k;
            return m;
    }
}

// The predicate over a thread's NS consecutive vector slots of V keys from e0 (bit
// u * V + c = element e0 + u * V + c; positions at or past n are 0), with one
// dispatch on the kind and one bounds mask for the whole run (NS * V <= 32).
template <typename KT, int NS, int V>
__device__ __forceinline__ unsigned pred_mask_run(const DPred &p, const KT (&kv)[NS][V], int64_t e0, int64_t n) {
    constexpr int PER = NS * V;
    static_assert(PER <= 32, "one 32-bit mask");
    constexpr unsigned ALL = PER == 32 ? ~0u : (1u << PER) - 1u;
    const unsigned valid = e0 + PER <= n ? ALL : (e0 >= n ? 0u : (1u << (unsigned)(n - e0)) - 1u);
    unsigned m = 0;
    switch (p.kind) {
        case IXP_P_TRUE: return valid;
        case IXP_P_LT:
            if (sizeof(KT) == 4) {
                if (p.b > (long long)INT32_MAX) return valid;
                if (p.b <= (long long)INT32_MIN) return 0u;
                const int32_t b = (int32_t)p.b;
#pragma unroll
                for (int u = 0; u < NS; u++)
#pragma unroll
                    for (int c = 0; c < V; c++) m |= (unsigned)((int32_t)kv[u][c] < b) << (u * V + c);
            } else {
#pragma unroll
                for (int u = 0; u < NS; u++)
#pragma unroll
                    for (int c = 0; c < V; c++) m |= (unsigned)((int64_t)kv[u][c] < p.b) << (u * V + c);
            }
            return m & valid;
        case IXP_P_MOD_EQ:
            if (p.b < 0 || p.b >= (long long)p.a) return 0u;
#pragma unroll
            for (int u = 0; u < NS; u++)
#pragma unroll
                for (int c = 0; c < V; c++) {
                    if (sizeof(KT) == 4) {
                        int32_t r = (int32_t)kv[u][c] % p.a;
                        r += r < 0 ? p.a : 0;
                        m |= (unsigned)(r == (int32_t)p.b) << (u * V + c);
                    } else {
                        int64_t r = (int64_t)kv[u][c] % (int64_t)p.a;
                        r += r < 0 ? (int64_t)p.a : 0;
                        m |= (unsigned)(r == p.b) << (u * V + c);
                    }
                }
            return m & valid;
        default:
#pragma unroll
            for (int e = 0; e < PER; e++) m |= (unsigned)(((valid >> e) & 1u) && __ldg(p.flags + e0 + e) != 0) << e;
            return m;
    }
}

// Loads V consecutive elements of type T at p0 (vector loads when aligned and
// in range, guarded scalar loads otherwise; missing elements read as 0).
template <typename T, int V>
__device__ __forceinline__ void load_vec(const T *p, int64_t p0, int64_t n, int vec_ok, T (&o)[V]) {
    constexpr int BYTES = (int)sizeof(T) * V;
    if (vec_ok && p0 + V <= n) {
        if (BYTES == 16 && sizeof(T) == 4) {
            int4 v = __ldcs(reinterpret_cast<const int4 *>(p + p0));
            o[0] = (T)v.x;
            o[1 % V] = (T)v.y;
            o[2 % V] = (T)v.z;
            o[3 % V] = (T)v.w;
            return;
        }
        if (BYTES == 16 && sizeof(T) == 8) {
            longlong2 v = __ldcs(reinterpret_cast<const longlong2 *>(p + p0));
            o[0] = (T)v.x;
            o[1 % V] = (T)v.y;
            return;
        }
        if (BYTES == 32) {
            longlong2 a = __ldcs(reinterpret_cast<const longlong2 *>(p + p0));
            longlong2 b = __ldcs(reinterpret_cast<const longlong2 *>(p + p0) + 1);
            o[0] = (T)a.x;
            o[1 % V] = (T)a.y;
            o[2 % V] = (T)b.x;
            o[3 % V] = (T)b.y;
            return;
        }
        if (BYTES == 8) {
            int2 v = __ldcs(reinterpret_cast<const int2 *>(p + p0));
            o[0] = (T)v.x;
            o[1 % V] = (T)v.y;
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < V; k++) o[k] = (p0 + k < n) ? p[p0 + k] : (T)0;
}

// Keys of one vector slot in their own type (keys may be NULL: zeros).
template <typename KT, int V>
__device__ __forceinline__ void load_slot(const KT *keys, int64_t p0, int64_t n, int vec_ok, KT (&kv)[V]) {
    if (keys) {
        load_vec<KT, V>(keys, p0, n, vec_ok, kv);
    } else {
#pragma unroll
        for (int k = 0; k < V; k++) kv[k] = (KT)0;
    }
}


inline DPred dpred(const ixp_pred &p) { return DPred{p.kind, p.a, (long long)p.b, p.flags}; }


inline bool pred_ok(const ixp_pred &p, bool have_keys) {
    switch (p.kind) {
        case IXP_P_TRUE: return true;
        case IXP_P_MOD_EQ: return have_keys && p.a > 0;
        case IXP_P_LT: return have_keys;
        case IXP_P_FLAGS: return p.flags != nullptr;
        default: return false;
    }
}

}  // namespace ixp
