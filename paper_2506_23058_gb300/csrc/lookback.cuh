// lookback.cuh - the decoupled look-back of a single-pass tile scan (Merrill &
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016):
// one 16-byte status word per tile, read and written with single 16-byte
// accesses, and the plain-sum look-back over it. Every wait is bounded by the
// process-wide Wait configuration; a wait that gives up records IXP_E_TIMEOUT.
#pragma once

#include "common.cuh"

namespace ixp {

struct Wait {
    long long spin_limit;  // polls before a wait gives up
    long long skip_tile;   // testing hook: this tile never publishes (-1: none)
};

// Process-wide wait bound (scan.cu): polls before a wait gives up, and the
// testing hook that names a tile that never publishes.
Wait wait_config();

// One 16-byte status word per tile: {value, flag}, written and read with single
// 16-byte accesses so that one load returns a consistent pair. flag: 0 empty,
// 1 aggregate, 2 inclusive prefix; bit 2: the aggregate holds a segment head.
struct Lookback {
    ulonglong2 *st;
};

__device__ __forceinline__ void publish_status(ulonglong2 *p, unsigned long long value, unsigned long long flag) {
    asm volatile("st.global.cg.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(value), "l"(flag) : "memory");
}
__device__ __forceinline__ ulonglong2 read_status(const ulonglong2 *p) {
    ulonglong2 v;
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}

// Look-back window: each lane reads LB_PER_LANE consecutive predecessors, so one
// round trip covers 32 * LB_PER_LANE tiles.
constexpr int LB_PER_LANE = 4;

// Plain-sum form of the look-back (no segment flags): the same protocol with
// addition; the window is reduced with a butterfly since order does not matter.
static __device__ unsigned long long lookback_sum(const Lookback L, int64_t t, unsigned long long agg, Hdr *h, Wait wt) {
    const int lane = threadIdx.x & 31;
    const bool publish = t != wt.skip_tile;
    if (t == 0) {
        if (lane == 0 && publish) publish_status(L.st, agg, 2ull);
        return 0ull;
    }
    if (lane == 0 && publish) publish_status(L.st + t, agg, 1ull);
    unsigned long long excl = 0;
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
            for (int q = 0; q < LB_PER_LANE; q++) pending |= w[q].y == 0ull;
            if (!__any_sync(FULL, pending)) break;
            if (++spins > wt.spin_limit) {
#pragma unroll
                for (int q = 0; q < LB_PER_LANE; q++)
                    if (w[q].y == 0ull) {
                        w[q] = make_ulonglong2(0ull, 2ull);
                        gave_up = true;
                    }
                break;
            }
            if (spins > 16) __nanosleep(32);
#pragma unroll
            for (int q = 0; q < LB_PER_LANE; q++) {
                const int64_t j = top - (int64_t)lane * LB_PER_LANE - q;
                if (w[q].y == 0ull) w[q] = read_status(L.st + j);
            }
        }
        unsigned long long mine = 0;
        bool stop_here = false;
#pragma unroll
        for (int q = 0; q < LB_PER_LANE; q++) {
            if (stop_here) continue;
            mine += w[q].x;
            stop_here = w[q].y == 2ull;
        }
        const unsigned stop = __ballot_sync(FULL, stop_here);
        const int L0 = stop ? __ffs(stop) - 1 : 32;
        if (lane > L0) mine = 0;
        excl += warp_sum_u64(mine);
        if (L0 < 32) break;
        top -= 32 * LB_PER_LANE;
    }
    if (gave_up && lane == 0) set_status(h, IXP_E_TIMEOUT);
    if (lane == 0 && publish) publish_status(L.st + t, excl + agg, 2ull);
    return excl;
}

}  // namespace ixp
