// lookback.cuh - the decoupled look-back of a single-pass tile scan (Merrill &
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016):
// one 16-byte status word per tile (two flagged 64-bit halves, see below), and
// the plain-sum look-back over it. Every wait is bounded by the
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

// One 16-byte status word per tile: a 64-bit value and a flag (0 empty, 1
// aggregate, 2 inclusive prefix; bit 2: the aggregate holds a segment head). The
// value is split into two 32-bit halves and each 64-bit half of the word carries
// the flag in its upper 32 bits. Both halves are written and read as relaxed
// gpu-scope 64-bit accesses (each single-copy atomic); the PTX memory model does
// not make the 16-byte pair atomic as a whole, so a load may combine halves from
// two different writes of the word. Such a mix has two different flags (the word
// goes 0 -> 1 -> 2, each state written once), and read_status reports it as not
// ready, so a flagged value is never assembled from two writes.
struct Lookback {
    ulonglong2 *st;
};

__device__ __forceinline__ void publish_status(ulonglong2 *p, unsigned long long value, unsigned long long flag) {
    const unsigned long long lo = (value & 0xffffffffull) | (flag << 32);
    const unsigned long long hi = (value >> 32) | (flag << 32);
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(lo), "l"(hi) : "memory");
}
// .x = the value, .y = the flag (0 while the two halves disagree)
__device__ __forceinline__ ulonglong2 read_status(const ulonglong2 *p) {
    unsigned long long lo, hi;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(p) : "memory");
    const unsigned long long f = lo >> 32;
    ulonglong2 v;
    v.x = (lo & 0xffffffffull) | (hi << 32);
    v.y = f == (hi >> 32) ? f : 0ull;
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
