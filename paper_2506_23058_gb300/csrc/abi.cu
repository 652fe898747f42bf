// abi.cu - workspace sizing, error strings, version, launch-shape helpers.
#include <algorithm>

#include "common.cuh"

namespace ixp {

size_t tiled_ws_bytes(int64_t n, int V, int64_t nseg);  // scan.cu
size_t bk_prefix_bytes(int64_t n);                       // checks.cu
size_t inj_any_span_ws_bytes(int64_t n);                 // checks.cu
size_t seg_ws_bytes(int64_t nseg);                       // segmented.cu
size_t gather_segments_ws_bytes(int64_t n_out);          // scatter.cu
size_t filtpart_classes_ws_bytes(int v, int64_t n, int64_t nseg);  // classes.cu
size_t filtpart_values_ws_bytes(int v, int64_t n, int64_t nseg);   // scan.cu
size_t inj_hist_ws_bytes(int64_t m);                                 // hist.cu
size_t smallest_pairs_ws_bytes(int itype, int64_t n, int64_t n_verts);  // hist.cu

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

// Enough 256-thread blocks for `per_thread` items per thread, capped at one wave
// of 4 resident blocks per SM (the streaming kernels are built for 4 blocks/SM,
// 64 registers per thread), at least one block.
int stream_grid(int64_t work_items, int per_thread) {
    int64_t per_block = (int64_t)STREAM_THREADS * std::max(1, per_thread);
    int64_t blocks = (work_items + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms() * 4;
    return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

}  // namespace ixp

using namespace ixp;


extern "C" size_t ixp_workspace_size(int op, int itype, int64_t n, int64_t extra) {
    if (n < 0) n = 0;
    const int es = itype == IXP_I64 ? 8 : 4;
    switch (op) {
        case IXP_OP_RANGE: return HDR_BYTES;
        case IXP_OP_MONO: return HDR_BYTES + chunk_lb_bytes(n);  // the table serves the segmented form
        case IXP_OP_INJ:
            if (extra < 0) return inj_any_span_ws_bytes(n);  // bitmaps + the hash set for any span
            [[fallthrough]];
        case IXP_OP_BIJ: {
            // large inputs also get the bucket pool (about 5 bytes per element)
            int64_t span = extra > 0 ? extra : n;
            if (span < (1 << 21)) span = 1 << 21;
            size_t words = (size_t)((span + 31) / 32);
            size_t prefix = n >= (1 << 18) ? bk_prefix_bytes(n) : HDR_BYTES;
            return prefix + round256(2 * words * 4 + 256);
        }
        case IXP_OP_SCAN: return tiled_ws_bytes(n, 16 / es, extra);
        case IXP_OP_PARTITION:
        case IXP_OP_FILTPART: return tiled_ws_bytes(n, 16 / es, extra);
        case IXP_OP_FLAGS: return tiled_ws_bytes(n, 2, 0);
        case IXP_OP_INJ_SEG:
        case IXP_OP_BIJ_SEG: return seg_ws_bytes(extra) + chunk_lb_bytes(n);
        case IXP_OP_GATHER_SEGMENTS: return gather_segments_ws_bytes(n);
        case IXP_OP_FILTPART_CLASSES: return filtpart_classes_ws_bytes(itype, n, extra);
        case IXP_OP_INJ_HIST: return inj_hist_ws_bytes(extra);
        case IXP_OP_SMALLEST_PAIRS: return smallest_pairs_ws_bytes(itype, n, extra);
        case IXP_OP_FILTPART_VALUES: return filtpart_values_ws_bytes(itype, n, extra);
        default: return 0;
    }
}

extern "C" const char *ixp_strerror(int code) {
    switch (code) {
        case IXP_OK: return "ok";
        case IXP_E_INVAL: return "invalid argument";
        case IXP_E_DTYPE: return "unsupported element type";
        case IXP_E_SPAN: return "value span exceeds the workspace bitmap";
        case IXP_E_WORKSPACE: return "workspace missing, misaligned or too small";
        case IXP_E_CUDA: return "CUDA launch failed";
        case IXP_E_TIMEOUT: return "bounded device wait gave up";
        case IXP_E_OOB: return "index out of bounds";
        default: return "unknown error";
    }
}

extern "C" int ixp_version(void) { return 100; }

extern "C" unsigned long long ixp_tu_kernels_checks(void);
extern "C" unsigned long long ixp_tu_kernels_scan(void);
extern "C" unsigned long long ixp_tu_kernels_scatter(void);
extern "C" unsigned long long ixp_tu_kernels_segmented(void);
extern "C" unsigned long long ixp_tu_kernels_batched(void);
extern "C" unsigned long long ixp_tu_kernels_classes(void);
extern "C" unsigned long long ixp_tu_kernels_hist(void);
extern "C" unsigned long long ixp_tu_kernels_ceilings(void);

extern "C" unsigned long long ixp_kernel_launches(void) {
    return ixp_tu_kernels_checks() + ixp_tu_kernels_scan() + ixp_tu_kernels_scatter() + ixp_tu_kernels_segmented() +
           ixp_tu_kernels_batched() + ixp_tu_kernels_classes() + ixp_tu_kernels_hist() +
           ixp_tu_kernels_ceilings();
}
