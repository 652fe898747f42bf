/*
 * ixp.h - C ABI of the GB300 (sm_103a) library for the index-array properties and
 * the scan/scatter combinators of "Verifying Properties of Index Arrays in a
 * Purely-Functional Data-Parallel Language" (arXiv 2506.23058).
 *
 * The paper proves these properties at compile time; this library decides them at
 * run time on concrete int32/int64 arrays in GPU memory, and provides the data-
 * parallel programs that build and use such arrays (scan, scatter, gather, stable
 * partition, flag arrays from shape arrays).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named d_* or described as "device" are CUDA device pointers. All
 *    arrays are contiguous, naturally aligned for their element type, and owned by
 *    the caller. The library never allocates device memory; scratch space comes
 *    from a caller-supplied workspace of at least ixp_workspace_size(...) bytes,
 *    256-byte aligned, which the call may overwrite.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream). Results (verdicts, totals, status words) are written to
 *    device memory, so the calls can be captured in CUDA graphs. Inputs must not be
 *    modified, and outputs/workspace not read, until the stream reaches that point.
 *  - The return value reports host-side validation and launch errors only. A
 *    property that does not hold is not an error: the call returns IXP_OK and the
 *    verdict says ok = 0. Device-side failures (a bitmap span above capacity, a
 *    bounded wait that gave up, an out-of-bounds gather index) are reported in the
 *    verdict's or call's device status word.
 *  - Index types: IXP_I32 (int32_t) or IXP_I64 (int64_t). n is an element count.
 *  - Segments (the paper's segmented shape (e^m, k, e_k), Sec. 2.3): `offsets` is a
 *    device int64_t[nseg + 1] with offsets[0] = 0, offsets[nseg] = n and
 *    offsets nondecreasing; empty segments are allowed. {NULL, 0} means one flat
 *    segment [0, n). Invalid offsets give unspecified results but every memory
 *    access stays inside [0, n).
 */
#ifndef IXP_H
#define IXP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ixp_stream; /* identical to cudaStream_t */

/* ---- return / status codes ------------------------------------------------ */
#define IXP_OK 0
#define IXP_E_INVAL (-1)     /* bad argument: null pointer, n < 0, lo > hi, Img outside Rcd, ... */
#define IXP_E_DTYPE (-2)     /* unsupported element type */
#define IXP_E_SPAN (-3)      /* value span larger than the workspace bitmap (device status) */
#define IXP_E_WORKSPACE (-4) /* workspace missing, misaligned or too small */
#define IXP_E_CUDA (-5)      /* a CUDA launch or memset failed */
#define IXP_E_TIMEOUT (-6)   /* a bounded device wait gave up (device status) */
#define IXP_E_OOB (-7)       /* gather index outside the source (device status) */

typedef enum { IXP_I32 = 0, IXP_I64 = 1 } ixp_itype;

/* Monotonic^op (Sec. 2.3, Fig. 5): op in {<=, <, >=, >}. */
typedef enum { IXP_LE = 0, IXP_LT = 1, IXP_GE = 2, IXP_GT = 3 } ixp_cmp;

/* Verdict kinds. */
enum {
    IXP_V_NONE = 0,
    IXP_V_OUT_OF_RANGE = 1, /* Range: index = first i with X[i] outside [lo, hi] */
    IXP_V_ORDER = 2,        /* Mono: index = later index j of the first failing pair */
    IXP_V_DUPLICATE = 3,    /* Inj/Bij: index = smallest i whose value repeats */
    IXP_V_OUT_OF_IMAGE = 4, /* Bij: index = first i with X[i] in Rcd but outside Img */
    IXP_V_MISSING = 5,      /* Bij: value = smallest image value no element takes */
    IXP_V_WRONG_DEST = 6    /* FiltPart: index = first i with a wrong destination */
};

/* Verdict of a property check, written to device memory (48 bytes).
 * ok = 1 holds, 0 violated, -1 undecided (status != IXP_OK). The meaning of
 * index/value/aux0/aux1 is given at each check. */
typedef struct {
    int32_t ok;
    int32_t kind;
    int64_t index;
    int64_t value;
    int64_t aux0;
    int64_t aux1;
    int32_t status;
    int32_t reserved;
} ixp_verdict;

/* Element predicate, the p of partition2 (Fig. 2) and the p^f / p^p of FiltPart
 * (Fig. 5), evaluated on keys[i] (or flags[i]):
 *   IXP_P_TRUE    always true (the "\_ -> true" of the paper)
 *   IXP_P_MOD_EQ  floored (keys[i] mod a) == b, a > 0
 *   IXP_P_LT      keys[i] < b (signed)
 *   IXP_P_FLAGS   flags[i] != 0, flags a device uint8_t[n] */
enum { IXP_P_TRUE = 0, IXP_P_MOD_EQ = 1, IXP_P_LT = 2, IXP_P_FLAGS = 3 };
typedef struct {
    int32_t kind;
    int32_t a;
    int64_t b;
    const uint8_t *flags;
} ixp_pred;

typedef struct {
    const int64_t *offsets; /* device int64_t[nseg + 1] or NULL */
    int64_t nseg;
} ixp_segs;

/* ---- workspace ------------------------------------------------------------- */
enum {
    IXP_OP_RANGE = 0,
    IXP_OP_MONO = 1,
    IXP_OP_INJ = 2,      /* extra = largest value span to support (bitmap bits); < 0: any span */
    IXP_OP_BIJ = 3,      /* extra = |Img| (bitmap bits) */
    IXP_OP_FILTPART = 4, /* extra = nseg */
    IXP_OP_SCAN = 5,     /* extra = nseg */
    IXP_OP_PARTITION = 6,/* extra = nseg */
    IXP_OP_FLAGS = 7,    /* n = m (number of segments) */
    IXP_OP_INJ_SEG = 8,  /* extra = nseg */
    IXP_OP_BIJ_SEG = 9,  /* extra = nseg */
    IXP_OP_GATHER_SEGMENTS = 10, /* n = output elements */
    IXP_OP_FILTPART_CLASSES = 11, /* itype = v (classes), extra = nseg (0 when flat) */
    IXP_OP_INJ_HIST = 12,         /* extra = m (bins) */
    IXP_OP_SMALLEST_PAIRS = 13,   /* extra = n_verts */
    IXP_OP_FILTPART_VALUES = 14   /* itype = v with a class array, 0 with a predicate; extra = nseg */
};

/* Bytes of workspace that call `op` needs for n elements of type itype and the
 * op-specific `extra` above. Returns 0 for an unknown op. */
size_t ixp_workspace_size(int op, int itype, int64_t n, int64_t extra);

/* Human-readable name of a return/status code. */
const char *ixp_strerror(int code);

/* Library version as major*10000 + minor*100 + patch. */
int ixp_version(void);

/* Number of this library's kernels that have run on the current device since the
 * library was loaded (each kernel counts itself once, from its first block). Reads
 * device memory: call it after synchronizing. 0 when no device is present. */
unsigned long long ixp_kernel_launches(void);

/* ---- property checks ------------------------------------------------------- */

/* Range X (lb, ub)  [Sec. 2.3, Fig. 5]: for all 0 <= i < n, lo <= X[i] <= hi.
 * Closed bounds; INT64_MIN / INT64_MAX stand for -inf / +inf. lo > hi is
 * IXP_E_INVAL. Verdict: index = first i outside the bounds, value = X[i],
 * aux0 = min X, aux1 = max X (INT64_MAX / INT64_MIN when n = 0). */
int ixp_check_range(const void *x, int itype, int64_t n, int64_t lo, int64_t hi, ixp_verdict *d_verdict,
                    void *ws, size_t ws_bytes, ixp_stream stream);

/* Monotonic^op X  [Sec. 2.3, Fig. 5]: for all i < j (inside one segment when
 * segmented), X[i] op X[j]; tested on adjacent pairs, which is equivalent for a
 * transitive op. Verdict: index = j of the first failing pair (X[j-1], X[j]),
 * value = X[j], aux0 = X[j-1]. d_seg_ok (nullable, device uint8_t[nseg]) gets 1/0
 * per segment. */
int ixp_check_mono(const void *x, int itype, int64_t n, int cmp, ixp_segs segs, ixp_verdict *d_verdict,
                   uint8_t *d_seg_ok, void *ws, size_t ws_bytes, ixp_stream stream);

/* Inj X Rcd  [Sec. 2.3, Fig. 5]: no two positions whose values lie in
 * Rcd = [rcd_lo, rcd_hi] hold the same value. Decided with a bitmap over the value
 * span: [rcd_lo, rcd_hi] when that is finite and fits, else [min, max] of the
 * in-Rcd values (one extra pass). A span wider than the workspace bitmaps is
 * decided with a hash set of the in-Rcd values instead when the workspace holds
 * one (ixp_workspace_size(IXP_OP_INJ, itype, n, extra < 0): any span, n < 2^32 - 1);
 * without it such a span gives verdict status IXP_E_SPAN. Verdict on a violation:
 * index = smallest i whose value occurs again, value = X[i], aux0 = smallest j > i
 * with X[j] = X[i] (0 when the property holds). */
int ixp_check_inj(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, ixp_verdict *d_verdict,
                  void *ws, size_t ws_bytes, ixp_stream stream);

/* Bij X Rcd Img  [Sec. 2.3, Fig. 5; rule BijF1, Sec. 3.2]: Inj X Rcd and the set
 * of in-Rcd values equals Img = [img_lo, img_hi], which must lie inside Rcd.
 * Verdict: the smaller of (first i with X[i] in Rcd outside Img -> OUT_OF_IMAGE)
 * and (smallest i with X[i] in Img repeated -> DUPLICATE); otherwise, if some
 * image value is not taken, MISSING with value = the smallest such value and
 * index = -1. aux0 = number of elements with values in Img, aux1 = |Img|
 * (reported whether or not the property holds). */
int ixp_check_bij(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, int64_t img_lo,
                  int64_t img_hi, ixp_verdict *d_verdict, void *ws, size_t ws_bytes, ixp_stream stream);

/* Inj of every segment  [Sec. 2.3, Fig. 5, read per segment]: within each segment
 * [e_k, e_{k+1}), no two positions whose values lie in Rcd = [rcd_lo, rcd_hi] hold
 * the same value; equal values in different segments are allowed. segs is
 * required (nseg >= 1, nseg < 2^32). A segment that increases strictly holds at
 * once (strict monotonicity implies injectivity); any other segment is checked
 * exactly. Limit: a segment that does not increase strictly and whose in-Rcd values
 * span more than 2^24 gives verdict status IXP_E_SPAN. Verdict: the first failing
 * segment decides; index = smallest i in it whose value repeats in the segment,
 * value = X[i], aux0 = the next j in the segment with X[j] = X[i]. d_seg_ok
 * (nullable, device uint8_t[nseg]) gets 1/0 per segment. */
int ixp_check_inj_seg(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, ixp_segs segs,
                      ixp_verdict *d_verdict, uint8_t *d_seg_ok, void *ws, size_t ws_bytes, ixp_stream stream);

/* Bij X Rcd (e^m, k, e_k, Img_k) with Img_k = [e_k, e_{k+1})  [Sec. 2.3, Fig. 5]:
 * every segment's in-Rcd values are exactly its own index range (a per-segment
 * permutation, what a segmented partition produces). Rcd must contain [0, n).
 * Verdict: the first failing segment decides: the smaller of its first
 * OUT_OF_IMAGE and first DUPLICATE position, else MISSING with value = its
 * smallest untaken image value (index -1); aux0 = that segment's in-image count,
 * aux1 = its length (summed over all segments when the property holds).
 * Segments longer than 2^24 give verdict status IXP_E_SPAN. */
int ixp_check_bij_seg(const void *x, int itype, int64_t n, int64_t rcd_lo, int64_t rcd_hi, ixp_segs segs,
                      ixp_verdict *d_verdict, uint8_t *d_seg_ok, void *ws, size_t ws_bytes, ixp_stream stream);

/* InvFiltPart Z (p^f, p^p)  [Sec. 2.3, Fig. 5 and the InvFiltPart prose]: Z is the
 * scatter-index array that turns X into its filter-partition, i.e. for each
 * segment k, the elements kept by `filt` go, stably, trues of `part` first, to
 * consecutive positions after all kept elements of segments < k, and every
 * dropped element's Z lies outside [0, N) (N = number of kept elements), so
 * scatter ignores it. Verdict: index = first i with a wrong destination,
 * value = Z[i], aux0 = N, aux1 = the expected destination (-1 if dropped).
 * keys may be NULL when both predicates are TRUE or FLAGS. */
int ixp_check_filtpart(const void *z, int ztype, int64_t n, const void *keys, int ktype, ixp_pred filt,
                       ixp_pred part, ixp_segs segs, ixp_verdict *d_verdict, void *ws, size_t ws_bytes,
                       ixp_stream stream);

/* InvFiltPart with v classes  [Sec. 2.3, FiltPart Y X (e_k, p^f, p^p_1..v)]: like
 * ixp_check_filtpart, but the kept elements of each segment are placed stably by
 * class, class 0 first: element i has class min(cls[i], v - 1) (the last class
 * takes what the first v - 1 class predicates leave). cls: device uint8_t[n];
 * 1 <= v <= 256; n < 2^32. Verdict as ixp_check_filtpart: index = first i with
 * a wrong destination, value = Z[i], aux0 = N (kept elements), aux1 = the expected
 * destination (-1 if dropped). Workspace: ixp_workspace_size(
 * IXP_OP_FILTPART_CLASSES, v, n, nseg) bytes, 256-byte aligned. */
int ixp_check_filtpart_classes(const void *z, int ztype, int64_t n, const void *keys, int ktype, ixp_pred filt,
                               const uint8_t *cls, int32_t v, ixp_segs segs, ixp_verdict *d_verdict, void *ws,
                               size_t ws_bytes, ixp_stream stream);

/* FiltPart, value form  [Sec. 2.3, FiltPart Y X (e_k, p^f, p^p_1..v)]: Y (ny rows of
 * row_bytes bytes, device) equals X (n rows, device) filtered by `filt` and
 * partitioned stably per segment, bitwise, and has length N (the number of kept
 * rows). The order is that of ixp_check_filtpart (cls == NULL, v = 2: trues of
 * `part` first) or of ixp_check_filtpart_classes (cls: uint8_t[n], 1 <= v <= 256,
 * class min(cls[i], v - 1)). Verdict: ok when Y matches; otherwise kind
 * IXP_V_WRONG_DEST with index = the first position of Y that differs and value =
 * the index in X of the row that belongs there, or, when ny != N, index = -1 and
 * value = ny; aux0 = N. row_bytes: a positive multiple of 4; X and Y 4-byte
 * aligned; n < 2^32. keys may be NULL when the predicates are TRUE or FLAGS; with
 * n = 0 every array may be NULL, and v != 2 then selects the class form.
 * Workspace: ixp_workspace_size(IXP_OP_FILTPART_VALUES, cls ? v : 0, n, nseg)
 * bytes, 256-byte aligned. */
int ixp_check_filtpart_values(const void *y, int64_t ny, const void *x, int64_t n, int32_t row_bytes,
                              const void *keys, int ktype, ixp_pred filt, ixp_pred part, const uint8_t *cls,
                              int32_t v, ixp_segs segs, ixp_verdict *d_verdict, void *ws, size_t ws_bytes,
                              ixp_stream stream);

/* FiltPart with v classes, index form  [Sec. 2.3; the partition3 / filter programs
 * of the evaluation]: out_idx[i] = the destination of element i in the filtered,
 * class-partitioned order (per segment, kept elements by class min(cls[i], v - 1),
 * stably, after all kept elements of the segments before), or -1 for an element
 * the filter drops; *d_kept (nullable) = N, the number of kept elements. Scattering
 * X by out_idx (ignoring -1) builds FiltPart's Y; ixp_check_filtpart_classes
 * accepts out_idx. Same arguments, limits and workspace as
 * ixp_check_filtpart_classes; out_type IXP_I32 needs n <= INT32_MAX. */
int ixp_filtpart_classes(const void *keys, int ktype, int64_t n, ixp_pred filt, const uint8_t *cls, int32_t v,
                         ixp_segs segs, void *out_idx, int out_type, int64_t *d_kept, void *ws, size_t ws_bytes,
                         ixp_stream stream);

/* ---- combinators ----------------------------------------------------------- */

/* scan (+) 0  [Sec. 2.1]: out[i] = sum_{j<i} in[j] (exclusive) or sum_{j<=i} in[j]
 * (inclusive), restarting at each segment start. Sums wrap in the output type
 * (two's complement). Types: i32->i32, i32->i64, i64->i64. d_totals (nullable,
 * device, output type) gets the sum of each segment (one entry when flat).
 * d_status (nullable, device int32) gets IXP_OK or IXP_E_TIMEOUT. */
int ixp_scan(const void *in, int in_type, void *out, int out_type, int64_t n, int inclusive, ixp_segs segs,
             void *d_totals, int32_t *d_status, void *ws, size_t ws_bytes, ixp_stream stream);

/* Stable two-way partition, partition2 of Fig. 2 (flat) and partition2L of Sec. 6
 * (segmented): out_indices[i] = the scatter destination of element i, which is
 * e_k + (number of trues before i in its segment) when pred(i) holds and
 * e_k + T_k + (number of falses before i in its segment) otherwise, T_k being the
 * segment's number of trues. d_num_true (device int64_t[max(1, nseg)]) gets T_k.
 * out_indices (nullable: then the destinations are only used to place the keys
 * and payload), out_keys / out_payload (nullable) receive keys / payload rows
 * scattered to their destinations (payload rows are row_bytes bytes, a multiple
 * of 4, at most 64).
 * keys may be NULL for a FLAGS or TRUE predicate. d_status as for ixp_scan. */
int ixp_partition(const void *keys, int ktype, int64_t n, ixp_pred pred, const void *payload, int32_t row_bytes,
                  void *out_indices, int out_type, void *out_keys, void *out_payload, int64_t *d_num_true,
                  ixp_segs segs, int32_t *d_status, void *ws, size_t ws_bytes, ixp_stream stream);

/* scatter dst is vs  [Sec. 2.1]: for each i, if 0 <= idx[i] < dst_len then row
 * dst[idx[i]] := vals[i] (mode IXP_SCATTER_ASSIGN) or += vals[i] (IXP_SCATTER_ADD,
 * float32 rows accumulated with float32 atomics, or float64 rows with float64
 * atomics). Out-of-bounds indices are ignored. ASSIGN is deterministic only when
 * the in-bounds indices are injective (check with ixp_check_inj). Rows are
 * row_elems elements of elem_bytes (4 or 8) bytes. */
enum { IXP_SCATTER_ASSIGN = 0, IXP_SCATTER_ADD = 1 };
int ixp_scatter(void *dst, int64_t dst_len, const void *idx, int itype, const void *vals, int64_t n,
                int32_t row_elems, int32_t elem_bytes, int32_t mode, ixp_stream stream);

/* Additive scatter of float32 rows accumulated in float64: acc[idx[i]] += vals[i]
 * for in-bounds idx[i], acc a device double[dst_len * row_elems] the caller zeroes
 * (or pre-loads). Rows of up to 8 values go through each block's shared-memory
 * cache of target rows held as exact 64-bit fixed-point values (native integer
 * atomics, one float64 rounding per cached row when the block ends); rows that
 * miss the cache, and values the fixed-point scale cannot hold exactly, are added
 * with float64 atomics, the lanes of a row covering its columns. Every addition
 * into acc rounds once in float64 (a cached partial sum is exact before its
 * rounding); the order of the additions is not fixed, so the low bits can differ
 * from run to run. */
int ixp_scatter_add_f32_to_f64(double *acc, int64_t dst_len, const void *idx, int itype, const float *vals,
                               int64_t n, int32_t row_elems, ixp_stream stream);

/* Rounds a float64 accumulator to float32 (out[i] = (float)acc[i], count elements). */
int ixp_f64_to_f32(float *out, const double *acc, int64_t count, ixp_stream stream);

/* Inverse of an index array, the is^-1 that rule Sc1 (Sec. 4, scatter conversion)
 * couples to a bijective scatter index: inv[idx[i]] = i for every in-bounds
 * idx[i] in [0, inv_len), and inv[j] = -1 for targets no index hits. idx must be
 * injective on its in-bounds entries (check with ixp_check_inj); otherwise which
 * i lands in inv[j] is unspecified. With inv, the adjoint of a gather by idx is the
 * gather by inv (out-of-range -1 rows read as zero), with no atomics. */
int ixp_invert(const void *idx, int itype, int64_t n, void *inv, int inv_type, int64_t inv_len, ixp_stream stream);

/* Widens float32 to float64 (out[i] = (double)in[i]); used to pre-load a float64
 * accumulator with a float32 destination before an additive scatter. */
int ixp_f32_to_f64(double *out, const float *in, int64_t count, ixp_stream stream);

/* gather: out[i] = src[idx[i]] (rows of row_elems * elem_bytes bytes). An index
 * outside [0, src_len) zero-fills its row and sets *d_status = IXP_E_OOB
 * (d_status nullable; it is not cleared, so zero it first). */
int ixp_gather(void *out, const void *src, int64_t src_len, const void *idx, int itype, int64_t n,
               int32_t row_elems, int32_t elem_bytes, int32_t *d_status, ixp_stream stream);

/* Gather of whole segments [Sec. 2.1 gather over the flattened layout of Fig. 2]:
 * output segment k (elements out_off[k] .. out_off[k+1] - 1) becomes a copy of
 * source segment seg_src[k] (src_off[s] .. src_off[s+1] - 1), i.e. the gather
 * out[j] = src[src_off[seg_src[II[j]]] + j - out_off[II[j]]] with II the mkII
 * segment ids of the output shape, without building II or the index array. Used
 * to move CSR rows (column indices, values) into a new row order; with the
 * inverse segment map it is its own adjoint. out_off: device int64[m + 1],
 * out_off[0] = 0, out_off[m] = n_out, nondecreasing; src_off: device
 * int64[src_m + 1] with src_off[src_m] = src_len; seg_src: device int32/int64[m]
 * in [0, src_m); elements of 4 or 8 bytes; out has n_out, src src_len elements.
 * Offsets or a map that do not describe equal-length segments set
 * *d_status = IXP_E_INVAL (results unspecified, every access stays in bounds;
 * d_status nullable and not cleared). Workspace: ixp_workspace_size(
 * IXP_OP_GATHER_SEGMENTS, 0, n_out, 0) bytes, 256-byte aligned. */
int ixp_gather_segments(void *out, int64_t n_out, const int64_t *out_off, int64_t m, const void *src,
                        int64_t src_len, const int64_t *src_off, int64_t src_m, const void *seg_src, int seg_type,
                        int32_t elem_bytes, int32_t *d_status, void *ws, size_t ws_bytes, ixp_stream stream);

/* mkSgmDescr shape xs  [Sec. 2.1, Fig. 2 right]: out (length sum(shape)) is zero
 * except out[e_k] = xs[k] (1 when xs is NULL) for every non-empty segment k, with
 * e_k the exclusive scan of shape; empty segments write nothing. shape is a device
 * int64_t[m] of non-negative sizes (Range shape (0, inf)); a negative size sets
 * *d_status = IXP_E_INVAL. d_offsets (nullable, device int64_t[m + 1]) gets e_0..e_m.
 * out_len must equal sum(shape), which the caller knows or reads from d_offsets of a
 * first call with out = NULL and out_len = 0 (then only the offsets are written). */
int ixp_flags_from_shape(const int64_t *shape, int64_t m, const int64_t *xs, void *out, int out_type,
                         int64_t out_len, int64_t *d_offsets, int32_t *d_status, void *ws, size_t ws_bytes,
                         ixp_stream stream);

/* sgmSum  [Fig. 2 with Sec. 2.1 scan]: scan with the segmented operator
 * (f1, v1) + (f2, v2) = (f1 or f2, f2 ? v2 : v1 + v2) over (flags[i] != 0, in[i]):
 * a segment starts at 0 and at every i with flags[i] != 0; the inclusive form is
 * out[i] = sum of in over [last start <= i, i], the exclusive form the same
 * without in[i]. Types and wrap-around as ixp_scan; flags: device uint8_t[n].
 * Workspace as ixp_scan (IXP_OP_SCAN, nseg = 0). */
int ixp_sgm_scan(const uint8_t *flags, const void *in, int in_type, void *out, int out_type, int64_t n, int inclusive,
                 int32_t *d_status, void *ws, size_t ws_bytes, ixp_stream stream);

/* mkII  [Fig. 2 right, with the prose reading: II[j] = k for e_k <= j < e_{k+1}]:
 * out (n = offsets[m] elements, int32 or int64) gets the segment index of every
 * position. offsets: device int64[m + 1], offsets[0] = 0, offsets[m] = n,
 * nondecreasing (empty segments allowed), e.g. the d_offsets of
 * ixp_flags_from_shape. Offsets that do not end at n set *d_status = IXP_E_INVAL
 * (d_status nullable, not cleared). Workspace: ixp_workspace_size(
 * IXP_OP_GATHER_SEGMENTS, 0, n, 0) bytes. */
int ixp_mkii(const int64_t *offsets, int64_t m, void *out, int out_type, int64_t n, int32_t *d_status, void *ws,
             size_t ws_bytes, ixp_stream stream);

/* ---- reduce-by-index and maxMatching ------------------------------------------- */

/* Reduce-by-index with min, Futhark's hist with the min operator  [Sec. 6: the
 * hist of get_smallest_pairs, Fig. 16, and of the dynamic verification of
 * scatter]: for every i with 0 <= idx[i] < m, H[idx[i]] = min(H[idx[i]],
 * vals[i]); indices out of bounds are ignored, as scatter ignores them (Sec. 2.1).
 * H: device htype[m] holding the neutral element on entry (the caller fills it).
 * vals: device htype[n], or NULL for vals[i] = i (n - 1 must then fit htype).
 * idx: device itype[n]. Signed comparison. The result does not depend on the
 * order of the updates. No workspace. */
int ixp_hist_min(void *H, int htype, int64_t m, const void *idx, int itype, const void *vals, int64_t n,
                 ixp_stream stream);

/* Inj on [0, m) decided the way a dynamic verification of scatter decides it
 * [Sec. 6: reduce-by-index with atomic min]: H = hist min over [0, m) of
 * iota n by x, then every i with 0 <= x[i] < m must have H[x[i]] == i. Same
 * property and verdict as ixp_check_inj(x, itype, n, 0, m - 1, ...): index = the
 * first occurrence of the earliest repeated value, value = x[index], aux0 = its
 * next occurrence. n < 2^32. Workspace: ixp_workspace_size(IXP_OP_INJ_HIST,
 * itype, n, m) bytes (4 m + 256), 256-byte aligned. */
int ixp_check_inj_hist(const void *x, int itype, int64_t n, int64_t m, ixp_verdict *d_verdict, void *ws,
                       size_t ws_bytes, ixp_stream stream);

/* get_smallest_pairs of maxMatching  [Sec. 6, Fig. 16]: H = hist min over n_verts
 * bins, neutral element n_es, of the priorities is by the vertices es; slot i is
 * kept when 0 <= es[i] < n_verts and H[es[i]] == is[i]; out_es / out_is get the
 * kept es[i] / is[i] in input order (filter_by) and *d_count their number. When
 * is is injective both outputs are injective, the property the paper proves.
 * es, is, out_es, out_is: device arrays of one itype (out_* need room for the kept
 * count, at most n); d_count: device int64. Workspace: ixp_workspace_size(
 * IXP_OP_SMALLEST_PAIRS, itype, n, n_verts) bytes, 256-byte aligned. */
int ixp_smallest_pairs(const void *es, const void *is, int itype, int64_t n, int64_t n_verts, int64_t n_es,
                       void *out_es, void *out_is, int64_t *d_count, void *ws, size_t ws_bytes, ixp_stream stream);

/* ---- hardware-rate microbenchmarks ------------------------------------------------ */

/* The rates that bound the kernels above, measured with minimal kernels so that a
 * kernel's time can be read against the rate it needs (the paper has no
 * counterpart; these serve the roofline report). Each writes one checksum word per
 * block or warp into d_sink (device uint32_t[ixp_sink_words()]) so that nothing is
 * optimised away; the checksums carry no meaning. */
int ixp_sink_words(void);

/* L2 atomic OR: for each i, bit pos[i] & (bits - 1) of the device bitmap (bits a
 * power of two, bits / 32 words) is set with atomicOr; with_return != 0 folds the
 * returned old word (what a bitmap duplicate test needs), 0 leaves it unused (a
 * fire-and-forget reduction). pos: device uint32_t[n], 16-byte aligned, n a
 * multiple of 4. */
int ixp_ceiling_atomic_or(unsigned *bitmap, int64_t bits, const unsigned *pos, int64_t n, int with_return,
                          unsigned *d_sink, ixp_stream stream);

/* Random 32-byte rows: item i reads row idx[i] & (nrows - 1) of rows (device,
 * 16-byte aligned, nrows a power of two up to 2^32, 32 bytes per row). idx: device
 * uint32_t[n], 16-byte aligned, n a multiple of 4. */
int ixp_ceiling_random_rows(const void *rows, int64_t nrows, const unsigned *idx, int64_t n, unsigned *d_sink,
                            ixp_stream stream);

/* Streaming read of bytes (a multiple of 16) from src (16-byte aligned). */
int ixp_ceiling_stream_read(const void *src, int64_t bytes, unsigned *d_sink, ixp_stream stream);

/* ---- batched pipeline over a jagged array ---------------------------------------- */

/* Launch shape of ixp_batch_run (the autotuner's search space): threads per CTA
 * (256 or 512), resident CTAs per SM (1..8), log2 of the shared bitmap in bits
 * (10..20) and elements per thread per sweep step (4 or 8). */
typedef struct {
    int32_t threads;
    int32_t ctas_per_sm;
    int32_t smem_bits_log2;
    int32_t chunk;
} ixp_batch_tuning;

/* Bytes of workspace ixp_batch_run needs for a tuning (NULL = defaults). */
size_t ixp_batch_workspace_size(const ixp_batch_tuning *tuning);

/* One persistent launch over the m segments of a jagged array of n = sum(shape)
 * int32 elements [Sec. 2.1 mkSgmDescr; Sec. 6 partition2L; Sec. 2.3 Fig. 5 checks].
 * For every segment k (e_k = shape[0] + ... + shape[k-1]):
 *   flags[e_k..e_{k+1})   = 1 at e_k, 0 elsewhere (mkSgmDescr with xs = 1)
 *   indices[e_k..e_{k+1}) = the stable partition destinations of the segment's
 *                           keys under pred (trues first), d_num_true[k] = T_k
 *   d_seg_ok[k]           = Mono< of iota inside the segment
 *   d_seg_ok[m + k]       = Inj of chk inside the segment
 *   d_seg_ok[2m + k]      = Bij of chk inside the segment onto [e_k, e_{k+1})
 * d_offsets (int64[m+1]) gets e_0..e_m; d_first_bad[0..2] the first segment
 * failing Mono / Inj / Bij (-1 if none). order (nullable) is the work list, a
 * permutation of [0, m) (longest segments first balances the launch). pred is
 * TRUE, MOD_EQ or LT. keys, chk, iota, flags and indices must be 16-byte aligned
 * (else IXP_E_INVAL). d_status gets IXP_E_INVAL for a negative size, a bad work
 * list or sum(shape) != n, and IXP_E_SPAN if a segment is longer than 2^21 or its
 * chk values, when some fall outside its image, span more than 2^21 (Inj/Bij then
 * read 0 for that segment). */
int ixp_batch_run(const int64_t *shape, int64_t m, const int32_t *keys, ixp_pred pred, const int32_t *chk,
                  const int32_t *iota, int64_t n, const int32_t *order, int32_t *flags, int32_t *indices,
                  int64_t *d_num_true, int64_t *d_offsets, uint8_t *d_seg_ok, int64_t *d_first_bad,
                  int32_t *d_status, const ixp_batch_tuning *tuning, void *ws, size_t ws_bytes, ixp_stream stream);

/* ---- allocation-free scan -------------------------------------------------------- */

/* ixp_scan for callers that cannot allocate device memory at all: a host runtime
 * whose device memory is fully planned before it starts, a process with a fixed
 * device-memory budget, or code on a path where a cudaMalloc (which can
 * synchronize the device) is not allowed. The paper has no counterpart; this is
 * a library convenience. It computes exactly what ixp_scan computes for a flat
 * array (segs = {NULL, 0}), but takes no workspace: its scratch (a 256-byte header
 * and 16 bytes per tile of 4096 int32 or 2048 int64 inputs) is a fixed array of
 * 262,400 bytes inside this library, which every GPU that loads the library holds
 * until the process exits. n above ixp_scan_noalloc_max_n(in_type) (2^26 for int32
 * input, 2^25 for int64) is rejected with IXP_E_INVAL; so are the argument errors
 * of ixp_scan. The call allocates nothing: it clears the part of the array it
 * uses with cudaMemsetAsync, then launches the scan.
 *  - The first call on each device looks up the array's device address (with that
 *    device current) and remembers it; make that first call before any stream
 *    capture. A failed lookup returns IXP_E_CUDA.
 *  - The array used is the current device's, so `stream` must belong to the
 *    current device (or be a default-stream handle); a stream of another device
 *    is rejected with IXP_E_INVAL.
 *  - Every call on a device shares the one array. Calls whose work overlaps on the
 *    GPU (different streams, or concurrent graph branches) race on it and give
 *    wrong results; order them on one stream or with events. */
int ixp_scan_noalloc(const void *in, int in_type, void *out, int out_type, int64_t n, int inclusive,
                     void *d_totals, int32_t *d_status, ixp_stream stream);

/* Largest n that ixp_scan_noalloc accepts for the given input type. */
int64_t ixp_scan_noalloc_max_n(int in_type);

/* ---- testing hook ------------------------------------------------------------ */

/* Sets the bound on every device-side wait of later calls in this process (number
 * of polls; <= 0 restores the default of 1048576, or the value of the environment
 * variable IXP_DEBUG_SPIN_LIMIT) and names one look-back tile that never
 * publishes its value (-1: none). Tests use it to make a wait run out and check
 * that the call reports IXP_E_TIMEOUT instead of hanging. */
int ixp_debug_set_wait(long long spin_limit, long long skip_tile);

#ifdef __cplusplus
}
#endif

#endif /* IXP_H */
