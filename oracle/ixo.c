/*
 * ixo.c - CPU oracle for the index-array properties and combinators of
 * "Verifying Properties of Index Arrays in a Purely-Functional Data-Parallel
 * Language" (arXiv 2506.23058).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, single-threaded
 * statement of what the GPU library computes. Only the tests, the smoke entry
 * point and the benchmark's CPU-baseline leg load it. It shares no code, header,
 * table or helper with the CUDA library, and the library never calls it.
 *
 * Every function follows the paper's definition in the paper's order; a library
 * primitive (qsort) is used as a step only where named. Readings taken where the
 * paper is silent or garbled are stated at each function.
 *
 * Integer results are exact. Sums use unsigned 64-bit arithmetic (two's-
 * complement wrap) and are truncated to the output width. Payload sums for the
 * additive scatter are accumulated in double.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IXO_OK 0
#define IXO_E_INVAL (-1)
#define IXO_E_DTYPE (-2)
#define IXO_E_NOMEM (-3)
#define IXO_E_OOB (-7)

enum { K_NONE = 0, K_OUT_OF_RANGE = 1, K_ORDER = 2, K_DUPLICATE = 3,
       K_OUT_OF_IMAGE = 4, K_MISSING = 5, K_WRONG_DEST = 6 };

enum { C_LE = 0, C_LT = 1, C_GE = 2, C_GT = 3 };

enum { P_TRUE = 0, P_MOD_EQ = 1, P_LT = 2, P_FLAGS = 3 };

typedef struct {
    int32_t ok;
    int32_t kind;
    int64_t index;
    int64_t value;
    int64_t aux0;
    int64_t aux1;
} ixo_verdict;

typedef struct {
    int32_t kind;
    int32_t a;
    int64_t b;
    const uint8_t *flags;
} ixo_pred;

/* ------------------------------------------------------------------ helpers */

static int64_t get(const void *x, int t, int64_t i)
{
    return t == 0 ? (int64_t)((const int32_t *)x)[i] : ((const int64_t *)x)[i];
}

static void put(void *x, int t, int64_t i, uint64_t v)
{
    if (t == 0)
        ((int32_t *)x)[i] = (int32_t)(uint32_t)v; /* truncation = wrap */
    else
        ((int64_t *)x)[i] = (int64_t)v;
}

static int bad_type(int t) { return t != 0 && t != 1; }

static void verdict_ok(ixo_verdict *v)
{
    v->ok = 1;
    v->kind = K_NONE;
    v->index = -1;
    v->value = 0;
    v->aux0 = 0;
    v->aux1 = 0;
}

/* Segment bounds: offsets == NULL means one segment [0, n). The paper's segmented
 * shape (Sec. 2.3, Fig. 5 preamble) requires e_0 = 0 and e_k nondecreasing; we also
 * require the last offset to be n. */
static int segs_valid(const int64_t *off, int64_t nseg, int64_t n)
{
    if (!off)
        return 1;
    if (nseg < 0 || off[0] != 0 || off[nseg] != n)
        return 0;
    for (int64_t k = 0; k < nseg; k++)
        if (off[k + 1] < off[k])
            return 0;
    return 1;
}

static int64_t seg_count(const int64_t *off, int64_t nseg) { return off ? nseg : 1; }
static int64_t seg_lo(const int64_t *off, int64_t k) { return off ? off[k] : 0; }
static int64_t seg_hi(const int64_t *off, int64_t k, int64_t n) { return off ? off[k + 1] : n; }

/* Floored remainder (result in [0, a) for a > 0). */
static int64_t floor_mod(int64_t key, int64_t a)
{
    int64_t r = key % a;
    if (r < 0)
        r += a;
    return r;
}

static int pred_eval(const ixo_pred *p, const void *keys, int kt, int64_t i)
{
    switch (p->kind) {
    case P_TRUE: return 1;
    case P_MOD_EQ: return floor_mod(get(keys, kt, i), p->a) == p->b;
    case P_LT: return get(keys, kt, i) < p->b;
    case P_FLAGS: return p->flags[i] != 0;
    }
    return 0;
}

static int pred_valid(const ixo_pred *p, const void *keys, int kt)
{
    if (p->kind == P_TRUE)
        return 1;
    if (p->kind == P_FLAGS)
        return p->flags != NULL;
    if (p->kind == P_MOD_EQ)
        return keys != NULL && !bad_type(kt) && p->a > 0;
    if (p->kind == P_LT)
        return keys != NULL && !bad_type(kt);
    return 0;
}

/* ------------------------------------------------------------------- Range
 * Fig. 5, Range X (lb, ub): for all 0 <= i < n, lb <= X[i] <= ub (closed bounds;
 * INT64_MIN / INT64_MAX stand for -inf / +inf). The verdict names the first i
 * that breaks the bound and its value; aux0/aux1 are min and max of X. */
int ixo_check_range(const void *x, int t, int64_t n, int64_t lo, int64_t hi, ixo_verdict *v)
{
    if (bad_type(t))
        return IXO_E_DTYPE;
    if (n < 0 || lo > hi || (n > 0 && !x) || !v)
        return IXO_E_INVAL;
    verdict_ok(v);
    v->aux0 = INT64_MAX;
    v->aux1 = INT64_MIN;
    for (int64_t i = 0; i < n; i++) {
        int64_t xi = get(x, t, i);
        if (xi < v->aux0)
            v->aux0 = xi;
        if (xi > v->aux1)
            v->aux1 = xi;
        if (v->ok && (xi < lo || xi > hi)) {
            v->ok = 0;
            v->kind = K_OUT_OF_RANGE;
            v->index = i;
            v->value = xi;
        }
    }
    return IXO_OK;
}

/* ------------------------------------------------------------- Monotonic
 * Fig. 5, Monotonic^op X: for all i < j, X[i] op X[j]. Reading: every pair in
 * [0, n) (the figure's "j < n - 1" would exempt the last element). Because op is
 * transitive, this equals the adjacent test X[j-1] op X[j] for 1 <= j < n. In the
 * segmented form only pairs inside one segment [e_k, e_{k+1}) are tested. The
 * verdict names the later index j of the first failing pair; aux0 = X[j-1]. */
static int cmp_holds(int c, int64_t a, int64_t b)
{
    switch (c) {
    case C_LE: return a <= b;
    case C_LT: return a < b;
    case C_GE: return a >= b;
    case C_GT: return a > b;
    }
    return 0;
}

int ixo_check_mono(const void *x, int t, int64_t n, int c, const int64_t *off, int64_t nseg,
                   ixo_verdict *v, uint8_t *seg_ok)
{
    if (bad_type(t))
        return IXO_E_DTYPE;
    if (n < 0 || c < 0 || c > 3 || (n > 0 && !x) || !v || !segs_valid(off, nseg, n))
        return IXO_E_INVAL;
    verdict_ok(v);
    for (int64_t k = 0; k < seg_count(off, nseg); k++) {
        int64_t a = seg_lo(off, k), b = seg_hi(off, k, n);
        int sok = 1;
        for (int64_t j = a + 1; j < b; j++) {
            int64_t p = get(x, t, j - 1), q = get(x, t, j);
            if (!cmp_holds(c, p, q)) {
                if (v->ok) {
                    v->ok = 0;
                    v->kind = K_ORDER;
                    v->index = j;
                    v->value = q;
                    v->aux0 = p;
                }
                sok = 0;
                break;
            }
        }
        if (seg_ok)
            seg_ok[k] = (uint8_t)sok;
    }
    return IXO_OK;
}

/* ---------------------------------------------------- first repeated value
 * Shared by Inj and Bij: among positions i in [a, b) whose value lies in [lo, hi],
 * find the smallest i whose value occurs again at some other position in [a, b)
 * (restricted to [lo, hi]), and the smallest such other position j > i. Reading
 * (the paper is a static verifier and names no witness): a violation of Inj is the
 * lexicographically smallest pair (i, j), i < j, X[i] = X[j].
 * Two plain methods, both exact: a saturating count per value when the value span
 * is small against the segment, otherwise qsort of (value, index) pairs. */
typedef struct { int64_t val, idx; } pair_t;

static int pair_cmp(const void *pa, const void *pb)
{
    const pair_t *a = pa, *b = pb;
    if (a->val != b->val)
        return a->val < b->val ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

static int first_repeat(const void *x, int t, int64_t a, int64_t b, int64_t lo, int64_t hi,
                        int64_t *out_i, int64_t *out_j)
{
    *out_i = -1;
    *out_j = -1;
    int64_t mn = INT64_MAX, mx = INT64_MIN, cnt = 0;
    for (int64_t i = a; i < b; i++) {
        int64_t xi = get(x, t, i);
        if (xi < lo || xi > hi)
            continue;
        cnt++;
        if (xi < mn)
            mn = xi;
        if (xi > mx)
            mx = xi;
    }
    if (cnt < 2)
        return IXO_OK;
    uint64_t span = (uint64_t)mx - (uint64_t)mn + 1u; /* mx >= mn here */
    if (span != 0 && span <= 4u * (uint64_t)(b - a) + 64u) {
        uint8_t *c = calloc(span, 1);
        if (!c)
            return IXO_E_NOMEM;
        for (int64_t i = a; i < b; i++) {
            int64_t xi = get(x, t, i);
            if (xi < lo || xi > hi)
                continue;
            uint8_t *ci = &c[(uint64_t)xi - (uint64_t)mn];
            if (*ci < 2)
                (*ci)++;
        }
        for (int64_t i = a; i < b && *out_i < 0; i++) {
            int64_t xi = get(x, t, i);
            if (xi >= lo && xi <= hi && c[(uint64_t)xi - (uint64_t)mn] >= 2)
                *out_i = i;
        }
        free(c);
    } else {
        pair_t *p = malloc((size_t)cnt * sizeof(pair_t));
        if (!p)
            return IXO_E_NOMEM;
        int64_t m = 0;
        for (int64_t i = a; i < b; i++) {
            int64_t xi = get(x, t, i);
            if (xi >= lo && xi <= hi) {
                p[m].val = xi;
                p[m].idx = i;
                m++;
            }
        }
        qsort(p, (size_t)m, sizeof(pair_t), pair_cmp);
        for (int64_t r = 0; r + 1 < m; r++)
            if (p[r].val == p[r + 1].val && (*out_i < 0 || p[r].idx < *out_i))
                *out_i = p[r].idx; /* p[r] is the first occurrence when r starts a run */
        free(p);
    }
    if (*out_i >= 0) {
        int64_t v0 = get(x, t, *out_i);
        for (int64_t j = *out_i + 1; j < b; j++)
            if (get(x, t, j) == v0) {
                *out_j = j;
                break;
            }
    }
    return IXO_OK;
}

/* ----------------------------------------------------------------- Inj
 * Fig. 5, Inj X Rcd: for j < i, X[i] in Rcd and X[j] in Rcd imply X[i] != X[j].
 * Rcd = [rlo, rhi] closed. Segmented: a reading, Inj applied to each segment on
 * its own (the paper extends only OrthogPreds, Bij, FiltPart, InvFiltPart to
 * segments). Verdict: index = i, value = X[i], aux0 = j (see first_repeat). */
int ixo_check_inj(const void *x, int t, int64_t n, int64_t rlo, int64_t rhi, const int64_t *off,
                  int64_t nseg, ixo_verdict *v, uint8_t *seg_ok)
{
    if (bad_type(t))
        return IXO_E_DTYPE;
    if (n < 0 || rlo > rhi || (n > 0 && !x) || !v || !segs_valid(off, nseg, n))
        return IXO_E_INVAL;
    verdict_ok(v);
    for (int64_t k = 0; k < seg_count(off, nseg); k++) {
        int64_t i, j;
        int rc = first_repeat(x, t, seg_lo(off, k), seg_hi(off, k, n), rlo, rhi, &i, &j);
        if (rc)
            return rc;
        if (seg_ok)
            seg_ok[k] = (uint8_t)(i < 0);
        if (i >= 0 && v->ok) {
            v->ok = 0;
            v->kind = K_DUPLICATE;
            v->index = i;
            v->value = get(x, t, i);
            v->aux0 = j;
        }
    }
    return IXO_OK;
}

/* ----------------------------------------------------------------- Bij
 * Fig. 5, Bij X Rcd (Img_k): Inj X Rcd and, per segment, the set of in-Rcd values
 * equals Img_k. The paper notes Img must lie inside Rcd (Sec. 2.3) and proves Bij
 * by counting (rule BijF1, Sec. 3.2: values inside Img, Inj, and |Img| equal to the
 * number of in-Rcd elements). Here the definition is tested directly, per segment:
 *   - the first position i with X[i] in Rcd but outside Img_k  -> OUT_OF_IMAGE
 *   - the first position i with X[i] in Img_k that occurs again -> DUPLICATE
 *     (the smaller of these two positions is reported)
 *   - otherwise, the smallest v in Img_k that no element takes  -> MISSING
 * seg_img != 0 selects Img_k = [e_k, e_{k+1} - 1]; otherwise Img_k = [ilo, ihi].
 * aux0 = number of elements with values in Img_k, aux1 = |Img_k| (for the
 * reported segment; summed over all segments when the property holds). */
int ixo_check_bij(const void *x, int t, int64_t n, int64_t rlo, int64_t rhi, int64_t ilo, int64_t ihi,
                  int seg_img, const int64_t *off, int64_t nseg, ixo_verdict *v, uint8_t *seg_ok)
{
    if (bad_type(t))
        return IXO_E_DTYPE;
    if (n < 0 || rlo > rhi || (n > 0 && !x) || !v || !segs_valid(off, nseg, n))
        return IXO_E_INVAL;
    if (seg_img && !off)
        return IXO_E_INVAL;
    if (!seg_img && (ilo > ihi || ilo < rlo || ihi > rhi || (uint64_t)ihi - (uint64_t)ilo >= ((uint64_t)1 << 40)))
        return IXO_E_INVAL;
    verdict_ok(v);
    int64_t sum_in = 0, sum_size = 0;
    for (int64_t k = 0; k < seg_count(off, nseg); k++) {
        int64_t a = seg_lo(off, k), b = seg_hi(off, k, n);
        int64_t lo = seg_img ? a : ilo, hi = seg_img ? b - 1 : ihi;
        if (seg_img && b > a && (lo < rlo || hi > rhi))
            return IXO_E_INVAL;
        int64_t bad_img = -1, in_img = 0;
        for (int64_t i = a; i < b; i++) {
            int64_t xi = get(x, t, i);
            if (xi < rlo || xi > rhi)
                continue;
            if (xi < lo || xi > hi) {
                if (bad_img < 0)
                    bad_img = i;
            } else {
                in_img++;
            }
        }
        int64_t di, dj;
        int rc = first_repeat(x, t, a, b, lo, hi, &di, &dj);
        if (rc)
            return rc;
        int64_t size = hi - lo + 1; /* 0 for an empty segment with seg_img */
        sum_in += in_img;
        sum_size += size;
        int sok = 1;
        if (bad_img >= 0 || di >= 0) {
            sok = 0;
            if (v->ok) {
                v->ok = 0;
                if (bad_img >= 0 && (di < 0 || bad_img < di)) {
                    v->kind = K_OUT_OF_IMAGE;
                    v->index = bad_img;
                    v->value = get(x, t, bad_img);
                } else {
                    v->kind = K_DUPLICATE;
                    v->index = di;
                    v->value = get(x, t, di);
                }
                v->aux0 = in_img;
                v->aux1 = size;
            }
        } else if (in_img < size) {
            /* injective and inside Img but not onto: find the smallest missing value */
            uint8_t *hit = calloc((size_t)size, 1);
            if (!hit)
                return IXO_E_NOMEM;
            for (int64_t i = a; i < b; i++) {
                int64_t xi = get(x, t, i);
                if (xi >= lo && xi <= hi)
                    hit[xi - lo] = 1;
            }
            int64_t miss = 0;
            while (miss < size && hit[miss])
                miss++;
            free(hit);
            sok = 0;
            if (v->ok) {
                v->ok = 0;
                v->kind = K_MISSING;
                v->index = -1;
                v->value = lo + miss;
                v->aux0 = in_img;
                v->aux1 = size;
            }
        }
        if (seg_ok)
            seg_ok[k] = (uint8_t)sok;
    }
    if (v->ok) {
        v->aux0 = sum_in;
        v->aux1 = sum_size;
    }
    return IXO_OK;
}

/* ------------------------------------------------------ FiltPart destinations
 * Fig. 5, FiltPart Y X (e_k, p^f, p^p_1..v): per segment k, filter the indices
 * [e_k, e_{k+1}) by p^f, partition them stably v ways (class 1 first, ...), gather X
 * at the result and flatten. The scatter-index form (InvFiltPart, Sec. 2.3) is the
 * array Z with scatter(Y0, Z, X) = Y: Z[i] is the position of i in that flattened
 * order for kept i, and dropped i must be ignored by scatter (Z[i] outside [0, N)).
 * Reading: InvFiltPart's four listed conditions alone admit non-filters (n = 2,
 * p^f = [T, F], Z = [5, 0]), so the check is the scatter equality itself.
 * Classes: cls[i] (0-based, entries >= v-1 fall in the last class v-1, which is
 * p^p_v = not(p_1 or ... or p_{v-1})), or, with cls == NULL, v = 2 and class 0 =
 * part(i) true. This routine writes ref[i] (or -1 for dropped i) and returns N. */
static int filtpart_ref(int64_t n, const void *keys, int kt, const ixo_pred *filt, const uint8_t *cls,
                        const ixo_pred *part, int v, const int64_t *off, int64_t nseg, int64_t *ref,
                        int64_t *N)
{
    int64_t pos = 0;
    int64_t *sigma = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!sigma)
        return IXO_E_NOMEM;
    for (int64_t i = 0; i < n; i++)
        ref[i] = -1;
    for (int64_t k = 0; k < seg_count(off, nseg); k++) {
        int64_t a = seg_lo(off, k), b = seg_hi(off, k, n);
        /* sigma = filter p^f [e_k .. e_{k+1}-1] */
        int64_t m = 0;
        for (int64_t i = a; i < b; i++)
            if (pred_eval(filt, keys, kt, i))
                sigma[m++] = i;
        /* sigma' = partition_v sigma; positions assigned in flattened order */
        for (int h = 0; h < v; h++)
            for (int64_t r = 0; r < m; r++) {
                int64_t i = sigma[r];
                int ci = cls ? (cls[i] >= v - 1 ? v - 1 : cls[i]) : (pred_eval(part, keys, kt, i) ? 0 : 1);
                if (ci == h)
                    ref[i] = pos++;
            }
    }
    free(sigma);
    *N = pos;
    return IXO_OK;
}

/* Index mode: verdict on Z. index = first i with a wrong destination, value = Z[i],
 * aux0 = N (length of the filtered-partitioned result), aux1 = expected
 * destination (-1 for a dropped element). */
int ixo_check_filtpart(const void *z, int zt, int64_t n, const void *keys, int kt, ixo_pred filt,
                       const uint8_t *cls, ixo_pred part, int v, const int64_t *off, int64_t nseg,
                       ixo_verdict *vd)
{
    if (bad_type(zt))
        return IXO_E_DTYPE;
    if (n < 0 || (n > 0 && !z) || !vd || !segs_valid(off, nseg, n) || v < 1 || v > 256)
        return IXO_E_INVAL;
    if (!pred_valid(&filt, keys, kt) || (!cls && (v != 2 || !pred_valid(&part, keys, kt))))
        return IXO_E_INVAL;
    int64_t *ref = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t)), N = 0;
    if (!ref)
        return IXO_E_NOMEM;
    int rc = filtpart_ref(n, keys, kt, &filt, cls, &part, v, off, nseg, ref, &N);
    if (rc) {
        free(ref);
        return rc;
    }
    verdict_ok(vd);
    vd->aux0 = N;
    for (int64_t i = 0; i < n; i++) {
        int64_t zi = get(z, zt, i);
        int bad = ref[i] >= 0 ? (zi != ref[i]) : (zi >= 0 && zi < N);
        if (bad) {
            vd->ok = 0;
            vd->kind = K_WRONG_DEST;
            vd->index = i;
            vd->value = zi;
            vd->aux1 = ref[i];
            break;
        }
    }
    free(ref);
    return IXO_OK;
}

/* Value mode: Y (row_bytes per element) equals the FiltPart of X bitwise and has
 * length N. Verdict index = first position p of Y that differs (value = p's source
 * index in X), or kind WRONG_DEST with index -1 when ny != N. */
int ixo_check_filtpart_values(const void *y, int64_t ny, const void *x, int64_t n, int row_bytes,
                              const void *keys, int kt, ixo_pred filt, const uint8_t *cls, ixo_pred part,
                              int v, const int64_t *off, int64_t nseg, ixo_verdict *vd)
{
    if (n < 0 || ny < 0 || row_bytes <= 0 || !vd || !segs_valid(off, nseg, n) || v < 1 || v > 256)
        return IXO_E_INVAL;
    if (!pred_valid(&filt, keys, kt) || (!cls && (v != 2 || !pred_valid(&part, keys, kt))))
        return IXO_E_INVAL;
    int64_t *ref = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t)), N = 0;
    if (!ref)
        return IXO_E_NOMEM;
    int rc = filtpart_ref(n, keys, kt, &filt, cls, &part, v, off, nseg, ref, &N);
    if (rc) {
        free(ref);
        return rc;
    }
    verdict_ok(vd);
    vd->aux0 = N;
    if (ny != N) {
        vd->ok = 0;
        vd->kind = K_WRONG_DEST;
        vd->index = -1;
        vd->value = ny;
    } else {
        int64_t best = -1, src = -1;
        for (int64_t i = 0; i < n; i++)
            if (ref[i] >= 0 && memcmp((const char *)y + ref[i] * row_bytes, (const char *)x + i * row_bytes,
                                      (size_t)row_bytes) != 0 &&
                (best < 0 || ref[i] < best)) {
                best = ref[i];
                src = i;
            }
        if (best >= 0) {
            vd->ok = 0;
            vd->kind = K_WRONG_DEST;
            vd->index = best;
            vd->value = src;
        }
    }
    free(ref);
    return IXO_OK;
}

/* ------------------------------------------------------------------ scan
 * Sec. 2.1: scan op ne [x0..x_{n-1}] = [x0, x0 op x1, ...] is inclusive; the
 * exclusive form shifts by one and starts at the neutral element 0. Segmented:
 * the sum restarts at each e_k. Overflow (the paper is silent): two's-complement
 * wrap in the output width. totals[k] = sum of segment k (one entry when flat). */
int ixo_scan(const void *in, int it, void *out, int ot, int64_t n, int inclusive, const int64_t *off,
             int64_t nseg, void *totals)
{
    if (bad_type(it) || bad_type(ot))
        return IXO_E_DTYPE;
    if (n < 0 || (n > 0 && (!in || !out)) || !segs_valid(off, nseg, n))
        return IXO_E_INVAL;
    for (int64_t k = 0; k < seg_count(off, nseg); k++) {
        uint64_t acc = 0;
        for (int64_t i = seg_lo(off, k); i < seg_hi(off, k, n); i++) {
            uint64_t xi = (uint64_t)get(in, it, i);
            if (inclusive) {
                acc += xi;
                put(out, ot, i, acc);
            } else {
                put(out, ot, i, acc);
                acc += xi;
            }
        }
        if (totals)
            put(totals, ot, k, acc);
    }
    return IXO_OK;
}

/* Segmented inclusive scan with a flag array, the sgmSum of Fig. 2 (right): the
 * lifted operator (f1, v1) + (f2, v2) = (f1 or f2, f2 ? v2 : v1 + v2), applied
 * left to right. Reading: the figure's variable names are garbled (f1/v1 vs fx/vx);
 * the operator above is the standard segmented-scan operator they denote. */
int ixo_sgm_scan(const uint8_t *flags, const void *in, int it, void *out, int ot, int64_t n)
{
    if (bad_type(it) || bad_type(ot))
        return IXO_E_DTYPE;
    if (n < 0 || (n > 0 && (!flags || !in || !out)))
        return IXO_E_INVAL;
    int f = 0;
    uint64_t acc = 0;
    for (int64_t i = 0; i < n; i++) {
        int f2 = flags[i] != 0;
        uint64_t v2 = (uint64_t)get(in, it, i);
        if (i == 0) {
            f = f2;
            acc = v2;
        } else {
            acc = f2 ? v2 : acc + v2;
            f = f || f2;
        }
        put(out, ot, i, acc);
    }
    (void)f;
    return IXO_OK;
}

/* -------------------------------------------------------------- scatter
 * Sec. 2.1: scatter dst is vs = for i in 0..m-1: if 0 <= is[i] < len(dst) then
 * dst[is[i]] := vs[i]. Reading: the printed bound "< m" is garbled; the prose says
 * indices out of bounds of dst are ignored, so the bound is len(dst). Rows of
 * row_bytes bytes are moved bitwise. Duplicates: later writes win (the paper
 * requires duplicate indices to carry equal values, which makes the order moot). */
int ixo_scatter(void *dst, int64_t dst_len, const void *idx, int it, const void *vals, int64_t n, int row_bytes)
{
    if (bad_type(it))
        return IXO_E_DTYPE;
    if (n < 0 || dst_len < 0 || row_bytes <= 0 || (n > 0 && (!idx || !vals)) || (dst_len > 0 && !dst))
        return IXO_E_INVAL;
    for (int64_t i = 0; i < n; i++) {
        int64_t d = get(idx, it, i);
        if (0 <= d && d < dst_len)
            memcpy((char *)dst + d * row_bytes, (const char *)vals + i * row_bytes, (size_t)row_bytes);
    }
    return IXO_OK;
}

/* Additive scatter, accumulated in double: dst[is[i]] += vs[i] for in-bounds is[i].
 * vals_bytes = 4 (float) or 8 (double), row_elems values per row. */
int ixo_scatter_add_f64(double *dst, int64_t dst_len, const void *idx, int it, const void *vals, int vals_bytes,
                        int64_t n, int row_elems)
{
    if (bad_type(it))
        return IXO_E_DTYPE;
    if (n < 0 || dst_len < 0 || row_elems <= 0 || (vals_bytes != 4 && vals_bytes != 8))
        return IXO_E_INVAL;
    for (int64_t i = 0; i < n; i++) {
        int64_t d = get(idx, it, i);
        if (d < 0 || d >= dst_len)
            continue;
        for (int c = 0; c < row_elems; c++) {
            double vi = vals_bytes == 4 ? (double)((const float *)vals)[i * row_elems + c]
                                        : ((const double *)vals)[i * row_elems + c];
            dst[d * row_elems + c] += vi;
        }
    }
    return IXO_OK;
}

/* Gather: out[i] = src[idx[i]]. An index outside [0, src_len) is an error; its
 * row is zero-filled and the call returns IXO_E_OOB after finishing the rest. */
int ixo_gather(void *out, const void *src, int64_t src_len, const void *idx, int it, int64_t n, int row_bytes)
{
    if (bad_type(it))
        return IXO_E_DTYPE;
    if (n < 0 || src_len < 0 || row_bytes <= 0 || (n > 0 && (!idx || !out)))
        return IXO_E_INVAL;
    int rc = IXO_OK;
    for (int64_t i = 0; i < n; i++) {
        int64_t s = get(idx, it, i);
        if (0 <= s && s < src_len) {
            memcpy((char *)out + i * row_bytes, (const char *)src + s * row_bytes, (size_t)row_bytes);
        } else {
            memset((char *)out + i * row_bytes, 0, (size_t)row_bytes);
            rc = IXO_E_OOB;
        }
    }
    return rc;
}

/* --------------------------------------------------------------- partition
 * Stable two-way partition (Sec. 2.1 and Fig. 2, partition2; Sec. 6, partition2L
 * for segments). What it computes: inside each segment [e_k, e_{k+1}) the elements
 * whose predicate holds come first and the others after them, each group keeping
 * its input order; indices[i] is the position element i moves to (the scatter
 * destination, Sec. 2.3), and num_true[k] is the size of segment k's first group.
 * Written as two ordered walks over each segment: the first hands out e_k, e_k+1,
 * ... to the elements whose predicate holds, the second continues the count for
 * the others. Optionally the keys and payload rows are moved to their positions. */
static void partition_move(int64_t i, int64_t d, void *out_idx, int ot, const void *keys, int kt,
                           void *out_keys, const void *payload, int row_bytes, void *out_payload)
{
    put(out_idx, ot, i, (uint64_t)d);
    if (out_keys)
        memcpy((char *)out_keys + d * (kt ? 8 : 4), (const char *)keys + i * (kt ? 8 : 4), kt ? 8 : 4);
    if (out_payload)
        memcpy((char *)out_payload + d * row_bytes, (const char *)payload + i * row_bytes, (size_t)row_bytes);
}

int ixo_partition(const void *keys, int kt, int64_t n, ixo_pred p, const void *payload, int row_bytes,
                  void *out_idx, int ot, void *out_keys, void *out_payload, int64_t *num_true,
                  const int64_t *off, int64_t nseg)
{
    if (bad_type(ot) || (keys && bad_type(kt)))
        return IXO_E_DTYPE;
    if (n < 0 || (n > 0 && !out_idx) || !num_true || !segs_valid(off, nseg, n) || !pred_valid(&p, keys, kt))
        return IXO_E_INVAL;
    if ((out_keys && !keys) || (out_payload && (!payload || row_bytes <= 0)))
        return IXO_E_INVAL;
    if (ot == 0 && n > INT32_MAX)
        return IXO_E_INVAL;
    for (int64_t k = 0; k < seg_count(off, nseg); k++) {
        int64_t a = seg_lo(off, k), b = seg_hi(off, k, n);
        int64_t next = a; /* the next free position of segment k */
        for (int64_t i = a; i < b; i++)
            if (pred_eval(&p, keys, kt, i))
                partition_move(i, next++, out_idx, ot, keys, kt, out_keys, payload, row_bytes, out_payload);
        num_true[off ? k : 0] = next - a;
        for (int64_t i = a; i < b; i++)
            if (!pred_eval(&p, keys, kt, i))
                partition_move(i, next++, out_idx, ot, keys, kt, out_keys, payload, row_bytes, out_payload);
    }
    return IXO_OK;
}

/* ------------------------------------------------------------ mkSgmDescr
 * mkSgmDescr shape xs (Fig. 2, right; Sec. 2.1): segment k occupies positions
 * [e_k, e_k + shape[k]) of a zero array of length sum(shape), where e_k is the sum
 * of the shapes before k; the first position of every non-empty segment holds
 * xs[k]. Written as one running offset over the segments. Precondition Range shape
 * (0, inf): negative shapes are rejected. xs == NULL means all ones (a plain flag
 * array). offsets (nullable) gets e_0 .. e_{m-1} followed by the total (m + 1
 * entries). */
int ixo_flags_from_shape(const int64_t *shape, int64_t m, const int64_t *xs, void *out, int ot, int64_t out_len,
                         int64_t *offsets)
{
    if (bad_type(ot))
        return IXO_E_DTYPE;
    if (m < 0 || (m > 0 && !shape))
        return IXO_E_INVAL;
    int64_t len = 0;
    for (int64_t k = 0; k < m; k++) {
        if (shape[k] < 0)
            return IXO_E_INVAL;
        len += shape[k];
    }
    if (len != out_len || (len > 0 && !out))
        return IXO_E_INVAL;
    for (int64_t j = 0; j < len; j++)
        put(out, ot, j, 0);
    int64_t e = 0;
    for (int64_t k = 0; k < m; k++) {
        if (offsets)
            offsets[k] = e;
        if (shape[k] > 0)
            put(out, ot, e, (uint64_t)(xs ? xs[k] : 1));
        e += shape[k];
    }
    if (offsets)
        offsets[m] = len;
    return IXO_OK;
}

/* ------------------------------------------------------------------ mkII
 * mkII shape (Fig. 2, right): II[j] = k for e_k <= j < e_{k+1}, the segment number
 * of every position (the prose of Sec. 2.1). Reading: the figure builds its flags
 * after subtracting one, which would miss a non-empty segment 0; the definition
 * above is what is computed. Written as a walk that repeats k shape[k] times. */
int ixo_mkii(const int64_t *shape, int64_t m, int64_t *out, int64_t out_len)
{
    if (m < 0 || (m > 0 && !shape))
        return IXO_E_INVAL;
    int64_t len = 0;
    for (int64_t k = 0; k < m; k++) {
        if (shape[k] < 0)
            return IXO_E_INVAL;
        len += shape[k];
    }
    if (len != out_len || (len > 0 && !out))
        return IXO_E_INVAL;
    int64_t j = 0;
    for (int64_t k = 0; k < m; k++)
        for (int64_t r = 0; r < shape[k]; r++)
            out[j++] = k;
    return IXO_OK;
}

/* ------------------------------------------------------------- hist min
 * Reduce-by-index with min, Futhark's `hist` with the min operator (Sec. 6:
 * get_smallest_pairs of maxMatching, Fig. 16, and the reduce-by-index that the
 * dynamic verification of scatter needs). H holds the neutral element on entry
 * (the caller fills it); for i = 0..n-1 in order, if 0 <= idx[i] < m then
 * H[idx[i]] = min(H[idx[i]], vals[i]). vals NULL means vals[i] = i. An index out of
 * bounds is ignored, as scatter ignores it (Sec. 2.1). H and vals share type ht. */
int ixo_hist_min(void *H, int ht, int64_t m, const void *idx, int it, const void *vals, int64_t n)
{
    if (bad_type(ht) || bad_type(it))
        return IXO_E_DTYPE;
    if (n < 0 || m < 0 || (n > 0 && !idx) || (m > 0 && !H))
        return IXO_E_INVAL;
    for (int64_t i = 0; i < n; i++) {
        int64_t k = get(idx, it, i);
        if (k < 0 || k >= m)
            continue;
        int64_t v = vals ? get(vals, ht, i) : i;
        if (v < get(H, ht, k))
            put(H, ht, k, (uint64_t)v);
    }
    return IXO_OK;
}

/* -------------------------------------------------- get_smallest_pairs
 * get_smallest_pairs of maxMatching (Sec. 6, Fig. 16): slot i is an edge endpoint
 * es[i] with priority is[i]. Slot i is kept when es[i] names a vertex of
 * [0, n_verts) and is[i] equals the smallest of n_es and the priorities of every
 * slot of that vertex; the kept (es[i], is[i]) pairs are written in input order.
 * Written as: the smallest priority per vertex (starting from n_es), then one
 * ordered walk that keeps the slots that attain it. Reading: the precondition
 * Range es (0, n_verts) is half-open (es indexes the vertex array); a slot outside
 * it names no vertex and is not kept. es and is share type t; out_es and out_is
 * have room for n entries; *count gets the number kept. */
int ixo_smallest_pairs(int64_t n_verts, int64_t n_es, const void *es, const void *is, int t, int64_t n,
                       void *out_es, void *out_is, int64_t *count)
{
    if (bad_type(t))
        return IXO_E_DTYPE;
    if (n < 0 || n_verts < 0 || (n > 0 && (!es || !is || !out_es || !out_is)) || !count)
        return IXO_E_INVAL;
    int64_t *best = malloc((size_t)(n_verts > 0 ? n_verts : 1) * 8);
    if (!best)
        return IXO_E_NOMEM;
    for (int64_t v = 0; v < n_verts; v++)
        best[v] = n_es;
    for (int64_t i = 0; i < n; i++) {
        int64_t v = get(es, t, i), pr = get(is, t, i);
        if (v >= 0 && v < n_verts && pr < best[v])
            best[v] = pr;
    }
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t v = get(es, t, i), pr = get(is, t, i);
        if (v >= 0 && v < n_verts && pr == best[v]) {
            put(out_es, t, c, (uint64_t)v);
            put(out_is, t, c, (uint64_t)pr);
            c++;
        }
    }
    *count = c;
    free(best);
    return IXO_OK;
}
