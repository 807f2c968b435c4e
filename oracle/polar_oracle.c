/*
 * Plain CPU oracle for Fast-SSC decoding of systematic polar codes
 * (Giard et al., "Low-Latency Software Polar Decoders", arXiv 1504.00353).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the GPU library. It is written for a
 * reader checking it against the paper, not for speed: recursion over the
 * decoder tree, one element at a time, in the order the paper states.
 *
 * Both LLR types run through one routine on binary32 values. For the int8
 * decoder every value is an integer in [-127, 127]; F, G, the Repetition sums
 * and the SPC magnitudes are then exact in binary32, and `sat` clamps each G
 * result (and each Repetition partial sum) to [-127, 127], which is the
 * saturating add followed by max(-127) that Sec. III-A and Listing 4 describe.
 * Clamping both ends keeps the range symmetric, so |a| never overflows in F.
 *
 * Parity status: every function here is pinned by tests under tests/ (closed
 * forms, brute force, invariants and the paper's worked example); see the
 * test files for which pin covers which part.
 */
#include "polar_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Element operations                                                  */
/* ------------------------------------------------------------------ */

/* Eq. 1: sgn(a) sgn(b) min(|a|, |b|). sgn(0) is taken as +1; the product only
 * matters when the magnitude is non-zero, so the choice never changes a value. */
static float f_op(float a, float b)
{
    float ma = a < 0.0f ? -a : a;
    float mb = b < 0.0f ? -b : b;
    float m = ma < mb ? ma : mb;
    int negative = (a < 0.0f) != (b < 0.0f);
    return negative ? -m : m;
}

static float clamp127(float v)
{
    if (v > 127.0f) return 127.0f;
    if (v < -127.0f) return -127.0f;
    return v;
}

/* Eq. 2: alpha_v[i + N_v/2] + alpha_v[i] when beta_l[i] = 0, else the
 * difference alpha_v[i + N_v/2] - alpha_v[i]. a = alpha_v[i],
 * b = alpha_v[i + N_v/2]. */
static float g_op(float a, float b, uint8_t beta_l, int sat)
{
    float r = beta_l ? (b - a) : (b + a);
    return sat ? clamp127(r) : r;
}

/* Eq. 4 / leaf threshold: alpha >= 0 decides 0 (a negative zero also
 * decides 0, since values are compared, not sign bits). */
static uint8_t hard(float a) { return a < 0.0f ? 1 : 0; }

float oracle_f_f32(float a, float b) { return f_op(a, b); }
float oracle_g_f32(float a, float b, uint8_t beta_l) { return g_op(a, b, beta_l, 0); }
int8_t oracle_f_i8(int8_t a, int8_t b) { return (int8_t)f_op((float)a, (float)b); }
int8_t oracle_g_i8(int8_t a, int8_t b, uint8_t beta_l)
{
    return (int8_t)g_op((float)a, (float)b, beta_l, 1);
}

/* ------------------------------------------------------------------ */
/* Encoding                                                            */
/* ------------------------------------------------------------------ */

static int is_pow2(uint32_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/* x = u * F_2^{(x)n}. With F_2 = [[1,0],[1,1]] a length-2 block maps
 * (u0, u1) to (u0 ^ u1, u1) (Fig. 1a); applying that butterfly at spans
 * 1, 2, ..., N/2 gives the Kronecker power (the N = 4 matrix of Sec. II-A). */
void oracle_encode(uint32_t N, const uint8_t *u, uint8_t *x)
{
    if (x != u) memcpy(x, u, N);
    for (uint32_t h = 1; h < N; h *= 2)
        for (uint32_t blk = 0; blk < N; blk += 2 * h)
            for (uint32_t i = blk; i < blk + h; i++)
                x[i] ^= x[i + h];
}

int oracle_encode_systematic(uint32_t N, const uint8_t *frozen, const uint8_t *d,
                             uint8_t *x)
{
    if (!is_pow2(N)) return -1;
    uint8_t *v = (uint8_t *)malloc(N);
    if (!v) return -1;
    uint32_t k = 0;
    for (uint32_t i = 0; i < N; i++) v[i] = frozen[i] ? 0 : d[k++];
    oracle_encode(N, v, v);
    for (uint32_t i = 0; i < N; i++)
        if (frozen[i]) v[i] = 0;
    oracle_encode(N, v, x);
    free(v);
    k = 0;
    for (uint32_t i = 0; i < N; i++)
        if (!frozen[i] && x[i] != d[k++]) return -1;
    return 0;
}

void oracle_extract_info(uint32_t N, const uint8_t *frozen, const uint8_t *xhat,
                         uint8_t *info_packed)
{
    uint32_t K = 0;
    for (uint32_t i = 0; i < N; i++) K += frozen[i] ? 0 : 1;
    memset(info_packed, 0, (K + 7) / 8);
    uint32_t k = 0;
    for (uint32_t i = 0; i < N; i++) {
        if (frozen[i]) continue;
        if (xhat[i]) info_packed[k / 8] |= (uint8_t)(1u << (k % 8));
        k++;
    }
}

/* ------------------------------------------------------------------ */
/* SC decoding (Sec. II-C)                                             */
/* ------------------------------------------------------------------ */

/* Decode the node whose input LLRs are a[0..n) and whose leaves are
 * frozen[0..n); write its bit estimates beta[0..n). work holds n floats. */
static void sc_node(const float *a, uint32_t n, const uint8_t *frozen, uint8_t *beta,
                    float *work, int sat)
{
    if (n == 1) {
        beta[0] = frozen[0] ? 0 : hard(a[0]);
        return;
    }
    uint32_t h = n / 2;
    float *child = work;
    for (uint32_t i = 0; i < h; i++) child[i] = f_op(a[i], a[i + h]);
    sc_node(child, h, frozen, beta, work + h, sat);
    for (uint32_t i = 0; i < h; i++) child[i] = g_op(a[i], a[i + h], beta[i], sat);
    sc_node(child, h, frozen + h, beta + h, work + h, sat);
    /* Eq. 3: left half XOR right half; the right half is copied as is. */
    for (uint32_t i = 0; i < h; i++) beta[i] ^= beta[i + h];
}

static int sc_decode(uint32_t N, const uint8_t *frozen, const float *llr, uint8_t *xhat,
                     int sat)
{
    if (!is_pow2(N)) return -1;
    float *work = (float *)malloc(sizeof(float) * (N + 1));
    if (!work) return -1;
    sc_node(llr, N, frozen, xhat, work, sat);
    free(work);
    return 0;
}

int oracle_sc_decode_f32(uint32_t N, const uint8_t *frozen, const float *llr,
                         uint8_t *xhat)
{
    return sc_decode(N, frozen, llr, xhat, 0);
}

int oracle_sc_decode_i8(uint32_t N, const uint8_t *frozen, const int8_t *llr,
                        uint8_t *xhat)
{
    float *a = (float *)malloc(sizeof(float) * N);
    if (!a) return -1;
    for (uint32_t i = 0; i < N; i++) a[i] = (float)llr[i];
    int rc = sc_decode(N, frozen, a, xhat, 1);
    free(a);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Fast-SSC decoding (Sec. II-D, Listing 1)                            */
/* ------------------------------------------------------------------ */

enum { NODE_R0, NODE_R1, NODE_REP, NODE_SPC, NODE_SPLIT };

typedef struct {
    uint32_t max_rep, max_spc;
    int sat;
    oracle_trace *trace;
} fssc_ctx;

/* Node type from its leaves, checked in this order: all frozen -> Rate-0;
 * none frozen -> Rate-1; only the last leaf is information -> Repetition;
 * only the first leaf is frozen -> SPC; otherwise the node is split.
 * (A size-2 node [frozen, info] is both Repetition and SPC; it is taken as
 * Repetition.) */
static int classify(const uint8_t *frozen, uint32_t n, const fssc_ctx *c)
{
    uint32_t nf = 0;
    for (uint32_t i = 0; i < n; i++) nf += frozen[i] ? 1 : 0;
    if (nf == n) return NODE_R0;
    if (nf == 0) return NODE_R1;
    if (nf == n - 1 && !frozen[n - 1] && n <= c->max_rep) return NODE_REP;
    if (nf == 1 && frozen[0] && n <= c->max_spc) return NODE_SPC;
    return NODE_SPLIT;
}

static void trace_op(fssc_ctx *c, uint32_t kind, uint32_t nv, uint32_t off)
{
    oracle_trace *t = c->trace;
    if (!t) return;
    if (t->n_ops >= t->cap_ops) {
        t->overflow = 1;
        return;
    }
    t->kind[t->n_ops] = kind;
    t->nv[t->n_ops] = nv;
    t->off[t->n_ops] = off;
    t->n_ops++;
}

static void trace_alpha(fssc_ctx *c, const float *v, uint32_t n)
{
    oracle_trace *t = c->trace;
    if (!t) return;
    if (t->n_alpha + n > t->cap_alpha) {
        t->overflow = 1;
        return;
    }
    memcpy(t->alpha + t->n_alpha, v, sizeof(float) * n);
    t->n_alpha += n;
}

/* Node decoders. a: the node's LLRs alpha_v, n = N_v, beta: its estimates. */

static void rate1_node(const float *a, uint32_t n, uint8_t *beta)
{
    for (uint32_t i = 0; i < n; i++) beta[i] = hard(a[i]); /* Eq. 4 */
}

/* Repetition: threshold of the sum of the LLRs, replicated. The sum is taken
 * as the halving folds t[i] <- t[i] + t[i + m/2] (m = n, n/2, ..., 2), which is
 * exactly what SC computes on this node (a chain of G with a zero left
 * estimate); the int8 decoder saturates after each fold, as G does. */
static void rep_node(const float *a, uint32_t n, uint8_t *beta, float *work, int sat)
{
    float *t = work;
    memcpy(t, a, sizeof(float) * n);
    for (uint32_t m = n; m > 1; m /= 2)
        for (uint32_t i = 0; i < m / 2; i++) {
            float s = t[i] + t[i + m / 2];
            t[i] = sat ? clamp127(s) : s;
        }
    uint8_t bit = t[0] < 0.0f ? 1 : 0; /* sum >= 0 decides 0 */
    for (uint32_t i = 0; i < n; i++) beta[i] = bit;
}

/* SPC: hard decisions, their parity, and if the parity is odd the decision
 * with the smallest |alpha| is flipped. Among equal magnitudes the lowest
 * index is flipped (Listing 2 returns the first lane equal to the minimum). */
static void spc_node(const float *a, uint32_t n, uint8_t *beta)
{
    uint8_t parity = 0;
    uint32_t jmin = 0;
    float mmin = a[0] < 0.0f ? -a[0] : a[0];
    for (uint32_t i = 0; i < n; i++) {
        beta[i] = hard(a[i]);
        parity ^= beta[i];
        float m = a[i] < 0.0f ? -a[i] : a[i];
        if (m < mmin) {
            mmin = m;
            jmin = i;
        }
    }
    beta[jmin] ^= parity;
}

/* Decode the node with LLRs a[0..n), leaves frozen[0..n) starting at leaf
 * index off; write beta[0..n). work: scratch of at least 2n floats. */
static void fssc_node(const float *a, uint32_t n, const uint8_t *frozen, uint32_t off,
                      uint8_t *beta, float *work, fssc_ctx *c)
{
    int type = classify(frozen, n, c);
    switch (type) {
    case NODE_R0:
        trace_op(c, ORACLE_OP_R0, n, off);
        memset(beta, 0, n);
        return;
    case NODE_R1:
        trace_op(c, ORACLE_OP_R1, n, off);
        rate1_node(a, n, beta);
        return;
    case NODE_REP:
        trace_op(c, ORACLE_OP_REP, n, off);
        rep_node(a, n, beta, work, c->sat);
        return;
    case NODE_SPC:
        trace_op(c, ORACLE_OP_SPC, n, off);
        spc_node(a, n, beta);
        return;
    default:
        break;
    }

    uint32_t h = n / 2;
    float *child = work; /* alpha of the child being decoded, h values */
    int left = classify(frozen, h, c);
    int right = classify(frozen + h, h, c);

    if (left == NODE_R0) {
        /* Left estimate is all-zero: G reduces to the plain sum (G_0R), the
         * left subtree needs no work, and the combine copies beta_r into the
         * left half (Combine_0R). */
        trace_op(c, ORACLE_OP_G0R, n, off);
        for (uint32_t i = 0; i < h; i++) child[i] = g_op(a[i], a[i + h], 0, c->sat);
        trace_alpha(c, child, h);
        fssc_node(child, h, frozen + h, off + h, beta + h, work + h, c);
        trace_op(c, ORACLE_OP_C0R, n, off);
        for (uint32_t i = 0; i < h; i++) beta[i] = beta[i + h];
        return;
    }

    trace_op(c, ORACLE_OP_F, n, off);
    for (uint32_t i = 0; i < h; i++) child[i] = f_op(a[i], a[i + h]);
    trace_alpha(c, child, h);
    fssc_node(child, h, frozen, off, beta, work + h, c);

    if (right == NODE_R0) {
        /* beta_r is all-zero: no G is needed and Eq. 3 leaves beta_l as is. */
        trace_op(c, ORACLE_OP_R0, h, off + h);
        memset(beta + h, 0, h);
        return;
    }

    trace_op(c, ORACLE_OP_G, n, off);
    for (uint32_t i = 0; i < h; i++) child[i] = g_op(a[i], a[i + h], beta[i], c->sat);
    trace_alpha(c, child, h);
    fssc_node(child, h, frozen + h, off + h, beta + h, work + h, c);
    trace_op(c, ORACLE_OP_C, n, off);
    for (uint32_t i = 0; i < h; i++) beta[i] ^= beta[i + h]; /* Eq. 3 */
}

static int fssc_decode(uint32_t N, const uint8_t *frozen, const float *llr,
                       uint32_t max_rep, uint32_t max_spc, uint8_t *xhat,
                       oracle_trace *trace, int sat)
{
    if (!is_pow2(N)) return -1;
    float *work = (float *)malloc(sizeof(float) * 2 * (N + 1));
    if (!work) return -1;
    fssc_ctx c;
    c.max_rep = max_rep;
    c.max_spc = max_spc;
    c.sat = sat;
    c.trace = trace;
    if (trace) {
        trace->n_ops = 0;
        trace->n_alpha = 0;
        trace->overflow = 0;
    }
    fssc_node(llr, N, frozen, 0, xhat, work, &c);
    free(work);
    return (trace && trace->overflow) ? -2 : 0;
}

int oracle_fastssc_decode_f32(uint32_t N, const uint8_t *frozen, const float *llr,
                              uint32_t max_rep, uint32_t max_spc, uint8_t *xhat,
                              oracle_trace *trace)
{
    return fssc_decode(N, frozen, llr, max_rep, max_spc, xhat, trace, 0);
}

int oracle_fastssc_decode_i8(uint32_t N, const uint8_t *frozen, const int8_t *llr,
                             uint32_t max_rep, uint32_t max_spc, uint8_t *xhat,
                             oracle_trace *trace)
{
    float *a = (float *)malloc(sizeof(float) * N);
    if (!a) return -1;
    for (uint32_t i = 0; i < N; i++) a[i] = (float)llr[i];
    int rc = fssc_decode(N, frozen, a, max_rep, max_spc, xhat, trace, 1);
    free(a);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Repetition-SPC node                                                 */
/* ------------------------------------------------------------------ */

/* Repetition-SPC node (Sec. II-D, "Repetition-SPC codes"): a node of n leaves
 * whose left child is a Repetition code and whose right child is an SPC code,
 * decoded speculatively. Three decodes are independent of one another: the
 * Repetition child on F of the node's LLRs (Eq. 1), and the SPC child on the
 * G outputs (Eq. 2) for a left estimate of all zeros and for one of all ones.
 * The Repetition decision then selects the matching SPC estimate, and Eq. 3
 * joins the halves. n is a power of two, 8 <= n. */
static int repspc_node(const float *a, uint32_t n, uint8_t *beta, int sat)
{
    uint32_t h = n / 2;
    float *buf = (float *)malloc(sizeof(float) * 4 * h);
    uint8_t *spc = (uint8_t *)malloc(2 * h);
    if (!buf || !spc) {
        free(buf);
        free(spc);
        return -1;
    }
    float *fl = buf, *g0 = buf + h, *g1 = buf + 2 * h, *work = buf + 3 * h;
    uint8_t rep[1];
    for (uint32_t i = 0; i < h; i++) {
        fl[i] = f_op(a[i], a[i + h]);
        g0[i] = g_op(a[i], a[i + h], 0, sat); /* left estimate all 0 */
        g1[i] = g_op(a[i], a[i + h], 1, sat); /* left estimate all 1 */
    }
    /* the Repetition decision is the same bit for every leaf of the left half */
    uint8_t *left = (uint8_t *)malloc(h);
    if (!left) {
        free(buf);
        free(spc);
        return -1;
    }
    rep_node(fl, h, left, work, sat);
    rep[0] = left[0];
    spc_node(g0, h, spc);
    spc_node(g1, h, spc + h);
    const uint8_t *right = rep[0] ? spc + h : spc;
    for (uint32_t i = 0; i < h; i++) {
        beta[i] = left[i] ^ right[i]; /* Eq. 3 */
        beta[i + h] = right[i];
    }
    free(left);
    free(buf);
    free(spc);
    return 0;
}

int oracle_repspc_f32(const float *alpha, uint32_t n, uint8_t *beta)
{
    if (!is_pow2(n) || n < 8) return -1;
    return repspc_node(alpha, n, beta, 0);
}

int oracle_repspc_i8(const int8_t *alpha, uint32_t n, uint8_t *beta)
{
    if (!is_pow2(n) || n < 8) return -1;
    float *a = (float *)malloc(sizeof(float) * n);
    if (!a) return -1;
    for (uint32_t i = 0; i < n; i++) a[i] = (float)alpha[i];
    int rc = repspc_node(a, n, beta, 1);
    free(a);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Batches                                                             */
/* ------------------------------------------------------------------ */

static int decode_batch(uint32_t N, const uint8_t *frozen, const float *llr_f,
                        const int8_t *llr_i, size_t n_frames, int algo,
                        uint32_t max_rep, uint32_t max_spc, uint8_t *out)
{
    if (!is_pow2(N)) return -1;
    uint32_t K = 0;
    for (uint32_t i = 0; i < N; i++) K += frozen[i] ? 0 : 1;
    size_t row = (K + 7) / 8;
    uint8_t *xhat = (uint8_t *)malloc(N);
    if (!xhat) return -1;
    int rc = 0;
    for (size_t f = 0; f < n_frames && rc == 0; f++) {
        if (llr_f) {
            const float *y = llr_f + f * (size_t)N;
            rc = algo == 1 ? oracle_sc_decode_f32(N, frozen, y, xhat)
                           : oracle_fastssc_decode_f32(N, frozen, y, max_rep, max_spc,
                                                       xhat, NULL);
        } else {
            const int8_t *y = llr_i + f * (size_t)N;
            rc = algo == 1 ? oracle_sc_decode_i8(N, frozen, y, xhat)
                           : oracle_fastssc_decode_i8(N, frozen, y, max_rep, max_spc,
                                                      xhat, NULL);
        }
        if (rc == 0 && row) oracle_extract_info(N, frozen, xhat, out + f * row);
    }
    free(xhat);
    return rc;
}

int oracle_decode_batch_f32(uint32_t N, const uint8_t *frozen, const float *llr,
                            size_t n_frames, int algo, uint32_t max_rep,
                            uint32_t max_spc, uint8_t *out)
{
    return decode_batch(N, frozen, llr, NULL, n_frames, algo, max_rep, max_spc, out);
}

int oracle_decode_batch_i8(uint32_t N, const uint8_t *frozen, const int8_t *llr,
                           size_t n_frames, int algo, uint32_t max_rep,
                           uint32_t max_spc, uint8_t *out)
{
    return decode_batch(N, frozen, NULL, llr, n_frames, algo, max_rep, max_spc, out);
}
