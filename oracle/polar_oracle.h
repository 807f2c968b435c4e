/*
 * Plain CPU oracle for Fast-SSC decoding of systematic polar codes
 * (Giard et al., "Low-Latency Software Polar Decoders", arXiv 1504.00353).
 *
 * TEST INFRASTRUCTURE ONLY. This file and polar_oracle.c are the slow,
 * obviously-correct restatement of the method used to check the CUDA decoder.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it. It shares no code, header, table or helper with the
 * GPU library, and the GPU library never calls it.
 *
 * Conventions (all arrays are natural-index, Sec. II-A: G_N = F_2^{(x)n}):
 *   - bits are one byte per bit (0/1) unless a name says "packed";
 *   - packed bit k lives in byte k/8 at bit position k%8 (LSB first);
 *   - frozen[i] = 1 marks a frozen bit-channel, 0 an information one;
 *   - the information set A is taken in increasing index order.
 * Floating point follows IEEE-754 binary32 round-to-nearest: each F is an exact
 * min/sign, each G is one add. Build without -ffast-math/-Ofast and with
 * -ffp-contract=off so no step is reassociated or fused.
 */
#ifndef POLAR_ORACLE_H
#define POLAR_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Operation kinds recorded by the Fast-SSC trace (names of Sec. III and
 * Listing 1: F, G, G_0R, Combine, Combine_0R, Info = Rate-1, Repetition, SPC;
 * R0 is the explicit zero fill of a Rate-0 right child). */
enum {
    ORACLE_OP_F = 0,
    ORACLE_OP_G = 1,
    ORACLE_OP_G0R = 2,
    ORACLE_OP_C = 3,
    ORACLE_OP_C0R = 4,
    ORACLE_OP_R0 = 5,
    ORACLE_OP_R1 = 6,
    ORACLE_OP_REP = 7,
    ORACLE_OP_SPC = 8
};

/* Optional record of a Fast-SSC decode, in execution (depth-first) order.
 * For every operation: kind, node size N_v and node offset (first leaf index).
 * For F, G and G_0R the N_v/2 output LLRs are appended to `alpha`
 * (int8 decodes store their integer values as floats). */
typedef struct {
    uint32_t *kind, *nv, *off; /* capacity cap_ops each */
    float *alpha;              /* capacity cap_alpha */
    size_t cap_ops, cap_alpha;
    size_t n_ops, n_alpha;     /* filled by the decoder */
    int overflow;              /* set when a capacity was exceeded */
} oracle_trace;

/* x = u * F_2^{(x)n} over GF(2) (Sec. II-A). u, x: N bytes; may alias. */
void oracle_encode(uint32_t N, const uint8_t *u, uint8_t *x);

/* Systematic encoding: x restricted to A equals d (K bytes).
 * Two-step method (the paper only consumes codewords; see the design notes):
 * v = d on A, 0 on A^c; w = v*G; w[A^c] = 0; x = w*G.
 * Returns 0, or -1 if the mask's K differs or x[A] != d (mask not
 * domination-contiguous). */
int oracle_encode_systematic(uint32_t N, const uint8_t *frozen, const uint8_t *d,
                             uint8_t *x);

/* Plain recursive SC (Sec. II-C, Eqs. 1-3). xhat: N bytes (estimated x). */
int oracle_sc_decode_f32(uint32_t N, const uint8_t *frozen, const float *llr,
                         uint8_t *xhat);
int oracle_sc_decode_i8(uint32_t N, const uint8_t *frozen, const int8_t *llr,
                        uint8_t *xhat);

/* Plain recursive Fast-SSC (Sec. II-D): Rate-0, Rate-1 (Info, Eq. 4),
 * Repetition and SPC nodes; G_0R / Combine_0R under a Rate-0 left child.
 * max_rep / max_spc cap the node size for Repetition / SPC (0 disables the
 * node, UINT32_MAX leaves it unlimited). trace may be NULL. */
int oracle_fastssc_decode_f32(uint32_t N, const uint8_t *frozen, const float *llr,
                              uint32_t max_rep, uint32_t max_spc, uint8_t *xhat,
                              oracle_trace *trace);
int oracle_fastssc_decode_i8(uint32_t N, const uint8_t *frozen, const int8_t *llr,
                             uint32_t max_rep, uint32_t max_spc, uint8_t *xhat,
                             oracle_trace *trace);

/* Information bits of a codeword estimate: out bit k = xhat[A[k]], packed
 * LSB-first into ceil(K/8) bytes (unused high bits of the last byte are 0). */
void oracle_extract_info(uint32_t N, const uint8_t *frozen, const uint8_t *xhat,
                         uint8_t *info_packed);

/* Decode n frames one after another (frame f reads llr + f*N) and write the
 * packed information bits of frame f to out + f*ceil(K/8).
 * algo: 0 = Fast-SSC, 1 = SC. Returns 0 or a negative error. */
int oracle_decode_batch_f32(uint32_t N, const uint8_t *frozen, const float *llr,
                            size_t n_frames, int algo, uint32_t max_rep,
                            uint32_t max_spc, uint8_t *out);
int oracle_decode_batch_i8(uint32_t N, const uint8_t *frozen, const int8_t *llr,
                           size_t n_frames, int algo, uint32_t max_rep,
                           uint32_t max_spc, uint8_t *out);

/* Single-element operations, exposed for unit pins.
 * f: Eq. 1 (min-sum); g: Eq. 2; the int8 forms saturate to [-127, 127]
 * (Sec. III-A: only G grows the amplitude and uses saturating adders). */
/* Repetition-SPC node decoded speculatively (Sec. II-D): n LLRs of a node whose
 * left child is a Repetition code and right child an SPC code (n a power of
 * two, n >= 8) -> its n estimates. Returns 0, or -1 for a bad n. */
int oracle_repspc_f32(const float *alpha, uint32_t n, uint8_t *beta);
int oracle_repspc_i8(const int8_t *alpha, uint32_t n, uint8_t *beta);

float oracle_f_f32(float a, float b);
float oracle_g_f32(float a, float b, uint8_t beta_l);
int8_t oracle_f_i8(int8_t a, int8_t b);
int8_t oracle_g_i8(int8_t a, int8_t b, uint8_t beta_l);

#ifdef __cplusplus
}
#endif
#endif
