/*
 * polar_gb300.h - C ABI of the GB300 (sm_103a) Fast-SSC decoder for systematic
 * polar codes.
 *
 * Method: Giard, Sarkis, Leroux, Thibeault, Gross, "Low-Latency Software Polar
 * Decoders" (arXiv 1504.00353). The decoder walks the code's Fast-SSC tree
 * depth first (Sec. II-C/II-D): min-sum F (Eq. 1), G (Eq. 2) and G_0R, the XOR
 * Combine (Eq. 3) and Combine_0R, and the Rate-0, Rate-1 (Eq. 4),
 * Repetition and SPC constituent decoders, on float32 or saturating int8 LLRs.
 *
 * Conventions shared by every call:
 *  - natural bit order (Sec. II-A, G_N = F_2^{(x)log2 N}, no bit reversal);
 *  - frozen_mask[i] = 1 marks a frozen bit-channel, 0 an information one;
 *    the information set A is used in increasing index order;
 *  - BPSK maps bit 0 to +1, so an LLR >= 0 decides bit 0 (Eq. 4);
 *  - packed bits are LSB first: bit k is byte k/8, bit position k%8; the unused
 *    high bits of a row's last byte are written as 0;
 *  - LLR and bit arrays are frame-major: frame f of an [n][N] LLR array starts
 *    at element f*N, frame f of the output at byte f*ceil(K/8).
 *
 * Threading: a polar_code_t is immutable after creation (its per-device tables
 * are filled once, under a lock) and may be used from several host threads and
 * streams at once. Every decode call is asynchronous on the stream it is given.
 *
 * Errors: calls return polar_status. Argument and launch errors are reported
 * synchronously; a device-side wait that ran out of time is recorded in the
 * code's status word and reported by polar_code_check(). No call aborts the
 * process.
 */
#ifndef POLAR_GB300_H
#define POLAR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct polar_code polar_code_t;

/* A CUDA stream handle (the same type as cudaStream_t); NULL is the legacy
 * default stream. */
typedef struct CUstream_st *polar_stream_t;

typedef enum {
    POLAR_OK = 0,
    POLAR_EINVAL = -1,   /* bad N, K, mask, handle, size or configuration */
    POLAR_ENOMEM = -2,   /* host or device allocation failed */
    POLAR_ECUDA = -3,    /* a CUDA runtime call failed (no device, launch error) */
    POLAR_EALIGN = -4,   /* an LLR pointer is not 16-byte aligned */
    POLAR_ETIMEOUT = -5  /* a bounded device-side wait expired (see polar_code_check) */
} polar_status;

/* Text for a status code (static storage, never NULL). */
const char *polar_status_str(polar_status s);

/* Create a code handle for an (N, K) polar code (Sec. II-A: the N-K frozen
 * bit-channels are fixed to zero).
 *   N           power of two, 2 <= N <= 2^20.
 *   K           number of information bits; must equal the number of zeros
 *               in frozen_mask, 0 <= K <= N.
 *   frozen_mask host array of N bytes, 1 = frozen, 0 = information; copied.
 *   out         receives the handle; untouched on error.
 * The host builds the depth-first Fast-SSC operation list (Listing 1 is this
 * list for the (8,5) code of Fig. 2a) and the tables that pack the decoded
 * information bits. When a CUDA device is present the tables are also copied
 * to the current device; other devices are filled on their first decode.
 * Returns POLAR_EINVAL for a bad N, K or mask, POLAR_ENOMEM on allocation
 * failure, POLAR_ECUDA if the upload to a present device fails. */
polar_status polar_code_create(uint32_t N, uint32_t K, const uint8_t *frozen_mask,
                               polar_code_t **out);

/* As polar_code_create, with the largest Repetition and SPC node sizes the
 * decoder may use (Sec. II-D). A larger node of that type is split into its
 * two children instead. 0 disables the node type; UINT32_MAX (the default of
 * polar_code_create) leaves it unlimited. Setting max_spc = 0 gives the
 * node set of the paper's GPU decoder (Sec. V: SPC nodes not used). */
polar_status polar_code_create_ex(uint32_t N, uint32_t K, const uint8_t *frozen_mask,
                                  uint32_t max_rep, uint32_t max_spc,
                                  polar_code_t **out);

/* Release a handle and its device tables. Synchronises with nothing: the
 * caller must ensure no decode that uses the handle is still running.
 * NULL is accepted. */
void polar_code_destroy(polar_code_t *code);

/* N, K and the length of the operation list. Any pointer may be NULL. */
polar_status polar_code_info(const polar_code_t *code, uint32_t *N, uint32_t *K,
                             uint32_t *n_ops);

/* Copy the operation list (depth-first order, Listing 1) to host arrays of
 * `capacity` entries: kind[i] (0 F, 1 G, 2 G_0R, 3 Combine, 4 Combine_0R,
 * 5 Rate-0 fill of a right child, 6 Rate-1/Info, 7 Repetition, 8 SPC),
 * nv[i] = node size N_v, off[i] = index of the node's first leaf.
 * *n_ops receives the list length. POLAR_EINVAL if capacity is too small. */
polar_status polar_code_schedule(const polar_code_t *code, uint32_t *kind, uint32_t *nv,
                                 uint32_t *off, size_t capacity, size_t *n_ops);

/* Systematic encoding on the host (the paper decodes codewords but does not
 * describe the encoder; this is the two-step encoder x = ((d on A) G)|_A G).
 *   info_packed     host, n_frames rows of ceil(K/8) bytes, packed LSB first.
 *   codeword_packed host, n_frames rows of ceil(N/8) bytes, packed LSB first.
 * Returns POLAR_EINVAL if the frozen set is not one for which the two-step
 * encoder is systematic (x restricted to A must equal the data). */
polar_status polar_encode_systematic(const polar_code_t *code, const uint8_t *info_packed,
                                     uint8_t *codeword_packed, size_t n_frames);

/* Fast-SSC decode of n_frames frames of float32 channel LLRs (Sec. II-D).
 *   llr       device, [n_frames][N] float32, 16-byte aligned; read only.
 *   bits_out  device, [n_frames][ceil(K/8)] bytes: the estimated codeword
 *             restricted to A (= the information bits of a systematic code),
 *             packed LSB first.
 *   stream    CUDA stream; the call is asynchronous on it.
 * n_frames = 0 (or K = 0 with nothing to write) is a no-op returning POLAR_OK.
 * Arithmetic: F is an exact min and sign, G one IEEE binary32 add, the
 * Repetition sum folds t[i] + t[i+m] for m = N_v/2, ..., 1 (the order SC
 * uses), SPC flips the lowest index of least |LLR|; results are bit-exact
 * with a scalar CPU evaluation in that order. The decoder specialised to this
 * code runs when polar_code_compile built one for the decode's launch shape,
 * the operation-list interpreter otherwise; both give the same bits. Device
 * scratch, when the code needs it, is taken on `stream` from the library's
 * stream-ordered memory pool (freed blocks stay cached in it for later calls)
 * and returned on it.
 * Returns POLAR_EALIGN for a misaligned llr, POLAR_EINVAL for NULL pointers,
 * POLAR_ECUDA when no device is present or the launch fails. */
polar_status polar_decode(const polar_code_t *code, const float *llr, uint8_t *bits_out,
                          size_t n_frames, polar_stream_t stream);

/* As polar_decode for int8 LLRs in [-127, 127] (-128 must not occur). G and
 * the Repetition sums saturate to [-127, 127] (Sec. III-A: saturating adders;
 * Listing 4: saturating add then max(-127)). */
polar_status polar_decode_i8(const polar_code_t *code, const int8_t *llr,
                             uint8_t *bits_out, size_t n_frames, polar_stream_t stream);

/* As polar_decode (float32 LLRs), for callers that cannot allocate device
 * memory: code that runs where cudaMalloc / cudaMallocAsync are unavailable or
 * forbidden (inside a host callback, under an allocator that must not grow,
 * in a process whose memory budget is fixed up front). No device memory is
 * allocated and nothing is freed; the paper has no counterpart of this call.
 *   Scratch: the alpha stages that do not fit in shared memory go to one
 *   static device array of 32 MiB, which every GPU that loads this library
 *   holds until the process exits. The grid is reduced so that the resident
 *   CTAs' stages fit in it. A launch shape whose single CTA would need more
 *   than 32 MiB is rejected with POLAR_EINVAL; with N <= 2^20 one CTA needs
 *   at most 4 MiB, so every valid code runs. Nothing in the array needs to
 *   start at zero (every stage is written before it is read).
 *   Sharing: all calls on a device use the same array, so calls whose kernels
 *   overlap on the GPU (two streams, or two host threads) race on it; order
 *   them on one stream or synchronise between them.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture. The handle's device tables must already be on
 *   the current device (polar_code_create uploads them to the device current
 *   at creation); otherwise POLAR_EINVAL, since uploading would allocate.
 * Always runs the operation-list interpreter, with the handle's launch shape.
 * Results are identical to polar_decode's. */
polar_status polar_decode_noalloc(const polar_code_t *code, const float *llr,
                                  uint8_t *bits_out, size_t n_frames, polar_stream_t stream);

/* Number of float values one frame writes to a trace (the summed N_v/2 of
 * every F, G and G_0R operation). */
size_t polar_code_trace_len(const polar_code_t *code);

/* Decode frames held in host memory: n_frames frames of N LLRs (float32
 * with is_i8 = 0, int8 in [-127, 127] with is_i8 = 1) at host_llr, packed
 * information bits to host_bits ([n][ceil(K/8)] bytes). The frames are cut
 * into chunks of chunk_frames (0 = n_frames / 8) that move through six
 * internal streams, so copies in and out overlap decoding; the paper's latency
 * likewise counts the copies into and out of decoder memory (Sec. III). Pinned
 * host memory (cudaMallocHost) is needed for the overlap. The device buffers of
 * the chunks in flight belong to the library and are kept between calls (they
 * grow to the largest chunk seen and are held until exit); calls on one device
 * run one after another. Blocking: returns when host_bits is complete;
 * POLAR_ETIMEOUT as polar_code_check. */
polar_status polar_decode_host(const polar_code_t *code, int is_i8, const void *host_llr,
                               uint8_t *host_bits, size_t n_frames, size_t chunk_frames);

/* Test/debug decode that also records, for every frame and in list order, the
 * N_v/2 output LLRs of each F, G and G_0R operation into
 *   alpha_trace  device, [n_frames][polar_code_trace_len()] float32
 *                (int8 decodes store their integer values as floats).
 * llr is float32 when is_i8 = 0 and int8 when is_i8 = 1. Same kernel code
 * path as the plain decode, with the trace stores added. */
polar_status polar_decode_trace(const polar_code_t *code, const void *llr, int is_i8,
                                uint8_t *bits_out, float *alpha_trace, size_t n_frames,
                                polar_stream_t stream);

/* Launch shape for one LLR type (is_i8 = 0 float32, 1 int8). 0 in any field
 * restores the automatic choice for that field.
 *   threads          threads per frame: per CTA, since a CTA decodes one frame
 *                    at a time, unless several frames per CTA are set
 *                    (polar_code_set_frames_per_cta, threads = 32); multiple
 *                    of 32, <= 1024.
 *   smem_stage_max   largest alpha stage (node size) kept in shared memory;
 *                    power of two >= 64. Wider stages live in per-CTA device
 *                    scratch.
 *   warp_stage_max   operations on nodes of size <= this run on one warp
 *                    without CTA barriers; power of two >= 2.
 *   ctas_per_sm      resident CTAs per SM for the persistent grid.
 *   stage_channel    1: copy each frame's LLRs into shared memory with a bulk
 *                    async copy (double buffered), 2: read them from device
 *                    memory in place, 0: automatic.
 * Not thread-safe against concurrent decodes of the same handle. */
polar_status polar_code_set_launch(polar_code_t *code, int is_i8, uint32_t threads,
                                   uint32_t smem_stage_max, uint32_t warp_stage_max,
                                   uint32_t ctas_per_sm, uint32_t stage_channel);

/* Several frames per CTA, one per warp (frames = 2, 4 or 8; 0 or 1 = one
 * frame per CTA), for throughput shapes of one warp per frame (threads = 32):
 * the CTA's warps decode different frames side by side with the same
 * straight-line decoder, kept in step by CTA barriers so that they share the
 * instructions they fetch. Applies to the specialised decoder only: compile
 * after setting it (polar_code_compile); decodes whose shape has no such
 * decoder, batch-1 shapes and the interpreter keep one frame per CTA.
 * Not thread-safe against concurrent decodes of the same handle. */
polar_status polar_code_set_frames_per_cta(polar_code_t *code, int is_i8, uint32_t frames);

/* Frames per CTA a decode of n_frames frames would run with now (1 when the
 * several-frames form does not apply or has not been compiled). */
polar_status polar_code_get_frames_per_cta(const polar_code_t *code, int is_i8, size_t n_frames,
                                           uint32_t *frames);

/* The launch shape a decode of n_frames frames would use now (after the
 * automatic choices), written to the non-NULL pointers. threads is per CTA
 * (32 x frames per CTA in the several-frames form), smem_bytes the dynamic
 * shared memory per CTA, grid the number of CTAs, scratch_bytes the
 * device scratch the call allocates, unrolled the register-subtree size of the
 * specialised decoder that will run (0: the operation-list interpreter). */
polar_status polar_code_get_launch(const polar_code_t *code, int is_i8, size_t n_frames,
                                   uint32_t *threads, uint32_t *smem_stage_max,
                                   uint32_t *warp_stage_max, uint32_t *ctas_per_sm,
                                   uint32_t *stage_channel, uint32_t *grid,
                                   size_t *smem_bytes, size_t *scratch_bytes,
                                   uint32_t *unrolled);

/* Build a decoder specialised to this code (Sec. III-B "Unrolled Decoder":
 * the code's operation list written out with every node size and offset a
 * compile-time constant), compiled at run time with NVRTC for the current
 * device, for the launch shape a decode of n_frames frames of this LLR type
 * uses (is_i8 = 0 float32, 1 int8). Later decodes whose shape matches run it
 * instead of the operation-list interpreter; results are bit-identical.
 *   reg_subtree  subtrees of at most this many leaves (power of two, 32..1024;
 *                0 = 256) are decoded entirely in the registers of one warp.
 * n_frames = 0 releases every specialised decoder of that LLR type. A decoder
 * already compiled for the same launch shape is kept (release first to build
 * one with another reg_subtree).
 * Blocking; takes seconds for long codes. Call before any stream capture.
 * Returns POLAR_ECUDA if NVRTC is unavailable or compilation fails (see
 * polar_code_compile_log); decodes then keep using the interpreter. */
polar_status polar_code_compile(polar_code_t *code, int is_i8, size_t n_frames,
                                uint32_t reg_subtree);

/* polar_code_compile with a choice of form. flags = 0: the full form
 * (every operation inlined with constant sizes) for lists of at most 4096
 * operations, else the compact form. POLAR_COMPILE_OUTLINE_SUBTREES emits
 * one out-of-line function per distinct register subtree (equal frozen
 * patterns share code); POLAR_COMPILE_OUTLINE_MEMORY calls memory-resident
 * operations out of line with run-time sizes; POLAR_COMPILE_COMPACT is both
 * (N = 2^20 codes, 28,465 operations, compile in about a minute);
 * POLAR_COMPILE_FULL forces the full form. POLAR_COMPILE_LOCAL_LEAVES (combinable
 * with any of these) decodes every split node of 4 to 16 leaves inside a
 * register subtree with each thread of the warp holding the whole node,
 * without shuffles: fewer dependent steps, more instructions, so it suits
 * single-frame (latency) shapes. Results are the same bits. */
#define POLAR_COMPILE_OUTLINE_SUBTREES 1u
#define POLAR_COMPILE_OUTLINE_MEMORY 2u
#define POLAR_COMPILE_COMPACT 3u
#define POLAR_COMPILE_FULL 4u
#define POLAR_COMPILE_LOCAL_LEAVES 8u
polar_status polar_code_compile_ex(polar_code_t *code, int is_i8, size_t n_frames,
                                   uint32_t reg_subtree, uint32_t flags);

/* NVRTC log of the last polar_code_compile on this handle (never NULL; valid
 * until the next compile or destroy). */
const char *polar_code_compile_log(const polar_code_t *code);

/* ---- Mixed-code batches: one persistent launch over frames of several codes ---- */

typedef struct polar_batch polar_batch_t;

/* Build a decoder for frames that belong to any of n_codes codes (1..64),
 * all of one LLR type (is_i8 = 0 float32, 1 int8). One kernel is generated
 * and compiled with NVRTC holding the decoder specialised to each code
 * (Sec. III-B, "Unrolled Decoder"); its CTAs claim frames from a work queue
 * with an atomic counter, so frames of different lengths balance across the
 * GPU in a single launch.
 *   codes           handles created with the current device current; they
 *                   must outlive the batch decoder.
 *   threads         threads per CTA (multiple of 32; 0 = 32: one warp per
 *                   frame, the shape that measured fastest for int8).
 *   smem_stage_max  per code, the largest alpha stage kept in shared memory
 *                   (power of two; NULL or 0 entries = 512 for 32 threads,
 *                   2048 otherwise). Larger stages use device scratch.
 *   warp_stage_max  per code, the largest node handled by warp 0 alone: the
 *                   tree depth at which work switches from CTA-wide to
 *                   warp-level (power of two; NULL or 0 entries = 2048;
 *                   raised to 256, the register-resident subtree size).
 *   ctas_per_sm     cap on resident CTAs (frames) per SM, which also sets the
 *                   register budget of the kernel (0 = as many as shared
 *                   memory allows, at most 32).
 * Returns POLAR_EINVAL for bad arguments or codes not created with this
 * device current, POLAR_ECUDA if NVRTC is missing or compilation fails (log:
 * polar_batch_log(NULL)), POLAR_ENOMEM if an allocation fails.
 * The descriptor table, the work counter and the scratch of every resident
 * CTA are allocated here, so polar_batch_decode allocates nothing and can be
 * captured in a CUDA graph. Blocking (NVRTC compile). */
polar_status polar_batch_create(polar_code_t *const *codes, uint32_t n_codes, int is_i8,
                                uint32_t threads, const uint32_t *smem_stage_max,
                                const uint32_t *warp_stage_max, uint32_t ctas_per_sm,
                                polar_batch_t **out);

/* polar_batch_create with a choice of form: flags = 0 inlines every body (as
 * polar_batch_create); POLAR_COMPILE_OUTLINE_SUBTREES makes each distinct
 * register subtree one out-of-line function shared by all the codes' bodies
 * (equal frozen patterns of different codes share code), which makes the
 * kernel smaller. POLAR_BATCH_FRAME_PER_WARP with threads = 32 x F (F = 2..8)
 * decodes F frames per CTA, one per warp: the CTA claims F consecutive frames
 * of the list and its warps run the frames' code body side by side (when the
 * F frames are of several codes, each code's body in turn); warp thresholds
 * then do not apply (every operation is warp-level) and per-code stage caps
 * size one shared-memory slot per warp. Other flag bits give POLAR_EINVAL.
 * Same bits in every form. */
#define POLAR_BATCH_FRAME_PER_WARP 16u
polar_status polar_batch_create_ex(polar_code_t *const *codes, uint32_t n_codes, int is_i8,
                                   uint32_t threads, const uint32_t *smem_stage_max,
                                   const uint32_t *warp_stage_max, uint32_t ctas_per_sm,
                                   uint32_t flags, polar_batch_t **out);

void polar_batch_destroy(polar_batch_t *batch);

/* Decode n_frames frames in one launch on `stream`. All arrays are device
 * memory owned by the caller:
 *   code_id[i]  index (into the codes given at creation) of frame i's code;
 *   llr_off[i]  element offset of frame i's N LLRs in `llr` (16-byte aligned
 *               frame start: a multiple of 4 for float32, 16 for int8);
 *   out_off[i]  byte offset of frame i's ceil(K/8) output bytes in bits_out.
 * n_frames is at most 2^32 - 1 (POLAR_EINVAL above: the work counter is 32-bit).
 * Frames are claimed in index order, so listing the longest codes first gives
 * the best balance. The grid is min(resident CTAs, n_frames). Calls on one
 * batch decoder share its work counter and scratch: they must not overlap on
 * the GPU (issue them on one stream; the serving loop below has its own
 * workspace per launch). */
polar_status polar_batch_decode(polar_batch_t *batch, const uint32_t *code_id,
                                const uint64_t *llr_off, const uint64_t *out_off,
                                const void *llr, uint8_t *bits_out, size_t n_frames,
                                polar_stream_t stream);

/* Launch shape of the batch decoder (non-NULL pointers are written). */
polar_status polar_batch_info(const polar_batch_t *batch, uint32_t *threads, uint32_t *grid,
                              size_t *smem_bytes, size_t *scratch_bytes);

/* NVRTC log of the batch decoder's compilation (never NULL). With batch =
 * NULL: the log of the last polar_batch_create that failed on this thread. */
const char *polar_batch_log(const polar_batch_t *batch);

/* ---- Serving loop: continuous batching onto a batch decoder ---- */

typedef struct polar_server polar_server_t;

/* One decode request: frame of code `code_id` (index into the batch decoder's
 * codes) whose N channel LLRs (float32 or int8, the batch decoder's type) are
 * at byte offset llr_off of the host input buffer and whose ceil(K/8) output
 * bytes (information bits packed LSB first, as polar_decode) go to byte
 * offset out_off of the host output buffer. Requests that follow one another
 * and whose data are adjacent in the host buffers move in one copy. */
typedef struct polar_request {
    uint32_t code_id;
    uint32_t reserved;
    uint64_t llr_off;
    uint64_t out_off;
} polar_request;

/* Start a serving loop on the current device (the batch decoder's). There is
 * no counterpart in the paper, which decodes one frame or one batch per call;
 * this is the serving form of the same decoder.
 *   reqs, capacity   circular request array owned by the caller: request i
 *                    is reqs[i % capacity]; it is read after polar_server_
 *                    publish covers i and may be overwritten once request
 *                    i is complete.
 *   host_llr, host_out  caller-owned buffers with their sizes in bytes, in
 *                    pinned host memory (e.g. from cudaMallocHost; copies are
 *                    asynchronous) or in device memory of this GPU (copies
 *                    stay on the device); they must outlive the server.
 *   done_ns          caller-owned array of `capacity` entries: the loop
 *                    writes done_ns[i % capacity] = completion time of
 *                    request i (CLOCK_MONOTONIC nanoseconds) before
 *                    counting it complete.
 *   device_budget_bytes  device memory for requests in flight (LLR ring and
 *                    output ring; at least one frame of the longest code):
 *                    a request is admitted when it fits.
 *   max_frames       frames per launch (at most).
 *   slots            launches in flight at once (1..64), each with its own
 *                    stream, work counter and alpha scratch; device memory
 *                    beyond the budget: slots x (scratch for max_frames
 *                    frames + 20 bytes per frame).
 *   flags            0, or POLAR_SERVE_LAUNCH_PER_CODE: each admission is
 *                    decoded by one launch per code present (one after
 *                    another on the slot's stream) instead of one launch for
 *                    all; with slots = 1 this is a plain queue feeding
 *                    one-launch-per-code batches, the baseline the mixed,
 *                    overlapped form is measured against.
 * A host thread admits published requests as slots and ring space free up,
 * one launch of the batch decoder per admission (longest codes first), and
 * retires finished launches in admission order. */
#define POLAR_SERVE_LAUNCH_PER_CODE 1u
polar_status polar_server_create(polar_batch_t *batch, const polar_request *reqs, size_t capacity,
                                 const void *host_llr, size_t host_llr_bytes, uint8_t *host_out,
                                 size_t host_out_bytes, uint64_t *done_ns,
                                 size_t device_budget_bytes, uint32_t max_frames, uint32_t slots,
                                 uint32_t flags, polar_server_t **out);

/* Requests [0, n_published) have arrived (n_published never decreases).
 * POLAR_EINVAL if a new request names an unknown code or lies outside the
 * host buffers, or if n_published would overrun requests not yet complete
 * (more than `capacity` outstanding); nothing is published then. */
polar_status polar_server_publish(polar_server_t *server, uint64_t n_published);

/* Requests completed (all of [0, *n_completed) are), admissions and kernel
 * launches issued so far (NULL pointers are skipped). Returns the loop's
 * sticky error: POLAR_ECUDA after a failed CUDA call (the loop then admits
 * nothing more). */
polar_status polar_server_progress(const polar_server_t *server, uint64_t *n_completed,
                                   uint64_t *n_admissions, uint64_t *n_launches);

/* Finish every published request (unless the loop failed), stop the loop and
 * free the server. Returns the loop's error status. */
polar_status polar_server_destroy(polar_server_t *server);

/* ---- Communication chain on the GPU (frame / bit error rates) ---- */

/* Uniform random information bits: row f (ceil(K/8) bytes, device memory)
 * from Philox-4x32-10 (Salmon et al., SC 2011) with key `seed` and counter
 * (word, frame0 + f, stream 1); bits at and beyond K are 0. Asynchronous. */
polar_status polar_random_info(const polar_code_t *code, uint8_t *info_packed, size_t n_frames,
                               uint64_t seed, uint64_t frame0, polar_stream_t stream);

/* Systematic encoding on the device (same result as polar_encode_systematic):
 * info_packed [n][ceil(K/8)] -> codeword_packed [n][ceil(N/8)], device
 * memory. POLAR_EINVAL if the frozen set is not one the two-step encoder
 * handles (checked once per handle on the host). Asynchronous. */
polar_status polar_encode_systematic_device(const polar_code_t *code, const uint8_t *info_packed,
                                            uint8_t *codeword_packed, size_t n_frames,
                                            polar_stream_t stream);

/* BPSK (bit 0 -> +1) over AWGN at Eb/N0 = ebn0_db with rate K/N:
 * sigma^2 = 1 / (2 R 10^(Eb/N0 / 10)), LLR = 2 y / sigma^2 written as float32
 * [n][N] (is_i8 = 0) or int8 q = clamp(rint(8 LLR), -127, 127) (is_i8 = 1).
 * Normals are Box-Muller pairs of Philox-4x32-10 words (key `seed`, counter
 * (element / 4, frame0 + f, stream 2)). Device memory; asynchronous. */
polar_status polar_channel_awgn(const polar_code_t *code, const uint8_t *codeword_packed,
                                void *llr, int is_i8, size_t n_frames, float ebn0_db,
                                uint64_t seed, uint64_t frame0, polar_stream_t stream);

/* counters[0] += frames whose ceil(K/8)-byte rows of `decoded` and `sent`
 * differ, counters[1] += differing bits. Device memory; asynchronous. */
polar_status polar_count_errors(const polar_code_t *code, const uint8_t *decoded,
                                const uint8_t *sent, size_t n_frames,
                                unsigned long long *counters, polar_stream_t stream);

/* Frame and bit errors of the decoder over n_frames frames at ebn0_db, run in
 * batches of `batch` frames (0 = 16384) entirely on the current device:
 * random information bits, systematic encoding, the AWGN channel, the decoder
 * (the specialised decoder if one was compiled for the batch's shape) and the
 * error count. Synchronous; the paper has no GPU chain (its error-rate
 * figures come from a CPU simulation). */
polar_status polar_fer_run(const polar_code_t *code, int is_i8, float ebn0_db, uint64_t seed,
                           size_t n_frames, size_t batch, uint64_t *frame_errors,
                           uint64_t *bit_errors);

/* Self-test of the device-side failure path (the paper has no counterpart):
 * launches one CTA whose mbarrier wait is never completed; the wait gives up
 * after limit_us microseconds (1..1,000,000), as the channel-staging wait does
 * after 2 s, and sets the handle's status word, so that the next
 * polar_code_check returns POLAR_ETIMEOUT. Nothing faults and nothing hangs;
 * the context stays usable. Asynchronous on `stream`. */
polar_status polar_selftest_bounded_wait(polar_code_t *code, uint32_t limit_us,
                                         polar_stream_t stream);

/* Wait for `stream`, then read and clear the handle's device status word on
 * the current device. POLAR_ETIMEOUT if a bounded device wait expired since
 * the last check, POLAR_OK otherwise. */
polar_status polar_code_check(polar_code_t *code, polar_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* POLAR_GB300_H */
