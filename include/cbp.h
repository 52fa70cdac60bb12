/* libcbp: check-belief propagation (CBP) decoding of QC-LDPC codes on sm_103a.
 *
 * Method: W. Guan and L. Liang, "Check-Belief Propagation Decoding of LDPC Codes",
 * Sec. IV.  Each check-node keeps a check-belief Omega_c (Eq. s4e1); in the
 * sequential order of the check-nodes, every edge (c_i, v) runs
 *   B2V  R^new_{c_j->v} = psi^-(Omega_{c_j}, Q_{v->c*})            Eq. (s4e18)
 *   V2C  Q^new = Q + R^new - R_{c_i->v},  Lambda = Q + R^new        Eqs. (s4e19), (s4e20)
 *   C2B  Omega_{c_i} <- psi^+(Omega_{c_i}, Q^new)                    Eq. (s4e21)
 * where c_j is the check that updated v last (Step 2 a).  Hard decisions follow
 * Eq. (s2e7); decoding of a frame stops after the first full sweep whose hard
 * decisions satisfy every parity check (syndrome stop).
 *
 * Code model (Sec. II): a quasi-cyclic parity-check matrix given by a base matrix
 * B (mb x nb, row-major, -1 = zero block, s in [0, Z) = identity shifted by s) and
 * the lifting Z:  H[r*Z + i][c*Z + (i + s) % Z] = 1.  N = nb*Z variables, M = mb*Z
 * checks, checks visited in ascending index r*Z + i, the variables of a check in
 * ascending base column.
 *
 * Numerics.  All algorithms compute in FP32 with a fixed operation order (no
 * contraction into fused multiply-adds outside phi).  phi(x) = -log tanh(x/2)
 * (Eq. s2e5) is evaluated as phi(clamp(x, phi(30), 30)) by a cubic Taylor
 * expansion around the nearest point of a fixed grid (32 points per binade below
 * 2, step 1/16 from 2 to 30), coefficients from the closed-form derivatives of phi.
 * The check-belief is stored as S_c = sum of phi(|Q|) with its sign (Appendix A,
 * Eqs. ae2-ae5).  A variable seen for the first time adds no C2V message; the C2V
 * store of Eq. (s4e22) writes the predecessor's slot R_{c_j->v}.
 *
 * Threading and streams.  Every call is asynchronous on the stream it is given and
 * may run concurrently with other calls that use distinct output and workspace
 * buffers.  A code handle belongs to the device that was current at creation.
 *
 * Errors.  Functions return CBP_OK (0) or a negative cbp_status.  Arguments are
 * checked on the host before anything is launched; a failed check launches
 * nothing and leaves the outputs untouched.  Device data (LLR values) is not
 * inspected: LLRs must be finite.
 */
#ifndef CBP_H
#define CBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque decoder description of one QC code on one device; immutable after creation. */
typedef struct cbp_code cbp_code_t;

/* A CUDA stream (cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st* cbp_stream_t;

typedef enum cbp_status {
  CBP_OK = 0,
  CBP_EINVAL = -1,        /* bad argument: null/misaligned pointer, size, shift, option */
  CBP_ENOMEM = -2,        /* device allocation failed (only cbp_code_create allocates) */
  CBP_ECUDA = -3,         /* a CUDA runtime call or a kernel launch failed */
  CBP_EUNSUPPORTED = -4,  /* valid code/option this build cannot run (e.g. Z > 1024) */
  CBP_EWORKSPACE = -5,    /* workspace smaller than cbp_workspace_bytes() */
  CBP_EDEVICE = -6        /* handle used on a device other than the one it was made on */
} cbp_status;

/* Decoding algorithm.  All share the check order, the hard decision and the stop. */
typedef enum cbp_alg {
  CBP_ALG_CBP_SP = 0,   /* CBP, log-tanh form (Sec. IV-C, Steps 1-3) */
  CBP_ALG_CBP_NMS = 1,  /* CBP normalized min-sum, Eqs. (s4e18xx), (s4e21xx) */
  CBP_ALG_LBP_NMS = 2,  /* layered normalized min-sum, Eqs. (s2e10), (s2e12) (comparator) */
  CBP_ALG_FBP_SP = 3    /* flooding sum-product BP, Eqs. (s3e1), (s3e2), (s2e6) (comparator) */
} cbp_alg;

typedef enum cbp_stop {
  CBP_STOP_SYNDROME = 0, /* stop a frame after the first sweep with H x^T = 0 */
  CBP_STOP_NONE = 1,     /* always run max_iter sweeps */
  /* The paper's own rule, Step 2 (3) and Step 3 of Sec. IV-C (CBP_ALG_CBP_SP only): the
   * decoding of a frame succeeds once M consecutive check updates (in the sequential
   * order, counted across sweeps) each leave Omega_c > 0 (Eq. s4e2) and flip no sign of
   * the posterior of Eq. (s4e20) against that variable's previous posterior (initially
   * its channel LLR), Eq. (s4e24).  Decoding stops right after that update, possibly in
   * the middle of a sweep; hard_out is the sign of each variable's latest Eq. (s4e20)
   * posterior ("generated in the V2C phase"), iters the sweep in which the window
   * filled (negated if it never did within max_iter sweeps).  No soft output; Z <= 384
   * and base-row degree <= 32 (CBP_EUNSUPPORTED otherwise).  A variable of weight 1
   * sends its channel LLR to its check in every sweep, so a wrong channel sign there
   * keeps that check's Omega negative and the rule never fires. */
  CBP_STOP_WINDOW = 2
} cbp_stop;

/* Options of cbp_decode_ex.  Zero-initialise, then set what you need;
 * alpha <= 0 means the default 0.75. */
typedef struct cbp_opts {
  int alg;          /* cbp_alg */
  float alpha;      /* min-sum normalisation (CBP_NMS, LBP_NMS); ignored otherwise */
  int stop_mode;    /* cbp_stop */
  float* soft_out;  /* optional device buffer [batch][N] fp32: the posterior LLR
                       (CBP: Eq. s4e20 evaluated at the end of the last sweep run) */
} cbp_opts_t;

/* Build a code handle from a host base matrix (row-major mb x nb, int32, -1 = zero
 * block, otherwise a shift in [0, Z)).  Every base row needs >= 2 entries and every
 * base column >= 1 (CBP_EINVAL otherwise).  Z <= 1024, mb, nb <= 4096 and at most
 * 65535 base entries (CBP_EUNSUPPORTED otherwise).  Allocates the device tables on
 * the current device; *out is set only on success.  Release with cbp_code_destroy. */
int cbp_code_create(const int32_t* base, int mb, int nb, int Z, cbp_code_t** out);

/* Release a handle and its device tables (NULL is ignored).  The caller makes sure
 * no decode using it is still running. */
void cbp_code_destroy(cbp_code_t* code);

/* Sizes: n = N, m = M, k = N - rank(H) if known (-1 if not computed), edges = E.
 * Any output pointer may be NULL. */
int cbp_code_info(const cbp_code_t* code, int* n, int* m, int* k, int* edges);

/* Bytes of device workspace a decode of `batch` frames with `opts` (NULL = defaults)
 * needs.  The workspace holds the per-frame-slot C2V messages; it is scratch
 * memory, its contents need no initialisation and are undefined afterwards. */
int cbp_workspace_bytes(const cbp_code_t* code, int batch, const cbp_opts_t* opts,
                        size_t* bytes);

/* Decode `batch` frames with CBP (log-tanh form) and the syndrome stop.
 *   llr        device, [batch][N] fp32 channel LLRs ln Pr(y|0)/Pr(y|1), 16-byte aligned
 *   hard_out   device, [batch][ceil(N/32)] uint32: bit (v % 32) of word v / 32 is x_v
 *   iters_out  device, [batch] int32: sweeps run, negated if the syndrome is non-zero
 *              after max_iter sweeps
 *   max_iter   >= 1 sweeps at most;  batch >= 0 (0 launches nothing)
 *   workspace  device, >= cbp_workspace_bytes(), 256-byte aligned, caller-owned
 * Asynchronous on `stream`; the library allocates nothing. */
int cbp_decode(const cbp_code_t* code, const float* llr, uint32_t* hard_out,
               int32_t* iters_out, int max_iter, int batch, void* workspace,
               size_t workspace_bytes, cbp_stream_t stream);

/* cbp_decode with an algorithm, stop mode and optional soft output (opts may be NULL). */
int cbp_decode_ex(const cbp_code_t* code, const float* llr, uint32_t* hard_out,
                  int32_t* iters_out, int max_iter, int batch, void* workspace,
                  size_t workspace_bytes, cbp_stream_t stream, const cbp_opts_t* opts);

/* ---- Decoding from host memory, copies overlapped with decoding -------------------
 * The same decode as cbp_decode_ex, with the LLRs and the results in host memory.  The
 * batch is cut into chunks of `chunk` frames; while chunk i is decoded, chunk i + 1 is
 * copied in (and chunk i - 1's results out) on a copy stream.  Even chunks decode on
 * `stream`, odd ones on a second decode stream, each with its own workspace, so the next
 * chunk's CTAs start on the SMs that the current chunk's last frames leave idle.  The call
 * creates and releases both extra streams, ordered after the work already queued on
 * `stream`.  Two chunk buffers and two workspaces live in the caller's device memory
 * `dev_buf` of at least cbp_host_buffer_bytes(code, chunk, opts) bytes (256-byte
 * aligned); the library allocates no device memory.  The paper has no counterpart.
 *   llr_host    host [batch][N] fp32; hard_host [batch][ceil(N/32)] uint32;
 *   iters_host  host [batch] int32.  Page-locked (pinned) host memory is needed for the
 *               copies to overlap the decoding; other host memory works but serialises.
 *   chunk       frames per chunk, >= 1 (chunks of a few times the frame slots in flight
 *               keep the launch tails short)
 * opts->soft_out must be NULL (no soft output from this entry point).  Asynchronous on
 * `stream`: the host buffers must stay valid until `stream` has completed the work.
 * Errors as cbp_decode_ex, and CBP_EWORKSPACE if dev_buf is too small. */
int cbp_host_buffer_bytes(const cbp_code_t* code, int chunk, const cbp_opts_t* opts,
                          size_t* bytes);
int cbp_decode_host(const cbp_code_t* code, const float* llr_host, uint32_t* hard_host,
                    int32_t* iters_host, int max_iter, int batch, int chunk, void* dev_buf,
                    size_t dev_bytes, cbp_stream_t stream, const cbp_opts_t* opts);

/* The launch a decode of `batch` frames with `opts` would use (for tuning and reports):
 *   info[0] resident frames per SM      info[1] threads per CTA
 *   info[2] CTAs per SM                 info[3] lane groups per CTA
 *   info[4] frames per lane group       info[5] 1 if the check state is in shared memory
 *   info[6] CTAs launched               info[7] lane groups per synchronising team
 *   info[8] dynamic shared bytes per CTA
 *   info[9] 1 if the CBP-SP instance for codes whose weight-1 edges end their rows runs
 *   info[10] 1 if the frame-parallel CBP-SP kernel runs (one frame per thread; chosen when
 *            the lane-parallel plan would keep fewer than 128 lanes per SM busy, e.g. for
 *            Z = 1 codes, or cannot place a frame in shared memory)
 *   info[11] 1 if the wavefront-schedule CBP-SP kernel runs (the checks of each level of
 *            the expanded graph's dependency order on parallel lanes, one group per frame;
 *            chosen before the frame-parallel kernel where a frame's state fits in shared
 *            memory)
 * `info` is a host array of 12 ints.  Nothing is launched. */
int cbp_launch_info(const cbp_code_t* code, int batch, const cbp_opts_t* opts, int* info);

/* ---- Weighted CBP: the differentiable decoder --------------------------------------
 * The B2V message of Eq. (s4e18) from check c_j is scaled by weights[tau * mb + b], where
 * tau in [0, T) is the sweep (0-based) in which c_j formed its belief and b is c_j's base
 * row: R^new = sgn * (w * phi(|S_cj - phi(|Q*_v|)|)).  The decoder runs exactly T sweeps
 * (no stop) and outputs the flushed posterior after the last sweep (tau = T - 1).  With
 * every weight 1 the output equals cbp_decode_ex(CBP_ALG_CBP_SP, CBP_STOP_NONE, T sweeps).
 * The paper has no weights; they follow the usual unrolled-decoder construction.
 *
 * Bytes of device workspace cbp_decode_weighted / cbp_decode_grad need for `batch` frames,
 * T sweeps and a state checkpoint every `ckpt_every` sweeps.  With ckpt_every = T the
 * forward records the backward's tape of all T sweeps and keeps no checkpoint, so the
 * backward recomputes nothing (the fastest backward; the tape takes 12 bytes per edge and
 * sweep); with ckpt_every < T the backward recomputes each segment of ckpt_every sweeps
 * from its checkpoint. */
int cbp_grad_workspace_bytes(const cbp_code_t* code, int batch, int T, int ckpt_every,
                             size_t* bytes);

/* Forward: soft_out [batch][N] fp32 (device) = the weighted decoder's posterior LLRs.
 *   weights  device fp32 [T][mb];  T >= 1, 1 <= ckpt_every <= T;  Z <= 512
 *   workspace receives the checkpoints cbp_decode_grad needs: keep it unchanged between
 *   the two calls.  Asynchronous on `stream`; allocates nothing. */
int cbp_decode_weighted(const cbp_code_t* code, const float* llr, const float* weights, int T,
                        int ckpt_every, int batch, float* soft_out, void* workspace,
                        size_t workspace_bytes, cbp_stream_t stream);

/* Backward of cbp_decode_weighted (same code, llr, weights, T, ckpt_every, batch and the
 * workspace that forward call left): from grad_soft = dLoss/dsoft_out [batch][N], writes
 * grad_weights [T][mb] (summed over the frames) and, if not NULL, grad_llr [batch][N].
 * Reverse-mode through the sweeps in reverse order, each checkpoint segment recomputed
 * (none when ckpt_every = T);
 * phi is differentiated as the evaluated cubic, |x| and the clamps with derivative 0 at
 * their kinks, signs as constants.  Summation order of the gradients is not fixed
 * (atomic adds). */
int cbp_decode_grad(const cbp_code_t* code, const float* llr, const float* weights, int T,
                    int ckpt_every, int batch, const float* grad_soft, float* grad_weights,
                    float* grad_llr, void* workspace, size_t workspace_bytes,
                    cbp_stream_t stream);

/* Size of the decoder scratch array compiled into the library for cbp_decode_noalloc. */
#define CBP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* cbp_decode for callers that cannot allocate device memory.  (The paper has no
 * counterpart: this is a deployment convenience of the library.)
 *
 * Some callers cannot call cudaMalloc or hand over a workspace: code running where an
 * allocation could fail or block at the wrong moment (a real-time receive loop, a
 * plugin inside a host application that owns all device memory), or a caller that has
 * no allocator at all.  This entry point decodes exactly like cbp_decode (CBP log-tanh
 * form, syndrome stop) but keeps its scratch in a fixed array of
 * CBP_NOALLOC_SCRATCH_BYTES that is part of the library's device image; every GPU on
 * which the library's kernels are loaded holds that array until the process exits.
 * The caller still passes the inputs and outputs (same layout as cbp_decode); the call
 * allocates nothing.
 *   - It runs the lane-parallel CBP-SP kernel only (never the frame-parallel one that
 *     cbp_decode picks for codes such as Z = 1 graphs): a code whose frame does not fit
 *     that kernel's shared memory returns CBP_EUNSUPPORTED, and a small-Z code decodes
 *     correctly but with few busy lanes.
 *   - Larger batches run with fewer frame slots in flight, so they fit the array; a code
 *     whose single frame slot needs more than the array returns CBP_EWORKSPACE.
 *   - Errors: CBP_EINVAL (null or misaligned pointers, max_iter < 1, batch < 0),
 *     CBP_EDEVICE (a code of another device), CBP_EUNSUPPORTED, CBP_EWORKSPACE,
 *     CBP_ECUDA (the symbol lookup or the launch failed).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the one array and it keeps the previous call's contents (the
 *     decoder writes every scratch value before reading it, so nothing needs clearing).
 *     Calls whose executions overlap on the GPU — different streams, or different host
 *     threads without ordering — race on the array: serialise them. */
int cbp_decode_noalloc(const cbp_code_t* code, const float* llr, uint32_t* hard_out,
                       int32_t* iters_out, int max_iter, int batch, cbp_stream_t stream);

/* ---- Several codes in one launch (CBP log-tanh form, Sec. IV) -----------------------
 * A receiver that serves several QC-LDPC codes at once (different lifting sizes Z,
 * rates, batch sizes) decodes them all in one persistent launch.  Each item names a
 * code handle and its own device buffers (the layout of cbp_decode).  The frames of
 * every item are cut into chunks of whole lane-group rounds; the launch's CTAs take
 * chunks from a work counter until none is left, the heaviest items first, so a small
 * item rides along with a large one without a launch of its own.  The decoding of each
 * frame is bit-identical to cbp_decode_ex(CBP_ALG_CBP_SP) of the same frame with the
 * same stop mode.  The paper decodes one code at a time; this is a deployment feature.
 *
 * Items (at most CBP_MULTI_MAX_ITEMS, all codes on the current device):
 *   code       handle;  llr, hard_out, iters_out, batch: as for cbp_decode
 *              (batch 0 is allowed and decodes nothing for that item)
 * Options (NULL = defaults; zero-initialise then set):
 *   frames_per_group  1 or 2 frames interleaved per lane group (0 = 1)
 *   chk_shared        1: check beliefs in shared memory, 0: in the workspace, -1 or
 *                     any other value: the library picks (shared when every code fits)
 *   threads           threads per CTA, a multiple of 32 up to 768 (fpt 1) or 384
 *                     (fpt 2); every code's Z must be <= threads (0 = the maximum)
 *   ctas_per_sm       CTAs resident per SM the shared-memory split aims at (0 = 1)
 *   rounds_per_chunk  frame rounds of a CTA's lane groups per chunk (0 = 4)
 *   stop_mode         cbp_stop (0 = CBP_STOP_SYNDROME)
 *   tail_percent      the last tail_percent % of each item's frames (rounded up to whole
 *                     rounds) are decoded in chunks of one round after all other chunks,
 *                     so that the launch ends on short chunks; 1..100, 0 = 20, -1 = none
 * Work order: every item's main chunks, heaviest item first, then the items' tail chunks
 * in the same order.
 * The workspace holds a work counter (the call zeroes it with cudaMemsetAsync on
 * `stream` before the launch, so the call can be captured into a CUDA graph) and the
 * per-CTA decoder state.  Errors: CBP_EINVAL (bad pointers, alignment, options,
 * more than CBP_MULTI_MAX_ITEMS items), CBP_EDEVICE (a code of another device),
 * CBP_EUNSUPPORTED (a code that does not fit the CTA shape), CBP_EWORKSPACE. */
#define CBP_MULTI_MAX_ITEMS 8

typedef struct cbp_multi_item {
  const cbp_code_t* code;
  const float* llr;
  uint32_t* hard_out;
  int32_t* iters_out;
  int batch;
} cbp_multi_item_t;

typedef struct cbp_multi_opts {
  int frames_per_group;
  int chk_shared;
  int threads;
  int ctas_per_sm;
  int rounds_per_chunk;
  int stop_mode;
  int tail_percent;
} cbp_multi_opts_t;

/* Bytes of workspace cbp_decode_multi needs for these items and options. */
int cbp_multi_workspace_bytes(const cbp_multi_item_t* items, int n_items,
                              const cbp_multi_opts_t* opts, size_t* bytes);

/* The launch cbp_decode_multi would use: info[0] CTAs, info[1] threads per CTA,
 * info[2] dynamic shared bytes per CTA, info[3] CTAs resident per SM, info[4] chunks,
 * info[5] 1 if check beliefs are in shared memory, info[6] frames per lane group,
 * info[7] 1 if every code ends its rows with its weight-1 edge (the kernel instance without
 * weight-1 branches in its edge loop runs), else 0.  `info` is a host array of 8 ints. */
int cbp_multi_launch_info(const cbp_multi_item_t* items, int n_items,
                          const cbp_multi_opts_t* opts, int* info);

/* Decode every item's frames in one launch on `stream` (asynchronous; nothing is
 * allocated).  max_iter >= 1 sweeps at most for every frame. */
int cbp_decode_multi(const cbp_multi_item_t* items, int n_items, int max_iter,
                     void* workspace, size_t workspace_bytes, cbp_stream_t stream,
                     const cbp_multi_opts_t* opts);

/* Evaluate the library's phi (Eq. s2e5, the clamped FP32 form used by the decoders)
 * on n device values: y[i] = phi(x[i]).  x, y device, 4-byte aligned, n >= 0. */
int cbp_phi(const float* x, float* y, int64_t n, cbp_stream_t stream);

/* The derivative of that phi as the library evaluates it (the adjoint cbp_decode_grad
 * uses for Eq. s2e5): the derivative of the cubic of x's grid centre, 0 where the clamp
 * holds (x below fl32(phi(30)) or above 30).  Same arguments as cbp_phi. */
int cbp_phi_deriv(const float* x, float* y, int64_t n, cbp_stream_t stream);

/* Device status of a code handle.  Kernels never trap on bad input: they set a bit in
 * the handle's status word and carry on (the frame's results are then undefined).
 *   CBP_STATUS_NONFINITE_LLR  some decoded frame's channel LLRs held NaN or +-Inf
 * cbp_device_status reads and clears the word in one atomic step on `stream`, waits for
 * `stream`, and stores the flags in *flags (0 = no event since the last read).  It
 * reports every decode with this handle that completed before the read, on any stream. */
#define CBP_STATUS_NONFINITE_LLR 1u
int cbp_device_status(const cbp_code_t* code, cbp_stream_t stream, uint32_t* flags);

/* Measurement helper (no counterpart in the paper): the compute ceiling of the CBP-SP
 * edge update.  Launches `ctas` CTAs of 512 threads (ctas <= 0: every SM filled to its
 * occupancy limit) in which each thread runs `iters` rounds of 4 independent edge updates
 * of Sec. IV-C Step 2 -- B2V (Eqs. s4e18, s4e13) with phi, V2C (s4e20, s4e19), C2B
 * (s4e21) with phi and the check-belief fold -- on register-resident values, with the
 * decoders' phi (table in shared memory).  No other memory is touched, so the edge
 * updates per second it reaches bound the decoder's from above.  *edge_updates receives
 * the number of edge updates the launch performs; time it with events on `stream`.
 *   sink        device array of sink_floats floats, >= (CTAs launched) * 512 (written
 *               only in a case that does not occur; it keeps the work observable)
 *   ctas_used   optional: the number of CTAs launched
 * Asynchronous; errors: CBP_EINVAL (iters < 1, NULL pointers, sink too small), CBP_ECUDA. */
int cbp_edge_ceiling(int ctas, int iters, float* sink, size_t sink_floats, cbp_stream_t stream,
                     int64_t* edge_updates, int* ctas_used);

/* Static description of an error code. */
const char* cbp_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* CBP_H */
