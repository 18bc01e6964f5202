/*
 * ifnso.h - C ABI of the GB300 (sm_103a) implementation of IFNSO,
 * Iteration-Free Newton-Schulz Orthogonalization (arXiv 2602.02500), and of
 * the Newton-Schulz iteration it is compared with.
 *
 * Conventions for every entry point
 *  - Matrices are row-major.  "Device pointer" means memory of the current
 *    CUDA device; "host pointer" means ordinary host memory.
 *  - Calls that take a cudaStream_t only enqueue work on that stream and
 *    return without synchronising, unless stated otherwise.  Host-detectable
 *    errors return a status at once and enqueue nothing; the message is
 *    available from ifnso_last_error() in the calling thread.
 *  - No C++ exception crosses this interface.  The caller owns every buffer
 *    it passes; a plan owns only its own metadata.
 *  - Conditions detected on the device (zero input, non-finite values,
 *    a pipeline wait that ran out of time) are recorded per matrix in the
 *    workspace and read back with ifnso_device_status().
 */
#ifndef IFNSO_H
#define IFNSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ifnso_stream_t; /* the same handle as cudaStream_t */

typedef enum {
  IFNSO_OK = 0,
  IFNSO_ERR_INVALID_ARG = 1,    /* a size, pointer, alignment or option is not accepted */
  IFNSO_ERR_UNSUPPORTED = 2,    /* a valid request this build does not implement */
  IFNSO_ERR_OOM = 3,            /* a host allocation of plan metadata failed */
  IFNSO_ERR_CUDA = 4,           /* a CUDA runtime/driver call failed (message has the CUDA error) */
  IFNSO_ERR_DEVICE_TIMEOUT = 5, /* a bounded device wait gave up (see ifnso_device_status) */
  IFNSO_ERR_WORKSPACE = 6       /* workspace missing, misaligned or smaller than required */
} ifnso_status;

typedef enum {
  IFNSO_F32 = 0,  /* FP32 storage and FP32 arithmetic (SIMT FP32 kernels) */
  IFNSO_BF16 = 1  /* BF16 storage, tensor-core products with FP32 accumulation */
} ifnso_dtype;

/* Options set with ifnso_plan_set(). */
typedef enum {
  /* Operand precision of the squaring chain and of the final product (BF16 plans).
   *   IFNSO_PREC_PLAIN: one FP16 operand per D_l, one BF16 operand for P.
   *   IFNSO_PREC_SPLIT: D_l = hi + lo (two FP16 parts, three products per
   *                     squaring), P = hi + lo (two BF16 parts, two products).
   *   IFNSO_PREC_MIXED: the first max(0, L - 8) squarings split, the last
   *                     ones plain (a rounding error of squaring l grows by up
   *                     to 2^(L - l) in the later squarings), P split.
   *   IFNSO_PREC_AUTO (default): PLAIN for L <= 4, MIXED for 5 <= L <= 14,
   *                     SPLIT for L >= 15. */
  IFNSO_OPT_PRECISION = 1,
  /* Input scaling.  IFNSO_SCALE_GRAM (default): X = A / ||A A^T||_F^(1/2)
   * (Eq. new_scale_formula, Sec. 2; o = ||T_0||_F in Algorithm 1).
   * IFNSO_SCALE_FROB: X = A / ||A||_F (Eq. constraint, Sec. 1).
   * IFNSO_SCALE_GELFAND2: X = A / ||(A A^T)^2||_F^(1/4), Gelfand's bound with
   * q = 2 (Eq. gelfand_formula, Eq. scale_formula_function), closer to the
   * largest singular value than q = 1; costs one extra product of D_1 with
   * itself (nothing stored) and a second prep.  Not with proposed
   * coefficients (IFNSO_ERR_UNSUPPORTED). */
  IFNSO_OPT_SCALE = 2,
  /* Upper bound on the CTAs of each persistent launch (0 = one per SM). */
  IFNSO_OPT_MAX_CTAS = 3,
  /* Testing aid: stop after this stage (0 = Gram only, 1 = Gram and the
   * D_1 / P initialisation, 2 + j = after squaring pass j+1).  -1 (default)
   * runs everything.  Intermediate buffers are read with ifnso_workspace_view(). */
  IFNSO_OPT_STOP_AFTER = 4,
  /* Measurement aid: when non-zero, every ifnso_orthogonalize / ns_iterate
   * call records a CUDA event on its stream before its first launch and after
   * each pass; ifnso_pass_times() returns the per-pass durations. */
  IFNSO_OPT_TIMING = 5,
  /* Limit, in milliseconds, of every pipeline wait inside the tensor-core
   * kernels (0, the default, means 4000).  A wait that runs out makes the CTA
   * record IFNSO_DEV_TIMEOUT for its matrix, let its copies and products
   * land, free its tensor memory and return. */
  IFNSO_OPT_WAIT_LIMIT_MS = 6,
  /* Testing aid for the failure path: when non-zero, the first CTA of the
   * Gram pass loads nothing, so that its waits run out (after the wait
   * limit) and the call reports IFNSO_DEV_TIMEOUT.  No memory is accessed out
   * of bounds and nothing is left running. */
  IFNSO_OPT_INJECT_STALL = 7,
  /* How the two CTAs of a cluster share the B operand of a pair of output
   * tiles in the tensor-core passes (the results agree bit for bit on every
   * case tested):
   * 1: each CTA issues its own M = 128 MMAs and loads the whole B tile into
   *    its own shared memory (the CTAs exchange nothing).
   * 2: MMAs of the CTA pair, M = 256 (tcgen05 cta_group::2); each CTA keeps
   *    its own half of B (a third fewer operand bytes per SM and product)
   *    and the odd CTA's copies complete on the even CTA's stage barrier.
   * 0 (default): the modes ifnso_plan_autotune chose, per pass kind; before
   *    any autotuning, 2 for the squarings with split operands, whose three
   *    products per stage hide the pair's handshakes, and 1 for every other
   *    pass (measured fastest on the 1B list). */
  IFNSO_OPT_CTA_GROUP = 8,
  /* Experiment on the first product (BF16 plans): when non-zero, T_0 = A A^T
   * is computed from an E4M3 copy of A s, s the power of two that maps
   * max |A_ij| into (224, 448] (rounded to nearest even, saturating), with
   * FP32 accumulation and T_0 = (A s)(A s)^T / s^2; the squarings and the
   * final product are unchanged.  E4M3 keeps 3 mantissa bits, so T_0 carries
   * a relative rounding error of about 2^-5 per input element.  The
   * workspace grows by h x round_up(w, 16) bytes per matrix.  0 (default):
   * the BF16 Gram. */
  IFNSO_OPT_GRAM_E4M3 = 9,
  /* Number of leading squarings that take split FP16 hi + lo operands in
   * IFNSO_PREC_MIXED (AUTO resolves to MIXED for 5 <= L <= 14): -1 (default)
   * means max(0, L - 8); n >= 0 means min(n, L - 1).  Fewer split squarings
   * are faster (a split squaring costs three products, a plain one one) and
   * less accurate: the rounding of D_l in a plain squaring l grows by up to
   * 2^(L - l) on small singular values.  Reading it back gives the number
   * the plan uses (L - 1 for SPLIT, 0 for PLAIN). */
  IFNSO_OPT_SPLIT_SQUARINGS = 10,
  /* Compute streams of ifnso_orthogonalize_host: 1 runs every group's
   * passes on the caller's stream; 2 (default) alternates the groups between
   * the caller's stream and a second stream of the plan, so that one
   * group's passes can start on the SMs another group's pass is leaving
   * (the groups share no buffers).  Either way the call is ordered after
   * earlier work on the caller's stream and later work waits for it. */
  IFNSO_OPT_HOST_STREAMS = 11,
  /* Shape bucket of matrices with h <= 128 (no counterpart in the paper's
   * code; Algorithm 1 is unchanged).  Such a matrix fits one 128 x 128
   * tensor-core tile, and one CTA can run the whole of Algorithm 1 on chip:
   * the Gram into tensor memory, D_l and P in shared and tensor memory
   * through all L - 1 squarings, then the product, in one launch for the
   * whole batch, where the tiled passes launch once per pass and pad h to
   * 256.  0 (default): the on-chip path when every matrix of a call has
   * h <= 128 and the call uses nothing it lacks (the proposal network inside
   * the call, IFNSO_SCALE_GELFAND2, IFNSO_OPT_GRAM_E4M3, ifnso_muon_step,
   * IFNSO_OPT_STOP_AFTER, IFNSO_OPT_INJECT_STALL), unless
   * ifnso_plan_autotune measured the tiled passes faster on such a batch;
   * 1: the on-chip path whenever it applies; 2: always the tiled passes.
   * With IFNSO_OPT_TIMING the on-chip path reports a single pass. */
  IFNSO_OPT_SMALL_MATRICES = 12,
  /* Read only (ifnso_plan_get): what ifnso_plan_autotune chose for batches
   * the on-chip path applies to: 0 not measured, 1 the on-chip path, 2 the
   * tiled passes. */
  IFNSO_OPT_SMALL_TUNED = 13,
  /* The MMA mode per pass kind that the tensor-core passes use when
   * IFNSO_OPT_CTA_GROUP is 0, packed two bits per kind (bits 0-1 the Gram,
   * 2-3 the split squarings, 4-5 the plain squarings, 6-7 the product; each
   * 1 or 2 as for IFNSO_OPT_CTA_GROUP).  Get: what ifnso_plan_autotune chose,
   * or 0 before it ran.  Set: those modes, e.g. another plan's choice on the
   * same batch; 0 returns to the untuned defaults.  ns_iterate runs its Gram,
   * its squaring S^2 and its product in the Gram's, the plain squarings' and
   * the product's modes. */
  IFNSO_OPT_CTA_GROUP_KINDS = 14,
  /* The final product Y = P A / sqrt(o) of MIXED-precision BF16 plans (AUTO
   * for 5 <= L <= 14), whose P is otherwise BF16 hi + lo (two products, P's
   * rounding below 2^-16 relative).  1 (default): one FP16 product of P (one
   * FP16 value) and an FP16 copy A s of the input (s a power of two from
   * ||A||_F that keeps every entry below 32768; written after the Gram, in
   * the workspace, which then grows by 2 bytes per input element; see
   * IFNSO_OPT_FP16_COPY_HOSTS for which kernels write it).  FP16
   * keeps 3 more mantissa bits than BF16, so P's rounding costs about 2^-11
   * times its largest entries.  0: BF16 hi + lo.  PLAIN plans keep their one
   * BF16 product of P and SPLIT plans (larger coefficients) hi + lo whatever
   * the value.  Set it before sizing the workspace; get returns whether the
   * plan uses it. */
  IFNSO_OPT_APPLY_F16 = 15,
  /* Read only: where the plan's last call wrote the FP16 copy of
   * IFNSO_OPT_APPLY_F16 (its last group, for ifnso_orthogonalize_host): the
   * number of squarings whose extra warps wrote it while they ran (the split
   * ones, or every squaring when fewer than three are split), or 0 when a
   * kernel of its own wrote it (batches too small to fill the GPU, or whose
   * squarings are too short to hide the copy) or no copy was needed. */
  IFNSO_OPT_FP16_COPY_HOSTS = 16,
  /* How many stages of its ring of operand buffers each kind of tensor-core
   * pass cycles through, packed 4 bits per kind (bits 0-3 the Gram, 4-7 the
   * split squarings, 8-11 the plain squarings, 12-15 the product, 16-19 the
   * final squaring, which reads P in its epilogue); 0 is the whole ring (up
   * to 6 stages, as many as shared memory holds), 2..15 a limit (a limit at or
   * above the ring's depth changes nothing).  A shallower ring leaves the
   * shared memory it does not allocate to the L1 cache and has fewer operand
   * bytes in flight, which can speed up a pass whose epilogue loads or stores
   * compete with them.  ifnso_plan_autotune chooses among the whole ring, 4
   * and 3 per kind (get returns its choice); set overrides it; the default is
   * 0.  Results do not depend on it. */
  IFNSO_OPT_STAGE_LIMITS = 17
} ifnso_option;

enum { IFNSO_PREC_AUTO = 0, IFNSO_PREC_PLAIN = 1, IFNSO_PREC_SPLIT = 2, IFNSO_PREC_MIXED = 3 };
enum { IFNSO_SCALE_GRAM = 0, IFNSO_SCALE_FROB = 1, IFNSO_SCALE_GELFAND2 = 2 };

/* Per-matrix device status bits (ifnso_device_status). */
enum {
  IFNSO_DEV_ZERO_INPUT = 1,   /* ||A A^T||_F = 0: the output is all zeros */
  IFNSO_DEV_NONFINITE = 2,    /* the norm scalar is not finite: the output is not meaningful */
  IFNSO_DEV_TIMEOUT = 4       /* a pipeline wait of a kernel ran out of time */
};

typedef struct ifnso_plan ifnso_plan;

/* A batch of independent matrices (one Muon step's gradient list, say).
 * Matrix i is rows[i] x cols[i], row-major with leading dimension ld[i]
 * elements, at device pointer in[i] (256-byte alignment recommended, 16 bytes
 * required; BF16: ld[i] a multiple of 8; F32: any ld >= cols).  The three
 * shape arrays and the pointer array are host arrays of `count` entries.
 * ld may be NULL (ld[i] = cols[i]).  A matrix with rows > cols is processed
 * as its transpose (Eq. 1, Sec. 1) and its result is returned in its own
 * shape. */
typedef struct {
  int32_t count;
  const void* const* in;
  const int64_t* rows;
  const int64_t* cols;
  const int64_t* ld;
} ifnso_batch_desc;

/* Coefficients of Y = sum_{l=0}^{L} w_l (I - X X^T)^{n_l} X over the plan's
 * exponents n = (0, 1, 2, 4, ..., 2^(L-1)) (Eq. generalized_matrix_formula and
 * the exponential selection of Sec. 2.2).  K = L + 1 slots; slot 0 is the
 * identity weight and is forced to 1 (y -> 1 as x -> 1, Eq. our_scalar_formula).
 * Exactly one of `host` (FP64, K values shared by every matrix), `device`
 * (FP32, count x K values, one row per matrix) and `mlp` is non-NULL.  With
 * `mlp` (a trained coefficient-proposal network with the same K; L >= 3; BF16
 * plans) the coefficients are proposed per matrix inside ifnso_orthogonalize
 * from the features the Gram and the first squaring produce, with the
 * network's fixed coefficients as the fallback.  The identity weight of the
 * equivalent D-basis form, 1 + sum w_l, is formed in FP64 on the device. */
typedef struct ifnso_mlp ifnso_mlp;

typedef struct {
  int32_t K;
  const double* host;
  const float* device;
  const ifnso_mlp* mlp;
} ifnso_coeffs;

/* ---------------------------------------------------------------------------
 * Plans
 * ------------------------------------------------------------------------- */

/* Create a plan for matrices whose oriented shape (h <= w after Eq. 1) is at
 * most h x w, stored as `dtype`.  `exponents` (host, K entries) must be
 * 0, 1, 2, 4, ..., 2^(K-2): the exponential term selection of Sec. 2.2, the
 * only exponents the repeated squaring of Sec. 2.4 produces; K >= 2, K <= 31.
 * On success *plan owns host metadata only (no device memory). */
ifnso_status ifnso_plan_create(ifnso_plan** plan, int64_t h, int64_t w, ifnso_dtype dtype,
                               const int32_t* exponents, int32_t K);

/* Set an ifnso_option; see the enum for values. */
ifnso_status ifnso_plan_set(ifnso_plan* plan, ifnso_option option, int64_t value);

/* Read back an option (after AUTO resolution for IFNSO_OPT_PRECISION). */
ifnso_status ifnso_plan_get(const ifnso_plan* plan, ifnso_option option, int64_t* value);

ifnso_status ifnso_plan_destroy(ifnso_plan* plan);

/* Bytes of device workspace ifnso_orthogonalize needs for this batch
 * (0 on error, with ifnso_last_error set).  Per matrix of oriented shape
 * h x w, with hp = h rounded up to 256: about 12 hp^2 bytes (SPLIT) or
 * 8 hp^2 (PLAIN) for BF16, 12 hp^2 for F32, plus metadata. */
size_t ifnso_workspace_bytes(const ifnso_plan* plan, const ifnso_batch_desc* batch);

/* ---------------------------------------------------------------------------
 * The hot path: Algorithm 1 (Sec. 2.4) for a whole batch
 * ------------------------------------------------------------------------- */

/* For every matrix M_i of the batch: A = M_i or M_i^T (h <= w); T_0 = A A^T;
 * o = ||T_0||_F; T_1 = I - T_0/o; T_l = T_{l-1}^2 (l = 2..L);
 * Y' = I + sum_l w_l T_l; Y = Y' A / sqrt(o) (Algorithm 1), computed in the
 * algebraically equal form D_1 = T_0/o, D_{l+1} = 2 D_l - D_l^2,
 * Y' = (1 + sum w_l) I - sum w_l D_l.  out[i] (device, rows[i] x cols[i],
 * row-major, leading dimension cols[i], 16-byte aligned, the input's dtype) receives Y in M_i's
 * shape; it must not overlap in[i] or the workspace.  `workspace` (device,
 * 1024-byte aligned, ifnso_workspace_bytes bytes) is scratch owned by the
 * caller; it must not be used by another call that runs concurrently.  The
 * call is asynchronous on `stream` and may be captured in a CUDA graph once
 * it has run outside capture with the same batch, outputs and workspace (the
 * first call uploads the launch metadata).  A workspace holds the metadata of
 * the plan that used it last: after another plan's call through it, this
 * plan's next call uploads its own again, but a graph captured before does
 * not, so a captured call needs a workspace no other plan uses. */
ifnso_status ifnso_orthogonalize(ifnso_plan* plan, const ifnso_batch_desc* batch,
                                 const ifnso_coeffs* coeffs, void* const* out,
                                 void* workspace, size_t workspace_bytes, ifnso_stream_t stream);

/* ifnso_orthogonalize (Algorithm 1, Sec. 2.4) for matrices held in host
 * memory; the copies and their overlap with the passes have no counterpart
 * in the paper.  host_in[i] holds matrix i in the layout dev_batch gives it
 * (rows[i] x cols[i], leading dimension ld[i], the plan's dtype); the call
 * copies it to dev_batch->in[i] (device memory the caller owns), runs every
 * pass, and copies the result from dev_out[i] (device, as `out` of
 * ifnso_orthogonalize) to host_out[i] (host, rows[i] x cols[i] contiguous).
 * The batch is cut into `groups` contiguous groups of about equal work (0
 * means 8; at most the batch count; F32 plans use one): the uploads run on a
 * copy stream of the plan, the downloads on another, and each group's passes
 * start as soon as its inputs have arrived, so the call costs about the
 * larger of the copies and the passes rather than their sum.  Host buffers
 * must be page-locked for the copies to overlap anything.  On hosts with
 * 64 KB base pages (Grace), buffers carved from one mapping backed by
 * transparent huge pages and registered once kept the copies at full speed,
 * where buffers page-locked one by one after another large process had
 * freed its memory intermittently copied at about a tenth of it.  Asynchronous:
 * everything the call does is ordered after earlier work on `stream` and
 * before later work on it; the host buffers must stay untouched until then.
 * Per-pass timing events (IFNSO_OPT_TIMING) and IFNSO_OPT_STOP_AFTER do not
 * apply.  Errors: IFNSO_ERR_INVALID_ARG for a NULL or misaligned pointer or
 * any argument ifnso_orthogonalize rejects; IFNSO_ERR_CUDA if a copy or a
 * launch fails (copies already queued then still run). */
/* Autotuning of the tensor-core launches for one batch (no counterpart in
 * the paper): runs ifnso_orthogonalize 1 + reps times with every pass forced
 * to per-CTA MMAs, and 1 + reps times forced to MMAs of the CTA pair
 * (IFNSO_OPT_CTA_GROUP 1 and 2), times every pass with CUDA events (the
 * first call of each set is not counted), and keeps in the plan, per pass
 * kind, the faster mode.  The kinds are the Gram, the split squarings, the
 * plain squarings and the final product.  Later calls with
 * IFNSO_OPT_CTA_GROUP = 0 (the default) use those modes.  `chosen` (host,
 * 4 entries, or NULL) receives them in that order.  In those modes it then
 * times the whole ring of operand stages, 4 and 3 stages for every pass
 * (1 + reps calls each) and keeps per kind, the final squaring counted
 * apart, the depth that is fastest by more than 2%
 * (IFNSO_OPT_STAGE_LIMITS).  When every matrix of the
 * batch has h <= 128 and the on-chip path applies to the call
 * (IFNSO_OPT_SMALL_MATRICES), it then also times that path (1 + reps calls)
 * against the tiled passes in their chosen modes and keeps the faster for
 * such batches (IFNSO_OPT_SMALL_TUNED).  Same arguments and rules as
 * ifnso_orthogonalize; `out` holds a valid result afterwards.  Synchronises
 * `stream`.  BF16 plans only (IFNSO_ERR_UNSUPPORTED otherwise); reps in
 * [1, 100]. */
ifnso_status ifnso_plan_autotune(ifnso_plan* plan, const ifnso_batch_desc* batch,
                                 const ifnso_coeffs* coeffs, void* const* out, void* workspace,
                                 size_t workspace_bytes, int32_t reps, int32_t* chosen,
                                 ifnso_stream_t stream);

ifnso_status ifnso_orthogonalize_host(ifnso_plan* plan, const void* const* host_in,
                                      const ifnso_batch_desc* dev_batch, const ifnso_coeffs* coeffs,
                                      void* const* dev_out, void* const* host_out, void* workspace,
                                      size_t workspace_bytes, int32_t groups, ifnso_stream_t stream);

/* One Muon step around the orthogonalization (the optimizer of Sec. 3.3;
 * the paper does not spell out its momentum, and this follows Muon's
 * published form).  For every matrix i of `grads` (BF16 gradients G, the
 * batch layout above):
 *   M <- beta M + G                          momentum[i]: FP32, rows x cols contiguous
 *   U <- G + beta M (nesterov = 1) or M      staging[i]: BF16, rows x cols, leading dimension ld[i]
 *   W <- W - lr sqrt(max(1, rows/cols)) Y    weights[i]: BF16, rows x cols contiguous
 * with Y the result of ifnso_orthogonalize on U (Algorithm 1, Sec. 2.4).
 * The update is fused into the final product's epilogue: Y is never
 * stored.  All four buffers are device memory owned by the caller, 16-byte
 * aligned and pairwise distinct; the workspace is ifnso_workspace_bytes of
 * `grads`.  beta in [0, 1), lr finite and >= 0, nesterov 0 or 1.  BF16
 * plans only (IFNSO_ERR_UNSUPPORTED otherwise).  Asynchronous on `stream`,
 * like ifnso_orthogonalize; capturable once it has run outside capture with
 * the same buffers. */
ifnso_status ifnso_muon_step(ifnso_plan* plan, const ifnso_batch_desc* grads, void* const* momentum,
                             void* const* staging, void* const* weights, const ifnso_coeffs* coeffs, double beta,
                             int32_t nesterov, double lr, void* workspace, size_t workspace_bytes,
                             ifnso_stream_t stream);

/* The comparison baseline, Newton-Schulz: X_0 = A/||A||_F (Eq. constraint),
 * then `steps` times X <- sum_n poly[n] (X X^T)^n X (Eq. general_eq_matrix):
 * degree 3 takes poly = (a, b) (the classical iteration is (1.5, -0.5),
 * Eq. one_iteration_matrix); degree 5 takes poly = (a, b, c) (Muon:
 * (3.4445, -4.7750, 2.0315), Eq. iteration_jordan).  Every product runs on
 * tensor cores for BF16 plans (BF16 storage of X, X X^T and the polynomial
 * in X X^T, FP32 accumulation) and in FP32 for F32 plans.  The plan's
 * exponents are ignored.  Same batch, output and stream rules as
 * ifnso_orthogonalize; workspace size from ns_workspace_bytes. */
ifnso_status ns_iterate(ifnso_plan* plan, const ifnso_batch_desc* batch, const double* poly,
                        int32_t degree, int32_t steps, void* const* out, void* workspace,
                        size_t workspace_bytes, ifnso_stream_t stream);

size_t ns_workspace_bytes(const ifnso_plan* plan, const ifnso_batch_desc* batch);

/* Synchronise `stream`, then copy the per-matrix device status words of the
 * last call that used `workspace` into per_matrix[0..count) (host), and the
 * per-matrix FP64 scalars into o_out / trace_out (host, count entries each,
 * either may be NULL): o = ||T_0||_F (or ||A||_F^2 under IFNSO_SCALE_FROB and
 * for ns_iterate) and tr(T_0) = ||A||_F^2.  Returns IFNSO_ERR_DEVICE_TIMEOUT
 * if any matrix has IFNSO_DEV_TIMEOUT set. */
ifnso_status ifnso_device_status(const ifnso_plan* plan, const void* workspace, int32_t count,
                                 int32_t* per_matrix, double* o_out, double* trace_out,
                                 ifnso_stream_t stream);

/* Per-pass durations (milliseconds, summed over every call made since the
 * last query with IFNSO_OPT_TIMING on) into ms_out[0..max_passes) (host);
 * *n_passes (host) receives the number of passes of the last call and
 * *n_calls (host, may be NULL) the number of calls summed.  Waits for the
 * recorded events.  A call captured into a CUDA graph counts once per query,
 * with the durations of the graph's latest replay (none before its first);
 * only the most recent capture is followed.  Pass order of
 * ifnso_orthogonalize: 0 Gram (with the
 * per-matrix scalars), 1 D_1 / P initialisation, 2 .. L squarings l = 1..L-1,
 * L + 1 the final product.  ns_iterate: 0 norm and scalars, then per step
 * Gram, squaring (degree 5 only), product. */
ifnso_status ifnso_pass_times(ifnso_plan* plan, double* ms_out, int32_t max_passes,
                              int32_t* n_passes, int32_t* n_calls);

/* Measurement aid (no counterpart in the paper): the timeline of the last
 * eager ifnso_orthogonalize_host call on a plan with IFNSO_OPT_TIMING on.
 * Waits for that call, then writes, for each of its *n_groups groups (at most
 * max_groups are written), three times in milliseconds since the call's
 * start into ms_out (host, 3 * max_groups entries): the group's uploads done,
 * its passes done, its downloads done.  group_first (host, may be NULL,
 * max_groups + 1 entries) receives the first matrix of each group and then
 * the matrix count.  *n_groups is 0 if no such call was made (or it was
 * captured into a graph). */
ifnso_status ifnso_host_timeline(ifnso_plan* plan, double* ms_out, int32_t max_groups, int32_t* n_groups,
                                 int32_t* group_first);

/* Testing aid: device pointer and leading dimension (elements) of an h_pad x
 * h_pad intermediate of matrix `index` in a workspace used by
 * ifnso_orthogonalize.  which: 0 = T_0 then P (FP32), 1/2 = D buffer 0 hi/lo
 * (FP16, or FP32 for F32 plans), 3/4 = D buffer 1 hi/lo, 5 = the FP32
 * coefficient row (c_0, w_1..w_L) the proposal network chose for the matrix
 * (ld = 32), 6 = the matrix's 64-byte record of FP64 scalars (ld = 8): [0]
 * ||T_0||_F^2, [1] tr(T_0), [2] the squared input scale, [3] the D-basis
 * identity weight 1 + sum w_l, [4] two FP32 reciprocals and two 32-bit words
 * (status bits, max |A_ij|), [6] ||D_1^2||_F^2 = tr(D_1^4) when the proposal
 * network ran (its third feature), [7] 1.0 where that network's fallback head
 * chose the fixed coefficients, else 0.0; 7 = the FP16 copy A s of
 * IFNSO_OPT_APPLY_F16 (M's shape, ld = its row pitch).  With that option, D
 * buffer hi of the final parity holds P as one FP16 value after the last
 * squaring.  BF16 plans keep these symmetric matrices on their 256 x 256
 * blocks on and above the diagonal only: element (i, j) with
 * i / 256 > j / 256 is the one at (j, i); the memory below is unspecified. */
ifnso_status ifnso_workspace_view(const ifnso_plan* plan, const ifnso_batch_desc* batch,
                                  void* workspace, int32_t index, int32_t which, void** ptr,
                                  int64_t* ld);

/* ---------------------------------------------------------------------------
 * Split-K Frobenius norm
 * ------------------------------------------------------------------------- */

/* norm2_out[i] (device, FP64, count entries) = ||M_i||_F^2, reduced as FP32
 * partial sums of squares per CTA and an FP64 final accumulation (the scaling
 * of Eq. constraint, Sec. 1).  dtype is that of the matrices.  The matrices'
 * descriptions go through a device buffer that the library allocates per
 * device on first use and grows; before overwriting it a call waits (on the
 * host) until the previous call's kernel on that device has read it, so
 * calls from several streams or threads are safe.  Otherwise asynchronous. */
ifnso_status ifnso_frobenius_norm2(const ifnso_batch_desc* batch, ifnso_dtype dtype,
                                   double* norm2_out, ifnso_stream_t stream);

/* Same result as ifnso_frobenius_norm2, without allocating device memory.
 * The paper has no counterpart: this exists for callers that cannot let a
 * library call cudaMalloc -- hosts that own all device memory through their
 * own pool (a framework's caching allocator, a serving process's arena) and
 * must not have memory taken or an out-of-memory raised behind their back,
 * and latency-critical callers that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree.  (ifnso_frobenius_norm2 allocates
 * its descriptor buffer on first use and grows it.)  The per-matrix
 * descriptors go to a fixed array compiled into the library (about 120 KB,
 * held on every GPU that loads the library until the process exits), so at
 * most IFNSO_STATIC_NORM_MAX_MATRICES matrices per call; a larger batch is
 * rejected with IFNSO_ERR_INVALID_ARG before anything is enqueued.  The
 * caller passes the inputs and norm2_out (device, FP64, count entries), which
 * the call zeroes before accumulating.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call
 * uploads its descriptors from pageable host memory.  Every call shares
 * the array and it keeps the last call's descriptors: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Asynchronous on `stream`. */
#define IFNSO_STATIC_NORM_MAX_MATRICES 1024
ifnso_status ifnso_frobenius_norm2_static(const ifnso_batch_desc* batch, ifnso_dtype dtype,
                                          double* norm2_out, ifnso_stream_t stream);

/* ---------------------------------------------------------------------------
 * Coefficient learning (Algorithm 1, "Coefficient learning"; Sec. 2.3, 3.1.1)
 * ------------------------------------------------------------------------- */

/* Learn w_1..w_{L-1} on the GPU in FP64 by minimising sum_j (f(x_j) - 1)^2
 * with f of Eq. overall_polynomial (w_L from Eq. b_approximation), using Adam
 * (moments from zero, bias corrections by running products of the betas 0.9
 * and 0.999, eps 1e-8) with learning rate lr * gamma^floor(t / step_size) at
 * iteration t, for `iters` iterations of `samples` points of (0, 1) each.
 * Sample j of iteration t is the FP64 uniform built from Philox4x32-10 words
 * 0 and 1 at counter (j, t, 0, 0), key (seed, 0x4C45524E):
 * ((w0 >> 5) 2^26 + (w1 >> 6) + 0.5) 2^-53.  Writes w_1..w_L to w_out (host,
 * L doubles).  Synchronous.  1 <= L <= 30, 1 <= samples <= 4096. */
ifnso_status ifnso_learn_coefficients(int32_t L, int32_t iters, int32_t samples, double lr,
                                      int32_t step_size, double gamma, uint32_t seed,
                                      double* w_out);

/* ---------------------------------------------------------------------------
 * Coefficient proposal: per-matrix coefficients from spectral features (the
 * paper's future work on dynamic coefficients, Sec. 4).
 *
 * Network (FP32): z = standardised [log tr(D)/h, log tr(D^2)/h, log tr(D^4)/h,
 * log h, log w, log ||A||_F] (D = A A^T / ||A A^T||_F) -> 64 GELU -> 64 GELU
 * -> K + 1 outputs.  Outputs 1..L: w_l = wfix_l + s_l out_l with
 * s_l = max(1, |wfix_l|)/10; output 0 (the identity weight) is projected onto
 * p(1) = 1; output K predicts log E(proposal) - log E(wfix), and the fixed
 * coefficients wfix are used whenever it is > 0.  E(c) = (1/h) sum_i
 * (f_c(x_i) - 1)^2 is the squared distance of Algorithm 1's output to the
 * polar factor U V^T (per h), exact from the singular values x_i of
 * X = A / ||A A^T||_F^(1/2).  Parameters: flat FP32 array W1 (64 x 6,
 * row-major) | b1 (64) | W2 (64 x 64) | b2 (64) | W3 ((K+1) x 64) | b3 (K+1).
 * The object owns its device memory (parameters, Adam moments, data).
 * ------------------------------------------------------------------------- */

/* Number of FP32 parameters for K = L + 1 coefficient slots. */
int32_t ifnso_mlp_param_count(int32_t K);

/* Create a network with K slots (3 <= K <= 31) around the fixed coefficients
 * wfix (host, K - 1 doubles w_1..w_L).  params (host, ifnso_mlp_param_count
 * floats) or NULL for a Philox-seeded Gaussian initialisation. */
ifnso_status ifnso_mlp_create(ifnso_mlp** mlp, int32_t K, const double* wfix, const float* params,
                              uint32_t seed);
ifnso_status ifnso_mlp_destroy(ifnso_mlp* mlp);

/* Copy parameters (host, param_count floats) and/or the 12 standardisation
 * constants (host: 6 means then 6 standard deviations) out of / into the
 * network; either pointer may be NULL.  Synchronous. */
ifnso_status ifnso_mlp_get_params(const ifnso_mlp* mlp, float* params, float* stats);
ifnso_status ifnso_mlp_set_params(ifnso_mlp* mlp, const float* params, const float* stats);

/* Attach a data set of n matrices given by their singular values: sigma
 * (device, FP32, concatenated), offsets (device, n + 1 int64: matrix i owns
 * sigma[offsets[i] .. offsets[i+1])), h and w (device int32, n each).  The
 * features are computed on the device; with fit_standardisation the
 * standardisation constants are refitted on this set.  Replaces the previous
 * data set.  Asynchronous on `stream`. */
ifnso_status ifnso_mlp_set_data(ifnso_mlp* mlp, int32_t n, const float* sigma, const int64_t* offsets,
                                const int32_t* h, const int32_t* w, int32_t fit_standardisation,
                                ifnso_stream_t stream);

/* Mean loss over the samples idx[0..batch) (device int32) of the data set,
 * and its gradient (device, param_count floats), by the forward and backward
 * kernels.  loss (device, 1 float).  Asynchronous. */
ifnso_status ifnso_mlp_loss_grad(ifnso_mlp* mlp, const int32_t* idx, int32_t batch, float* grad, float* loss,
                                 ifnso_stream_t stream);

/* `steps` Adam steps (moments from zero at creation, betas 0.9 / 0.999,
 * eps 1e-8) of learning rate lr on batches of `batch` samples drawn with
 * replacement (Philox4x32-10 word 0 of counter (j, step), key (seed,
 * 0x4D4C5042), modulo n).  loss_curve (device, steps floats) or NULL.
 * Asynchronous. */
ifnso_status ifnso_mlp_train(ifnso_mlp* mlp, int32_t steps, int32_t batch, float lr, uint32_t seed,
                             float* loss_curve, ifnso_stream_t stream);

/* For samples idx[0..n) (device; NULL = 0..n-1): E of the coefficients the
 * network proposes after the fallback rule (e_mlp), E of the fixed
 * coefficients (e_fix), the coefficient rows (coeffs, n x K, may be NULL)
 * and the fallback flags (fallback, may be NULL); all device arrays.
 * Asynchronous. */
ifnso_status ifnso_mlp_evaluate(const ifnso_mlp* mlp, const int32_t* idx, int32_t n, float* e_mlp,
                                float* e_fix, float* coeffs, int32_t* fallback, ifnso_stream_t stream);

/* ---------------------------------------------------------------------------
 * Synthetic inputs (benchmark and test data; not part of the method)
 * ------------------------------------------------------------------------- */

/* Fill out (device, BF16, rows x cols, leading dimension ld) with the
 * rank-32 signal plus noise matrix of seed `seed`: element (i, j) is
 * fl(fl(fl(alpha * S_ij) + N_ij) * beta) rounded to nearest even BF16, where
 * S = L R^T with L_ir / R_jr the byte sums of Philox4x32-10 word 0 at counter
 * (i, r, 0, 0) / (j, r, 0, 0), keys (seed, 0x4C524B31) / (seed, 0x4C524B32),
 * minus 510, and N_ij = the four 16-bit halves of words 0 and 1 at counter
 * (j, i, 0, 0), key (seed, 0x4E4F4953), summed, minus 131070.  Asynchronous. */
ifnso_status ifnso_synth_lowrank_bf16(void* out, int64_t rows, int64_t cols, int64_t ld,
                                      uint32_t seed, float alpha, float beta,
                                      ifnso_stream_t stream);

/* ---------------------------------------------------------------------------
 * Errors and build information
 * ------------------------------------------------------------------------- */

/* Message of the last error in the calling thread ("" if none). */
const char* ifnso_last_error(void);

/* Number of kernel launches enqueued by this library since the process
 * started (counting every launch of every entry point). */
uint64_t ifnso_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* IFNSO_H */
