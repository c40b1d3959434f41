/*
 * qtp.h - C ABI of libqtp, the GB300 (sm_103a) fast T-product of third-order
 * quaternion tensors.
 *
 * Method: Zheng & Ni, "Block diagonalization of block circulant quaternion
 * matrices and the fast calculation for T-product of quaternion tensors"
 * (arXiv 2212.14318), Algorithm 5.1 with Theorem 5.1.  For A in Q^{m x n x p}
 * and B in Q^{n x s x p} the library returns C = A * B in Q^{m x s x p}, the
 * T-product of Definition 2.3, C = fold(bcirc(A) . unfold(B)).
 *
 * ------------------------------------------------------------------------
 * Data layout ("tube-contiguous complex-pair planes")
 * ------------------------------------------------------------------------
 * A quaternion q = a + b i + c j + d k is stored by its Cayley-Dickson halves
 * q = q1 + q2 j with q1 = a + b i, q2 = c + d i (Sec. 2.2).  A tensor
 * X in Q^{R x K x p} is ONE buffer of 2*R*K*p complex FP32 numbers, each
 * complex number two consecutive floats (real, imag):
 *
 *     X[plane][r][k][t]  at float offset  2 * (((plane*R + r)*K + k)*p + t)
 *
 * plane 0 holds X1 = (a, b), plane 1 holds X2 = (c, d); t is the index along
 * the third mode (frontal slice), so every tube X(r, k, :) is contiguous.
 * Every tensor pointer must be 16-byte aligned.
 *
 * ------------------------------------------------------------------------
 * Ownership, streams, errors
 * ------------------------------------------------------------------------
 * - The caller owns every tensor and the workspace; all of them are device
 *   memory unless the entry point's name ends in _host.  The plan owns only
 *   its twiddle tables, its device error word and tuned parameters.
 * - Everything after plan creation is asynchronous on the caller's stream
 *   (a cudaStream_t passed as void*; NULL = legacy default stream).  Only
 *   qtp_plan_create / qtp_plan_destroy allocate, free or synchronise.
 * - Every call returns a qtp_status and never throws.  Invalid shapes, null
 *   or misaligned pointers, an unsupported precision and an undersized
 *   workspace are rejected on the host before any launch.  A failed launch
 *   maps to QTP_ERR_CUDA.  Kernels that wait on a barrier give up after a
 *   bounded time (2 s), record it in the plan's error word and return;
 *   qtp_plan_sync reports that as QTP_ERR_TIMEOUT.  For tests of that path
 *   the environment variables QTP_INJECT_WITHHOLD=<k> and
 *   QTP_INJECT_WAIT_NS=<ns>, read at every tensor-core launch, make the
 *   products' operand producer skip K step k (its operands never arrive) and
 *   bound every wait by ns nanoseconds: the waits expire, the kernels unwind
 *   and the next sync returns QTP_ERR_TIMEOUT.  Unset, they change nothing.
 * - qtp_last_error() returns a thread-local message for the last failure.
 */
#ifndef QTP_H_
#define QTP_H_

#include <stddef.h>

#if defined(__GNUC__)
#define QTP_API __attribute__((visibility("default")))
#else
#define QTP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QTP_OK = 0,
  QTP_ERR_INVALID_ARG = 1,  /* bad shape, null or misaligned pointer       */
  QTP_ERR_UNSUPPORTED = 2,  /* precision or size the library does not do */
  QTP_ERR_WORKSPACE = 3,    /* workspace missing or smaller than required */
  QTP_ERR_CUDA = 4,         /* a CUDA runtime/driver call failed          */
  QTP_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up         */
  QTP_ERR_INTERNAL = 6,
  QTP_ERR_NOT_CONVERGED = 7 /* an iteration stopped at its limit (T-SVD)  */
} qtp_status;

/* Arithmetic of the per-frequency products (Alg. 5.1 Step 2).  The tube FFTs
 * (Steps 1 and 3) always run in FP32.
 *   QTP_PREC_FP32   : FP32 FMA on CUDA cores ("plain FP32 path").
 *   QTP_PREC_BF16X3 : each FP32 operand x is split x = hi + lo with
 *                     hi = bf16(x), lo = bf16(x - hi); the products
 *                     hi*hi + hi*lo + lo*hi run on the tcgen05 tensor cores
 *                     with FP32 accumulation (relative error 4e-6 to 7e-6 on
 *                     N(0,1) data, at most 1e-5, for every reduction length:
 *                     long reductions fold their tensor-core partial sums
 *                     into FP32 at least every 512 terms).
 *   QTP_PREC_BF16   : hi*hi only (relative error ~1e-3; comparison only). */
typedef enum { QTP_PREC_FP32 = 0, QTP_PREC_BF16X3 = 1, QTP_PREC_BF16 = 2 } qtp_precision;

typedef struct qtp_plan qtp_plan;

/* Plan flags. */
#define QTP_PLAN_AUTOTUNE 1u  /* time the tensor-core tile shapes for this shape at plan creation */

/* Create a plan for C = A * B with A in Q^{m x n x p}, B in Q^{n x s x p}.
 * Requires 1 <= m, n, s <= 2^20, 1 <= p <= 4096 and m*n*p, n*s*p, m*s*p
 * each below 2^31 complex entries per plane.  Allocates the twiddle table
 * w^e = exp(-2 pi i e / p), e in [0, p) (eq. DFT, generated in FP64 and
 * rounded to FP32) and synchronises the current device.  flags: 0 or
 * QTP_PLAN_AUTOTUNE.  With QTP_PLAN_AUTOTUNE the plan times, on scratch
 * buffers it allocates and frees, (BF16 precisions) for the forward and both
 * backward product kinds every tensor-core tile shape that keeps the
 * split-BF16 accuracy bound for that kind's reduction length, and (p > 128)
 * every form of the forward and of the inverse tube transform (one kernel,
 * two passes with runtime-radix sub-transforms, two passes with compile-time
 * ones for every split p = N1 N2 they allow), and keeps the fastest of each;
 * choices are cached per (device,
 * shape, precision) in the process and appended to the file named by the
 * environment variable QTP_AUTOTUNE_CACHE, if set, which later processes
 * read. */
QTP_API qtp_status qtp_plan_create(qtp_plan** out, int m, int n, int s, int p,
                           int precision, unsigned flags);
QTP_API qtp_status qtp_plan_destroy(qtp_plan* plan);

/* Tile shapes the plan uses for its (forward, dA, dB) products: 0 = built-in
 * rule, 1 = 256 wide, 2 = 128 wide, 3 = 128 wide with split accumulators,
 * 4 = 128 wide with accumulators promoted to FP32 every 512 terms of the
 * reduction.  The built-in rule picks by the reduction length K per half
 * (n forward, s for dA, m for dB): 1 or 2 up to 384, 3 up to 1024, 4 beyond,
 * which keeps QTP_PREC_BF16X3 within 1e-5 relative error for every K the
 * plan accepts. */
QTP_API qtp_status qtp_plan_get_tiles(const qtp_plan* plan, int* tiles3);

/* Kernel launches that one qtp_forward call (*forward) and one qtp_backward
 * call with both outputs requested (*backward) issue for this plan: 3 and 5
 * (Steps 1, 2, 3 of Algorithm 5.1; the backward transforms A and B, then dC,
 * forms dA and dB, and transforms both back in one launch), or 1 forward
 * launch for products small enough to run whole in one CTA.  Long tubes
 * (p > 128 without a one-kernel compile-time transform that factor as
 * p = N1 N2 with N2 in {128, 256, 100, 64} and N1 <= 32, or from p = 2048 with
 * any factor between 4 and sqrt(p)) transform in two launches per transform
 * step (through an intermediate in the workspace): up to 5 and 8.  Tensor-core
 * plans with small m and s (max(m, s) <= 128, min(m, s) <= 64, n <= 384 in
 * split-BF16) and p >= 256 form their forward products in the grouped kernel,
 * one tile per frequency, after a one-block copy of the problem record: one
 * forward launch more (QTP_SMALL_TILES = 0 in the environment at plan creation
 * keeps the single-product kernel).  The training pair issues *forward
 * (qtp_forward_saving, never the one-CTA route) and *backward minus the
 * transform launches of A and B (qtp_backward_saved).  Library extension
 * with no counterpart in the paper; for launch accounting.
 * Errors: QTP_ERR_INVALID_ARG for a NULL plan or output pointer. */
QTP_API qtp_status qtp_plan_launch_count(const qtp_plan* plan, int* forward, int* backward);

/* Bytes of device workspace qtp_forward needs: the spectra of A and B in the
 * GEMM operand format of the plan's precision plus the FP32 spectrum of C,
 * and for long tubes (see qtp_plan_launch_count) the FP32 intermediate of the
 * two-pass transforms. */
QTP_API qtp_status qtp_workspace_size(const qtp_plan* plan, size_t* bytes);

/* Bytes of device workspace qtp_backward needs (spectra of A, B and dC and
 * the FP32 spectra of dA and dB). */
QTP_API qtp_status qtp_backward_workspace_size(const qtp_plan* plan, size_t* bytes);

/* C = A * B (Definition 2.3) by Algorithm 5.1:
 *   Step 1 (Thm 4.4, eq. fft-Q): FFT of every tube of both halves of A and B
 *          along the third mode, omega = exp(-2 pi i / p), unnormalised.
 *   Step 2 (Thm 5.1, eqs. TC/TC2): for every frequency f, with f' = (-f) mod p
 *          (the paper's 1-based p+2-i),
 *            C1_f = A1_f B1_f - A2_f conj(B2_f'),  C2_f = A1_f B2_f + A2_f conj(B1_f')
 *          i.e. one complex m x 2n x 2s product per frequency.  This is the
 *          paper's eqs. TC/TC2 after absorbing its conjugations into the
 *          transform (fft(conj x) = conj(fft(x)) reversed in frequency).
 *   Step 3 (eq. ifft-C): inverse FFT of every tube of C1, C2 with scale 1/p.
 * A: 2*m*n*p complex, B: 2*n*s*p complex, C: 2*m*s*p complex (layout above).
 * C may not alias A, B or the workspace.  workspace_bytes must be at least
 * qtp_workspace_size(plan).  Asynchronous on stream.  Products small enough
 * to hold A, B and all three spectra in 96 KB of shared memory (p <= 64) run
 * the three steps in one CTA with FP32 arithmetic, whatever the plan's
 * precision (environment variable QTP_NO_FUSED=1: the three launches). */
QTP_API qtp_status qtp_forward(const qtp_plan* plan, const float* A, const float* B, float* C,
                       void* workspace, size_t workspace_bytes, void* stream);

/* Same product with A, B and C in HOST memory (pinned for full speed).  The
 * call copies A and B to the device, runs qtp_forward and copies C back, all
 * asynchronously on stream; the caller synchronises before reading C.
 * dev_buffer (device, 16-byte aligned) must hold at least
 * qtp_host_buffer_size(plan) bytes: device copies of A, B, C plus the
 * workspace. */
QTP_API qtp_status qtp_host_buffer_size(const qtp_plan* plan, size_t* bytes);
QTP_API qtp_status qtp_forward_host(const qtp_plan* plan, const float* A_host, const float* B_host,
                            float* C_host, void* dev_buffer, size_t dev_buffer_bytes, void* stream);

/* A sequence of count independent products of the plan's shape with every
 * operand in HOST memory (pinned for full speed): C_host[i] = A_host[i] *
 * B_host[i], i < count, each by the three steps of qtp_forward.  The device
 * holds two products at a time (two slots of A, B, C and one workspace), so
 * the copies of product i + 1 to the device run while product i is computed
 * and its C is copied back: host-to-device and device-to-host copies go on
 * two streams of the plan's own, the compute on stream.  A long sequence then
 * runs at the host link's rate instead of the sum of the copy and compute
 * times.
 * Arguments: A_host, B_host, C_host are arrays of count host pointers (each
 * 16-byte aligned; layout of qtp_forward).  The products must be independent:
 * no C_host[i] may overlap another C_host[j], an A_host[j] or a B_host[j].
 * dev_buffer (device, 16-byte aligned, caller-owned) must hold at least
 * qtp_host_many_buffer_size(plan) bytes.
 * Ordering: work enqueued on stream before the call completes before the
 * first copy starts; the last copy of the call is joined back onto stream, so
 * the caller synchronises stream before reading any C_host[i] or reusing any
 * buffer.  Calls on one plan must not run concurrently from several host
 * threads (the copy streams are the plan's).
 * Errors: count < 0, NULL arrays or pointers, misalignment and an undersized
 * dev_buffer are rejected before anything is enqueued; count == 0 is a
 * no-op.  A failed launch returns QTP_ERR_CUDA with the copies already queued
 * joined onto stream. */
QTP_API qtp_status qtp_host_many_buffer_size(const qtp_plan* plan, size_t* bytes);
QTP_API qtp_status qtp_forward_host_many(const qtp_plan* plan, int count, const float* const* A_host,
                                 const float* const* B_host, float* const* C_host, void* dev_buffer,
                                 size_t dev_buffer_bytes, void* stream);

/* Training pair: the backward pass reuses the forward's spectra of A and B
 * instead of transforming them again (Step 1 of the backward then transforms
 * only dC).  qtp_forward_saving computes C = A * B like qtp_forward, always
 * by the three steps (never the one-CTA route), and leaves the spectra of A
 * and B in `saved` (device, caller-owned, at least qtp_workspace_size(plan)
 * bytes), which the caller keeps unchanged until the matching
 * qtp_backward_saved.  qtp_backward_saved computes dA = dC * B^H and
 * dB = A^H * dC as qtp_backward does, reading A's and B's spectra from
 * `saved` (A and B themselves are not needed); dA or dB may be NULL;
 * workspace_bytes >= qtp_backward_workspace_size(plan).  Both asynchronous
 * on stream.  Errors as qtp_forward / qtp_backward, and QTP_ERR_WORKSPACE
 * for an undersized `saved`. */
QTP_API qtp_status qtp_forward_saving(const qtp_plan* plan, const float* A, const float* B, float* C, void* saved,
                              size_t saved_bytes, void* stream);
QTP_API qtp_status qtp_backward_saved(const qtp_plan* plan, const float* dC, const void* saved, size_t saved_bytes,
                              float* dA, float* dB, void* workspace, size_t workspace_bytes, void* stream);

/* T-SVD of a quaternion tensor under the T-product.  The paper names
 * T-SVD-type (low-tubal-rank) methods as what its fast T-product opens up
 * (Sec. 6) but defines none; this one rests on the per-frequency structure
 * of Thm 5.1: with A1_hat = fft(A1), A2_hat = fft(A2) along mode 3 and
 * g = (-f) mod p, the 2m x 2n complex matrices
 *     M_f(A) = [[A1_hat(f), A2_hat(f)], [-conj A2_hat(g), conj A1_hat(g)]]
 * satisfy M_f(X * Y) = M_f(X) M_f(Y) and M_f(X^H) = M_f(X)^H, so one SVD per
 * frequency pair {f, g} gives
 *     A = U * S * V^H,   U^H * U = I_k,   V^H * V = I_k,   k = min(m, n),
 * with S f-diagonal (every frontal slice diagonal, no j part).  S's spectra
 * at f and g are the odd- and even-ranked singular values of M_f (f < g);
 * at f = g (f = 0, and p / 2 for even p) M_f's singular values come in equal
 * pairs and the factors are a quaternion SVD.  Truncating U, S, V to their
 * first r columns gives the tubal-rank-r approximation that keeps the 2r
 * largest singular values of every M_f.
 * A: m x n x p (layout of qtp_forward); outputs U: m x k x p, S: k x k x p,
 * V: n x k x p (same layout), sigma: p x k floats, sigma[f][i] = S's spectrum
 * at frequency f, entry (i, i) (real, decreasing in i).  All device memory,
 * caller-owned, 16-byte aligned; workspace_bytes >= qtp_tsvd_workspace_size.
 * FP32 one-sided Jacobi per frequency pair.  Limits: min(m, n) <=
 * QTP_TSVD_MAX_K, max(m, n) <= QTP_TSVD_MAX_MN, p <= 4096 (QTP_ERR_UNSUPPORTED
 * beyond).  Asynchronous on stream.  When a pair's columns are kept in
 * registers (2 max(m, n) <= 256, buffers past 200 KB) a cluster of up to 8 CTAs
 * shares it, the count taken from the cluster occupancy at the first call of
 * a shape; QTP_TSVD_CLUSTER = n in the environment fixes it (for
 * measurement; the results do not depend on it). */
#define QTP_TSVD_MAX_K 64
#define QTP_TSVD_MAX_MN 1024
QTP_API qtp_status qtp_tsvd_workspace_size(int m, int n, int p, size_t* bytes);
QTP_API qtp_status qtp_tsvd(int m, int n, int p, const float* A, float* U, float* S, float* V, float* sigma,
                    void* workspace, size_t workspace_bytes, void* stream);

/* Synchronise stream after a qtp_tsvd call of this shape on this workspace
 * and report whether every frequency pair's Jacobi sweeps converged: each of
 * the two sweep phases (before and after the Newton-Schulz step that keeps V
 * unitary) stops after a sweep whose column pairs were all orthogonal to
 * within a relative off-diagonal |x^H y| / (|x| |y|) of 1e-3 (the first
 * phase) or 1e-4 (the second) when visited, or after 40 sweeps; a pair that
 * missed the bound in its 40th sweep gets factors that are written as usual
 * but may miss the orthogonality bound, and this call then returns
 * QTP_ERR_NOT_CONVERGED (else QTP_OK; QTP_ERR_CUDA if the stream reports an
 * error).  The status lives in the workspace and is cleared by the next
 * qtp_tsvd on it. */
QTP_API qtp_status qtp_tsvd_sync(int m, int n, int p, const void* workspace, void* stream);

/* Gradients of a real loss L(C), C = A * B, with each quaternion entry taken
 * as four independent reals (not in the paper; a training-style use of it):
 *     dA = dC * B^H,   dB = A^H * dC,
 * where X^H(:,:,1) = X(:,:,1)^*, X^H(:,:,k) = X(:,:,p+2-k)^* (quaternion
 * conjugate transpose of the slices, Kilmer-Martin convention), so both are
 * T-products computed by the same three steps.  dC has C's shape, dA A's, dB
 * B's.  dA or dB may be NULL to skip it.  workspace_bytes must be at least
 * qtp_backward_workspace_size(plan).  Asynchronous on stream. */
QTP_API qtp_status qtp_backward(const qtp_plan* plan, const float* dC, const float* A, const float* B,
                        float* dA, float* dB, void* workspace, size_t workspace_bytes,
                        void* stream);

/* ------------------------------------------------------------------------
 * Batches: thousands of independent products of uneven shapes in one call
 * ------------------------------------------------------------------------ */

/* Shape of one product of a batch: A is m x n x p, B is n x s x p. */
typedef struct {
  int m, n, s, p;
} qtp_shape;

typedef struct qtp_batch_plan qtp_batch_plan;

/* Flags of qtp_batch_plan_create. */
#define QTP_BATCH_NO_GRAPH 1u  /* launch the kernels directly instead of replaying a CUDA graph */
#define QTP_BATCH_AUTOTUNE 2u  /* time the products' routing at plan creation (BF16 precisions) */

/* Plan a batch of `count` products C_i = A_i * B_i (Definition 2.3, each by
 * Algorithm 5.1).  Shapes are copied; each must satisfy the limits of
 * qtp_plan_create.  The plan orders the products by tube length p and then
 * size (the order the grouped kernels walk them; results are unaffected),
 * lays out every product's spectra in one workspace, builds the device job
 * and tile tables and the twiddle tables of every distinct p, and
 * synchronises the device.  Each forward call runs grouped launches (the
 * tube FFTs of A and B, one launch per distinct p; all per-frequency products
 * in one persistent tensor-core launch, or one FP32 launch; the inverse FFTs,
 * one launch per distinct p), replayed from a
 * CUDA graph captured on the first call (and again after the workspace
 * pointer changes) on a stream the plan owns, ordered after and before the
 * caller's stream with events. */
QTP_API qtp_status qtp_batch_plan_create(qtp_batch_plan** out, const qtp_shape* shapes, int count,
                                         int precision, unsigned flags);
QTP_API qtp_status qtp_batch_plan_destroy(qtp_batch_plan* plan);
QTP_API qtp_status qtp_batch_workspace_size(const qtp_batch_plan* plan, size_t* bytes);

/* A, B, C: HOST arrays of `count` DEVICE pointers (product i in the order of
 * the shapes given to qtp_batch_plan_create), each 16-byte aligned, layout as
 * for qtp_forward.  The pointer arrays are copied before the call returns.
 * Asynchronous on stream. */
QTP_API qtp_status qtp_forward_batched(qtp_batch_plan* plan, const float* const* A, const float* const* B,
                                       float* const* C, void* workspace, size_t workspace_bytes, void* stream);

/* Routing of a batch's tensor-core products (library extension; the paper has
 * no counterpart).  Step 2 runs every product either in the grouped kernel
 * (128 x 64 tiles that compute both output halves) or in the single-product
 * kernel (128 x 256 / 128 x 128 tiles per output half, one launch each,
 * spread over eight streams of the plan inside the graph, concurrent with
 * the grouped kernel): products whose
 * split-BF16 reduction exceeds 384 per half always take the latter, and so do
 * products with min(m, s) >= *route_min.  Without QTP_BATCH_AUTOTUNE
 * *route_min is INT_MAX (every other product grouped; the environment
 * variable QTP_BATCH_ROUTE_MIN overrides it).  With QTP_BATCH_AUTOTUNE the
 * plan times the products on a zeroed scratch workspace it allocates and
 * frees for the thresholds INT_MAX, 192, 128, 96, 64, 48 and keeps the
 * fastest (cached per device, precision and shapes for the process);
 * tuned_ms[i] (i < *tuned_count <= 8) receives those times in that order.
 * Any output pointer may be NULL. */
QTP_API qtp_status qtp_batch_plan_route(const qtp_batch_plan* plan, int* route_min, float* tuned_ms,
                                        int* tuned_count);

/* Tracing of batched calls: four events around the three stages (forward
 * transforms, products, inverse transforms); ms3 receives their durations for
 * the last traced call (waits for it). */
QTP_API qtp_status qtp_batch_plan_set_tracing(qtp_batch_plan* plan, int enable);
QTP_API qtp_status qtp_batch_stage_times(const qtp_batch_plan* plan, float* ms3);

/* As qtp_plan_sync, for a batch plan. */
QTP_API qtp_status qtp_batch_plan_sync(const qtp_batch_plan* plan, void* stream);

/* Synchronise stream, then read and clear the plan's device error word.
 * Returns QTP_ERR_TIMEOUT if a kernel gave up on a bounded wait since the
 * last call, QTP_ERR_CUDA if the stream reports an error, else QTP_OK. */
QTP_API qtp_status qtp_plan_sync(const qtp_plan* plan, void* stream);

/* Tracing.  While enabled, every qtp_forward / qtp_forward_host /
 * qtp_backward call records four CUDA events on its stream: before Step 1,
 * after Step 1 (tube FFTs), after Step 2 (per-frequency products) and after
 * Step 3 (inverse FFTs); a one-CTA forward counts entirely as Step 2.
 * qtp_plan_stage_times waits for the events of the last traced call and
 * writes the three stage durations (ms) to ms3[0..2].
 * Enabling creates the events (no device memory); disabling destroys them. */
QTP_API qtp_status qtp_plan_set_tracing(qtp_plan* plan, int enable);
QTP_API qtp_status qtp_plan_stage_times(const qtp_plan* plan, float* ms3);

/* C = A * B, exactly as qtp_forward, for callers that may not allocate device
 * memory (the paper has no counterpart; this is a property of the library).
 * Some host programs cannot call cudaMalloc: their device memory belongs to
 * another allocator (a framework's caching pool, a fixed memory budget) that
 * must stay the only one, or they cannot afford cudaMalloc's implicit
 * synchronisation.  Plans allocate and qtp_forward needs a workspace, so this
 * entry point takes neither: dimensions and precision are passed directly, and
 * the twiddle table, error word and spectra live in one static device array
 * of QTP_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading the library
 * holds until the process exits.  A, B and C are the caller's device tensors
 * (layout as above).  It calls no cudaMalloc, cudaFree or allocating routine.
 * - Products whose scratch (twiddles + spectra of A, B and C, see
 *   qtp_workspace_size) exceeds the array are rejected with
 *   QTP_ERR_WORKSPACE before any launch.
 * - Every call looks up the array's device address in the current device's
 *   context (cudaGetSymbolAddress, which allocates nothing), so the address
 *   stays valid after a device reset.  The first call on a device loads the
 *   library's module there; make that first call before any stream capture
 *   begins.
 * - All calls share the one array and it keeps the last call's contents; each
 *   call clears its error word and rewrites its twiddles.  Calls that overlap
 *   on the GPU (other streams, other threads) race on the array: order them.
 * - A device-side wait that gives up (see qtp_plan_sync) cannot be reported
 *   here: there is no plan to read it from. */
#define QTP_NOALLOC_SCRATCH_BYTES (32 << 20)
QTP_API qtp_status qtp_forward_noalloc(int m, int n, int s, int p, int precision, const float* A,
                                       const float* B, float* C, void* stream);

/* Thread-local description of the last failure in this thread ("" if none). */
QTP_API const char* qtp_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
QTP_API int qtp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QTP_H_ */
