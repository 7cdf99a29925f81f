/*
 * qtt.h -- C ABI of the GB300 QTT denoising-convolution library (libqtt.so).
 *
 * The library computes, on one GPU, the hot path of "Denoising Convolution
 * Algorithms and Applications to SAR Signal Processing" (arXiv 2301.13339):
 *
 *   noisy samples on a 2^d (1D) or 2^dy x 2^dx (2D) grid
 *     -> QTT reshape (Sec. 4)
 *     -> TT-SVD with the max-rank modification (Alg. 1, Sec. 5 (1)):
 *        the rank truncation is the denoiser (Sec. 6)
 *     -> convolution with the sinc imaging kernel (Eq. GAF, Eq. sinc_kern1/2)
 *        as a QTT Toeplitz operator applied core by core, then TT-rounding
 *     -> Full (Alg. 3) back to the dense array.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Dense arrays are caller-owned DEVICE memory, contiguous; a 2D image is
 *   row-major F[y][x] (x fast).  Sizes are powers of two given as log2.
 * - QTT tensors (qtt_tensor) and operators (qtt_op) are library-owned handles
 *   living in device memory; free them with qtt_free / qtt_op_free.
 * - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls are asynchronous on that stream unless stated otherwise; TT ranks
 *   stay on the device, so the decompose -> convolve -> full chain never
 *   waits for the host.  qtt_get_ranks / qtt_get_cores / qtt_op_create
 *   synchronise the stream.
 * - Element types: QTT_F64 (real double, FP64 arithmetic throughout) and
 *   QTT_C64 (complex float = interleaved re,im float pairs, FP32
 *   arithmetic with FP64 only in the reductions that feed rank decisions).
 * - Errors: every call returns a qtt_status; qtt_last_error() gives a
 *   thread-local message.  Errors detected on the device (an iteration limit
 *   reached, a rank above its capacity) are recorded in a device status word
 *   of the handle and returned by the next qtt_get_ranks.  No call aborts the
 *   process or traps the device.
 * - The library allocates its own device workspace (grow-only, reused); it is
 *   released by qtt_release_workspace().
 */
#ifndef QTT_H_
#define QTT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QTT_OK = 0,
  QTT_EINVAL = -1,        /* bad argument (sizes not powers of two, NULL ...) */
  QTT_ENOMEM = -2,        /* device allocation failed                          */
  QTT_ECUDA = -3,         /* a CUDA runtime call failed                        */
  QTT_ETIMEOUT = -4,      /* a device iteration limit was reached              */
  QTT_ERANK = -5,         /* a rank exceeded its capacity                      */
  QTT_EUNSUPPORTED = -6,  /* valid request this build does not implement       */
  QTT_ENUMERIC = -7       /* non-finite values (NaN / Inf) met in the data     */
} qtt_status;

/* Element type of dense arrays and QTT cores.  This build computes with
 * QTT_F64 (real double: FP64 arithmetic throughout) and QTT_C64 (complex
 * float, interleaved re,im pairs: FP32 arithmetic with FP64 reductions for
 * rank decisions).  QTT_F32 and QTT_C128 name the other two storage types of
 * the problem statement; every entry point answers them with
 * QTT_EUNSUPPORTED (real single-precision data takes the FP32 path as
 * complex64 with zero imaginary part). */
typedef enum { QTT_F64 = 0, QTT_F32 = 1, QTT_C64 = 2, QTT_C128 = 3 } qtt_dtype;

/* Arithmetic of a TT-SVD or rounding.  QTT_PREC_AUTO: the element type's own
 * (FP64 for QTT_F64, FP32 for QTT_C64); QTT_PREC_FP64 / QTT_PREC_FP32 must
 * match it (else QTT_EINVAL).  QTT_PREC_TF32_REFINED (complex64 TT-SVD,
 * qtt_decompose only): the first Gram pass of every factored unfolding with
 * at least 32 rows runs on the tensor cores (tcgen05 MMAs of kind tf32 on
 * each operand's TF32 head and remainder -- three products, FP32-level
 * products -- FP32 accumulation, FP64 sum of the per-CTA partials); its eigenvectors
 * only seed the second, FP32 pass (the projected Gram and the
 * relative-accuracy Jacobi, which decides the ranks), so the result keeps
 * the FP32 path's accuracy (Alg. 1; the refinement is what makes the Gram
 * route as accurate as an SVD).  Other calls answer it, and every call
 * answers QTT_PREC_BF16_REFINED, with QTT_EUNSUPPORTED. */
typedef enum {
  QTT_PREC_AUTO = 0,
  QTT_PREC_FP64 = 1,
  QTT_PREC_FP32 = 2,
  QTT_PREC_BF16_REFINED = 3,
  QTT_PREC_TF32_REFINED = 4
} qtt_prec;

/* Truncation parameters of one TT-SVD or rounding sweep.
 *   eps    relative accuracy; per-cut threshold tau = eps/sqrt(d-1)*||A||_F,
 *          rank = smallest r with sqrt(sum_{i>r} sigma_i^2) <= tau
 *          (Sec. 4 eps-rank, Alg. 1).  eps = 0: cap only.
 *   rmax   rank cap R_max (Sec. 5 modification (1)); <= 0: no cap beyond the
 *          library's capacity QTT_RANK_CAP.
 *   refine 1: second Gram pass on the projected unfolding before the rank
 *          decision (relative accuracy of small singular values); 0: single
 *          pass.  FP64 calls always refine.
 *   delta  0 < delta < 1: the SV drop-off rule (Sec. 5 modification (3))
 *          replaces the eps rule: rank = the first k with
 *          sigma_{k+1}/sigma_k < delta, all singular values if there is no
 *          such drop, then the cap rmax.  <= 0: off.
 *   prec   qtt_prec (QTT_PREC_AUTO = 0 for the element type's arithmetic).
 *   fixed_ranks  NULL, or d+1 host ints r_0..r_d (r_0 = r_d = 1, 1 <= r_k <=
 *          min(2^k, 2^(d-k), QTT_RANK_CAP)): forced ranks, the parity mode
 *          that takes another implementation's rank decisions -- cut k keeps
 *          exactly r_k singular triplets (the dominant ones) and eps, delta
 *          and rmax are not used.  In a rounding the sketch rank also bounds
 *          r_k.  Read during the call only. */
typedef struct {
  double eps;
  int rmax;
  int refine;
  double delta;
  int prec;
  const int* fixed_ranks;
} qtt_trunc;

/* Largest TT rank of a decomposition or of an eps-truncated rounding
 * (capacity of the one-CTA eigen-solvers behind every rank decision). */
#define QTT_RANK_CAP 64

/* Largest sketch rank of the large-rank rounding mode (sketch >
 * QTT_RANK_CAP, complex64 only; see qtt_conv_sinc): its range finder factors
 * matrices of up to 2 x QTT_SKETCH_CAP_BIG rows by blocked Householder QR. */
#define QTT_SKETCH_CAP_BIG 512

typedef struct qtt_tensor qtt_tensor;
typedef struct qtt_op qtt_op;

/* qtt_decompose -- Alg. 2 steps 1-2: QTT reshape + TT-SVD (Alg. 1) with the
 * max-rank modification (Sec. 5 (1)).
 *   x           device array, 2^d elements of dt (1D) or 2^dy x 2^dx (2D,
 *               row-major).  Not modified.
 *   ndim        1 or 2;  log2_shape = {d} or {dy, dx}.
 *   interleave  2D only: 1 = bit-interleaved QTT modes x1,y1,x2,y2,...
 *               0 = x bits then y bits.
 *   tr          truncation (eps, rmax, refine).
 *   out         receives a new handle (caller frees with qtt_free).
 * Asynchronous; ranks stay on the device.  QTT_EINVAL on bad sizes or
 * d < 2 or d > 30. */
qtt_status qtt_decompose(const void* x, qtt_dtype dt, int ndim, const int* log2_shape,
                         int interleave, const qtt_trunc* tr, void* stream,
                         qtt_tensor** out);

/* Max rank TT-RSVD (Sec. 5 modification (2); App. A, Algs. 4-5) of a 1D
 * vector: Alg. 1 with the SVD of every unfolding A^{k} (m_k x n_k) replaced by
 * the randomized SVD with k = rmax and oversampling p -- Y = A Omega with a
 * Gaussian n_k x (rmax + p) test matrix Omega, Q R = Y, B = Q^* A, the SVD of
 * B (from its Gram by the relative-accuracy Jacobi solver), U = Q U~ -- each
 * level keeping min(rmax, ...) triplets (no threshold: the cap alone); a
 * level with min(m_k, n_k) <= rmax + p reverts to the max rank TT-SVD.
 * x: device array of 2^log2_len elements (QTT_C64: complex64, QTT_F64:
 * double), QTT order.  1 <= rmax <= 64, p >= 1, rmax + p <= 96.
 * omega: NULL = the test matrices are drawn on the device (N(0, 1) by
 * Philox4x32-10 with counter (index, level) and key seed, Box-Muller);
 * otherwise a device array of the real type (float for QTT_C64, double for
 * QTT_F64) holding, for k = 1 .. log2_len-1 in order, the n_k x (rmax + p)
 * block of level k column-major, n_k = 2^(log2_len - k) (every level has a
 * block; the levels that revert to the SVD ignore theirs).  Asynchronous;
 * returns a library-owned handle in *out (free with qtt_free); errors:
 * QTT_EINVAL (arguments), QTT_ENOMEM, QTT_ECUDA. */
qtt_status qtt_decompose_rsvd(const void* x, qtt_dtype dt, int log2_len, int rmax, int p,
                              const void* omega, unsigned long long seed, void* stream,
                              qtt_tensor** out);

/* qtt_conv_sinc -- Alg. 2 step 3 with the convolution done by the QTT
 * Toeplitz operator of the sinc kernel (Sec. 1 [KKT13]; kernel Eq. GAF with
 * Delta_x = 1/B on the midpoint grid of [0,1]^D, h = 2^-d per axis), then
 * TT-rounding.  2D: the x operator then the y operator, each followed by a
 * rounding.
 *   B          ndim bandwidths (B_x, B_y order for 2D).
 *   normalize  1: kernel divided by its midpoint-rule integral (Eq.
 *              sinc_kern1/2), 0: A = 1.
 *   eps_op     accuracy of the operator's generating vector QTT.
 *   round_tr   truncation of the rounding (eps_round, R_round cap, refine).
 *   sketch     rank of the random sketch used by the rounding (>= the
 *              rounded rank + oversampling).  <= 0: QTT_RANK_CAP.
 *              QTT_RANK_CAP < sketch <= QTT_SKETCH_CAP_BIG (complex64 only)
 *              selects the large-rank mode for products whose eps-ranks
 *              exceed QTT_RANK_CAP (2D images): the randomised range finder
 *              of the rounding alone, without its truncation sweep, so the
 *              result has the fixed ranks min(sketch, 2^k, 2^(d-k), P_k r_k)
 *              and round_tr's eps / rmax / delta are not applied; its error
 *              is that of the range finder (close to the best approximation
 *              at those ranks less the oversampling).  Larger sketch:
 *              QTT_EINVAL; a float64 tensor: QTT_EUNSUPPORTED.
 *   seed       seed of the sketch's counter-based generator.
 * Operators are built on first use and cached per (n, B, normalize, eps_op,
 * dtype); building synchronises the stream once.  out: new handle. */
qtt_status qtt_conv_sinc(const qtt_tensor* f, const double* B, int normalize, double eps_op,
                         const qtt_trunc* round_tr, int sketch, unsigned long long seed,
                         void* stream, qtt_tensor** out);

/* qtt_round -- TT-rounding of t in place (randomized sketch of rank
 * `sketch`, right orthogonalisation, left-to-right truncated SVD sweep with
 * the thresholds of tr). */
qtt_status qtt_round(qtt_tensor* t, const qtt_trunc* tr, int sketch, unsigned long long seed,
                     void* stream);

/* qtt_to_full -- Alg. 2 step 4 / Alg. 3 (Full): expand t into the caller's
 * device array y (same element type and shape as the decomposed input, 2D
 * written back in row-major array order).  Asynchronous. */
qtt_status qtt_to_full(const qtt_tensor* t, void* y, void* stream);

/* qtt_to_full_noalloc -- the same expansion as qtt_to_full, for callers that
 * must not allocate device memory after start-up: latency-critical loops in
 * which a cudaMalloc (it can synchronise the device and its latency is
 * unbounded) is not acceptable, and processes whose device memory is already
 * reserved by another allocator, where a cudaMalloc could fail.  The paper
 * has no counterpart: this is an interface variant, not a step of the method.
 *   t, y    as qtt_to_full (the caller owns y; t is read only).
 * Scratch: a static 16 MiB device array inside the library (every GPU that
 * loads the library holds it until the process exits).  The expansion needs
 * 2 (2^a + 2^(d-a)) rmax elements plus 8 (2^a + 2^(d-a)) bytes of index
 * tables (a = d/2); QTT_EINVAL with a message when that exceeds 16 MiB.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (no allocation); make that first call before any
 * stream capture.  No call allocates: no cudaMalloc, cudaFree or allocating
 * library routine.  All calls share the one array and it keeps the last
 * call's contents: calls that overlap on the GPU (different streams or
 * threads) race and must be serialised by the caller.  Asynchronous. */
qtt_status qtt_to_full_noalloc(const qtt_tensor* t, void* y, void* stream);

/* qtt_conv_adjoint -- the adjoint of qtt_conv_sinc's operator applied to a
 * QTT tensor r, then TT-rounded with round_tr, and optionally the core
 * gradients of the least-squares deconvolution loss.  This is the
 * differentiation of the convolution step (Alg. 2 step 3) for gradient-based
 * deconvolution with the kernel of Eq. GAF; the paper itself only applies T.
 *   f          QTT tensor whose core gradients are wanted (may be NULL when
 *              grad_cores is NULL); same shape, type and mode order as r.
 *   r          the residual full(T f) - g in QTT form (read only).
 *   B, normalize, eps_op   the forward operator's parameters, as in
 *              qtt_conv_sinc.  T^H is built from the forward operator's
 *              cores with j and i swapped (the cores are real), so it is the
 *              exact adjoint of the discrete operator qtt_conv_sinc applies;
 *              for the even sinc it is correlation with the flipped kernel
 *              and equals T up to eps_op.  2D: T^H = T_x^H T_y^H, each
 *              factor followed by a rounding.
 *   round_tr, sketch, seed  rounding of T^H r, as in qtt_conv_sinc.
 *   grad_cores NULL, or d device pointers; pointer k receives, in f's core
 *              layout at f's current ranks (r_{k-1} x 2 x r_k column-major),
 *              the gradient 2 dL/dconj(F_k) of L(F) = ||full(T F) - g||^2,
 *              i.e. the contraction of w = 2 T^H r with the left and right
 *              partial products of f's cores (environment sweeps).  For real
 *              data this is the ordinary gradient; for complex data it is
 *              the convention of PyTorch's complex autograd.
 *   adj_out    NULL, or receives a new handle holding round(T^H r).
 * Asynchronous.  QTT_EINVAL on mismatched handles or NULL grad pointers;
 * QTT_EUNSUPPORTED when f's and the adjoint's rank capacities exceed the
 * environment sweep's shared memory (max rank product above 64 x 64 for
 * complex64 / real float64 handles with wider products). */
qtt_status qtt_conv_adjoint(const qtt_tensor* f, const qtt_tensor* r, const double* B,
                            int normalize, double eps_op, const qtt_trunc* round_tr,
                            int sketch, unsigned long long seed, void* const* grad_cores,
                            qtt_tensor** adj_out, void* stream);

/* qtt_core_grads -- the chain rule through Full (Alg. 3) alone: for a QTT
 * vector w of f's shape, grad_k = alpha * C_k(f, w) + beta * grad_k where
 * C_k(f, w)[a, i, b] = sum over the other modes of w * conj(left partial
 * product of f up to core k-1)[., a] * conj(right partial product of f from
 * core k+1)[b, .].  Used with w = T^H g to subtract the target's share from
 * the gradient.  grad_cores as in qtt_conv_adjoint (beta = 0: overwrite).
 * Asynchronous. */
qtt_status qtt_core_grads(const qtt_tensor* f, const qtt_tensor* w, double alpha, double beta,
                          void* const* grad_cores, void* stream);

/* qtt_dot -- <x, y> = sum_n conj(x[n]) y[n] of two QTT tensors of the same
 * shape (left-to-right environment sweep, O(d r^3)).  out_dev: DEVICE
 * memory for two doubles (real, imaginary part).  Asynchronous.  The sum is
 * carried in the handles' arithmetic (FP32 for QTT_C64). */
qtt_status qtt_dot(const qtt_tensor* x, const qtt_tensor* y, double* out_dev, void* stream);

/* qtt_add -- new handle alpha x + beta y (the TT sum: block-diagonal
 * cores, ranks r_x + r_y in the interior, each at most QTT_PRODUCT_CAP; no
 * rounding -- follow with qtt_round).  Asynchronous. */
qtt_status qtt_add(double alpha, const qtt_tensor* x, double beta, const qtt_tensor* y,
                   void* stream, qtt_tensor** out);

/* qtt_from_device_cores -- new handle holding copies of d cores given in
 * DEVICE memory, core k at cores[k] in the packed column-major layout
 * r_{k-1} x 2 x r_k (ranks: d+1 host ints, r_0 = r_d = 1).  The caller keeps
 * ownership of its buffers.  Asynchronous (stream-ordered copies). */
qtt_status qtt_from_device_cores(const void* const* cores, const int* ranks, int d, qtt_dtype dt,
                                 int ndim, const int* log2_shape, int interleave, void* stream,
                                 qtt_tensor** out);

/* Batched lines (many independent 1D signals of uneven length, bandwidth
 * and rank cap): Alg. 2 steps 1-4 for every line -- qtt_decompose with
 * (eps, rmax[i], refine), qtt_conv_sinc with (B[i], normalize, eps_op,
 * round_tr) and qtt_to_full -- with the lines spread over internal streams
 * so that their chains run concurrently.  Lines are independent; the paper's
 * method is applied to each unchanged.
 *
 * qtt_batch_create: plans for nlines lines (log2_len[i], B[i], rmax[i]; host
 *   arrays, copied).  nstreams <= 0: 16.  Builds every line's operator plan
 *   (synchronises `stream` once per distinct (log2_len, B)).
 * qtt_batch_run: eager submission.  x[i] / y[i]: caller-owned device arrays
 *   of 2^log2_len[i] elements of dt (y written).  Forks from and joins back
 *   to `stream`; asynchronous.
 * qtt_batch_capture: runs the batch once eagerly (synchronising `stream`),
 *   then captures the same submission for these x / y buffers into a CUDA
 *   graph (relaxed capture mode); `stream` must not be the legacy default
 *   stream.  The buffers must stay valid while the graph is used.
 * qtt_batch_launch: replays the captured graph on `stream` (one launch for
 *   the whole batch); asynchronous.
 * qtt_batch_info: internal stream count and graph node count (0 if none).
 * qtt_batch_free: synchronises the device and releases streams and graph.
 * qtt_batch_conv_sinc: create + run + release in one call (asynchronous;
 *   the internal streams are released when their work completes). */
typedef struct qtt_batch qtt_batch;
qtt_status qtt_batch_create(int nlines, const int* log2_len, const double* B, const int* rmax,
                            double eps, int refine, int normalize, double eps_op,
                            const qtt_trunc* round_tr, qtt_dtype dt, int nstreams, void* stream,
                            qtt_batch** out);
qtt_status qtt_batch_run(qtt_batch* b, const void* const* x, void* const* y, void* stream);
qtt_status qtt_batch_capture(qtt_batch* b, const void* const* x, void* const* y, void* stream);
qtt_status qtt_batch_launch(qtt_batch* b, void* stream);
/* Tile settings of the lines' TT-SVD Gram passes (the autotuner's knobs):
 * gram_parts_per_sm partial-Gram CTAs per SM (the passes' grid; 0: the
 * library default of 2) and chunk_div, a divisor of the column-chunk width
 * each CTA stages (its tile; 0 or 1: the default, 2 or 4: narrower).  They
 * change the order of the FP32 sums, not the method.  They take effect at
 * the next run or capture; a captured graph is dropped.  Out-of-range
 * values: QTT_EINVAL. */
qtt_status qtt_batch_set_tiles(qtt_batch* b, int gram_parts_per_sm, int chunk_div);
qtt_status qtt_batch_info(const qtt_batch* b, int* nstreams, int* graph_nodes);
void qtt_batch_free(qtt_batch* b);
qtt_status qtt_batch_conv_sinc(int nlines, const void* const* x, const int* log2_len,
                               const double* B, const int* rmax, double eps, int refine,
                               int normalize, double eps_op, const qtt_trunc* round_tr,
                               void* const* y, qtt_dtype dt, void* stream);

/* Handle inspection and construction (tests, checkpoints). */
/* ranks_host: d+1 ints r_0..r_d.  Synchronises; returns the device status. */
qtt_status qtt_get_ranks(const qtt_tensor* t, int* ranks_host, void* stream);
/* qtt_get_margins -- how close each rank decision of the call that made t
 * came to its threshold (Alg. 1's eps-rank rule): margins_host[k], k = 0..d,
 * receives min(|sqrt(tail(r_k)) - tau|, |sqrt(tail(r_k - 1)) - tau|) / tau
 * for cut k, tail(r) = the sum of the eigenvalues sigma_i^2 beyond r that
 * the decision saw, tau the cut's threshold; a margin near the working
 * precision (1e-7 in FP32) says that another implementation may decide
 * differently (rerun with fixed_ranks).  NaN where no eps rule decided
 * (k = 0, d, a rank set by the cap, eps = 0, the drop-off rule, forced
 * ranks, the large-rank rounding).  Synchronises. */
qtt_status qtt_get_margins(const qtt_tensor* t, double* margins_host, void* stream);
/* d, element type, ndim and log2 shape of a handle (host-side, no sync). */
qtt_status qtt_get_info(const qtt_tensor* t, int* d, qtt_dtype* dt, int* ndim,
                        int* log2_shape, int* interleave);
/* Copy the cores to host memory, packed core after core, each core
 * r_{k-1} x 2 x r_k column-major (alpha fastest, then i_k, then beta).
 * host_buf must hold sum_k 2 r_{k-1} r_k elements.  Synchronises. */
qtt_status qtt_get_cores(const qtt_tensor* t, void* host_buf, void* stream);
/* Build a handle from host cores in the packed layout above (ranks given
 * as d+1 ints with r_0 = r_d = 1, each <= QTT_RANK_CAP). */
qtt_status qtt_from_cores(const void* host_cores, const int* ranks, int d, qtt_dtype dt,
                          int ndim, const int* log2_shape, int interleave, void* stream,
                          qtt_tensor** out);
/* Release a handle without synchronising.  Every call that uses a handle
 * records the handle's last-use event on its stream when it returns;
 * qtt_free releases the storage on a library stream after that event (so
 * after the last call's work, on whatever stream it ran; work that a caller
 * enqueued on other streams after that call is the caller's to order, as for
 * any stream-ordered free).  qtt_free_async releases it in the order of the
 * given stream (the stream the handle was last used on).  Calls made while
 * their stream is being captured into a CUDA graph record no last-use
 * event: a handle created or used inside a capture is released with
 * qtt_free_async on the capturing stream. */
void qtt_free(qtt_tensor* t);
void qtt_free_async(qtt_tensor* t, void* stream);

/* Operator plan of the 1D sinc Toeplitz operator on 2^d points (Sec. 1
 * [KKT13], Eq. GAF / sinc_kern1): generating vector chat[t] = c(t - 2^d)
 * (chat[0] = 0), its QTT by TT-SVD at eps_op, and operator cores
 * O_k[(b,alpha), j, i, (b',beta)] from the borrow chain of j - i.
 * Synchronises the stream (plan-time). */
qtt_status qtt_op_create(int d, double B, int normalize, double eps_op, qtt_dtype dt,
                         void* stream, qtt_op** out);
/* Operator ranks P_0..P_d (d+1 ints) on the host. */
qtt_status qtt_op_get_ranks(const qtt_op* op, int* ranks_host);
/* Operator cores to host, packed, each P_{k-1} x 2 (j) x 2 (i) x P_k
 * column-major (p fastest, then j, then i, then q), element type real
 * double for QTT_F64 operators and real float for QTT_C64 operators. */
qtt_status qtt_op_get_cores(const qtt_op* op, void* host_buf);
void qtt_op_free(qtt_op* op);

/* Operator x vector without rounding (tests): out has ranks P_k r_k, each
 * at most QTT_PRODUCT_CAP; QTT_EINVAL otherwise. */
#define QTT_PRODUCT_CAP 4096
qtt_status qtt_matvec(const qtt_op* op, const qtt_tensor* x, void* stream, qtt_tensor** out);

/* qtt_fft -- QTT-FFT / QTT-iFFT (Sec. 4, the QTT-FFT of [DKS12]; truncated
 * as Sec. 5 prescribes for the transforms of Alg. 2): the radix-2
 * decimation-in-frequency FFT as one rank-2 QTT operator per bit, the input
 * and every stage TT-rounded with tr, then the chain of cores reversed
 * (bit reversal).
 *   x        QTT_C64 handle (a real handle cannot hold a spectrum:
 *            QTT_EUNSUPPORTED): 1D; 2D plain (interleave 0); or 2D
 *            interleaved with dy == dx (else QTT_EUNSUPPORTED).  Not
 *            modified.
 *   inverse  0: X[k] = sum_n x[n] exp(-2 pi i k n / N) per axis (the Sec. 2
 *            DFT); 1: the inverse DFT including 1/N^D.
 *   tr       truncation of every rounding: rmax = R^_max, or eps, or the
 *            SV drop-off delta (rmax <= 0 and eps = 0: cap QTT_RANK_CAP).
 *   sketch, seed  as qtt_round (the seed advances by one per stage).
 *   out      new handle.  1D: the transform in natural order.  2D: the
 *            transform laid out as the TRANSPOSED image (log2 shape
 *            {dx, dy}, same interleave flag), so that the inverse of a
 *            product of two transforms returns the input layout.
 * The axes are transformed in the order of their least significant bit's
 * mode.  Asynchronous; device status flags of the roundings carry over. */
qtt_status qtt_fft(const qtt_tensor* x, int inverse, const qtt_trunc* tr, int sketch,
                   unsigned long long seed, void* stream, qtt_tensor** out);

/* qtt_sinc_padded -- the kernel array g of Alg. 2 for the sinc kernel, padded
 * as in Sec. 2: g[j] = c(j - (N-1)/2) for j < N (the kernel at the N points
 * of the grid, centred), 0 for N <= j < n = 2^log2_n, where c(m) = h A
 * sinc(pi B m h) with h = 1/n and, for normalize = 1, h A = 1 / the sum of
 * sinc(pi B m h) over m = -(n-1)..n-1 (the normalisation qtt_conv_sinc
 * uses); normalize = 0: A = 1.
 *   N      odd, 1 <= N and 2N - 1 <= n (room for the circular convolution
 *          to equal the linear one), else QTT_EINVAL.
 *   g_dev  caller-owned DEVICE array of n elements of dt (QTT_C64: real
 *          part set, imaginary part 0).
 * Asynchronous. */
qtt_status qtt_sinc_padded(int log2_n, long long N, double B, int normalize, qtt_dtype dt,
                           void* g_dev, void* stream);

/* qtt_hadamard -- new handle holding the entrywise product x .* y (the
 * product of Alg. 2 Step 3) of two handles of the same layout: core k is
 * Z[(a + ra a'), i, (b + rb b')] = X[a, i, b] Y[a', i, b'], ranks multiply
 * (each at most QTT_PRODUCT_CAP, else QTT_EINVAL); no rounding.
 * Asynchronous. */
qtt_status qtt_hadamard(const qtt_tensor* x, const qtt_tensor* y, void* stream, qtt_tensor** out);

/* Per-kernel timing.  When enabled, each kernel launch of the library is
 * bracketed by CUDA events on its stream (adds ~2 event records per launch).
 * qtt_profile_read synchronises the device and writes, for up to cap kernel
 * names, the name (names + i*name_stride, NUL-terminated), the summed
 * milliseconds and the launch count; it returns the number of names.
 * qtt_profile_reset drops the records. */
void qtt_profile_enable(int on);
int qtt_profile_read(char* names, int name_stride, double* ms, int* counts, int cap);
void qtt_profile_reset(void);
/* Algorithmic work recorded while profiling was on, summed over the launches
 * of kernel `name` (the same names as qtt_profile_read): *flops = arithmetic
 * operations the method needs (complex multiply-add = 8), *bytes = the
 * operand bytes the launch has to move at least.  Returns 1 if the name
 * recorded any, else 0 (outputs untouched).  Launch sites without a
 * closed-form count record nothing. */
int qtt_profile_work(const char* name, double* flops, double* bytes);

/* qtt_small_eigh -- the one-CTA Hermitian eigen-decomposition behind every
 * truncation (Alg. 1 "compute truncated SVD", done as eigen-decomposition of
 * the unfolding's Gram matrix).  G: device n x n Hermitian as interleaved
 * double pairs (re, im), column-major, n <= 128.  U: device, element type dt
 * (QTT_C64: FP32 arithmetic, QTT_F64: real part of G, FP64 arithmetic),
 * column-major n x n, columns ordered by descending eigenvalue.  lam: device
 * double[n], descending.  Asynchronous. */
qtt_status qtt_small_eigh(const void* G, int n, qtt_dtype dt, void* U, double* lam, void* stream);

/* Diagnostics: if dev32 is not NULL (device, 32 long long), the following
 * eigen-solves of the FP32 path store clock64() values there; the last
 * solve of each kind leaves its values.  Tridiagonal solver (qtt_small_eigh
 * and the solves inside decompose and round): slots 0-9 = its 10 phase
 * boundaries (start, load, tridiagonalisation, eigenvalues, eigenvectors,
 * orthogonalisation, hand-off, Newton-Schulz, back-transformation, output),
 * slots 10-12 = the end of the Gram-Schmidt sweeps, the number of
 * degenerate copies replaced and the number of vectors in clusters of more
 * than one member.  Jacobi solver: through qtt_small_eigh (with that solver
 * selected) slots 0-3 = start, load, end of the sweeps, end, slot 4 = sweep
 * count, slots 13-15 = ends of the ordering, of the Newton-Schulz Gram and
 * of the output; inside decompose and round the same at slots 16 + those.
 * NULL switches it off. */
void qtt_debug_small_eigh_clocks(long long* dev32);

/* Diagnostics: eigen-solver of the FP32 path (0 = Householder tridiagonal
 * + bisection, the default; 1 = cyclic Jacobi; 2 = for qtt_small_eigh only,
 * the relative-accuracy Jacobi of the refinement passes, up to 20 sweeps
 * and stopping at the first sweep without a rotation: for n > 32 the
 * three-launch data-movement solve).  FP64 always uses Jacobi. */
void qtt_debug_set_eig_solver(int which);

/* Diagnostics: sweep count of the FP32 relative-accuracy Jacobi passes
 * (refinement pass of the TT-SVD and of the rounding); default 2; 0 = run
 * to the convergence test; negative = back to the default. */
void qtt_debug_set_refine_sweeps(int sweeps);

/* Diagnostics: per-CTA partial Grams of the TT-SVD passes per SM (1-16;
 * default 2; anything else restores the default).  Each partial sums its
 * columns in FP32 and the partials are added in FP64, so more partials
 * shorten the FP32 sums. */
void qtt_debug_set_gram_parts(int per_sm);

/* Diagnostics: FP32 tridiagonal solver's orthogonalisation.  Eigenvalues
 * closer than ortol_rel * ||T|| chain into clusters orthogonalised by
 * Gram-Schmidt (default 1e-6); ns_steps Newton-Schulz steps follow
 * (default 3).  Non-positive values restore the defaults. */
void qtt_debug_set_heev_cluster(double ortol_rel, int ns_steps);

/* Diagnostics: the tensor-core (tcgen05) MMA path checked on its own --
 * C (128 x N, row-major, FP32) = A (128 x K, row-major) B^T, B (N x K,
 * row-major), with TF32 operands staged in shared memory and FP32
 * accumulators in tensor memory, one CTA, one 8-deep K step per MMA.
 * A, B, C, err_dev: DEVICE pointers; *err_dev is set to 1 if a wait on the
 * MMA completion ran out (the kernel then frees its tensor memory and
 * returns).  N in {32, 64, 128, 256}, K a positive multiple of 8, else
 * QTT_EINVAL.  Asynchronous. */
qtt_status qtt_debug_tc_selftest(const float* A, const float* B, float* C, int N, int K,
                                 int* err_dev, void* stream);

/* Diagnostics: the complex tensor-core GEMM of the large-rank rounding on
 * its own -- C (M x N) = op(A) B with A (M x K), B (K x N), C all complex64
 * column-major DEVICE arrays (interleaved re, im), op(A) = conj(A) when
 * conjA != 0.  The complex product runs as one real product over the
 * stacking [[Re A, -Im A], [Im A, Re A]] [Re B; Im B] on tcgen05 MMAs
 * (kind::tf32) with each operand split into a TF32 head and its FP32
 * remainder (three products: FP32-level accuracy).  Each chunk of 8 k is
 * summed in a fresh FP32 accumulator in tensor memory and the chunk sums
 * are added in registers with compensation; runs of k above 1024 are split
 * and the partials added with compensation.  *status_dev (a device int, QTT_OK on entry) receives
 * QTT_ETIMEOUT if a wait on the MMA completion ran out.  Negative sizes, a
 * NULL status_dev or a NULL array of nonzero size: QTT_EINVAL; K = 0 gives
 * C = 0.  Asynchronous. */
qtt_status qtt_debug_tc_cgemm(const void* A, const void* B, void* C, int M, int N, int K,
                              int conjA, int* status_dev, void* stream);

/* Diagnostics: 1 (default) re-orthonormalises every complex64 TT-SVD core
 * after its eigen-solves (C <- C (I - E/2), E = C^H C - I with compensated
 * sums, the projection basis of the next unfolding corrected alike); 0
 * keeps the cores as the FP32 eigen-solves give them. */
void qtt_debug_set_orth_fix(int on);

/* Diagnostics: allocates `bytes` from the library's stream-ordered memory
 * pool, fills them with the byte `value` and returns them to the pool, so
 * that the next scratch allocations start from known contents (a check that
 * no kernel reads scratch it did not write).  Synchronises the stream. */
qtt_status qtt_debug_fill_pool(size_t bytes, int value, void* stream);

/* Diagnostics: the FP32 eigen-solves with n <= 32 in the QTT-FFT route's
 * calls (qtt_fft, qtt_hadamard), whose roundings meet spectra degenerate at
 * FP32 resolution.  1 (default): the tridiagonal solver, which checks its
 * eigenvectors' orthonormality, with a Jacobi solve of the same Gram queued
 * behind it and run only when the check fails; 2: the cyclic Jacobi solver
 * for all of them; 0: the tridiagonal solver alone.  Other calls are not
 * affected. */
void qtt_debug_set_heev_repair(int on);

/* Diagnostics: 1 runs every complex64 environment sweep (qtt_dot, core
 * gradients) through its strided-GEMM form, which otherwise serves only rank
 * capacities whose environments exceed one CTA's shared memory; 0 (default)
 * restores that choice. */
void qtt_debug_set_env_big(int on);

/* Diagnostics: accumulator of the complex64 TT-SVD's projections W = U^H M
 * (the m-term sums): 0 (default) Dot2 (exact products, compensated sums),
 * 1 Kahan-compensated sums of rounded products, 2 plain FMA. */
void qtt_debug_set_proj_acc(int which);

/* Diagnostics of QTT_PREC_TF32_REFINED: split = 3 (default) feeds the first
 * pass's tensor-core Gram a TF32 head and remainder of every operand
 * (3xTF32), 1 plain TF32 operands; pass2 != 0 also moves the second pass's
 * Gram to the tensor cores (3xTF32; default 0: the FP32 CUDA-core pass,
 * which decides the ranks). */
void qtt_debug_set_tc_gram(int split, int pass2);

/* Diagnostics: the tensor-core Gram pass on its own -- per-CTA partial
 * Grams X X^H of X (m x n complex64, column-major DEVICE array, 1 <= m <=
 * 128) written to gram_part (DEVICE, max_parts x ldp x ldp complex64,
 * element (a, b) of a partial at a + ldp b, zero outside m x m; m <= ldp <=
 * 128), as the TF32-refined TT-SVD's first pass computes them: split 1 feeds
 * TF32-rounded operands, split 3 a TF32 head and remainder (3xTF32).
 * Returns the number of partials written (<= max_parts; their sum is the
 * Gram), or a negative qtt_status (QTT_EINVAL for bad arguments).
 * *status_dev receives QTT_ETIMEOUT if a wait ran out.  Asynchronous. */
int qtt_debug_tc_gram(const void* X, int m, long long n, int split, void* gram_part, int ldp,
                      int max_parts, int* status_dev, void* stream);

/* Diagnostics: 1 routes the large-rank rounding's products (sketch ranks
 * above 64) to the tensor-core GEMM, 2 only those with k <= 64, 0 (default)
 * all to the CUDA-core GEMM with compensated chunk sums.  The 3xTF32
 * operands keep ~2^-22 of each value (FP32: 2^-24), and along the range
 * finder's chain of products that reaches the result (exact-regime E2
 * ~9e-6 against ~2e-6 on the CUDA cores), so the default stays on the CUDA
 * cores. */
void qtt_debug_set_tc_gemm(int on);

/* Diagnostics: the blocked Householder QR of the large-rank rounding on its
 * own (the orthonormal basis of the randomised range finder, Sec. 5's
 * TT-rounding with a sketch).  A: m x n column-major DEVICE array of dtype
 * QTT_C64 (interleaved re, im floats) or QTT_F64, read only (the
 * factorisation runs on a copy).  Q: m x nq column-major DEVICE array of the
 * same dtype, caller-owned, receives the first nq columns of
 * Q = H_1 ... H_min(m,n) (H_k = I - tau_k v_k v_k^H), so that A = Q R with R
 * upper triangular and Q^H Q = I also where A is rank deficient.  Accepts
 * 1 <= m <= 1024, n >= 1, 1 <= nq <= m; anything else, a NULL array or
 * another dtype: QTT_EINVAL.  Asynchronous on `stream`. */
qtt_status qtt_debug_big_qr(const void* A, int m, int n, int nq, int dtype, void* Q, void* stream);

/* Release the library's cached workspace and operator plans. */
void qtt_release_workspace(void);

/* Thread-local description of the last error ("" if none). */
const char* qtt_last_error(void);

/* Version string. */
const char* qtt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QTT_H_ */
