/*
 * ffca.h - C ABI of the GB300 FastFCA-AS library (libffca.so).
 *
 * FastFCA-AS (Ito & Nakatani, "FastFCA-AS: joint diagonalization based
 * acceleration of full-rank spatial covariance analysis for separating any
 * number of sources", arXiv 1805.09498) estimates, for an STFT mixture
 * y(n,f) in C^I of J sources, the parameters of the jointly diagonalised
 * full-rank spatial covariance model (Sec. 4.1, Eq. diagconst)
 *     R_j(n,f) = v_j(n,f) P(f)^{-H} Lambda_j(f) P(f)^{-1}
 * by maximising the log-likelihood L2 (Eq. L2) with the hybrid algorithm of
 * Sec. 4.4: one EM iteration for (v, Lambda) (Eqs. mutilde0, Phitilde0,
 * updatev, Lambdaupdate), then K fixed-point sweeps for P (Eq. FPI).  It
 * also exposes the conventional FCA EM (Sec. 3.3) as a baseline.
 *
 * Conventions for every entry point:
 *  - All array pointers in the descriptors are DEVICE pointers owned by the
 *    caller.  The library never allocates or frees device memory; it borrows
 *    the pointers for the lifetime of the context and updates parameters in
 *    place.  The only host allocation is the small context object.
 *  - Work is enqueued on the caller's CUDA stream (desc.stream, a
 *    cudaStream_t; NULL = legacy default stream).  Calls that return host
 *    values (a trace, a log-likelihood, a status) synchronise that stream.
 *  - Errors are returned as ffca_status codes; nothing is thrown across the
 *    ABI and no device code traps.  Device-side failures (non-finite values,
 *    singular per-frequency systems) are latched in a status word inside the
 *    workspace and reported by the next synchronising call.
 *
 * Layouts ("mic-planar"; ld = frame stride, ld >= N and ld % 4 == 0):
 *  - y      [I][F][ld] complex  mixture y(n,f) (some texts call it x(n,f));
 *                               interleaved (re, im); complex128 for
 *                               FFCA_PREC_FP64, complex64 for FFCA_PREC_MIXED
 *  - v      [J][F][ld] real     source power spectra v_j(n,f) > 0; double
 *                               for FP64, float for MIXED; in/out
 *  - lambda [F][J][I] double    diagonal of Lambda_j(f), > 0; in/out
 *  - P      [F][I][I] complex128 row-major: P[f][a][i] = [P(f)]_{a,i}, so
 *                               column i is p_i of Eq. FPI; in/out
 * Base pointers must be 16-byte aligned.  Frames n >= N of each row are
 * padding: they are read but never used; v's padding is written back
 * unchanged and the Wiener output's padding is set to zero.
 *
 * Precision (ffca_precision):
 *  - FFCA_PREC_FP64:  every per-(n,f) operation and reduction in FP64.
 *  - FFCA_PREC_MIXED: per-(n,f) arithmetic in FP32 on complex64/float data;
 *    Lambda, P, the per-frequency I x I solves and the log-likelihood totals
 *    are FP64.  Sums over the frames n: each thread's running sum is
 *    Kahan-compensated in FP32 (folded every few tiles) where a thread holds
 *    at most 32 sums, so that the registers hold a compensation term for
 *    each (pass A for I <= 4, pass B for I <= 3, the normal EM's pass when
 *    J I^2 + 2 <= 32); elsewhere (pass B at I = 4, both passes at I = 8, the
 *    normal EM's pass with more sums) a thread's plain FP32 sum is flushed
 *    into the FP64 partial sums every 64 (pass B and the normal EM's pass at
 *    I = 8: 128) units of two frames, so that no FP32 sum runs over more
 *    frames than that however long the mixture is.  The 32 lanes
 *    of a warp are then summed by a five-level pairwise tree in FP32, the
 *    warps' sums in double-float (TwoSum), and the partial sums in FP64.
 *
 * Supported shapes: I in {1, 2, 3, 4, 8}, 1 <= J <= 6 (FFCA_ERR_UNSUPPORTED
 * otherwise), N >= 1, F >= 0 (F == 0 is a
 * no-op).
 */
#ifndef FFCA_H
#define FFCA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FFCA_OK = 0,
  FFCA_ERR_ARG = 1,         /* invalid argument: sizes, null/misaligned pointers, stride */
  FFCA_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
  FFCA_ERR_NONFINITE = 3,   /* a non-finite or non-positive Lambda / log-likelihood appeared */
  FFCA_ERR_SINGULAR = 4,    /* a per-frequency I x I system (P or V_i) was singular */
  FFCA_ERR_TIMEOUT = 5,     /* reserved: a bounded device-side wait ran out */
  FFCA_ERR_INTERNAL = 6,    /* library bug */
  FFCA_ERR_UNSUPPORTED = 7  /* (I, J) outside the compiled set */
} ffca_status;

typedef enum { FFCA_PREC_FP64 = 0, FFCA_PREC_MIXED = 1 } ffca_precision;

/* Problem and state of one FastFCA-AS estimation (device pointers). */
typedef struct {
  int I;                  /* microphones: 1, 2, 3, 4 or 8 */
  int J;                  /* sources, 1..6 */
  int F;                  /* frequency bins, >= 0 */
  int N;                  /* frames, >= 1 */
  int ld;                 /* frame stride of y, v and the Wiener output; >= N, multiple of 4 */
  int K;                  /* fixed-point sweeps per iteration (the paper uses K = 1), >= 1 */
  int prec;               /* ffca_precision */
  const void* y;          /* [I][F][ld] complex, read only */
  void* v;                /* [J][F][ld] real, in/out */
  double* lambda;         /* [F][J][I], in/out */
  double* P;              /* [F][I][I] complex128 interleaved, in/out */
  void* workspace;        /* device scratch, ffca_workspace_size() bytes, 256-byte aligned */
  size_t workspace_bytes;
  void* stream;           /* cudaStream_t */
} ffca_desc;

typedef struct ffca_ctx ffca_ctx;

/* Bytes of device workspace the descriptor needs on the current device
 * (partial sums, counters, per-frequency scalars, the trace).  Returns 0 if
 * the descriptor's sizes are invalid. */
size_t ffca_workspace_size(const ffca_desc* desc);

/* Validate the descriptor, plan the launch grid for the current device and
 * clear the workspace (enqueued on desc->stream).  On success *out receives
 * a context to pass to the calls below and to release with ffca_destroy. */
ffca_status ffca_init(ffca_ctx** out, const ffca_desc* desc);

/* Run `iters` >= 0 hybrid iterations (Sec. 4.4) in place on (v, lambda, P).
 * Each iteration: pass A (E-step, Eq. updatev, Eq. Lambdaupdate, L2 of the
 * entering state), pass B (V_i of Eq. FPI), then the per-frequency FP64
 * fixed-point update of P (K sweeps, (I+1)K small inversions per frequency).
 * ll_trace: host array of iters + 1 doubles or NULL.  When given, ll_trace[t]
 * receives L2 (Eq. L2, natural log, including -I ln(pi) per point) of the
 * state entering iteration t and ll_trace[iters] that of the final state;
 * the call then synchronises and returns the latched device status.  When
 * NULL the work is only enqueued (errors surface at the next sync call). */
ffca_status ffca_iterate(ffca_ctx* ctx, int iters, double* ll_trace);

/* L2 (Eq. L2) of the current state, synchronously, into *ll (host). */
ffca_status ffca_loglik(ffca_ctx* ctx, double* ll);

/* Multichannel Wiener filter (Eq. MMSE0 with Eq. covmodelprop):
 * out[j][a][f][n] = [P^{-H} diag(v_j lambda_j / sigma) P^H y(n,f)]_a with
 * sigma_i = sum_j v_j lambda_ji.  out: device, [J][I][F][ld] complex of the
 * precision's type, caller-owned; padding frames are written as zero.  For a
 * batch context out holds the mixtures' blocks one after another, mixture m's
 * block [J][I][F][ld_m] starting at element J I F frame_offset[m] (the layout
 * of y and v in ffca_batch_desc).  Enqueued only. */
ffca_status ffca_wiener(ffca_ctx* ctx, void* out);

/* Wait for the context's stream and return the latched device status. */
ffca_status ffca_sync(ffca_ctx* ctx);

/* Frequency index of the first latched device error (-1 if none); valid
 * after a synchronising call returned an error.  For a batch context the
 * index is that of the problem, m F + f. */
int ffca_error_frequency(const ffca_ctx* ctx);

/* Number of per-frequency I x I inversions the update of P has performed
 * since ffca_init ((I+1) F K per iteration for the fixed point, Sec. 4.5;
 * see ffca_set_p_update for the others).  Syncs. */
ffca_status ffca_inversion_count(ffca_ctx* ctx, unsigned long long* count);

/* Update of P in each hybrid iteration.  FFCA_P_FIXED_POINT (the default)
 * is Eq. FPI.  The other two are alternatives the paper names without
 * stating them (Sec. 4.6), read as K ascent steps on L2 of step size mu with
 * the V_i of Eq. FPI held fixed, along G / N for G = dL2/dP^* (Eq. partialP):
 *   FFCA_P_GRADIENT          p_i <- p_i + mu ([P^{-H}]_i - V_i p_i)
 *   FFCA_P_NATURAL_GRADIENT  p_i <- p_i + mu (p_i - P P^H V_i p_i)
 * The natural (relative) gradient is P P^H G / N; it inverts no matrix and
 * is equivariant under a change of microphone basis.  The gradient method
 * inverts P once per step.  ffca_inversion_count counts F K per iteration
 * for the gradient and nothing for the natural gradient.  Neither method
 * guarantees an increase of L2 for a large mu: the trace monitors it. */
/* FFCA_P_EM is the normal EM algorithm for P, the fourth alternative of
 * Sec. 4.6, read with the source images x_j of Eq. fullrank as complete data:
 * the M-step for P has Eq. FPI's form with V_i replaced by W_i / (J N),
 *   W_i = P^{-H} (sum_j T_j / lambda_ji^new) P^{-1},
 *   T_j = sum_n (mu~_j mu~_j^H + diag phi~_j) / v_j^new
 * (posterior of the entering state, Eqs. mutilde0 / Phitilde0; the new v and
 * Lambda of Eqs. updatev / Lambdaupdate), K sweeps of it per iteration.  Its
 * sums come from pass A, so an iteration streams y and v once (no pass B);
 * it counts (I+1) F K inversions per iteration like the fixed point, ignores
 * mu and guarantees an L2 that does not decrease (an EM step).  At I = 8
 * each unit of the pass is shared by eight threads (the 336 sums of T_j's
 * off-diagonal entries at J = 6 split over them). */
/* FFCA_P_NEWTON is Newton's method on L2 with the V_i of Eq. FPI held fixed
 * (Sec. 4.6 names it), in the 2 I^2 real coordinates of P, off the I
 * directions p_i -> e^{i t} p_i along which L2 does not change: K steps of
 * size mu per iteration, each solving (Q' H Q' - Pi) s = -Q' g (H and g the
 * Hessian and gradient of L2 / N, Pi the projector on those directions, Q' =
 * 1 - Pi) and moving P by mu s; two inversions per step (P and the system).
 * It converges quadratically near a maximum and is not globally convergent
 * (mu damps it).  At I = 8 one CTA per problem holds the 128 x 128 system
 * in shared memory (a thread per column). */
typedef enum {
  FFCA_P_FIXED_POINT = 0,
  FFCA_P_GRADIENT = 1,
  FFCA_P_NATURAL_GRADIENT = 2,
  FFCA_P_EM = 3,
  FFCA_P_NEWTON = 4
} ffca_p_update;

/* Select the update of P for later iterations of a single or batch context.
 * mu: step size, finite and > 0 for the gradient methods and Newton's
 * (ignored for the fixed point and the EM).  Drops a captured graph.
 * FFCA_ERR_ARG for an unknown method or an invalid mu (the context keeps
 * its previous choice).  With the EM, ffca_timing_read
 * counts its streaming pass as FFCA_KERNEL_ESTEP and its per-problem step as
 * FFCA_KERNEL_PSOLVE, and ffca_batch_autotune tunes the EM pass on pass A's
 * candidates.  The allocation-free call always uses the fixed point. */
ffca_status ffca_set_p_update(ffca_ctx* ctx, int method, double mu);

/* Mask-based initialisation (Sec. 5 initialises the parameters by mask-based
 * covariance matrix estimation from time-frequency masks; the masks are the
 * caller's, the masking method is not part of this library).  Writes the
 * context's v, lambda and P from its mixture y and the masks:
 *  1. R_j(f) = sum_n m_j(n,f) y y^H / sum_n m_j(n,f)  (FP64 sums);
 *  2. P(f) the generalized eigenvectors of (R_1, R_y), R_y = sum_j R_j, in
 *     ascending order of their eigenvalues, each column turned in phase so
 *     that its entry of largest magnitude is real and positive (the GEVD that
 *     gives P and Lambda for two sources, Sec. 4.1; exact for any J whenever
 *     the R_j are jointly diagonalisable), then `sweeps` alternations
 *     lambda_ji = p_i^H R_j p_i, p_i <- V_i^{-1} [P^{-H}]_i with
 *     V_i = (1/J) sum_j R_j / lambda_ji (Eq. FPI on the covariances), and
 *     lambda_ji = p_i^H R_j p_i of the final P;
 *  3. v_j(n,f) = max(m_j(n,f), delta) (1/I) sum_i |[P^H y]_i|^2 / lambda_ji
 *     (frames n >= N untouched).
 * masks: device, the layout and real type of v ([J][F][ld]; a batch: the
 * batch layout of v), 16-byte aligned, m_j >= 0 with sum_n m_j(n,f) > 0 for
 * every (j, f).  sweeps: 0 .. 1000 (10 is a good start); delta in (0, 1].
 * Synchronises and returns the device status: FFCA_ERR_NONFINITE for an
 * all-zero mask row, FFCA_ERR_SINGULAR for a singular R_y or sweep. */
ffca_status ffca_mask_init(ffca_ctx* ctx, const void* masks, int sweeps, double delta);

/* With enable != 0, later calls of ffca_iterate / ffca_batch_iterate (with
 * the fixed-point update of P) run the hybrid iterations with each problem
 * resident on chip: one CTA per problem holds the problem's y and v in shared
 * memory for up to 32 iterations per launch (pass A, the new Lambda and L2,
 * pass B, the P step, all inside the CTA), so that a short problem streams
 * its data from HBM once per launch instead of twice per iteration and an
 * iteration costs no launch.  Same results as the streaming kernels up to
 * the order of the floating-point sums; the trace as ffca_iterate.  For
 * problems of at most the frames the shared memory holds (about 5600 frames
 * at I = J = 3 in the mixed precision, 2300 at I = 8, J = 6; half in FP64):
 * FFCA_ERR_UNSUPPORTED otherwise (the context keeps streaming).  With another
 * update of P selected the iterations stream as usual.  Drops a captured
 * graph. */
ffca_status ffca_set_resident(ffca_ctx* ctx, int enable);

/* Fault injection for tests of failure detection (no GPU fault is made).
 * FFCA_FAULT_PASS_A_NO_COPIES: from the next call on, the producer warps of
 * pass A issue none of their copies, so its consumers' bounded waits run
 * out (after about a second), latch FFCA_ERR_TIMEOUT and skip their tiles;
 * every kernel still ends and the GPU context stays usable.  The context's
 * status then stays latched and its state is not meaningful: release it and
 * make a new context.  FFCA_FAULT_NONE switches the fault off.  Drops a
 * captured graph.  FFCA_ERR_ARG for an unknown kind. */
#define FFCA_FAULT_NONE 0
#define FFCA_FAULT_PASS_A_NO_COPIES 1
ffca_status ffca_test_fault(ffca_ctx* ctx, int kind);

/* Host-buffer transfers for callers whose data live in host memory: copy
 * y, v, lambda and P (same layouts as the device arrays; any may be NULL to
 * skip it) from host to the context's device arrays, or v, lambda and P back
 * to host.  Enqueued on the context stream; ffca_download synchronises.
 * Batch contexts use the batch layouts (rows of ld frames, M F problems).
 * Pinned (page-locked) host memory gives asynchronous, full-speed copies. */
ffca_status ffca_upload(ffca_ctx* ctx, const void* y_host, const void* v_host,
                        const double* lambda_host, const double* P_host);
ffca_status ffca_download(ffca_ctx* ctx, void* v_host, double* lambda_host, double* P_host);

/* Multichannel Wiener filter for host-memory callers: runs ffca_wiener into
 * the caller's device buffer out_dev ([J][I][F][ld] complex; a batch: J I F ld
 * elements in total) and copies it to out_host (same layout), then
 * synchronises. */
ffca_status ffca_wiener_host(ffca_ctx* ctx, void* out_dev, void* out_host);

/* ---------------------------------------------------------------------------
 * Gradients (adjoint) at the context's current state (v, lambda, P), with the
 * per-point posteriors recomputed in one streaming pass over y and v (no
 * state is kept from the iterations), for two losses:
 *
 *   NLL = -L2 (Eq. L2, with the -I ln(pi) term), summed over the N frames
 *         and the F bins;
 *   SE  = sum_{j,a,n,f} |x^_ja(n,f) - s_ja(n,f)|^2, x^ the Wiener estimate
 *         of ffca_wiener (Eq. MMSE0 with Eq. covmodelprop) and s given
 *         reference source images.
 *
 * Outputs (device, caller-owned, overwritten):
 *   dv    [J][F][ld] real of the precision's type: dLoss/dv_j(n,f) for n < N
 *         (16-byte aligned; entries of frames >= N in the last vector units
 *         are written as 0, frames beyond untouched)
 *   dlam  [F][J][I] double: dLoss/dlambda_ji(f)
 *   dP    [F][I][I] complex128: dLoss/dP(f)^*, the conjugate Wirtinger
 *         derivative (for a real loss dLoss = 2 Re sum conj(dP) dP; the NLL
 *         one is minus Eq. partialP's dL2/dP^*)
 *   loss  host double or NULL: the loss value (the call then synchronises)
 * s: device [J][I][F][ld] complex of the precision's type (the layout of the
 * ffca_wiener output).  Enqueued on the context stream.  For a batch context
 * every array takes the batch layout (dv that of v, dlam and dP stacked per
 * mixture as lambda and P, s that of the batch Wiener output), N is each
 * mixture's N[m], and loss is the sum over the mixtures.  At I = 8 each
 * unit of the pass is shared by eight threads (thread e: y~_e, sigma_e and
 * column e of dP^*). */
ffca_status ffca_nll_grad(ffca_ctx* ctx, void* dv, double* dlam, double* dP, double* loss);
ffca_status ffca_wiener_se_grad(ffca_ctx* ctx, const void* s, void* dv, double* dlam, double* dP,
                                double* loss);

/* Kernel kinds reported by ffca_timing_read. */
#define FFCA_KERNEL_PREP 0      /* per-frequency ln|det P|^2 and P^{-H} */
#define FFCA_KERNEL_ESTEP 1     /* pass A with the M-step */
#define FFCA_KERNEL_LOGLIK 2    /* pass A, log-likelihood only */
#define FFCA_KERNEL_WCOV 3      /* pass B: weighted covariance partial sums */
#define FFCA_KERNEL_WIENER 4
#define FFCA_KERNEL_PSOLVE 5    /* per-frequency FP64 fixed-point update of P */
#define FFCA_KERNEL_AFINAL 6    /* per-frequency finalise of pass A: Lambda, log-likelihood */
#define FFCA_KERNEL_ADJ 7       /* adjoint streaming pass (ffca_nll_grad, ffca_wiener_se_grad) */
#define FFCA_KERNEL_ADJ_FINAL 8 /* adjoint per-frequency finalise */
#define FFCA_KERNEL_RESIDENT 9  /* iterations with each problem resident on chip (ffca_set_resident) */
#define FFCA_KERNEL_KINDS 10

/* Profiling: while enabled, each kernel the context launches is bracketed by
 * two CUDA events on the context stream.  ffca_timing_read synchronises,
 * writes per kind the summed device milliseconds (ms) and the number of
 * launches (launches; counted whether or not timing is enabled) since the
 * last read, and resets both.  Either output may be NULL. */
ffca_status ffca_timing_enable(ffca_ctx* ctx, int enable);
ffca_status ffca_timing_read(ffca_ctx* ctx, double* ms, unsigned long long* launches);

/* Hybrid iterations for callers that cannot allocate any memory (the paper
 * has no counterpart; this is an interface for embedding).  A real-time
 * audio thread must not call cudaMalloc, which can block and synchronise the
 * device, and a plugin or a system with a fixed memory map may have no
 * allocator at hand.  This call allocates nothing, neither device nor host
 * memory: the context lives on its stack and its scratch is a static array of
 * FFCA_NOALLOC_SCRATCH_BYTES bytes in the library image, which every GPU that
 * loads libffca.so keeps until the process exits.
 *  - desc: as for ffca_init; desc->workspace and desc->workspace_bytes are
 *    ignored.  Problems whose workspace (ffca_workspace_size) exceeds
 *    FFCA_NOALLOC_SCRATCH_BYTES are rejected with FFCA_ERR_ARG.
 *  - iters, ll_trace: as for ffca_iterate.  Once the call has enqueued
 *    work it waits for desc->stream before it returns, on success (then
 *    returning the device status) and on every error alike, so that none of
 *    its kernels still uses the shared array when the next call clears it.
 *    Errors found before anything is enqueued (bad sizes, too large a
 *    problem) return at once.
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current); make that first call before any
 *    stream capture.
 *  - All calls share the one array, and each starts by clearing it.  Calls
 *    that overlap on the GPU (other threads, other streams) race; serialise
 *    them. */
#define FFCA_NOALLOC_SCRATCH_BYTES (8u << 20)
ffca_status ffca_iterate_noalloc(const ffca_desc* desc, int iters, double* ll_trace);

/* Release the context (host memory only; the device arrays stay the caller's). */
void ffca_destroy(ffca_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batches of independent mixtures of uneven length (same I, J, F), run by
 * the same kernels in one launch per pass: every (mixture, frequency) pair is
 * one problem of the work partition.  The method couples nothing across
 * frequencies (the log-likelihood of Eq. L2 and every update of Sec. 4 are
 * per-frequency), so a batch is the same computation as M separate runs;
 * the trace entry of an iteration is the sum of the M mixtures' L2.
 * Mixture-major layout: mixture m has rows of ld_m = frame_offset[m+1] -
 * frame_offset[m] frames (its first N[m] used); its y block [I][F][ld_m]
 * starts at element I F frame_offset[m] of y, its v block [J][F][ld_m] at
 * element J F frame_offset[m] of v, so the blocks of the M mixtures follow
 * one another.  Parameters are stacked per mixture. */
typedef struct {
  int I, J, F;                    /* as in ffca_desc */
  int M;                          /* mixtures, >= 1 */
  int K;                          /* fixed-point sweeps per iteration */
  int prec;                       /* ffca_precision */
  const long long* frame_offset;  /* HOST [M+1]: 0 = off[0] < ... < off[M] = ld, each a multiple of 4 */
  const int* N;                   /* HOST [M]: frames of mixture m, 1 <= N[m] <= off[m+1] - off[m] */
  long long ld;                   /* total row length = frame_offset[M] (< 2^30) */
  const void* y;                  /* device: M blocks [I][F][ld_m] complex, I F ld elements */
  void* v;                        /* device: M blocks [J][F][ld_m] real, J F ld elements, in/out */
  double* lambda;                 /* device [M][F][J][I], in/out */
  double* P;                      /* device [M][F][I][I] complex128, in/out */
  void* workspace;                /* ffca_batch_workspace_size() bytes, 256-byte aligned */
  size_t workspace_bytes;
  void* stream;                   /* cudaStream_t */
} ffca_batch_desc;

typedef struct ffca_ctx ffca_batch_ctx;

/* Workspace bytes for the batch on the current device (0 if invalid). */
size_t ffca_batch_workspace_size(const ffca_batch_desc* desc);
/* Validate, plan, clear the workspace and upload the per-problem tables
 * (host arrays are read during the call only; synchronises the stream). */
ffca_status ffca_batch_init(ffca_batch_ctx** out, const ffca_batch_desc* desc);
/* `iters` hybrid iterations of every mixture.  ll_trace: host array of
 * iters + 1 doubles (L2 summed over the mixtures, as ffca_iterate) or NULL. */
ffca_status ffca_batch_iterate(ffca_batch_ctx* ctx, int iters, double* ll_trace);
/* L2 of each mixture's current state into the host array ll[M]; synchronises. */
ffca_status ffca_batch_loglik(ffca_batch_ctx* ctx, double* ll);
/* With enable != 0, ffca_iterate / ffca_batch_iterate without a trace replay
 * the whole launch sequence of the call from a CUDA graph, captured (on a
 * private stream) on the first call for a given iteration count and
 * launched on the context stream; per-kernel timing is not recorded for
 * replays, launch counts are.  Works on single and batch contexts.  On a
 * single context ffca_iterate with a trace replays too (iters < 4096, not
 * with the resident form): the graph writes the trace into the workspace,
 * then one copy brings it to ll_trace and the call synchronises and reads
 * the status, as without the graph. */
ffca_status ffca_set_graph(ffca_ctx* ctx, int enable);
/* Batch work partitions: ffca_batch_config_count() candidates per streaming
 * pass, each a choice of the per-problem cost the CTA ranges balance and of
 * the grid size; candidate 0 is the default.  All candidates give the same
 * estimates up to the order of the floating-point sums.
 *
 * ffca_batch_autotune runs rounds x ffca_batch_config_count() hybrid
 * iterations of the batch (they advance the estimate like ffca_batch_iterate),
 * candidate q on iteration q of each round, times pass A and pass B of each
 * with CUDA events, and keeps the fastest candidate of each pass.  Outputs
 * (any may be NULL): the chosen candidates, and per-candidate mean pass times
 * in ms (host arrays of ffca_batch_config_count() doubles).  Synchronises.
 * ffca_batch_set_config selects candidates directly (for reproducible
 * summation order across runs). */
int ffca_batch_config_count(void);
ffca_status ffca_batch_autotune(ffca_batch_ctx* ctx, int rounds, int* cand_a, int* cand_b, double* ms_a,
                                double* ms_b);
ffca_status ffca_batch_set_config(ffca_batch_ctx* ctx, int cand_a, int cand_b);
/* Release a batch context (host memory only; the graph, if any). */
void ffca_batch_destroy(ffca_batch_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Conventional FCA EM (Sec. 3.3 of the paper; the baseline FastFCA-AS is
 * measured against).  Model (Eqs. srcmodel, fullrank): R_j(n,f) =
 * v_j(n,f) S_j(f) with full Hermitian positive definite S_j(f).  Each
 * iteration: per (n,f) the E-step of Eqs. MMSE and postquadexp with a full
 * I x I inverse of R = sum_j R_j and the products R_j R^{-1}, (R_j R^{-1}) R_j;
 * the v update of Eq. vupdate with the current S_j^{-1}; then per frequency
 * S_j <- (1/N) sum_n (mu_j mu_j^H + Phi_j) / v_j (Eq. Supdate) in FP64.
 * Same conventions (device pointers, caller's stream, status codes) and the
 * same y / v layouts and precisions as FastFCA-AS. */
typedef struct {
  int I, J, F, N, ld;     /* as in ffca_desc (I 1..4 or 8, J 1..6) */
  int prec;               /* ffca_precision */
  const void* y;          /* [I][F][ld] complex, read only */
  void* v;                /* [J][F][ld] real, in/out */
  double* S;              /* [F][J][I][I] complex128 row-major, Hermitian PD, in/out */
  void* workspace;        /* ffca_fca_workspace_size() bytes, 256-byte aligned */
  size_t workspace_bytes;
  void* stream;           /* cudaStream_t */
} ffca_fca_desc;

typedef struct ffca_fca_ctx ffca_fca_ctx;

/* Workspace bytes for the descriptor on the current device (0 if invalid). */
size_t ffca_fca_workspace_size(const ffca_fca_desc* desc);
/* Validate, plan and clear the workspace; *out receives the context. */
ffca_status ffca_fca_init(ffca_fca_ctx** out, const ffca_fca_desc* desc);
/* `iters` EM iterations in place on (v, S); ll_trace as for ffca_iterate,
 * with L1 (Eq. L1) in place of L2. */
ffca_status ffca_fca_iterate(ffca_fca_ctx* ctx, int iters, double* ll_trace);
/* L1 (Eq. L1) of the current state, synchronously. */
ffca_status ffca_fca_loglik(ffca_fca_ctx* ctx, double* ll);
/* Matrix inversions and matrix-matrix multiplications performed since
 * ffca_fca_init, counted as Sec. 3.4 counts them: (J+N)F inversions and 2JNF
 * multiplications per iteration.  Synchronises. */
ffca_status ffca_fca_op_counts(ffca_fca_ctx* ctx, unsigned long long* inversions,
                               unsigned long long* multiplications);
/* Frequency of the first latched device error (-1 if none). */
int ffca_fca_error_frequency(const ffca_fca_ctx* ctx);
void ffca_fca_destroy(ffca_fca_ctx* ctx);

/* ---------------------------------------------------------------------------
 * STFT front end and overlap-add back end with the paper's analysis
 * conditions (Table 1: frame length L = 1024 samples, frame shift H = 512,
 * square root of the Hann window; F = L/2 + 1 = 513 bins up to the Nyquist
 * frequency, Sec. 2), so that time-domain mixtures enter and separated
 * time-domain images leave the estimation API.  The window is the periodic
 * Hann window's square root, w(t) = sin(pi t / L), so that analysis and
 * synthesis windows together sum to one over the overlapping frames.
 * Arithmetic in FP32 (complex64 spectra, float signals); every pointer is a
 * DEVICE pointer owned by the caller; enqueued on `stream`.
 *
 * ffca_stft: x [C][S] float (C channels of S samples, 4-byte aligned) ->
 *   out [C][F][ld] complex64 (16-byte aligned; the mic-planar layout of y in
 *   ffca_desc), N = 1 + (S - L) / H frames (0 if S < L; frame n holds samples
 *   n H .. n H + L - 1, no padding):
 *     out[c][f][n] = sum_t w(t) x[c][n H + t] exp(-2 pi i f t / L);
 *   frames N .. ld - 1 are written as zero.  ld >= N, ld % 4 == 0.
 * ffca_istft: in [C][F][ld] complex64 (first N frames used) -> out [C][(N+1) H]
 *   float: out[c][s] = sum_n w(s - n H) x_n(s - n H), x_n the inverse DFT
 *   (1/L, Hermitian extension; the imaginary parts of bins 0 and L/2 are
 *   ignored, as for the spectrum of a real signal) of frame n.  Samples H .. N H - 1, covered by
 *   two frames, reconstruct the signal that ffca_stft analysed.
 * FFCA_ERR_ARG on bad sizes, strides or alignment; C and N of 0 are no-ops. */
ffca_status ffca_stft(const float* x, int C, long long S, void* out, int ld, void* stream);
ffca_status ffca_istft(const void* in, int C, int N, int ld, float* out, void* stream);

/* ---------------------------------------------------------------------------
 * Measurement (not part of the method).  ffca_peak_fp64 runs a kernel of
 * independent FP64 FMA chains over every SM of the current device on
 * `stream` (a cudaStream_t) and writes the best of three timed launches as
 * GFLOP/s (2 flops per FMA) to *gflops (host); it synchronises the stream.
 * This is the measured FP64 peak the FP64 path's ALU roofline is reported
 * against. */
ffca_status ffca_peak_fp64(void* stream, double* gflops);

const char* ffca_status_str(ffca_status s);

/* Text of the last CUDA call the library saw fail in the calling thread
 * ("" if none): which call, and CUDA's message.  Valid until the next
 * failure in that thread. */
const char* ffca_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FFCA_H */
