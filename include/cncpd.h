/*
 * cncpd.h -- C ABI of the GB300 (sm_103a) implementation of CoNCPD-APG and
 * lraCoNCPD-APG (coupled nonnegative CP decomposition by alternating
 * proximal gradient, with optional low-rank approximation; arXiv 2302.05119).
 *
 * Model (Eq. tensormodel): K nonnegative N-th order tensors X^(k) with
 *   X^(k) ~ [[D^(k); U^(1,k), ..., U^(N,k)]],  U^(n,k) = [U_C^(n) U_I^(n,k)],
 * the first L_n columns U_C^(n) of mode n shared by every block, D^(k)
 * super-diagonal (vector lambda^(k)).  Objective (Eq. costfunc):
 *   F = 1/2 sum_k || X^(k) - [[D^(k); U^(.,k)]] ||_F^2,  U >= 0, D >= 0.
 *
 * Conventions for every entry point:
 *  - Return 0 (CNCPD_OK) on success or a negative CNCPD_E* code; the message
 *    of the last failure on the calling thread is cncpd_last_error().
 *    Nothing is thrown across the ABI.
 *  - Tensors are dense, C order (last mode fastest): element (i_1..i_N) of
 *    block k sits at sum_n i_n * prod_{m>n} I_m^(k).  Factor matrices are
 *    row-major I_n x R_k (element (i, r) at i * R_k + r).
 *  - A "void*" data pointer may be host memory (pageable or pinned) or
 *    device memory of the context's GPU; the library tells them apart with
 *    unified addressing.  The caller keeps ownership of every pointer it
 *    passes; the library copies what it needs before the call returns and
 *    never touches caller memory afterwards.
 *  - Calls on one handle are not thread-safe; different handles are
 *    independent.  Every call that launches work synchronises the
 *    library's stream before it returns.
 *  - The library has no CPU fallback: without a usable CUDA device every
 *    call that needs one fails with CNCPD_ECUDA.
 */
#ifndef CNCPD_H
#define CNCPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cncpd_ctx *cncpd_t;

/* Element types.  CNCPD_BF16X2 stores each tensor element as a pair of
 * bfloat16 numbers hi = bf16(x), lo = bf16(x - hi) whose sum carries about
 * 16 significand bits; it is only a storage format for X. */
typedef enum {
  CNCPD_F64 = 0,
  CNCPD_F32 = 1,
  CNCPD_BF16 = 2,
  CNCPD_BF16X2 = 3
} cncpd_dtype;

enum {
  CNCPD_OK = 0,
  CNCPD_EINVAL = -1,     /* bad argument (sizes, ranks, L_n > min_k R_k, ...) */
  CNCPD_ENOMEM = -2,     /* device allocation failed */
  CNCPD_ECUDA = -3,      /* CUDA runtime error (message has the CUDA text) */
  CNCPD_ENONFINITE = -4, /* objective or a Lipschitz constant became NaN/Inf */
  CNCPD_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
  CNCPD_ESTATE = -6,     /* call not valid in the handle's current state */
  CNCPD_ESINGULAR = -7   /* ALS normal matrix not positive definite */
};

/* Solver options; cncpd_default_opts() fills the paper's settings. */
typedef struct {
  double eps;        /* stop when |RelErr_k - RelErr_{k-1}| < eps; 1e-8 (Sec. III-C) */
  int max_it;        /* iteration cap of cncpd_fit; 1000 (Sec. III-C) */
  double lra_eps;    /* ALS stop threshold of the LRA step; 1e-4 (Sec. III-C) */
  int lra_max_it;    /* ALS sweep cap; 200 (Sec. III-C) */
  double delta_w;    /* delta_w of Eqs. eqextrawd/eqextrawu; 0.9999 (App. A) */
  int use_core;      /* 1: update the super-diagonal cores D^(k) (Eq. solD); 0: D = I */
  int reupdate;      /* 1: non-monotone safeguard of Algorithm 1 (redo with w = 0) when
                        F(k) - F(k-1) > tol * F(k-1); tol = 1e-13 for FP64 storage and
                        1e-6 otherwise (the FP32 objective is accurate to a few 1e-7) */
  int storage;       /* cncpd_dtype of X on the device, or -1 = same as the input
                        (F64 input -> F64 path; anything else -> F32 factors) */
  int use_graph;     /* 1: replay each sweep as a CUDA graph */
  int profile;       /* 1: time the tensor-streaming kernels with CUDA events on the
                        first iteration of each cncpd_step / cncpd_fit call and every
                        8th one after it (and every re-update); the other iterations
                        replay a graph without event nodes */
  int tensor_cores;  /* 1: BF16-stored third-order tensors with ranks up to 32 stream
                        through tcgen05 tensor-core passes; 0: CUDA-core passes only */
  int autotune;      /* 1: the first cncpd_step / cncpd_fit of a handle times every
                        candidate split-K plan of the lead-mode pass (1, 2, 3, 4, 6 or 8
                        units per SM) with CUDA events and keeps the fastest; the winner
                        is cached per problem shape for later handles of the process.
                        0: the plan of the cost model only */
  int tf32;          /* 1 (with tensor_cores): FP32-stored third-order tensors with ranks
                        up to 32 take the trailing-mode pass on the TF32 tensor cores, X
                        and the factor each split into two TF32 parts (FP32-accurate:
                        MTTKRP within 3e-7 of FP64 on uniform data).  Off by default: on
                        GB300 it is slower than the CUDA-core pass (96 against 63 us on
                        5 x 256^3, R = 10) */
  int stream_x;      /* 1: keep only one block's stored values on the device (a window
                        the size of the largest block); cncpd_create takes ||X^(k)||^2
                        block by block, cncpd_lra runs each block's ALS with its tensor
                        in the window, and cncpd_global_fit streams the blocks again.
                        The caller's tensors must stay valid for the handle's lifetime
                        (device or page-locked host memory is read in place).  Only the
                        lraCoNCPD-APG iterations run without X: cncpd_step, cncpd_fit,
                        cncpd_mttkrp and cncpd_objective_grad(_at) return CNCPD_ESTATE
                        before cncpd_lra */
  int reserved[2];
} cncpd_opts;

/* Results of a solver call. */
typedef struct {
  int iters;          /* iterations run by this call */
  int total_iters;    /* iterations since the handle was created (or since cncpd_lra) */
  int reupdates;      /* iterations of this call that were re-updated with w = 0 */
  int converged;      /* 1 if the eps test stopped the call */
  double F;           /* objective after the last iteration (Eq. costfunc; after
                         cncpd_lra, Eq. cosfunclra on the approximation) */
  double relerr;      /* RelErr (Sec. III-C) of the same quantity */
  double fit;         /* 1 - relerr */
  double seconds;     /* host wall time of the call */
  double x_bytes;     /* algorithmic bytes of X streamed by this call's MTTKRP passes */
  double stream_ms;   /* summed CUDA-event time of those passes (opts.profile = 1) */
  int stream_launches;/* number of timed tensor-streaming launches */
  int lra_sweeps;     /* cncpd_lra: largest ALS sweep count over the blocks */
  double lra_relerr;  /* cncpd_lra: mean ||X - [[U~]]|| / ||X|| after ALS */
  double trail_ms;    /* part of stream_ms spent in the trailing-mode contraction */
  double lead_ms;     /* part of stream_ms spent in the lead-mode contraction */
  long long launches; /* kernels launched by this call */
  int lead_plan;      /* lead-pass units per SM in use (chosen by the measuring tuner when
                         opts.autotune is set; 0: not a persistent-pass problem) */
  int lead_plan_tuned;/* 1 if that plan was measured (this call or a cached earlier one) */
  int trail_ranges;   /* most column ranges any block's rows are cut into by the trailing
                         FP32/BF16 pass (1: whole rows; the ranges' partial products are
                         added in range order by one extra launch per sweep) */
  int trail_tensor_cores; /* 1 if the trailing pass runs on the tensor cores (BF16 storage,
                         or FP32 storage split into two TF32 parts, third order, R <= 32) */
} cncpd_stats;

/* Fill *opts with the defaults listed above. */
void cncpd_default_opts(cncpd_opts *opts);

/*
 * Create a problem (Eq. tensormodel, Algorithm 1 input).
 *  K        number of blocks (1..64)
 *  N        tensor order (3..8)
 *  dims     K*N sizes, block-major: dims[k*N + n] = I_n^(k) >= 1
 *  X        K pointers to the tensors (C order, element type x_dtype =
 *           CNCPD_F64 or CNCPD_F32); host or device memory
 *  R        K ranks (1..64)
 *  L        N coupling counts, 0 <= L_n <= min_k R_k (Sec. II-C); a mode
 *           with L_n > 0 must have the same I_n in every block
 *  nonneg   N flags (NULL: all 1); 0 skips the projection max(0, .) in
 *           that mode (the operator P of Sec. II-B is user-defined)
 *  opts     NULL for the defaults
 *  stream   cudaStream_t whose prior work the copy of X waits for (NULL:
 *           the legacy default stream)
 * X is quantised into library-owned device memory in opts->storage and
 * ||X^(k)||^2 taken in FP64 of the stored values.  Page-locked host memory
 * is read in place by the quantising kernel (no staging copy); other host
 * memory goes through a device staging buffer.  Initial factors are
 * Uniform[0,1] from a fixed counter-based generator until
 * cncpd_set_factors overrides them; cores start at 1.
 */
int cncpd_create(cncpd_t *out, int K, int N, const int64_t *dims,
                 const void *const *X, cncpd_dtype x_dtype, const int *R,
                 const int *L, const unsigned char *nonneg,
                 const cncpd_opts *opts, void *stream);

/* Set the initial U^(n,k) (I_n x R_k row-major, dtype F64 or F32; host or
 * device).  The shared first L_n columns are taken from block 0 only: a call
 * for k = 0 writes them into every block, a call for k > 0 writes only the
 * individual columns.  Resets the iteration history (Sec. IV: the factors
 * are the algorithm's initialisation). */
int cncpd_set_factors(cncpd_t h, int k, int n, const void *U, cncpd_dtype dtype);

/* cncpd_set_factors for every block and mode in one call: U holds K*N
 * pointers, block-major (U[k*N + n]), all of one dtype; the same rules for
 * the shared columns (block 0's are written first).  One synchronisation at
 * the end instead of one per factor. */
int cncpd_set_factors_all(cncpd_t h, const void *const *U, cncpd_dtype dtype);

/* Set the initial core lambda^(k) (R_k doubles, host memory). */
int cncpd_set_core(cncpd_t h, int k, const double *lambda);

/*
 * Step (i) of lraCoNCPD-APG (Sec. III-B, Algorithm 2): an unconstrained
 * rank-R_tilde^(k) CPD of every block by ALS (opts lra_eps / lra_max_it),
 * after which cncpd_step / cncpd_fit use the collapsed products of
 * Eqs. eqlrag and eqlrau and never read X again.
 *  R_tilde  K ranks (1..64)
 *  Ut0      K*N pointers (block-major) to the initial ALS factors
 *           (I_n x R_tilde^(k), dtype F64 or F32), or NULL for Uniform[0,1]
 *           from the library's generator
 * Returns CNCPD_ESINGULAR if an ALS normal matrix is not positive definite.
 */
int cncpd_lra(cncpd_t h, const int *R_tilde, const void *const *Ut0,
              cncpd_dtype dtype, cncpd_stats *out);

/* Run n_iters iterations of Algorithm 1 (or its LRA form), each with the
 * safeguard re-update, without the eps test. */
int cncpd_step(cncpd_t h, int n_iters, cncpd_stats *out);

/* Run Algorithm 1 until |RelErr_k - RelErr_{k-1}| < eps or max_it. */
int cncpd_fit(cncpd_t h, cncpd_stats *out);

/* Copy U^(n,k) out (I_n x R_k row-major) as dtype F64 or F32 into host or
 * device memory. */
int cncpd_factors(cncpd_t h, int k, int n, void *dst, cncpd_dtype dtype);

/* Copy lambda^(k) out (R_k doubles, host memory). */
int cncpd_core(cncpd_t h, int k, double *lambda);

/* Copy the LRA factor U_tilde^(n,k) out (I_n x R_tilde^(k)). */
int cncpd_lra_factors(cncpd_t h, int k, int n, void *dst, cncpd_dtype dtype);

/* Fit = 1 - (1/K) sum_k ||X^(k) - X_hat^(k)|| / ||X^(k)|| against the
 * stored tensors (Sec. IV), one extra pass over X; valid on both paths. */
int cncpd_global_fit(cncpd_t h, double *fit);

/*
 * Objective and gradient at the current factors (no extrapolation):
 *  *F       = Eq. costfunc (Eq. cosfunclra after cncpd_lra)
 *  gradU    K*N device or host pointers (block-major, NULL entries skipped)
 *           receiving dF/dU^(n,k) = U D (U^T U)^{circledast_-n} D
 *           - X_(n) U^{odot_-n} D (Eq. solbpgU), I_n x R_k row-major, dtype
 *  gradC    N pointers (NULL entries skipped) receiving the gradient of the
 *           shared U_C^(n): sum_k of the first L_n columns (App. A), I_n x L_n
 * Either array may be NULL.
 */
int cncpd_objective_grad(cncpd_t h, double *F, void *const *gradU,
                         void *const *gradC, cncpd_dtype dtype);

/*
 * Objective and gradient as cncpd_objective_grad, but at the factors U
 * given by the caller instead of the handle's current iterate:
 *  U        K*N pointers (block-major) to U^(n,k), I_n x R_k row-major, dtype
 *           udtype (F64 or F32), host or device memory; the shared first L_n
 *           columns are read from block 0 only (as cncpd_set_factors does)
 *  F, gradU, gradC, dtype: as cncpd_objective_grad
 * The handle's iterate, previous iterate, cores, Lipschitz history, momentum
 * and objective history are left exactly as they were, so evaluating the
 * loss in the middle of a fit does not restart the APG extrapolation (the
 * differentiable-loss use).  The first call allocates a copy of the factor
 * arena that the handle keeps.
 */
int cncpd_objective_grad_at(cncpd_t h, const void *const *U, cncpd_dtype udtype,
                            double *F, void *const *gradU, void *const *gradC,
                            cncpd_dtype dtype);

/* X_(n)^(k) U^{odot_-n} at the current factors (Eq. solapgU second term,
 * without D), I_n x R_k row-major, into host or device memory. */
int cncpd_mttkrp(cncpd_t h, int k, int n, void *dst, cncpd_dtype dtype);

/* Largest eigenvalue of the symmetric PSD R x R matrix H (host memory,
 * row-major, R <= 64) as the GPU solver computes Lipschitz constants
 * (Eqs. eqLipsLd/eqLipsLu). */
int cncpd_lipschitz(const double *H, int R, double *lmax);

/* Opaque checkpoint of the solver state (factors, previous iterates, cores,
 * Lipschitz history, momentum, objective history).  cncpd_save_state writes
 * a malloc'ed blob the caller releases with cncpd_free_blob. */
int cncpd_save_state(cncpd_t h, void **blob, size_t *nbytes);
int cncpd_load_state(cncpd_t h, const void *blob, size_t nbytes);
void cncpd_free_blob(void *blob);

/*
 * Failure-detection self-test (Section III-A's algorithm has no counterpart;
 * this checks the library's own guard against a stalled pipeline).  Every
 * wait of the tensor passes on an mbarrier is bounded in time; one that runs
 * out sets the handle's device error word and the call that launched it
 * returns CNCPD_ETIMEOUT.  This call runs a one-CTA kernel on the handle's
 * stream whose single wait expects an arrival that never comes, with no
 * copy or MMA in flight, and a limit of limit_ms (0.001 .. 2000 ms).
 * Returns CNCPD_ETIMEOUT (the expected result) after clearing the error
 * word; the iteration history is discarded as after any timeout, so the
 * next cncpd_step starts Algorithm 1 afresh from the current factors.  The
 * handle stays usable.  CNCPD_EINVAL for a limit out of range.
 */
int cncpd_check_wait_timeout(cncpd_t h, double limit_ms);

/*
 * Allocation-free MTTKRP for callers that must not let this library call
 * cudaMalloc (their device memory is owned by another allocator or a fixed
 * arena, they run under a strict memory budget, or an allocation's implicit
 * device synchronisation is unacceptable to them).  The paper has no
 * counterpart: it is a service of this library.
 *
 * Computes M[j, r] = sum_{i0, i1} X[i0, i1, j] U0[i0, r] U1[i1, r], the
 * last-mode MTTKRP X_(3) (U1 (.) U0) of one third-order FP32 tensor, on
 * `stream` (NULL: legacy default stream), without synchronising it.
 *  X   device, C order I0 x I1 x I2;  U0: device, I0 x R;  U1: device, I1 x R
 *      (this entry point alone does not accept host memory)
 *  M   device output, I2 x R (row-major);  1 <= R <= 64
 * Scratch: a fixed 8 MiB device array inside the library (2^21 floats),
 * held on every GPU that loads the library until the process exits.
 * I2 * R above 2^21 is rejected with CNCPD_EINVAL.  Nothing in the scratch
 * needs to start at zero.  All calls share that array, so calls that overlap
 * on the GPU (different streams, or different host threads on one device)
 * race and give wrong results; serialise them.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress); under
 * CUDA's lazy module loading that first lookup is also when the library's
 * device code is loaded and the 8 MiB are reserved on that device.  So make
 * one eager warm-up call per device (any valid small problem) before stream
 * capture or latency-sensitive work.  Calls no allocating routine.  X, U0,
 * U1 and M must be device (or managed) memory of the current device:
 * anything else is refused with CNCPD_EINVAL before a kernel is launched.
 */
int cncpd_mttkrp_last_mode_noalloc(const float *X, int64_t I0, int64_t I1,
                                   int64_t I2, const float *U0,
                                   const float *U1, int R, float *M,
                                   void *stream);

/* Release every device allocation of the handle (NULL is ignored). */
void cncpd_destroy(cncpd_t h);

/* Message of the last failing call on this thread ("" if none). */
const char *cncpd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CNCPD_H */
