// Internal definitions shared by the translation units of libcncpd.
//
// Device data layout (all in HBM, allocated once per handle):
//  - X^(k): dense C-order tensor in the storage type (f64, f32, bf16, or two
//    bf16 planes hi/lo).  The tensor is viewed as a matrix with
//    lead_rows = prod_{m<h} I_m rows and trail_cols = prod_{m>=h} I_m
//    columns (h = number of "lead" modes of the two-level dimension tree).
//  - factors U1 (current iterate), U2 (previous iterate), S (snapshot of U2
//    at the start of an iteration) live in three arenas of identical layout;
//    U^(n,k) is row-major I_n x R_k.
//  - Grams G^(n,k) = U^T U are R_k x R_k in FP64.
//  - Pl^(k) (lead_rows x R) and Pt^(k) (trail_cols x R) hold the level-1
//    partial contractions of the dimension tree; M^(n,k) (I_n x R_k) the
//    MTTKRP of the mode being updated.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>

#define CNCPD_KMAX 64
#define CNCPD_NMAX 8
#define CNCPD_RMAX 64

namespace cncpd {

enum Storage { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2, ST_BF16X2 = 3 };

// Scalars that live on the device so that a whole sweep can be replayed as a
// CUDA graph without host round trips.
struct DevScalars {
  double t;          // momentum sequence t_{k} (Appendix A)
  double w_hat;      // hat w of the current iteration
  int have_prev;     // L_prev valid (false in the first iteration)
  int have_cur;      // L_cur written by a sweep
  int nonfinite;     // set when F or a Lipschitz constant is NaN/Inf
  int timeout;       // set when a bounded device-side wait gave up
  double F;          // objective of the last evaluated iterate
  double relerr;     // mean relative error of the same
  double Fk[CNCPD_KMAX];
  double relk[CNCPD_KMAX];
  double xnorm2[CNCPD_KMAX];               // ||X^(k)||^2 (or ||X~^(k)||^2 on the LRA path)
  double Lprev_u[CNCPD_NMAX][CNCPD_KMAX];  // L_u^(n,k) of the previous accepted sweep
  double Lcur_u[CNCPD_NMAX][CNCPD_KMAX];
  double LCprev[CNCPD_NMAX], LCcur[CNCPD_NMAX];
  double Ldprev[CNCPD_KMAX], Ldcur[CNCPD_KMAX];
  double cterm[CNCPD_KMAX][CNCPD_RMAX];    // (U^{odot})^T vec(X^(k)) at the current factors
  double cterm_save[CNCPD_KMAX][CNCPD_RMAX];
  double lam1[CNCPD_KMAX][CNCPD_RMAX];     // cores: current, previous, snapshot
  double lam2[CNCPD_KMAX][CNCPD_RMAX];
  double lamS[CNCPD_KMAX][CNCPD_RMAX];
  double xnorm2_orig[CNCPD_KMAX];          // ||X^(k)||^2 of the stored tensors (global fit)
  double inv_xnorm2[CNCPD_KMAX];           // 1 / xnorm2 and 1 / xnorm2_orig (0 for a zero tensor)
  double inv_xnorm2_orig[CNCPD_KMAX];
  double out_relk[CNCPD_KMAX];             // per-block relative error of an uncommitted evaluation
  int done_counter[CNCPD_NMAX + 2];        // arrival counters of last-CTA reductions (reset by the last CTA)
  unsigned int seq;                        // objectives published to the host mirror
};

// Pinned, mapped host memory that the objective's last CTA writes directly,
// so the host learns an iteration's F without a copy or a stream sync: the
// fields first, then (after a system-scope fence) the sequence number.
struct HostMirror {
  double F, relerr;
  int nonfinite, timeout;
  volatile unsigned int seq;
  int pad;
};

struct DevDesc {
  int K, N, h;        // blocks, order, number of lead modes
  int Rmax;
  int lra;            // 1: collapsed (LRA) products replace the tensor passes
  int pad0;
  int R[CNCPD_KMAX];
  int Rt[CNCPD_KMAX];  // LRA ranks
  int L[CNCPD_NMAX];
  int nonneg[CNCPD_NMAX];
  int64_t dims[CNCPD_KMAX][CNCPD_NMAX];
  int64_t lead_rows[CNCPD_KMAX];
  int64_t trail_cols[CNCPD_KMAX];
  const void* X[CNCPD_KMAX];
  const void* Xlo[CNCPD_KMAX];
  void* U1[CNCPD_KMAX][CNCPD_NMAX];
  void* U2[CNCPD_KMAX][CNCPD_NMAX];
  void* M[CNCPD_KMAX][CNCPD_NMAX];
  double* G[CNCPD_KMAX][CNCPD_NMAX];
  void* Pl[CNCPD_KMAX];
  void* Pt[CNCPD_KMAX];
  void* H[CNCPD_KMAX];          // D (*_{m!=n} G) D of the mode being updated, in the factor type
  // LRA step
  void* Ut[CNCPD_KMAX][CNCPD_NMAX];    // U~^(n,k), I_n x Rt_k
  double* Gt[CNCPD_KMAX][CNCPD_NMAX];  // U~^T U~ (Rt x Rt)
  double* C[CNCPD_KMAX][CNCPD_NMAX];   // U~^T U (Rt x R)
  void* Vinv[CNCPD_KMAX];              // ALS: V^{-1} in the factor type (Rt x Rt)
  // split-K partials of the lead-mode contraction
  void* partial;
  int64_t partial_off[CNCPD_KMAX];     // element offset of block k's partials
  int nsplit[CNCPD_KMAX];
  int64_t split_rows[CNCPD_KMAX];
  const CUtensorMap* tmap_trail;        // per-block TMA descriptors of X, boxes of 256 rows x 128 bytes (swizzled)
  const CUtensorMap* tmap_lead;         // per-block TMA descriptors of X, boxes of 32 KiB x 256 columns
  int use_tma;                          // 1: the TMA kernels run the level-1 contractions
  int lt_rows;                          // rows per tile of the trailing contraction (64 or 256)
  int tt_cols;                          // columns per tile of the lead contraction
  int pad2;
  int64_t pitch[CNCPD_KMAX];            // row pitch of X^(k) in elements (multiple of 16)
  int lt_prefix[CNCPD_KMAX + 1];       // cumulative units (row tiles x column splits) of the trailing-mode contraction
  // column splits of the trailing TMA pass: block k's 256-row tiles are cut
  // into lt_js[k] ranges of lt_jc[k] columns (a multiple of one stage); with
  // lt_js[k] > 1 each range leaves a partial Pl at Pl_part + plp_off[k] +
  // split * lead_rows * R, added in split order by k_reduce_trail_splits
  int lt_js[CNCPD_KMAX];
  int lt_jc[CNCPD_KMAX];
  void* Pl_part;
  int64_t plp_off[CNCPD_KMAX];
  int trail_split;                     // 1: some block has lt_js > 1
  int pad6;
  int tt_prefix[CNCPD_KMAX + 1];       // cumulative (column tile x split) units of the lead-mode contraction
  int tt_ctiles[CNCPD_KMAX];           // column tiles per block
  int tt_cpt;                          // columns per thread of that kernel
  int pad1;
  // balanced unit lists of the TMA passes (null: unit g goes to CTA g mod grid).
  // Layout: grid + 1 start offsets, then the unit ids of CTA 0, CTA 1, ...
  const int* lt_sched;
  const int* tt_sched;
  int lt_grid, tt_grid;                // CTAs the lists were made for
  DevScalars* sc;
  int* err;                            // device error word (bounded waits, bad state)
  HostMirror* hm;                      // device address of the host mirror (null: none)
  // factor arenas U1 and S (snapshot of U2 at the start of an iteration); the
  // snapshot of U^(n,k) sits at the same offset in S as U1[k][n] in U1
  char* A1base;
  char* ASbase;
  // Grams and H live in arenas: G^(m,k) = Gbase + (k*N + m)*Rmax^2, H^(k) = Hbase + k*Rmax^2
  double* Gbase;
  void* Hbase;
  // H^(k) of the mode being updated also in FP64 (the objective of the last
  // mode takes ||X_hat||^2 = <H^(N-1,k), G^(N-1,k)> from it): H64base + k*Rmax^2
  double* H64base;
  // Gram partials of each mode (null: Grams are formed by one CTA per factor).
  // Rows of U^(n,k) are cut into chunks of gr[n] rows; chunk c of block k
  // holds its partial sums, in the factor type, at Gp[n] + (k*gnc[n] + c)*Rmax^2.
  void* Gp[CNCPD_NMAX];
  int gr[CNCPD_NMAX];
  int gnc[CNCPD_NMAX];
  // LRA path: chunk values of the cross Grams C^(n,k) = U~^T U, chunks of
  // CROSS_ROWS rows; chunk c of block k at Cp[n] + (k*cgnc[n] + c)*cld.
  void* Cp[CNCPD_NMAX];
  int cgnc[CNCPD_NMAX];
  int cld, pad3;
  // tcgen05 passes (BF16 storage, N = 3): the split factors that are the B
  // operands (3 NP rows, row pitch bt_pitch / bl_pitch elements) and their
  // TMA descriptors; tmap_lead3 views X^(k) as (J, I1, I0) in boxes of 64 x 64 x 1
  // objective fused into the last mode's update: per-CTA sums of <M, U_new>,
  // [chunk CTA][block][RP] in the factor type (null: separate objective kernel)
  void* dotp;
  double* xxp;                          // per-CTA shares of ||X_hat^(k)||^2 of that objective: [chunk CTA][block]
  int use_umma, umma_np;
  // FP32 storage, third order, R <= 32: the trailing pass runs on the TF32
  // tensor cores (Bt holds the factor's two TF32 parts, tmap_bt their map);
  // the lead pass stays on the CUDA cores
  int use_tf32, pad7;
  void* Bt[CNCPD_KMAX];
  void* Bl[CNCPD_KMAX];
  int64_t bt_pitch[CNCPD_KMAX];
  int64_t bl_pitch[CNCPD_KMAX];
  const CUtensorMap* tmap_lead3;
  const CUtensorMap* tmap_bt;
  const CUtensorMap* tmap_bl;
  // BF16 hi + lo storage: the lo planes' maps; both planes stream through the
  // same MMAs (the lo plane's K chunks follow the hi plane's, same B operand)
  const CUtensorMap* tmap_trail_lo;
  const CUtensorMap* tmap_lead3_lo;
  int umma_planes, pad4;               // 1 (BF16) or 2 (BF16 hi + lo)
};

constexpr int CROSS_ROWS = 32;

// -------------------------------------------------------------- helpers ----

template <typename T> struct Acc;  // accumulator type of the level-2 partial sums
template <> struct Acc<float> { typedef float type; };  // short in-kernel sums
template <> struct Acc<double> { typedef double type; };

template <int ST, typename T>
__device__ __forceinline__ T load_x(const void* __restrict__ x, const void* __restrict__ xlo, int64_t i) {
  if constexpr (ST == ST_F64) {
    return (T)__ldg(reinterpret_cast<const double*>(x) + i);
  } else if constexpr (ST == ST_F32) {
    return (T)__ldg(reinterpret_cast<const float*>(x) + i);
  } else if constexpr (ST == ST_BF16) {
    return (T)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(x)[i]);
  } else {
    return (T)(__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(x)[i]) +
               __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(xlo)[i]));
  }
}

// One entry of the lead-mode contraction from its split-K partial sums
// (ns splits, stride elements apart), the splits added in order; the loads of
// up to 32 splits are issued before any of them is added.
template <typename T>
__device__ __forceinline__ T sum_splits(const T* __restrict__ p, int ns, int64_t stride) {
  T s = T(0);
  for (int i0 = 0; i0 < ns; i0 += 32) {
    T x[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = p[(int64_t)min(i0 + j, ns - 1) * stride];  // clamped: no predicate
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (i0 + j < ns) s += x[j];
  }
  return s;
}

// Mixed-radix decode of a flat C-order index over modes [m0, m1) of block k.
__device__ __forceinline__ void decode(const DevDesc* d, int k, int m0, int m1, int64_t flat, int* idx) {
  for (int m = m1 - 1; m >= m0; --m) {
    int64_t I = d->dims[k][m];
    idx[m] = (int)(flat % I);
    flat /= I;
  }
}

__device__ __forceinline__ int ceil_div_i(int a, int b) { return (a + b - 1) / b; }

// Bucketed padded rank used as a compile-time register count.
#define CNCPD_FOR_EACH_RP(X) X(4) X(8) X(10) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64)

inline int rank_bucket(int R) {
  const int b[] = {4, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64};
  for (int v : b) if (R <= v) return v;
  return -1;
}

// Every kernel of the sweep asks for the largest shared-memory carveout, so
// consecutive kernels (the TMA passes need almost all of it) run with one
// L1 / shared split and the SMs are not reconfigured between launches.  Set
// once per kernel and device, before the kernel's first launch.
// Compensated FP32 addition (hi, lo) += x (Knuth's TwoSum); FP64 is slow on
// this part, and a pair of FP32 values carries about 48 bits.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// Sum of the first nch chunk values of entry p (stride rr), in chunk order
// (compensated FP32 for FP32 factors, FP64 otherwise); the loads of up to 32
// chunks are issued before any of them is added.
// CG = true reads through L2 only (values other CTAs of the same kernel wrote).
template <typename T, bool CG = false>
__device__ __forceinline__ double gram_sum(const T* __restrict__ gp, int nch, int rr, int p) {
  auto ld = [](const T* q) -> T {
    if constexpr (CG) return __ldcg(q);
    else return *q;
  };
  if constexpr (sizeof(T) == 4) {
    float hi = 0.f, lo = 0.f;
    for (int c0 = 0; c0 < nch; c0 += 32) {
      float x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = ld(gp + (size_t)min(c0 + j, nch - 1) * rr + p);  // clamped: no predicate
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < nch) ff_add(hi, lo, x[j]);
    }
    return (double)hi + (double)lo;
  } else {
    double s = 0.0;
    for (int c0 = 0; c0 < nch; c0 += 32) {
      double x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = ld(gp + (size_t)min(c0 + j, nch - 1) * rr + p);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < nch) s += x[j];
    }
    return s;
  }
}

template <auto Kernel>
inline void carve() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_relaxed) & bit) return;
  if (cudaFuncSetAttribute(Kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    cudaGetLastError();
  done.fetch_or(bit);
}

// ------------------------------------------- programmatic dependent launch --
// The kernels of a sweep are launched with programmatic stream serialisation:
// a kernel may be launched while its predecessor on the stream is still
// finishing.  Each such kernel calls pdl_wait() before it reads anything an
// earlier kernel of the sweep wrote and before it writes anything (the wait
// returns once the predecessor grid has completed and its memory is
// visible; without a programmatic predecessor it returns at once).  The
// small kernels call pdl_trigger() right after their wait, which lets their
// successor be launched; the tensor passes leave that to their exit.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// kernel<<<grid, block, smem, stream>>>(args...) with programmatic stream
// serialisation allowed (the kernel must call pdl_wait() as described above).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ----------------------------------------------------- launch wrappers ----
// Implemented in mttkrp.cu / update.cu / lra.cu.  `fp64` selects the FP64
// factor path (storage ST_F64); otherwise factors are FP32.

// Record the message returned by cncpd_last_error() on this thread; returns code.
int set_error(int code, const char* msg);

struct LaunchCfg {
  cudaStream_t stream;
  int num_sms;
};

// trailing-mode contraction -> Pl ; lead-mode contraction (split-K + fixed-order reduction) -> Pt
cudaError_t launch_trailing_contract(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int st, int RP);
cudaError_t launch_lead_contract(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int st, int RP,
                                 const int64_t* d_red_prefix, int with_reduce = 1);
int lead_cpt(int fp64, int RP);
bool tma_rank_supported(int RP);
cudaError_t launch_reduce_splits(const LaunchCfg& c, const DevDesc& h_desc, int fp64);
// TMA-staged passes for FP32 (st = ST_F32) and BF16 (st = ST_BF16) storage
cudaError_t launch_trailing_tma(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int RP, int st);
// Pl of every block with column splits = the sum of its partials, in split order.
cudaError_t launch_reduce_trail_splits(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc);
cudaError_t launch_lead_tma(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int RP, int st);
int lead_tma_rows(int st);
// One-CTA kernel whose bounded mbarrier wait gets no arrival and gives up
// after limit_ns, setting *err (the failure-detection self-test).
cudaError_t launch_wait_selftest(cudaStream_t s, int* err, uint64_t limit_ns);
// tcgen05 passes for BF16 third-order tensors (ranks up to 32)
int umma_np(int Rmax);
cudaError_t launch_split_factor(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int which);
cudaError_t launch_trailing_umma(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc);
// TF32 tensor-core trailing pass of FP32 third-order tensors (use_tf32): the
// factor's two TF32 parts, then the pass.
cudaError_t launch_split_factor_tf32(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc);
cudaError_t launch_trailing_tf32(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc);
cudaError_t launch_lead_umma(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc);
cudaError_t launch_level2(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int RP, int n);
cudaError_t launch_gram(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n_begin, int n_end, int which);
// Level-2 of mode n (two-mode groups) and H / L of mode n in one launch
// (CTAs 0..K-1: Lipschitz; the rest: level 2).  with_level2 = 0: Lipschitz only.
cudaError_t launch_mode_prep(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n,
                             int use_core, int prev, int with_level2, int begin = 0);
bool level2_is_pair(const DevDesc& h_desc, int n);
// prev >= 0: first form the Gram of mode `prev` (updated just before)
// begin = 1: the launch also does the iteration bookkeeping of k_iter_begin
// (no core tensor).
cudaError_t launch_lipschitz(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n, int use_core,
                             int prev, int begin = 0);
// msplit = 1: M of mode n (the last mode, a one-mode trailing group) is summed
// here from the lead contraction's split-K partials (and stored).
// with_objective = 1 (the last mode of a sweep, update_fuses_objective true):
// the update also evaluates and publishes the objective, as launch_objective
// with commit = 1 and reduce_last = 1 would.
cudaError_t launch_update(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int RP, int n,
                          int use_w, double delta_w, int use_core, int msplit, int with_objective = 0);
bool update_fuses_objective(const DevDesc& h_desc, int fp64, int RP);
// commit = 1: write F/relerr/core term of the solver state; 0: only out_relk against xnorm2_orig.
// reduce_last = 1: the Gram of the last mode is first summed from the chunk values the update left.
cudaError_t launch_objective(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int RP, int commit,
                             int reduce_last);
cudaError_t launch_core_update(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int use_w, double delta_w);
cudaError_t launch_iter_begin(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int use_core);
// Rows per Gram chunk of a mode with at most imax rows (the rows of one update CTA).
int gram_chunk_rows(int RP, int K, int64_t imax, int fp64);
cudaError_t launch_redo_prepare(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc);
// Quantise a rows x cols tensor (C order) into storage with row pitch `pitch` (padding zeroed).
cudaError_t launch_quantize(cudaStream_t s, const void* src, int src_f64, void* dst, void* dst_lo, int st,
                            int64_t rows, int64_t cols, int64_t pitch, double* norm2_out, double* norm2_scratch,
                            int nblk);
cudaError_t launch_convert(cudaStream_t s, const void* src, int src_f64, void* dst, int dst_f64, int64_t n);
cudaError_t launch_uniform_init(cudaStream_t s, void* dst, int fp64, int64_t n, uint64_t seed);
cudaError_t launch_lmax_host(const double* d_H, int R, double* d_out, cudaStream_t s);
cudaError_t launch_grad(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int RP, int n, int use_core);
// Sum over blocks of the first L_n gradient columns (after launch_grad of mode n) into out (I_n x L_n).
cudaError_t launch_common_grad(cudaStream_t s, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n, void* out,
                               int out_f64);
// LRA
cudaError_t launch_cross_gram(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n_begin, int n_end);
cudaError_t launch_collapsed_m(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n);
cudaError_t launch_lra_objective(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int use_core);
cudaError_t launch_als_solve(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n,
                             const int* active, int* status);
cudaError_t launch_als_apply(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, int n, const int* active);
cudaError_t launch_als_relerr(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc, int fp64, double* relk);
cudaError_t launch_lra_xnorm(const LaunchCfg& c, const DevDesc* d_desc, const DevDesc& h_desc);

}  // namespace cncpd
