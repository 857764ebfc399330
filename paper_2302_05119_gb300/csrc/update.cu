// Small per-mode kernels of the APG sweep: Grams, Hadamard products and
// Lipschitz constants, the fused extrapolate / gradient / step / projection
// update with the coupled common-column sum, the objective, the core update,
// and the bookkeeping of iterations and re-updates.
#include <algorithm>

#include "cncpd_internal.cuh"

namespace cncpd {

// ---------------------------------------------------------------------------
// Per-mode views passed to the small kernels by value.  Every pointer and size
// a kernel needs is resolved on the host, so a kernel starts by issuing its
// data loads instead of walking the device descriptor through dependent
// global loads.
// ---------------------------------------------------------------------------
template <typename T>
struct LipArgs {            // H^(n,k) and L^(n,k) for every block
  int K, N, n, prev;        // prev >= 0: first reduce the Gram partials of mode prev
  int use_core, want_L, rr, gnc_prev;
  int gr_prev, begin;       // begin: also the iteration bookkeeping (no core tensor)
  DevScalars* sc;
  double* G;                // Gram arena: G^(m,k) at G + (k*N + m)*rr
  T* H;                     // H arena: H^(k) at H + k*rr
  double* H64;              // the same in FP64
  const T* Gp_prev;         // partials of mode prev
  int R[CNCPD_KMAX];
  int Iprev[CNCPD_KMAX];
};

template <typename T>
struct PairArgs {           // level 2 of a two-mode group
  int K, first, ni, nsl;     // rows per CTA; slices of the a range (n last in its group)
  int In[CNCPD_KMAX], Io[CNCPD_KMAX], R[CNCPD_KMAX];
  int cta0[CNCPD_KMAX + 1];  // first CTA of each block
  const T* P[CNCPD_KMAX];
  const T* W[CNCPD_KMAX];
  T* M[CNCPD_KMAX];
};

template <typename T>
struct UpdArgs {            // fused APG update of mode n
  int K, n, Ln, nonneg;
  int use_w, use_core, gr, gnc;
  int rr, stage_rows;       // stage_rows: the CTA keeps its new rows in shared memory
  double delta_w;
  DevScalars* sc;
  T* Gp;                    // Gram partials of mode n (written)
  int R[CNCPD_KMAX];
  int I[CNCPD_KMAX];
  T* U1[CNCPD_KMAX];
  T* U2[CNCPD_KMAX];
  T* S[CNCPD_KMAX];          // snapshot of U2 at the start of the iteration (written here)
  T* M[CNCPD_KMAX];
  const T* H[CNCPD_KMAX];
  const T* part[CNCPD_KMAX];  // non-null: M is summed from these split-K partials
  int nsplit[CNCPD_KMAX];
  // obj = 1: the objective is fused into this (last-mode) update; every CTA
  // leaves its <M, U_new> sums in dotp[cta][k][RP], the last CTA to finish
  // evaluates F and publishes it
  int obj, N;
  double inv_K;
  T* dotp;
  double* xxp;              // per-CTA <H^(n,k), chunk of G^(n,k)> in FP64: xxp[cta][k]
  int gram_last;            // 1: the tail also stores G^(n) (summed from its chunks)
  double* G;
  const double* H64;        // H^(n,k) in FP64 (written by the Lipschitz kernel of mode n)
  HostMirror* hm;
};

template <typename T>
struct ObjArgs {            // objective with the last mode just updated
  int K, N, rr, gnc;
  int gr, commit, reduce_last, pad;
  double inv_K;             // 1 / K
  DevScalars* sc;
  HostMirror* hm;
  double* G;
  const T* Gp_last;
  int R[CNCPD_KMAX];
  int I[CNCPD_KMAX];
  const T* M[CNCPD_KMAX];
  const T* U[CNCPD_KMAX];
};

// ---------------------------------------------------------------------------
// Largest eigenvalue of a symmetric PSD R x R matrix (R <= RP), called by a
// whole CTA: ||H||_2 of Eqs. eqLipsLd / eqLipsLu.  Normalised repeated
// squaring A <- A^2 / tr(A^2) in FP32 on the zero-padded RP x RP matrix
// converges to the projector on the leading eigenvector (eigenvalue ratios
// are raised to the power 2^s); the value is the Rayleigh quotient of H at a
// column of that limit, evaluated in TT (the factor precision), so its error
// is quadratic in the FP32 accuracy of the eigenvector.  Returns 0 for a zero
// matrix and propagates NaN/Inf.
// ---------------------------------------------------------------------------
template <int RP>
struct LmaxSmem {
  float Hf[RP * RP];  // H in FP32 (R x R, row stride R), written by the caller
  float A[RP * RP];
  float B[RP * RP];
  double v[RP];
  double w[RP];
  double scal[2];
  float red[32];
};

// Shared memory of one Lipschitz CTA: H in FP64, then the squaring scratch.
template <int RP>
__host__ __device__ constexpr size_t lip_smem_bytes() {
  return (size_t)RP * RP * sizeof(double) + sizeof(LmaxSmem<RP>);
}

template <typename TT, int RP>
__device__ double lmax_rp(const double* Hs, int R, LmaxSmem<RP>* s) {
  // Hs: H in FP64 (read only when TT is double); s->Hf: H in FP32
  constexpr int RR = RP * RP;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  __syncthreads();
  // every thread forms the trace (the same sum in the same order) and its inverse
  float tr = 0.f;
  for (int i = 0; i < R; ++i) tr += s->Hf[i * R + i];
  if (!isfinite(tr)) return (double)tr;
  if (!(tr > 0.f)) return 0.0;
  const float itr = 1.f / tr;
  for (int e = tid; e < RR; e += nt) {
    const int i = e / RP, j = e % RP;
    s->A[e] = (i < R && j < R) ? s->Hf[i * R + j] * itr : 0.f;
  }
  __syncthreads();
  for (int it = 0; it < 32; ++it) {
    for (int e = tid; e < RR; e += nt) {
      const int i = e / RP, j = e % RP;
      float acc = 0.f;
#pragma unroll
      for (int l = 0; l < RP; ++l) acc = fmaf(s->A[i * RP + l], s->A[l * RP + j], acc);
      s->B[e] = acc;
    }
    __syncthreads();
    float trb = 0.f;
#pragma unroll
    for (int i = 0; i < RP; ++i) trb += s->B[i * RP + i];
    float dmax = 0.f;
    if (trb > 0.f) {
      for (int e = tid; e < RR; e += nt) {
        const float nv = s->B[e] / trb;
        dmax = fmaxf(dmax, fabsf(nv - s->A[e]));
        s->A[e] = nv;
      }
    }
    if ((it & 3) != 3 && trb > 0.f) {
      __syncthreads();
      continue;
    }
    // every fourth squaring: CTA max of the last change
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((tid & 31) == 0) s->red[tid >> 5] = dmax;
    __syncthreads();
    float m = 0.f;
    for (int i = 0; i < (nt + 31) / 32; ++i) m = fmaxf(m, s->red[i]);
    __syncthreads();
    if (!(trb > 0.f) || m < 4e-6f) break;
  }
  // v: the column of the limit with the largest diagonal entry; warp 0 forms
  // the Rayleigh quotient v^T H v / v^T v
  int jm = 0;
  float dm = -1.f;
  for (int i = 0; i < R; ++i)
    if (s->A[i * RP + i] > dm) { dm = s->A[i * RP + i]; jm = i; }
  if (tid < 32) {
    TT num = TT(0), den = TT(0);
    for (int i = tid; i < R; i += 32) {
      const TT vi = (TT)s->A[i * RP + jm];
      TT acc = TT(0);
      if constexpr (sizeof(TT) == 4) {
        for (int l = 0; l < R; ++l) acc = fma(s->Hf[i * R + l], s->A[l * RP + jm], acc);
      } else {
        for (int l = 0; l < R; ++l) acc = fma(Hs[i * R + l], (TT)s->A[l * RP + jm], acc);
      }
      num = fma(vi, acc, num);
      den = fma(vi, vi, den);
    }
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (tid == 0) s->v[0] = den > TT(0) ? (double)(num / den) : 0.0;
  }
  __syncthreads();
  const double L = s->v[0];
  __syncthreads();
  return L;
}

template <typename KernelT>
static cudaError_t allow_smem(KernelT kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename TT>
__device__ __forceinline__ TT extrap_weight(double w_hat, int have_prev, double Lprev, double Lcur, double delta_w) {
  // Eqs. eqextrawd / eqextrawu; first iteration reads the ratio as 1.  TT is
  // the factor precision (FP32 on the FP32 path; FP64 is slow on this part).
  if (!(Lcur > 0.0)) return TT(0);
  const TT ratio = have_prev ? (TT)Lprev / (TT)Lcur : TT(1);
  return min((TT)w_hat, (TT)delta_w * sqrt(ratio));
}

// ---------------------------------------------------------------------------
// Grams G = U^T U (Table II operation 1).  The rows of U^(n,k) are cut into
// chunks of gr[n] rows.  For every chunk and every entry (a, b) an FMA chain
// in the factor type runs over the chunk's rows in order and is stored in
// FP64; the Gram is the sum of the chunk values in chunk order, in FP64.  The
// update kernel writes the chunk values of the mode it has just updated, the
// next kernel that needs the Gram adds them up; k_gram_chunks /
// k_gram_reduce do both for whole factors.  Every path follows the same
// order, so a Gram is bit-identical wherever it is formed.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T gram_chain(const T* U, int64_t row0, int rows, int R, int a, int b) {
  // plain loads: the update kernel reads rows it has just written
  T s = T(0);
  for (int i = 0; i < rows; ++i) s = fma(U[(row0 + i) * R + a], U[(row0 + i) * R + b], s);
  return s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gram_chunks(const DevDesc* __restrict__ d, int n0, int n1) {
  const int nm = n1 - n0;
  const int k = blockIdx.y / nm, n = n0 + blockIdx.y % nm;
  const int c = blockIdx.x;
  const int gr = d->gr[n];
  const int64_t I = d->dims[k][n];
  const int64_t row0 = (int64_t)c * gr;
  if (c >= d->gnc[n] || row0 >= I) return;
  const int rows = (int)min((int64_t)gr, I - row0);
  const int R = d->R[k];
  const int rr = d->Rmax * d->Rmax;
  const T* U = reinterpret_cast<const T*>(d->U1[k][n]);
  T* out = reinterpret_cast<T*>(d->Gp[n]) + ((size_t)k * d->gnc[n] + c) * rr;
  for (int p = threadIdx.x; p < R * R; p += blockDim.x) out[p] = gram_chain<T>(U, row0, rows, R, p / R, p % R);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gram_reduce(const DevDesc* __restrict__ d, int n0, int n1) {
  const int nm = n1 - n0;
  const int k = blockIdx.x / nm, n = n0 + blockIdx.x % nm;
  const int R = d->R[k];
  const int rr = d->Rmax * d->Rmax;
  const int nch = (int)((d->dims[k][n] + d->gr[n] - 1) / d->gr[n]);
  const T* gp = reinterpret_cast<const T*>(d->Gp[n]) + (size_t)k * d->gnc[n] * rr;
  double* G = d->G[k][n];
  for (int p = threadIdx.x; p < R * R; p += blockDim.x) G[p] = gram_sum<T>(gp, nch, rr, p);
}

// Gram of one I x R factor by one CTA (factors without chunk partials: the
// LRA factors and the ALS step): U staged through shared memory, FMA chains
// in the factor type over tiles of GRAM_TILE rows, tile sums added in FP64.
constexpr int GRAM_TILE = 64;

template <typename T>
__device__ void block_gram(const T* __restrict__ U, int64_t I, int R, double* __restrict__ G, T* buf, int cap_rows) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  const int RR = R * R;
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  for (int64_t s0 = 0; s0 < I; s0 += cap_rows) {
    const int ns = (int)min((int64_t)cap_rows, I - s0);
    __syncthreads();
    for (int e = tid; e < ns * R; e += nt) buf[e] = U[s0 * R + e];
    __syncthreads();
    for (int t0 = 0; t0 < ns; t0 += GRAM_TILE) {
      const int n = min(GRAM_TILE, ns - t0);
      const T* tile = buf + t0 * R;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int p = q * nt + tid;
        if (p < RR) {
          const int a = p / R, b = p % R;
          T s = T(0);
#pragma unroll 4
          for (int i = 0; i < n; ++i) s = fma(tile[i * R + a], tile[i * R + b], s);
          acc[q] += (double)s;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p = q * nt + tid;
    if (p < RR) G[p] = acc[q];
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_gram_block(const DevDesc* __restrict__ d, int n_begin, int n_end, int which) {
  constexpr int CAP = (32768 / (int)sizeof(T)) / CNCPD_RMAX / GRAM_TILE * GRAM_TILE;
  __shared__ T tile[CAP * CNCPD_RMAX];
  const int nm = n_end - n_begin;
  const int k = blockIdx.x / nm;
  const int n = n_begin + blockIdx.x % nm;
  const T* U = reinterpret_cast<const T*>(which ? d->Ut[k][n] : d->U1[k][n]);
  const int R = which ? d->Rt[k] : d->R[k];
  double* G = which ? d->Gt[k][n] : d->G[k][n];
  block_gram<T>(U, d->dims[k][n], R, G, tile, CAP * CNCPD_RMAX / R / GRAM_TILE * GRAM_TILE);
}

cudaError_t launch_gram(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n_begin, int n_end,
                        int which) {
  if (n_end <= n_begin) return cudaSuccess;
  const int nm = n_end - n_begin;
  if (which == 0 && hd.Gp[n_begin]) {
    int cmax = 1;
    for (int n = n_begin; n < n_end; ++n) cmax = std::max(cmax, hd.gnc[n]);
    dim3 grid((unsigned)cmax, (unsigned)(hd.K * nm));
    if (fp64) {
      carve<k_gram_chunks<double>>();
      k_gram_chunks<double><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end);
    } else {
      carve<k_gram_chunks<float>>();
      k_gram_chunks<float><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (fp64) {
      carve<k_gram_reduce<double>>();
      k_gram_reduce<double><<<hd.K * nm, 256, 0, c.stream>>>(dd, n_begin, n_end);
    } else {
      carve<k_gram_reduce<float>>();
      k_gram_reduce<float><<<hd.K * nm, 256, 0, c.stream>>>(dd, n_begin, n_end);
    }
    return cudaGetLastError();
  }
  const int grid = hd.K * nm;
  if (fp64) k_gram_block<double><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end, which);
  else k_gram_block<float><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end, which);
  return cudaGetLastError();
}

// Update kernel geometry of one mode.  When K * RP <= 512 and the shared
// memory fits, one CTA covers (column, block, row) with RP * K * TY threads
// (k_update_kp); otherwise RP * (128 / RP) threads walk the blocks
// (k_update).  A CTA handles gr = TY * passes rows -- enough passes that no
// block has more than 32 Gram chunks -- and gr is also the Gram chunk size.
struct UpdGeom {
  int kp, ty, gr;
  size_t smem;
};

static UpdGeom update_geometry(int RP, int K, int64_t imax, size_t es) {
  UpdGeom g{};
  auto rows = [&](int ty) {
    const int64_t passes = std::max<int64_t>(1, ((imax + ty - 1) / ty + 31) / 32);
    return (int)(ty * passes);
  };
  if (RP * K <= 512) {
    g.ty = std::min(64, std::max(1, 512 / (RP * K)));
    g.gr = rows(g.ty);
    g.smem = ((size_t)K * RP * RP + 2 * (size_t)g.ty * K * RP + (size_t)K * g.gr * RP) * es;
    if (g.smem <= 200 * 1024) {
      g.kp = 1;
      return g;
    }
  }
  g.kp = 0;
  g.ty = std::max(1, 128 / RP);
  g.gr = rows(g.ty);
  g.smem = 0;
  return g;
}

int gram_chunk_rows(int RP, int K, int64_t imax, int fp64) {
  return update_geometry(RP, K, imax, fp64 ? 8 : 4).gr;
}

// ---------------------------------------------------------------------------
// H^(n,k) = D (*_{m != n} G^(m,k)) D (Eq. solapgU first term; Table II
// operation 4) and L_u^(n,k) = ||H||_2 (Eq. eqLipsLu).  One CTA per block;
// the Gram of the mode updated just before is first summed from its chunks.
// ---------------------------------------------------------------------------
template <typename T, int RP>
__device__ void lip_body(const LipArgs<T>& a, int k, unsigned char* smem) {
  double* Hs = reinterpret_cast<double*>(smem);
  LmaxSmem<RP>* ls = reinterpret_cast<LmaxSmem<RP>*>(smem + (size_t)RP * RP * sizeof(double));
  const int R = a.R[k], N = a.N, rr = a.rr, n = a.n, prev = a.prev;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* Gk = a.G + (size_t)k * N * rr;
  DevScalars* sc = a.sc;
  const int nch = prev >= 0 ? (a.Iprev[k] + a.gr_prev - 1) / a.gr_prev : 0;
  const T* gp = prev >= 0 ? a.Gp_prev + (size_t)k * a.gnc_prev * rr : nullptr;
  if (a.begin) {
    // Iteration bookkeeping (Appendix A): t_k, hat w, and the Lipschitz
    // constants of the last accepted sweep become L_{k-2}.  This CTA's own
    // L^(n,k) is copied by the thread that overwrites it below; CTA 0 does
    // the rest.  Every reader of these values runs after this kernel.
    const int have_cur = sc->have_cur;
    if (tid == 0 && have_cur) sc->Lprev_u[n][k] = sc->Lcur_u[n][k];
    if (k == 0) {
      const int K = a.K;
      for (int e = tid; e < N * K; e += nt) {
        const int m = e / K, kk = e % K;
        if (m != n && have_cur) sc->Lprev_u[m][kk] = sc->Lcur_u[m][kk];
      }
      for (int m = tid; m < N; m += nt)
        if (have_cur) sc->LCprev[m] = sc->LCcur[m];
      // the last thread (idle in the H loop below while R^2 < nt) takes the
      // momentum step, off the critical path of thread 0
      if (tid == nt - 1) {
        const double t = sc->t;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        sc->w_hat = (t - 1.0) / tn;
        sc->t = tn;
        if (have_cur) sc->have_prev = 1;
      }
    }
  }
  for (int p = tid; p < R * R; p += nt) {
    double gm[CNCPD_NMAX];
#pragma unroll
    for (int m = 0; m < CNCPD_NMAX; ++m) gm[m] = (m < N && m != n && m != prev) ? Gk[(size_t)m * rr + p] : 1.0;
    if (prev >= 0) {
      const double g = gram_sum<T>(gp, nch, rr, p);
      Gk[(size_t)prev * rr + p] = g;
#pragma unroll
      for (int m = 0; m < CNCPD_NMAX; ++m)
        if (m == prev && m != n) gm[m] = g;
    }
    double h = 1.0;
#pragma unroll
    for (int m = 0; m < CNCPD_NMAX; ++m)
      if (m < N && m != n) h *= gm[m];
    if (a.use_core) h *= sc->lam1[k][p / R] * sc->lam1[k][p % R];
    if constexpr (sizeof(T) == 8) Hs[p] = h;
    ls->Hf[p] = (float)h;
    a.H[(size_t)k * rr + p] = (T)h;
    a.H64[(size_t)k * rr + p] = h;
  }
  if (!a.want_L) return;
  const double L = lmax_rp<T, RP>(Hs, R, ls);
  if (tid == 0) {
    sc->Lcur_u[n][k] = L;
    if (!isfinite(L)) atomicExch(&sc->nonfinite, 1);
  }
}

template <typename T, int RP>
__global__ void __launch_bounds__(256) k_lipschitz(const __grid_constant__ LipArgs<T> a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  lip_body<T, RP>(a, blockIdx.x, smem_raw);
}

// Level 2 of a two-mode group (third- and fourth-order tensors).  With n
// first in its group, P[i_n][b][r] is contiguous per i_n:
//   M[i_n, r] = sum_b P[i_n, b, r] W[b, r];
// thread t keeps r = t mod R and strides over (b, r) by a multiple of R; a
// CTA produces ni rows.  With n last, P[a][i_n][r]:
//   M[i_n, r] = sum_a P[a, i_n, r] W[a, r];
// a CTA produces ni*R consecutive outputs (a contiguous run of every P[a]),
// thread (e, slice) summing output e over the slice's a values; the slices
// are added in order.
template <typename T>
__device__ void pair_body(const PairArgs<T>& a, int b, T* red) {
  int k = 0;
  while (k + 1 < a.K && a.cta0[k + 1] <= b) ++k;
  const int bx = b - a.cta0[k];
  const int In = a.In[k], Io = a.Io[k], R = a.R[k];
  const int i0 = bx * a.ni;
  if (i0 >= In) return;
  const int ni = min(a.ni, In - i0);
  const T* __restrict__ P = a.P[k];
  const T* __restrict__ W = a.W[k];
  T* M = a.M[k];
  const int t = threadIdx.x;
  if (a.first) {
    // ni <= 2 rows; 12 columns e of the (b, r) range per batch, all loads first
    const int BR = Io * R;
    const int stride = (256 / R) * R;
    T acc0 = T(0), acc1 = T(0);
    if (t < stride) {
      const T* P0 = P + (int64_t)i0 * BR;
      const T* P1 = ni > 1 ? P0 + BR : P0;
      for (int e0 = t; e0 < BR; e0 += 12 * stride) {
        T wv[12], p0v[12], p1v[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) {
          const int e = min(e0 + j * stride, BR - 1);  // clamped: every load issues at once
          wv[j] = W[e];
          p0v[j] = P0[e];
          p1v[j] = P1[e];
        }
#pragma unroll
        for (int j = 0; j < 12; ++j)
          if (e0 + j * stride < BR) {
            acc0 = fma(p0v[j], wv[j], acc0);
            acc1 = fma(p1v[j], wv[j], acc1);
          }
      }
    }
    red[t] = acc0;
    red[256 + t] = acc1;
    __syncthreads();
    if (t < ni * R) {
      const int q = t / R, r = t % R;
      T s = T(0);
      for (int u = r; u < stride; u += R) s += red[q * 256 + u];
      M[(int64_t)(i0 + q) * R + r] = s;
    }
  } else {
    // outputs e < ni*R of rows i0 .. i0+ni-1, the a range cut into nsl slices;
    // 12 a per batch
    const int OF = a.ni * R, nsl = a.nsl;
    const int e = t % OF, sl = t / OF;
    T acc = T(0);
    if (sl < nsl && e < ni * R) {
      const T* Pe = P + (int64_t)i0 * R + e;
      const T* We = W + e % R;
      const int64_t ps = (int64_t)In * R;
      for (int x0 = sl; x0 < Io; x0 += 12 * nsl) {
        T pv[12], wv[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          const int x = min(x0 + q * nsl, Io - 1);  // clamped: every load issues at once
          pv[q] = Pe[(int64_t)x * ps];
          wv[q] = We[x * R];
        }
#pragma unroll
        for (int q = 0; q < 12; ++q)
          if (x0 + q * nsl < Io) acc = fma(pv[q], wv[q], acc);
      }
    }
    red[t] = acc;
    __syncthreads();
    if (t < ni * R) {
      T s = T(0);
      for (int u = 0; u < nsl; ++u) s += red[u * OF + t];
      M[(int64_t)i0 * R + t] = s;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_level2_pair(const __grid_constant__ PairArgs<T> a) {
  pdl_wait();
  pdl_trigger();
  __shared__ T red[8 * 256];
  pair_body<T>(a, blockIdx.x, red);
}

// CTAs [0, K): H and L of mode n, block blockIdx.x; the rest: level 2.
template <typename T, int RP>
__global__ void __launch_bounds__(256, 4) k_mode_prep(const __grid_constant__ LipArgs<T> la,
                                                   const __grid_constant__ PairArgs<T> pa) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if ((int)blockIdx.x < la.K) lip_body<T, RP>(la, blockIdx.x, smem_raw);
  else pair_body<T>(pa, blockIdx.x - la.K, reinterpret_cast<T*>(smem_raw));
}

bool level2_is_pair(const DevDesc& hd, int n) {
  const int gsize = (n < hd.h) ? hd.h : hd.N - hd.h;
  return gsize == 2;
}

template <typename T>
static LipArgs<T> lip_args(const DevDesc& hd, int n, int use_core, int prev, int want_L, int begin = 0) {
  LipArgs<T> a{};
  a.begin = begin;
  a.K = hd.K;
  a.N = hd.N;
  a.n = n;
  a.prev = (prev >= 0 && hd.Gp[prev]) ? prev : -1;
  a.use_core = use_core;
  a.want_L = want_L;
  a.rr = hd.Rmax * hd.Rmax;
  a.sc = hd.sc;
  a.G = hd.Gbase;
  a.H = reinterpret_cast<T*>(hd.Hbase);
  a.H64 = hd.H64base;
  if (a.prev >= 0) {
    a.Gp_prev = reinterpret_cast<const T*>(hd.Gp[prev]);
    a.gnc_prev = hd.gnc[prev];
    a.gr_prev = hd.gr[prev];
  }
  for (int k = 0; k < hd.K; ++k) {
    a.R[k] = hd.R[k];
    a.Iprev[k] = a.prev >= 0 ? (int)hd.dims[k][prev] : 0;
  }
  return a;
}

template <typename T>
static PairArgs<T> pair_args(const DevDesc& hd, int n, int num_sms, int* ctas) {
  PairArgs<T> a{};
  const int h = hd.h;
  const int m0 = (n < h) ? 0 : h;
  const int other = (n == m0) ? n + 1 : m0;
  a.K = hd.K;
  a.first = (n == m0);
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = std::max<int64_t>(imax, hd.dims[k][n]);
  int ni;
  if (a.first) {
    // one or two rows per CTA: two unless that leaves fewer than ~4 CTAs per SM
    ni = ((imax + 1) / 2) * hd.K >= 4LL * num_sms ? 2 : 1;
  } else {
    // about 24 a values per thread; the rest of the 256 threads take more rows
    int iomax = 1, rmax = 1;
    for (int k = 0; k < hd.K; ++k) {
      iomax = std::max<int>(iomax, (int)hd.dims[k][other]);
      rmax = std::max(rmax, hd.R[k]);
    }
    a.nsl = std::max(1, std::min((iomax + 23) / 24, 256 / rmax));
    ni = std::max(1, 256 / (rmax * a.nsl));
  }
  a.ni = ni;
  int tot = 0;
  for (int k = 0; k < hd.K; ++k) {
    a.In[k] = (int)hd.dims[k][n];
    a.Io[k] = (int)hd.dims[k][other];
    a.R[k] = hd.R[k];
    a.cta0[k] = tot;
    // no CTAs for a block whose tensor pass had no units (inactive in a
    // restricted descriptor): its level-1 product is not new
    const bool act = (n < h) ? hd.lt_prefix[k + 1] > hd.lt_prefix[k] : hd.tt_prefix[k + 1] > hd.tt_prefix[k];
    if (act) tot += (int)((hd.dims[k][n] + ni - 1) / ni);
    a.P[k] = reinterpret_cast<const T*>((n < h) ? hd.Pl[k] : hd.Pt[k]);
    a.W[k] = reinterpret_cast<const T*>(hd.U1[k][other]);
    a.M[k] = reinterpret_cast<T*>(hd.M[k][n]);
  }
  a.cta0[hd.K] = tot;
  *ctas = tot;
  return a;
}

template <typename T, int RP>
static cudaError_t mode_prep_impl(const LaunchCfg& c, const DevDesc& hd, int n, int use_core, int prev,
                                  int with_level2, int begin) {
  // with_level2: 0 = Lipschitz only, 1 = Lipschitz + level 2, 2 = level 2 only
  int ctas = 0;
  PairArgs<T> pa{};
  if (with_level2) pa = pair_args<T>(hd, n, c.num_sms, &ctas);
  if (with_level2 == 2) {
    if (ctas == 0) return cudaSuccess;
    carve<k_level2_pair<T>>();
    cudaError_t el = launch_pdl(k_level2_pair<T>, dim3(ctas), dim3(256), 0, c.stream, pa);
    if (el != cudaSuccess) return el;
    return cudaGetLastError();
  }
  LipArgs<T> la = lip_args<T>(hd, n, use_core, prev, 1, begin);
  const size_t sm = std::max(lip_smem_bytes<RP>(), with_level2 ? sizeof(T) * 8 * 256 : (size_t)0);
  if (with_level2 == 0) {
    cudaError_t e = allow_smem(k_lipschitz<T, RP>, sm);
    if (e != cudaSuccess) return e;
    carve<k_lipschitz<T, RP>>();
    e = launch_pdl(k_lipschitz<T, RP>, dim3(hd.K), dim3(RP <= 16 ? 128 : 256), sm, c.stream, la);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  cudaError_t e = allow_smem(k_mode_prep<T, RP>, sm);
  if (e != cudaSuccess) return e;
  carve<k_mode_prep<T, RP>>();
  e = launch_pdl(k_mode_prep<T, RP>, dim3(hd.K + ctas), dim3(256), sm, c.stream, la, pa);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

static int rank_bucket_of(const DevDesc& hd) { return rank_bucket(hd.Rmax); }

static cudaError_t mode_prep_any(const LaunchCfg& c, const DevDesc& hd, int fp64, int n, int use_core, int prev,
                                 int with_level2, int begin) {
#define MCASE(V)                                                                                       \
  case V:                                                                                              \
    return fp64 ? mode_prep_impl<double, V>(c, hd, n, use_core, prev, with_level2, begin)              \
                : mode_prep_impl<float, V>(c, hd, n, use_core, prev, with_level2, begin);
  switch (rank_bucket_of(hd)) { CNCPD_FOR_EACH_RP(MCASE) }
#undef MCASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_mode_prep(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n, int use_core,
                             int prev, int with_level2, int begin) {
  (void)dd;
  return mode_prep_any(c, hd, fp64, n, use_core, prev, with_level2, begin);
}

cudaError_t launch_lipschitz(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n, int use_core,
                             int prev, int begin) {
  (void)dd;
  return mode_prep_any(c, hd, fp64, n, use_core, prev, 0, begin);
}

// H of mode n for every block, without L (the gradient path).
template <typename T, int RP>
static cudaError_t hmat_impl(const LaunchCfg& c, const DevDesc& hd, int n, int use_core) {
  LipArgs<T> la = lip_args<T>(hd, n, use_core, -1, 0);
  const size_t sm = lip_smem_bytes<RP>();
  cudaError_t e = allow_smem(k_lipschitz<T, RP>, sm);
  if (e != cudaSuccess) return e;
  carve<k_lipschitz<T, RP>>();
  k_lipschitz<T, RP><<<hd.K, 256, sm, c.stream>>>(la);
  return cudaGetLastError();
}

static cudaError_t launch_hmat(const LaunchCfg& c, const DevDesc& hd, int fp64, int n, int use_core) {
#define HCASE(V) \
  case V: return fp64 ? hmat_impl<double, V>(c, hd, n, use_core) : hmat_impl<float, V>(c, hd, n, use_core);
  switch (rank_bucket_of(hd)) { CNCPD_FOR_EACH_RP(HCASE) }
#undef HCASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Fused update of mode n for every block (Eqs. eqextraPU, solapgU, solUns,
// solUnC, solUnsI):
//   U_hat = U1 + w (U1 - U2)            (shared columns: one weight w_C)
//   G_hat = U_hat H - M D
//   individual columns: U1 <- P(U_hat - G_hat / L_u^(n,k))
//   shared columns:     U1 <- P(U_hat_C - sum_k G_hat_C / sum_k L_u^(n,k)),
//                       the same value written to every block
//   U2 <- old U1,
// then the Gram chunk values of the new rows (one chunk per CTA).  Thread
// (c, y) owns column c of row y of each pass over the CTA's rows and walks
// the blocks in chunks of KC, keeping the shared-column gradient sum in a
// register, so the coupled sum needs no cross-CTA communication.  Rows are
// owned by exactly one CTA, so the in-place write is race free.
// ---------------------------------------------------------------------------
template <typename T, int RP>
struct UpdCfg {
  static constexpr int ROWS = (128 / RP) > 0 ? 128 / RP : 1;
  static constexpr int KC_ = (int)((10240 * 4 / sizeof(T)) / (RP * RP));
  static constexpr int KC = KC_ < 1 ? 1 : (KC_ > 8 ? 8 : KC_);
};

template <typename T, int RP>
__global__ void __launch_bounds__(128) k_update(const __grid_constant__ UpdArgs<T> a) {
  pdl_wait();
  pdl_trigger();
  constexpr int TY = UpdCfg<T, RP>::ROWS;
  constexpr int KC = UpdCfg<T, RP>::KC;
  constexpr int NT = RP * TY;
  __shared__ T Hs[KC][RP * RP];
  __shared__ T uh[KC][TY][RP];
  __shared__ T wsh[CNCPD_KMAX + 1];
  __shared__ T Lsh[CNCPD_KMAX];
  __shared__ double LCs;
  // new rows of the CTA for the Gram chunk values (all blocks in one chunk
  // of KC; otherwise null and the rows are read back from global memory)
  extern __shared__ __align__(16) unsigned char nv_raw[];
  T* nvs = a.stage_rows ? reinterpret_cast<T*>(nv_raw) : nullptr;

  const int c = threadIdx.x;
  const int y = threadIdx.y;
  const int tid = c + y * RP;
  const int K = a.K, n = a.n, Ln = a.Ln;
  DevScalars* sc = a.sc;
  const int64_t row0 = (int64_t)blockIdx.x * a.gr;
  const int nchunk = (K + KC - 1) / KC;

  // H of the first chunk of blocks (all of them when K <= KC)
  auto load_h = [&](int k0) {
    for (int e = tid; e < KC * RP * RP; e += NT) {
      const int kk = e / (RP * RP), q = e % (RP * RP);
      const int k = k0 + kk;
      const int ra = q / RP, rb = q % RP;
      T v = T(0);
      if (k < K) {
        const int R = a.R[k];
        if (ra < R && rb < R) v = a.H[k][ra * R + rb];
      }
      Hs[kk][q] = v;
    }
  };
  load_h(0);
  {
    // extrapolation weights (Eqs. eqextrawu and reading R3) and L, one
    // evaluation per block
    const double w_hat = a.use_w ? sc->w_hat : 0.0;
    const int have_prev = sc->have_prev;
    for (int k = tid; k < K; k += NT) {
      const double Lc = sc->Lcur_u[n][k];
      wsh[k] = extrap_weight<T>(w_hat, have_prev, sc->Lprev_u[n][k], Lc, a.delta_w);
      Lsh[k] = Lc > 0.0 ? (T)Lc : T(0);
    }
    if (tid == 0) {
      double LC = 0.0;
      for (int k = 0; k < K; ++k) LC += sc->Lcur_u[n][k];
      LCs = LC;
      wsh[K] = extrap_weight<T>(w_hat, have_prev, sc->LCprev[n], LC, a.delta_w);
      if (blockIdx.x == 0) {
        sc->LCcur[n] = LC;
        sc->have_cur = 1;
      }
    }
  }
  __syncthreads();
  const double LC = LCs;
  const T wC = wsh[K];

  for (int p0 = 0; p0 < a.gr; p0 += TY) {
    const int64_t i = (p0 + y < a.gr) ? row0 + p0 + y : INT64_MAX;  // rows past the chunk belong to the next CTA
    T sumC = T(0), uhC = T(0), u1C = T(0), u2C = T(0);
    for (int k0 = 0; k0 < K; k0 += KC) {
      if (nchunk > 1) {
        __syncthreads();
        load_h(k0);
      }
      T u1[KC], u2[KC], mv[KC];
      T lam[KC];
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        const int k = k0 + kk;
        u1[kk] = u2[kk] = mv[kk] = T(0);
        lam[kk] = T(1);
        const bool valid = k < K && i < a.I[k] && c < a.R[k];
        if (valid) {
          const int R = a.R[k];
          u1[kk] = a.U1[k][i * R + c];
          u2[kk] = a.U2[k][i * R + c];
          if (a.part[0]) {
            mv[kk] = sum_splits<T>(a.part[k] + i * R + c, a.nsplit[k], (int64_t)a.I[k] * R);
            a.M[k][i * R + c] = mv[kk];
          } else {
            mv[kk] = a.M[k][i * R + c];
          }
          if (a.use_core) lam[kk] = (T)sc->lam1[k][c];
        }
        const T w = (c < Ln) ? wC : (k < K ? wsh[k] : T(0));
        uh[kk][y][c] = valid ? u1[kk] + w * (u1[kk] - u2[kk]) : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        const int k = k0 + kk;
        if (k < K && i < a.I[k] && c < a.R[k]) {
          const int R = a.R[k];
          const T uhat = uh[kk][y][c];
          T g = -mv[kk] * lam[kk];
#pragma unroll
          for (int q = 0; q < RP; ++q) g = fma(uh[kk][y][q], Hs[kk][q * RP + c], g);
          if (c >= Ln) {
            T nv = u1[kk];
            const T Lk = Lsh[k];
            if (Lk > T(0)) {
              nv = uhat - g / Lk;
              if (a.nonneg) nv = nv > T(0) ? nv : T(0);
            }
            a.S[k][i * R + c] = u2[kk];
            a.U2[k][i * R + c] = u1[kk];
            a.U1[k][i * R + c] = nv;
            if (nvs) nvs[((size_t)kk * a.gr + p0 + y) * RP + c] = nv;
          } else {
            sumC += g;
            uhC = uhat;
            u1C = u1[kk];
            u2C = u2[kk];
          }
        }
      }
      __syncthreads();
    }
    if (c < Ln && i < a.I[0]) {
      T nv = u1C;
      if (LC > 0.0) {
        nv = uhC - sumC / (T)LC;
        if (a.nonneg) nv = nv > T(0) ? nv : T(0);
      }
      for (int k = 0; k < K; ++k) {
        const int R = a.R[k];
        a.S[k][i * R + c] = u2C;
        a.U2[k][i * R + c] = u1C;
        a.U1[k][i * R + c] = nv;
        if (nvs) nvs[((size_t)k * a.gr + p0 + y) * RP + c] = nv;
      }
    }
  }
  if (!a.Gp) return;
  __syncthreads();  // the CTA's new rows are visible to the whole CTA
  for (int e = tid; e < K * RP * RP; e += NT) {
    const int k = e / (RP * RP), q = e % (RP * RP);
    const int ra = q / RP, rb = q % RP;
    const int R = a.R[k];
    const int64_t I = a.I[k];
    if (ra < R && rb < R && row0 < I) {
      const int rows = (int)min((int64_t)a.gr, I - row0);
      T gv;
      if (nvs) {
        const T* Uk = nvs + (size_t)k * a.gr * RP;
        gv = T(0);
        for (int ii = 0; ii < rows; ++ii) gv = fma(Uk[ii * RP + ra], Uk[ii * RP + rb], gv);
      } else {
        gv = gram_chain<T>(a.U1[k], row0, rows, R, ra, rb);
      }
      a.Gp[((size_t)k * a.gnc + blockIdx.x) * a.rr + ra * R + rb] = gv;
    }
  }
}

// Objective of Eq. costfunc at the end of the last mode's update, by the last
// CTA to finish (the other CTAs' Gram chunk values of mode n and <M, U_new>
// sums are read through L2).  Full warps take the blocks; per block the
// lanes sum the Gram of mode n from its chunks (stored as G^(n,k)), the
// lambda^T (*_m G^(m)) lambda terms and lambda^T c with c the column sums of
// <M, U_new> (the next core term); warp 0 then adds the blocks up in order.
// Objective of Eq. costfunc after the last mode's update, run by the last
// CTA of that update to finish (every CTA has left its <M, U_new> column
// sums and its share of ||X_hat||^2):
//   ||X_hat^(k)||^2 = <H^(n,k), G^(n,k)> = sum over CTAs c of
//     <H^(n,k), chunk c of G^(n,k)>, H^(n,k) = D (*_{m != n} G^(m,k)) D in
//     FP64 from the Lipschitz kernel of this mode, the shares added in CTA
//     order;
//   <X^(k), X_hat^(k)> = sum_r lambda_r (M^(n,k)^T U^(n,k))_{rr}, the column
//     sums added in CTA order (also kept as the core term);
//   F_k = (||X||^2 - 2 <X, X_hat> + ||X_hat||^2) / 2, RelErr_k = sqrt(2 F_k) / ||X||.
// Each block's terms are added by one warp in a fixed order, so the result
// does not depend on timing.  G^(n) itself is summed from its chunks by the
// next sweep's first Lipschitz launch, or here when the cores are updated
// (their update at the start of the next sweep reads it).
template <typename T, int RP>
__device__ void update_objective_tail(const UpdArgs<T>& a, int tid, int NT, unsigned char* smem) {
  constexpr int RR = RP * RP;
  const int K = a.K, N = a.N, n = a.n, rr = a.rr;
  DevScalars* sc = a.sc;
  double* xb = reinterpret_cast<double*>(smem);  // [K][RR]: H * G_new
  double* ib = xb + (size_t)K * RR;              // [K][RP]: lambda * core term
  double* fk = ib + (size_t)K * RP;              // [K]
  double* rk = fk + K;                           // [K]
  double x2 = 0.0, ix2 = 0.0;
  if (tid < K) {
    x2 = sc->xnorm2[tid];
    ix2 = sc->inv_xnorm2[tid];
  }
  // what the publish at the end reads, loaded now: the flags are only set by
  // earlier kernels (and below, by this thread, when F is not finite)
  unsigned int seq0 = 0;
  int nonfinite0 = 0, timeout0 = 0;
  if (tid == 0) {
    seq0 = *((volatile unsigned int*)&sc->seq);
    nonfinite0 = *((volatile int*)&sc->nonfinite);
    timeout0 = *((volatile int*)&sc->timeout);
  }
  if (a.gram_last) {
    // G^(n) for the next sweep's core update, summed from its chunks
    for (int e = tid; e < K * RR; e += NT) {
      const int kk = e / RR, q = e % RR, ra = q / RP, rb = q % RP;
      const int Rk = a.R[kk];
      if (ra < Rk && rb < Rk) {
        const int p = ra * Rk + rb;
        const int nch = (a.I[kk] + a.gr - 1) / a.gr;
        a.G[((size_t)kk * N + n) * rr + p] = gram_sum<T, true>(a.Gp + (size_t)kk * a.gnc * rr, nch, rr, p);
      }
    }
  }
  // ||X_hat^(k)||^2: the CTAs' shares in CTA order (a warp per block below)
  const int nct = (int)gridDim.x;
  for (int e = tid; e < K * RR; e += NT) {
    const int kk = e / RR, c0 = e % RR;
    xb[e] = c0 < nct ? __ldcg(a.xxp + (size_t)c0 * K + kk) : 0.0;
  }
  for (int e = tid; e < K * RP; e += NT) {
    const int kk = e / RP, cc = e % RP;
    double v = 0.0;
    if (cc < a.R[kk]) {
      const double lam = sc->lam1[kk][cc];
      const double cr = gram_sum<T, true>(a.dotp + (size_t)kk * RP, (int)gridDim.x, K * RP, cc);
      sc->cterm[kk][cc] = cr;
      v = lam * cr;
    }
    ib[e] = v;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, nw = NT >> 5;  // whole warps only
  if (warp < nw) {
    for (int kk = warp; kk < K; kk += nw) {
      double xx = 0.0, ip = 0.0;
      for (int q = lane; q < min(RR, nct); q += 32) xx += xb[(size_t)kk * RR + q];
      for (int q = lane; q < RP; q += 32) ip += ib[(size_t)kk * RP + q];
      for (int o = 16; o > 0; o >>= 1) {
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
        ip += __shfl_xor_sync(0xffffffffu, ip, o);
      }
      if (lane == 0) {
        fk[kk] = xx;
        rk[kk] = ip;
      }
    }
  }
  __syncthreads();
  if (tid < K) {
    const double Fk = 0.5 * (x2 + fk[tid] - 2.0 * rk[tid]);
    const double rel = sqrt(fmax(2.0 * Fk, 0.0) * ix2);
    sc->Fk[tid] = Fk;
    sc->relk[tid] = rel;
    fk[tid] = Fk;
    rk[tid] = rel;
  }
  __syncthreads();
  if (tid < 32) {
    double F = 0.0, rel = 0.0;
    for (int q = tid; q < K; q += 32) {
      F += fk[q];
      rel += rk[q];
    }
    for (int o = 16; o > 0; o >>= 1) {
      F += __shfl_xor_sync(0xffffffffu, F, o);
      rel += __shfl_xor_sync(0xffffffffu, rel, o);
    }
    if (tid == 0) {
      const double relerr = rel * a.inv_K;
      const int nonfinite = nonfinite0 | (isfinite(F) ? 0 : 1);
      sc->F = F;
      sc->relerr = relerr;
      if (nonfinite) sc->nonfinite = 1;
      sc->done_counter[1] = 0;
      const unsigned int q = seq0 + 1;
      sc->seq = q;
      if (a.hm) {
        HostMirror* hm = a.hm;
        hm->F = F;
        hm->relerr = relerr;
        hm->nonfinite = nonfinite;
        hm->timeout = timeout0;
        __threadfence_system();
        hm->seq = q;
      }
    }
  }
}

// Shared memory the objective tail needs (it reuses the update's).
__host__ __device__ constexpr size_t objective_tail_smem(int K, int RP) {
  return ((size_t)K * RP * RP + (size_t)K * RP + 2 * (size_t)K) * sizeof(double);
}

// The same update with one thread per (column c, block k, row y): the loads
// of a pass are issued together, the shared-column gradient sum is formed in
// shared memory in block order, and the CTA's new rows stay in shared memory
// for the Gram chunk values.
template <typename T, int RP>
__global__ void __launch_bounds__(512) k_update_kp(const __grid_constant__ UpdArgs<T> a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = a.K, Ln = a.Ln, n = a.n;
  const int c = threadIdx.x, k = threadIdx.y, y = threadIdx.z, TY = blockDim.z;
  const int tid = c + RP * (k + K * y);
  const int NT = RP * K * TY;
  T* Hs = reinterpret_cast<T*>(sm_raw);       // [K][RP][RP]
  T* uh = Hs + (size_t)K * RP * RP;           // [TY][K][RP]
  T* gC = uh + (size_t)TY * K * RP;           // [TY][K][RP]
  T* nvs = gC + (size_t)TY * K * RP;          // [K][gr][RP]
  T* mvs = nvs + (size_t)K * a.gr * RP;        // [K][gr][RP], with the fused objective
  // with the fused objective: H^(n,k) in FP64, then H * (this CTA's Gram chunk)
  double* xsb = reinterpret_cast<double*>(mvs + (size_t)K * a.gr * RP);  // [K][RP][RP]
  __shared__ T wsh[CNCPD_KMAX + 1];
  __shared__ T Lsh[CNCPD_KMAX];
  __shared__ T LCsh;
  __shared__ int is_last;
  double LCd = 0.0;  // sum_k L^(n,k), held by thread K until the end of the kernel
  DevScalars* sc = a.sc;
  const int64_t row0 = (int64_t)blockIdx.x * a.gr;
  const int R = a.R[k];
  const int64_t I = a.I[k];

  // The rows of the first pass are loaded before anything else, and with at
  // most 32 split-K partials those are loaded too (added after the staging
  // below, so that every load of the prologue is in flight at once).
  T u1_0 = T(0), u2_0 = T(0), mv_0 = T(0);
  T pv[32];
  const int64_t i_0 = row0 + y;
  const bool valid_0 = y < a.gr && i_0 < I && c < R;
  const size_t off_0 = valid_0 ? (size_t)i_0 * R + c : 0;
  const int ns_0 = a.part[0] ? a.nsplit[k] : 0;
  if (valid_0) {
    u1_0 = a.U1[k][off_0];
    u2_0 = a.U2[k][off_0];
    if (!a.part[0]) {
      mv_0 = a.M[k][off_0];
    } else if (ns_0 <= 32) {
      const T* pp = a.part[k] + off_0;
      const int64_t stride = I * R;
#pragma unroll
      for (int j = 0; j < 32; ++j) pv[j] = pp[(int64_t)min(j, ns_0 - 1) * stride];  // clamped: no predicate
    }
  }

  // H of every block (zero-padded to RP x RP)
#pragma unroll 4
  for (int e = tid; e < K * RP * RP; e += NT) {
    const int kk = e / (RP * RP), q = e % (RP * RP);
    const int ra = q / RP, rb = q % RP;
    const int Rk = a.R[kk];
    Hs[e] = (ra < Rk && rb < Rk) ? a.H[kk][ra * Rk + rb] : T(0);
    if (a.obj) xsb[e] = (ra < Rk && rb < Rk) ? a.H64[(size_t)kk * a.rr + ra * Rk + rb] : 0.0;
  }
  // extrapolation weights (Eqs. eqextrawu and reading R3), one per block
  if (tid <= K) {
    const double w_hat = a.use_w ? sc->w_hat : 0.0;
    const int have_prev = sc->have_prev;
    if (tid < K) {
      const double Lc = sc->Lcur_u[n][tid];
      wsh[tid] = extrap_weight<T>(w_hat, have_prev, sc->Lprev_u[n][tid], Lc, a.delta_w);
      Lsh[tid] = Lc > 0.0 ? (T)Lc : T(0);
    } else {
      double LC = 0.0;
#pragma unroll 8
      for (int kk = 0; kk < K; ++kk) LC += sc->Lcur_u[n][kk];
      wsh[K] = extrap_weight<T>(w_hat, have_prev, sc->LCprev[n], LC, a.delta_w);
      LCsh = LC > 0.0 ? (T)LC : T(0);
      LCd = LC;
    }
  }
  const T lam = (a.use_core && c < R) ? (T)sc->lam1[k][c] : T(1);
  if (valid_0 && a.part[0]) {
    if (ns_0 <= 32) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < ns_0) acc += pv[j];
      mv_0 = acc;
    } else {
      mv_0 = sum_splits<T>(a.part[k] + off_0, ns_0, I * R);
    }
  }
  for (int p0 = 0; p0 < a.gr; p0 += TY) {
    const bool inchunk = p0 + y < a.gr;
    const int64_t i = row0 + p0 + y;
    const bool valid = inchunk && i < I && c < R;
    const size_t off = valid ? (size_t)i * R + c : 0;
    T u1, u2, mv;
    if (p0 == 0) {
      u1 = u1_0;
      u2 = u2_0;
      mv = mv_0;
    } else {
      u1 = valid ? a.U1[k][off] : T(0);
      u2 = valid ? a.U2[k][off] : T(0);
      mv = T(0);
      if (valid) mv = a.part[0] ? sum_splits<T>(a.part[k] + off, a.nsplit[k], I * R) : a.M[k][off];
    }
    if (a.part[0] && valid) a.M[k][off] = mv;
    if (a.obj && inchunk) mvs[((size_t)k * a.gr + p0 + y) * RP + c] = mv;
    __syncthreads();  // weights and H staged; the previous pass is done with uh / gC
    const T w = (c < Ln) ? wsh[K] : wsh[k];
    const T uhat = u1 + w * (u1 - u2);
    uh[((size_t)y * K + k) * RP + c] = valid ? uhat : T(0);
    __syncthreads();
    if (valid) {
      const T* uy = uh + ((size_t)y * K + k) * RP;
      const T* Hk = Hs + (size_t)k * RP * RP + c;
      T g = -mv * lam;
#pragma unroll
      for (int q = 0; q < RP; ++q) g = fma(uy[q], Hk[q * RP], g);
      if (c >= Ln) {
        T nv = u1;
        const T Lk = Lsh[k];
        if (Lk > T(0)) {
          nv = uhat - g / Lk;
          if (a.nonneg) nv = nv > T(0) ? nv : T(0);
        }
        a.S[k][off] = u2;
        a.U2[k][off] = u1;
        a.U1[k][off] = nv;
        nvs[((size_t)k * a.gr + p0 + y) * RP + c] = nv;
      } else {
        gC[((size_t)y * K + k) * RP + c] = g;
      }
    }
    __syncthreads();
    if (k == 0 && valid && c < Ln) {
      // shared columns: one step from the sum of every block's gradient
      T s = T(0);
      for (int kk = 0; kk < K; ++kk) s += gC[((size_t)y * K + kk) * RP + c];
      T nv = u1;
      const T LC = LCsh;
      if (LC > T(0)) {
        nv = uhat - s / LC;
        if (a.nonneg) nv = nv > T(0) ? nv : T(0);
      }
      for (int kk = 0; kk < K; ++kk) {
        const size_t o = (size_t)i * a.R[kk] + c;
        a.S[kk][o] = u2;
        a.U2[kk][o] = u1;
        a.U1[kk][o] = nv;
        nvs[((size_t)kk * a.gr + p0 + y) * RP + c] = nv;
      }
    }
  }
  if (blockIdx.x == 0 && tid == K) {  // the sweep's record of sum_k L (read by later kernels only)
    sc->LCcur[n] = LCd;
    sc->have_cur = 1;
  }
  if (!a.Gp) return;
  __syncthreads();
  for (int e = tid; e < K * RP * RP; e += NT) {
    const int kk = e / (RP * RP), q = e % (RP * RP);
    const int ra = q / RP, rb = q % RP;
    const int Rk = a.R[kk];
    const int64_t Ik = a.I[kk];
    if (ra < Rk && rb < Rk && row0 < Ik) {
      const int rows = (int)min((int64_t)a.gr, Ik - row0);
      const T* Uk = nvs + (size_t)kk * a.gr * RP;
      T gv = T(0);
      for (int ii = 0; ii < rows; ++ii) gv = fma(Uk[ii * RP + ra], Uk[ii * RP + rb], gv);
      a.Gp[((size_t)kk * a.gnc + blockIdx.x) * a.rr + ra * Rk + rb] = gv;
      if (a.obj) xsb[e] *= (double)gv;
    } else if (a.obj) {
      xsb[e] = 0.0;
    }
  }
  if (!a.obj) return;
  // <M, U_new> over this CTA's rows per (block, column): thread (c, k, y)
  // takes rows y, y + TY, ..., then the TY sums are added in order
  T ds = T(0);
  for (int p = y; p < a.gr; p += TY) {
    if (row0 + p < I && c < R)
      ds = fma(mvs[((size_t)k * a.gr + p) * RP + c], nvs[((size_t)k * a.gr + p) * RP + c], ds);
  }
  gC[((size_t)y * K + k) * RP + c] = ds;  // gC is free: the update loop is done with it
  __syncthreads();
  if (y == 0) {
    T s;
    if constexpr (sizeof(T) == 4) {
      float hi = 0.f, lo = 0.f;
      for (int yy = 0; yy < TY; ++yy) ff_add(hi, lo, gC[((size_t)yy * K + k) * RP + c]);
      s = hi + lo;
    } else {
      s = T(0);
      for (int yy = 0; yy < TY; ++yy) s += gC[((size_t)yy * K + k) * RP + c];
    }
    a.dotp[((size_t)blockIdx.x * K + k) * RP + c] = s;
  }
  {
    // this CTA's share of ||X_hat^(k)||^2 = <H^(n,k), G^(n,k)>, one warp per
    // block in a fixed order (xsb was completed before the barrier above)
    const int warp = tid >> 5, lane = tid & 31, nw = NT >> 5;
    if (warp < nw) {
      for (int kk = warp; kk < K; kk += nw) {
        double v = 0.0;
        for (int q = lane; q < RP * RP; q += 32) v += xsb[(size_t)kk * RP * RP + q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) a.xxp[(size_t)blockIdx.x * K + kk] = v;
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&sc->done_counter[1], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  update_objective_tail<T, RP>(a, tid, NT, sm_raw);
}

// Shared memory of the block-parallel update with the fused objective (the
// rows of M staged next to the new rows), 0 when the objective stays a
// kernel of its own (no chunk buffers, no scratch, not the block-parallel
// kernel, or not enough shared memory).
template <typename T>
static size_t fused_objective_smem(const DevDesc& hd, int RP) {
  const int n = hd.N - 1;
  if (!hd.dotp || !hd.Gp[n]) return 0;
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = std::max<int64_t>(imax, hd.dims[k][n]);
  const UpdGeom geo = update_geometry(RP, hd.K, imax, sizeof(T));
  if (!geo.kp) return 0;
  // the last CTA evaluates the objective with at least two whole warps per
  // block; with fewer the separate objective kernel (one CTA per block) is faster
  if ((RP * hd.K * geo.ty) / 32 < 2 * hd.K) return 0;
  // the tail reads the CTAs' shares through a K x RP^2 buffer
  if (hd.gnc[n] > RP * RP) return 0;
  const size_t smem = std::max<size_t>(geo.smem + (size_t)hd.K * geo.gr * RP * sizeof(T) +
                                           (size_t)hd.K * RP * RP * sizeof(double),
                                       objective_tail_smem(hd.K, RP));
  return smem <= 200 * 1024 ? smem : 0;
}

bool update_fuses_objective(const DevDesc& hd, int fp64, int RP) {
  return fp64 ? fused_objective_smem<double>(hd, RP) > 0 : fused_objective_smem<float>(hd, RP) > 0;
}

template <typename T, int RP>
static cudaError_t update_impl(const LaunchCfg& c, const DevDesc& hd, int n, int use_w, double delta_w,
                               int use_core, int msplit, int with_objective) {
  UpdArgs<T> a{};
  a.K = hd.K;
  a.n = n;
  a.Ln = hd.L[n];
  a.nonneg = hd.nonneg[n];
  a.use_w = use_w;
  a.use_core = use_core;
  a.delta_w = delta_w;
  a.sc = hd.sc;
  a.rr = hd.Rmax * hd.Rmax;
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = std::max<int64_t>(imax, hd.dims[k][n]);
  const UpdGeom geo = update_geometry(RP, hd.K, imax, sizeof(T));
  a.gr = geo.gr;
  if (hd.Gp[n]) {
    a.Gp = reinterpret_cast<T*>(hd.Gp[n]);
    a.gnc = hd.gnc[n];
    if (hd.gr[n] != geo.gr) return cudaErrorInvalidValue;  // chunking must match the partial buffers
  }
  for (int k = 0; k < hd.K; ++k) {
    a.R[k] = hd.R[k];
    a.I[k] = (int)hd.dims[k][n];
    a.U1[k] = reinterpret_cast<T*>(hd.U1[k][n]);
    a.U2[k] = reinterpret_cast<T*>(hd.U2[k][n]);
    a.S[k] = reinterpret_cast<T*>(hd.ASbase + (static_cast<const char*>(hd.U1[k][n]) - hd.A1base));
    a.M[k] = reinterpret_cast<T*>(hd.M[k][n]);
    a.H[k] = reinterpret_cast<const T*>(hd.Hbase) + (size_t)k * a.rr;
    if (msplit) {
      a.part[k] = reinterpret_cast<const T*>(hd.partial) + hd.partial_off[k];
      a.nsplit[k] = hd.nsplit[k];
    }
  }
  const unsigned grid = (unsigned)((imax + a.gr - 1) / a.gr);
  size_t smem = geo.smem;
  if (with_objective) {
    smem = fused_objective_smem<T>(hd, RP);
    if (n != hd.N - 1 || smem == 0 || (unsigned)hd.gnc[n] < grid) return cudaErrorInvalidValue;
    a.obj = 1;
    a.N = hd.N;
    a.inv_K = 1.0 / hd.K;
    a.dotp = reinterpret_cast<T*>(hd.dotp);
    a.xxp = hd.xxp;
    a.gram_last = use_core;
    a.G = hd.Gbase;
    a.H64 = hd.H64base;
    a.hm = hd.hm;
  }
  if (geo.kp) {
    a.stage_rows = 1;
    cudaError_t e = allow_smem(k_update_kp<T, RP>, smem);
    if (e != cudaSuccess) return e;
    carve<k_update_kp<T, RP>>();
    e = launch_pdl(k_update_kp<T, RP>, dim3(grid), dim3(RP, hd.K, geo.ty), smem, c.stream, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  size_t dyn = 0;
  if (a.Gp && hd.K <= UpdCfg<T, RP>::KC) {
    dyn = (size_t)hd.K * a.gr * RP * sizeof(T);
    if (dyn <= 96 * 1024) a.stage_rows = 1;
    else dyn = 0;
  }
  cudaError_t e = allow_smem(k_update<T, RP>, dyn);
  if (e != cudaSuccess) return e;
  carve<k_update<T, RP>>();
  e = launch_pdl(k_update<T, RP>, dim3(grid), dim3(RP, UpdCfg<T, RP>::ROWS), dyn, c.stream, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_update(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int n,
                          int use_w, double delta_w, int use_core, int msplit, int with_objective) {
  (void)dd;
#define UCASE(V)                                                                                   \
  case V:                                                                                          \
    return fp64 ? update_impl<double, V>(c, hd, n, use_w, delta_w, use_core, msplit, with_objective) \
                : update_impl<float, V>(c, hd, n, use_w, delta_w, use_core, msplit, with_objective);
  switch (RP) { CNCPD_FOR_EACH_RP(UCASE) }
#undef UCASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Objective (Eq. costfunc) by the Gram expansion
//   F_k = 1/2 (||X||^2 - 2 <X, X_hat> + ||X_hat||^2),
//   <X, X_hat> = sum_r lambda_r sum_i M^(N-1)[i, r] U^(N-1)[i, r],
//   ||X_hat||^2 = lambda^T (*_m G^(m)) lambda,
// with M^(N-1) the MTTKRP of the last mode (computed before its update) and
// U^(N-1) the updated factor: together they give <X, [[U]]> at the new point.
// The per-r sums are the core term (U^{odot})^T vec(X) of Eq. solapgG for the
// next core update.  RelErr per Section III-C.  One CTA per block, threads
// (r, y); the last CTA to finish adds the blocks up in order.
// ---------------------------------------------------------------------------
template <typename T, int RP>
__global__ void __launch_bounds__(256) k_objective(const __grid_constant__ ObjArgs<T> a) {
  pdl_wait();
  pdl_trigger();
  constexpr int Y = 256 / RP;
  constexpr int NT = RP * Y;
  const int tid = threadIdx.x;
  const int r = tid % RP, y = tid / RP;  // threads >= NT only join the reductions
  const int N = a.N, n = N - 1;
  const int k = blockIdx.x;
  DevScalars* sc = a.sc;
  __shared__ T red[256];
  __shared__ double cr[RP];
  __shared__ double wsum[2][8];
  __shared__ float fsum[2][8];
  __shared__ int is_last;
  const int R = a.R[k];
  const int64_t I = a.I[k];
  const T* __restrict__ M = a.M[k];
  const T* __restrict__ U = a.U[k];
  const int rr = a.rr;
  double* Gk = a.G + (size_t)k * N * rr;
  // the scalars thread 0 needs at the end, loaded now
  double x2 = 0.0, ix2 = 0.0;
  if (tid == 0) {
    x2 = a.commit ? sc->xnorm2[k] : sc->xnorm2_orig[k];
    ix2 = a.commit ? sc->inv_xnorm2[k] : sc->inv_xnorm2_orig[k];
  }
  // <M, U> per column: an FMA chain in the factor type per thread
  T acc_t = T(0);
  if (r < R && y < Y) {
    for (int64_t i0 = y; i0 < I; i0 += 16 * Y) {
      T mv[16], uv[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int64_t i = min(i0 + (int64_t)j * Y, I - 1);  // clamped: every load issues at once
        mv[j] = M[i * R + r];
        uv[j] = U[i * R + r];
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (i0 + (int64_t)j * Y < I) acc_t = fma(mv[j], uv[j], acc_t);
    }
  }
  // ||X_hat||^2 terms in FP64; the Gram of the last mode is summed from its chunks
  double xx = 0.0;
  const int nch = a.reduce_last ? (int)((I + a.gr - 1) / a.gr) : 0;
  const T* gp = a.reduce_last ? a.Gp_last + (size_t)k * a.gnc * rr : nullptr;
  for (int p = tid; p < R * R; p += 256) {
    double gm[CNCPD_NMAX];
#pragma unroll
    for (int m = 0; m < CNCPD_NMAX; ++m) gm[m] = (m < N && !(a.reduce_last && m == n)) ? Gk[(size_t)m * rr + p] : 1.0;
    if (a.reduce_last) {
      const double g = gram_sum<T>(gp, nch, rr, p);
      Gk[(size_t)n * rr + p] = g;
#pragma unroll
      for (int m = 0; m < CNCPD_NMAX; ++m)
        if (m == n) gm[m] = g;
    }
    double g = sc->lam1[k][p / R] * sc->lam1[k][p % R];
#pragma unroll
    for (int m = 0; m < CNCPD_NMAX; ++m)
      if (m < N) g *= gm[m];
    xx += g;
  }
  if (tid < NT) red[tid] = acc_t;
  __syncthreads();
  if (y == 0 && r < R) {
    // the Y chains of column r, added in order
    double s;
    if constexpr (sizeof(T) == 4) {
      float hi = 0.f, lo = 0.f;
      for (int yy = 0; yy < Y; ++yy) ff_add(hi, lo, red[yy * RP + r]);
      s = (double)hi + (double)lo;
    } else {
      s = 0.0;
      for (int yy = 0; yy < Y; ++yy) s += red[yy * RP + r];
    }
    cr[r] = s;
    if (a.commit) sc->cterm[k][r] = s;
  }
  __syncthreads();
  // ||X_hat||^2 - 2 <X, X_hat> over the CTA: for FP32 factors in compensated
  // FP32 pairs (FP64 adds are slow here), FP64 only for the last additions
  if (tid < R) xx -= 2.0 * sc->lam1[k][tid] * cr[tid];
  if constexpr (sizeof(T) == 4) {
    float hi = (float)xx;
    float lo = (float)(xx - (double)hi);
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
      const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
      ff_add(hi, lo, oh);
      lo += ol;
    }
    if ((tid & 31) == 0) {
      fsum[0][tid >> 5] = hi;
      fsum[1][tid >> 5] = lo;
    }
  } else {
    for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(0xffffffffu, xx, o);
    if ((tid & 31) == 0) {
      wsum[0][tid >> 5] = xx;
      wsum[1][tid >> 5] = 0.0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double t;
    if constexpr (sizeof(T) == 4) {
      // the eight warp sums as one compensated FP32 pair, one conversion
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        ff_add(hi, lo, fsum[0][q]);
        lo += fsum[1][q];
      }
      t = (double)hi + (double)lo;
    } else {
      t = 0.0;
      for (int q = 0; q < 8; ++q) t += wsum[0][q];
    }
    const double Fk = 0.5 * (x2 + t);
    const double rel = sqrt(fmax(2.0 * Fk, 0.0) * ix2);
    if (a.commit) {
      sc->Fk[k] = Fk;
      sc->relk[k] = rel;
    } else {
      sc->out_relk[k] = rel;
    }
  }
  if (!a.commit) return;
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&sc->done_counter[1], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (is_last && tid < 32) {
    // the blocks' F_k and RelErr_k added by warp 0 (lane q holds blocks q,
    // q + 32, ...), in a fixed order
    __threadfence();
    double F = 0.0, rel = 0.0;
    for (int q = tid; q < (int)gridDim.x; q += 32) {
      F += __ldcg(&sc->Fk[q]);
      rel += __ldcg(&sc->relk[q]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      F += __shfl_xor_sync(0xffffffffu, F, o);
      rel += __shfl_xor_sync(0xffffffffu, rel, o);
    }
    if (tid == 0) {
      const double relerr = rel * a.inv_K;
      sc->F = F;
      sc->relerr = relerr;
      if (!isfinite(F)) sc->nonfinite = 1;
      sc->done_counter[1] = 0;
      if (a.hm) {
        HostMirror* hm = a.hm;
        hm->F = F;
        hm->relerr = relerr;
        hm->nonfinite = *((volatile int*)&sc->nonfinite);
        hm->timeout = *((volatile int*)&sc->timeout);
        const unsigned int q = sc->seq + 1;
        sc->seq = q;
        __threadfence_system();
        hm->seq = q;
      }
    }
  }
}

template <typename T, int RP>
static cudaError_t objective_impl(const LaunchCfg& c, const DevDesc& hd, int commit, int reduce_last) {
  ObjArgs<T> a{};
  const int n = hd.N - 1;
  a.K = hd.K;
  a.N = hd.N;
  a.rr = hd.Rmax * hd.Rmax;
  a.commit = commit;
  a.reduce_last = (reduce_last && hd.Gp[n]) ? 1 : 0;
  a.inv_K = 1.0 / hd.K;
  a.sc = hd.sc;
  a.hm = commit ? hd.hm : nullptr;
  a.G = hd.Gbase;
  if (a.reduce_last) {
    a.Gp_last = reinterpret_cast<const T*>(hd.Gp[n]);
    a.gnc = hd.gnc[n];
    a.gr = hd.gr[n];
  }
  for (int k = 0; k < hd.K; ++k) {
    a.R[k] = hd.R[k];
    a.I[k] = (int)hd.dims[k][n];
    a.M[k] = reinterpret_cast<const T*>(hd.M[k][n]);
    a.U[k] = reinterpret_cast<const T*>(hd.U1[k][n]);
  }
  carve<k_objective<T, RP>>();
  {
    cudaError_t eo = launch_pdl(k_objective<T, RP>, dim3(hd.K), dim3(256), 0, c.stream, a);
    if (eo != cudaSuccess) return eo;
  }
  return cudaGetLastError();
}

cudaError_t launch_objective(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int commit,
                             int reduce_last) {
  (void)dd;
#define OCASE(V)                                                                 \
  case V:                                                                        \
    return fp64 ? objective_impl<double, V>(c, hd, commit, reduce_last)          \
                : objective_impl<float, V>(c, hd, commit, reduce_last);
  switch (RP) { CNCPD_FOR_EACH_RP(OCASE) }
#undef OCASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Core update of Eqs. solD / solapgG / eqextraPG with L_d = ||(U^T U)^*||_2
// (Eq. eqLipsLd) and the weight of Eq. eqextrawd.  One CTA per block, FP64.
// ---------------------------------------------------------------------------
template <int RP>
__global__ void __launch_bounds__(256) k_core_update(const DevDesc* __restrict__ d, int use_w, double delta_w) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.x;
  const int R = d->R[k], N = d->N;
  DevScalars* sc = d->sc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Hs = reinterpret_cast<double*>(smem_raw);
  LmaxSmem<RP>* ls = reinterpret_cast<LmaxSmem<RP>*>(smem_raw + (size_t)RP * RP * sizeof(double));
  __shared__ double lh[CNCPD_RMAX];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double h = 1.0;
    for (int m = 0; m < N; ++m) h *= d->G[k][m][e];
    Hs[e] = h;
    ls->Hf[e] = (float)h;
  }
  const double Ld = lmax_rp<double, RP>(Hs, R, ls);
  const double w = extrap_weight<double>(use_w ? sc->w_hat : 0.0, sc->have_prev, sc->Ldprev[k], Ld, delta_w);
  for (int a = threadIdx.x; a < R; a += blockDim.x) lh[a] = sc->lam1[k][a] + w * (sc->lam1[k][a] - sc->lam2[k][a]);
  __syncthreads();
  if (Ld > 0.0) {
    for (int a = threadIdx.x; a < R; a += blockDim.x) {
      double g = -sc->cterm[k][a];
      for (int b = 0; b < R; ++b) g = fma(Hs[a * R + b], lh[b], g);
      const double nv = fmax(0.0, lh[a] - g / Ld);
      sc->lam2[k][a] = sc->lam1[k][a];
      sc->lam1[k][a] = nv;
    }
  } else {
    for (int a = threadIdx.x; a < R; a += blockDim.x) sc->lam2[k][a] = sc->lam1[k][a];
  }
  if (threadIdx.x == 0) {
    sc->Ldcur[k] = Ld;
    if (!isfinite(Ld)) sc->nonfinite = 1;
  }
}

template <int RP>
static cudaError_t core_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int use_w, double delta_w) {
  const size_t sm = lip_smem_bytes<RP>();
  cudaError_t e = allow_smem(k_core_update<RP>, sm);
  if (e != cudaSuccess) return e;
  carve<k_core_update<RP>>();
  k_core_update<RP><<<hd.K, 256, sm, c.stream>>>(dd, use_w, delta_w);
  return cudaGetLastError();
}

cudaError_t launch_core_update(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int use_w, double delta_w) {
#define CCASE(V) \
  case V: return core_impl<V>(c, dd, hd, use_w, delta_w);
  switch (rank_bucket_of(hd)) { CNCPD_FOR_EACH_RP(CCASE) }
#undef CCASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Iteration bookkeeping.  Begin: t_k and hat w (Appendix A), commit the
// Lipschitz constants of the last accepted sweep as L_{k-2}, snapshot the
// core term and lambda_2 (the factor snapshot is a device memcpy).
// Redo: restore lambda and the core term for the w = 0 re-update.
// One element per thread, so every load is issued at once.
// ---------------------------------------------------------------------------
struct IterArgs {
  int K, N, use_core, pad;
  DevScalars* sc;
};

__global__ void __launch_bounds__(1024) k_iter_begin(const __grid_constant__ IterArgs a) {
  pdl_wait();
  pdl_trigger();
  DevScalars* sc = a.sc;
  const int K = a.K, N = a.N;
  const int tid = threadIdx.x;
  const int have_cur = sc->have_cur;
  if (tid < N * K) {
    const int n = tid / K, k = tid % K;
    const double L = sc->Lcur_u[n][k];
    if (have_cur) sc->Lprev_u[n][k] = L;
  } else if (tid < N * K + N) {
    const int n = tid - N * K;
    const double L = sc->LCcur[n];
    if (have_cur) sc->LCprev[n] = L;
  } else if (tid < N * K + N + K) {
    const int k = tid - N * K - N;
    const double L = sc->Ldcur[k];
    if (have_cur) sc->Ldprev[k] = L;
  } else if (tid == N * K + N + K) {
    const double t = sc->t;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc->w_hat = (t - 1.0) / tn;
    sc->t = tn;
    if (have_cur) sc->have_prev = 1;
  }
  if (a.use_core)
    for (int e = tid; e < K * CNCPD_RMAX; e += blockDim.x) {
      const int k = e / CNCPD_RMAX, r = e % CNCPD_RMAX;
      sc->cterm_save[k][r] = sc->cterm[k][r];
      sc->lamS[k][r] = sc->lam2[k][r];
    }
}

__global__ void k_redo_prepare(const DevDesc* __restrict__ d) {
  pdl_wait();
  pdl_trigger();
  DevScalars* sc = d->sc;
  const int K = d->K;
  for (int e = threadIdx.x; e < K * CNCPD_RMAX; e += blockDim.x) {
    const int k = e / CNCPD_RMAX, r = e % CNCPD_RMAX;
    sc->lam1[k][r] = sc->lam2[k][r];
    sc->lam2[k][r] = sc->lamS[k][r];
    sc->cterm[k][r] = sc->cterm_save[k][r];
  }
}

cudaError_t launch_iter_begin(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int use_core) {
  (void)dd;
  IterArgs a{hd.K, hd.N, use_core, 0, hd.sc};
  const int need = hd.N * hd.K + hd.N + hd.K + 1;
  int nt = 256;
  while (nt < need && nt < 1024) nt *= 2;
  carve<k_iter_begin>();
  k_iter_begin<<<1, nt, 0, c.stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_redo_prepare(const LaunchCfg& c, const DevDesc* dd, const DevDesc&) {
  carve<k_redo_prepare>();
  k_redo_prepare<<<1, 256, 0, c.stream>>>(dd);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gradient at the current factors (no extrapolation), Eq. solbpgU:
//   dF/dU^(n,k) = U D (U^T U)^{*-n} D - X_(n) U^{odot-n} D,
// written over the M buffer of (n, k).  Threads (c, y) like the update.
// ---------------------------------------------------------------------------
template <typename T, int RP>
__global__ void k_grad(const DevDesc* __restrict__ d, int n, int use_core) {
  constexpr int ROWS = 256 / RP;
  __shared__ T Hs[RP * RP];
  __shared__ T us[ROWS][RP];
  const int c = threadIdx.x, y = threadIdx.y;
  const int64_t i = (int64_t)blockIdx.x * ROWS + y;
  const int k = blockIdx.y;
  const int R = d->R[k];
  const int64_t In = d->dims[k][n];
  DevScalars* sc = d->sc;
  const T* Hk = reinterpret_cast<const T*>(d->H[k]);
  for (int e = threadIdx.x + threadIdx.y * RP; e < RP * RP; e += RP * ROWS) {
    const int a = e / RP, b = e % RP;
    Hs[e] = (a < R && b < R) ? Hk[a * R + b] : T(0);
  }
  const bool valid = (i < In) && (c < R);
  const T* U1 = reinterpret_cast<const T*>(d->U1[k][n]);
  us[y][c] = valid ? U1[i * R + c] : T(0);
  __syncthreads();
  if (valid) {
    T* M = reinterpret_cast<T*>(d->M[k][n]);
    const T lam = use_core ? (T)sc->lam1[k][c] : T(1);
    T g = -M[i * R + c] * lam;
#pragma unroll
    for (int a = 0; a < RP; ++a) g = fma(us[y][a], Hs[a * RP + c], g);
    M[i * R + c] = g;
  }
}

// Gradient of the shared columns U_C^(n) (App. A): out[i, r] = sum_k of
// column r < L_n of block k's gradient (left in M[k][n] by k_grad), the
// blocks added in order in FP64, written as O.
template <typename T, typename O>
__global__ void k_common_grad(const DevDesc* __restrict__ d, int n, O* __restrict__ out) {
  const int Ln = d->L[n];
  const int64_t total = d->dims[0][n] * Ln;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Ln;
    const int r = (int)(e % Ln);
    double s = 0.0;
    for (int k = 0; k < d->K; ++k) s += (double)reinterpret_cast<const T*>(d->M[k][n])[i * d->R[k] + r];
    out[e] = (O)s;
  }
}

cudaError_t launch_common_grad(cudaStream_t s, const DevDesc* dd, const DevDesc& hd, int fp64, int n, void* out,
                               int out_f64) {
  const int64_t total = hd.dims[0][n] * hd.L[n];
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(1024, (total + 255) / 256);
  if (fp64) {
    if (out_f64) k_common_grad<double, double><<<grid, 256, 0, s>>>(dd, n, static_cast<double*>(out));
    else k_common_grad<double, float><<<grid, 256, 0, s>>>(dd, n, static_cast<float*>(out));
  } else {
    if (out_f64) k_common_grad<float, double><<<grid, 256, 0, s>>>(dd, n, static_cast<double*>(out));
    else k_common_grad<float, float><<<grid, 256, 0, s>>>(dd, n, static_cast<float*>(out));
  }
  return cudaGetLastError();
}

cudaError_t launch_grad(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int n,
                        int use_core) {
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][n] > imax ? hd.dims[k][n] : imax;
  {
    cudaError_t e = launch_hmat(c, hd, fp64, n, use_core);
    if (e != cudaSuccess) return e;
  }
#define GCASE(V)                                                                        \
  case V: {                                                                             \
    dim3 grid((unsigned)((imax + 256 / V - 1) / (256 / V)), hd.K);                      \
    if (fp64) k_grad<double, V><<<grid, dim3(V, 256 / V), 0, c.stream>>>(dd, n, use_core); \
    else k_grad<float, V><<<grid, dim3(V, 256 / V), 0, c.stream>>>(dd, n, use_core);    \
    return cudaGetLastError();                                                          \
  }
  switch (RP) { CNCPD_FOR_EACH_RP(GCASE) }
#undef GCASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Data preparation: quantise X into the storage type and take ||X_stored||^2
// in FP64 (per-CTA partial sums, then a fixed-order sum).
// ---------------------------------------------------------------------------
// One element: stored at o in the storage type; returns the stored value.
__device__ __forceinline__ double quantize_one(double x, void* dst, void* dst_lo, int st, int64_t o) {
  if (st == ST_F64) {
    reinterpret_cast<double*>(dst)[o] = x;
    return x;
  }
  if (st == ST_F32) {
    const float f = (float)x;
    reinterpret_cast<float*>(dst)[o] = f;
    return f;
  }
  if (st == ST_BF16) {
    const __nv_bfloat16 b = __double2bfloat16(x);
    reinterpret_cast<__nv_bfloat16*>(dst)[o] = b;
    return (double)__bfloat162float(b);
  }
  const float f = (float)x;
  const __nv_bfloat16 hi = __float2bfloat16_rn(f);
  const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
  reinterpret_cast<__nv_bfloat16*>(dst)[o] = hi;
  reinterpret_cast<__nv_bfloat16*>(dst_lo)[o] = lo;
  return (double)(__bfloat162float(hi) + __bfloat162float(lo));
}

// The source may be page-locked host memory read in place, so it is read in
// 16-byte vectors, four per thread in flight, when its address allows; each
// element then goes to (row, col) of the pitched store.
template <typename S>
__global__ void k_quantize(const S* __restrict__ src, void* dst, void* dst_lo, int st, int64_t rows, int64_t cols,
                           int64_t pitch, double* part) {
  constexpr int V = 16 / sizeof(S);  // elements per 16-byte vector
  double acc = 0.0;
  const int64_t n = rows * cols;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t done = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int64_t nv = n / V;  // whole vectors
    const uint4* sv = reinterpret_cast<const uint4*>(src);
    for (int64_t v0 = t; v0 < nv; v0 += 4 * nthreads) {
      uint4 buf[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t v = v0 + u * nthreads;
        buf[u] = v < nv ? sv[v] : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t v = v0 + u * nthreads;
        if (v >= nv) break;
        const S* e = reinterpret_cast<const S*>(&buf[u]);
#pragma unroll
        for (int j = 0; j < V; ++j) {
          const int64_t i = v * V + j;
          const int64_t row = i / cols;
          const double q = quantize_one((double)e[j], dst, dst_lo, st, row * pitch + (i - row * cols));
          acc = fma(q, q, acc);
        }
      }
    }
    done = nv * V;
  }
  for (int64_t i = done + t; i < n; i += nthreads) {
    const int64_t row = i / cols;
    const double q = quantize_one((double)src[i], dst, dst_lo, st, row * pitch + (i - row * cols));
    acc = fma(q, q, acc);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* part, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

cudaError_t launch_quantize(cudaStream_t s, const void* src, int src_f64, void* dst, void* dst_lo, int st,
                            int64_t rows, int64_t cols, int64_t pitch, double* norm2_out, double* scratch, int nblk) {
  if (src_f64)
    k_quantize<double><<<nblk, 256, 0, s>>>(reinterpret_cast<const double*>(src), dst, dst_lo, st, rows, cols, pitch,
                                            scratch);
  else
    k_quantize<float><<<nblk, 256, 0, s>>>(reinterpret_cast<const float*>(src), dst, dst_lo, st, rows, cols, pitch,
                                           scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_partials<<<1, 32, 0, s>>>(scratch, nblk, norm2_out);
  return cudaGetLastError();
}

__global__ void k_convert(const void* src, int src_f64, void* dst, int dst_f64, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = src_f64 ? reinterpret_cast<const double*>(src)[i] : (double)reinterpret_cast<const float*>(src)[i];
    if (dst_f64) reinterpret_cast<double*>(dst)[i] = v;
    else reinterpret_cast<float*>(dst)[i] = (float)v;
  }
}

cudaError_t launch_convert(cudaStream_t s, const void* src, int src_f64, void* dst, int dst_f64, int64_t n) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  k_convert<<<grid, 256, 0, s>>>(src, src_f64, dst, dst_f64, n);
  return cudaGetLastError();
}

// Uniform[0,1) from the SplitMix64 finaliser of (seed, index) (Steele,
// Lea and Flood, OOPSLA 2014) -- the library's default initialisation.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_uniform(void* dst, int fp64, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = splitmix64(seed ^ splitmix64((uint64_t)i));
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    if (fp64) reinterpret_cast<double*>(dst)[i] = u;
    else reinterpret_cast<float*>(dst)[i] = (float)u;
  }
}

cudaError_t launch_uniform_init(cudaStream_t s, void* dst, int fp64, int64_t n, uint64_t seed) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 1024) grid = 1024;
  k_uniform<<<grid, 256, 0, s>>>(dst, fp64, n, seed);
  return cudaGetLastError();
}

template <int RP>
__global__ void k_lmax_one(const double* H, int R, double* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Hs = reinterpret_cast<double*>(smem_raw);
  LmaxSmem<RP>* ls = reinterpret_cast<LmaxSmem<RP>*>(smem_raw + (size_t)RP * RP * sizeof(double));
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    Hs[e] = H[e];
    ls->Hf[e] = (float)H[e];
  }
  const double L = lmax_rp<double, RP>(Hs, R, ls);
  if (threadIdx.x == 0) *out = L;
}

template <int RP>
static cudaError_t lmax_one_impl(const double* d_H, int R, double* d_out, cudaStream_t s) {
  const size_t sm = lip_smem_bytes<RP>();
  cudaError_t e = allow_smem(k_lmax_one<RP>, sm);
  if (e != cudaSuccess) return e;
  k_lmax_one<RP><<<1, 256, sm, s>>>(d_H, R, d_out);
  return cudaGetLastError();
}

cudaError_t launch_lmax_host(const double* d_H, int R, double* d_out, cudaStream_t s) {
#define LCASE(V) \
  case V: return lmax_one_impl<V>(d_H, R, d_out, s);
  switch (rank_bucket(R)) { CNCPD_FOR_EACH_RP(LCASE) }
#undef LCASE
  return cudaErrorInvalidValue;
}

}  // namespace cncpd
