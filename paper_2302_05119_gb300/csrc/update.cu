// Small per-mode kernels of the APG sweep: Grams, Hadamard products and
// Lipschitz constants, the fused extrapolate / gradient / step / projection
// update with the coupled common-column sum, the objective, the core update,
// and the bookkeeping of iterations and re-updates.
#include <algorithm>

#include "cncpd_internal.cuh"

namespace cncpd {

// ---------------------------------------------------------------------------
// Largest eigenvalue of a symmetric PSD R x R matrix (R <= 64), called by a
// whole CTA.  ||H||_2 of Eqs. eqLipsLd / eqLipsLu.  Normalised repeated
// squaring A <- A^2 / tr(A^2) in FP32 converges to the projector on the
// leading eigenvector (ratios of eigenvalues are raised to the power 2^s).
// The FP64 value is the Rayleigh quotient of H at a column of the limit.
// Returns 0 for a zero matrix and propagates NaN/Inf.
// ---------------------------------------------------------------------------
// Shared-memory layout of lmax_psd for an R x R problem (dynamic smem):
// Hs (R*R doubles), v, w (R doubles each), A, B (R*R floats each), red (32 floats).
__host__ __device__ inline size_t lmax_smem_bytes(int R) {
  return (size_t)R * R * 8 + 2 * (size_t)R * 8 + 2 * (size_t)R * R * 4 + 32 * 4 + 16;
}

struct LmaxScratch {
  double* Hs;
  double* v;
  double* w;
  float* A;
  float* B;
  float* red;
  __device__ void carve(unsigned char* base, int R) {
    Hs = reinterpret_cast<double*>(base);
    v = Hs + R * R;
    w = v + R;
    A = reinterpret_cast<float*>(w + R);
    B = A + R * R;
    red = B + R * R;
  }
};

template <typename TT>
__device__ double lmax_psd(const double* Hs, int R, LmaxScratch* s) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  __syncthreads();
  double tr = 0.0;
  for (int i = 0; i < R; ++i) tr += Hs[i * R + i];
  if (!isfinite(tr)) return tr;
  if (!(tr > 0.0)) return 0.0;
  const int RR = R * R;
  const double itr = 1.0 / tr;
  for (int e = tid; e < RR; e += nt) s->A[e] = (float)(Hs[e] * itr);
  __syncthreads();
  for (int it = 0; it < 32; ++it) {
    for (int e = tid; e < RR; e += nt) {
      const int i = e / R, j = e % R;
      float acc = 0.f;
      for (int l = 0; l < R; ++l) acc = fmaf(s->A[i * R + l], s->A[l * R + j], acc);
      s->B[e] = acc;
    }
    __syncthreads();
    float trb = 0.f;
    for (int i = 0; i < R; ++i) trb += s->B[i * R + i];
    float dmax = 0.f;
    if (trb > 0.f) {
      for (int e = tid; e < RR; e += nt) {
        const float nv = s->B[e] / trb;
        dmax = fmaxf(dmax, fabsf(nv - s->A[e]));
        s->A[e] = nv;
      }
    }
    if ((it & 3) != 3 && (trb > 0.f)) {
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
  // v: column of the limit with the largest diagonal entry (FP32 accuracy in
  // every non-leading direction).  One FP64 product y = H v and the Rayleigh
  // quotient v^T y / v^T v, reduced by warp 0, give L with error quadratic in
  // that accuracy.  (When the two largest eigenvalues agree to within FP32
  // resolution the squaring still ends in a rank-one limit, and the error is
  // bounded by their relative gap.)
  int jm = 0;
  float dm = -1.f;
  for (int i = 0; i < R; ++i)
    if (s->A[i * R + i] > dm) { dm = s->A[i * R + i]; jm = i; }
  // (TT = float on the FP32 path: L to FP32 accuracy is ample there and
  // FP64 arithmetic is slow on this part; TT = double on the FP64 path.)
  for (int i = tid; i < R; i += nt) {
    const TT vi = (TT)s->A[i * R + jm];
    TT a = TT(0);
    for (int l = 0; l < R; ++l) a = fma((TT)Hs[i * R + l], (TT)s->A[l * R + jm], a);
    s->v[i] = (double)(vi * a);   // v_i (H v)_i
    s->w[i] = (double)(vi * vi);  // v_i^2
  }
  __syncthreads();
  if (tid < 32) {
    TT num = TT(0), den = TT(0);
    for (int i = tid; i < R; i += 32) {
      num += (TT)s->v[i];
      den += (TT)s->w[i];
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
// Gram G = U^T U (Table II operation 1) of one I x R factor, computed by a
// whole CTA: U is staged through shared memory GT rows at a time; for every
// (a, b) an FMA chain in the factor type runs over each tile and the tile
// sums are added in FP64 in order.  Every kernel that forms a Gram calls
// this routine, so all of them give bit-identical results.
// ---------------------------------------------------------------------------
constexpr int GRAM_TILE = 64;

template <typename T>
__device__ void block_gram(const T* __restrict__ U, int64_t I, int R, double* __restrict__ G, T* buf, int cap_rows) {
  // buf holds cap_rows rows (a multiple of GRAM_TILE); rows are staged in as
  // few round trips as the buffer allows.  For small R each pair's rows are
  // split into SL = max(1, 256 / R^2) interleaved slices (an FMA chain in the
  // factor type each); per tile the slice sums are added in slice order in
  // FP64, tiles in order.  The order depends only on R, so every kernel that
  // calls this routine gets bit-identical Grams.
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nt = blockDim.x * blockDim.y;
  const int RR = R * R;
  const int SL = max(1, 256 / RR);
  const int items = RR * SL;  // <= 256 whenever SL > 1
  __shared__ double slice_sum[256];
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
      if (SL == 1) {
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
      } else {
        for (int wi = tid; wi < items; wi += nt) {
          const int p = wi / SL, sl = wi % SL;
          const int a = p / R, b = p % R;
          T s = T(0);
#pragma unroll 4
          for (int i = sl; i < n; i += SL) s = fma(tile[i * R + a], tile[i * R + b], s);
          slice_sum[wi] = (double)s;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int p = q * nt + tid;
          if (p < RR) {
            double t = 0.0;
            for (int sl = 0; sl < SL; ++sl) t += slice_sum[p * SL + sl];
            acc[q] += t;
          }
        }
        __syncthreads();
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

// Grams of modes [n_begin, n_end) of every block; which = 0: the factors
// U1, which = 1: the LRA factors U~.  One CTA per (block, mode).
template <typename T>
__global__ void __launch_bounds__(256) k_gram(const DevDesc* __restrict__ d, int n_begin, int n_end, int which) {
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
  const int grid = hd.K * (n_end - n_begin);
  if (fp64) k_gram<double><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end, which);
  else k_gram<float><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end, which);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// H^(n,k) = D (*_{m != n} G^(m,k)) D (Eq. solapgU first term; Table II
// operation 4) and L_u^(n,k) = ||H||_2 (Eq. eqLipsLu).  One CTA per block.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void lipschitz_body(const DevDesc* __restrict__ d, int k, int n, int use_core, int want_L, int prev,
                               int gram_rows, unsigned char* smem_raw) {
  const int R = d->R[k], N = d->N;
  if (prev >= 0)  // Gram of the mode updated just before (Table II operation 1)
    block_gram<T>(reinterpret_cast<const T*>(d->U1[k][prev]), d->dims[k][prev], R, d->G[k][prev],
                  reinterpret_cast<T*>(smem_raw), gram_rows);
  LmaxScratch scr;
  scr.carve(smem_raw, R);
  double* Hs = scr.Hs;
  DevScalars* sc = d->sc;
  T* Hout = reinterpret_cast<T*>(d->H[k]);
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double h = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) h *= d->G[k][m][e];
    if (use_core) h *= sc->lam1[k][e / R] * sc->lam1[k][e % R];
    Hs[e] = h;
    Hout[e] = (T)h;
  }
  if (!want_L) return;
  const double L = lmax_psd<T>(Hs, R, &scr);
  if (threadIdx.x == 0) {
    sc->Lcur_u[n][k] = L;
    if (!isfinite(L)) atomicExch(&sc->nonfinite, 1);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_lipschitz(const DevDesc* __restrict__ d, int n, int use_core, int want_L,
                                                   int prev, int gram_rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  lipschitz_body<T>(d, blockIdx.x, n, use_core, want_L, prev, gram_rows, smem_raw);
}

// Two-mode groups (third- and fourth-order tensors).  With n first in its
// group, P[i_n][b][r] is contiguous per i_n:  M[i_n, r] = sum_b P W[b, r].
// With n last, P[a][i_n][r]:  M[i_n, r] = sum_a P W[a, r], and ni
// consecutive i_n of one a are contiguous.  W is the other mode's factor
// (read through the read-only cache); a CTA produces ni rows of M.
template <typename T>
__device__ void level2_pair_body(const DevDesc* __restrict__ d, int k, int bx, int n, int ni_max) {
  __shared__ T red[256];
  const int N = d->N, h = d->h;
  const int m0 = (n < h) ? 0 : h;
  const int other = (n == m0) ? n + 1 : m0;   // the group's other mode
  const bool first = (n == m0);
  const int In = (int)d->dims[k][n];
  const int Io = (int)d->dims[k][other];
  const int R = d->R[k];
  const int i0 = bx * ni_max;
  if (i0 >= In) return;
  const int ni = min(ni_max, In - i0);
  const T* P = reinterpret_cast<const T*>((n < h) ? d->Pl[k] : d->Pt[k]);
  const T* W = reinterpret_cast<const T*>(d->U1[k][other]);
  T* M = reinterpret_cast<T*>(d->M[k][n]);
  const int t = threadIdx.x;
  if (first) {
    const int BR = Io * R;
    const int stride = (blockDim.x / R) * R;
    T acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = T(0);
    if (t < stride) {
#pragma unroll 2
      for (int e = t; e < BR; e += stride) {
        const T w = __ldg(W + e);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < ni) acc[q] = fma(P[(int64_t)(i0 + q) * BR + e], w, acc[q]);
      }
    }
    for (int q = 0; q < ni; ++q) {
      red[t] = acc[q];
      __syncthreads();
      if (t < R) {
        T s = T(0);
        for (int u = t; u < stride; u += R) s += red[u];
        M[(int64_t)(i0 + q) * R + t] = s;
      }
      __syncthreads();
    }
  } else {
    const int JR = ni * R;
    const int nsl = max(1, (int)blockDim.x / JR);
    const int j = t % JR, sl = t / JR;
    T acc = T(0);
    if (sl < nsl && t < nsl * JR) {
      const int r = j % R;
#pragma unroll 8
      for (int a = sl; a < Io; a += nsl) acc = fma(P[((int64_t)a * In + i0) * R + j], __ldg(W + a * R + r), acc);
    }
    red[t] = acc;
    __syncthreads();
    if (t < JR) {
      T s = T(0);
      for (int u = 0; u < nsl; ++u) s += red[u * JR + t];
      M[(int64_t)i0 * R + t] = s;
    }
  }
}

// CTAs [0, nlip): H and L of mode n for block blockIdx.x; the rest: level 2
// of mode n, nx CTAs per block.
template <typename T>
__global__ void __launch_bounds__(256) k_mode_prep(const DevDesc* __restrict__ d, int n, int use_core, int prev,
                                                   int gram_rows, int nlip, int nx, int ni) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if ((int)blockIdx.x < nlip) {
    lipschitz_body<T>(d, blockIdx.x, n, use_core, 1, prev, gram_rows, smem_raw);
  } else {
    const int b = blockIdx.x - nlip;
    level2_pair_body<T>(d, b / nx, b % nx, n, ni);
  }
}

static void lipschitz_smem(const DevDesc& hd, int fp64, int* gram_rows, size_t* sm) {
  // Gram staging: up to 32 KiB of rows (whole factor when it fits)
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k)
    for (int m = 0; m < hd.N; ++m) imax = std::max<int64_t>(imax, hd.dims[k][m]);
  const int es = fp64 ? 8 : 4;
  int64_t rows = std::min<int64_t>((imax + GRAM_TILE - 1) / GRAM_TILE * GRAM_TILE,
                                   std::max<int64_t>(GRAM_TILE, (32768 / es / std::max(1, hd.Rmax)) / GRAM_TILE * GRAM_TILE));
  *gram_rows = (int)rows;
  *sm = std::max(lmax_smem_bytes(hd.Rmax), (size_t)rows * hd.Rmax * es);
}

bool level2_is_pair(const DevDesc& hd, int n) {
  const int gsize = (n < hd.h) ? hd.h : hd.N - hd.h;
  return gsize == 2;
}

cudaError_t launch_mode_prep(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n, int use_core,
                             int prev, int with_level2) {
  // with_level2: 0 = Lipschitz only, 1 = Lipschitz + level 2, 2 = level 2 only
  int gram_rows = GRAM_TILE;
  size_t sm = 0;
  const int nlip = (with_level2 == 2) ? 0 : hd.K;
  if (nlip) lipschitz_smem(hd, fp64, &gram_rows, &sm);
  int nx = 0, ni = 1;
  if (with_level2) {
    int64_t imax = 0;
    for (int k = 0; k < hd.K; ++k) imax = std::max<int64_t>(imax, hd.dims[k][n]);
    // rows per CTA: small enough for ~4 CTAs per SM over all blocks, ni*R <= 256
    ni = std::max(1, std::min(8, 256 / std::max(1, hd.Rmax)));
    while (ni > 1 && ((imax + ni - 1) / ni) * hd.K < 4LL * c.num_sms) ni /= 2;
    nx = (int)((imax + ni - 1) / ni);
  }
  const int grid = nlip + nx * hd.K;
  if (grid == 0) return cudaSuccess;
  cudaError_t e = fp64 ? allow_smem(k_mode_prep<double>, sm) : allow_smem(k_mode_prep<float>, sm);
  if (e != cudaSuccess) return e;
  if (fp64) k_mode_prep<double><<<grid, 256, sm, c.stream>>>(dd, n, use_core, prev, gram_rows, nlip, nx, ni);
  else k_mode_prep<float><<<grid, 256, sm, c.stream>>>(dd, n, use_core, prev, gram_rows, nlip, nx, ni);
  return cudaGetLastError();
}

cudaError_t launch_lipschitz(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n, int use_core,
                             int prev) {
  int gram_rows;
  size_t sm;
  lipschitz_smem(hd, fp64, &gram_rows, &sm);
  cudaError_t e = fp64 ? allow_smem(k_lipschitz<double>, sm) : allow_smem(k_lipschitz<float>, sm);
  if (e != cudaSuccess) return e;
  const int nt = hd.Rmax <= 16 ? 128 : 256;
  if (fp64) k_lipschitz<double><<<hd.K, nt, sm, c.stream>>>(dd, n, use_core, 1, prev, gram_rows);
  else k_lipschitz<float><<<hd.K, nt, sm, c.stream>>>(dd, n, use_core, 1, prev, gram_rows);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused update of mode n for every block (Eqs. eqextraPU, solapgU, solUns,
// solUnC, solUnsI):
//   U_hat = U1 + w (U1 - U2)            (shared columns: one weight w_C)
//   G_hat = U_hat H - M D
//   individual columns: U1 <- P(U_hat - G_hat / L_u^(n,k))
//   shared columns:     U1 <- P(U_hat_C - sum_k G_hat_C / sum_k L_u^(n,k)),
//                       the same value written to every block
//   U2 <- old U1.
// (The Gram of the new factor is formed by the next kernel that needs it.)
// Thread (c, y) owns column c of row blockIdx.x * ROWS + y and walks the
// blocks in chunks of KC, keeping the shared-column gradient sum in a
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
__global__ void __launch_bounds__(128) k_update(const DevDesc* __restrict__ d, int n, int use_w, double delta_w,
                                                int use_core) {
  constexpr int ROWS = UpdCfg<T, RP>::ROWS;
  constexpr int KC = UpdCfg<T, RP>::KC;
  __shared__ T Hs[KC][RP * RP];
  __shared__ T uh[KC][ROWS][RP];

  const int c = threadIdx.x;
  const int y = threadIdx.y;
  const int tid = c + y * RP;
  constexpr int NT = RP * ROWS;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  const int64_t i = row0 + y;
  const int K = d->K;
  const int Ln = d->L[n];
  const int nonneg = d->nonneg[n];
  DevScalars* sc = d->sc;
  __shared__ T wsh[CNCPD_KMAX + 1];
  __shared__ double LCs;
  {
    // extrapolation weights (Eqs. eqextrawu and reading R3), one FP64
    // evaluation per block instead of one per thread
    const double w_hat = use_w ? sc->w_hat : 0.0;
    const int have_prev = sc->have_prev;
    if (tid < K) wsh[tid] = extrap_weight<T>(w_hat, have_prev, sc->Lprev_u[n][tid], sc->Lcur_u[n][tid], delta_w);
    if (tid == K) {
      double LC = 0.0;
      for (int k = 0; k < K; ++k) LC += sc->Lcur_u[n][k];
      LCs = LC;
      wsh[K] = extrap_weight<T>(w_hat, have_prev, sc->LCprev[n], LC, delta_w);
      if (blockIdx.x == 0) {
        sc->LCcur[n] = LC;
        sc->have_cur = 1;
      }
    }
    __syncthreads();
  }
  const double LC = LCs;
  const T wC = wsh[K];

  T sumC = T(0), uhC = T(0), u1C = T(0);
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kn = min(KC, K - k0);
    __syncthreads();
    T u1[KC], u2[KC], mv[KC];
    for (int kk = 0; kk < kn; ++kk) {
      const int k = k0 + kk;
      const int R = d->R[k];
      const T* Hk = reinterpret_cast<const T*>(d->H[k]);
      for (int e = tid; e < RP * RP; e += NT) {
        const int a = e / RP, b = e % RP;
        Hs[kk][e] = (a < R && b < R) ? Hk[a * R + b] : T(0);
      }
      const bool valid = (i < d->dims[k][n]) && (c < R);
      u1[kk] = u2[kk] = mv[kk] = T(0);
      if (valid) {
        u1[kk] = reinterpret_cast<const T*>(d->U1[k][n])[i * R + c];
        u2[kk] = reinterpret_cast<const T*>(d->U2[k][n])[i * R + c];
        mv[kk] = reinterpret_cast<const T*>(d->M[k][n])[i * R + c];
      }
      const T w = (c < Ln) ? wC : wsh[k];
      uh[kk][y][c] = valid ? u1[kk] + w * (u1[kk] - u2[kk]) : T(0);
    }
    __syncthreads();
    for (int kk = 0; kk < kn; ++kk) {
      const int k = k0 + kk;
      const int R = d->R[k];
      if ((i < d->dims[k][n]) && (c < R)) {
        const double Lk = sc->Lcur_u[n][k];
        const T lam = use_core ? (T)sc->lam1[k][c] : T(1);
        const T uhat = uh[kk][y][c];
        T g = -mv[kk] * lam;
#pragma unroll
        for (int a = 0; a < RP; ++a) g = fma(uh[kk][y][a], Hs[kk][a * RP + c], g);
        if (c >= Ln) {
          T nv = u1[kk];
          if (Lk > 0.0) {
            nv = uhat - g / (T)Lk;
            if (nonneg) nv = nv > T(0) ? nv : T(0);
          }
          reinterpret_cast<T*>(d->U2[k][n])[i * R + c] = u1[kk];
          reinterpret_cast<T*>(d->U1[k][n])[i * R + c] = nv;
        } else {
          sumC += g;
          uhC = uhat;
          u1C = u1[kk];
        }
      }
    }
  }
  if (c < Ln && i < d->dims[0][n]) {
    T nv = u1C;
    if (LC > 0.0) {
      nv = uhC - sumC / (T)LC;
      if (nonneg) nv = nv > T(0) ? nv : T(0);
    }
    for (int k = 0; k < K; ++k) {
      const int R = d->R[k];
      reinterpret_cast<T*>(d->U2[k][n])[i * R + c] = u1C;
      reinterpret_cast<T*>(d->U1[k][n])[i * R + c] = nv;
    }
  }

}

template <typename T, int RP>
static cudaError_t update_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int n, int use_w,
                               double delta_w, int use_core) {
  constexpr int ROWS = UpdCfg<T, RP>::ROWS;
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][n] > imax ? hd.dims[k][n] : imax;
  const unsigned grid = (unsigned)((imax + ROWS - 1) / ROWS);
  k_update<T, RP><<<grid, dim3(RP, ROWS), 0, c.stream>>>(dd, n, use_w, delta_w, use_core);
  return cudaGetLastError();
}

cudaError_t launch_update(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int n,
                          int use_w, double delta_w, int use_core) {
#define UCASE(V)                                                                       \
  case V:                                                                              \
    return fp64 ? update_impl<double, V>(c, dd, hd, n, use_w, delta_w, use_core)       \
                : update_impl<float, V>(c, dd, hd, n, use_w, delta_w, use_core);
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
// next core update.  RelErr per Section III-C.  One CTA, threads (r, y).
// ---------------------------------------------------------------------------
template <typename T, int RP>
__global__ void __launch_bounds__(256) k_objective(const DevDesc* __restrict__ d, int commit) {
  const int r = threadIdx.x, y = threadIdx.y, Y = blockDim.y;
  const int tid = r + y * RP;
  const int NT = RP * Y;
  const int N = d->N, n = N - 1;
  const int k = blockIdx.x;
  DevScalars* sc = d->sc;
  __shared__ double red[256];
  __shared__ double cr[RP];
  __shared__ int is_last;
  constexpr int CAP = (16384 / (int)sizeof(T)) / RP / GRAM_TILE * GRAM_TILE > 0
                          ? (16384 / (int)sizeof(T)) / RP / GRAM_TILE * GRAM_TILE : GRAM_TILE;
  __shared__ T tile[CAP * RP];
  const int R = d->R[k];
  if (commit)  // Gram of the last mode, just updated
    block_gram<T>(reinterpret_cast<const T*>(d->U1[k][n]), d->dims[k][n], R, d->G[k][n], tile, CAP);
  const int64_t I = d->dims[k][n];
  const T* M = reinterpret_cast<const T*>(d->M[k][n]);
  const T* U = reinterpret_cast<const T*>(d->U1[k][n]);
  double acc = 0.0;
  if (r < R)
    for (int64_t i = y; i < I; i += Y) acc = fma((double)M[i * R + r], (double)U[i * R + r], acc);
  red[tid] = acc;
  __syncthreads();
  if (y == 0) {
    double s = 0.0;
    for (int yy = 0; yy < Y; ++yy) s += red[yy * RP + r];
    cr[r] = s;
    if (r < R && commit) sc->cterm[k][r] = s;
  }
  __syncthreads();
  // ||X_hat||^2 = lambda^T (*_m G^(m)) lambda and <X, X_hat> = lambda^T c
  double xx = 0.0;
  for (int p = tid; p < R * R; p += NT) {
    const int a = p / R, b = p % R;
    double g = sc->lam1[k][a] * sc->lam1[k][b];
    for (int m = 0; m < N; ++m) g *= d->G[k][m][p];
    xx += g;
  }
  if (tid < R) xx -= 2.0 * sc->lam1[k][tid] * cr[tid];
  for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(0xffffffffu, xx, o);
  if ((tid & 31) == 0) red[tid >> 5] = xx;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < (NT + 31) / 32; ++q) t += red[q];
    const double x2 = commit ? sc->xnorm2[k] : sc->xnorm2_orig[k];
    const double Fk = 0.5 * (x2 + t);
    const double rel = x2 > 0.0 ? sqrt(fmax(2.0 * Fk, 0.0) / x2) : 0.0;
    if (commit) {
      sc->Fk[k] = Fk;
      sc->relk[k] = rel;
    } else {
      sc->out_relk[k] = rel;
    }
  }
  if (!commit) return;
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(&sc->done_counter[1], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (is_last && tid == 0) {
    __threadfence();
    double F = 0.0, rel = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) {
      F += __ldcg(&sc->Fk[q]);
      rel += __ldcg(&sc->relk[q]);
    }
    sc->F = F;
    sc->relerr = rel / gridDim.x;
    if (!isfinite(F)) sc->nonfinite = 1;
    sc->done_counter[1] = 0;
  }
}

cudaError_t launch_objective(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int commit) {
#define OCASE(V)                                                                                  \
  case V:                                                                                         \
    if (fp64) k_objective<double, V><<<hd.K, dim3(V, 256 / V), 0, c.stream>>>(dd, commit);        \
    else k_objective<float, V><<<hd.K, dim3(V, 256 / V), 0, c.stream>>>(dd, commit);              \
    return cudaGetLastError();
  switch (RP) { CNCPD_FOR_EACH_RP(OCASE) }
#undef OCASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Core update of Eqs. solD / solapgG / eqextraPG with L_d = ||(U^T U)^*||_2
// (Eq. eqLipsLd) and the weight of Eq. eqextrawd.  One CTA per block, FP64.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_core_update(const DevDesc* __restrict__ d, int use_w, double delta_w) {
  const int k = blockIdx.x;
  const int R = d->R[k], N = d->N;
  DevScalars* sc = d->sc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LmaxScratch scr;
  scr.carve(smem_raw, R);
  double* Hs = scr.Hs;
  __shared__ double lh[CNCPD_RMAX];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double h = 1.0;
    for (int m = 0; m < N; ++m) h *= d->G[k][m][e];
    Hs[e] = h;
  }
  const double Ld = lmax_psd<double>(Hs, R, &scr);
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

cudaError_t launch_core_update(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int use_w, double delta_w) {
  const size_t sm = lmax_smem_bytes(hd.Rmax);
  cudaError_t e = allow_smem(k_core_update, sm);
  if (e != cudaSuccess) return e;
  k_core_update<<<hd.K, 256, sm, c.stream>>>(dd, use_w, delta_w);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Iteration bookkeeping.  Begin: t_k and hat w (Appendix A), commit the
// Lipschitz constants of the last accepted sweep as L_{k-2}, snapshot the
// core term and lambda_2 (the factor snapshot is a device memcpy).
// Redo: restore lambda and the core term for the w = 0 re-update.
// ---------------------------------------------------------------------------
__global__ void k_iter_begin(const DevDesc* __restrict__ d) {
  DevScalars* sc = d->sc;
  const int K = d->K, N = d->N;
  const int tid = threadIdx.x;
  const int have_cur = sc->have_cur;
  __syncthreads();
  if (tid == 0) {
    const double t = sc->t;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc->w_hat = (t - 1.0) / tn;
    sc->t = tn;
  }
  if (have_cur) {
    for (int e = tid; e < N * CNCPD_KMAX; e += blockDim.x) {
      const int n = e / CNCPD_KMAX, k = e % CNCPD_KMAX;
      sc->Lprev_u[n][k] = sc->Lcur_u[n][k];
    }
    for (int n = tid; n < N; n += blockDim.x) sc->LCprev[n] = sc->LCcur[n];
    for (int k = tid; k < K; k += blockDim.x) sc->Ldprev[k] = sc->Ldcur[k];
  }
  for (int e = tid; e < K * CNCPD_RMAX; e += blockDim.x) {
    const int k = e / CNCPD_RMAX, r = e % CNCPD_RMAX;
    sc->cterm_save[k][r] = sc->cterm[k][r];
    sc->lamS[k][r] = sc->lam2[k][r];
  }
  __syncthreads();
  if (tid == 0 && have_cur) sc->have_prev = 1;
}

__global__ void k_redo_prepare(const DevDesc* __restrict__ d) {
  DevScalars* sc = d->sc;
  const int K = d->K;
  for (int e = threadIdx.x; e < K * CNCPD_RMAX; e += blockDim.x) {
    const int k = e / CNCPD_RMAX, r = e % CNCPD_RMAX;
    sc->lam1[k][r] = sc->lam2[k][r];
    sc->lam2[k][r] = sc->lamS[k][r];
    sc->cterm[k][r] = sc->cterm_save[k][r];
  }
}

cudaError_t launch_iter_begin(const LaunchCfg& c, const DevDesc* dd, const DevDesc&) {
  k_iter_begin<<<1, 256, 0, c.stream>>>(dd);
  return cudaGetLastError();
}

cudaError_t launch_redo_prepare(const LaunchCfg& c, const DevDesc* dd, const DevDesc&) {
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

cudaError_t launch_grad(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int n,
                        int use_core) {
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][n] > imax ? hd.dims[k][n] : imax;
  {
    const size_t sm = lmax_smem_bytes(hd.Rmax);
    cudaError_t e = fp64 ? allow_smem(k_lipschitz<double>, sm) : allow_smem(k_lipschitz<float>, sm);
    if (e != cudaSuccess) return e;
    if (fp64) k_lipschitz<double><<<hd.K, 256, sm, c.stream>>>(dd, n, use_core, 0, -1, GRAM_TILE);
    else k_lipschitz<float><<<hd.K, 256, sm, c.stream>>>(dd, n, use_core, 0, -1, GRAM_TILE);
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
template <typename S>
__global__ void k_quantize(const S* __restrict__ src, void* dst, void* dst_lo, int st, int64_t rows, int64_t cols,
                           int64_t pitch, double* part) {
  double acc = 0.0;
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / cols;
    const int64_t o = row * pitch + (i - row * cols);
    const double x = (double)src[i];
    double q;
    if (st == ST_F64) {
      reinterpret_cast<double*>(dst)[o] = x;
      q = x;
    } else if (st == ST_F32) {
      const float f = (float)x;
      reinterpret_cast<float*>(dst)[o] = f;
      q = f;
    } else if (st == ST_BF16) {
      const __nv_bfloat16 b = __double2bfloat16(x);
      reinterpret_cast<__nv_bfloat16*>(dst)[o] = b;
      q = (double)__bfloat162float(b);
    } else {
      const float f = (float)x;
      const __nv_bfloat16 hi = __float2bfloat16_rn(f);
      const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
      reinterpret_cast<__nv_bfloat16*>(dst)[o] = hi;
      reinterpret_cast<__nv_bfloat16*>(dst_lo)[o] = lo;
      q = (double)(__bfloat162float(hi) + __bfloat162float(lo));
    }
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

__global__ void k_lmax_one(const double* H, int R, double* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LmaxScratch scr;
  scr.carve(smem_raw, R);
  double* Hs = scr.Hs;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) Hs[e] = H[e];
  const double L = lmax_psd<double>(Hs, R, &scr);
  if (threadIdx.x == 0) *out = L;
}

cudaError_t launch_lmax_host(const double* d_H, int R, double* d_out, cudaStream_t s) {
  const size_t sm = lmax_smem_bytes(R);
  cudaError_t e = allow_smem(k_lmax_one, sm);
  if (e != cudaSuccess) return e;
  k_lmax_one<<<1, 256, sm, s>>>(d_H, R, d_out);
  return cudaGetLastError();
}

}  // namespace cncpd
