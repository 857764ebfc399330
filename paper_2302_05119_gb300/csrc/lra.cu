// lraCoNCPD-APG kernels (Section III-B, Algorithm 2).
//
// Step (i): unconstrained rank-R~ CPD of every block by ALS (Section IV
// settings): per mode, U~^(n) = X_(n) U~^{odot_-n} V^{-1} with
// V = (U~^T U~)^{circledast_-n}; the MTTKRP reuses the dimension-tree kernels
// with the LRA factors, V^{-1} comes from an FP64 Cholesky factorisation.
// Step (ii): the APG sweep with the collapsed products
//   X_(n) U^{odot_-n}   = U~^(n) (U~^T U)^{circledast_-n}     (Eq. eqlrau)
//   (U^{odot})^T vec(X) = (U^T U~)^{circledast} 1              (Eq. eqlrag)
// and the objective of Eq. cosfunclra by the Gram expansion.
#include "cncpd_internal.cuh"

namespace cncpd {

// C^(n,k) = U~^(n,k)^T U^(n,k) (R~ x R), FP64 output (Table II operations 8, 9).
template <typename T>
__global__ void __launch_bounds__(256) k_cross_gram(const DevDesc* __restrict__ d, int n_begin, int n_end) {
  const int nm = n_end - n_begin;
  const int k = blockIdx.x / nm;
  const int n = n_begin + blockIdx.x % nm;
  const T* A = reinterpret_cast<const T*>(d->Ut[k][n]);
  const T* B = reinterpret_cast<const T*>(d->U1[k][n]);
  const int Ra = d->Rt[k], Rb = d->R[k];
  double* C = d->C[k][n];
  const int64_t I = d->dims[k][n];
  const int P = Ra * Rb;
  __shared__ double red[256];
  const int tid = threadIdx.x;
  for (int p0 = 0; p0 < P; p0 += 256) {
    const int np = min(256, P - p0);
    const int Y = max(1, 256 / np);
    const int p = p0 + tid % np;
    const int y = tid / np;
    double acc = 0.0;
    if (tid < np * Y) {
      const int a = p / Rb, b = p % Rb;
      T part = T(0);
      int cnt = 0;
      for (int64_t i = y; i < I; i += Y) {
        part = fma(A[i * Ra + a], B[i * Rb + b], part);
        if (++cnt == 64) { acc += (double)part; part = T(0); cnt = 0; }
      }
      acc += (double)part;
    }
    red[tid] = acc;
    __syncthreads();
    if (tid < np) {
      double s = 0.0;
      for (int yy = 0; yy < Y; ++yy) s += red[yy * np + tid];
      C[p0 + tid] = s;
    }
    __syncthreads();
  }
}

cudaError_t launch_cross_gram(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n_begin,
                              int n_end) {
  if (n_end <= n_begin) return cudaSuccess;
  const int grid = hd.K * (n_end - n_begin);
  if (fp64) k_cross_gram<double><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end);
  else k_cross_gram<float><<<grid, 256, 0, c.stream>>>(dd, n_begin, n_end);
  return cudaGetLastError();
}

// M^(n,k) = U~^(n) Hc with Hc = (U~^T U)^{circledast_-n} (R~ x R).  Grid
// (row tiles, blocks); threads (r, y).
template <typename T>
__global__ void __launch_bounds__(256) k_collapsed_m(const DevDesc* __restrict__ d, int n) {
  const int k = blockIdx.y;
  const int Rt = d->Rt[k], R = d->R[k], N = d->N;
  const int64_t I = d->dims[k][n];
  __shared__ T Hc[CNCPD_RMAX * CNCPD_RMAX];
  for (int e = threadIdx.x; e < Rt * R; e += blockDim.x) {
    double h = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) h *= d->C[k][m][e];
    Hc[e] = (T)h;
  }
  __syncthreads();
  const T* Ut = reinterpret_cast<const T*>(d->Ut[k][n]);
  T* M = reinterpret_cast<T*>(d->M[k][n]);
  const int rows_per = max(1, (int)blockDim.x / R);
  const int r = threadIdx.x % R;
  const int y = threadIdx.x / R;
  if (y >= rows_per) return;
  for (int64_t i = (int64_t)blockIdx.x * rows_per + y; i < I; i += (int64_t)gridDim.x * rows_per) {
    T acc = T(0);
    for (int q = 0; q < Rt; ++q) acc = fma(Ut[i * Rt + q], Hc[q * R + r], acc);
    M[i * R + r] = acc;
  }
}

cudaError_t launch_collapsed_m(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n) {
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][n] > imax ? hd.dims[k][n] : imax;
  const int rows_per = 256 / (hd.Rmax > 0 ? hd.Rmax : 1);
  unsigned gx = (unsigned)((imax + rows_per - 1) / rows_per);
  if (gx > 1024) gx = 1024;
  dim3 grid(gx, hd.K);
  if (fp64) k_collapsed_m<double><<<grid, 256, 0, c.stream>>>(dd, n);
  else k_collapsed_m<float><<<grid, 256, 0, c.stream>>>(dd, n);
  return cudaGetLastError();
}

// Objective of Eq. cosfunclra at the current factors:
//   F_k = 1/2 (||X~||^2 - 2 lambda^T c + lambda^T (*_m G^(m)) lambda),
//   c_r = sum_q prod_m C^(m)[q, r]  (Eq. eqlrag; also the next core term).
__global__ void __launch_bounds__(64) k_lra_objective(const DevDesc* __restrict__ d) {
  const int K = d->K, N = d->N;
  DevScalars* sc = d->sc;
  __shared__ double cr[CNCPD_RMAX];
  for (int k = 0; k < K; ++k) {
    const int R = d->R[k], Rt = d->Rt[k];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < Rt; ++q) {
        double p = 1.0;
        for (int m = 0; m < N; ++m) p *= d->C[k][m][q * R + r];
        s += p;
      }
      cr[r] = s;
      sc->cterm[k][r] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ip = 0.0, xx = 0.0;
      for (int a = 0; a < R; ++a) {
        const double la = sc->lam1[k][a];
        ip += la * cr[a];
        for (int b = 0; b < R; ++b) {
          double g = 1.0;
          for (int m = 0; m < N; ++m) g *= d->G[k][m][a * R + b];
          xx += la * sc->lam1[k][b] * g;
        }
      }
      const double x2 = sc->xnorm2[k];
      const double Fk = 0.5 * (x2 - 2.0 * ip + xx);
      sc->Fk[k] = Fk;
      sc->relk[k] = x2 > 0.0 ? sqrt(fmax(2.0 * Fk, 0.0) / x2) : 0.0;
      sc->ip[k] = ip;
      sc->xhat2[k] = xx;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double F = 0.0, rel = 0.0;
    for (int k = 0; k < K; ++k) { F += sc->Fk[k]; rel += sc->relk[k]; }
    sc->F = F;
    sc->relerr = rel / K;
    if (!isfinite(F)) sc->nonfinite = 1;
  }
}

cudaError_t launch_lra_objective(const LaunchCfg& c, const DevDesc* dd, const DevDesc&, int, int) {
  k_lra_objective<<<1, 64, 0, c.stream>>>(dd);
  return cudaGetLastError();
}

// ||X~^(k)||^2 = 1^T (*_m U~^(m)^T U~^(m)) 1.
__global__ void k_lra_xnorm(const DevDesc* __restrict__ d) {
  const int k = blockIdx.x;
  const int Rt = d->Rt[k], N = d->N;
  __shared__ double red[256];
  double s = 0.0;
  for (int e = threadIdx.x; e < Rt * Rt; e += blockDim.x) {
    double g = 1.0;
    for (int m = 0; m < N; ++m) g *= d->Gt[k][m][e];
    s += g;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
    d->sc->xnorm2[k] = t;
  }
}

cudaError_t launch_lra_xnorm(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  k_lra_xnorm<<<hd.K, 256, 0, c.stream>>>(dd);
  return cudaGetLastError();
}

// ALS: V = (U~^T U~)^{circledast_-n}, Cholesky V = L L^T in FP64, V^{-1}
// written in the factor type.  status[k] = 1 if V is not positive definite.
template <typename T>
__global__ void __launch_bounds__(64) k_als_solve(const DevDesc* __restrict__ d, int n, const int* active, int* status) {
  const int k = blockIdx.x;
  if (!active[k]) return;
  const int Rt = d->Rt[k], N = d->N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* V = reinterpret_cast<double*>(smem_raw);
  double* Lc = V + Rt * Rt;
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < Rt * Rt; e += blockDim.x) {
    double g = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) g *= d->Gt[k][m][e];
    V[e] = g;
    Lc[e] = 0.0;
  }
  __syncthreads();
  // right-looking Cholesky, column j at a time
  for (int j = 0; j < Rt; ++j) {
    if (tid == 0) {
      double s = V[j * Rt + j];
      for (int l = 0; l < j; ++l) s -= Lc[j * Rt + l] * Lc[j * Rt + l];
      if (!(s > 0.0) || !isfinite(s)) bad = 1;
      Lc[j * Rt + j] = (s > 0.0) ? sqrt(s) : 1.0;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < Rt; i += blockDim.x) {
      double s = V[i * Rt + j];
      for (int l = 0; l < j; ++l) s -= Lc[i * Rt + l] * Lc[j * Rt + l];
      Lc[i * Rt + j] = s / Lc[j * Rt + j];
    }
    __syncthreads();
  }
  // inverse: column c of V^{-1} solves L L^T x = e_c (one thread per column)
  T* Vinv = reinterpret_cast<T*>(d->Vinv[k]);
  for (int c = tid; c < Rt; c += blockDim.x) {
    double z[CNCPD_RMAX];
    for (int i = 0; i < Rt; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l = 0; l < i; ++l) s -= Lc[i * Rt + l] * z[l];
      z[i] = s / Lc[i * Rt + i];
    }
    for (int i = Rt - 1; i >= 0; --i) {
      double s = z[i];
      for (int l = i + 1; l < Rt; ++l) s -= Lc[l * Rt + i] * z[l];
      z[i] = s / Lc[i * Rt + i];
    }
    for (int i = 0; i < Rt; ++i) Vinv[i * Rt + c] = (T)z[i];
  }
  __syncthreads();
  if (tid == 0 && bad) status[k] = 1;
}

cudaError_t launch_als_solve(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n,
                             const int* active, int* status) {
  int rmax = 1;
  for (int k = 0; k < hd.K; ++k) rmax = hd.Rt[k] > rmax ? hd.Rt[k] : rmax;
  const size_t sm = 2 * (size_t)rmax * rmax * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = fp64 ? cudaFuncSetAttribute(k_als_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                         : cudaFuncSetAttribute(k_als_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  if (fp64) k_als_solve<double><<<hd.K, 64, sm, c.stream>>>(dd, n, active, status);
  else k_als_solve<float><<<hd.K, 64, sm, c.stream>>>(dd, n, active, status);
  return cudaGetLastError();
}

// U~^(n)[i, :] = M[i, :] V^{-1}  (the ALS descriptor's M holds X_(n) U~^{odot_-n}).
template <typename T>
__global__ void __launch_bounds__(256) k_als_apply(const DevDesc* __restrict__ d, int n, const int* active) {
  const int k = blockIdx.y;
  if (!active[k]) return;
  const int Rt = d->Rt[k];
  const int64_t I = d->dims[k][n];
  __shared__ T Vs[CNCPD_RMAX * CNCPD_RMAX];
  const T* Vinv = reinterpret_cast<const T*>(d->Vinv[k]);
  for (int e = threadIdx.x; e < Rt * Rt; e += blockDim.x) Vs[e] = Vinv[e];
  __syncthreads();
  const T* M = reinterpret_cast<const T*>(d->M[k][n]);
  T* Ut = reinterpret_cast<T*>(d->Ut[k][n]);
  const int rows_per = max(1, (int)blockDim.x / Rt);
  const int r = threadIdx.x % Rt, y = threadIdx.x / Rt;
  if (y >= rows_per) return;
  for (int64_t i = (int64_t)blockIdx.x * rows_per + y; i < I; i += (int64_t)gridDim.x * rows_per) {
    T acc = T(0);
    for (int q = 0; q < Rt; ++q) acc = fma(M[i * Rt + q], Vs[q * Rt + r], acc);
    Ut[i * Rt + r] = acc;
  }
}

cudaError_t launch_als_apply(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n,
                             const int* active) {
  int64_t imax = 0;
  int rmax = 1;
  for (int k = 0; k < hd.K; ++k) {
    imax = hd.dims[k][n] > imax ? hd.dims[k][n] : imax;
    rmax = hd.Rt[k] > rmax ? hd.Rt[k] : rmax;
  }
  const int rows_per = 256 / rmax;
  unsigned gx = (unsigned)((imax + rows_per - 1) / rows_per);
  if (gx > 1024) gx = 1024;
  dim3 grid(gx, hd.K);
  if (fp64) k_als_apply<double><<<grid, 256, 0, c.stream>>>(dd, n, active);
  else k_als_apply<float><<<grid, 256, 0, c.stream>>>(dd, n, active);
  return cudaGetLastError();
}

// ALS relative error ||X - [[U~]]|| / ||X|| per block by the Gram expansion:
// <X, [[U~]]> = sum_{i,q} M^(N-1)[i, q] U~^(N-1)[i, q] with M^(N-1) taken
// before the last mode's update and U~^(N-1) after it.
template <typename T>
__global__ void __launch_bounds__(256) k_als_relerr(const DevDesc* __restrict__ d, double* relk) {
  const int k = blockIdx.x;
  const int Rt = d->Rt[k], N = d->N, n = N - 1;
  const int64_t I = d->dims[k][n];
  const T* M = reinterpret_cast<const T*>(d->M[k][n]);
  const T* U = reinterpret_cast<const T*>(d->Ut[k][n]);
  __shared__ double red[256];
  double ip = 0.0;
  for (int64_t e = threadIdx.x; e < I * Rt; e += blockDim.x) ip = fma((double)M[e], (double)U[e], ip);
  double xx = 0.0;
  for (int e = threadIdx.x; e < Rt * Rt; e += blockDim.x) {
    double g = 1.0;
    for (int m = 0; m < N; ++m) g *= d->Gt[k][m][e];
    xx += g;
  }
  red[threadIdx.x] = xx - 2.0 * ip;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) s += red[i];
    const double x2 = d->sc->xnorm2_orig[k];
    relk[k] = x2 > 0.0 ? sqrt(fmax(x2 + s, 0.0) / x2) : 0.0;
  }
}

cudaError_t launch_als_relerr(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, double* relk) {
  if (fp64) k_als_relerr<double><<<hd.K, 256, 0, c.stream>>>(dd, relk);
  else k_als_relerr<float><<<hd.K, 256, 0, c.stream>>>(dd, relk);
  return cudaGetLastError();
}

}  // namespace cncpd
