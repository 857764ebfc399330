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

// C^(n,k) = U~^(n,k)^T U^(n,k) (R~ x R), FP64 output (Table II operations 8, 9),
// formed like the Grams: the rows are cut into chunks of CROSS_ROWS rows, each
// chunk gives one FMA chain in the factor type per entry (k_cross_chunks, one
// CTA per chunk, rows staged in shared memory), and the chunk values are
// added in chunk order (k_cross_reduce, compensated FP32 for FP32 factors).
template <typename T>
__global__ void __launch_bounds__(256) k_cross_chunks(const DevDesc* __restrict__ d, int n0, int n1) {
  const int nm = n1 - n0;
  const int k = blockIdx.y / nm, n = n0 + blockIdx.y % nm;
  const int c = blockIdx.x;
  const int64_t I = d->dims[k][n];
  const int64_t row0 = (int64_t)c * CROSS_ROWS;
  if (c >= d->cgnc[n] || row0 >= I) return;
  const int rows = (int)min((int64_t)CROSS_ROWS, I - row0);
  const int Ra = d->Rt[k], Rb = d->R[k];
  __shared__ T As[CROSS_ROWS * CNCPD_RMAX];
  __shared__ T Bs[CROSS_ROWS * CNCPD_RMAX];
  const T* __restrict__ A = reinterpret_cast<const T*>(d->Ut[k][n]) + row0 * Ra;
  const T* __restrict__ B = reinterpret_cast<const T*>(d->U1[k][n]) + row0 * Rb;
#pragma unroll 4
  for (int e = threadIdx.x; e < rows * Ra; e += 256) As[e] = A[e];
#pragma unroll 4
  for (int e = threadIdx.x; e < rows * Rb; e += 256) Bs[e] = B[e];
  __syncthreads();
  T* out = reinterpret_cast<T*>(d->Cp[n]) + ((size_t)k * d->cgnc[n] + c) * d->cld;
  for (int p = threadIdx.x; p < Ra * Rb; p += 256) {
    const int a = p / Rb, b = p % Rb;
    T s = T(0);
    for (int i = 0; i < rows; ++i) s = fma(As[i * Ra + a], Bs[i * Rb + b], s);
    out[p] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_cross_reduce(const DevDesc* __restrict__ d, int n0, int n1) {
  const int nm = n1 - n0;
  const int k = blockIdx.x / nm, n = n0 + blockIdx.x % nm;
  const int P = d->Rt[k] * d->R[k];
  const int nch = (int)((d->dims[k][n] + CROSS_ROWS - 1) / CROSS_ROWS);
  const T* gp = reinterpret_cast<const T*>(d->Cp[n]) + (size_t)k * d->cgnc[n] * d->cld;
  double* C = d->C[k][n];
  for (int p = threadIdx.x; p < P; p += 256) C[p] = gram_sum<T>(gp, nch, d->cld, p);
}

template <typename T>
static cudaError_t cross_gram_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int n_begin, int n_end) {
  const int nm = n_end - n_begin;
  int cmax = 1;
  for (int n = n_begin; n < n_end; ++n) cmax = hd.cgnc[n] > cmax ? hd.cgnc[n] : cmax;
  k_cross_chunks<T><<<dim3((unsigned)cmax, (unsigned)(hd.K * nm)), 256, 0, c.stream>>>(dd, n_begin, n_end);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_cross_reduce<T><<<hd.K * nm, 256, 0, c.stream>>>(dd, n_begin, n_end);
  return cudaGetLastError();
}

cudaError_t launch_cross_gram(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int n_begin,
                              int n_end) {
  if (n_end <= n_begin) return cudaSuccess;
  return fp64 ? cross_gram_impl<double>(c, dd, hd, n_begin, n_end) : cross_gram_impl<float>(c, dd, hd, n_begin, n_end);
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
// One CTA per block, FP64 throughout; the last CTA to finish adds the blocks
// up in order and publishes F to the host mirror.
__global__ void __launch_bounds__(256) k_lra_objective(const DevDesc* __restrict__ d) {
  const int N = d->N, k = blockIdx.x, tid = threadIdx.x;
  DevScalars* sc = d->sc;
  const int R = d->R[k], Rt = d->Rt[k];
  __shared__ double pr[CNCPD_RMAX * CNCPD_RMAX];
  __shared__ double part[8][CNCPD_RMAX];
  __shared__ double wsum[8];
  __shared__ int is_last;
  // prod_m C^(m)[q, r] for every (q, r)
  for (int p = tid; p < Rt * R; p += 256) {
    double v = 1.0;
    for (int m = 0; m < N; ++m) v *= d->C[k][m][p];
    pr[p] = v;
  }
  // lambda^T (*_m G^(m)) lambda, one term per thread and (a, b)
  double xx = 0.0;
  for (int p = tid; p < R * R; p += 256) {
    double g = sc->lam1[k][p / R] * sc->lam1[k][p % R];
    for (int m = 0; m < N; ++m) g *= d->G[k][m][p];
    xx += g;
  }
  __syncthreads();
  // c_r: the rows q = y, y + Y, ... in thread (y, r), then the Y partial sums in order
  const int Y = min(8, 256 / R);
  if (tid < Y * R) {
    const int y = tid / R, r = tid % R;
    double s = 0.0;
    for (int q = y; q < Rt; q += Y) s += pr[q * R + r];
    part[y][r] = s;
  }
  __syncthreads();
  if (tid < R) {
    double s = 0.0;
    for (int y = 0; y < Y; ++y) s += part[y][tid];
    sc->cterm[k][tid] = s;
    xx -= 2.0 * sc->lam1[k][tid] * s;
  }
  for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(0xffffffffu, xx, o);
  if ((tid & 31) == 0) wsum[tid >> 5] = xx;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += wsum[q];
    const double x2 = sc->xnorm2[k];
    const double Fk = 0.5 * (x2 + t);
    sc->Fk[k] = Fk;
    sc->relk[k] = sqrt(fmax(2.0 * Fk, 0.0) * sc->inv_xnorm2[k]);
  }
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
    const double relerr = rel / gridDim.x;
    sc->F = F;
    sc->relerr = relerr;
    if (!isfinite(F)) sc->nonfinite = 1;
    sc->done_counter[1] = 0;
    if (d->hm) {
      HostMirror* hm = d->hm;
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

cudaError_t launch_lra_objective(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int, int) {
  k_lra_objective<<<hd.K, 256, 0, c.stream>>>(dd);
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
