// Dimension-tree MTTKRP kernels (the tensor-streaming hot path).
//
// The MTTKRP of Eq. solapgU, X_(n) U^{odot_-n}, is computed for every mode of
// a sweep from two level-1 contractions that each stream X once (Table II
// operations 6 and 7 without forming the Khatri-Rao matrix):
//   trailing contraction  Pl[row, r] = sum_col X[row, col] * W_t[col, r]
//   lead contraction      Pt[col, r] = sum_row X[row, col] * W_l[row, r]
// where X^(k) is viewed as a lead_rows x trail_cols matrix (modes [0,h) and
// [h,N)), W_t[col, r] = prod_{m>=h} U^(m)[i_m, r] and
// W_l[row, r] = prod_{m<h} U^(m)[i_m, r].  A level-2 kernel then contracts
// Pl (or Pt) with the remaining factors of its group to give M^(n).
// Gauss-Seidel order is kept: the trailing contraction uses the trailing
// factors before the lead modes are updated, the lead contraction uses the
// freshly updated lead factors.
#include <algorithm>

#include "cncpd_internal.cuh"

namespace cncpd {

// 32-bit mixed-radix decode over modes [m0, m1) (each level-1 index range is
// below 2^31, checked at creation).
__device__ __forceinline__ void decode32(const DevDesc* d, int k, int m0, int m1, int flat, int* idx) {
  for (int m = m1 - 1; m >= m0; --m) {
    const int I = (int)d->dims[k][m];
    idx[m] = flat % I;
    flat /= I;
  }
}

// ---------------------------------------------------------------------------
// Trailing contraction: one warp owns 64 consecutive rows (lane l: rows l and
// l + 32) and walks the columns in chunks of 32.  A 64 x 32 chunk of X is
// loaded row-coalesced (128-bit loads when the row length allows) into a
// padded shared tile and read back transposed as float4 (row stride 36
// floats: conflict-free); the 32 x R chunk of W_t is formed by the warp
// itself, so warps never wait on each other.
// ---------------------------------------------------------------------------
template <typename T> struct TrailCfg;
template <> struct TrailCfg<float> { static constexpr int XS = 36; };
template <> struct TrailCfg<double> { static constexpr int XS = 34; };

template <int ST, typename T, int RP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_trailing_contract(const DevDesc* __restrict__ d) {
  constexpr int XS = TrailCfg<T>::XS;
  constexpr int TR = 64;  // rows per warp tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*xs)[TR][XS] = reinterpret_cast<T (*)[TR][XS]>(smem_raw);
  T (*ws)[32][RP] = reinterpret_cast<T (*)[32][RP]>(smem_raw + sizeof(T) * WARPS * TR * XS);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int K = d->K, N = d->N, h = d->h;
  const int total = d->lt_prefix[K];
  for (int g = blockIdx.x * WARPS + warp; g < total; g += gridDim.x * WARPS) {
    int k = 0;
    while (d->lt_prefix[k + 1] <= g) ++k;
    const int64_t row0 = (int64_t)(g - d->lt_prefix[k]) * TR;
    const int64_t rows = d->lead_rows[k];
    const int64_t J = d->trail_cols[k];
    const int R = d->R[k];
    const void* X = d->X[k];
    const void* Xlo = d->Xlo[k];
    const int64_t pitch = d->pitch[k];
    const bool vec = (ST == ST_F32) && (pitch % 4 == 0);
    T acc0[RP], acc1[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) acc0[r] = acc1[r] = T(0);
    for (int64_t j0 = 0; j0 < J; j0 += 32) {
      // W_t chunk: lane forms the row for column j0 + lane.
      {
        const int64_t j = j0 + lane;
        T w[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) w[r] = (r < R && j < J) ? T(1) : T(0);
        if (j < J) {
          int idx[CNCPD_NMAX];
          decode32(d, k, h, N, (int)j, idx);
          for (int m = h; m < N; ++m) {
            const T* U = reinterpret_cast<const T*>(d->U1[k][m]) + (int64_t)idx[m] * R;
#pragma unroll
            for (int r = 0; r < RP; ++r)
              if (r < R) w[r] *= U[r];
          }
        }
#pragma unroll
        for (int r = 0; r < RP; ++r) ws[warp][lane][r] = w[r];
      }
      // X chunk (64 x 32) into the padded tile
      if constexpr (ST == ST_F32) {
        if (vec && j0 + 32 <= J) {
          const float* Xf = reinterpret_cast<const float*>(X);
          const int cq = (lane & 7) * 4;
          float4 v[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int64_t row = row0 + q * 4 + (lane >> 3);
            v[q] = (row < rows) ? __ldg(reinterpret_cast<const float4*>(Xf + row * pitch + j0 + cq))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) *reinterpret_cast<float4*>(&xs[warp][q * 4 + (lane >> 3)][cq]) = v[q];
        } else {
          const int64_t j = j0 + lane;
#pragma unroll 8
          for (int q = 0; q < TR; ++q) {
            const int64_t row = row0 + q;
            xs[warp][q][lane] = (j < J && row < rows) ? load_x<ST, T>(X, Xlo, row * pitch + j) : T(0);
          }
        }
      } else {
        const int64_t j = j0 + lane;
#pragma unroll 8
        for (int q = 0; q < TR; ++q) {
          const int64_t row = row0 + q;
          xs[warp][q][lane] = (j < J && row < rows) ? load_x<ST, T>(X, Xlo, row * pitch + j) : T(0);
        }
      }
      __syncwarp();
      if constexpr (sizeof(T) == 4) {
#pragma unroll 2
        for (int jj = 0; jj < 32; jj += 4) {
          const float4 xa = *reinterpret_cast<const float4*>(&xs[warp][lane][jj]);
          const float4 xb = *reinterpret_cast<const float4*>(&xs[warp][lane + 32][jj]);
          const float a4[4] = {xa.x, xa.y, xa.z, xa.w};
          const float b4[4] = {xb.x, xb.y, xb.z, xb.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int r = 0; r < RP; ++r) {
              const T wv = ws[warp][jj + q][r];
              acc0[r] = fma(a4[q], wv, acc0[r]);
              acc1[r] = fma(b4[q], wv, acc1[r]);
            }
          }
        }
      } else {
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) {
          const T xa = xs[warp][lane][jj];
          const T xb = xs[warp][lane + 32][jj];
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            const T wv = ws[warp][jj][r];
            acc0[r] = fma(xa, wv, acc0[r]);
            acc1[r] = fma(xb, wv, acc1[r]);
          }
        }
      }
      __syncwarp();
    }
    T* P = reinterpret_cast<T*>(d->Pl[k]);
    if (row0 + lane < rows) {
#pragma unroll
      for (int r = 0; r < RP; ++r)
        if (r < R) P[(row0 + lane) * R + r] = acc0[r];
    }
    if (row0 + lane + 32 < rows) {
#pragma unroll
      for (int r = 0; r < RP; ++r)
        if (r < R) P[(row0 + lane + 32) * R + r] = acc1[r];
    }
  }
}

// ---------------------------------------------------------------------------
// Lead contraction (split over rows): a CTA owns CPT*64 consecutive columns
// and a slice of rows; thread (tx, ty) owns CPT columns and every second row
// of the slice.  W_l for a chunk of 64 rows is formed cooperatively in shared
// memory.  Each CTA writes its partial Pt slice to the split buffer; a second
// kernel adds the slices in fixed order (deterministic).
// ---------------------------------------------------------------------------
template <int ST, typename T, int CPT>
struct VecLoad {
  static __device__ __forceinline__ void run(const void* X, const void* Xlo, int64_t base, int64_t col0,
                                             int64_t J, bool vec_ok, T* x) {
    const int64_t i = base + col0;
    if (vec_ok && col0 + CPT <= J) {
      if constexpr (ST == ST_F32 && CPT == 4) {
        float4 v = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + i));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
        return;
      } else if constexpr (ST == ST_F32 && CPT == 2) {
        float2 v = __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(X) + i));
        x[0] = v.x; x[1] = v.y;
        return;
      } else if constexpr (ST == ST_F64 && CPT == 2) {
        double2 v = __ldg(reinterpret_cast<const double2*>(reinterpret_cast<const double*>(X) + i));
        x[0] = v.x; x[1] = v.y;
        return;
      } else if constexpr ((ST == ST_BF16 || ST == ST_BF16X2) && CPT == 4) {
        uint2 v = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(X) + i));
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&v.x);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&v.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        x[0] = fa.x; x[1] = fa.y; x[2] = fb.x; x[3] = fb.y;
        if constexpr (ST == ST_BF16X2) {
          uint2 u = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(Xlo) + i));
          __nv_bfloat162 c = *reinterpret_cast<__nv_bfloat162*>(&u.x);
          __nv_bfloat162 e = *reinterpret_cast<__nv_bfloat162*>(&u.y);
          float2 fc = __bfloat1622float2(c), fe = __bfloat1622float2(e);
          x[0] += fc.x; x[1] += fc.y; x[2] += fe.x; x[3] += fe.y;
        }
        return;
      }
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) x[c] = (col0 + c < J) ? load_x<ST, T>(X, Xlo, i + c) : T(0);
  }
};

template <int ST, typename T, int RP, int CPT>
__global__ void __launch_bounds__(256)
k_lead_contract(const DevDesc* __restrict__ d) {
  constexpr int CH = 64;   // rows per W_l chunk
  constexpr int GR = 4;    // row groups (threads 64*g .. 64*g+63)
  constexpr int UNR = 4;   // rows loaded per batch by one thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*wsm)[RP] = reinterpret_cast<T (*)[RP]>(smem_raw);
  T* red = reinterpret_cast<T*>(smem_raw + sizeof(T) * CH * RP);
  const int tx = threadIdx.x & 63;
  const int ty = threadIdx.x >> 6;
  const int K = d->K, h = d->h;
  const int total = d->tt_prefix[K];
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    int k = 0;
    while (d->tt_prefix[k + 1] <= u) ++k;
    const int local = u - d->tt_prefix[k];
    const int ctile = local % d->tt_ctiles[k];
    const int split = local / d->tt_ctiles[k];
    const int64_t rows = d->lead_rows[k];
    const int64_t J = d->trail_cols[k];
    const int R = d->R[k];
    const int64_t rb = (int64_t)split * d->split_rows[k];
    const int64_t re = min(rows, rb + d->split_rows[k]);
    const int64_t col0 = (int64_t)ctile * 64 * CPT + (int64_t)tx * CPT;
    const int64_t pitch = d->pitch[k];
    const bool vec_ok = (pitch % CPT) == 0;
    const void* X = d->X[k];
    const void* Xlo = d->Xlo[k];
    T acc[CPT][RP];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
      for (int r = 0; r < RP; ++r) acc[c][r] = T(0);
    for (int64_t r0 = rb; r0 < re; r0 += CH) {
      __syncthreads();
      for (int e = threadIdx.x; e < CH * RP; e += blockDim.x) {
        const int i = e / RP, r = e % RP;
        const int64_t row = r0 + i;
        T w = T(0);
        if (row < re && r < R) {
          int idx[CNCPD_NMAX];
          decode32(d, k, 0, h, (int)row, idx);
          w = T(1);
          for (int m = 0; m < h; ++m) w *= reinterpret_cast<const T*>(d->U1[k][m])[(int64_t)idx[m] * R + r];
        }
        wsm[i][r] = w;
      }
      __syncthreads();
      const int nrow = (int)min((int64_t)CH, re - r0);
      if (col0 < J) {
        for (int i = ty; i < nrow; i += GR * UNR) {
          T x[UNR][CPT];
#pragma unroll
          for (int q = 0; q < UNR; ++q) {
            const int ii = i + q * GR;
            if (ii < nrow) {
              VecLoad<ST, T, CPT>::run(X, Xlo, (r0 + ii) * pitch, col0, J, vec_ok, x[q]);
            } else {
#pragma unroll
              for (int c = 0; c < CPT; ++c) x[q][c] = T(0);
            }
          }
#pragma unroll
          for (int q = 0; q < UNR; ++q) {
            const int ii = min(i + q * GR, CH - 1);
#pragma unroll
            for (int r = 0; r < RP; ++r) {
              const T w = wsm[ii][r];
#pragma unroll
              for (int c = 0; c < CPT; ++c) acc[c][r] = fma(x[q][c], w, acc[c][r]);
            }
          }
        }
      }
    }
    // reduce the GR row groups (groups 1..GR-1 park their sums in shared memory)
    __syncthreads();
    if (ty > 0) {
#pragma unroll
      for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int r = 0; r < RP; ++r) red[((ty - 1) * 64 * CPT + tx * CPT + c) * RP + r] = acc[c][r];
    }
    __syncthreads();
    if (ty == 0) {
      T* part = reinterpret_cast<T*>(d->partial) + d->partial_off[k] + (int64_t)split * J * R;
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int64_t col = col0 + c;
        if (col < J) {
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            if (r < R) {
              T s = acc[c][r];
              for (int g = 1; g < GR; ++g) s += red[((g - 1) * 64 * CPT + tx * CPT + c) * RP + r];
              part[col * R + r] = s;
            }
          }
        }
      }
    }
  }
}

// Sum of the split partials into Pt: a CTA takes 32 consecutive entries;
// thread group g (of 8) adds splits g, g + 8, ... and the 8 group sums are
// added in group order (fixed order: deterministic).
template <typename T>
struct SplitArgs {
  int K, pad;
  int64_t prefix[CNCPD_KMAX + 1];  // first output element of each block
  int64_t stride[CNCPD_KMAX];      // elements per split (trail_cols * R)
  int nsplit[CNCPD_KMAX];
  const T* part[CNCPD_KMAX];
  T* out[CNCPD_KMAX];
};

// One thread per output element, the splits added in order (sum_splits).
template <typename T>
__global__ void __launch_bounds__(256) k_reduce_splits(const __grid_constant__ SplitArgs<T> a) {
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t total = a.prefix[a.K];
  if (e >= total) return;
  int k = 0;
  while (a.prefix[k + 1] <= e) ++k;
  const int64_t local = e - a.prefix[k];
  a.out[k][local] = sum_splits<T>(a.part[k] + local, a.nsplit[k], a.stride[k]);
}

// ---------------------------------------------------------------------------
// Level 2: with the level-1 partial P of n's group viewed as [A][I_n][B][R]
// (A = product of the group's sizes before n, B = after n),
//   M^(n)[i_n, r] = sum_{a,b} P[a, i_n, b, r] * Wa[a, r] * Wb[b, r],
// Wa / Wb the Khatri-Rao rows of the group's other factors.  One CTA per
// (i_n, block); thread t keeps r = t mod R fixed and strides over the flat
// (a, b, r) range, so consecutive threads read consecutive P entries.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T kr_row(const DevDesc* d, int k, int m0, int m1, int flat, int r, int R) {
  // prod_{m in [m0, m1)} U^(m)[i_m(flat), r]  (C-order mixed radix; 32-bit:
  // the level-1 partials are limited to 2^31 entries)
  if (m1 - m0 == 1) return reinterpret_cast<const T*>(d->U1[k][m0])[flat * R + r];
  T w = T(1);
  for (int m = m1 - 1; m >= m0; --m) {
    const int I = (int)d->dims[k][m];
    const int im = flat % I;
    flat /= I;
    w *= reinterpret_cast<const T*>(d->U1[k][m])[im * R + r];
  }
  return w;
}

template <typename T>
__global__ void __launch_bounds__(256) k_level2(const DevDesc* __restrict__ d, int n) {
  // Generic form (groups of three or more modes): one CTA per (i_n, block).
  const int k = blockIdx.y;
  const int64_t in = blockIdx.x;
  const int N = d->N, h = d->h;
  const int m0 = (n < h) ? 0 : h, m1 = (n < h) ? h : N;
  const int64_t In = d->dims[k][n];
  if (in >= In) return;
  // a block whose tensor pass had no units (inactive in a restricted
  // descriptor) has no new level-1 product
  if ((n < h) ? d->lt_prefix[k + 1] == d->lt_prefix[k] : d->tt_prefix[k + 1] == d->tt_prefix[k]) return;
  const int R = d->R[k];
  const T* P = reinterpret_cast<const T*>((n < h) ? d->Pl[k] : d->Pt[k]);
  int A = 1, B = 1;
  for (int m = m0; m < n; ++m) A *= (int)d->dims[k][m];
  for (int m = n + 1; m < m1; ++m) B *= (int)d->dims[k][m];
  const int BR = B * R;
  const int stride = (blockDim.x / R) * R;
  const int t = threadIdx.x;
  typedef typename Acc<T>::type AT;
  AT acc = 0;
  const int r = t % R;
  if (t < stride) {
    const int total = A * BR;
    const int sq = stride / BR, sr = stride % BR;
    int a = t / BR, e = t % BR, b = e / R;
    const int bq = sr / R;  // stride and BR are multiples of R
    for (int f = t; f < total; f += stride) {
      T p = P[((int64_t)a * In + in) * BR + e];
      if (n > m0) p *= kr_row<T>(d, k, m0, n, a, r, R);
      if (n + 1 < m1) p *= kr_row<T>(d, k, n + 1, m1, b, r, R);
      acc += (AT)p;
      a += sq;
      e += sr;
      b += bq;
      if (e >= BR) { e -= BR; b -= B; ++a; }
    }
  }
  __shared__ AT red[256];
  red[t] = acc;
  __syncthreads();
  if (t < R) {
    AT s = 0;
    for (int q = t; q < stride; q += R) s += red[q];
    reinterpret_cast<T*>(d->M[k][n])[in * R + t] = (T)s;
  }
}

// ------------------------------------------------------------- launchers ----

template <int ST, typename T, int RP>
static cudaError_t trailing_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  const int total = hd.lt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  constexpr int WARPS = (sizeof(T) == 8 && RP > 16) ? 4 : 8;
  constexpr size_t smem = sizeof(T) * WARPS * (64 * TrailCfg<T>::XS + 32 * RP);
  auto kern = k_trailing_contract<ST, T, RP, WARPS>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int grid = (total + WARPS - 1) / WARPS;
  int per_sm = 0;  // trailing tiles are 64 rows
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  grid = grid < c.num_sms * per_sm ? grid : c.num_sms * per_sm;
  kern<<<grid, WARPS * 32, smem, c.stream>>>(dd);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t reduce_splits_impl(const LaunchCfg& c, const DevDesc& hd) {
  SplitArgs<T> a{};
  a.K = hd.K;
  a.prefix[0] = 0;
  for (int k = 0; k < hd.K; ++k) {
    a.stride[k] = hd.trail_cols[k] * hd.R[k];
    a.prefix[k + 1] = a.prefix[k] + a.stride[k];
    a.nsplit[k] = hd.nsplit[k];
    a.part[k] = reinterpret_cast<const T*>(hd.partial) + hd.partial_off[k];
    a.out[k] = reinterpret_cast<T*>(hd.Pt[k]);
  }
  const int64_t blocks = (a.prefix[hd.K] + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  carve<k_reduce_splits<T>>();
  cudaError_t e = launch_pdl(k_reduce_splits<T>, dim3((unsigned)blocks), dim3(256), 0, c.stream, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_reduce_splits(const LaunchCfg& c, const DevDesc& hd, int fp64) {
  return fp64 ? reduce_splits_impl<double>(c, hd) : reduce_splits_impl<float>(c, hd);
}

template <int ST, typename T, int RP>
static cudaError_t lead_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, const int64_t* d_red_prefix,
                             int with_reduce) {
  const int total = hd.tt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  constexpr int CPT = (sizeof(T) == 8) ? (RP <= 16 ? 2 : 1) : (RP <= 20 ? 4 : (RP <= 32 ? 2 : 1));
  constexpr size_t smem = sizeof(T) * (64 * RP + 3 * 64 * CPT * RP);
  auto kern = k_lead_contract<ST, T, RP, CPT>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (per_sm < 1) per_sm = 1;
  int grid = total < c.num_sms * per_sm ? total : c.num_sms * per_sm;
  kern<<<grid, 256, smem, c.stream>>>(dd);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  (void)d_red_prefix;
  if (!with_reduce) return cudaSuccess;
  return launch_reduce_splits(c, hd, sizeof(T) == 8);
}

int lead_cpt(int fp64, int RP) {
  if (fp64) return RP <= 16 ? 2 : 1;
  return RP <= 20 ? 4 : (RP <= 32 ? 2 : 1);
}

#define CNCPD_DISPATCH_ST_RP(FN, ...)                                              \
  switch (st) {                                                                     \
    case ST_F64:                                                                    \
      switch (RP) {                                                                 \
        case 4: return FN<ST_F64, double, 4>(__VA_ARGS__);                          \
        case 8: return FN<ST_F64, double, 8>(__VA_ARGS__);                          \
        case 10: return FN<ST_F64, double, 10>(__VA_ARGS__);                        \
        case 12: return FN<ST_F64, double, 12>(__VA_ARGS__);                        \
        case 16: return FN<ST_F64, double, 16>(__VA_ARGS__);                        \
        case 20: return FN<ST_F64, double, 20>(__VA_ARGS__);                        \
        case 24: return FN<ST_F64, double, 24>(__VA_ARGS__);                        \
        case 32: return FN<ST_F64, double, 32>(__VA_ARGS__);                        \
        case 40: return FN<ST_F64, double, 40>(__VA_ARGS__);                        \
        case 48: return FN<ST_F64, double, 48>(__VA_ARGS__);                        \
        case 64: return FN<ST_F64, double, 64>(__VA_ARGS__);                        \
      }                                                                             \
      break;                                                                        \
    case ST_F32:                                                                    \
      switch (RP) {                                                                 \
        case 4: return FN<ST_F32, float, 4>(__VA_ARGS__);                           \
        case 8: return FN<ST_F32, float, 8>(__VA_ARGS__);                           \
        case 10: return FN<ST_F32, float, 10>(__VA_ARGS__);                         \
        case 12: return FN<ST_F32, float, 12>(__VA_ARGS__);                         \
        case 16: return FN<ST_F32, float, 16>(__VA_ARGS__);                         \
        case 20: return FN<ST_F32, float, 20>(__VA_ARGS__);                         \
        case 24: return FN<ST_F32, float, 24>(__VA_ARGS__);                         \
        case 32: return FN<ST_F32, float, 32>(__VA_ARGS__);                         \
        case 40: return FN<ST_F32, float, 40>(__VA_ARGS__);                         \
        case 48: return FN<ST_F32, float, 48>(__VA_ARGS__);                         \
        case 64: return FN<ST_F32, float, 64>(__VA_ARGS__);                         \
      }                                                                             \
      break;                                                                        \
    case ST_BF16:                                                                   \
      switch (RP) {                                                                 \
        case 4: return FN<ST_BF16, float, 4>(__VA_ARGS__);                          \
        case 8: return FN<ST_BF16, float, 8>(__VA_ARGS__);                          \
        case 10: return FN<ST_BF16, float, 10>(__VA_ARGS__);                        \
        case 12: return FN<ST_BF16, float, 12>(__VA_ARGS__);                        \
        case 16: return FN<ST_BF16, float, 16>(__VA_ARGS__);                        \
        case 20: return FN<ST_BF16, float, 20>(__VA_ARGS__);                        \
        case 24: return FN<ST_BF16, float, 24>(__VA_ARGS__);                        \
        case 32: return FN<ST_BF16, float, 32>(__VA_ARGS__);                        \
        case 40: return FN<ST_BF16, float, 40>(__VA_ARGS__);                        \
        case 48: return FN<ST_BF16, float, 48>(__VA_ARGS__);                        \
        case 64: return FN<ST_BF16, float, 64>(__VA_ARGS__);                        \
      }                                                                             \
      break;                                                                        \
    case ST_BF16X2:                                                                 \
      switch (RP) {                                                                 \
        case 4: return FN<ST_BF16X2, float, 4>(__VA_ARGS__);                        \
        case 8: return FN<ST_BF16X2, float, 8>(__VA_ARGS__);                        \
        case 10: return FN<ST_BF16X2, float, 10>(__VA_ARGS__);                      \
        case 12: return FN<ST_BF16X2, float, 12>(__VA_ARGS__);                      \
        case 16: return FN<ST_BF16X2, float, 16>(__VA_ARGS__);                      \
        case 20: return FN<ST_BF16X2, float, 20>(__VA_ARGS__);                      \
        case 24: return FN<ST_BF16X2, float, 24>(__VA_ARGS__);                      \
        case 32: return FN<ST_BF16X2, float, 32>(__VA_ARGS__);                      \
        case 40: return FN<ST_BF16X2, float, 40>(__VA_ARGS__);                      \
        case 48: return FN<ST_BF16X2, float, 48>(__VA_ARGS__);                      \
        case 64: return FN<ST_BF16X2, float, 64>(__VA_ARGS__);                      \
      }                                                                             \
      break;                                                                        \
  }                                                                                 \
  return cudaErrorInvalidValue;

cudaError_t launch_trailing_contract(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int st, int RP) {
  CNCPD_DISPATCH_ST_RP(trailing_impl, c, dd, hd)
}

cudaError_t launch_lead_contract(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int st, int RP,
                                  const int64_t* d_red_prefix, int with_reduce) {
  CNCPD_DISPATCH_ST_RP(lead_impl, c, dd, hd, d_red_prefix, with_reduce)
}

cudaError_t launch_level2(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int n) {
  (void)RP;
  const int gsize = (n < hd.h) ? hd.h : hd.N - hd.h;
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][n] > imax ? hd.dims[k][n] : imax;
  if (gsize == 2) return launch_mode_prep(c, dd, hd, fp64, n, 0, -1, 2);
  dim3 grid((unsigned)imax, hd.K);
  if (fp64) k_level2<double><<<grid, 256, 0, c.stream>>>(dd, n);
  else k_level2<float><<<grid, 256, 0, c.stream>>>(dd, n);
  return cudaGetLastError();
}

}  // namespace cncpd
