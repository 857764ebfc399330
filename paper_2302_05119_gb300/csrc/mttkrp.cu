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
#include "cncpd_internal.cuh"

namespace cncpd {

// ---------------------------------------------------------------------------
// Trailing contraction: one warp owns 32 consecutive rows (one per lane) and
// walks the columns in chunks of 32.  A chunk of X (32 rows x 32 columns) is
// loaded row-coalesced into shared memory and read back transposed; the
// 32 x R chunk of W_t is formed by the warp itself, so warps never wait on
// each other.
// ---------------------------------------------------------------------------
template <int ST, typename T, int RP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_trailing_contract(const DevDesc* __restrict__ d) {
  constexpr int XS = 33;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T (*xs)[32][XS] = reinterpret_cast<T (*)[32][XS]>(smem_raw);
  T (*ws)[32][RP] = reinterpret_cast<T (*)[32][RP]>(smem_raw + sizeof(T) * WARPS * 32 * XS);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int K = d->K, N = d->N, h = d->h;
  const int total = d->lt_prefix[K];
  for (int g = blockIdx.x * WARPS + warp; g < total; g += gridDim.x * WARPS) {
    int k = 0;
    while (d->lt_prefix[k + 1] <= g) ++k;
    const int64_t row0 = (int64_t)(g - d->lt_prefix[k]) * 32;
    const int64_t rows = d->lead_rows[k];
    const int64_t J = d->trail_cols[k];
    const int R = d->R[k];
    const void* X = d->X[k];
    const void* Xlo = d->Xlo[k];
    T acc[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) acc[r] = T(0);
    for (int64_t j0 = 0; j0 < J; j0 += 32) {
      // W_t chunk: lane forms the row for column j0 + lane.
      {
        const int64_t j = j0 + lane;
        T w[RP];
        if (j < J) {
          int idx[CNCPD_NMAX];
          decode(d, k, h, N, j, idx);
#pragma unroll
          for (int r = 0; r < RP; ++r) w[r] = (r < R) ? T(1) : T(0);
          for (int m = h; m < N; ++m) {
            const T* U = reinterpret_cast<const T*>(d->U1[k][m]) + (int64_t)idx[m] * R;
#pragma unroll
            for (int r = 0; r < RP; ++r)
              if (r < R) w[r] *= U[r];
          }
        } else {
#pragma unroll
          for (int r = 0; r < RP; ++r) w[r] = T(0);
        }
#pragma unroll
        for (int r = 0; r < RP; ++r) ws[warp][lane][r] = w[r];
      }
      // X chunk, row-coalesced: instruction q loads 32 consecutive columns of row row0+q.
      {
        const int64_t j = j0 + lane;
        const bool jok = j < J;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
          const int64_t row = row0 + q;
          T v = T(0);
          if (jok && row < rows) v = load_x<ST, T>(X, Xlo, row * J + j);
          xs[warp][q][lane] = v;
        }
      }
      __syncwarp();
#pragma unroll 4
      for (int jj = 0; jj < 32; ++jj) {
        const T x = xs[warp][lane][jj];
#pragma unroll
        for (int r = 0; r < RP; ++r) acc[r] = fma(x, ws[warp][jj][r], acc[r]);
      }
      __syncwarp();
    }
    const int64_t row = row0 + lane;
    if (row < rows) {
      T* P = reinterpret_cast<T*>(d->Pl[k]) + row * R;
#pragma unroll
      for (int r = 0; r < RP; ++r)
        if (r < R) P[r] = acc[r];
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
__global__ void __launch_bounds__(128)
k_lead_contract(const DevDesc* __restrict__ d) {
  constexpr int CH = 64;  // rows per W_l chunk
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
    const bool vec_ok = (J % CPT) == 0;
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
          decode(d, k, 0, h, row, idx);
          w = T(1);
          for (int m = 0; m < h; ++m) w *= reinterpret_cast<const T*>(d->U1[k][m])[(int64_t)idx[m] * R + r];
        }
        wsm[i][r] = w;
      }
      __syncthreads();
      const int nrow = (int)min((int64_t)CH, re - r0);
      if (col0 < J) {
#pragma unroll 2
        for (int i = ty; i < nrow; i += 2) {
          T x[CPT];
          VecLoad<ST, T, CPT>::run(X, Xlo, (r0 + i) * J, col0, J, vec_ok, x);
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            const T w = wsm[i][r];
#pragma unroll
            for (int c = 0; c < CPT; ++c) acc[c][r] = fma(x[c], w, acc[c][r]);
          }
        }
      }
    }
    __syncthreads();
    if (ty == 1) {
#pragma unroll
      for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int r = 0; r < RP; ++r) red[(tx * CPT + c) * RP + r] = acc[c][r];
    }
    __syncthreads();
    if (ty == 0) {
      T* part = reinterpret_cast<T*>(d->partial) + d->partial_off[k] + (int64_t)split * J * R;
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int64_t col = col0 + c;
        if (col < J) {
#pragma unroll
          for (int r = 0; r < RP; ++r)
            if (r < R) part[col * R + r] = acc[c][r] + red[(tx * CPT + c) * RP + r];
        }
      }
    }
  }
}

// Sum of the split partials in fixed order s = 0, 1, ... into Pt.
template <typename T>
__global__ void k_reduce_splits(const DevDesc* __restrict__ d, const int64_t* __restrict__ prefix) {
  const int K = d->K;
  const int64_t total = prefix[K];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (prefix[k + 1] <= e) ++k;
    const int64_t local = e - prefix[k];
    const int64_t stride = d->trail_cols[k] * d->R[k];
    const T* part = reinterpret_cast<const T*>(d->partial) + d->partial_off[k] + local;
    T s = T(0);
    const int ns = d->nsplit[k];
    for (int i = 0; i < ns; ++i) s += part[(int64_t)i * stride];
    reinterpret_cast<T*>(d->Pt[k])[local] = s;
  }
}

// ---------------------------------------------------------------------------
// Level 2: M^(n)[i_n, r] = sum over the other modes of n's group of
// P[.., r] * prod U^(m)[i_m, r].  One CTA per (i_n, block); threads (r, y).
// ---------------------------------------------------------------------------
template <typename T, int RP>
__global__ void k_level2(const DevDesc* __restrict__ d, int n) {
  const int k = blockIdx.y;
  const int64_t in = blockIdx.x;
  const int N = d->N, h = d->h;
  const int m0 = (n < h) ? 0 : h, m1 = (n < h) ? h : N;
  const int64_t In = d->dims[k][n];
  if (in >= In) return;
  const int R = d->R[k];
  const T* P = reinterpret_cast<const T*>((n < h) ? d->Pl[k] : d->Pt[k]);
  T* M = reinterpret_cast<T*>(d->M[k][n]);
  const int64_t total = (n < h) ? d->lead_rows[k] : d->trail_cols[k];
  const int64_t Q = total / In;
  const int r = threadIdx.x;
  const int y = threadIdx.y, Y = blockDim.y;
  typedef typename Acc<T>::type A;
  A acc = 0;
  if (r < R) {
    for (int64_t q = y; q < Q; q += Y) {
      // decode q over the group's modes other than n (C order), then compose the row.
      int idx[CNCPD_NMAX];
      int64_t f = q;
      for (int m = m1 - 1; m >= m0; --m) {
        if (m == n) continue;
        const int64_t I = d->dims[k][m];
        idx[m] = (int)(f % I);
        f /= I;
      }
      idx[n] = (int)in;
      int64_t row = 0;
      for (int m = m0; m < m1; ++m) row = row * d->dims[k][m] + idx[m];
      T p = P[row * R + r];
      for (int m = m0; m < m1; ++m)
        if (m != n) p *= reinterpret_cast<const T*>(d->U1[k][m])[(int64_t)idx[m] * R + r];
      acc += (A)p;
    }
  }
  __shared__ A red[256];
  red[y * RP + r] = acc;
  __syncthreads();
  if (y == 0 && r < R) {
    A s = 0;
    for (int yy = 0; yy < Y; ++yy) s += red[yy * RP + r];
    M[in * R + r] = (T)s;
  }
}

// ------------------------------------------------------------- launchers ----

template <int ST, typename T, int RP>
static cudaError_t trailing_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  const int total = hd.lt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  constexpr int WARPS = (sizeof(T) == 8 && RP > 16) ? 4 : 8;
  constexpr size_t smem = sizeof(T) * WARPS * 32 * (33 + RP);
  auto kern = k_trailing_contract<ST, T, RP, WARPS>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int grid = (total + WARPS - 1) / WARPS;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  grid = grid < c.num_sms * per_sm ? grid : c.num_sms * per_sm;
  kern<<<grid, WARPS * 32, smem, c.stream>>>(dd);
  return cudaGetLastError();
}

template <int ST, typename T, int RP>
static cudaError_t lead_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, const int64_t* d_red_prefix) {
  const int total = hd.tt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  constexpr int CPT = (sizeof(T) == 8) ? (RP <= 16 ? 2 : 1) : (RP <= 20 ? 4 : (RP <= 32 ? 2 : 1));
  constexpr size_t smem = sizeof(T) * (64 * RP + 64 * CPT * RP);
  auto kern = k_lead_contract<ST, T, RP, CPT>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
  if (per_sm < 1) per_sm = 1;
  int grid = total < c.num_sms * per_sm ? total : c.num_sms * per_sm;
  kern<<<grid, 128, smem, c.stream>>>(dd);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_splits<T><<<c.num_sms * 4, 256, 0, c.stream>>>(dd, d_red_prefix);
  return cudaGetLastError();
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
                                  const int64_t* d_red_prefix) {
  CNCPD_DISPATCH_ST_RP(lead_impl, c, dd, hd, d_red_prefix)
}

template <typename T, int RP>
static cudaError_t level2_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int n) {
  int64_t imax = 0;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][n] > imax ? hd.dims[k][n] : imax;
  dim3 block(RP, 256 / RP);
  dim3 grid((unsigned)imax, hd.K);
  k_level2<T, RP><<<grid, block, 0, c.stream>>>(dd, n);
  return cudaGetLastError();
}

cudaError_t launch_level2(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int fp64, int RP, int n) {
#define L2CASE(V) \
  case V: return fp64 ? level2_impl<double, V>(c, dd, hd, n) : level2_impl<float, V>(c, dd, hd, n);
  switch (RP) { CNCPD_FOR_EACH_RP(L2CASE) }
#undef L2CASE
  return cudaErrorInvalidValue;
}

}  // namespace cncpd
