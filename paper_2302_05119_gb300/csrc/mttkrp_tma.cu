// TMA-staged level-1 contractions of the dimension tree for FP32 and BF16
// tensors (BF16 elements are widened to FP32 in registers; FP32 accumulate).
//
// Both kernels stream X^(k) (viewed as lead_rows x trail_cols, row pitch a
// multiple of 16 elements) from HBM exactly once.  One thread issues
// cp.async.bulk.tensor copies of X tiles into a ring of shared-memory stages
// guarded by mbarriers (arrive.expect_tx), three warps take turns writing the
// matching Khatri-Rao rows of the factors next to them (a stage is full after
// both arrivals and all bytes), and eight consumer warps accumulate with
// packed fma.rn.f32x2.  CTAs are persistent (one per SM) and walk a static list of
// work units.  Every mbarrier wait is bounded in time: on expiry the kernel
// sets the error word, stops issuing copies, waits for the copies already in
// flight and returns.
#include <algorithm>

#include "cncpd_internal.cuh"
#include "tma.cuh"

namespace cncpd {

// 32-bit mixed-radix decode over modes [m0, m1).
__device__ __forceinline__ void decode32_t(const DevDesc* d, int k, int m0, int m1, int flat, int* idx) {
  for (int m = m1 - 1; m >= m0; --m) {
    const int I = (int)d->dims[k][m];
    idx[m] = flat % I;
    flat /= I;
  }
}

// The work units of this CTA: the host's balanced list when there is one,
// else every gridDim.x-th unit.  unit(j) for j = first; j < end; j += step.
struct Units {
  const int* ids;
  int first, end, step;
  __device__ __forceinline__ Units(const int* sched, int total) {
    if (sched) {
      ids = sched + gridDim.x + 1;
      first = __ldg(sched + blockIdx.x);
      end = __ldg(sched + blockIdx.x + 1);
      step = 1;
    } else {
      ids = nullptr;
      first = blockIdx.x;
      end = total;
      step = gridDim.x;
    }
  }
  __device__ __forceinline__ int unit(int j) const { return ids ? __ldg(ids + j) : j; }
};

// Unit g of the trailing pass: block k, first row, and the column range
// [jb, je) of its split (the whole row when the block is not split).
struct TrailUnit {
  int k, row0, jb, je, split;
  __device__ __forceinline__ TrailUnit(const DevDesc* d, int g, int rows_per_tile) {
    k = 0;
    while (d->lt_prefix[k + 1] <= g) ++k;
    const int local = g - d->lt_prefix[k];
    const int js = d->lt_js[k];
    split = local % js;
    row0 = (local / js) * rows_per_tile;
    const int J = (int)d->trail_cols[k];
    jb = split * d->lt_jc[k];
    je = min(J, jb + d->lt_jc[k]);
  }
};

// Sixteen bytes of X as FP32 values: four FP32 or eight BF16 elements.
template <typename XT>
struct XChunk {
  static constexpr int N = 16 / (int)sizeof(XT);
};

__device__ __forceinline__ void widen(const uint4& raw, float (&v)[4], float) {
  v[0] = __uint_as_float(raw.x);
  v[1] = __uint_as_float(raw.y);
  v[2] = __uint_as_float(raw.z);
  v[3] = __uint_as_float(raw.w);
}
// BF16 -> FP32 is exact: the 16 bits become the high half of the FP32 word.
__device__ __forceinline__ void widen(const uint4& raw, float (&v)[8], __nv_bfloat16) {
  const uint32_t u[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(u[i] << 16);
    v[2 * i + 1] = __uint_as_float(u[i] & 0xffff0000u);
  }
}
// Four consecutive elements (16 bytes of FP32, 8 bytes of BF16).
__device__ __forceinline__ float4 load4(const unsigned char* p, float) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 load4(const unsigned char* p, __nv_bfloat16) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                     __uint_as_float(u.y & 0xffff0000u));
}

// ---------------------------------------------------------------------------
// Trailing contraction Pl[row, r] = sum_col X[row, col] W_t[col, r].
// Tile = 256 rows; stage = 256 rows x 128 bytes (32 FP32 or 64 BF16 columns,
// 32 KiB, 128-byte swizzle).  Consumer warp w owns rows 32 w .. 32 w + 31 of
// the tile; lane (i, cq) = (lane mod 8, lane / 8) takes rows 32 w + i + 8 t
// (t = 0..3) and the cq-th quarter of the stage's columns, so each
// Khatri-Rao value read from shared memory feeds four rows, and the four
// quarters of a row meet in one warp: the tile's sums are two butterfly
// shuffles, with no barrier across warps.  A warp's 32 rows are 32 R
// consecutive floats of Pl: they go out through the warp's own staging rows
// in shared memory as coalesced stores (scattered 4-byte stores of the rows
// cost about 9 us of the 256^3 pass).  The Khatri-Rao rows of a stage are
// stored with 16 bytes of padding per column quarter, so the four quarters'
// rows read by a warp fall in distinct banks.
// ---------------------------------------------------------------------------
constexpr int TT_ROWS = 256;
constexpr int TT_CONS = 8;  // 32 rows each
constexpr size_t SMEM_LIMIT = 232448;  // 227 KiB of dynamic shared memory per CTA
constexpr int NKR = 3;  // Khatri-Rao warps, stage i handled by warp i mod NKR

template <int RP, typename XT>
struct TrailTma {
  static constexpr int BC = 128 / (int)sizeof(XT);  // columns per stage
  static constexpr int CPC = XChunk<XT>::N;         // columns per 16-byte chunk
  static constexpr int WST = (RP + 3) / 4 * 4;
  static constexpr uint32_t X_BYTES = TT_ROWS * 128;
  static constexpr int QC = BC / 4;                  // columns per quarter
  static constexpr uint32_t W_BYTES = BC * WST * 4 + 4 * 16;  // + 16 bytes of padding per quarter
  // as many stages as fit (at most 6): bytes in flight hide the memory latency
  static constexpr uint32_t OUT_BYTES = TT_CONS * 32 * (RP + 1) * 4;  // output staging, 32 rows per warp
  // at most 5 stages: on the 256^3 workload 4, 5 and 6 stages took 64.9, 62.6
  // and 64.6 us (a deeper ring only adds to the queues in front of DRAM)
  static constexpr int STAGES_FIT = (int)((SMEM_LIMIT - 1024 - 128 - OUT_BYTES) / (X_BYTES + W_BYTES));
  static constexpr int STAGES = STAGES_FIT > 5 ? 5 : STAGES_FIT;
  static constexpr size_t SMEM = 1024 + STAGES * (size_t)(X_BYTES + W_BYTES) + OUT_BYTES + 2 * STAGES * 8;
  // float offset of the Khatri-Rao row of column jj within a stage
  static __device__ __forceinline__ int wrow(int jj) { return jj * WST + (jj / QC) * 4; }
  // A Khatri-Rao warp takes every NKR-th stage; with more warps than stages it
  // could reach a slot two phases ahead of its consumers, which a parity wait
  // cannot tell from the phase it wants.
  static_assert(STAGES >= NKR, "the stage ring must hold at least one stage per Khatri-Rao warp");
};

template <int RP, typename XT>
__global__ void __launch_bounds__((TT_CONS + NKR + 1) * 32, 1) k_trailing_tma(const DevDesc* __restrict__ d) {
  using S = TrailTma<RP, XT>;
  constexpr int TT_BC = S::BC;
  constexpr int TST = S::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* xs = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* ws = reinterpret_cast<float*>(xs + TST * S::X_BYTES);
  float* ostg = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(ws) + TST * S::W_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(ostg) + S::OUT_BYTES);
  uint64_t* empty = full + TST;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* err = &d->sc->timeout;
  const CUtensorMap* maps = d->tmap_trail;
  const uint64_t pol = l2_evict_first_policy();
  if (threadIdx.x == 0) {
    for (int s = 0; s < TST; ++s) {
      mbar_init(smem_u32(&full[s]), 2);  // TMA issuer (with the byte count) + Khatri-Rao warp
      mbar_init(smem_u32(&empty[s]), TT_CONS);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const int K = d->K, N = d->N, h = d->h;
  const Units us(d->lt_sched, d->lt_prefix[K]);

  if (warp == TT_CONS + NKR) {
    // ------------------------------------------- TMA issuer (one thread)
    if (lane != 0) return;
    uint32_t it = 0;
    bool ok = true;
    for (int j = us.first; j < us.end && ok; j += us.step) {
      const TrailUnit tu(d, us.unit(j), TT_ROWS);
      const int k = tu.k;
      const int nch = (tu.je - tu.jb + TT_BC - 1) / TT_BC;
      prefetch_tmap(&maps[k]);
      for (int c = 0; c < nch; ++c, ++it) {
        const int s = it % TST;
        const uint32_t ph = (it / TST) & 1;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, err)) { ok = false; break; }
        mbar_arrive_expect_tx(smem_u32(&full[s]), S::X_BYTES);
        tma_load_2d_hint(smem_u32(xs + s * S::X_BYTES), &maps[k], smem_u32(&full[s]), tu.jb + c * TT_BC, tu.row0,
                         pol);
      }
    }
    // copies still in flight land before the CTA leaves
    for (uint32_t i = it > TST ? it - TST : 0; i < it; ++i)
      mbar_wait_drain(smem_u32(&full[i % TST]), (i / TST) & 1);
    return;
  }

  if (warp >= TT_CONS) {
    // ------------------------------------------------- Khatri-Rao warps
    pdl_wait();  // the factors come from the previous kernel of the sweep
    const int kw = warp - TT_CONS;
    uint32_t it = 0;
    bool ok = true;
    for (int jn = us.first; jn < us.end && ok; jn += us.step) {
      const TrailUnit tu(d, us.unit(jn), TT_ROWS);
      const int k = tu.k;
      const int J = tu.je;  // columns past the split's end (or past J) get zero rows
      const int R = d->R[k];
      const int nch = (tu.je - tu.jb + TT_BC - 1) / TT_BC;
      for (int c = 0; c < nch; ++c, ++it) {
        if ((int)(it % NKR) != kw) continue;
        const int s = it % TST;
        const uint32_t ph = (it / TST) & 1;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, err)) { ok = false; break; }
        // Khatri-Rao rows of the trailing factors for the columns of this stage
#pragma unroll
        for (int jj = lane; jj < TT_BC; jj += 32) {
          const int j = tu.jb + c * TT_BC + jj;
          float w[S::WST];
#pragma unroll
          for (int r = 0; r < S::WST; ++r) w[r] = (j < J && r < R) ? 1.f : 0.f;
          if (j < J) {
            int idx[CNCPD_NMAX];
            decode32_t(d, k, h, N, j, idx);
            for (int m = h; m < N; ++m) {
              const float* U = reinterpret_cast<const float*>(d->U1[k][m]) + (int64_t)idx[m] * R;
#pragma unroll
              for (int r = 0; r < RP; ++r)
                if (r < R) w[r] *= __ldg(U + r);
            }
          }
          float4* wrow = reinterpret_cast<float4*>(ws + s * (S::W_BYTES / 4) + S::wrow(jj));
#pragma unroll
          for (int q = 0; q < S::WST / 4; ++q) wrow[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&full[s]));
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  pdl_wait();
  uint32_t it = 0;
  const int li = lane & 7, cq = lane >> 3;  // row offset, column quarter
  constexpr int RH = RP / 2;
  for (int jn = us.first; jn < us.end; jn += us.step) {
    const TrailUnit tu(d, us.unit(jn), TT_ROWS);
    const int k = tu.k;
    const int row0 = tu.row0;
    const int R = d->R[k];
    const int nch = (tu.je - tu.jb + TT_BC - 1) / TT_BC;
    uint64_t acc[4][RH];  // [row t][pair of ranks]
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int p = 0; p < RH; ++p) acc[t][p] = 0ull;
    for (int c = 0; c < nch; ++c, ++it) {
      const int s = it % TST;
      const uint32_t ph = (it / TST) & 1;
      if (!mbar_wait(smem_u32(&full[s]), ph, err)) continue;  // error recorded; keep the barrier schedule
      const unsigned char* xt = xs + s * S::X_BYTES;
      const float* wt = ws + s * (S::W_BYTES / 4);
#pragma unroll
      for (int q = 2 * cq; q < 2 * cq + 2; ++q) {
        float xv[4][S::CPC];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          // 128-byte swizzle: 16-byte chunk q of row r sits at chunk q ^ (r & 7), and r & 7 = li
          const int r = 32 * warp + li + 8 * t;
          widen(*reinterpret_cast<const uint4*>(xt + r * 128 + ((q ^ li) << 4)), xv[t], XT());
        }
#pragma unroll
        for (int e = 0; e < S::CPC; ++e) {
          const uint64_t* wr = reinterpret_cast<const uint64_t*>(wt + S::wrow(S::CPC * q + e));
          uint64_t x2[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) x2[t] = pack2(xv[t][e], xv[t][e]);
#pragma unroll
          for (int p = 0; p + 2 <= RH; p += 2) {
            const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(wr + p);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              ffma2x(acc[t][p], x2[t], w.x);
              ffma2x(acc[t][p + 1], x2[t], w.y);
            }
          }
          if constexpr (RH % 2 == 1) {
            const uint64_t w = wr[RH - 1];
#pragma unroll
            for (int t = 0; t < 4; ++t) ffma2x(acc[t][RH - 1], x2[t], w);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
    }
    // the four quarters of each row, by butterfly over lanes li, li + 8, li + 16,
    // li + 24 (every lane ends with the same sums); lane (li, cq) stages row
    // li + 8 cq of the warp, then the warp's rows go out as one run of Pl
    float* stg = ostg + warp * 32 * (RP + 1);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
#pragma unroll
      for (int p = 0; p < RH; ++p) {
        float2 v = unpack2(acc[t][p]);
        v.x += __shfl_xor_sync(0xffffffffu, v.x, 8);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, 8);
        v.x += __shfl_xor_sync(0xffffffffu, v.x, 16);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, 16);
        if (t == cq) {
          stg[(li + 8 * t) * (RP + 1) + 2 * p] = v.x;
          stg[(li + 8 * t) * (RP + 1) + 2 * p + 1] = v.y;
        }
      }
    }
    __syncwarp();
    const int64_t wrow0 = (int64_t)row0 + 32 * warp;
    const int64_t rows = d->lead_rows[k];
    const int nrow = rows - wrow0 < 32 ? (int)(rows - wrow0) : 32;
    const int ne = nrow > 0 ? nrow * R : 0;
    // a split block's unit leaves its partial rows for k_reduce_trail_splits
    float* dst = (d->lt_js[k] > 1 ? reinterpret_cast<float*>(d->Pl_part) + d->plp_off[k] + (int64_t)tu.split * rows * R
                                  : reinterpret_cast<float*>(d->Pl[k])) +
                 wrow0 * R;
    if (R == RP) {
      for (int e = lane; e < ne; e += 32) dst[e] = stg[(e / RP) * (RP + 1) + e % RP];
    } else {
      for (int e = lane; e < ne; e += 32) dst[e] = stg[(e / R) * (RP + 1) + e % R];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Lead contraction (split over rows) Pt[col, r] = sum_row X[row, col] W_l[row, r].
// Unit = 256 columns x one row split; stage = 32 KiB = 32 FP32 or 64 BF16
// rows x 256 columns.  Consumer warp w owns columns 128 (w % 2) + 4 lane .. + 3
// and the (w / 2)-th quarter of the stage's rows, so each Khatri-Rao value
// read from shared memory feeds four columns; the four row quarters are added
// at the end of the unit.
// ---------------------------------------------------------------------------
constexpr int LT_COLS = 256;
constexpr int LT_CONS = 8;

template <int RP, typename XT>
struct LeadTma {
  static constexpr int ROWS = 128 / (int)sizeof(XT);  // rows per stage (32 KiB)
  static constexpr int WST = (RP + 3) / 4 * 4;
  static constexpr uint32_t X_BYTES = ROWS * LT_COLS * (int)sizeof(XT);
  static constexpr uint32_t W_BYTES = ROWS * WST * 4;
  static constexpr uint32_t RED_BYTES = 3 * LT_COLS * RP * 4;  // partial sums of row quarters 1..3, [quarter][rank][slot]
  static constexpr int STAGES_FIT = (int)((SMEM_LIMIT - 1024 - 128 - RED_BYTES) / (X_BYTES + W_BYTES));
  static constexpr int STAGES = STAGES_FIT > 6 ? 6 : STAGES_FIT;
  static constexpr size_t SMEM = 1024 + STAGES * (size_t)(X_BYTES + W_BYTES) + RED_BYTES + 2 * STAGES * 8;
  static_assert(STAGES >= NKR, "the stage ring must hold at least one stage per Khatri-Rao warp");
};

template <int RP, typename XT>
__global__ void __launch_bounds__((LT_CONS + NKR + 1) * 32, 1) k_lead_tma(const DevDesc* __restrict__ d) {
  using S = LeadTma<RP, XT>;
  constexpr int LT_ROWS = S::ROWS;
  constexpr int ST = S::STAGES;
  constexpr int RH = RP / 2;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* xs = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* ws = reinterpret_cast<float*>(xs + ST * S::X_BYTES);
  float* red = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(ws) + ST * S::W_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(red) + S::RED_BYTES);
  uint64_t* empty = full + ST;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* err = &d->sc->timeout;
  const CUtensorMap* maps = d->tmap_lead;
  const uint64_t pol = l2_evict_first_policy();
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 2);  // TMA issuer (with the byte count) + Khatri-Rao warp
      mbar_init(smem_u32(&empty[s]), LT_CONS);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const int K = d->K, h = d->h;
  const Units us(d->tt_sched, d->tt_prefix[K]);

  if (warp == LT_CONS + NKR) {
    // ------------------------------------------- TMA issuer (one thread)
    if (lane != 0) return;
    uint32_t it = 0;
    bool ok = true;
    for (int j = us.first; j < us.end && ok; j += us.step) {
      const int u = us.unit(j);
      int k = 0;
      while (d->tt_prefix[k + 1] <= u) ++k;
      const int local = u - d->tt_prefix[k];
      const int ctile = local % d->tt_ctiles[k];
      const int split = local / d->tt_ctiles[k];
      const int rows = (int)d->lead_rows[k];
      const int rb = split * (int)d->split_rows[k];
      const int re = min(rows, rb + (int)d->split_rows[k]);
      prefetch_tmap(&maps[k]);
      for (int r0 = rb; r0 < re; r0 += LT_ROWS, ++it) {
        const int s = it % ST;
        const uint32_t ph = (it / ST) & 1;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, err)) { ok = false; break; }
        mbar_arrive_expect_tx(smem_u32(&full[s]), S::X_BYTES);
        tma_load_2d_hint(smem_u32(xs + s * S::X_BYTES), &maps[k], smem_u32(&full[s]), ctile * LT_COLS, r0, pol);
      }
    }
    for (uint32_t i = it > (uint32_t)ST ? it - ST : 0; i < it; ++i)
      mbar_wait_drain(smem_u32(&full[i % ST]), (i / ST) & 1);
    return;
  }

  if (warp >= LT_CONS) {
    // ------------------------------------------------- Khatri-Rao warps
    pdl_wait();  // the factors come from the previous kernel of the sweep
    const int kw = warp - LT_CONS;
    uint32_t it = 0;
    bool ok = true;
    for (int j = us.first; j < us.end && ok; j += us.step) {
      const int u = us.unit(j);
      int k = 0;
      while (d->tt_prefix[k + 1] <= u) ++k;
      const int local = u - d->tt_prefix[k];
      const int split = local / d->tt_ctiles[k];
      const int rows = (int)d->lead_rows[k];
      const int R = d->R[k];
      const int rb = split * (int)d->split_rows[k];
      const int re = min(rows, rb + (int)d->split_rows[k]);
      for (int r0 = rb; r0 < re; r0 += LT_ROWS, ++it) {
        if ((int)(it % NKR) != kw) continue;
        const int s = it % ST;
        const uint32_t ph = (it / ST) & 1;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, err)) { ok = false; break; }
        // Khatri-Rao rows of the lead factors for the rows of this stage
#pragma unroll
        for (int ii = lane; ii < LT_ROWS; ii += 32) {
          const int row = r0 + ii;
          float w[S::WST];
#pragma unroll
          for (int r = 0; r < S::WST; ++r) w[r] = (row < re && r < R) ? 1.f : 0.f;
          if (row < re) {
            int idx[CNCPD_NMAX];
            decode32_t(d, k, 0, h, row, idx);
            for (int m = 0; m < h; ++m) {
              const float* U = reinterpret_cast<const float*>(d->U1[k][m]) + (int64_t)idx[m] * R;
#pragma unroll
              for (int r = 0; r < RP; ++r)
                if (r < R) w[r] *= __ldg(U + r);
            }
          }
          float4* dst = reinterpret_cast<float4*>(ws + s * (S::W_BYTES / 4) + ii * S::WST);
#pragma unroll
          for (int q = 0; q < S::WST / 4; ++q) dst[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&full[s]));
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  pdl_wait();
  const int ch = warp & 1, rq = warp >> 1;  // column half (128 columns, 4 per lane), row quarter (8 rows)
  const int colw = ch * 128 + 4 * lane;    // first of this lane's four columns within the tile
  uint32_t it = 0;
  for (int j = us.first; j < us.end; j += us.step) {
    const int u = us.unit(j);
    int k = 0;
    while (d->tt_prefix[k + 1] <= u) ++k;
    const int local = u - d->tt_prefix[k];
    const int ctile = local % d->tt_ctiles[k];
    const int split = local / d->tt_ctiles[k];
    const int rows = (int)d->lead_rows[k];
    const int J = (int)d->trail_cols[k];
    const int R = d->R[k];
    const int rb = split * (int)d->split_rows[k];
    const int re = min(rows, rb + (int)d->split_rows[k]);
    uint64_t acc[4][RH];  // [column][pair of ranks]
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int p = 0; p < RH; ++p) acc[c][p] = 0ull;
    for (int r0 = rb; r0 < re; r0 += LT_ROWS, ++it) {
      const int s = it % ST;
      const uint32_t ph = (it / ST) & 1;
      if (!mbar_wait(smem_u32(&full[s]), ph, err)) continue;  // error recorded; keep the barrier schedule
      const unsigned char* xt = xs + s * S::X_BYTES;
      const float* wt = ws + s * (S::W_BYTES / 4);
      constexpr int RQ = LT_ROWS / 4;  // rows per quarter
#pragma unroll 4
      for (int i = rq * RQ; i < rq * RQ + RQ; ++i) {
        const float4 x = load4(xt + (i * LT_COLS + colw) * (int)sizeof(XT), XT());
        const uint64_t x0 = pack2(x.x, x.x), x1 = pack2(x.y, x.y), x2 = pack2(x.z, x.z), x3 = pack2(x.w, x.w);
        const uint64_t* wr = reinterpret_cast<const uint64_t*>(wt + i * S::WST);
#pragma unroll
        for (int p = 0; p + 2 <= RH; p += 2) {
          const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(wr + p);
          ffma2x(acc[0][p], x0, w.x);
          ffma2x(acc[0][p + 1], x0, w.y);
          ffma2x(acc[1][p], x1, w.x);
          ffma2x(acc[1][p + 1], x1, w.y);
          ffma2x(acc[2][p], x2, w.x);
          ffma2x(acc[2][p + 1], x2, w.y);
          ffma2x(acc[3][p], x3, w.x);
          ffma2x(acc[3][p + 1], x3, w.y);
        }
        if constexpr (RH % 2 == 1) {
          const uint64_t w = wr[RH - 1];
          ffma2x(acc[0][RH - 1], x0, w);
          ffma2x(acc[1][RH - 1], x1, w);
          ffma2x(acc[2][RH - 1], x2, w);
          ffma2x(acc[3][RH - 1], x3, w);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
    }
    // row quarters 1..3 park their sums; quarter 0 adds them in order
    named_bar(1, LT_CONS * 32);
    // slot c * 64 + ch * 32 + lane holds column colw + c: consecutive lanes,
    // consecutive words
    if (rq > 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int p = 0; p < RH; ++p) {
          const float2 v = unpack2(acc[c][p]);
          const int slot = c * 64 + ch * 32 + lane;
          red[((rq - 1) * RP + 2 * p) * LT_COLS + slot] = v.x;
          red[((rq - 1) * RP + 2 * p + 1) * LT_COLS + slot] = v.y;
        }
    }
    named_bar(1, LT_CONS * 32);
    if (rq == 0) {
      float* part = reinterpret_cast<float*>(d->partial) + d->partial_off[k] + (int64_t)split * J * R;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = ctile * LT_COLS + colw + c;
        if (col < J) {
#pragma unroll
          for (int p = 0; p < RH; ++p) {
            const float2 v = unpack2(acc[c][p]);
            float o0 = v.x, o1 = v.y;
#pragma unroll
            const int slot = c * 64 + ch * 32 + lane;
#pragma unroll
            for (int q4 = 0; q4 < 3; ++q4) {
              o0 += red[(q4 * RP + 2 * p) * LT_COLS + slot];
              o1 += red[(q4 * RP + 2 * p + 1) * LT_COLS + slot];
            }
            if (2 * p < R) part[(int64_t)col * R + 2 * p] = o0;
            if (2 * p + 1 < R) part[(int64_t)col * R + 2 * p + 1] = o1;
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------- launchers ----

template <int RP, typename XT>
static cudaError_t trailing_tma_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  const int total = hd.lt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  const size_t smem = TrailTma<RP, XT>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_trailing_tma<RP, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = hd.lt_sched ? hd.lt_grid : (total < c.num_sms ? total : c.num_sms);
  // the issuer streams X (constant) from the start; the other warps wait for
  // the previous kernel of the sweep (programmatic dependent launch)
  e = launch_pdl(k_trailing_tma<RP, XT>, dim3(grid), dim3((TT_CONS + NKR + 1) * 32), smem, c.stream, dd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int RP, typename XT>
static cudaError_t lead_tma_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  const int total = hd.tt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  const size_t smem = LeadTma<RP, XT>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_lead_tma<RP, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = hd.tt_sched ? hd.tt_grid : (total < c.num_sms ? total : c.num_sms);
  e = launch_pdl(k_lead_tma<RP, XT>, dim3(grid), dim3((LT_CONS + NKR + 1) * 32), smem, c.stream, dd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

#define CNCPD_TMA_RP(X) X(4) X(8) X(10) X(12) X(16) X(20) X(24) X(32)

bool tma_rank_supported(int RP) {
#define TCASE(V) if (RP == V) return true;
  CNCPD_TMA_RP(TCASE)
#undef TCASE
  return false;
}

// Rows of the lead contraction per TMA stage (the split-K plan keeps every
// split a multiple of this).
int lead_tma_rows(int st) { return st == ST_BF16 ? LeadTma<4, __nv_bfloat16>::ROWS : LeadTma<4, float>::ROWS; }

cudaError_t launch_trailing_tma(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int RP, int st) {
#define TCASE(V)                                                                             \
  case V:                                                                                    \
    return st == ST_BF16 ? trailing_tma_impl<V, __nv_bfloat16>(c, dd, hd) : trailing_tma_impl<V, float>(c, dd, hd);
  switch (RP) { CNCPD_TMA_RP(TCASE) }
#undef TCASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_lead_tma(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int RP, int st) {
#define TCASE(V)                                                                             \
  case V:                                                                                    \
    return st == ST_BF16 ? lead_tma_impl<V, __nv_bfloat16>(c, dd, hd) : lead_tma_impl<V, float>(c, dd, hd);
  switch (RP) { CNCPD_TMA_RP(TCASE) }
#undef TCASE
  return cudaErrorInvalidValue;
}

// Pl^(k) = sum over the column splits of block k's partial rows, added in
// split order (blocks without splits are skipped).  One thread per element.
__global__ void __launch_bounds__(256) k_reduce_trail_splits(const DevDesc* __restrict__ d) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.y;
  const int js = d->lt_js[k];
  if (js <= 1) return;
  const int64_t n = d->lead_rows[k] * d->R[k];
  const float* __restrict__ part = reinterpret_cast<const float*>(d->Pl_part) + d->plp_off[k];
  float* Pl = reinterpret_cast<float*>(d->Pl[k]);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = part[(int64_t)min(q, js - 1) * n + e];  // clamped: every load issues at once
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < js) sum += v[q];
    for (int q = 8; q < js; ++q) sum += part[(int64_t)q * n + e];
    Pl[e] = sum;
  }
}

cudaError_t launch_reduce_trail_splits(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  if (!hd.trail_split) return cudaSuccess;
  int64_t nmax = 0;
  for (int k = 0; k < hd.K; ++k)
    if (hd.lt_js[k] > 1) nmax = std::max<int64_t>(nmax, hd.lead_rows[k] * hd.R[k]);
  const unsigned gx = (unsigned)std::min<int64_t>(256, (nmax + 255) / 256);
  return launch_pdl(k_reduce_trail_splits, dim3(gx, hd.K), dim3(256), 0, c.stream, dd);
}

// Self-test of the bounded-wait path: one thread waits on the phase-0
// completion of an mbarrier that expects one arrival and never gets it, with
// no copy or MMA in flight, so the wait runs out after `limit_ns` and sets
// the error word exactly as a stalled pipeline would.
__global__ void k_wait_selftest(int* err, uint64_t limit_ns) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, err, limit_ns);
  __syncthreads();
}

cudaError_t launch_wait_selftest(cudaStream_t s, int* err, uint64_t limit_ns) {
  k_wait_selftest<<<1, 32, 0, s>>>(err, limit_ns);
  return cudaGetLastError();
}

}  // namespace cncpd
