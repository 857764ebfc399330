// Trailing-mode contraction of FP32-stored third-order tensors on the TF32
// tensor cores (tcgen05.mma .kind::tf32, A from tensor memory), opt-in via
// cncpd_opts.tf32.  See the comment above k_trailing_tf32 for the split of
// the operands, the roles and the barriers.
#include "cncpd_internal.cuh"
#include "tma.cuh"
#include "umma.cuh"

namespace cncpd {

namespace {

constexpr size_t T_SMEM_LIMIT = 232448;  // 227 KiB of dynamic shared memory per CTA

// The units of this CTA (the host's balanced list, else every gridDim.x-th
// unit).
struct TUnits {
  const int* ids;
  int first, end, step;
  __device__ __forceinline__ TUnits(const int* sched, int total) {
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

}  // namespace

// ---------------------------------------------------------------------------
// Trailing contraction of FP32-stored third-order tensors on the TF32 tensor
// cores, FP32-accurate by splitting both operands into two TF32 parts:
//   x = xb + xs (+ a rounding error below 2^-23 |x|),  u = ub + us (likewise),
// (X by Veltkamp splitting on the FP32 pipe, so |x| < 2^114 is required: the
// host enables the pass only when ||X^(k)|| is below that),
//   x u = xb ub + xb us + xs ub + xs us,
// every product exact in the FP32 accumulator.  The factor's parts are the
// B operand [ub; us] (2 NP rows, k_split_factor_tf32, staged by TMA with each
// X tile); the X tile (256 rows x 32 FP32 columns, 128-byte swizzle, the
// same box as the CUDA-core pass) is split by eight CUDA-core warps into xb
// and xs, which they store straight into tensor memory as the MMA's A
// operand (tcgen05.st), so shared memory sees only the TMA write and one
// read of X.  Two MMAs (A = xb, A = xs) per K step and half tile add into
// one accumulator whose two NP-column halves hold the ub- and us-products.
//
// The tensor cores round each MMA's addition into the accumulator toward
// zero (measured on GB300: a chain of MMAs over J = 256 columns left the
// MTTKRP 2e-6 low, over J = 1024 8.5e-6 low, growing with the chain).  So
// every stage (32 columns: 8 MMAs) starts a fresh accumulator, and the
// warps add the stages' sums in FP32 with round-to-nearest; the bias left
// is that of an 8-MMA chain on one stage's share (2.5e-7 measured).
//
// Warp roles (320 threads): 0 TMA producer, 1 MMA issuer and TMEM owner,
// 2-9 workers.  Worker w takes half tile (w - 2) / 4 and TMEM lanes
// 32 (w mod 4) .. + 31, i.e. rows 32 (w mod 4) + lane of that half: it
// splits its rows of each stage into the A slot, then drains the
// accumulator rows of the stage NB - 1 back into its running sums, and
// writes its rows of Pl when a unit's last stage is drained.  TMEM: NB
// accumulator buffers (4 for R <= 16, else 2) x two half tiles (2 NP columns
// each), then two A slots of 128 columns (per half tile 32 columns of xb and
// 32 of xs); stage `it` uses A slot it mod 2 and buffer it mod NB.  Barriers: full[s] (TMA bytes), empty[s] (the
// eight workers have read the tile and the MMAs have read its B part),
// afull / aempty per A slot, tfull / tempty per accumulator buffer.  Every
// wait is bounded in time, as in the other passes.
// ---------------------------------------------------------------------------
namespace {

constexpr int T_THREADS = 320;
constexpr int T_WORKERS = 8;

template <int NP>
struct Tf32Cfg {
  static constexpr uint32_t X_BYTES = 32768;         // 256 rows x 32 FP32 columns
  static constexpr uint32_t B_BYTES = 2 * NP * 128;  // [ub; us]: 2 NP rows x 32 K values
  static constexpr uint32_t STAGE = X_BYTES + B_BYTES;
  static constexpr uint32_t OUT_BYTES = T_WORKERS * 32 * (NP + 1) * 4;  // a staging block per worker
  static constexpr int STAGES_FIT = (int)((T_SMEM_LIMIT - 1024 - 256 - OUT_BYTES) / STAGE);
  static constexpr int STAGES = STAGES_FIT > 6 ? 6 : STAGES_FIT;
  static constexpr uint32_t ACC = 2 * NP;            // TMEM columns of one M = 128 accumulator
  static constexpr int NB = NP <= 16 ? 4 : 2;        // accumulator buffers (stage it uses it mod NB)
  static constexpr int LAG = NB - 1;                 // a worker drains stage it - LAG after splitting it
  static constexpr uint32_t ABASE = NB * 2 * ACC;    // A slots after NB buffers x 2 halves
  static constexpr uint32_t ASLOT = 128;             // 2 halves x (32 xb + 32 xs) columns
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256 + OUT_BYTES;
  static_assert(STAGE % 1024 == 0, "stages must keep 1 KiB alignment");
  static_assert(STAGES >= 3, "stage ring too small");
  static_assert(ABASE + 2 * ASLOT <= TMEM_COLS, "TMEM plan exceeds the allocation");
  static_assert((2 * STAGES + 4 + 2 * NB + 1) * 8 + 4 <= 256, "barrier area too small");
};

}  // namespace

// B operand of the TF32 trailing pass: U = U^(k)_(N-1) as 2 NP rows of
// length I (row pitch bt_pitch) in FP32 with TF32 values: row r holds
// ub = tf32(u) of U[:, r], row NP + r holds us = tf32(u - ub); rows r >= R
// are zero.
__global__ void __launch_bounds__(256) k_split_factor_tf32(const DevDesc* __restrict__ d) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.y;
  const int m = d->N - 1;
  const int NP = d->umma_np;
  const int R = d->R[k];
  const int64_t I = d->dims[k][m];
  const int64_t ld = d->bt_pitch[k];
  const float* __restrict__ U = reinterpret_cast<const float*>(d->U1[k][m]);
  uint32_t* dst = reinterpret_cast<uint32_t*>(d->Bt[k]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += (int64_t)gridDim.x * blockDim.x) {
    for (int r = 0; r < NP; ++r) {
      const float w = r < R ? U[i * R + r] : 0.f;
      const uint32_t ub = tf32_round_bits(__float_as_uint(w));
      const uint32_t us = tf32_round_bits(__float_as_uint(w - __uint_as_float(ub)));
      dst[(int64_t)r * ld + i] = ub;
      dst[(int64_t)(NP + r) * ld + i] = us;
    }
  }
}

// x rounded to 11 significant bits (a TF32 value) by Veltkamp's splitting
// with the constant 2^13 + 1, on the FP32 pipe: three rounded operations, no
// contraction.  Exact for |x| below 2^114 (the caller's data bound).
__device__ __forceinline__ float tf32_split_hi(float x) {
  const float t = __fmul_rn(x, 8193.0f);
  return __fsub_rn(t, __fsub_rn(t, x));
}

template <int NP>
__global__ void __launch_bounds__(T_THREADS, 1) k_trailing_tf32(const DevDesc* __restrict__ d) {
  using S = Tf32Cfg<NP>;
  constexpr int ST = S::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + ST * S::STAGE);
  uint64_t* empty = full + ST;
  constexpr int NB = S::NB;
  uint64_t* afull = empty + ST;   // [2]
  uint64_t* aempty = afull + 2;   // [2]
  uint64_t* tfull = aempty + 2;   // [NB]
  uint64_t* tempty = tfull + NB;  // [NB]
  uint64_t* drain = tempty + NB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);                // producer (arrive + byte count)
      mbar_init(smem_u32(&empty[s]), T_WORKERS + 1);   // the workers + the MMA commit
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&afull[q]), T_WORKERS);   // the workers' splits
      mbar_init(smem_u32(&aempty[q]), 1);          // MMA commit
    }
    for (int q = 0; q < NB; ++q) {
      mbar_init(smem_u32(&tfull[q]), 1);           // MMA commit
      mbar_init(smem_u32(&tempty[q]), T_WORKERS);  // the workers' drains
    }
    mbar_init(smem_u32(drain), 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), S::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // the split factor and the factors come from earlier kernels of the sweep
  const uint32_t tmem = *tmem_slot;
  int* err = &d->sc->timeout;
  const int K = d->K;
  const TUnits us(d->lt_sched, d->lt_prefix[K]);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      const uint64_t pol = l2_evict_first_policy();
      uint32_t it = 0;
      bool ok = true;
      for (int jn = us.first; jn < us.end && ok; jn += us.step) {
        const int g = us.unit(jn);
        int k = 0;
        while (d->lt_prefix[k + 1] <= g) ++k;
        const int row0 = (g - d->lt_prefix[k]) * 256;
        const int nch = (int)((d->trail_cols[k] + 31) / 32);
        prefetch_tmap(&d->tmap_trail[k]);
        prefetch_tmap(&d->tmap_bt[k]);
        for (int c = 0; c < nch; ++c, ++it) {
          const int s = it % ST;
          if (!mbar_wait(smem_u32(&empty[s]), ((it / ST) & 1) ^ 1, err)) { ok = false; break; }
          const uint32_t sa = smem_u32(base + s * S::STAGE);
          const uint32_t fb = smem_u32(&full[s]);
          mbar_arrive_expect_tx(fb, S::STAGE);
          tma_load_2d_hint(sa, &d->tmap_trail[k], fb, c * 32, row0, pol);
          tma_load_2d(sa + S::X_BYTES, &d->tmap_bt[k], fb, c * 32, 0);
        }
      }
      for (uint32_t i = it > (uint32_t)ST ? it - ST : 0; i < it; ++i)
        mbar_wait_drain(smem_u32(&full[i % ST]), (i / ST) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------ MMA issuer
      constexpr uint32_t IDESC = umma_idesc_tf32(128, 2 * NP);
      uint32_t it = 0;
      bool ok = true;
      for (int jn = us.first; jn < us.end && ok; jn += us.step) {
        const int g = us.unit(jn);
        int k = 0;
        while (d->lt_prefix[k + 1] <= g) ++k;
        const int nch = (int)((d->trail_cols[k] + 31) / 32);
        for (int c = 0; c < nch; ++c, ++it) {
          const int s = it % ST;
          const int a = it & 1;        // A slot of this stage
          const int b = it % NB;       // accumulator buffer of this stage
          if (!mbar_wait(smem_u32(&tempty[b]), ((it / NB) & 1) ^ 1, err) ||
              !mbar_wait(smem_u32(&full[s]), (it / ST) & 1, err) ||
              !mbar_wait(smem_u32(&afull[a]), (it >> 1) & 1, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ba = smem_u32(base + s * S::STAGE) + S::X_BYTES;
#pragma unroll
          for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                umma_tf32_ta(tmem + (uint32_t)((b * 2 + half) * S::ACC),
                             tmem + S::ABASE + (uint32_t)(a * S::ASLOT + half * 64 + p * 32 + ks * 8),
                             umma_desc_sw128(ba + ks * 32, 16, 1024), IDESC, (p > 0 || ks > 0) ? 1u : 0u);
          umma_commit(smem_u32(&empty[s]));
          umma_commit(smem_u32(&aempty[a]));
          umma_commit(smem_u32(&tfull[b]));
        }
      }
      // every MMA issued by this thread completes before TMEM is freed
      umma_commit(smem_u32(drain));
      mbar_wait_drain(smem_u32(drain), 0);
    }
  } else {
    // ------------------------------------------------------------ workers
    const int half = (warp - 2) >> 2;
    const int q = warp & 3;                     // TMEM lanes 32 q .. 32 q + 31
    const int r = half * 128 + 32 * q + lane;   // this lane's row of each tile
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    float* stg = reinterpret_cast<float*>(base + ST * S::STAGE + 256) + (warp - 2) * 32 * (NP + 1);
    float sum[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) sum[j] = 0.f;
    // Drain of stage pit (its accumulator rows added to sum); when it ends
    // its unit, the warp's 32 rows of Pl go out as one coalesced run.
    auto drain_stage = [&](uint32_t pit, bool last, int pk, int64_t prow0) -> bool {
      const int b = pit % NB;
      if (!mbar_wait(smem_u32(&tfull[b]), (pit / NB) & 1, err)) return false;
      tc_fence_after();
      uint32_t v[2 * NP];
      const uint32_t t = lane_base + (uint32_t)((b * 2 + half) * S::ACC);
#pragma unroll
      for (int c0 = 0; c0 < 2 * NP; c0 += 16) tmem_ld16(t + c0, *reinterpret_cast<uint32_t(*)[16]>(&v[c0]));
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
#pragma unroll
      for (int j = 0; j < NP; ++j) sum[j] += __uint_as_float(v[j]) + __uint_as_float(v[NP + j]);
      if (last) {
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          stg[lane * (NP + 1) + j] = sum[j];
          sum[j] = 0.f;
        }
        __syncwarp();
        const int64_t rows = d->lead_rows[pk];
        const int R = d->R[pk];
        const int64_t wrow0 = prow0 + half * 128 + 32 * q;  // first row of this warp
        const int64_t nrow = rows - wrow0 < 32 ? rows - wrow0 : 32;
        const int ne = nrow > 0 ? (int)nrow * R : 0;
        float* dst = reinterpret_cast<float*>(d->Pl[pk]) + wrow0 * R;
        for (int e = lane; e < ne; e += 32) dst[e] = stg[(e / R) * (NP + 1) + e % R];
        __syncwarp();
      }
      return true;
    };
    // The drains follow the splits S::LAG stages behind, walking the same
    // unit list with their own cursor, so an accumulator is read only after
    // the MMAs have had LAG splits' time to finish it.
    int djn = us.first, dc = 0, dk = 0, dnch = 0;
    int64_t drow0 = 0;
    uint32_t dit = 0;
    auto dload = [&]() {
      if (djn < us.end) {
        const int g = us.unit(djn);
        dk = 0;
        while (d->lt_prefix[dk + 1] <= g) ++dk;
        drow0 = (int64_t)(g - d->lt_prefix[dk]) * 256;
        dnch = (int)((d->trail_cols[dk] + 31) / 32);
      }
    };
    auto drain_next = [&]() -> bool {
      if (!drain_stage(dit, dc == dnch - 1, dk, drow0)) return false;
      ++dit;
      if (++dc == dnch) {
        dc = 0;
        djn += us.step;
        dload();
      }
      return true;
    };
    dload();
    uint32_t it = 0;
    bool ok = true;
    for (int jn = us.first; jn < us.end && ok; jn += us.step) {
      const int g = us.unit(jn);
      int k = 0;
      while (d->lt_prefix[k + 1] <= g) ++k;
      const int nch = (int)((d->trail_cols[k] + 31) / 32);
      for (int c = 0; c < nch; ++c, ++it) {
        // split this lane's row of stage it: eight 16-byte chunks (chunk c
        // of row r sits at c ^ (r mod 8) under the 128-byte swizzle, and
        // r mod 8 = lane mod 8); xb = x to 11 bits, xs = (x - xb) to 11 bits
        const int s = it % ST;
        const int a = it & 1;
        if (!mbar_wait(smem_u32(&full[s]), (it / ST) & 1, err) ||
            !mbar_wait(smem_u32(&aempty[a]), ((it >> 1) & 1) ^ 1, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const unsigned char* xrow = base + s * S::STAGE + r * 128;
        uint32_t xb[32], xs[32];
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const uint4 v = *reinterpret_cast<const uint4*>(xrow + ((ch ^ (lane & 7)) << 4));
          const uint32_t e4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float x = __uint_as_float(e4[e]);
            const float hb = tf32_split_hi(x);
            const float rs = __fsub_rn(x, hb);  // exact
            xb[4 * ch + e] = __float_as_uint(hb);
            xs[4 * ch + e] = __float_as_uint(tf32_split_hi(rs));
          }
        }
        const uint32_t ta = lane_base + S::ABASE + (uint32_t)(a * S::ASLOT + half * 64);
        tmem_st32(ta, xb);
        tmem_st32(ta + 32, xs);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_u32(&empty[s]));
          mbar_arrive(smem_u32(&afull[a]));
        }
        if (it >= (uint32_t)S::LAG && !drain_next()) {
          ok = false;
          break;
        }
      }
    }
    while (ok && dit < it)
      if (!drain_next()) break;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, S::TMEM_COLS);
}

// ------------------------------------------------------------- launchers ----

template <int NP>
static cudaError_t trailing_tf32_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  const int total = hd.lt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  const size_t smem = Tf32Cfg<NP>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_trailing_tf32<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = hd.lt_sched ? hd.lt_grid : (total < c.num_sms ? total : c.num_sms);
  e = launch_pdl(k_trailing_tf32<NP>, dim3(grid), dim3(T_THREADS), smem, c.stream, dd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_split_factor_tf32(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  int64_t imax = 1;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][hd.N - 1] > imax ? hd.dims[k][hd.N - 1] : imax;
  const unsigned gx = (unsigned)((imax + 255) / 256);
  cudaError_t e = launch_pdl(k_split_factor_tf32, dim3(gx, hd.K), dim3(256), 0, c.stream, dd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_trailing_tf32(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  if (hd.umma_np == 16) return trailing_tf32_impl<16>(c, dd, hd);
  if (hd.umma_np == 32) return trailing_tf32_impl<32>(c, dd, hd);
  return cudaErrorInvalidValue;
}

}  // namespace cncpd
