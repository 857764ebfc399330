// Level-1 contractions of the dimension tree for BF16-stored third-order
// tensors on the fifth-generation tensor cores (tcgen05.mma .kind::f16,
// BF16 x BF16 -> FP32 accumulators in TMEM).
//
// Each pass multiplies X by one factor; the other contracted factor, if any,
// enters as a scale per slab of X:
//   trailing pass  Pl[a, r] = sum_j X[a, j] U2[j, r]                     (a = (i0, i1))
//   lead pass      Pt[j, r] = sum_i0 U0[i0, r] sum_i1 X[i0, i1, j] U1[i1, r]
// so the MMA's B operand is a factor, the same for every tile of the pass.
// k_split_factor writes it once per pass as three BF16 parts hi + mid + lo
// (hi = bf16(u), mid = bf16(u - hi), lo = bf16(u - hi - mid): 24 significant
// bits, the FP32 value up to the last bit) stacked as the 3 NP rows of a
// K-major operand in global memory, and TMA stages it next to each X tile.
// One MMA per K step forms the three partial products side by side in TMEM;
// the epilogue adds them (lo + mid, then hi).  The lead pass keeps one
// accumulator per i0 slab (double-buffered in TMEM); the epilogue warps scale
// each slab by U0[i0, :] and add the slabs of a unit in registers, in slab
// order, and write the unit's split-K partial.
//
// BF16 hi + lo storage (two planes, x = hi + lo) runs the same MMAs over
// twice the K chunks: the lo plane's chunks follow the hi plane's with the
// same B operand, into the same accumulator.
//
// Warp roles (192 threads): 0 TMA producer, 1 MMA issuer and TMEM owner,
// 2-5 epilogue (warp w reads TMEM lanes 32 (w mod 4) .. + 31).  Each mbarrier
// is waited on by one role that sees every phase in order, so a parity wait
// always names the phase it wants.  Every wait is bounded in time; on expiry
// the kernel records the error, lets its copies and MMAs finish (bounded) and
// frees its TMEM before returning.
#include <cuda_bf16.h>

#include "cncpd_internal.cuh"
#include "tma.cuh"
#include "umma.cuh"

namespace cncpd {

namespace {

constexpr int U_THREADS = 192;
constexpr size_t U_SMEM_LIMIT = 232448;  // 227 KiB of dynamic shared memory per CTA

// OUT: the kernel stages its output rows in shared memory (trailing pass).
template <int NP, bool OUT>
struct UmmaCfg {
  static constexpr uint32_t A_BYTES = 32768;         // X: 256 x 64 (trailing) or 64 x 256 (lead) BF16
  static constexpr uint32_t B_BYTES = 3 * NP * 128;  // 3 NP rows x 64 K values
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;  // a multiple of 1 KiB (swizzle atoms stay aligned)
  // output staging of the trailing epilogue: 32 rows x (NP + 1) floats per epilogue warp
  static constexpr uint32_t OUT_BYTES = OUT ? 4 * 32 * (NP + 1) * 4 : 0;
  static constexpr int STAGES_FIT = (int)((U_SMEM_LIMIT - 1024 - 256 - OUT_BYTES) / STAGE);
  static constexpr int STAGES = STAGES_FIT > 6 ? 6 : STAGES_FIT;
  static constexpr uint32_t ACC = 3 * NP;  // TMEM columns of one M = 128 accumulator
  static constexpr uint32_t TMEM_COLS = 4 * ACC <= 256 ? 256 : 512;  // 2 buffers x 2 halves
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256 + OUT_BYTES;
  static_assert(STAGE % 1024 == 0, "stages must keep 1 KiB alignment");
  static_assert(STAGES >= 2, "stage ring too small");
};

// Barriers and the TMEM base address after the stage ring.
struct UmmaBars {
  uint64_t *full, *empty, *tfull, *tempty, *drain;
  uint32_t* tmem_slot;
};

template <class S>
__device__ __forceinline__ UmmaBars umma_setup(unsigned char* base) {
  UmmaBars b;
  b.full = reinterpret_cast<uint64_t*>(base + S::STAGES * S::STAGE);
  b.empty = b.full + S::STAGES;
  b.tfull = b.empty + S::STAGES;  // [2]
  b.tempty = b.tfull + 2;         // [2]
  b.drain = b.tempty + 2;
  b.tmem_slot = reinterpret_cast<uint32_t*>(b.drain + 1);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S::STAGES; ++s) {
      mbar_init(smem_u32(&b.full[s]), 1);   // producer (arrive + byte count)
      mbar_init(smem_u32(&b.empty[s]), 1);  // MMA completion
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&b.tfull[q]), 1);   // MMA completion of an accumulator
      mbar_init(smem_u32(&b.tempty[q]), 4);  // the four epilogue warps
    }
    mbar_init(smem_u32(b.drain), 1);
    fence_mbar_init();
  }
  if ((threadIdx.x >> 5) == 1) tmem_alloc(smem_u32(b.tmem_slot), S::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return b;
}

// The work units of this CTA (the host's balanced list, else every
// gridDim.x-th unit).
struct UUnits {
  const int* ids;
  int first, end, step;
  __device__ __forceinline__ UUnits(const int* sched, int total) {
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

// Three 16-column groups (hi, mid, lo parts) of the warp's 32 TMEM lanes at
// column c0 of the accumulator at t, added as hi + (mid + lo).
template <int NP>
__device__ __forceinline__ void tmem_parts16(uint32_t t, int c0, float (&v)[16]) {
  uint32_t vh[16], vm[16], vl[16];
  tmem_ld16(t + c0, vh);
  tmem_ld16(t + NP + c0, vm);
  tmem_ld16(t + 2 * NP + c0, vl);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(vh[j]) + (__uint_as_float(vm[j]) + __uint_as_float(vl[j]));
}

}  // namespace

// ---------------------------------------------------------------------------
// B operand of a pass: factor U (I x R, FP32) as 3 NP rows of length I (row
// pitch ld elements) in BF16: row p NP + r, column i holds part p of U[i, r]
// (rows r >= R are zero).  which = 0: mode N-1 for the trailing pass; 1: mode
// h-1 for the lead pass.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_split_factor(const DevDesc* __restrict__ d, int which) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.y;
  const int m = which ? d->h - 1 : d->N - 1;
  const int NP = d->umma_np;
  const int R = d->R[k];
  const int64_t I = d->dims[k][m];
  const int64_t ld = which ? d->bl_pitch[k] : d->bt_pitch[k];
  const float* __restrict__ U = reinterpret_cast<const float*>(d->U1[k][m]);
  __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(which ? d->Bl[k] : d->Bt[k]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += (int64_t)gridDim.x * blockDim.x) {
    for (int r = 0; r < NP; ++r) {
      const float w = r < R ? U[i * R + r] : 0.f;
      const __nv_bfloat16 hi = __float2bfloat16_rn(w);
      const float r1 = w - __bfloat162float(hi);
      const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
      const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
      dst[(int64_t)r * ld + i] = hi;
      dst[(int64_t)(NP + r) * ld + i] = mid;
      dst[(int64_t)(2 * NP + r) * ld + i] = lo;
    }
  }
}

// ---------------------------------------------------------------------------
// Trailing contraction.  Unit = 256 rows of X (two M = 128 MMAs); stage = 256
// rows x 64 columns of X (K-major, 128-byte swizzle) + the 64 matching
// columns of the split factor.
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(U_THREADS, 1) k_trailing_umma(const DevDesc* __restrict__ d) {
  using S = UmmaCfg<NP, true>;
  constexpr int ST = S::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const UmmaBars bars = umma_setup<S>(base);
  pdl_wait();  // the split factor and the factors come from earlier kernels of the sweep
  const uint32_t tmem = *bars.tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* err = &d->sc->timeout;
  const int K = d->K;
  const int planes = d->umma_planes;
  const UUnits us(d->lt_sched, d->lt_prefix[K]);

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
        const int nch = (int)((d->trail_cols[k] + 63) / 64);
        prefetch_tmap(&d->tmap_trail[k]);
        if (planes > 1) prefetch_tmap(&d->tmap_trail_lo[k]);
        prefetch_tmap(&d->tmap_bt[k]);
        // hi + lo storage: the lo plane's chunks follow the hi plane's
        for (int c = 0; c < planes * nch; ++c, ++it) {
          const int s = it % ST;
          const int cc = c < nch ? c : c - nch;
          if (!mbar_wait(smem_u32(&bars.empty[s]), ((it / ST) & 1) ^ 1, err)) { ok = false; break; }
          const uint32_t sa = smem_u32(base + s * S::STAGE);
          const uint32_t fb = smem_u32(&bars.full[s]);
          mbar_arrive_expect_tx(fb, S::STAGE);
          tma_load_2d_hint(sa, c < nch ? &d->tmap_trail[k] : &d->tmap_trail_lo[k], fb, cc * 64, row0, pol);
          tma_load_2d(sa + S::A_BYTES, &d->tmap_bt[k], fb, cc * 64, 0);
        }
      }
      for (uint32_t i = it > (uint32_t)ST ? it - ST : 0; i < it; ++i)
        mbar_wait_drain(smem_u32(&bars.full[i % ST]), (i / ST) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------ MMA issuer
      constexpr uint32_t IDESC = umma_idesc_bf16(128, 3 * NP, 0, 0);
      uint32_t it = 0, tc = 0;
      bool ok = true;
      for (int jn = us.first; jn < us.end && ok; jn += us.step, ++tc) {
        const int g = us.unit(jn);
        int k = 0;
        while (d->lt_prefix[k + 1] <= g) ++k;
        const int nch = (int)((d->trail_cols[k] + 63) / 64);
        const int b = tc & 1;
        if (!mbar_wait(smem_u32(&bars.tempty[b]), ((tc >> 1) & 1) ^ 1, err)) { ok = false; break; }
        tc_fence_after();
        for (int c = 0; c < planes * nch; ++c, ++it) {
          const int s = it % ST;
          if (!mbar_wait(smem_u32(&bars.full[s]), (it / ST) & 1, err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t xa = smem_u32(base + s * S::STAGE);
          const uint32_t ba = xa + S::A_BYTES;
#pragma unroll
          for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              umma_bf16(tmem + (uint32_t)((b * 2 + half) * S::ACC), umma_desc_sw128(xa + half * 16384 + ks * 32, 16, 1024),
                        umma_desc_sw128(ba + ks * 32, 16, 1024), IDESC, (c > 0 || ks > 0) ? 1u : 0u);
          umma_commit(smem_u32(&bars.empty[s]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&bars.tfull[b]));
      }
      // every MMA issued by this thread completes before TMEM is freed
      umma_commit(smem_u32(bars.drain));
      mbar_wait_drain(smem_u32(bars.drain), 0);
    }
  } else {
    // ---------------------------------------------------------- epilogue
    // The warp's 32 rows of a half tile are 32 R consecutive floats of Pl:
    // they go through the warp's staging rows in shared memory (stride
    // NP + 1: conflict-free) and out as coalesced stores.
    const int q = warp & 3;  // TMEM lanes 32 q .. 32 q + 31
    float* stg = reinterpret_cast<float*>(base + ST * S::STAGE + 256) + (warp - 2) * 32 * (NP + 1);
    uint32_t tc = 0;
    for (int jn = us.first; jn < us.end; jn += us.step, ++tc) {
      const int g = us.unit(jn);
      int k = 0;
      while (d->lt_prefix[k + 1] <= g) ++k;
      const int b = tc & 1;
      if (!mbar_wait(smem_u32(&bars.tfull[b]), (tc >> 1) & 1, err)) break;
      tc_fence_after();
      const int64_t row0 = (int64_t)(g - d->lt_prefix[k]) * 256;
      const int64_t rows = d->lead_rows[k];
      const int R = d->R[k];
      float* P = reinterpret_cast<float*>(d->Pl[k]);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const uint32_t t = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((b * 2 + half) * S::ACC);
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16) {
          float v[16];
          tmem_parts16<NP>(t, c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) stg[lane * (NP + 1) + c0 + j] = v[j];
        }
        __syncwarp();
        const int64_t wrow0 = row0 + half * 128 + 32 * q;  // first row of this warp
        const int64_t nrow = rows - wrow0 < 32 ? rows - wrow0 : 32;
        const int ne = nrow > 0 ? (int)nrow * R : 0;
        float* dst = P + wrow0 * R;
        for (int e = lane; e < ne; e += 32) dst[e] = stg[(e / R) * (NP + 1) + e % R];
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars.tempty[b]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, S::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Lead contraction.  Unit = 256 columns j x a range of i0 slabs (one split);
// per slab the K loop runs over i1 in stages of 64: X[i0, i1 .. i1+63, j ..
// j+255] as four 64 x 64 boxes of the 3-D view (MN-major A, 128-byte swizzle)
// + the 64 matching columns of the split U1.
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(U_THREADS, 1) k_lead_umma(const DevDesc* __restrict__ d) {
  using S = UmmaCfg<NP, false>;
  constexpr int ST = S::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const UmmaBars bars = umma_setup<S>(base);
  pdl_wait();  // the split factor and the factors come from earlier kernels of the sweep
  const uint32_t tmem = *bars.tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* err = &d->sc->timeout;
  const int K = d->K;
  const int planes = d->umma_planes;
  const UUnits us(d->tt_sched, d->tt_prefix[K]);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      const uint64_t pol = l2_evict_first_policy();
      uint32_t it = 0;
      bool ok = true;
      for (int jn = us.first; jn < us.end && ok; jn += us.step) {
        const int u = us.unit(jn);
        int k = 0;
        while (d->tt_prefix[k + 1] <= u) ++k;
        const int local = u - d->tt_prefix[k];
        const int ctile = local % d->tt_ctiles[k];
        const int split = local / d->tt_ctiles[k];
        const int I0 = (int)d->dims[k][0], I1 = (int)d->dims[k][1];
        const int per = (int)(d->split_rows[k] / I1);  // slabs per split
        const int a0 = split * per, a1 = min(I0, a0 + per);
        const int nst = (I1 + 63) / 64;
        prefetch_tmap(&d->tmap_lead3[k]);
        if (planes > 1) prefetch_tmap(&d->tmap_lead3_lo[k]);
        prefetch_tmap(&d->tmap_bl[k]);
        for (int i0 = a0; i0 < a1 && ok; ++i0)
          for (int st = 0; st < planes * nst; ++st, ++it) {  // hi + lo: the lo plane's stages follow
            const int s = it % ST;
            const int ss = st < nst ? st : st - nst;
            const CUtensorMap* xm = st < nst ? &d->tmap_lead3[k] : &d->tmap_lead3_lo[k];
            if (!mbar_wait(smem_u32(&bars.empty[s]), ((it / ST) & 1) ^ 1, err)) { ok = false; break; }
            const uint32_t sa = smem_u32(base + s * S::STAGE);
            const uint32_t fb = smem_u32(&bars.full[s]);
            mbar_arrive_expect_tx(fb, S::STAGE);
#pragma unroll
            for (int qb = 0; qb < 4; ++qb)
              tma_load_3d_hint(sa + qb * 8192, xm, fb, ctile * 256 + qb * 64, ss * 64, i0, pol);
            tma_load_2d(sa + S::A_BYTES, &d->tmap_bl[k], fb, ss * 64, 0);
          }
      }
      for (uint32_t i = it > (uint32_t)ST ? it - ST : 0; i < it; ++i)
        mbar_wait_drain(smem_u32(&bars.full[i % ST]), (i / ST) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------ MMA issuer
      constexpr uint32_t IDESC = umma_idesc_bf16(128, 3 * NP, 1, 0);
      uint32_t it = 0, sc = 0;  // stages, slabs
      bool ok = true;
      for (int jn = us.first; jn < us.end && ok; jn += us.step) {
        const int u = us.unit(jn);
        int k = 0;
        while (d->tt_prefix[k + 1] <= u) ++k;
        const int local = u - d->tt_prefix[k];
        const int split = local / d->tt_ctiles[k];
        const int I0 = (int)d->dims[k][0], I1 = (int)d->dims[k][1];
        const int per = (int)(d->split_rows[k] / I1);
        const int a0 = split * per, a1 = min(I0, a0 + per);
        const int nst = (I1 + 63) / 64;
        for (int i0 = a0; i0 < a1 && ok; ++i0, ++sc) {
          const int b = sc & 1;
          if (!mbar_wait(smem_u32(&bars.tempty[b]), ((sc >> 1) & 1) ^ 1, err)) { ok = false; break; }
          tc_fence_after();
          for (int st = 0; st < planes * nst; ++st, ++it) {
            const int s = it % ST;
            if (!mbar_wait(smem_u32(&bars.full[s]), (it / ST) & 1, err)) { ok = false; break; }
            tc_fence_after();
            const uint32_t xa = smem_u32(base + s * S::STAGE);
            const uint32_t ba = xa + S::A_BYTES;
#pragma unroll
            for (int half = 0; half < 2; ++half)
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                umma_bf16(tmem + (uint32_t)((b * 2 + half) * S::ACC),
                          umma_desc_sw128(xa + half * 16384 + ks * 2048, 8192, 1024),
                          umma_desc_sw128(ba + ks * 32, 16, 1024), IDESC, (st > 0 || ks > 0) ? 1u : 0u);
            umma_commit(smem_u32(&bars.empty[s]));
          }
          if (!ok) break;
          umma_commit(smem_u32(&bars.tfull[b]));
        }
      }
      umma_commit(smem_u32(bars.drain));
      mbar_wait_drain(smem_u32(bars.drain), 0);
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;
    uint32_t sc = 0;
    bool ok = true;
    for (int jn = us.first; jn < us.end && ok; jn += us.step) {
      const int u = us.unit(jn);
      int k = 0;
      while (d->tt_prefix[k + 1] <= u) ++k;
      const int local = u - d->tt_prefix[k];
      const int ctile = local % d->tt_ctiles[k];
      const int split = local / d->tt_ctiles[k];
      const int I0 = (int)d->dims[k][0], I1 = (int)d->dims[k][1];
      const int per = (int)(d->split_rows[k] / I1);
      const int a0 = split * per, a1 = min(I0, a0 + per);
      const int R = d->R[k];
      const float* __restrict__ U0 = reinterpret_cast<const float*>(d->U1[k][0]);
      float acc[2][NP];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < NP; ++r) acc[h][r] = 0.f;
      for (int i0 = a0; i0 < a1; ++i0, ++sc) {
        // U0[i0, :] (zero past R); the loads issue before the wait
        float u0[NP];
#pragma unroll
        for (int r = 0; r < NP; ++r) u0[r] = __ldg(U0 + (int64_t)i0 * R + min(r, R - 1));
#pragma unroll
        for (int r = 0; r < NP; ++r)
          if (r >= R) u0[r] = 0.f;
        const int b = sc & 1;
        if (!mbar_wait(smem_u32(&bars.tfull[b]), (sc >> 1) & 1, err)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const uint32_t t = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((b * 2 + half) * S::ACC);
#pragma unroll
          for (int c0 = 0; c0 < NP; c0 += 16) {
            float v[16];
            tmem_parts16<NP>(t, c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[half][c0 + j] = fmaf(u0[c0 + j], v[j], acc[half][c0 + j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars.tempty[b]));
      }
      if (!ok) break;
      const int J = (int)d->trail_cols[k];
      float* part = reinterpret_cast<float*>(d->partial) + d->partial_off[k] + (int64_t)split * J * R;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int col = ctile * 256 + half * 128 + 32 * q + lane;
        if (col < J) {
#pragma unroll
          for (int r = 0; r < NP; ++r)
            if (r < R) part[(int64_t)col * R + r] = acc[half][r];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, S::TMEM_COLS);
}

// ------------------------------------------------------------- launchers ----

cudaError_t launch_split_factor(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd, int which) {
  const int m = which ? hd.h - 1 : hd.N - 1;
  int64_t imax = 1;
  for (int k = 0; k < hd.K; ++k) imax = hd.dims[k][m] > imax ? hd.dims[k][m] : imax;
  const unsigned gx = (unsigned)((imax + 255) / 256);
  cudaError_t e = launch_pdl(k_split_factor, dim3(gx, hd.K), dim3(256), 0, c.stream, dd, which);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NP>
static cudaError_t trailing_umma_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  const int total = hd.lt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  const size_t smem = UmmaCfg<NP, true>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_trailing_umma<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = hd.lt_sched ? hd.lt_grid : (total < c.num_sms ? total : c.num_sms);
  e = launch_pdl(k_trailing_umma<NP>, dim3(grid), dim3(U_THREADS), smem, c.stream, dd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int NP>
static cudaError_t lead_umma_impl(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  const int total = hd.tt_prefix[hd.K];
  if (total == 0) return cudaSuccess;
  const size_t smem = UmmaCfg<NP, false>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_lead_umma<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = hd.tt_sched ? hd.tt_grid : (total < c.num_sms ? total : c.num_sms);
  e = launch_pdl(k_lead_umma<NP>, dim3(grid), dim3(U_THREADS), smem, c.stream, dd);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int umma_np(int Rmax) { return Rmax <= 16 ? 16 : Rmax <= 32 ? 32 : 0; }

cudaError_t launch_trailing_umma(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  if (hd.umma_np == 16) return trailing_umma_impl<16>(c, dd, hd);
  if (hd.umma_np == 32) return trailing_umma_impl<32>(c, dd, hd);
  return cudaErrorInvalidValue;
}

cudaError_t launch_lead_umma(const LaunchCfg& c, const DevDesc* dd, const DevDesc& hd) {
  if (hd.umma_np == 16) return lead_umma_impl<16>(c, dd, hd);
  if (hd.umma_np == 32) return lead_umma_impl<32>(c, dd, hd);
  return cudaErrorInvalidValue;
}

}  // namespace cncpd
