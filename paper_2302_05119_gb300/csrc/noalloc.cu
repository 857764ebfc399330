// Allocation-free MTTKRP of the last mode of one third-order FP32 tensor.
//
// Some callers cannot let this library call cudaMalloc: code whose device
// memory is owned entirely by another allocator (a caching allocator or a
// fixed arena that has already reserved the GPU's memory), code running under
// a strict per-process memory budget, or code in the middle of latency-
// sensitive work where a cudaMalloc may implicitly synchronise the device.
// For them this entry point keeps its only scratch -- the split-K partial
// sums of the lead-mode contraction -- in a file-scope device array of fixed
// size instead of allocating it, and takes every input and output from the
// caller.
//
// The array below is reserved on every GPU that loads the library, for the
// life of the process.  In host code its name is only a host-side stand-in
// for the device symbol, so its device address is fetched once per device
// with cudaGetSymbolAddress (on the first call made with that device
// current) and that address is what the kernels receive.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/cncpd.h"
#include "cncpd_internal.cuh"

namespace {

constexpr int64_t kScratchFloats = 2 * 1024 * 1024;  // 8 MiB of FP32 partial sums
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

std::mutex g_mu;
float* g_scratch_addr[kMaxDevices] = {nullptr};

int fail(int code, const char* msg) { return cncpd::set_error(code, msg); }

// Variant of the lead-mode contraction: partial[s][j][r] = sum over the rows
// of split s of X[row, j] * U0[i0(row), r] * U1[i1(row), r], row = i0*I1 + i1.
// Thread (tx, ty): column j = blockIdx.x * 64 + tx, every second row of the
// split (ty = 0, 1); the two row halves are added through shared memory.
// RMAXL is the rank bucket (16, 32 or 64): the accumulators are indexed by
// compile-time constants only, so they stay in registers.
template <int RMAXL>
__global__ void __launch_bounds__(128) k_lead_noalloc(const float* __restrict__ X, int64_t I0, int64_t I1,
                                                      int64_t J, const float* __restrict__ U0,
                                                      const float* __restrict__ U1, int R, int64_t split_rows,
                                                      float* __restrict__ partial) {
  __shared__ float w[64][RMAXL];
  __shared__ float red[64][RMAXL];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t j = (int64_t)blockIdx.x * 64 + tx;
  const int64_t rows = I0 * I1;
  const int64_t rb = (int64_t)blockIdx.y * split_rows;
  const int64_t re = rb + split_rows < rows ? rb + split_rows : rows;
  float acc[RMAXL];
#pragma unroll
  for (int r = 0; r < RMAXL; ++r) acc[r] = 0.f;
  for (int64_t r0 = rb; r0 < re; r0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * R; e += blockDim.x) {
      const int i = e / R, r = e % R;
      const int64_t row = r0 + i;
      w[i][r] = row < re ? U0[(row / I1) * R + r] * U1[(row % I1) * R + r] : 0.f;
    }
    __syncthreads();
    const int nrow = (int)(re - r0 < 64 ? re - r0 : 64);
    if (j < J)
      for (int i = ty; i < nrow; i += 2) {
        const float x = X[(r0 + i) * J + j];
#pragma unroll
        for (int r = 0; r < RMAXL; ++r)
          if (r < R) acc[r] = fmaf(x, w[i][r], acc[r]);
      }
  }
  __syncthreads();
  if (ty == 1) {
#pragma unroll
    for (int r = 0; r < RMAXL; ++r)
      if (r < R) red[tx][r] = acc[r];
  }
  __syncthreads();
  if (ty == 0 && j < J) {
#pragma unroll
    for (int r = 0; r < RMAXL; ++r)
      if (r < R) partial[((int64_t)blockIdx.y * J + j) * R + r] = acc[r] + red[tx][r];
  }
}

// M[j, r] = sum_s partial[s][j][r], splits added in order.
__global__ void k_reduce_noalloc(const float* __restrict__ partial, int nsplit, int64_t JR, float* __restrict__ M) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < JR; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < nsplit; ++i) s += partial[(int64_t)i * JR + e];
    M[e] = s;
  }
}

int scratch_for_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CNCPD_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(CNCPD_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(CNCPD_ECUDA, cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return CNCPD_OK;
}

// Every array of this entry point must be device (or managed) memory of the
// current device: unlike the handle-based calls it copies nothing, so a host
// pointer is refused here instead of faulting in the kernel.
// cudaPointerGetAttributes allocates nothing.
int check_device_pointer(const void* p, int dev, const char* name) {
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CNCPD_EINVAL, "pointer attributes not available");
  }
  const bool ok = (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
  if (!ok) {
    static thread_local char msg[128];
    snprintf(msg, sizeof msg, "%s must be device or managed memory of the current device", name);
    return fail(CNCPD_EINVAL, msg);
  }
  return CNCPD_OK;
}

template <int RB>
void launch_lead_noalloc(dim3 grid, cudaStream_t s, const float* X, int64_t I0, int64_t I1, int64_t J,
                         const float* U0, const float* U1, int R, int64_t split_rows, float* partial) {
  k_lead_noalloc<RB><<<grid, 128, 0, s>>>(X, I0, I1, J, U0, U1, R, split_rows, partial);
}

}  // namespace

extern "C" int cncpd_mttkrp_last_mode_noalloc(const float* X, int64_t I0, int64_t I1, int64_t I2, const float* U0,
                                              const float* U1, int R, float* M, void* stream) {
  if (!X || !U0 || !U1 || !M) return fail(CNCPD_EINVAL, "NULL pointer argument");
  if (I0 < 1 || I1 < 1 || I2 < 1 || R < 1 || R > 64) return fail(CNCPD_EINVAL, "sizes must be >= 1 and R <= 64");
  const int64_t per_split = I2 * R;
  if (per_split > kScratchFloats)
    return fail(CNCPD_EINVAL, "I2 * R exceeds the fixed scratch of 2097152 floats (8 MiB)");
  int dev = 0;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return fail(CNCPD_ECUDA, cudaGetErrorString(de));
  int rc = check_device_pointer(X, dev, "X");
  if (rc == CNCPD_OK) rc = check_device_pointer(U0, dev, "U0");
  if (rc == CNCPD_OK) rc = check_device_pointer(U1, dev, "U1");
  if (rc == CNCPD_OK) rc = check_device_pointer(M, dev, "M");
  if (rc != CNCPD_OK) return rc;
  float* scratch = nullptr;
  rc = scratch_for_current_device(&scratch);
  if (rc != CNCPD_OK) return rc;
  const int64_t rows = I0 * I1;
  // about 600 CTAs in total, at least 64 rows each, within the scratch
  const int64_t ctiles = (I2 + 63) / 64;
  int64_t want = 600 / ctiles;
  if (want < 1) want = 1;
  int64_t cap = kScratchFloats / per_split;
  if (want > cap) want = cap;
  int64_t split_rows = (rows + want - 1) / want;
  if (split_rows < 64) split_rows = 64;
  const int64_t nsplit = (rows + split_rows - 1) / split_rows;
  if (nsplit > 65535) return fail(CNCPD_EINVAL, "tensor too large for the split grid");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dim3 grid((unsigned)ctiles, (unsigned)nsplit);
  if (R <= 16) launch_lead_noalloc<16>(grid, s, X, I0, I1, I2, U0, U1, R, split_rows, scratch);
  else if (R <= 32) launch_lead_noalloc<32>(grid, s, X, I0, I1, I2, U0, U1, R, split_rows, scratch);
  else launch_lead_noalloc<64>(grid, s, X, I0, I1, I2, U0, U1, R, split_rows, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    int grid = (int)((per_split + 255) / 256);
    if (grid > 1024) grid = 1024;
    k_reduce_noalloc<<<grid, 256, 0, s>>>(scratch, (int)nsplit, per_split, M);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(CNCPD_ECUDA, cudaGetErrorString(e));
  return CNCPD_OK;
}
