// C ABI and host orchestration of CoNCPD-APG (Algorithm 1) and
// lraCoNCPD-APG (Algorithm 2) on one GPU.
//
// One iteration = one sweep (cores, then modes 1..N for all blocks) + the
// objective, replayed as a CUDA graph; the host reads F(k) and, if it did not
// decrease, replays the re-update graph (Algorithm 1 safeguard: restore the
// iterate of the start of the iteration and sweep again with every
// extrapolation weight 0).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/cncpd.h"
#include "cncpd_internal.cuh"

using namespace cncpd;

namespace {

thread_local std::string g_err;

int set_err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(expr)                                                                         \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return set_err(_e == cudaErrorMemoryAllocation ? CNCPD_ENOMEM : CNCPD_ECUDA,       \
                     "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
  } while (0)

#define TRY(expr)           \
  do {                      \
    int _r = (expr);        \
    if (_r != CNCPD_OK) return _r; \
  } while (0)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct HostScalars {  // mirror of the head of DevScalars read back each iteration
  double t, w_hat;
  int have_prev, have_cur, nonfinite, timeout;
  double F, relerr;
};

}  // namespace

int cncpd::set_error(int code, const char* msg) { return set_err(code, "%s", msg); }

struct cncpd_ctx {
  int device = 0, num_sms = 0;
  int K = 0, N = 0, h = 0;
  std::vector<int64_t> dims;  // K*N
  std::vector<int> R, L, nonneg;
  int Rmax = 0, RP = 0;
  cncpd_opts opts{};
  int st = ST_F32, fp64 = 0;
  size_t fsz = 4;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;

  // factor arenas
  size_t arena_elems = 0;
  std::vector<size_t> foff;  // K*N element offsets
  char *A1 = nullptr, *A2 = nullptr, *AS = nullptr;
  char* A_eval = nullptr;        // cncpd_objective_grad_at: the iterate kept aside (allocated on first use)
  char* sc_eval = nullptr;       // and the solver scalars

  DevDesc hd{};
  DevDesc* dd = nullptr;
  DevScalars* sc = nullptr;
  std::vector<double> lam_init;  // K*RMAX
  std::vector<double> xnorm2;    // K
  int64_t* d_red_prefix = nullptr;
  HostScalars* hs = nullptr;     // pinned

  // solver state on the host
  bool dirty = true;             // factors/cores changed: re-initialise history
  // "F did not increase" (Algorithm 1 safeguard) when F - F_prev <= tie_tol * |F_prev|:
  // 1e-13 with FP64 factors; 1e-6 with FP32 factors, whose objective is only
  // accurate to a few 1e-7 relative (cancellation in the Gram expansion)
  double tie_tol = 1e-13;
  double F_prev = 0.0, rel_prev = 0.0;
  int total_iters = 0;

  // two main graphs used alternately (each records its own profile events, so
  // one iteration's pass times are read while the next one runs) and the
  // re-update graph (event set 2)
  cudaGraphExec_t g_main[2] = {nullptr, nullptr}, g_redo = nullptr;
  // with profile = 1 only every PROFILE_EVERY-th main sweep records events
  // (event nodes in a graph cost several microseconds each); the others
  // replay g_plain
  cudaGraphExec_t g_plain = nullptr;
  int main_runs = 0, redo_runs = 0, prof_runs = 0, timed_runs = 0;
  bool rec_on = true;
  cudaEvent_t ev[3][4] = {};
  int ev_set = 0;
  HostMirror* hm = nullptr;      // pinned, mapped; written by the objective kernel
  HostMirror* hm_dev = nullptr;
  cudaStream_t side = nullptr;                // branch for work independent of a tensor pass
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // opts.stream_x: one device window holds the stored values of one block at
  // a time; the caller's tensors (xsrc, in x_dtype) are quantised into it on
  // demand (load_block)
  std::vector<const void*> xsrc;
  int x_src_f64 = 0;
  void* window = nullptr;
  void* window_lo = nullptr;
  void* xstage = nullptr;        // staging buffer for pageable sources
  size_t window_bytes = 0;
  int window_block = -1;
  double* wscratch = nullptr;    // norm partials of a window load
  double* wnorm = nullptr;

  // lead-pass split plan: units per SM in use, whether it was measured, and
  // the partial-sum capacity (elements) every candidate plan fits in
  int lead_mult = 0;
  bool lead_tuned = false;
  size_t partial_cap = 0;

  // LRA
  bool lra = false;
  std::vector<int> Rt;
  DevDesc hd_als{};
  DevDesc* dd_als = nullptr;
  DevDesc* dd_tmp = nullptr;     // a restricted copy of hd (streamed X: one block's passes)
  int RPt = 0;
  int64_t* d_red_prefix_als = nullptr;
  int* d_active = nullptr;
  int* d_status = nullptr;
  double* d_relk = nullptr;

  int64_t dim(int k, int n) const { return dims[(size_t)k * N + n]; }
  void* U1p(int k, int n) const { return A1 + foff[(size_t)k * N + n] * fsz; }
  void* U2p(int k, int n) const { return A2 + foff[(size_t)k * N + n] * fsz; }
};

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D tensor map (FP32 or BF16 elements) over a rows x cols matrix with row
// pitch `pitch` elements, box (box_cols x box_rows), out-of-range elements
// read as zero.
bool encode_map(CUtensorMap* m, const void* base, int st, int64_t rows, int64_t cols, int64_t pitch, int box_cols,
                int box_rows, CUtensorMapSwizzle swz) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const int esz = st == ST_BF16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * esz)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, st == ST_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3-D tensor map of a BF16 third-order tensor stored as (I0 I1) rows of J
// elements (row pitch `pitch`): dims (J, I1, I0), boxes of 64 x 64 x 1 with
// the 128-byte swizzle.
bool encode_x3(CUtensorMap* m, const void* base, int64_t J, int64_t I1, int64_t I0, int64_t pitch) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)J, (cuuint64_t)I1, (cuuint64_t)I0};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * 2), (cuuint64_t)(I1 * pitch * 2)};
  cuuint32_t box[3] = {64, 64, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int dalloc(cncpd_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(CNCPD_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return CNCPD_OK;
}

// tcgen05 passes of a BF16 third-order problem with ranks up to 32: buffers
// for the split factors that are the MMAs' B operands and the TMA
// descriptors of the 3-D view of X and of the split factors.  d.use_umma
// stays 0 when the problem does not qualify (the CUDA-core passes run).
int setup_umma(cncpd_ctx* c, DevDesc& d, int Rmax) {
  d.use_umma = 0;
  d.umma_np = 0;
  d.umma_planes = 1;
  const int np = umma_np(Rmax);
  const bool x2 = c->st == ST_BF16X2;
  if (!c->opts.tensor_cores || !(c->st == ST_BF16 || x2) || d.N != 3 || d.h != 2 || np == 0 ||
      !tensor_map_encoder())
    return CNCPD_OK;
  if (!x2 && !d.tmap_trail) return CNCPD_OK;
  // [lead3 | Bt | Bl | trail hi | trail lo | lead3 lo] (the last three with hi + lo storage)
  std::vector<CUtensorMap> maps(6 * CNCPD_KMAX);
  for (int k = 0; k < d.K; ++k) {
    const int64_t J = d.trail_cols[k], I1 = d.dims[k][1], I0 = d.dims[k][0];
    d.bt_pitch[k] = (J + 7) / 8 * 8;
    d.bl_pitch[k] = (I1 + 7) / 8 * 8;
    TRY(dalloc(c, &d.Bt[k], (size_t)3 * np * d.bt_pitch[k] * 2));
    TRY(dalloc(c, &d.Bl[k], (size_t)3 * np * d.bl_pitch[k] * 2));
    if (!encode_x3(&maps[k], d.X[k], J, I1, I0, d.pitch[k]) ||
        !encode_map(&maps[CNCPD_KMAX + k], d.Bt[k], ST_BF16, 3 * np, J, d.bt_pitch[k], 64, 3 * np,
                    CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_map(&maps[2 * CNCPD_KMAX + k], d.Bl[k], ST_BF16, 3 * np, I1, d.bl_pitch[k], 64, 3 * np,
                    CU_TENSOR_MAP_SWIZZLE_128B))
      return CNCPD_OK;
    if (x2 && (!encode_map(&maps[3 * CNCPD_KMAX + k], d.X[k], ST_BF16, d.lead_rows[k], J, d.pitch[k], 64, 256,
                           CU_TENSOR_MAP_SWIZZLE_128B) ||
               !encode_map(&maps[4 * CNCPD_KMAX + k], d.Xlo[k], ST_BF16, d.lead_rows[k], J, d.pitch[k], 64, 256,
                           CU_TENSOR_MAP_SWIZZLE_128B) ||
               !encode_x3(&maps[5 * CNCPD_KMAX + k], d.Xlo[k], J, I1, I0, d.pitch[k])))
      return CNCPD_OK;
  }
  CUtensorMap* dm = nullptr;
  TRY(dalloc(c, (void**)&dm, maps.size() * sizeof(CUtensorMap)));
  CU(cudaMemcpyAsync(dm, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  d.tmap_lead3 = dm;
  d.tmap_bt = dm + CNCPD_KMAX;
  d.tmap_bl = dm + 2 * CNCPD_KMAX;
  if (x2) {
    d.tmap_trail = dm + 3 * CNCPD_KMAX;
    d.tmap_trail_lo = dm + 4 * CNCPD_KMAX;
    d.tmap_lead3_lo = dm + 5 * CNCPD_KMAX;
    d.umma_planes = 2;
  }
  d.umma_np = np;
  d.use_umma = 1;
  return CNCPD_OK;
}

// TF32 trailing pass of an FP32 third-order problem with ranks up to 32: the
// buffers of the factor's two TF32 parts (the B operand) and their TMA
// descriptors.  d.use_tf32 stays 0 when the problem does not qualify.
int setup_tf32(cncpd_ctx* c, DevDesc& d, int Rmax) {
  d.use_tf32 = 0;
  const int np = umma_np(Rmax);
  if (d.use_umma || !d.use_tma || !c->opts.tensor_cores || !c->opts.tf32 || c->st != ST_F32 || d.N != 3 ||
      d.h != 2 || np == 0 ||
      !d.tmap_trail || !tensor_map_encoder())
    return CNCPD_OK;
  // the kernel's split of X (Veltkamp, x * (2^13 + 1)) needs |x| < 2^114:
  // guaranteed when every ||X^(k)||^2 is below 2^228
  CU(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < d.K; ++k)
    if (!(c->xnorm2[k] < std::ldexp(1.0, 228))) return CNCPD_OK;
  std::vector<CUtensorMap> maps(CNCPD_KMAX);
  for (int k = 0; k < d.K; ++k) {
    const int64_t J = d.trail_cols[k];
    d.bt_pitch[k] = (J + 31) / 32 * 32;
    TRY(dalloc(c, &d.Bt[k], (size_t)2 * np * d.bt_pitch[k] * sizeof(float)));
    if (!encode_map(&maps[k], d.Bt[k], ST_F32, 2 * np, J, d.bt_pitch[k], 32, 2 * np, CU_TENSOR_MAP_SWIZZLE_128B))
      return CNCPD_OK;
  }
  CUtensorMap* dm = nullptr;
  TRY(dalloc(c, (void**)&dm, maps.size() * sizeof(CUtensorMap)));
  CU(cudaMemcpyAsync(dm, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  d.tmap_bt = dm;
  d.umma_np = np;
  d.use_tf32 = 1;
  return CNCPD_OK;
}

// Assign units of cost cost[u] to P persistent CTAs, longest first, each to
// the CTA with the least work so far (ties: lowest index); every CTA then
// walks its units in increasing id.  Returns P + 1 start offsets followed by
// the ids.  With equal costs this is the plain round-robin order.
std::vector<int> lpt_schedule(const std::vector<int64_t>& cost, int P) {
  const int n = (int)cost.size();
  std::vector<int> order(n);
  for (int u = 0; u < n; ++u) order[u] = u;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  using Slot = std::pair<int64_t, int>;  // (load, CTA)
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  for (int p = 0; p < P; ++p) heap.push({0, p});
  std::vector<std::vector<int>> lists(P);
  for (int u : order) {
    Slot s = heap.top();
    heap.pop();
    lists[s.second].push_back(u);
    heap.push({s.first + cost[u], s.second});
  }
  std::vector<int> out(P + 1 + n);
  int pos = P + 1;
  for (int p = 0; p < P; ++p) {
    out[p] = pos - (P + 1);
    std::sort(lists[p].begin(), lists[p].end());
    for (int u : lists[p]) out[pos++] = u;
  }
  out[P] = n;
  return out;
}

// Largest total cost of a CTA when lpt_schedule assigns `cost` to P CTAs.
int64_t lpt_makespan(const std::vector<int64_t>& cost, int P) {
  const std::vector<int> sched = lpt_schedule(cost, P);
  int64_t worst = 0;
  for (int p = 0; p < P; ++p) {
    int64_t load = 0;
    for (int q = sched[p]; q < sched[p + 1]; ++q) load += cost[sched[P + 1 + q]];
    worst = std::max(worst, load);
  }
  return worst;
}

// Cost of one unit of the persistent passes, in bytes of DRAM time: the
// larger of the bytes of X it reads (`valid` elements) and its arithmetic on
// the whole tile (`tile` elements, out-of-range parts included): R FMAs per
// element on the CUDA cores, 0.16 byte-times each (R = 25 matches the HBM
// rate of FP32 data on this GPU), or about a quarter of the DRAM time of a
// full tile on the tensor cores; plus four 32 KiB stages for the unit's
// epilogue and pipeline refill (measured on the 256^3 workload: 1, 2, 4 and 8
// lead units per SM took 56, 60, 67 and 74 us).
int64_t unit_cost(const DevDesc& d, int st, int64_t valid, int64_t tile, bool tensor_cores) {
  const int64_t es = st == ST_BF16 ? 2 : 4;
  const int64_t work = tensor_cores ? tile / 2 : tile * d.Rmax * 16 / 100;
  return std::max(valid * es, work) + 4 * 32768;
}

// Split-K plan of the lead-mode contraction for rank bucket RP, aiming at
// about target_units units in all (per_block: for every block, which then
// runs alone, as with streamed X).
void plan_lead_units(cncpd_ctx* c, DevDesc& d, int RP, int fp64, int64_t target_units, size_t* partial_elems,
                     bool per_block = false) {
  const int cpt = lead_cpt(fp64, RP);
  const int tile_cols = (d.use_tma || d.use_umma) ? 256 : 64 * cpt;
  int64_t tot_rows = 0;
  for (int k = 0; k < d.K; ++k) tot_rows += d.lead_rows[k];
  d.tt_prefix[0] = 0;
  size_t off = 0;
  for (int k = 0; k < d.K; ++k) {
    const int64_t J = d.trail_cols[k];
    const int ctiles = (int)((J + tile_cols - 1) / tile_cols);
    const int64_t rows = d.lead_rows[k];
    const int64_t share = per_block ? rows : tot_rows;
    int64_t want = std::max<int64_t>(1, (target_units * rows) / std::max<int64_t>(1, share) / ctiles);
    int64_t split_rows = (rows + want - 1) / want;
    if (d.use_umma) {
      const int64_t I1 = d.dims[k][1];
      split_rows = (split_rows + I1 - 1) / I1 * I1;  // whole i0 slabs of the tensor-core pass
    } else {
      split_rows = std::max<int64_t>(split_rows, 64);
      split_rows = ((split_rows + 63) / 64) * 64;  // whole stages of the lead contraction
    }
    const int ns = (int)((rows + split_rows - 1) / split_rows);
    d.tt_ctiles[k] = ctiles;
    d.nsplit[k] = ns;
    d.split_rows[k] = split_rows;
    d.partial_off[k] = (int64_t)off;
    off += (size_t)ns * J * d.R[k];
    d.tt_prefix[k + 1] = d.tt_prefix[k] + ctiles * ns;
  }
  d.tt_cpt = cpt;
  d.tt_cols = tile_cols;
  *partial_elems = off;
}

// Unit costs of the current lead plan (unit order of tt_prefix).
std::vector<int64_t> lead_unit_costs(const cncpd_ctx* c, const DevDesc& d) {
  std::vector<int64_t> tt;
  for (int k = 0; k < d.K; ++k) {
    const int64_t rows = d.lead_rows[k], J = d.trail_cols[k];
    for (int s = 0; s < d.nsplit[k]; ++s) {
      const int64_t rb = s * d.split_rows[k];
      const int64_t re = std::min<int64_t>(rows, rb + d.split_rows[k]);
      for (int t = 0; t < d.tt_ctiles[k]; ++t) {
        const int64_t cols = std::min<int64_t>(d.tt_cols, J - (int64_t)t * d.tt_cols);
        tt.push_back(unit_cost(d, c->st, (re - rb) * cols, (re - rb) * d.tt_cols, d.use_umma));
      }
    }
  }
  return tt;
}

// Split-K plan of the lead pass.  The generic kernel takes about two
// 256-thread CTAs per SM.  For the persistent passes (one CTA per SM walking
// a longest-first unit list) the plan is the one, among about 1, 2, 3, 4, 6
// or 8 units per SM, whose list has the smallest largest load; ties go to
// fewer units (fewer split-K partials to add up).
constexpr int kLeadMults[] = {1, 2, 3, 4, 6, 8};

int plan_lead_splits(cncpd_ctx* c, DevDesc& d, int RP, int fp64, size_t* partial_elems) {
  if (!d.use_tma && !d.use_umma) {
    plan_lead_units(c, d, RP, fp64, (int64_t)c->num_sms * 2, partial_elems, c->opts.stream_x != 0);
    return 0;
  }
  if (c->opts.stream_x) {
    // blocks run one at a time: two units per SM for each
    plan_lead_units(c, d, RP, fp64, (int64_t)c->num_sms * 2, partial_elems, true);
    return 2;
  }
  int best = 1;
  int64_t best_span = -1;
  for (int mult : kLeadMults) {
    plan_lead_units(c, d, RP, fp64, (int64_t)c->num_sms * mult, partial_elems);
    const std::vector<int64_t> cost = lead_unit_costs(c, d);
    const int P = std::min<int>((int)cost.size(), c->num_sms);
    const int64_t span = lpt_makespan(cost, P);
    if (best_span < 0 || span < best_span) {
      best_span = span;
      best = mult;
    }
  }
  plan_lead_units(c, d, RP, fp64, (int64_t)c->num_sms * best, partial_elems);
  return best;
}

// Partial-sum elements of the largest candidate lead plan.
size_t lead_partial_cap(cncpd_ctx* c, DevDesc d, int RP, int fp64) {
  size_t cap = 0, pel = 0;
  if (!d.use_tma && !d.use_umma) {
    plan_lead_units(c, d, RP, fp64, (int64_t)c->num_sms * 2, &pel, c->opts.stream_x != 0);
    return pel;
  }
  if (c->opts.stream_x) {
    plan_lead_units(c, d, RP, fp64, (int64_t)c->num_sms * 2, &pel, true);
    return pel;
  }
  for (int mult : kLeadMults) {
    plan_lead_units(c, d, RP, fp64, (int64_t)c->num_sms * mult, &pel);
    cap = std::max(cap, pel);
  }
  return cap;
}

// Units of the trailing contraction: 256-row tiles (64 for the generic
// kernel).  On the FP32/BF16 CUDA-core pass (allow_split) a tile holding
// more than half of a CTA's share of X (X over the SM count) is cut along its
// columns into ranges of whole stages, so that one long-row block (say 4544
// x 19200) cannot outlast the others; each range leaves a partial Pl that a
// small kernel adds up in range order.  Returns the partial elements needed.
size_t plan_trailing_tiles(DevDesc& d, int num_sms, int st, int allow_split) {
  d.lt_rows = (d.use_tma || d.use_umma || d.use_tf32) ? 256 : 64;
  d.lt_prefix[0] = 0;
  d.trail_split = 0;
  d.Pl_part = nullptr;
  int64_t xtot = 0;
  for (int k = 0; k < d.K; ++k) xtot += d.lead_rows[k] * d.trail_cols[k];
  const int64_t cap = std::max<int64_t>(1, xtot / std::max(1, num_sms) / 2);
  const int64_t bc = st == ST_BF16 ? 64 : 32;  // columns of one 128-byte stage
  size_t off = 0;
  for (int k = 0; k < d.K; ++k) {
    const int64_t J = d.trail_cols[k];
    int js = 1;
    int64_t jc = J;
    if (allow_split && d.use_tma && !d.use_umma && !d.use_tf32 && (int64_t)d.lt_rows * J > cap) {
      const int64_t want = std::min<int64_t>(16, ((int64_t)d.lt_rows * J + cap - 1) / cap);
      jc = ((J + want - 1) / want + bc - 1) / bc * bc;
      js = (int)((J + jc - 1) / jc);
    }
    d.lt_js[k] = js;
    d.lt_jc[k] = (int)jc;
    d.plp_off[k] = (int64_t)off;
    if (js > 1) {
      d.trail_split = 1;
      off += (size_t)js * d.lead_rows[k] * d.R[k];
    }
    d.lt_prefix[k + 1] = d.lt_prefix[k] + js * (int)((d.lead_rows[k] + d.lt_rows - 1) / d.lt_rows);
  }
  return off;
}

// Unit costs of the current trailing plan (unit order of lt_prefix).
std::vector<int64_t> trailing_unit_costs(const cncpd_ctx* c, const DevDesc& d) {
  std::vector<int64_t> lt;
  for (int k = 0; k < d.K; ++k) {
    const int64_t rows = d.lead_rows[k], J = d.trail_cols[k];
    const int js = d.lt_js[k];
    for (int g = d.lt_prefix[k]; g < d.lt_prefix[k + 1]; ++g) {
      const int local = g - d.lt_prefix[k];
      const int64_t r0 = (int64_t)(local / js) * d.lt_rows;
      const int64_t jb = (int64_t)(local % js) * d.lt_jc[k];
      const int64_t cols = std::min<int64_t>(J, jb + d.lt_jc[k]) - jb;
      lt.push_back(unit_cost(d, c->st, std::min<int64_t>(d.lt_rows, rows - r0) * cols, (int64_t)d.lt_rows * cols,
                             d.use_umma || d.use_tf32));
    }
  }
  return lt;
}

// Trailing plan with column splits where they shorten the longest unit list
// by more than the extra launch that adds the ranges up costs (about 3 us,
// one SM's share of DRAM time for 128 KiB); else whole rows.  Returns the
// partial elements of the chosen plan.
size_t choose_trailing_plan(const cncpd_ctx* c, DevDesc& d, int allow_split) {
  const size_t plp = plan_trailing_tiles(d, c->num_sms, c->st, allow_split);
  if (!plp) return 0;
  auto span = [&](const DevDesc& x) {
    const std::vector<int64_t> cost = trailing_unit_costs(c, x);
    return lpt_makespan(cost, std::min<int>((int)cost.size(), c->num_sms));
  };
  DevDesc whole = d;
  plan_trailing_tiles(whole, c->num_sms, c->st, 0);
  if (span(d) + 4 * 32768 < span(whole)) return plp;
  d = whole;
  return 0;
}

// Balanced unit lists of the two TMA passes.  A unit's cost is the number of
// tensor elements it reads (the in-range part of its tiles) plus two stages'
// worth for its epilogue.
int plan_tma_schedules(cncpd_ctx* c, DevDesc& d) {
  d.lt_sched = d.tt_sched = nullptr;
  d.lt_grid = d.tt_grid = 0;
  if (!d.use_tma && !d.use_umma) return CNCPD_OK;
  const std::vector<int64_t> lt = trailing_unit_costs(c, d);
  const std::vector<int64_t> tt = lead_unit_costs(c, d);
  const std::vector<int64_t>* costs[2] = {&lt, &tt};
  for (int which = 0; which < 2; ++which) {
    const std::vector<int64_t>& cost = *costs[which];
    if (cost.empty()) continue;
    const int P = std::min<int>((int)cost.size(), c->num_sms);
    const std::vector<int> sched = lpt_schedule(cost, P);
    int* dev = nullptr;
    TRY(dalloc(c, (void**)&dev, sched.size() * sizeof(int)));
    CU(cudaMemcpyAsync(dev, sched.data(), sched.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (which == 0) {
      d.lt_sched = dev;
      d.lt_grid = P;
    } else {
      d.tt_sched = dev;
      d.tt_grid = P;
    }
  }
  return CNCPD_OK;
}

int upload_desc(cncpd_ctx* c) {
  CU(cudaMemcpyAsync(c->dd, &c->hd, sizeof(DevDesc), cudaMemcpyHostToDevice, c->stream));
  if (c->dd_als) CU(cudaMemcpyAsync(c->dd_als, &c->hd_als, sizeof(DevDesc), cudaMemcpyHostToDevice, c->stream));
  return CNCPD_OK;
}

int sync(cncpd_ctx* c) {
  CU(cudaStreamSynchronize(c->stream));
  return CNCPD_OK;
}

void destroy_graphs(cncpd_ctx* c) {
  for (auto& g : c->g_main) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  if (c->g_redo) cudaGraphExecDestroy(c->g_redo);
  c->g_redo = nullptr;
  if (c->g_plain) cudaGraphExecDestroy(c->g_plain);
  c->g_plain = nullptr;
  c->main_runs = c->redo_runs = c->prof_runs = c->timed_runs = 0;
}

// Copy the shared first L_n columns of block 0 into every other block (arena A).
int propagate_common(cncpd_ctx* c, char* arena) {
  for (int n = 0; n < c->N; ++n) {
    const int Ln = c->L[n];
    if (Ln == 0) continue;
    const char* src = arena + c->foff[n] * c->fsz;
    for (int k = 1; k < c->K; ++k) {
      char* dst = arena + c->foff[(size_t)k * c->N + n] * c->fsz;
      CU(cudaMemcpy2DAsync(dst, c->R[k] * c->fsz, src, c->R[0] * c->fsz, Ln * c->fsz, c->dim(0, n),
                           cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  return CNCPD_OK;
}

// ----------------------------------------------------------- the sweep -----

int record(cncpd_ctx* c, int which_ev) {
  if (!c->opts.profile || !c->rec_on) return CNCPD_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(c->stream, &cs));
  CU(cudaEventRecordWithFlags(c->ev[c->ev_set][which_ev], c->stream,
                              cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault));
  return CNCPD_OK;
}

// M^(n) for every block at the current factors of the other modes, given
// that the level-1 partial of n's group is current.
int enqueue_mode_m(cncpd_ctx* c, int n) {
  LaunchCfg lc{c->stream, c->num_sms};
  if (c->lra) {
    CU(launch_collapsed_m(lc, c->dd, c->hd, c->fp64, n));
    return CNCPD_OK;
  }
  const int gsize = (n < c->h) ? c->h : c->N - c->h;
  if (gsize > 1) CU(launch_level2(lc, c->dd, c->hd, c->fp64, c->RP, n));
  return CNCPD_OK;
}

int enqueue_trailing(cncpd_ctx* c, const DevDesc* dd, const DevDesc& hd, int RP) {
  LaunchCfg lc{c->stream, c->num_sms};
  if (hd.use_umma) CU(launch_split_factor(lc, dd, hd, 0));
  if (hd.use_tf32) CU(launch_split_factor_tf32(lc, dd, hd));
  TRY(record(c, 0));
  if (hd.use_umma) {
    CU(launch_trailing_umma(lc, dd, hd));
  } else if (hd.use_tf32) {
    CU(launch_trailing_tf32(lc, dd, hd));
  } else if (hd.use_tma) {
    CU(launch_trailing_tma(lc, dd, hd, RP, c->st));
    CU(launch_reduce_trail_splits(lc, dd, hd));
  } else {
    CU(launch_trailing_contract(lc, dd, hd, c->st, RP));
  }
  TRY(record(c, 1));
  return CNCPD_OK;
}

// with_reduce = 0: the split-K partials are left for the consumer to sum
// (the update of the last mode when the trailing group is that mode alone).
int enqueue_lead(cncpd_ctx* c, const DevDesc* dd, const DevDesc& hd, int RP, const int64_t* red_prefix,
                 int with_reduce = 1) {
  LaunchCfg lc{c->stream, c->num_sms};
  if (hd.use_umma) CU(launch_split_factor(lc, dd, hd, 1));
  TRY(record(c, 2));
  if (hd.use_umma) {
    CU(launch_lead_umma(lc, dd, hd));
    TRY(record(c, 3));
    if (with_reduce) CU(launch_reduce_splits(lc, hd, c->fp64));
  } else if (hd.use_tma) {
    CU(launch_lead_tma(lc, dd, hd, RP, c->st));
    TRY(record(c, 3));
    if (with_reduce) CU(launch_reduce_splits(lc, hd, c->fp64));
  } else {
    CU(launch_lead_contract(lc, dd, hd, c->st, RP, red_prefix, with_reduce));
    TRY(record(c, 3));
  }
  return CNCPD_OK;
}

// The sweep does the iteration bookkeeping inside its first Lipschitz launch
// (no separate k_iter_begin) on the tensor-pass path without a core tensor.
bool begin_in_sweep(const cncpd_ctx* c) { return !c->lra && !c->opts.use_core; }

// The lead pass of a third-order problem is the last mode's MTTKRP; the
// update of that mode sums its split-K partials itself.
bool fused_last_reduce(const cncpd_ctx* c) { return !c->lra && c->N - c->h == 1; }

// The update of the last mode also evaluates and publishes the objective
// (tensor-pass path, block-parallel update with room for the rows of M).
bool fused_objective(const cncpd_ctx* c) { return !c->lra && update_fuses_objective(c->hd, c->fp64, c->RP); }

// Mode of the Gram the first Lipschitz launch of a sweep sums from its
// chunks: with the fused objective and no cores, the last mode's Gram is
// left in chunks by its update (the objective does not need the sum).
int first_prev(const cncpd_ctx* c) { return (fused_objective(c) && !c->opts.use_core) ? c->N - 1 : -1; }

// Launch H / L of mode n (with the Gram of mode n-1) on the side stream so
// that it runs concurrently with the tensor pass enqueued next on the main
// stream; the main stream joins before the update of mode n.
int fork_lipschitz(cncpd_ctx* c, int n, int core, int begin) {
  LaunchCfg ls{c->side, c->num_sms};
  CU(cudaEventRecord(c->ev_fork, c->stream));
  CU(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  CU(launch_lipschitz(ls, c->dd, c->hd, c->fp64, n, core, n - 1, begin));
  CU(cudaEventRecord(c->ev_join, c->side));
  return CNCPD_OK;
}

// begin = 1: a main (not re-update) sweep, whose first Lipschitz launch
// also does the iteration bookkeeping when begin_in_sweep holds.
int enqueue_sweep(cncpd_ctx* c, int use_w, int begin) {
  LaunchCfg lc{c->stream, c->num_sms};
  const double dw = c->opts.delta_w;
  const int core = c->opts.use_core;
  const int fuse_reduce = fused_last_reduce(c);
  if (core) CU(launch_core_update(lc, c->dd, c->hd, use_w, dw));
  for (int n = 0; n < c->N; ++n) {
    const int beg = (n == 0 && begin && begin_in_sweep(c)) ? 1 : 0;
    if (!c->lra && n == 0) {
      // trailing pass alone on the GPU, then level 2 and H / L of mode 0 (with
      // the iteration bookkeeping) in one launch
      TRY(enqueue_trailing(c, c->dd, c->hd, c->RP));
      if (level2_is_pair(c->hd, n)) {
        CU(launch_mode_prep(lc, c->dd, c->hd, c->fp64, n, core, first_prev(c), 1, beg));
      } else {
        TRY(enqueue_mode_m(c, n));
        CU(launch_lipschitz(lc, c->dd, c->hd, c->fp64, n, core, first_prev(c), beg));
      }
    } else if (!c->lra && n == c->h) {
      // the lead pass needs the factors updated so far; H / L of mode h only
      // needs the Grams, which are final as well: run them side by side
      TRY(fork_lipschitz(c, n, core, 0));
      TRY(enqueue_lead(c, c->dd, c->hd, c->RP, c->d_red_prefix, fuse_reduce ? 0 : 1));
      if (level2_is_pair(c->hd, n)) CU(launch_mode_prep(lc, c->dd, c->hd, c->fp64, n, core, -1, 2));
      else TRY(enqueue_mode_m(c, n));
      CU(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    } else if (!c->lra && level2_is_pair(c->hd, n)) {
      // level 2 of mode n and H / L of mode n (with the Gram of mode n-1) in one launch
      CU(launch_mode_prep(lc, c->dd, c->hd, c->fp64, n, core, n - 1, 1));
    } else {
      TRY(enqueue_mode_m(c, n));
      CU(launch_lipschitz(lc, c->dd, c->hd, c->fp64, n, core, n - 1, beg));  // also the Gram of mode n-1
    }
    const int last = n == c->N - 1;
    CU(launch_update(lc, c->dd, c->hd, c->fp64, c->RP, n, use_w, dw, core, (fuse_reduce && last) ? 1 : 0,
                     (last && fused_objective(c)) ? 1 : 0));
    if (c->lra) CU(launch_cross_gram(lc, c->dd, c->hd, c->fp64, n, n + 1));
  }
  if (c->lra) {
    CU(launch_gram(lc, c->dd, c->hd, c->fp64, c->N - 1, c->N, 0));
    CU(launch_lra_objective(lc, c->dd, c->hd, c->fp64, core));
  } else if (!fused_objective(c)) {
    CU(launch_objective(lc, c->dd, c->hd, c->fp64, c->RP, 1, 1));
  }
  return CNCPD_OK;
}

int enqueue_readback(cncpd_ctx* c) {
  CU(cudaMemcpyAsync(c->hs, c->sc, sizeof(HostScalars), cudaMemcpyDeviceToHost, c->stream));
  return CNCPD_OK;
}

size_t arena_bytes(cncpd_ctx* c) { return c->arena_elems * c->fsz; }

// A bounded device-side wait gave up: clear the flag (so the handle can be
// used again after the caller's decision) and report it.
int timeout_error(cncpd_ctx* c) {
  cudaMemsetAsync(&c->sc->timeout, 0, sizeof(int), c->stream);
  cudaStreamSynchronize(c->stream);
  c->dirty = true;
  return set_err(CNCPD_ETIMEOUT, "a bounded device-side wait expired (pipeline stalled); iteration state discarded");
}

// The objective at the end of a sweep publishes F to the host mirror.
// (The snapshot S of U2 taken for a re-update is written by the update kernels.)
int enqueue_main(cncpd_ctx* c) {
  LaunchCfg lc{c->stream, c->num_sms};
  if (!begin_in_sweep(c)) CU(launch_iter_begin(lc, c->dd, c->hd, c->opts.use_core));
  return enqueue_sweep(c, 1, 1);
}

int enqueue_redo(cncpd_ctx* c) {
  LaunchCfg lc{c->stream, c->num_sms};
  CU(launch_redo_prepare(lc, c->dd, c->hd));
  CU(cudaMemcpyAsync(c->A1, c->A2, arena_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(c->A2, c->AS, arena_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  CU(launch_gram(lc, c->dd, c->hd, c->fp64, 0, c->N, 0));
  if (c->lra) CU(launch_cross_gram(lc, c->dd, c->hd, c->fp64, 0, c->N));
  return enqueue_sweep(c, 0, 0);
}

int capture(cncpd_ctx* c, int (*fn)(cncpd_ctx*), cudaGraphExec_t* out) {
  CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int r = fn(c);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (r != CNCPD_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return set_err(CNCPD_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return set_err(CNCPD_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return CNCPD_OK;
}

constexpr int PROFILE_EVERY = 8;

// The first replay of each kind runs eagerly (so that every kernel's
// attributes are set outside stream capture); later ones replay the graph.
// Timed main replays (every one without profiling, every PROFILE_EVERY-th
// with it) alternate between event sets 0 and 1; *set_used is the set, or
// -1 for a replay that records no events.
int run_main(cncpd_ctx* c, int* set_used) {
  if (c->opts.profile && c->prof_runs++ % PROFILE_EVERY != 0) {
    *set_used = -1;
    c->rec_on = false;
    int r = CNCPD_OK;
    if (c->opts.use_graph && c->main_runs++ > 0) {
      if (!c->g_plain) r = capture(c, enqueue_main, &c->g_plain);
      if (r == CNCPD_OK && cudaGraphLaunch(c->g_plain, c->stream) != cudaSuccess)
        r = set_err(CNCPD_ECUDA, "graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    } else {
      r = enqueue_main(c);
    }
    c->rec_on = true;
    return r;
  }
  const int set = c->timed_runs++ & 1;
  *set_used = set;
  c->ev_set = set;
  if (c->opts.use_graph && c->main_runs++ > 0) {
    if (!c->g_main[set]) TRY(capture(c, enqueue_main, &c->g_main[set]));
    CU(cudaGraphLaunch(c->g_main[set], c->stream));
    return CNCPD_OK;
  }
  return enqueue_main(c);
}

int run_redo(cncpd_ctx* c) {
  c->ev_set = 2;
  if (c->opts.use_graph && c->redo_runs++ > 0) {
    if (!c->g_redo) TRY(capture(c, enqueue_redo, &c->g_redo));
    CU(cudaGraphLaunch(c->g_redo, c->stream));
    return CNCPD_OK;
  }
  return enqueue_redo(c);
}

// Wait until the objective kernel has published a sequence number other than
// s0 to the host mirror.  The stream is queried now and then, so that a
// failed launch or a fault ends the wait; a bounded time limit guards
// against anything else.
int wait_published(cncpd_ctx* c, unsigned int s0) {
  const double t0 = now_s();
  for (unsigned long n = 1;; ++n) {
    if (c->hm->seq != s0) {
      std::atomic_thread_fence(std::memory_order_acquire);
      return CNCPD_OK;
    }
    if ((n & 255) == 0) {
      const cudaError_t e = cudaStreamQuery(c->stream);
      if (e == cudaSuccess) {
        if (c->hm->seq != s0) continue;
        return set_err(CNCPD_ECUDA, "the sweep finished without publishing its objective");
      }
      if (e != cudaErrorNotReady) return set_err(CNCPD_ECUDA, "sweep failed: %s", cudaGetErrorString(e));
      if (now_s() - t0 > 60.0) return set_err(CNCPD_ETIMEOUT, "a sweep did not finish within 60 s");
    }
  }
}

// Reset the iteration history (first iteration of Algorithm 1) and evaluate
// F(0) at the current factors.
int initialise(cncpd_ctx* c) {
  LaunchCfg lc{c->stream, c->num_sms};
  // U_{-1} := U_0 (reading R2)
  CU(cudaMemcpyAsync(c->A2, c->A1, arena_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  // scalars: t_0 = 1, no Lipschitz history, cores from lam_init
  std::vector<char> buf(sizeof(DevScalars), 0);
  DevScalars* s = reinterpret_cast<DevScalars*>(buf.data());
  s->t = 1.0;
  for (int k = 0; k < c->K; ++k) {
    s->xnorm2_orig[k] = c->xnorm2[k];
    s->xnorm2[k] = c->xnorm2[k];
    for (int r = 0; r < CNCPD_RMAX; ++r) {
      const double v = c->opts.use_core ? c->lam_init[(size_t)k * CNCPD_RMAX + r] : 1.0;
      s->lam1[k][r] = s->lam2[k][r] = s->lamS[k][r] = v;
    }
  }
  if (c->lra) {
    // ||X~||^2 is computed on the device; keep it.
    CU(cudaMemcpyAsync(c->hs, c->sc, sizeof(HostScalars), cudaMemcpyDeviceToHost, c->stream));
    std::vector<double> xt(c->K);
    CU(cudaMemcpyAsync(xt.data(), c->sc->xnorm2, sizeof(double) * c->K, cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    for (int k = 0; k < c->K; ++k) s->xnorm2[k] = xt[k];
  }
  for (int k = 0; k < c->K; ++k) {
    s->inv_xnorm2[k] = s->xnorm2[k] > 0.0 ? 1.0 / s->xnorm2[k] : 0.0;
    s->inv_xnorm2_orig[k] = s->xnorm2_orig[k] > 0.0 ? 1.0 / s->xnorm2_orig[k] : 0.0;
  }
  CU(cudaMemcpyAsync(c->sc, buf.data(), sizeof(DevScalars), cudaMemcpyHostToDevice, c->stream));
  CU(launch_gram(lc, c->dd, c->hd, c->fp64, 0, c->N, 0));
  const int n = c->N - 1;
  if (c->lra) {
    CU(launch_cross_gram(lc, c->dd, c->hd, c->fp64, 0, c->N));
    CU(launch_lra_objective(lc, c->dd, c->hd, c->fp64, c->opts.use_core));
  } else {
    TRY(enqueue_lead(c, c->dd, c->hd, c->RP, c->d_red_prefix));
    TRY(enqueue_mode_m(c, n));
    CU(launch_objective(lc, c->dd, c->hd, c->fp64, c->RP, 1, 0));
  }
  TRY(enqueue_readback(c));
  TRY(sync(c));
  if (c->hs->timeout) return timeout_error(c);
  if (c->hs->nonfinite || !std::isfinite(c->hs->F))
    return set_err(CNCPD_ENONFINITE, "initial objective is not finite (F = %g)", c->hs->F);
  c->F_prev = c->hs->F;
  c->rel_prev = c->hs->relerr;
  c->total_iters = 0;
  c->dirty = false;
  return CNCPD_OK;
}

double pass_bytes(cncpd_ctx* c) {
  double b = 0;
  const double es = c->st == ST_F64 ? 8 : c->st == ST_F32 ? 4 : c->st == ST_BF16 ? 2 : 4;
  for (int k = 0; k < c->K; ++k) {
    double n = 1;
    for (int m = 0; m < c->N; ++m) n *= (double)c->dim(k, m);
    b += n * es;
  }
  return b;
}

// Kernels launched by one main (redo = 0) or re-update (redo = 1) replay.
long long kernels_per_replay(cncpd_ctx* c, int redo) {
  long long n = c->opts.use_core ? 1 : 0;                 // core update
  if (!redo && !begin_in_sweep(c)) n += 1;                // iteration bookkeeping
  if (redo) n += 1 + 2 + (c->lra ? 2 : 0);                // restore, Grams (chunks + sums), cross Grams (same)
  if (!c->lra) n += 2 + (fused_last_reduce(c) ? 0 : 1);  // both tensor passes (+ split reduction)
  if (!c->lra && c->hd.use_umma) n += 2;                  // split factors of the tensor-core passes
  if (!c->lra && c->hd.use_tf32) n += 1;                  // TF32 parts of the trailing factor
  if (!c->lra && c->hd.trail_split) n += 1;               // column ranges of the trailing pass added up
  for (int m = 0; m < c->N; ++m) {
    n += 2;                                               // Lipschitz (alone or with level 2), update
    if (c->lra) {
      n += 3;                                             // collapsed M, cross Gram (chunks + sums)
    } else {
      const int gsize = (m < c->h) ? c->h : c->N - c->h;
      const bool forked = (m == c->h);
      if (gsize > 2 || (gsize == 2 && forked)) n += 1;   // level 2 in its own launch
    }
  }
  n += c->lra ? 3 : (fused_objective(c) ? 0 : 1);         // (last Gram: chunks + sums) + objective
  return n;
}

int read_profile(cncpd_ctx* c, cncpd_stats* st, int set) {
  if (!c->opts.profile || c->lra) return CNCPD_OK;
  float a = 0, b = 0;
  CU(cudaEventSynchronize(c->ev[set][3]));
  CU(cudaEventElapsedTime(&a, c->ev[set][0], c->ev[set][1]));
  CU(cudaEventElapsedTime(&b, c->ev[set][2], c->ev[set][3]));
  st->stream_ms += a + b;
  st->trail_ms += a;
  st->lead_ms += b;
  st->stream_launches += 2;
  return CNCPD_OK;
}

// Measured choice of the lead pass's split-K plan.  Every candidate (1, 2,
// 3, 4, 6 or 8 units per SM) is planned, its balanced unit list uploaded, and
// the pass alone (no split reduction) run once to warm up and then three
// times between CUDA events on the handle's stream; the fastest plan wins
// (ties: fewer units).  The winner is cached per problem shape for the
// process.  Runs before any graph is captured (graphs bake in the plan).
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;

std::string shape_key(const cncpd_ctx* c) {
  std::string k = std::to_string(c->st) + "/" + std::to_string(c->fp64) + "/" + std::to_string(c->num_sms) + "/" +
                  std::to_string(c->hd.use_umma) + "/" + std::to_string(c->RP);
  for (int b = 0; b < c->K; ++b) {
    k += ";" + std::to_string(c->R[b]);
    for (int n = 0; n < c->N; ++n) k += "," + std::to_string(c->dim(b, n));
  }
  return k;
}

int apply_lead_plan(cncpd_ctx* c, int mult) {
  size_t pel = 0;
  plan_lead_units(c, c->hd, c->RP, c->fp64, (int64_t)c->num_sms * mult, &pel);
  if (pel > c->partial_cap) return set_err(CNCPD_ESTATE, "lead plan exceeds the partial-sum buffer");
  TRY(plan_tma_schedules(c, c->hd));
  TRY(upload_desc(c));
  c->lead_mult = mult;
  return CNCPD_OK;
}

int tune_lead(cncpd_ctx* c) {
  c->lead_tuned = true;
  if (!c->opts.autotune || c->lra || (!c->hd.use_tma && !c->hd.use_umma)) return CNCPD_OK;
  const std::string key = shape_key(c);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return apply_lead_plan(c, it->second);
  }
  destroy_graphs(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  int best = c->lead_mult;
  float best_ms = -1.f;
  int rc = CNCPD_OK;
  for (int mult : kLeadMults) {
    size_t pel = 0;
    DevDesc probe = c->hd;
    plan_lead_units(c, probe, c->RP, c->fp64, (int64_t)c->num_sms * mult, &pel);
    if (pel > c->partial_cap) continue;
    rc = apply_lead_plan(c, mult);
    if (rc != CNCPD_OK) break;
    float ms = 0.f;
    for (int rep = 0; rep < 4 && rc == CNCPD_OK; ++rep) {
      if (rep == 1 && cudaEventRecord(e0, c->stream) != cudaSuccess) rc = set_err(CNCPD_ECUDA, "event record failed");
      if (rc == CNCPD_OK) rc = enqueue_lead(c, c->dd, c->hd, c->RP, c->d_red_prefix, 0);
    }
    if (rc != CNCPD_OK) break;
    if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = set_err(CNCPD_ECUDA, "autotune timing failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    if (c->hs && c->sc) {  // a pass that timed out must not win
      rc = enqueue_readback(c);
      if (rc == CNCPD_OK) rc = sync(c);
      if (rc == CNCPD_OK && c->hs->timeout) {
        rc = timeout_error(c);
        break;
      }
    }
    if (best_ms < 0.f || ms < best_ms * 0.995f) {
      best_ms = ms;
      best = mult;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TRY(rc);
  TRY(apply_lead_plan(c, best));
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  return CNCPD_OK;
}

int need_resident_x(const cncpd_ctx* c) {
  if (c->opts.stream_x && !c->lra)
    return set_err(CNCPD_ESTATE, "opts.stream_x keeps one block of X on the device: run cncpd_lra first "
                                 "(only the lraCoNCPD-APG iterations run without X)");
  return CNCPD_OK;
}

int run_iterations(cncpd_ctx* c, int n_iters, bool use_eps, cncpd_stats* out) {
  TRY(need_resident_x(c));
  cncpd_stats st{};
  const double t0 = now_s();
  if (!c->lead_tuned) TRY(tune_lead(c));
  if (c->dirty) TRY(initialise(c));
  const double pb = c->lra ? 0.0 : 2.0 * pass_bytes(c);
  c->prof_runs = 0;  // the first sweep of every call records its pass times
  int pending = -1;  // event set of a main replay whose pass times are not read yet
  for (int it = 0; it < n_iters; ++it) {
    const unsigned int s0 = c->hm->seq;
    int set = -1;
    TRY(run_main(c, &set));
    // the previous timed iteration's pass times, read while this one runs
    if (set >= 0) {
      if (pending >= 0) TRY(read_profile(c, &st, pending));
      pending = set;
    }
    TRY(wait_published(c, s0));
    st.x_bytes += pb;
    st.launches += kernels_per_replay(c, 0);
    double F = c->hm->F;
    const bool redo = c->opts.reupdate && (F - c->F_prev) > c->tie_tol * std::fabs(c->F_prev);
    if (redo) {
      const unsigned int s1 = c->hm->seq;
      TRY(run_redo(c));
      TRY(wait_published(c, s1));
      TRY(read_profile(c, &st, 2));
      st.x_bytes += pb;
      st.launches += kernels_per_replay(c, 1);
      F = c->hm->F;
      st.reupdates++;
    }
    const int timeout = c->hm->timeout;
    const int nonfinite = c->hm->nonfinite;
    if (timeout) {
      TRY(sync(c));
      return timeout_error(c);
    }
    if (nonfinite || !std::isfinite(F)) {
      TRY(sync(c));
      return set_err(CNCPD_ENONFINITE, "objective or Lipschitz constant not finite at iteration %d",
                     c->total_iters + 1);
    }
    const double rel = c->hm->relerr;
    c->total_iters++;
    st.iters++;
    c->F_prev = F;
    const bool stop = use_eps && std::fabs(rel - c->rel_prev) < c->opts.eps;
    c->rel_prev = rel;
    if (stop) {
      st.converged = 1;
      break;
    }
  }
  TRY(sync(c));
  if (pending >= 0) TRY(read_profile(c, &st, pending));
  st.total_iters = c->total_iters;
  st.lead_plan = c->lead_mult;
  st.lead_plan_tuned = (c->opts.autotune && c->lead_mult > 0) ? 1 : 0;
  st.trail_tensor_cores = (c->hd.use_umma || c->hd.use_tf32) ? 1 : 0;
  st.trail_ranges = 1;
  for (int k = 0; k < c->K; ++k) st.trail_ranges = std::max(st.trail_ranges, c->hd.lt_js[k]);
  st.F = c->F_prev;
  st.relerr = c->rel_prev;
  st.fit = 1.0 - c->rel_prev;
  st.seconds = now_s() - t0;
  if (out) *out = st;
  return CNCPD_OK;
}

// M^(n) for every mode at the current factors (no updates in between):
// both level-1 contractions, then level 2.  Used by the gradient, the
// MTTKRP hook and the global fit.
int all_modes_m(cncpd_ctx* c) {
  LaunchCfg lc{c->stream, c->num_sms};
  TRY(enqueue_trailing(c, c->dd, c->hd, c->RP));
  TRY(enqueue_lead(c, c->dd, c->hd, c->RP, c->d_red_prefix));
  for (int n = 0; n < c->N; ++n) {
    const int gsize = (n < c->h) ? c->h : c->N - c->h;
    if (gsize > 1) CU(launch_level2(lc, c->dd, c->hd, c->fp64, c->RP, n));
  }
  return CNCPD_OK;
}

// opts.stream_x: make the window hold block k's stored values (quantised
// from the caller's tensor: in place when it is device or page-locked
// memory, else through the staging buffer).
int load_block(cncpd_ctx* c, int k) {
  if (c->window_block == k) return CNCPD_OK;
  const DevDesc& d = c->hd;
  const size_t xes = (c->st == ST_F64) ? 8 : (c->st == ST_F32) ? 4 : 2;
  const int64_t ne = d.lead_rows[k] * d.trail_cols[k];
  const int64_t nstore = d.lead_rows[k] * d.pitch[k];
  if (d.pitch[k] != d.trail_cols[k]) {
    CU(cudaMemsetAsync(c->window, 0, nstore * xes, c->stream));
    if (c->window_lo) CU(cudaMemsetAsync(c->window_lo, 0, nstore * xes, c->stream));
  }
  const void* src = c->xsrc[k];
  const size_t ses = c->x_src_f64 ? 8 : 4;
  cudaPointerAttributes pa;
  bool on_dev = false;
  if (cudaPointerGetAttributes(&pa, src) == cudaSuccess) {
    on_dev = (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
      src = pa.devicePointer;
      on_dev = true;
    }
  } else {
    cudaGetLastError();
  }
  if (!on_dev) {
    if (!c->xstage) {
      int64_t maxel = 0;
      for (int b = 0; b < c->K; ++b) maxel = std::max(maxel, d.lead_rows[b] * d.trail_cols[b]);
      TRY(dalloc(c, &c->xstage, maxel * ses));
    }
    CU(cudaMemcpyAsync(c->xstage, src, ne * ses, cudaMemcpyHostToDevice, c->stream));
    src = c->xstage;
  }
  CU(launch_quantize(c->stream, src, c->x_src_f64, c->window, c->window_lo, c->st, d.lead_rows[k], d.trail_cols[k],
                     d.pitch[k], c->wnorm, c->wscratch, 1024));
  c->window_block = k;
  return CNCPD_OK;
}

// A copy of `full` whose tensor-pass unit lists cover only the blocks with
// active[k] set (the balanced per-CTA lists number every block's units, so
// they are dropped unless every block is active).
DevDesc restrict_units(const DevDesc& full, const int* active) {
  DevDesc aa = full;
  int nact = 0;
  aa.lt_prefix[0] = aa.tt_prefix[0] = 0;
  for (int k = 0; k < full.K; ++k) {
    nact += active[k] ? 1 : 0;
    aa.lt_prefix[k + 1] = aa.lt_prefix[k] + (active[k] ? full.lt_prefix[k + 1] - full.lt_prefix[k] : 0);
    aa.tt_prefix[k + 1] = aa.tt_prefix[k] + (active[k] ? full.tt_prefix[k + 1] - full.tt_prefix[k] : 0);
  }
  if (nact < full.K) aa.lt_sched = aa.tt_sched = nullptr;
  return aa;
}

int check_handle(cncpd_t h) {
  if (!h) return set_err(CNCPD_EINVAL, "null handle");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return set_err(CNCPD_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return CNCPD_OK;
}

int copy_matrix_out(cncpd_ctx* c, const void* src, int src_f64, int64_t n, void* dst, cncpd_dtype dt) {
  if (dt != CNCPD_F64 && dt != CNCPD_F32) return set_err(CNCPD_EINVAL, "output dtype must be F64 or F32");
  const int dst_f64 = dt == CNCPD_F64;
  if (dst_f64 == src_f64) {
    CU(cudaMemcpyAsync(dst, src, n * (src_f64 ? 8 : 4), cudaMemcpyDefault, c->stream));
  } else {
    void* tmp = nullptr;
    CU(cudaMallocAsync(&tmp, n * (dst_f64 ? 8 : 4) + 16, c->stream));
    CU(launch_convert(c->stream, src, src_f64, tmp, dst_f64, n));
    CU(cudaMemcpyAsync(dst, tmp, n * (dst_f64 ? 8 : 4), cudaMemcpyDefault, c->stream));
    CU(cudaFreeAsync(tmp, c->stream));
  }
  return sync(c);
}

}  // namespace

// =============================================================== C ABI ====

extern "C" {

void cncpd_default_opts(cncpd_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->eps = 1e-8;
  o->max_it = 1000;
  o->lra_eps = 1e-4;
  o->lra_max_it = 200;
  o->delta_w = 0.9999;
  o->use_core = 0;
  o->reupdate = 1;
  o->storage = -1;
  o->use_graph = 1;
  o->profile = 0;
  o->tensor_cores = 1;
  o->autotune = 1;
}

const char* cncpd_last_error(void) { return g_err.c_str(); }

void cncpd_destroy(cncpd_t h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  destroy_graphs(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->hs) cudaFreeHost(h->hs);
  if (h->hm) cudaFreeHost(h->hm);
  for (auto& set : h->ev)
    for (auto& e : set)
      if (e) cudaEventDestroy(e);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int cncpd_create(cncpd_t* out, int K, int N, const int64_t* dims, const void* const* X, cncpd_dtype x_dtype,
                 const int* R, const int* L, const unsigned char* nonneg, const cncpd_opts* opts, void* stream) {
  g_err.clear();
  if (!out) return set_err(CNCPD_EINVAL, "out is NULL");
  *out = nullptr;
  if (K < 1 || K > CNCPD_KMAX) return set_err(CNCPD_EINVAL, "K = %d outside 1..%d", K, CNCPD_KMAX);
  if (N < 3 || N > CNCPD_NMAX) return set_err(CNCPD_EINVAL, "N = %d outside 3..%d", N, CNCPD_NMAX);
  if (!dims || !X || !R || !L) return set_err(CNCPD_EINVAL, "dims, X, R and L are required");
  if (x_dtype != CNCPD_F64 && x_dtype != CNCPD_F32) return set_err(CNCPD_EINVAL, "x_dtype must be F64 or F32");
  int minR = 1 << 30;
  for (int k = 0; k < K; ++k) {
    if (R[k] < 1 || R[k] > CNCPD_RMAX) return set_err(CNCPD_EINVAL, "R[%d] = %d outside 1..%d", k, R[k], CNCPD_RMAX);
    minR = std::min(minR, R[k]);
    if (!X[k]) return set_err(CNCPD_EINVAL, "X[%d] is NULL", k);
    for (int n = 0; n < N; ++n)
      if (dims[(size_t)k * N + n] < 1) return set_err(CNCPD_EINVAL, "dims[%d][%d] < 1", k, n);
  }
  for (int n = 0; n < N; ++n) {
    if (L[n] < 0 || L[n] > minR)
      return set_err(CNCPD_EINVAL, "L[%d] = %d outside 0..min_k R_k = %d", n, L[n], minR);
    if (L[n] > 0)
      for (int k = 1; k < K; ++k)
        if (dims[(size_t)k * N + n] != dims[n])
          return set_err(CNCPD_EINVAL, "coupled mode %d has different sizes across blocks", n);
  }
  cncpd_opts o;
  if (opts) o = *opts;
  else cncpd_default_opts(&o);
  int st = o.storage < 0 ? (x_dtype == CNCPD_F64 ? ST_F64 : ST_F32) : o.storage;
  if (st < 0 || st > 3) return set_err(CNCPD_EINVAL, "bad storage type %d", o.storage);
  if (o.delta_w <= 0 || o.delta_w >= 1.0) return set_err(CNCPD_EINVAL, "delta_w must be in (0, 1)");

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return set_err(CNCPD_ECUDA, "no CUDA device: %s", cudaGetErrorString(ce));

  cncpd_ctx* c = new cncpd_ctx();
  c->device = dev;
  c->K = K;
  c->N = N;
  c->h = (N + 1) / 2;
  c->dims.assign(dims, dims + (size_t)K * N);
  c->R.assign(R, R + K);
  c->L.assign(L, L + N);
  c->nonneg.assign(N, 1);
  if (nonneg)
    for (int n = 0; n < N; ++n) c->nonneg[n] = nonneg[n] ? 1 : 0;
  c->Rmax = *std::max_element(c->R.begin(), c->R.end());
  c->RP = rank_bucket(c->Rmax);
  c->opts = o;
  c->st = st;
  c->fp64 = (st == ST_F64);
  c->tie_tol = c->fp64 ? 1e-13 : 1e-6;
  c->fsz = c->fp64 ? 8 : 4;
  c->lam_init.assign((size_t)K * CNCPD_RMAX, 1.0);
  c->xnorm2.assign(K, 0.0);

  auto fail = [&](int code) {
    std::string msg = g_err;
    cncpd_destroy(c);
    g_err = msg;
    return code;
  };
#define CTRY(expr)                 \
  do {                             \
    int _r = (expr);               \
    if (_r != CNCPD_OK) return fail(_r); \
  } while (0)
#define CCU(expr)                                                                                   \
  do {                                                                                              \
    cudaError_t _e = (expr);                                                                        \
    if (_e != cudaSuccess) return fail(set_err(CNCPD_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e))); \
  } while (0)

  CCU(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
  CCU(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  CCU(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  CCU(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CCU(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CCU(cudaMallocHost((void**)&c->hs, sizeof(HostScalars)));
  CCU(cudaHostAlloc((void**)&c->hm, sizeof(HostMirror), cudaHostAllocMapped));
  std::memset((void*)c->hm, 0, sizeof(HostMirror));
  CCU(cudaHostGetDevicePointer((void**)&c->hm_dev, c->hm, 0));
  for (auto& set : c->ev)
    for (auto& e : set) CCU(cudaEventCreate(&e));
  // order after the caller's stream
  if (stream) {
    cudaEvent_t ev;
    CCU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CCU(cudaEventRecord(ev, (cudaStream_t)stream));
    CCU(cudaStreamWaitEvent(c->stream, ev, 0));
    cudaEventDestroy(ev);
  } else {
    CCU(cudaStreamSynchronize(0));
  }

  DevDesc& d = c->hd;
  std::memset(&d, 0, sizeof d);
  d.K = K;
  d.N = N;
  d.h = c->h;
  d.Rmax = c->Rmax;
  for (int k = 0; k < K; ++k) {
    d.R[k] = R[k];
    int64_t lr = 1, tc = 1;
    for (int n = 0; n < N; ++n) {
      d.dims[k][n] = c->dim(k, n);
      if (n < c->h) lr *= c->dim(k, n);
      else tc *= c->dim(k, n);
    }
    d.lead_rows[k] = lr;
    d.trail_cols[k] = tc;
    if (lr * R[k] >= (1LL << 31) || tc * R[k] >= (1LL << 31)) {
      std::string msg = "block too large for the two-level tree (level-1 partial above 2^31 entries)";
      cncpd_destroy(c);
      return set_err(CNCPD_EINVAL, "%s", msg.c_str());
    }
  }
  for (int n = 0; n < N; ++n) {
    d.L[n] = c->L[n];
    d.nonneg[n] = c->nonneg[n];
  }

  // --- X: quantise into library storage
  const size_t xes = (st == ST_F64) ? 8 : (st == ST_F32) ? 4 : 2;
  const int src_f64 = x_dtype == CNCPD_F64;
  const size_t ses = src_f64 ? 8 : 4;
  int64_t maxel = 0;
  for (int k = 0; k < K; ++k) maxel = std::max(maxel, d.lead_rows[k] * d.trail_cols[k]);
  void* stage = nullptr;
  double* nscratch = nullptr;
  double* nout = nullptr;
  const int nblk = 1024;
  CTRY(dalloc(c, (void**)&nscratch, nblk * sizeof(double)));
  CTRY(dalloc(c, (void**)&nout, CNCPD_KMAX * sizeof(double)));
  const bool streamed = c->opts.stream_x != 0;
  if (streamed) {
    // one window for the largest stored block (and its lo plane)
    size_t wmax = 0;
    for (int k = 0; k < K; ++k) {
      d.pitch[k] = (d.trail_cols[k] + 15) / 16 * 16;
      wmax = std::max(wmax, (size_t)(d.lead_rows[k] * d.pitch[k]) * xes);
    }
    c->window_bytes = wmax;
    CTRY(dalloc(c, &c->window, wmax));
    if (st == ST_BF16X2) CTRY(dalloc(c, &c->window_lo, wmax));
    c->xsrc.assign(X, X + K);
    c->x_src_f64 = src_f64;
    CTRY(dalloc(c, (void**)&c->wscratch, nblk * sizeof(double)));
    CTRY(dalloc(c, (void**)&c->wnorm, sizeof(double)));
  }
  for (int k = 0; k < K; ++k) {
    const int64_t ne = d.lead_rows[k] * d.trail_cols[k];
    const int64_t pitch = (d.trail_cols[k] + 15) / 16 * 16;  // rows start on 64-byte (FP32) boundaries
    d.pitch[k] = pitch;
    const int64_t nstore = d.lead_rows[k] * pitch;
    void* xb = nullptr;
    void* xlo = nullptr;
    if (streamed) {
      // every block's stored values go through the window (here for ||X||^2)
      xb = c->window;
      xlo = c->window_lo;
      if (pitch != d.trail_cols[k]) {
        CCU(cudaMemsetAsync(xb, 0, nstore * xes, c->stream));
        if (xlo) CCU(cudaMemsetAsync(xlo, 0, nstore * xes, c->stream));
      }
    } else {
      CTRY(dalloc(c, &xb, nstore * xes));
      if (pitch != d.trail_cols[k]) CCU(cudaMemsetAsync(xb, 0, nstore * xes, c->stream));
      if (st == ST_BF16X2) {
        CTRY(dalloc(c, &xlo, nstore * xes));
        if (pitch != d.trail_cols[k]) CCU(cudaMemsetAsync(xlo, 0, nstore * xes, c->stream));
      }
    }
    const void* src = X[k];
    cudaPointerAttributes pa;
    bool on_dev = false;
    if (cudaPointerGetAttributes(&pa, src) == cudaSuccess) {
      on_dev = (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
      // page-locked host memory is mapped into the device's address space:
      // the quantising kernel reads it in place (no staging copy)
      if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
        src = pa.devicePointer;
        on_dev = true;
      }
    } else {
      cudaGetLastError();
    }
    if (!on_dev) {
      if (!stage) CTRY(dalloc(c, &stage, maxel * ses));
      CCU(cudaMemcpyAsync(stage, src, ne * ses, cudaMemcpyHostToDevice, c->stream));
      src = stage;
    }
    CCU(launch_quantize(c->stream, src, src_f64, xb, xlo, st, d.lead_rows[k], d.trail_cols[k], pitch, nout + k,
                        nscratch, nblk));
    d.X[k] = xb;
    d.Xlo[k] = xlo;
    if (streamed) c->window_block = k;
  }
  if (streamed && stage) c->xstage = stage;
  CCU(cudaMemcpyAsync(c->xnorm2.data(), nout, K * sizeof(double), cudaMemcpyDeviceToHost, c->stream));

  // --- factor arenas
  c->foff.resize((size_t)K * N);
  size_t off = 0;
  for (int k = 0; k < K; ++k)
    for (int n = 0; n < N; ++n) {
      c->foff[(size_t)k * N + n] = off;
      off += ((size_t)c->dim(k, n) * R[k] + 31) / 32 * 32;
    }
  c->arena_elems = off;
  // 64 elements of slack past the last factor: kernels read factor rows as
  // whole 16-byte vectors up to the padded rank
  CTRY(dalloc(c, (void**)&c->A1, (off + 64) * c->fsz));
  CTRY(dalloc(c, (void**)&c->A2, (off + 64) * c->fsz));
  CTRY(dalloc(c, (void**)&c->AS, (off + 64) * c->fsz));
  const size_t rr = (size_t)c->Rmax * c->Rmax;
  CTRY(dalloc(c, (void**)&d.Gbase, (size_t)K * N * rr * sizeof(double)));
  CTRY(dalloc(c, &d.Hbase, (size_t)K * rr * c->fsz));
  CTRY(dalloc(c, (void**)&d.H64base, (size_t)K * rr * sizeof(double)));
  for (int n = 0; n < N; ++n) {
    int64_t imax = 0;
    for (int k = 0; k < K; ++k) imax = std::max<int64_t>(imax, c->dim(k, n));
    d.gr[n] = gram_chunk_rows(c->RP, K, imax, c->fp64);
    d.gnc[n] = (int)((imax + d.gr[n] - 1) / d.gr[n]);
    CTRY(dalloc(c, &d.Gp[n], (size_t)K * d.gnc[n] * rr * c->fsz));
  }
  // per-CTA <M, U_new> sums of the objective fused into the last update
  CTRY(dalloc(c, &d.dotp, (size_t)d.gnc[N - 1] * K * c->RP * c->fsz));
  CTRY(dalloc(c, (void**)&d.xxp, (size_t)d.gnc[N - 1] * K * sizeof(double)));
  for (int k = 0; k < K; ++k)
    for (int n = 0; n < N; ++n) {
      d.U1[k][n] = c->U1p(k, n);
      d.U2[k][n] = c->U2p(k, n);
      void* m = nullptr;
      CTRY(dalloc(c, &m, (size_t)c->dim(k, n) * R[k] * c->fsz));
      d.M[k][n] = m;
      d.G[k][n] = d.Gbase + ((size_t)k * N + n) * rr;
    }
  for (int k = 0; k < K; ++k) {
    void* p = nullptr;
    CTRY(dalloc(c, &p, (size_t)d.lead_rows[k] * R[k] * c->fsz));
    d.Pl[k] = p;
    if (N - c->h == 1) {
      d.Pt[k] = d.M[k][N - 1];  // the lead contraction is the last mode's MTTKRP
    } else {
      CTRY(dalloc(c, &p, (size_t)d.trail_cols[k] * R[k] * c->fsz));
      d.Pt[k] = p;
    }
    d.H[k] = static_cast<char*>(d.Hbase) + (size_t)k * rr * c->fsz;
  }
  // TMA descriptors of X for the FP32 / BF16 kernels (two box shapes per
  // block: 256 rows x 128 bytes, swizzled, for the trailing pass; 256 columns
  // x 32 KiB for the lead pass)
  if ((st == ST_F32 || st == ST_BF16) && tensor_map_encoder()) {
    std::vector<CUtensorMap> maps(2 * CNCPD_KMAX);
    bool ok = true;
    const int esz = st == ST_BF16 ? 2 : 4;
    for (int k = 0; k < K && ok; ++k) {
      ok = encode_map(&maps[k], d.X[k], st, d.lead_rows[k], d.trail_cols[k], d.pitch[k], 128 / esz, 256,
                      CU_TENSOR_MAP_SWIZZLE_128B) &&
           encode_map(&maps[CNCPD_KMAX + k], d.X[k], st, d.lead_rows[k], d.trail_cols[k], d.pitch[k], 256,
                      lead_tma_rows(st), CU_TENSOR_MAP_SWIZZLE_NONE);
    }
    if (ok) {
      CUtensorMap* dm = nullptr;
      CTRY(dalloc(c, (void**)&dm, maps.size() * sizeof(CUtensorMap)));
      CCU(cudaMemcpyAsync(dm, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream));
      d.tmap_trail = dm;
      d.tmap_lead = dm + CNCPD_KMAX;
    }
  }
  d.use_tma = (d.tmap_trail != nullptr) && tma_rank_supported(c->RP);
  CTRY(setup_umma(c, d, c->Rmax));
  CTRY(setup_tf32(c, d, c->Rmax));
  size_t pel = 0;
  c->lead_mult = plan_lead_splits(c, d, c->RP, c->fp64, &pel);
  const size_t plp = choose_trailing_plan(c, d, 1);
  if (plp) CTRY(dalloc(c, &d.Pl_part, plp * sizeof(float)));
  CTRY(plan_tma_schedules(c, d));
  c->partial_cap = std::max(pel, lead_partial_cap(c, d, c->RP, c->fp64));
  CTRY(dalloc(c, &d.partial, c->partial_cap * c->fsz));

  {
    std::vector<int64_t> pre(K + 1, 0);
    for (int k = 0; k < K; ++k) pre[k + 1] = pre[k] + d.trail_cols[k] * R[k];
    CTRY(dalloc(c, (void**)&c->d_red_prefix, (K + 1) * sizeof(int64_t)));
    CCU(cudaMemcpyAsync(c->d_red_prefix, pre.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    CCU(cudaStreamSynchronize(c->stream));
  }
  CTRY(dalloc(c, (void**)&c->sc, sizeof(DevScalars)));
  CTRY(dalloc(c, (void**)&d.err, sizeof(int)));
  CCU(cudaMemsetAsync(d.err, 0, sizeof(int), c->stream));
  d.sc = c->sc;
  d.hm = c->hm_dev;
  d.A1base = c->A1;
  d.ASbase = c->AS;
  CTRY(dalloc(c, (void**)&c->dd, sizeof(DevDesc)));
  CTRY(upload_desc(c));

  // default initial factors: Uniform[0,1] (Section IV), shared columns from block 0
  for (int k = 0; k < K; ++k)
    for (int n = 0; n < N; ++n)
      CCU(launch_uniform_init(c->stream, c->U1p(k, n), c->fp64, (int64_t)c->dim(k, n) * R[k],
                              0x5eedULL * 1000003ULL + (uint64_t)(k * CNCPD_NMAX + n)));
  CTRY(propagate_common(c, c->A1));
  CCU(cudaStreamSynchronize(c->stream));
  c->dirty = true;
  *out = c;
#undef CTRY
#undef CCU
  return CNCPD_OK;
}

}  // extern "C"

namespace {

// Write U^(n,k) (host or device, F64 or F32) into the current-iterate arena;
// the shared first L_n columns only from block 0 (copied to every block).
int write_factor(cncpd_t h, int k, int n, const void* U, cncpd_dtype dtype) {
  if (k < 0 || k >= h->K || n < 0 || n >= h->N || !U) return set_err(CNCPD_EINVAL, "bad block/mode or NULL data");
  if (dtype != CNCPD_F64 && dtype != CNCPD_F32) return set_err(CNCPD_EINVAL, "factor dtype must be F64 or F32");
  const int64_t I = h->dim(k, n);
  const int R = h->R[k];
  const int src_f64 = dtype == CNCPD_F64;
  const size_t ses = src_f64 ? 8 : 4;
  void* tmp = nullptr;
  CU(cudaMallocAsync(&tmp, I * R * ses + 16, h->stream));
  CU(cudaMemcpyAsync(tmp, U, I * R * ses, cudaMemcpyDefault, h->stream));
  void* conv = tmp;
  void* tmp2 = nullptr;
  if (src_f64 != h->fp64) {
    CU(cudaMallocAsync(&tmp2, I * R * h->fsz + 16, h->stream));
    CU(launch_convert(h->stream, tmp, src_f64, tmp2, h->fp64, I * R));
    conv = tmp2;
  }
  const int Ln = h->L[n];
  char* dst = (char*)h->U1p(k, n);
  if (k == 0 || Ln == 0) {
    CU(cudaMemcpyAsync(dst, conv, I * R * h->fsz, cudaMemcpyDeviceToDevice, h->stream));
  } else if (Ln < R) {
    CU(cudaMemcpy2DAsync(dst + Ln * h->fsz, R * h->fsz, (char*)conv + Ln * h->fsz, R * h->fsz, (R - Ln) * h->fsz, I,
                         cudaMemcpyDeviceToDevice, h->stream));
  }
  if (k == 0) TRY(propagate_common(h, h->A1));
  CU(cudaFreeAsync(tmp, h->stream));
  if (tmp2) CU(cudaFreeAsync(tmp2, h->stream));
  return CNCPD_OK;
}

// Objective and gradient at the factors in the current-iterate arena (no
// extrapolation); gradients into host or device memory.
int eval_objective_grad(cncpd_t h, double* F, void* const* gradU, void* const* gradC, cncpd_dtype dtype) {
  LaunchCfg lc{h->stream, h->num_sms};
  CU(launch_gram(lc, h->dd, h->hd, h->fp64, 0, h->N, 0));
  if (h->lra) {
    CU(launch_cross_gram(lc, h->dd, h->hd, h->fp64, 0, h->N));
    CU(launch_lra_objective(lc, h->dd, h->hd, h->fp64, h->opts.use_core));
    for (int n = 0; n < h->N; ++n) CU(launch_collapsed_m(lc, h->dd, h->hd, h->fp64, n));
  } else {
    TRY(all_modes_m(h));
    CU(launch_objective(lc, h->dd, h->hd, h->fp64, h->RP, 1, 0));
  }
  TRY(enqueue_readback(h));
  TRY(sync(h));
  if (F) *F = h->hs->F;
  const int dst_f64 = dtype == CNCPD_F64;
  for (int n = 0; n < h->N; ++n) {
    CU(launch_grad(lc, h->dd, h->hd, h->fp64, h->RP, n, h->opts.use_core));
    if (gradU)
      for (int k = 0; k < h->K; ++k)
        if (gradU[(size_t)k * h->N + n])
          TRY(copy_matrix_out(h, h->hd.M[k][n], h->fp64, h->dim(k, n) * h->R[k], gradU[(size_t)k * h->N + n], dtype));
    if (gradC && gradC[n] && h->L[n] > 0) {
      const size_t bytes = (size_t)h->dim(0, n) * h->L[n] * (dst_f64 ? 8 : 4);
      void* tmp = nullptr;
      CU(cudaMallocAsync(&tmp, bytes + 16, h->stream));
      CU(launch_common_grad(h->stream, h->dd, h->hd, h->fp64, n, tmp, dst_f64));
      CU(cudaMemcpyAsync(gradC[n], tmp, bytes, cudaMemcpyDefault, h->stream));
      CU(cudaFreeAsync(tmp, h->stream));
    }
    TRY(sync(h));
  }
  return CNCPD_OK;
}

// Bytes of DevScalars that describe the solver state: everything before the
// publish sequence number, which must keep counting up so that the host's
// wait for the next objective sees a new value.
constexpr size_t kStateScalarBytes = offsetof(DevScalars, seq);

}  // namespace

extern "C" {

int cncpd_set_factors(cncpd_t h, int k, int n, const void* U, cncpd_dtype dtype) {
  TRY(check_handle(h));
  TRY(write_factor(h, k, n, U, dtype));
  TRY(sync(h));
  h->dirty = true;
  return CNCPD_OK;
}

int cncpd_set_factors_all(cncpd_t h, const void* const* U, cncpd_dtype dtype) {
  TRY(check_handle(h));
  if (!U) return set_err(CNCPD_EINVAL, "U is NULL");
  for (int k = 0; k < h->K; ++k)
    for (int n = 0; n < h->N; ++n) TRY(write_factor(h, k, n, U[(size_t)k * h->N + n], dtype));
  TRY(sync(h));
  h->dirty = true;
  return CNCPD_OK;
}

int cncpd_set_core(cncpd_t h, int k, const double* lambda) {
  TRY(check_handle(h));
  if (k < 0 || k >= h->K || !lambda) return set_err(CNCPD_EINVAL, "bad block or NULL lambda");
  for (int r = 0; r < h->R[k]; ++r) {
    if (!(lambda[r] >= 0.0)) return set_err(CNCPD_EINVAL, "core entries must be >= 0");
    h->lam_init[(size_t)k * CNCPD_RMAX + r] = lambda[r];
  }
  h->dirty = true;
  return CNCPD_OK;
}

int cncpd_step(cncpd_t h, int n_iters, cncpd_stats* out) {
  TRY(check_handle(h));
  if (n_iters < 0) return set_err(CNCPD_EINVAL, "n_iters < 0");
  return run_iterations(h, n_iters, false, out);
}

int cncpd_fit(cncpd_t h, cncpd_stats* out) {
  TRY(check_handle(h));
  return run_iterations(h, h->opts.max_it, true, out);
}

int cncpd_factors(cncpd_t h, int k, int n, void* dst, cncpd_dtype dtype) {
  TRY(check_handle(h));
  if (k < 0 || k >= h->K || n < 0 || n >= h->N || !dst) return set_err(CNCPD_EINVAL, "bad block/mode or NULL dst");
  return copy_matrix_out(h, h->U1p(k, n), h->fp64, h->dim(k, n) * h->R[k], dst, dtype);
}

int cncpd_core(cncpd_t h, int k, double* lambda) {
  TRY(check_handle(h));
  if (k < 0 || k >= h->K || !lambda) return set_err(CNCPD_EINVAL, "bad block or NULL lambda");
  if (h->dirty) {
    for (int r = 0; r < h->R[k]; ++r)
      lambda[r] = h->opts.use_core ? h->lam_init[(size_t)k * CNCPD_RMAX + r] : 1.0;
    return CNCPD_OK;
  }
  CU(cudaMemcpyAsync(lambda, h->sc->lam1[k], h->R[k] * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return sync(h);
}

int cncpd_mttkrp(cncpd_t h, int k, int n, void* dst, cncpd_dtype dtype) {
  TRY(check_handle(h));
  if (k < 0 || k >= h->K || n < 0 || n >= h->N || !dst) return set_err(CNCPD_EINVAL, "bad block/mode or NULL dst");
  TRY(need_resident_x(h));
  if (h->lra) {
    LaunchCfg lc{h->stream, h->num_sms};
    CU(launch_cross_gram(lc, h->dd, h->hd, h->fp64, 0, h->N));
    CU(launch_collapsed_m(lc, h->dd, h->hd, h->fp64, n));
  } else {
    TRY(all_modes_m(h));
  }
  return copy_matrix_out(h, h->hd.M[k][n], h->fp64, h->dim(k, n) * h->R[k], dst, dtype);
}

int cncpd_objective_grad(cncpd_t h, double* F, void* const* gradU, void* const* gradC, cncpd_dtype dtype) {
  TRY(check_handle(h));
  TRY(need_resident_x(h));
  if (dtype != CNCPD_F64 && dtype != CNCPD_F32) return set_err(CNCPD_EINVAL, "dtype must be F64 or F32");
  if (h->dirty) TRY(initialise(h));
  return eval_objective_grad(h, F, gradU, gradC, dtype);
}

int cncpd_objective_grad_at(cncpd_t h, const void* const* U, cncpd_dtype udtype, double* F, void* const* gradU,
                            void* const* gradC, cncpd_dtype dtype) {
  TRY(check_handle(h));
  TRY(need_resident_x(h));
  if (!U) return set_err(CNCPD_EINVAL, "U is NULL");
  if (dtype != CNCPD_F64 && dtype != CNCPD_F32) return set_err(CNCPD_EINVAL, "dtype must be F64 or F32");
  if (h->dirty) TRY(initialise(h));
  const size_t ab = arena_bytes(h);
  if (!h->A_eval) TRY(dalloc(h, (void**)&h->A_eval, ab));
  if (!h->sc_eval) TRY(dalloc(h, (void**)&h->sc_eval, kStateScalarBytes));
  // keep the current iterate and solver scalars; evaluate at U; put them back
  CU(cudaMemcpyAsync(h->A_eval, h->A1, ab, cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->sc_eval, h->sc, kStateScalarBytes, cudaMemcpyDeviceToDevice, h->stream));
  int r = CNCPD_OK;
  for (int k = 0; k < h->K && r == CNCPD_OK; ++k)
    for (int n = 0; n < h->N && r == CNCPD_OK; ++n) r = write_factor(h, k, n, U[(size_t)k * h->N + n], udtype);
  if (r == CNCPD_OK) r = eval_objective_grad(h, F, gradU, gradC, dtype);
  const std::string msg = g_err;
  CU(cudaMemcpyAsync(h->A1, h->A_eval, ab, cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->sc, h->sc_eval, kStateScalarBytes, cudaMemcpyDeviceToDevice, h->stream));
  LaunchCfg lc{h->stream, h->num_sms};
  CU(launch_gram(lc, h->dd, h->hd, h->fp64, 0, h->N, 0));
  if (h->lra) CU(launch_cross_gram(lc, h->dd, h->hd, h->fp64, 0, h->N));
  TRY(sync(h));
  if (r != CNCPD_OK) g_err = msg;
  return r;
}

int cncpd_global_fit(cncpd_t h, double* fit) {
  TRY(check_handle(h));
  if (!fit) return set_err(CNCPD_EINVAL, "fit is NULL");
  if (h->dirty) TRY(initialise(h));
  LaunchCfg lc{h->stream, h->num_sms};
  const bool was_lra = h->lra;
  h->lra = false;
  CU(launch_gram(lc, h->dd, h->hd, h->fp64, 0, h->N, 0));
  int r = CNCPD_OK;
  if (h->opts.stream_x) {
    // one block at a time through the window: its lead pass alone (the
    // split-K sums of the other blocks are formed from their own partials)
    if (!h->dd_tmp) r = dalloc(h, (void**)&h->dd_tmp, sizeof(DevDesc));
    std::vector<int> one(CNCPD_KMAX, 0);
    for (int k = 0; k < h->K && r == CNCPD_OK; ++k) {
      r = load_block(h, k);
      if (r != CNCPD_OK) break;
      std::fill(one.begin(), one.end(), 0);
      one[k] = 1;
      const DevDesc t = restrict_units(h->hd, one.data());
      cudaError_t e = cudaMemcpyAsync(h->dd_tmp, &t, sizeof(DevDesc), cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) r = set_err(CNCPD_ECUDA, "%s", cudaGetErrorString(e));
      if (r == CNCPD_OK) r = enqueue_lead(h, h->dd_tmp, t, h->RP, h->d_red_prefix);
      // the descriptor copy must not change before the kernels have read it
      if (r == CNCPD_OK) r = sync(h);
    }
  } else {
    r = enqueue_lead(h, h->dd, h->hd, h->RP, h->d_red_prefix);
  }
  if (r == CNCPD_OK) r = enqueue_mode_m(h, h->N - 1);
  h->lra = was_lra;
  TRY(r);
  CU(launch_objective(lc, h->dd, h->hd, h->fp64, h->RP, 0, 0));
  std::vector<double> rel(h->K);
  CU(cudaMemcpyAsync(rel.data(), h->sc->out_relk, h->K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  TRY(sync(h));
  double s = 0;
  for (double v : rel) s += v;
  *fit = 1.0 - s / h->K;
  return CNCPD_OK;
}

int cncpd_lipschitz(const double* H, int R, double* lmax) {
  g_err.clear();
  if (!H || !lmax || R < 1 || R > CNCPD_RMAX) return set_err(CNCPD_EINVAL, "bad arguments");
  double* d = nullptr;
  CU(cudaMalloc(&d, (size_t)(R * R + 1) * sizeof(double)));
  cudaError_t e = cudaMemcpy(d, H, (size_t)R * R * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_lmax_host(d, R, d + R * R, 0);
  if (e == cudaSuccess) e = cudaMemcpy(lmax, d + R * R, sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return set_err(CNCPD_ECUDA, "lipschitz: %s", cudaGetErrorString(e));
  return CNCPD_OK;
}

int cncpd_check_wait_timeout(cncpd_t h, double limit_ms) {
  g_err.clear();
  TRY(check_handle(h));
  if (!(limit_ms >= 0.001 && limit_ms <= 2000.0)) return set_err(CNCPD_EINVAL, "limit_ms must be in [0.001, 2000]");
  cncpd_ctx* c = h;
  TRY(sync(c));
  CU(launch_wait_selftest(c->stream, &c->sc->timeout, (uint64_t)(limit_ms * 1e6)));
  TRY(enqueue_readback(c));
  TRY(sync(c));
  if (c->hs->timeout) return timeout_error(c);
  return set_err(CNCPD_ECUDA, "the self-test wait completed although nothing arrived on its barrier");
}

// ------------------------------------------------------------- LRA -------

int cncpd_lra(cncpd_t h, const int* R_tilde, const void* const* Ut0, cncpd_dtype dtype, cncpd_stats* out) {
  TRY(check_handle(h));
  if (h->lra) return set_err(CNCPD_ESTATE, "cncpd_lra already ran on this handle");
  if (!R_tilde) return set_err(CNCPD_EINVAL, "R_tilde is NULL");
  if (Ut0 && dtype != CNCPD_F64 && dtype != CNCPD_F32) return set_err(CNCPD_EINVAL, "Ut0 dtype must be F64 or F32");
  const double t0 = now_s();
  const int K = h->K, N = h->N;
  h->Rt.assign(R_tilde, R_tilde + K);
  int rtmax = 0;
  for (int k = 0; k < K; ++k) {
    if (R_tilde[k] < 1 || R_tilde[k] > CNCPD_RMAX) return set_err(CNCPD_EINVAL, "R_tilde[%d] outside 1..64", k);
    rtmax = std::max(rtmax, R_tilde[k]);
    h->hd.Rt[k] = R_tilde[k];
  }
  h->RPt = rank_bucket(rtmax);
  DevDesc& a = h->hd_als;
  a = h->hd;
  a.Rmax = rtmax;
  // ALS Grams are formed by one CTA per factor (no chunk partials, no arenas)
  a.Gbase = nullptr;
  a.Hbase = nullptr;
  a.H64base = nullptr;
  for (int n = 0; n < N; ++n) {
    a.Gp[n] = nullptr;
    a.gr[n] = a.gnc[n] = 0;
  }
  for (int k = 0; k < K; ++k) {
    a.R[k] = a.Rt[k] = R_tilde[k];
    for (int n = 0; n < N; ++n) {
      void* u = nullptr;
      TRY(dalloc(h, &u, ((size_t)h->dim(k, n) * R_tilde[k] + 64) * h->fsz));  // slack for whole-row reads
      h->hd.Ut[k][n] = a.Ut[k][n] = a.U1[k][n] = u;
      a.U2[k][n] = nullptr;
      double* g = nullptr;
      TRY(dalloc(h, (void**)&g, (size_t)R_tilde[k] * R_tilde[k] * sizeof(double)));
      h->hd.Gt[k][n] = a.Gt[k][n] = a.G[k][n] = g;
      TRY(dalloc(h, (void**)&g, (size_t)R_tilde[k] * h->R[k] * sizeof(double)));
      h->hd.C[k][n] = a.C[k][n] = g;
      void* m = nullptr;
      TRY(dalloc(h, &m, (size_t)h->dim(k, n) * R_tilde[k] * h->fsz));
      a.M[k][n] = m;
    }
    void* p = nullptr;
    TRY(dalloc(h, &p, (size_t)a.lead_rows[k] * R_tilde[k] * h->fsz));
    a.Pl[k] = p;
    if (N - h->h == 1) {
      a.Pt[k] = a.M[k][N - 1];
    } else {
      TRY(dalloc(h, &p, (size_t)a.trail_cols[k] * R_tilde[k] * h->fsz));
      a.Pt[k] = p;
    }
    TRY(dalloc(h, &p, (size_t)R_tilde[k] * R_tilde[k] * h->fsz));
    h->hd.Vinv[k] = a.Vinv[k] = p;
  }
  // chunk values of the cross Grams (main descriptor only)
  h->hd.cld = rtmax * h->hd.Rmax;
  for (int n = 0; n < N; ++n) {
    int64_t imax = 0;
    for (int k = 0; k < K; ++k) imax = std::max<int64_t>(imax, h->dim(k, n));
    h->hd.cgnc[n] = (int)((imax + CROSS_ROWS - 1) / CROSS_ROWS);
    TRY(dalloc(h, &h->hd.Cp[n], (size_t)K * h->hd.cgnc[n] * h->hd.cld * h->fsz));
  }
  size_t pel = 0;
  a.use_tma = (a.tmap_trail != nullptr) && tma_rank_supported(h->RPt);
  TRY(setup_umma(h, a, rtmax));
  TRY(setup_tf32(h, a, rtmax));
  (void)plan_lead_splits(h, a, h->RPt, h->fp64, &pel);
  (void)plan_trailing_tiles(a, h->num_sms, h->st, 0);
  TRY(plan_tma_schedules(h, a));
  TRY(dalloc(h, &a.partial, pel * h->fsz));
  std::vector<int64_t> pre(K + 1, 0);
  for (int k = 0; k < K; ++k) pre[k + 1] = pre[k] + a.trail_cols[k] * R_tilde[k];
  TRY(dalloc(h, (void**)&h->d_red_prefix_als, (K + 1) * sizeof(int64_t)));
  TRY(dalloc(h, (void**)&h->d_active, CNCPD_KMAX * sizeof(int)));
  TRY(dalloc(h, (void**)&h->d_status, CNCPD_KMAX * sizeof(int)));
  TRY(dalloc(h, (void**)&h->d_relk, CNCPD_KMAX * sizeof(double)));
  TRY(dalloc(h, (void**)&h->dd_als, sizeof(DevDesc)));
  CU(cudaMemcpyAsync(h->d_red_prefix_als, pre.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  // initial ALS factors
  for (int k = 0; k < K; ++k)
    for (int n = 0; n < N; ++n) {
      const int64_t ne = h->dim(k, n) * R_tilde[k];
      if (Ut0 && Ut0[(size_t)k * N + n]) {
        void* tmp = nullptr;
        const int src_f64 = dtype == CNCPD_F64;
        CU(cudaMallocAsync(&tmp, ne * (src_f64 ? 8 : 4) + 16, h->stream));
        CU(cudaMemcpyAsync(tmp, Ut0[(size_t)k * N + n], ne * (src_f64 ? 8 : 4), cudaMemcpyDefault, h->stream));
        CU(launch_convert(h->stream, tmp, src_f64, a.Ut[k][n], h->fp64, ne));
        CU(cudaFreeAsync(tmp, h->stream));
      } else {
        CU(launch_uniform_init(h->stream, a.Ut[k][n], h->fp64, ne, 0x1a5eedULL * 7919ULL + (uint64_t)(k * CNCPD_NMAX + n)));
      }
    }
  // ||X||^2 of the stored tensors for the ALS relative error
  {
    std::vector<char> buf(sizeof(DevScalars), 0);
    DevScalars* s = reinterpret_cast<DevScalars*>(buf.data());
    for (int k = 0; k < K; ++k) s->xnorm2_orig[k] = s->xnorm2[k] = h->xnorm2[k];
    CU(cudaMemcpyAsync(h->sc->xnorm2_orig, s->xnorm2_orig, sizeof(double) * CNCPD_KMAX, cudaMemcpyHostToDevice,
                       h->stream));
  }
  TRY(upload_desc(h));
  LaunchCfg lc{h->stream, h->num_sms};
  CU(launch_gram(lc, h->dd_als, h->hd_als, h->fp64, 0, N, 0));
  std::vector<int> active(CNCPD_KMAX, 0), sweeps(K, 0);
  std::vector<double> rel_prev(K, -1.0), rel(K, 0.0);
  const DevDesc full = h->hd_als;
  // The blocks' ALS runs are independent.  With X resident they run together;
  // with opts.stream_x one block at a time, each with its tensor in the window.
  const bool streamed = h->opts.stream_x != 0;
  for (int g0 = 0; g0 < K; g0 = streamed ? g0 + 1 : K) {
    const int g1 = streamed ? g0 + 1 : K;
    if (streamed) TRY(load_block(h, g0));
    std::fill(active.begin(), active.end(), 0);
    for (int k = g0; k < g1; ++k) active[k] = 1;
    // relative error of the initial factors, from M^(N-1) at those factors
    h->hd_als = restrict_units(full, active.data());
    CU(cudaMemcpyAsync(h->dd_als, &h->hd_als, sizeof(DevDesc), cudaMemcpyHostToDevice, h->stream));
    TRY(enqueue_lead(h, h->dd_als, h->hd_als, h->RPt, h->d_red_prefix_als));
    if (N - h->h > 1) CU(launch_level2(lc, h->dd_als, h->hd_als, h->fp64, h->RPt, N - 1));
    CU(launch_als_relerr(lc, h->dd_als, h->hd_als, h->fp64, h->d_relk));
    {
      std::vector<double> r0(K, 0.0);
      CU(cudaMemcpyAsync(r0.data(), h->d_relk, K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      TRY(sync(h));
      for (int k = g0; k < g1; ++k) rel_prev[k] = r0[k];
    }
    for (int s = 1; s <= h->opts.lra_max_it; ++s) {
      int nact = 0;
      for (int k = 0; k < K; ++k) nact += active[k];
      if (nact == 0) break;
      // only active blocks stream X
      h->hd_als = restrict_units(full, active.data());
      CU(cudaMemcpyAsync(h->dd_als, &h->hd_als, sizeof(DevDesc), cudaMemcpyHostToDevice, h->stream));
      CU(cudaMemcpyAsync(h->d_active, active.data(), CNCPD_KMAX * sizeof(int), cudaMemcpyHostToDevice, h->stream));
      CU(cudaMemsetAsync(h->d_status, 0, CNCPD_KMAX * sizeof(int), h->stream));
      for (int n = 0; n < N; ++n) {
        if (n == 0) TRY(enqueue_trailing(h, h->dd_als, h->hd_als, h->RPt));
        if (n == h->h) TRY(enqueue_lead(h, h->dd_als, h->hd_als, h->RPt, h->d_red_prefix_als));
        const int gsize = (n < h->h) ? h->h : N - h->h;
        if (gsize > 1) CU(launch_level2(lc, h->dd_als, h->hd_als, h->fp64, h->RPt, n));
        CU(launch_als_solve(lc, h->dd_als, h->hd_als, h->fp64, n, h->d_active, h->d_status));
        CU(launch_als_apply(lc, h->dd_als, h->hd_als, h->fp64, n, h->d_active));
        CU(launch_gram(lc, h->dd_als, h->hd_als, h->fp64, n, n + 1, 0));
      }
      CU(launch_als_relerr(lc, h->dd_als, h->hd_als, h->fp64, h->d_relk));
      std::vector<int> status(K, 0);
      CU(cudaMemcpyAsync(rel.data(), h->d_relk, K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CU(cudaMemcpyAsync(status.data(), h->d_status, K * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      TRY(sync(h));
      for (int k = 0; k < K; ++k) {
        if (!active[k]) continue;
        if (status[k]) return set_err(CNCPD_ESINGULAR, "ALS normal matrix of block %d not positive definite", k);
        sweeps[k] = s;
        if (std::fabs(rel[k] - rel_prev[k]) < h->opts.lra_eps) active[k] = 0;
        rel_prev[k] = rel[k];
      }
    }
  }
  h->hd_als = full;
  // switch to the collapsed products; ||X~||^2 for the objective of Eq. cosfunclra
  h->hd.lra = 1;
  h->lra = true;
  destroy_graphs(h);
  TRY(upload_desc(h));
  CU(launch_gram(lc, h->dd, h->hd, h->fp64, 0, N, 1));
  CU(launch_lra_xnorm(lc, h->dd, h->hd));
  TRY(sync(h));
  h->dirty = true;
  if (out) {
    cncpd_stats st{};
    st.lra_sweeps = *std::max_element(sweeps.begin(), sweeps.end());
    double m = 0;
    for (double v : rel_prev) m += v;
    st.lra_relerr = m / K;
    st.seconds = now_s() - t0;
    *out = st;
  }
  return CNCPD_OK;
}

int cncpd_lra_factors(cncpd_t h, int k, int n, void* dst, cncpd_dtype dtype) {
  TRY(check_handle(h));
  if (!h->lra) return set_err(CNCPD_ESTATE, "cncpd_lra has not run");
  if (k < 0 || k >= h->K || n < 0 || n >= h->N || !dst) return set_err(CNCPD_EINVAL, "bad block/mode or NULL dst");
  return copy_matrix_out(h, h->hd.Ut[k][n], h->fp64, h->dim(k, n) * h->Rt[k], dst, dtype);
}

// ------------------------------------------------------- checkpoint -------

struct BlobHeader {
  char magic[8];
  int K, N, fp64, lra;
  int total_iters, pad;
  double F_prev, rel_prev;
  uint64_t arena_bytes, scalars_bytes;
};

int cncpd_save_state(cncpd_t h, void** blob, size_t* nbytes) {
  TRY(check_handle(h));
  if (!blob || !nbytes) return set_err(CNCPD_EINVAL, "NULL output");
  if (h->dirty) TRY(initialise(h));
  const size_t ab = arena_bytes(h);
  const size_t total = sizeof(BlobHeader) + 2 * ab + sizeof(DevScalars);
  char* p = (char*)std::malloc(total);
  if (!p) return set_err(CNCPD_ENOMEM, "host malloc failed");
  BlobHeader hdr{};
  std::memcpy(hdr.magic, "CNCPDst1", 8);
  hdr.K = h->K;
  hdr.N = h->N;
  hdr.fp64 = h->fp64;
  hdr.lra = h->lra;
  hdr.total_iters = h->total_iters;
  hdr.F_prev = h->F_prev;
  hdr.rel_prev = h->rel_prev;
  hdr.arena_bytes = ab;
  hdr.scalars_bytes = sizeof(DevScalars);
  std::memcpy(p, &hdr, sizeof hdr);
  cudaError_t e = cudaMemcpyAsync(p + sizeof hdr, h->A1, ab, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + sizeof hdr + ab, h->A2, ab, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + sizeof hdr + 2 * ab, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::free(p);
    return set_err(CNCPD_ECUDA, "save_state: %s", cudaGetErrorString(e));
  }
  *blob = p;
  *nbytes = total;
  return CNCPD_OK;
}

int cncpd_load_state(cncpd_t h, const void* blob, size_t nbytes) {
  TRY(check_handle(h));
  if (!blob || nbytes < sizeof(BlobHeader)) return set_err(CNCPD_EINVAL, "blob too small");
  BlobHeader hdr;
  std::memcpy(&hdr, blob, sizeof hdr);
  const size_t ab = arena_bytes(h);
  if (std::memcmp(hdr.magic, "CNCPDst1", 8) != 0 || hdr.K != h->K || hdr.N != h->N || hdr.fp64 != h->fp64 ||
      hdr.lra != (int)h->lra || hdr.arena_bytes != ab || hdr.scalars_bytes != sizeof(DevScalars) ||
      nbytes != sizeof(BlobHeader) + 2 * ab + sizeof(DevScalars))
    return set_err(CNCPD_EINVAL, "blob does not match this problem");
  const char* p = (const char*)blob + sizeof hdr;
  CU(cudaMemcpyAsync(h->A1, p, ab, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(h->A2, p + ab, ab, cudaMemcpyHostToDevice, h->stream));
  // the publish sequence number keeps its current value (see kStateScalarBytes)
  CU(cudaMemcpyAsync(h->sc, p + 2 * ab, kStateScalarBytes, cudaMemcpyHostToDevice, h->stream));
  LaunchCfg lc{h->stream, h->num_sms};
  CU(launch_gram(lc, h->dd, h->hd, h->fp64, 0, h->N, 0));
  if (h->lra) CU(launch_cross_gram(lc, h->dd, h->hd, h->fp64, 0, h->N));
  TRY(sync(h));
  h->total_iters = hdr.total_iters;
  h->F_prev = hdr.F_prev;
  h->rel_prev = hdr.rel_prev;
  h->dirty = false;
  return CNCPD_OK;
}

void cncpd_free_blob(void* blob) { std::free(blob); }

}  // extern "C"
