// lst_api.cu -- C-ABI and runtime of the GB300 LST library: context, resident geometry and
// network, per-event device buffers (event slots), the one-launch-per-stage pipeline over
// a batch of events, a CUDA-graph cache for batched runs, and candidate export.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lst_internal.cuh"

namespace lstk {
// kernels (lst_kernels.cu, lst_score.cu, lst_mma.cu)
__global__ void k_reset(const EvDesc *, DevGeom);
__global__ void k_bin_count(const EvDesc *, int, DevGeom);
__global__ void k_bin_scan(const EvDesc *, DevGeom);
__global__ void k_bin_scatter(const EvDesc *, int, DevGeom);
__global__ void k_md(const EvDesc *, int, DevGeom, lst_cuts);
__global__ void k_md_scan(const EvDesc *, DevGeom);
__global__ void k_md_scatter(const EvDesc *, int);
__global__ void k_md_sort(const EvDesc *, int);
__global__ void k_ls(const EvDesc *, int, DevGeom, lst_cuts, int *, const int32_t *, int, int);
__global__ void k_ls_scan(const EvDesc *);
__global__ void k_ls_scatter(const EvDesc *, int);
__global__ void k_t3(const EvDesc *, int, lst_cuts, int *, int);
__global__ void k_t3_scan(const EvDesc *);
__global__ void k_t3_scatter(const EvDesc *, int);
__global__ void k_t5(const EvDesc *, int, lst_cuts);
__global__ void k_score_fp32(const EvDesc *, int, DevGeom, lst_cuts, const float *, int);
__global__ void k_features(const EvDesc *, DevGeom, float, float *, int);
__global__ void k_score_feat_fp32(const float *, int64_t, const float *, int, float *);
__global__ void k_gather(const EvDesc *, int, int, int32_t *, float *, uint8_t *);
__global__ void k_collect(const EvDesc *, int, int *);
__global__ void k_tc_count(const EvDesc *, int);
__global__ void k_tc_scan(const EvDesc *);
__global__ void k_tc_scatter(const EvDesc *, int);
__global__ void k_tc_decide(const EvDesc *, int);
__global__ void k_gather_tc(const EvDesc *, int, int *, int32_t *, float *, uint8_t *, int64_t);
__global__ void k_graph_rows(const EvDesc *, int, int32_t *);
__global__ void k_graph_fill(const EvDesc *, DevGeom, int, const int32_t *, int32_t *, float *, float *);
cudaError_t launch_score_bf16_events(int, cudaStream_t, const EvDesc *, int, DevGeom, lst_cuts, const uint16_t *,
                                     const float *, int, int *, long long, bool split, int skip_mma);
cudaError_t launch_score_bf16_features(int, cudaStream_t, DevGeom, lst_cuts, const uint16_t *, const float *, int,
                                       const float *, int64_t, float *, int *, long long, bool split, int skip_mma);
int score_bf16_blocks_per_sm(bool split);
cudaError_t pix_launch_bin(const PixDesc *, int, bool, int, cudaStream_t);
cudaError_t pix_launch_rebin(const PixDesc *, int, bool, int, cudaStream_t);
cudaError_t pix_launch_stage_begin(const PixDesc *, int, int, cudaStream_t);
cudaError_t pix_launch_round(const EvDesc *, const PixDesc *, int, int, lst_pixel_cuts, int, int *, cudaStream_t);
cudaError_t pix_launch_mark(const EvDesc *, const PixDesc *, int, int, cudaStream_t);
cudaError_t pix_launch_rows(const EvDesc *, const PixDesc *, int, int, cudaStream_t);
void pack_weights_bf16(const float *wflat, int n_hidden, uint16_t *out);
}  // namespace lstk

using namespace lstk;

namespace {

thread_local std::string g_err;

lst_status fail(lst_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) {                                                              \
      return fail(_e == cudaErrorMemoryAllocation ? LST_ERR_NOMEM : LST_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(_e));                     \
    }                                                                                     \
  } while (0)

// NVTX ranges (domain "lst") around the public calls and, while a launch sequence is
// enqueued, around each stage's launches, so that a profiler attributes kernels to steps
// (ncu --nvtx --nvtx-include). Without a tool attached the NVTX calls return at once.
nvtxDomainHandle_t nvtx_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("lst");
  return d;
}
void nvtx_push(const char *name) {
  nvtxEventAttributes_t a{};
  a.version = NVTX_VERSION;
  a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  a.messageType = NVTX_MESSAGE_TYPE_ASCII;
  a.message.ascii = name;
  nvtxDomainRangePushEx(nvtx_domain(), &a);
}
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtx_push(name); }
  ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
};
// consecutive stage ranges of one launch sequence; the open one closes on scope exit
struct NvtxStages {
  bool open = false;
  void next(const char *name) {
    if (open) nvtxDomainRangePop(nvtx_domain());
    open = name != nullptr;
    if (open) nvtx_push(name);
  }
  ~NvtxStages() { next(nullptr); }
};
const char *const STAGE_NAMES[LST_N_STAGES] = {"hit grouping", "step 1: MD", "step 2: LS", "LS grouping",
                                               "step 3: T3", "step 4: T5", "T5-DNN score", "track candidates"};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Slot {
  EvDesc d{};
  void *mem = nullptr;
  size_t bytes = 0;
  int64_t hit_cap = 0;
  int md_cap = 0, ls_cap = 0, t3_cap = 0, t5_cap = 0;
  void *in_mem = nullptr;          // staging for host inputs
  int64_t in_cap = 0;
  bool mem_pooled = false, in_pooled = false;  // mem / in_mem came from the context's pool
  void *pix_mem = nullptr;         // pixel-seed matching (lst_match_pixel_seeds)
  size_t pix_bytes = 0;
  int64_t pix_rows = -1;           // its track candidates, -1 before a matching
  const int32_t *pix_rows_ptr = nullptr;  // where they are (in pix_mem)
  bool busy = false;
  int lane = -1;                   // lane whose last batch holds this slot's counters
  int lane_pos = -1;
  uint64_t lane_gen = 0;
  int32_t cnt[C_NCOUNTERS] = {0};  // harvested counters
  bool have_cnt = false;
  int64_t n_hits = 0;
};

// Batches of lst_run_batch in flight at once: the lanes are taken round robin and a launch
// on a lane first waits for that lane's previous batch, so a caller that keeps two earlier
// batches pending while the third runs leaves the GPU a full batch of slack.
constexpr int BATCH_LANES = 3;

struct Lane {
  EvDesc *d_desc = nullptr;        // [MAX_EVENTS]
  EvDesc *h_desc = nullptr;        // pinned
  int *d_work = nullptr;           // [16]
  int *d_counts = nullptr;         // [MAX_EVENTS * C_NCOUNTERS]
  int *h_counts = nullptr;         // pinned
  int slots[MAX_EVENTS];
  int n = 0;
  uint64_t gen = 0;
  bool inflight = false;
  cudaEvent_t done = nullptr;
  cudaEvent_t tev[LST_N_STAGES + 1] = {};  // stage boundaries of the last launch (when timed)
  bool timed = false;
  cudaStream_t cap_stream = nullptr;
  std::map<long long, cudaGraphExec_t> graphs;
};

}  // namespace

struct lst_ctx_s {
  int device = 0;
  lst_config cfg{};
  int n_sm = 0;
  bool have_geom = false;
  DevGeom g{};
  int8_t *d_subdet = nullptr, *d_layer = nullptr;
  int32_t *d_map_off = nullptr, *d_map_tgt = nullptr;
  int32_t *d_ls_units = nullptr;  // [n_mod + 1] prefix of step-2 units per module for small launches
  int ls_units_per_event = 0;
  lst_cuts cuts{};
  int n_hidden = 2;
  float *d_w = nullptr;
  int n_w = 0;
  uint16_t *d_wpack = nullptr;   // BF16 weights in the tensor-core operand layout
  int *d_err = nullptr;          // device error word (bounded waits of the tensor-core kernel)
  long long wait_limit = 1ll << 26;
  int skip_mma = 0;                // test aid: the tensor-core score kernels issue no MMA
  std::atomic<int> fail_allocs{0};  // test aid: that many event-buffer allocations fail next
  int grid_bf[2] = {0, 0};   // tensor-core score grid: plain BF16, split BF16
  std::vector<Slot> slots;
  std::vector<Lane> lanes;     // lane 0: lst_run_event; lanes 1..: batches, round robin
  int next_lane = 1;
  float r_md, r_ls, r_t3, r_t5;
  // launch shapes (autotuned)
  int md_threads = 256, md_buf = 128;
  int ls_threads = 128, ls_list = 1024;
  int t3_threads = 256;
  int t3_mds = 0;                  // step-3 unit size in middle MDs; 0: chosen per launch
  int t5_threads = 256;
  int sc_threads = 256;
  int grid_md = 0, grid_ls = 0, grid_t3 = 0, grid_t5 = 0, grid_sc = 0;
  // grids of the 256-thread grid-stride kernels: as many CTAs as are resident at once (an
  // event-major loop must not leave a second wave of CTAs to redo every event)
  int grid_bin_count = 0, grid_bin_scatter = 0, grid_md_scatter = 0, grid_md_sort = 0, grid_ls_scatter = 0,
      grid_t3_scatter = 0;
  int grid_tc_count = 0, grid_tc_scatter = 0, grid_tc_decide = 0;
  // per-stage device times accumulated over timed launches
  bool timing = false;
  double stage_sum[LST_N_STAGES] = {0};
  int64_t stage_n = 0;
  cudaStream_t aux = nullptr;
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  // event-slot buffers and input staging of the serving workers: stream-ordered allocations
  // from a pool of the context that keeps its memory, so that a slot grows without waiting
  // for the device
  cudaMemPool_t pool = nullptr;
};

struct lst_event_s {
  lst_ctx ctx;
  int slot;
  int status;
};

namespace {

constexpr int LS_WARP_BYTES = 5456;     // sizeof(LsWarp): each warp's targets, inner MDs and pair queue
constexpr int LS_SMALL_TB = 8;          // target modules per step-2 unit in small launches
size_t ls_smem(const lst_ctx_s *c) { return (size_t)(c->ls_threads / 32) * LS_WARP_BYTES; }
size_t md_smem(const lst_ctx_s *c) { return (size_t)(c->md_threads / 32) * (512 + 3 * 128 + 2 * 256); }
size_t t3_smem(const lst_ctx_s *c) { return (size_t)(c->t3_threads / 32) * 6288; }   // sizeof(T3Warp)
size_t t5_smem(const lst_ctx_s *c) { return (size_t)(c->t5_threads / 32) * (4 * 128 + 3 * 512); }
int mlp_floats_host(int nh) { return NHID * NFEAT + NHID + (nh - 1) * (NHID * NHID + NHID) + NHID + 1; }

lst_status compute_grids(lst_ctx_s *c) {
  // Function attributes are process-wide (shared by every context): allow the device's
  // opt-in maximum once, so that no context's launch shape limits another's.
  int optin = 0;
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  auto allow = [&](const void *fn) -> cudaError_t {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
  };
  CU(allow((const void *)k_ls));
  CU(allow((const void *)k_md));
  CU(allow((const void *)k_t3));
  CU(allow((const void *)k_t5));
  CU(allow((const void *)k_score_fp32));
  CU(allow((const void *)k_score_feat_fp32));
  int occ = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ls, c->ls_threads, ls_smem(c)));
  c->grid_ls = std::max(1, occ) * c->n_sm;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_md, c->md_threads, md_smem(c)));
  c->grid_md = std::max(1, occ) * c->n_sm;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_t3, c->t3_threads, t3_smem(c)));
  c->grid_t3 = std::max(1, occ) * c->n_sm;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_t5, c->t5_threads, t5_smem(c)));
  c->grid_t5 = std::max(1, occ) * c->n_sm;
  const size_t sw = (size_t)mlp_floats_host(4) * 4;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_score_fp32, c->sc_threads, sw));
  c->grid_sc = std::max(1, occ) * c->n_sm;
  auto resident = [&](const void *fn, int &grid) -> cudaError_t {
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, 256, 0);
    grid = std::max(1, o) * c->n_sm;
    return e;
  };
  CU(resident((const void *)k_bin_count, c->grid_bin_count));
  CU(resident((const void *)k_bin_scatter, c->grid_bin_scatter));
  CU(resident((const void *)k_md_scatter, c->grid_md_scatter));
  CU(resident((const void *)k_md_sort, c->grid_md_sort));
  CU(resident((const void *)k_ls_scatter, c->grid_ls_scatter));
  CU(resident((const void *)k_t3_scatter, c->grid_t3_scatter));
  CU(resident((const void *)k_tc_count, c->grid_tc_count));
  CU(resident((const void *)k_tc_scatter, c->grid_tc_scatter));
  CU(resident((const void *)k_tc_decide, c->grid_tc_decide));
  c->grid_bf[0] = score_bf16_blocks_per_sm(false) * c->n_sm;
  c->grid_bf[1] = score_bf16_blocks_per_sm(true) * c->n_sm;
  return LST_OK;
}

// capacities for n hits with the context's current ratios
void caps_for(const lst_ctx_s *c, int64_t n, int &md, int &ls, int &t3, int &t5) {
  const double nmd = std::ceil(c->r_md * (double)n) + 256;
  md = (int)std::min(nmd, 2.0e9);
  ls = (int)std::min(std::ceil(c->r_ls * nmd) + 1024, 2.0e9);
  t3 = (int)std::min(std::ceil(c->r_t3 * nmd) + 1024, 2.0e9);
  t5 = (int)std::min(std::ceil(c->r_t5 * nmd) + 1024, 2.0e9);
}

// Byte offsets of one event's buffers in its slot allocation (H hits, nm modules, md/ls/t3/t5
// object capacities); `total` is the allocation size.
struct SlotLayout {
  size_t hit, om, hrank, scnt, soff, manc, mk, mmod, mh, mst, mcn, uanc, uk, umod, uh, urank, mperm, mq;
  size_t lin, lout, lst, lcn, lost, locn, lsu, t3, t3k, t3s, t3c, t3u, t3uk, t5a, t5b, t5s, t5e, tcc, tcp, tcl,
      tcf, cnt;
  size_t total;
};
SlotLayout slot_layout(int64_t H, size_t nm, size_t md, size_t ls, size_t t3, size_t t5) {
  SlotLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  L.hit = take(16 * (size_t)H); L.om = take(8 * (size_t)H);
  L.hrank = take(4 * (size_t)H);
  L.scnt = take(4 * 2 * nm); L.soff = take(4 * (2 * nm + 1));
  L.manc = take(16 * md); L.mk = take(8 * md); L.mmod = take(4 * md); L.mh = take(8 * md);
  L.mst = take(4 * nm); L.mcn = take(4 * nm);
  L.uanc = take(16 * md); L.uk = take(8 * md); L.umod = take(4 * md); L.uh = take(8 * md);
  L.urank = take(4 * md); L.mperm = take(4 * md); L.mq = take(4 * md);
  L.lin = take(4 * ls); L.lout = take(4 * ls);
  L.lst = take(4 * md); L.lcn = take(4 * md); L.lost = take(4 * md); L.locn = take(4 * md); L.lsu = take(16 * ls);
  L.t3 = take(16 * t3); L.t3k = take(4 * t3); L.t3s = take(4 * md); L.t3c = take(4 * md);
  L.t3u = take(16 * t3); L.t3uk = take(4 * t3);
  L.t5a = take(16 * t5); L.t5b = take(16 * t5); L.t5s = take(4 * t5); L.t5e = take(t5);
  L.tcc = take(4 * md); L.tcp = take(4 * md); L.tcl = take(20 * t5); L.tcf = take(t5);
  L.cnt = take(4 * C_NCOUNTERS);
  L.total = off;
  return L;
}

// test aid (lst_test_fail_alloc): consume one pending injected allocation failure
bool injected_alloc_failure(lst_ctx_s *c) {
  int v = c->fail_allocs.load();
  while (v > 0)
    if (c->fail_allocs.compare_exchange_weak(v, v - 1)) return true;
  return false;
}

// Short-lived device staging of the exports and the pixel matching, from the context's own
// pool: its freed blocks stay reserved (release threshold: never), so a call does not map
// new memory each time (the device's default pool hands freed memory back at every
// synchronisation, and the next call maps it again while the driver holds its locks).
// Every kernel that writes such staging either writes the same values on every run or
// bounds its writes (a profiler replay may not restore pool memory between its passes).
cudaError_t tmp_alloc(lst_ctx_s *c, void **p, size_t bytes, cudaStream_t st) {
  return cudaMallocFromPoolAsync(p, bytes, c->pool, st);
}

// Device buffers of a slot. The serving workers take them from the context's stream-ordered
// pool (pooled): the slot is idle when it grows (its last launch was harvested when its
// event was released and every export synchronises before it returns), so the old buffers
// go back to the pool at once and the new ones are ready in stream order on `st`, the
// stream of the slot's next launch, without waiting for the device. The other callers use
// plain allocations, after a device synchronisation when a buffer is replaced (a profiler
// replaying kernels saves and restores those, which it may not do for pool memory).
cudaError_t slot_buf_alloc(lst_ctx_s *c, void **p, size_t bytes, cudaStream_t st, bool pooled) {
  return pooled ? cudaMallocFromPoolAsync(p, bytes, c->pool, st) : cudaMalloc(p, bytes);
}
cudaError_t slot_buf_free(void *p, cudaStream_t st, bool pooled) {
  if (!p) return cudaSuccess;
  if (pooled) return cudaFreeAsync(p, st);
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(p);
  return e;
}

// (Re)size the buffers of slot s for an event of n_hits.
lst_status slot_alloc(lst_ctx_s *c, Slot &s, int64_t n_hits, cudaStream_t st, bool pooled) {
  int md, ls, t3, t5;
  caps_for(c, n_hits, md, ls, t3, t5);
  const int64_t hcap = std::max<int64_t>(n_hits, 1024);
  if (s.mem && s.hit_cap >= n_hits && s.md_cap >= md && s.ls_cap >= ls && s.t3_cap >= t3 && s.t5_cap >= t5)
    return LST_OK;
  // grow with headroom
  const int64_t H = std::max<int64_t>(s.hit_cap, (int64_t)(hcap * 1.1));
  md = std::max(s.md_cap, md); ls = std::max(s.ls_cap, ls); t3 = std::max(s.t3_cap, t3); t5 = std::max(s.t5_cap, t5);
  const SlotLayout L = slot_layout(H, (size_t)c->g.n_mod, md, ls, t3, t5);
  const size_t off = L.total;
  if (s.mem) {
    CU(slot_buf_free(s.mem, st, s.mem_pooled));
    s.mem = nullptr;
    s.hit_cap = 0; s.md_cap = 0; s.ls_cap = 0; s.t3_cap = 0; s.t5_cap = 0;
  }
  if (injected_alloc_failure(c))
    return fail(LST_ERR_NOMEM, "cudaMalloc(event buffers): injected failure (lst_test_fail_alloc)");
  CU(slot_buf_alloc(c, &s.mem, off, st, pooled));
  s.mem_pooled = pooled;
  s.bytes = off;
  char *b = (char *)s.mem;
  EvDesc &d = s.d;
  d.hit = (float4 *)(b + L.hit); d.hit_om = (int2 *)(b + L.om);
  d.hit_rank = (int32_t *)(b + L.hrank);
  d.sens_cnt = (int32_t *)(b + L.scnt); d.sens_off = (int32_t *)(b + L.soff);
  d.md_anchor = (float4 *)(b + L.manc); d.md_kappa = (float2 *)(b + L.mk); d.md_mod = (int32_t *)(b + L.mmod);
  d.md_hits = (int2 *)(b + L.mh); d.md_start = (int32_t *)(b + L.mst); d.md_cnt = (int32_t *)(b + L.mcn);
  d.mdu_anchor = (float4 *)(b + L.uanc); d.mdu_kappa = (float2 *)(b + L.uk);
  d.mdu_mod = (int32_t *)(b + L.umod); d.mdu_hits = (int2 *)(b + L.uh); d.mdu_rank = (int32_t *)(b + L.urank);
  d.md_perm = (int32_t *)(b + L.mperm); d.md_q = (float *)(b + L.mq);
  d.ls_to = (int32_t *)(b + L.lin); d.ls_from = (int32_t *)(b + L.lout);
  d.ls_start = (int32_t *)(b + L.lst); d.ls_cnt = (int32_t *)(b + L.lcn);
  d.lso_start = (int32_t *)(b + L.lost); d.lso_cnt = (int32_t *)(b + L.locn);
  d.lsu = (int4 *)(b + L.lsu);
  d.t3_md = (int4 *)(b + L.t3); d.t3_kappa = (float *)(b + L.t3k); d.t3_pos = (int32_t *)(b + L.t3s);
  d.t3_cnt = (int32_t *)(b + L.t3c); d.t3u_md = (int4 *)(b + L.t3u); d.t3u_kappa = (float *)(b + L.t3uk);
  d.t5_a = (int4 *)(b + L.t5a); d.t5_b = (int4 *)(b + L.t5b); d.t5_score = (float *)(b + L.t5s);
  d.t5_sel = (uint8_t *)(b + L.t5e); d.cnt = (int32_t *)(b + L.cnt);
  d.tc_cnt = (int32_t *)(b + L.tcc); d.tc_pos = (int32_t *)(b + L.tcp); d.tc_list = (int32_t *)(b + L.tcl);
  d.t5_tc = (uint8_t *)(b + L.tcf);
  s.hit_cap = H; s.md_cap = md; s.ls_cap = ls; s.t3_cap = t3; s.t5_cap = t5;
  d.md_cap = md; d.ls_cap = ls; d.t3_cap = t3; d.t5_cap = t5;
  return LST_OK;
}

// stage host inputs into the slot's own device buffer (copies on `st`)
lst_status slot_inputs(lst_ctx_s *c, Slot &s, const float *x, const float *y, const float *z,
                       const int32_t *sensor, int64_t n, cudaStream_t st, bool pooled) {
  s.d.n_hits = (int32_t)n;
  s.n_hits = n;
  const bool dev = n == 0 || is_device_ptr(x);
  if (dev) {
    s.d.x = x; s.d.y = y; s.d.z = z; s.d.sensor = sensor;
    return LST_OK;
  }
  if (s.in_cap < n) {
    if (s.in_mem) { CU(slot_buf_free(s.in_mem, st, s.in_pooled)); s.in_mem = nullptr; s.in_cap = 0; }
    if (injected_alloc_failure(c))
      return fail(LST_ERR_NOMEM, "cudaMalloc(input staging): injected failure (lst_test_fail_alloc)");
    const int64_t cap = (int64_t)(n * 1.1) + 1024;
    CU(slot_buf_alloc(c, &s.in_mem, (size_t)cap * 16, st, pooled));
    s.in_pooled = pooled;
    s.in_cap = cap;
  }
  float *b = (float *)s.in_mem;
  float *dx = b, *dy = b + s.in_cap, *dz = b + 2 * s.in_cap;
  int32_t *ds = (int32_t *)(b + 3 * s.in_cap);
  CU(cudaMemcpyAsync(dx, x, 4 * n, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(dy, y, 4 * n, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(dz, z, 4 * n, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(ds, sensor, 4 * n, cudaMemcpyHostToDevice, st));
  s.d.x = dx; s.d.y = dy; s.d.z = dz; s.d.sensor = ds;
  return LST_OK;
}

lst_status lane_init(Lane &L) {
  CU(cudaMalloc(&L.d_desc, sizeof(EvDesc) * MAX_EVENTS));
  CU(cudaMallocHost(&L.h_desc, sizeof(EvDesc) * MAX_EVENTS));
  CU(cudaMalloc(&L.d_work, sizeof(int) * 16));
  CU(cudaMalloc(&L.d_counts, sizeof(int) * MAX_EVENTS * C_NCOUNTERS));
  CU(cudaMallocHost(&L.h_counts, sizeof(int) * MAX_EVENTS * C_NCOUNTERS));
  CU(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
  for (auto &e : L.tev) CU(cudaEventCreate(&e));
  CU(cudaStreamCreateWithFlags(&L.cap_stream, cudaStreamNonBlocking));
  return LST_OK;
}

// Wait for the lane's last batch and copy its counters into the slots.
lst_status lane_harvest(lst_ctx_s *c, Lane &L) {
  if (!L.inflight) return LST_OK;
  CU(cudaEventSynchronize(L.done));
  for (int i = 0; i < L.n; i++) {
    Slot &s = c->slots[L.slots[i]];
    if (s.lane_gen == L.gen && s.lane == (int)(&L - c->lanes.data())) {
      std::memcpy(s.cnt, L.h_counts + i * C_NCOUNTERS, sizeof(s.cnt));
      s.have_cnt = true;
    }
  }
  if (L.timed) {
    for (int k = 0; k < LST_N_STAGES; k++) {
      float ms = 0.0f;
      CU(cudaEventElapsedTime(&ms, L.tev[k], L.tev[k + 1]));
      c->stage_sum[k] += ms;
    }
    c->stage_n++;
  }
  L.inflight = false;
  return LST_OK;
}

// Enqueue the whole pipeline for the lane's current batch (desc already on device).
lst_status enqueue_pipeline(lst_ctx_s *c, Lane &L, int n, cudaStream_t st, bool timed, bool capturing) {
  const DevGeom g = c->g;
  // stage boundary events; inside a capture they become event-record nodes of the graph
  NvtxStages ranges;
  auto mark = [&](int i) {
    ranges.next(i < LST_N_STAGES ? STAGE_NAMES[i] : nullptr);
    if (timed) cudaEventRecordWithFlags(L.tev[i], st, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  };
  mark(0);
  k_reset<<<dim3(std::max(1, c->n_sm / n + 1), n), 256, 0, st>>>(L.d_desc, g);
  k_bin_count<<<c->grid_bin_count, 256, 0, st>>>(L.d_desc, n, g);
  k_bin_scan<<<n, 1024, 0, st>>>(L.d_desc, g);
  k_bin_scatter<<<c->grid_bin_scatter, 256, 0, st>>>(L.d_desc, n, g);
  CU(cudaMemsetAsync(L.d_work, 0, sizeof(int) * 16, st));
  mark(1);
  k_md<<<c->grid_md, c->md_threads, md_smem(c), st>>>(L.d_desc, n, g, c->cuts);
  k_md_scan<<<n, 1024, 0, st>>>(L.d_desc, g);
  k_md_scatter<<<c->grid_md_scatter, 256, 0, st>>>(L.d_desc, n);
  k_md_sort<<<c->grid_md_sort, 256, 0, st>>>(L.d_desc, n);
  mark(2);
  {
    // few events: units of LS_SMALL_TB target modules, so that dense modules spread over
    // several warps; many events: one unit per module
    const bool small = (long long)n * g.n_mod < 16ll * c->grid_ls * (c->ls_threads / 32);
    if (small)
      k_ls<<<c->grid_ls, c->ls_threads, ls_smem(c), st>>>(L.d_desc, n, g, c->cuts, L.d_work + 1, c->d_ls_units,
                                                         c->ls_units_per_event, LS_SMALL_TB);
    else
      k_ls<<<c->grid_ls, c->ls_threads, ls_smem(c), st>>>(L.d_desc, n, g, c->cuts, L.d_work + 1, nullptr, g.n_mod,
                                                         0);
  }
  mark(3);
  k_ls_scan<<<2 * n, 1024, 0, st>>>(L.d_desc);
  k_ls_scatter<<<c->grid_ls_scatter, 256, 0, st>>>(L.d_desc, n);
  mark(4);
  // step-3 units: few middle MDs when few events share the launch, so that the heaviest
  // unit (the longest warp) stays short against the launch
  const int t3_mds = c->t3_mds > 0 ? c->t3_mds : (n >= 16 ? 16 : n >= 4 ? 4 : 2);
  k_t3<<<c->grid_t3, c->t3_threads, t3_smem(c), st>>>(L.d_desc, n, c->cuts, L.d_work + 2, t3_mds);
  k_t3_scan<<<n, 1024, 0, st>>>(L.d_desc);
  k_t3_scatter<<<c->grid_t3_scatter, 256, 0, st>>>(L.d_desc, n);
  mark(5);
  k_t5<<<c->grid_t5, c->t5_threads, t5_smem(c), st>>>(L.d_desc, n, c->cuts);
  mark(6);
  if (c->cfg.precision != LST_FP32)
    CU(launch_score_bf16_events(c->grid_bf[c->cfg.precision == LST_BF16X3], st, L.d_desc, n, g, c->cuts, c->d_wpack,
                                c->d_w, c->n_hidden, c->d_err, c->wait_limit, c->cfg.precision == LST_BF16X3,
                                c->skip_mma));
  else
    k_score_fp32<<<c->grid_sc, c->sc_threads, (size_t)mlp_floats_host(c->n_hidden) * 4, st>>>(
        L.d_desc, n, g, c->cuts, c->d_w, c->n_hidden);
  mark(7);
  k_tc_count<<<c->grid_tc_count, 256, 0, st>>>(L.d_desc, n);
  k_tc_scan<<<n, 1024, 0, st>>>(L.d_desc);
  k_tc_scatter<<<c->grid_tc_scatter, 256, 0, st>>>(L.d_desc, n);
  k_tc_decide<<<c->grid_tc_decide, 256, 0, st>>>(L.d_desc, n);
  mark(8);
  k_collect<<<(n + 127) / 128, 128, 0, st>>>(L.d_desc, n, L.d_counts);
  CU(cudaMemcpyAsync(L.h_counts, L.d_counts, sizeof(int) * C_NCOUNTERS * n, cudaMemcpyDeviceToHost, st));
  CU(cudaGetLastError());
  return LST_OK;
}

int find_free_slot(lst_ctx_s *c) {
  for (size_t i = 0; i < c->slots.size(); i++)
    if (!c->slots[i].busy) return (int)i;
  return -1;
}

void grow_ratios(lst_ctx_s *c, const Slot &s, const int32_t *cnt) {
  const int f = cnt[C_FLAGS];
  const double n = std::max<double>(1.0, (double)s.n_hits);
  const double nmd = std::max<double>(1.0, std::ceil(c->r_md * n) + 256);
  // the overflowed stage counted all its objects; at least double in any case
  if (f & F_OVF_MD) c->r_md = std::max(2.0f * c->r_md, (float)(1.3 * cnt[C_MD] / n));
  if (f & F_OVF_LS) c->r_ls = std::max(2.0f * c->r_ls, (float)(1.3 * cnt[C_LS] / nmd));
  if (f & F_OVF_T3) c->r_t3 = std::max(2.0f * c->r_t3, (float)(1.3 * cnt[C_T3] / nmd));
  if (f & F_OVF_T5) c->r_t5 = std::max(2.0f * c->r_t5, (float)(1.3 * cnt[C_T5] / nmd));
}

lst_status status_of(const int32_t *cnt) {
  if (cnt[C_FLAGS] & F_CHECK) return LST_ERR_CUDA;   // failed device bounds check (LST_CHECK builds)
  if (cnt[C_FLAGS] & F_TIMEOUT) return LST_ERR_TIMEOUT;
  if (cnt[C_FLAGS] & F_INPUT) return LST_ERR_INPUT;
  if (cnt[C_FLAGS] & (F_OVF_MD | F_OVF_LS | F_OVF_T3 | F_OVF_T5)) return LST_ERR_CAPACITY;
  return LST_OK;
}

lst_status wait_event(lst_event ev) {
  lst_ctx_s *c = ev->ctx;
  Slot &s = c->slots[ev->slot];
  if (!s.have_cnt) {
    if (s.lane < 0) return fail(LST_ERR_NOT_READY, "event has no pending work");
    lst_status st = lane_harvest(c, c->lanes[s.lane]);
    if (st != LST_OK) return st;
    if (!s.have_cnt) return fail(LST_ERR_NOT_READY, "event counters unavailable");
  }
  // the lane may have been harvested through another event of the same batch
  if (ev->status == LST_ERR_NOT_READY) {
    ev->status = status_of(s.cnt);
    if (ev->status == LST_ERR_CAPACITY) grow_ratios(c, s, s.cnt);
  }
  return LST_OK;
}

}  // namespace

namespace lstk {
__global__ void k_collect(const EvDesc *__restrict__ evs, int n, int *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n)
    for (int k = 0; k < C_NCOUNTERS; k++) out[e * C_NCOUNTERS + k] = evs[e].cnt[k];
}
}  // namespace lstk

namespace {
// Track candidates of one event into caller buffers (device or host), any order.
lst_status gather_tc(lst_ctx_s *c, const EvDesc *dd, int n_t5, int64_t n, int32_t *hit_idx, float *score,
                     uint8_t *selected) {
  const bool dev_out = is_device_ptr(hit_idx);
  const size_t bytes = 256 + (dev_out ? 0 : (size_t)n * 40 + (size_t)n * 4 + (size_t)n);
  void *tmp = nullptr;
  CU(tmp_alloc(c, &tmp, bytes, c->aux));
  int *d_counter = (int *)tmp;
  int32_t *d_idx = dev_out ? hit_idx : (int32_t *)((char *)tmp + 256);
  float *d_sc = dev_out ? score : (float *)(d_idx + (size_t)n * 10);
  uint8_t *d_sel = dev_out ? selected : (uint8_t *)(d_sc + n);
  CU(cudaMemsetAsync(d_counter, 0, sizeof(int), c->aux));
  const int grid = (int)std::min<int64_t>((n_t5 + 255) / 256, 4 * c->n_sm);
  if (grid > 0) k_gather_tc<<<grid, 256, 0, c->aux>>>(dd, n_t5, d_counter, d_idx, d_sc, d_sel, n);
  CU(cudaGetLastError());
  if (!dev_out) {
    CU(cudaMemcpyAsync(hit_idx, d_idx, (size_t)n * 40, cudaMemcpyDeviceToHost, c->aux));
    if (score) CU(cudaMemcpyAsync(score, d_sc, (size_t)n * 4, cudaMemcpyDeviceToHost, c->aux));
    if (selected) CU(cudaMemcpyAsync(selected, d_sel, (size_t)n, cudaMemcpyDeviceToHost, c->aux));
  }
  CU(cudaFreeAsync(tmp, c->aux));
  CU(cudaStreamSynchronize(c->aux));
  return LST_OK;
}
}  // namespace

// =========================================================================== C-ABI
extern "C" {

const char *lst_status_str(int32_t s) {
  switch (s) {
    case LST_OK: return "LST_OK";
    case LST_ERR_ARG: return "LST_ERR_ARG";
    case LST_ERR_CAPACITY: return "LST_ERR_CAPACITY";
    case LST_ERR_CUDA: return "LST_ERR_CUDA";
    case LST_ERR_TIMEOUT: return "LST_ERR_TIMEOUT";
    case LST_ERR_NOT_READY: return "LST_ERR_NOT_READY";
    case LST_ERR_INPUT: return "LST_ERR_INPUT";
    case LST_ERR_NOMEM: return "LST_ERR_NOMEM";
    default: return "LST_ERR_UNKNOWN";
  }
}

const char *lst_last_error(void) { return g_err.c_str(); }

lst_status lst_default_config(lst_config *cfg) {
  if (!cfg) return fail(LST_ERR_ARG, "cfg is NULL");
  std::memset(cfg, 0, sizeof *cfg);
  cfg->precision = LST_FP32;
  cfg->max_events = 1;
  cfg->use_graphs = 1;
  cfg->md_per_hit = 0.75f;
  cfg->ls_per_md = 16.0f;
  cfg->t3_per_md = 3.0f;
  cfg->t5_per_md = 2.0f;
  return LST_OK;
}

lst_status lst_create(int cuda_device, const lst_config *cfg, lst_ctx *out) {
  if (!out) return fail(LST_ERR_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (cuda_device < 0 || cuda_device >= ndev) return fail(LST_ERR_ARG, "bad device index");
  lst_config d;
  lst_default_config(&d);
  const lst_config &c = cfg ? *cfg : d;
  if (c.max_events < 1 || c.max_events > MAX_EVENTS) return fail(LST_ERR_ARG, "max_events out of range");
  if (c.precision != LST_FP32 && c.precision != LST_BF16 && c.precision != LST_BF16X3)
    return fail(LST_ERR_ARG, "bad precision");
  DeviceGuard gd(cuda_device);
  lst_ctx_s *x = new lst_ctx_s();
  x->device = cuda_device;
  x->cfg = c;
  x->r_md = c.md_per_hit > 0 ? c.md_per_hit : d.md_per_hit;
  x->r_ls = c.ls_per_md > 0 ? c.ls_per_md : d.ls_per_md;
  x->r_t3 = c.t3_per_md > 0 ? c.t3_per_md : d.t3_per_md;
  x->r_t5 = c.t5_per_md > 0 ? c.t5_per_md : d.t5_per_md;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, cuda_device) != cudaSuccess) { delete x; return fail(LST_ERR_CUDA, "device properties"); }
  x->n_sm = p.multiProcessorCount;
  x->slots.resize(c.max_events);
  x->lanes.resize(1 + BATCH_LANES);
  for (auto &L : x->lanes) {
    lst_status s = lane_init(L);
    if (s != LST_OK) { lst_destroy(x); return s; }
  }
  cudaStreamCreateWithFlags(&x->aux, cudaStreamNonBlocking);
  {
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = cuda_device;
    if (cudaMemPoolCreate(&x->pool, &pp) != cudaSuccess) {
      x->pool = nullptr;
      lst_destroy(x);
      return fail(LST_ERR_CUDA, "memory pool creation");
    }
    uint64_t keep = ~0ull;     // freed blocks stay in the pool for the next slot growth
    cudaMemPoolSetAttribute(x->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (cudaMalloc(&x->d_err, sizeof(int)) != cudaSuccess || cudaMemset(x->d_err, 0, sizeof(int)) != cudaSuccess) {
    lst_destroy(x);
    return fail(LST_ERR_NOMEM, "device error word");
  }
  lst_status s = compute_grids(x);
  if (s != LST_OK) { lst_destroy(x); return s; }
  *out = x;
  return LST_OK;
}

lst_status lst_load_geometry(lst_ctx c, const lst_module *mods, int32_t n_mod, const int32_t *map_off,
                             const int32_t *map_tgt, const lst_cuts *cuts, const lst_mlp *weights) {
  if (!c || !mods || !map_off || !cuts || n_mod <= 0) return fail(LST_ERR_ARG, "null argument or n_mod <= 0");
  if (map_off[0] != 0) return fail(LST_ERR_ARG, "map_off[0] != 0");
  for (int32_t m = 0; m < n_mod; m++) {
    if (mods[m].layer < 1 || mods[m].layer > 11) return fail(LST_ERR_ARG, "module layer out of range");
    if (mods[m].subdet != 0 && mods[m].subdet != 1) return fail(LST_ERR_ARG, "module subdet out of range");
    if (map_off[m + 1] < map_off[m]) return fail(LST_ERR_ARG, "map_off not monotonic");
    if (map_off[m + 1] - map_off[m] > MAX_FANOUT) return fail(LST_ERR_ARG, "module map fan-out above 512");
  }
  const int32_t nl = map_off[n_mod];
  if (nl > 0 && !map_tgt) return fail(LST_ERR_ARG, "map_tgt is NULL");
  for (int32_t i = 0; i < nl; i++)
    if (map_tgt[i] < 0 || map_tgt[i] >= n_mod) return fail(LST_ERR_ARG, "map target out of range");
  int nh = 2;
  if (weights) {
    nh = weights->n_hidden;
    if (nh < 1 || nh > 4 || !weights->w) return fail(LST_ERR_ARG, "n_hidden must be 1..4 with weights");
  }
  DeviceGuard gd(c->device);
  CU(cudaDeviceSynchronize());
  for (auto &L : c->lanes) {
    for (auto &kv : L.graphs) cudaGraphExecDestroy(kv.second);
    L.graphs.clear();
  }
  cudaFree(c->d_subdet); cudaFree(c->d_layer); cudaFree(c->d_map_off); cudaFree(c->d_map_tgt); cudaFree(c->d_w);
  cudaFree(c->d_ls_units);
  c->d_subdet = nullptr; c->d_layer = nullptr; c->d_map_off = nullptr; c->d_map_tgt = nullptr; c->d_w = nullptr;
  c->d_ls_units = nullptr;
  std::vector<int8_t> sd(n_mod), ly(n_mod);
  for (int32_t m = 0; m < n_mod; m++) { sd[m] = (int8_t)mods[m].subdet; ly[m] = (int8_t)mods[m].layer; }
  CU(cudaMalloc(&c->d_subdet, n_mod));
  CU(cudaMalloc(&c->d_layer, n_mod));
  CU(cudaMalloc(&c->d_map_off, 4 * ((size_t)n_mod + 1)));
  CU(cudaMalloc(&c->d_map_tgt, 4 * (size_t)std::max(nl, 1)));
  CU(cudaMemcpy(c->d_subdet, sd.data(), n_mod, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->d_layer, ly.data(), n_mod, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->d_map_off, map_off, 4 * ((size_t)n_mod + 1), cudaMemcpyHostToDevice));
  if (nl > 0) CU(cudaMemcpy(c->d_map_tgt, map_tgt, 4 * (size_t)nl, cudaMemcpyHostToDevice));
  {
    // step-2 units of small launches: LS_SMALL_TB target modules each (at least one per module)
    std::vector<int32_t> uo((size_t)n_mod + 1, 0);
    for (int32_t m = 0; m < n_mod; m++) {
      const int32_t fan = map_off[m + 1] - map_off[m];
      uo[m + 1] = uo[m] + std::max(1, (fan + LS_SMALL_TB - 1) / LS_SMALL_TB);
    }
    CU(cudaMalloc(&c->d_ls_units, 4 * ((size_t)n_mod + 1)));
    CU(cudaMemcpy(c->d_ls_units, uo.data(), 4 * ((size_t)n_mod + 1), cudaMemcpyHostToDevice));
    c->ls_units_per_event = uo[n_mod];
  }
  c->n_hidden = nh;
  c->n_w = mlp_floats_host(nh);
  std::vector<float> w(c->n_w, 0.0f);
  if (weights) std::memcpy(w.data(), weights->w, 4 * (size_t)c->n_w);
  CU(cudaMalloc(&c->d_w, 4 * (size_t)c->n_w));
  CU(cudaMemcpy(c->d_w, w.data(), 4 * (size_t)c->n_w, cudaMemcpyHostToDevice));
  {
    std::vector<uint16_t> pk(2 * (32 * 48 + 3 * 32 * 32), 0);   // hi parts, then lo parts
    pack_weights_bf16(w.data(), nh, pk.data());
    cudaFree(c->d_wpack);
    c->d_wpack = nullptr;
    CU(cudaMalloc(&c->d_wpack, pk.size() * 2));
    CU(cudaMemcpy(c->d_wpack, pk.data(), pk.size() * 2, cudaMemcpyHostToDevice));
  }
  c->g.n_mod = n_mod;
  c->g.subdet = c->d_subdet;
  c->g.layer = c->d_layer;
  c->g.map_off = c->d_map_off;
  c->g.map_tgt = c->d_map_tgt;
  c->cuts = *cuts;
  // slot buffers depend on n_mod: drop them
  for (auto &s : c->slots) {
    if (s.mem) cudaFree(s.mem);
    s.mem = nullptr; s.hit_cap = 0; s.md_cap = s.ls_cap = s.t3_cap = s.t5_cap = 0;
    s.busy = false; s.have_cnt = false; s.lane = -1;
  }
  c->have_geom = true;
  return LST_OK;
}

// The lane's graph of the whole pipeline for n events (captured on first use): the kernels
// read the events' descriptors from the lane's device array, so one graph serves every
// batch of n events.
static lst_status lane_graph(lst_ctx c, Lane &L, int n, bool timed, cudaGraphExec_t *out) {
  const long long key = (long long)n * 16 + c->cfg.precision * 2 + (timed ? 1 : 0);
  auto it = L.graphs.find(key);
  if (it == L.graphs.end()) {
    cudaGraph_t graph;
    CU(cudaStreamBeginCapture(L.cap_stream, cudaStreamCaptureModeThreadLocal));
    lst_status s = enqueue_pipeline(c, L, n, L.cap_stream, timed, true);
    cudaError_t e = cudaStreamEndCapture(L.cap_stream, &graph);
    if (s != LST_OK) return s;
    if (e != cudaSuccess) return fail(LST_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(LST_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    it = L.graphs.emplace(key, exec).first;
  }
  *out = it->second;
  return LST_OK;
}

static lst_status run_lane(lst_ctx c, Lane &L, int n, const int *slot_ids, cudaStream_t st, bool allow_graph,
                           bool timed) {
  L.gen++;
  L.n = n;
  for (int i = 0; i < n; i++) {
    L.slots[i] = slot_ids[i];
    Slot &s = c->slots[slot_ids[i]];
    s.d.md_cap = s.md_cap; s.d.ls_cap = s.ls_cap; s.d.t3_cap = s.t3_cap; s.d.t5_cap = s.t5_cap;
    L.h_desc[i] = s.d;
    s.lane = (int)(&L - c->lanes.data());
    s.lane_pos = i;
    s.lane_gen = L.gen;
    s.have_cnt = false;
  }
  CU(cudaMemcpyAsync(L.d_desc, L.h_desc, sizeof(EvDesc) * n, cudaMemcpyHostToDevice, st));
  if (allow_graph && c->cfg.use_graphs) {
    cudaGraphExec_t exec = nullptr;
    lst_status s = lane_graph(c, L, n, timed, &exec);
    if (s != LST_OK) return s;
    CU(cudaGraphLaunch(exec, st));
  } else {
    lst_status s = enqueue_pipeline(c, L, n, st, timed, false);
    if (s != LST_OK) return s;
  }
  L.timed = timed;
  CU(cudaEventRecord(L.done, st));
  L.inflight = true;
  return LST_OK;
}

lst_status lst_run_event(lst_ctx c, const float *x, const float *y, const float *z, const int32_t *sensor,
                         int64_t n_hits, void *cuda_stream, lst_event *out) {
  NvtxRange nvtx_range("lst_run_event");
  if (!c || !out) return fail(LST_ERR_ARG, "null ctx/out");
  *out = nullptr;
  if (n_hits < 0 || n_hits > (int64_t)1 << 30) return fail(LST_ERR_ARG, "n_hits out of range");
  if (n_hits > 0 && (!x || !y || !z || !sensor)) return fail(LST_ERR_ARG, "null hit array");
  if (!c->have_geom) return fail(LST_ERR_NOT_READY, "no geometry loaded");
  DeviceGuard gd(c->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Lane &L = c->lanes[0];
  lst_status s = lane_harvest(c, L);
  if (s != LST_OK) return s;
  const int si = find_free_slot(c);
  if (si < 0) return fail(LST_ERR_NOT_READY, "no free event slot (release events)");
  Slot &S = c->slots[si];
  for (int attempt = 0; attempt < 6; attempt++) {
    s = slot_alloc(c, S, n_hits, st, false);
    if (s != LST_OK) return s;
    s = slot_inputs(c, S, x, y, z, sensor, n_hits, st, false);
    if (s != LST_OK) return s;
    s = run_lane(c, L, 1, &si, st, false, c->timing);
    if (s != LST_OK) return s;
    s = lane_harvest(c, L);
    if (s != LST_OK) return s;
    const lst_status es = status_of(S.cnt);
    if (es == LST_ERR_CAPACITY) { grow_ratios(c, S, S.cnt); continue; }
    if (S.cnt[C_FLAGS] & F_CHECK) {
      char msg[128];
      std::snprintf(msg, sizeof msg, "device bounds check failed at site %d, index %d", S.cnt[C_DBG_SITE],
                    S.cnt[C_DBG_VAL]);
      return fail(LST_ERR_CUDA, msg);
    }
    S.busy = true;
    lst_event ev = new lst_event_s{c, si, es};
    *out = ev;
    if (es == LST_ERR_INPUT) return fail(es, "invalid hit in input (sensor id or coordinate)");
    if (es != LST_OK) return fail(es, "a bounded device wait ran out (tensor-core score)");
    return LST_OK;
  }
  return fail(LST_ERR_CAPACITY, "object buffers kept overflowing");
}

lst_status lst_run_batch(lst_ctx c, int32_t n, const float *const *x, const float *const *y,
                         const float *const *z, const int32_t *const *sensor, const int64_t *n_hits,
                         void *cuda_stream, lst_event *out) {
  NvtxRange nvtx_range("lst_run_batch");
  if (!c || !out || !x || !y || !z || !sensor || !n_hits) return fail(LST_ERR_ARG, "null argument");
  if (n < 1 || n > (int32_t)c->slots.size()) return fail(LST_ERR_ARG, "batch size outside 1..max_events");
  if (!c->have_geom) return fail(LST_ERR_NOT_READY, "no geometry loaded");
  for (int i = 0; i < n; i++) {
    if (n_hits[i] < 0 || n_hits[i] > (int64_t)1 << 30) return fail(LST_ERR_ARG, "n_hits out of range");
    if (n_hits[i] > 0 && (!x[i] || !y[i] || !z[i] || !sensor[i])) return fail(LST_ERR_ARG, "null hit array");
  }
  DeviceGuard gd(c->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int li = c->next_lane;
  c->next_lane = 1 + (c->next_lane % ((int)c->lanes.size() - 1));
  Lane &L = c->lanes[li];
  lst_status s = lane_harvest(c, L);
  if (s != LST_OK) return s;
  std::vector<int> ids;
  for (size_t i = 0; i < c->slots.size() && (int)ids.size() < n; i++)
    if (!c->slots[i].busy) ids.push_back((int)i);
  if ((int)ids.size() < n) return fail(LST_ERR_NOT_READY, "not enough free event slots");
  for (int i = 0; i < n; i++) {
    Slot &S = c->slots[ids[i]];
    if (S.lane >= 0 && S.lane != li) { s = lane_harvest(c, c->lanes[S.lane]); if (s != LST_OK) return s; }
    s = slot_alloc(c, S, n_hits[i], st, false);
    if (s != LST_OK) return s;
    s = slot_inputs(c, S, x[i], y[i], z[i], sensor[i], n_hits[i], st, false);
    if (s != LST_OK) return s;
  }
  s = run_lane(c, L, n, ids.data(), st, true, c->timing);
  if (s != LST_OK) return s;
  for (int i = 0; i < n; i++) {
    c->slots[ids[i]].busy = true;
    out[i] = new lst_event_s{c, ids[i], LST_ERR_NOT_READY};
  }
  return LST_OK;
}

lst_status lst_event_counts(lst_event ev, lst_counts *out) {
  if (!ev || !out) return fail(LST_ERR_ARG, "null argument");
  DeviceGuard gd(ev->ctx->device);
  lst_status s = wait_event(ev);
  if (s != LST_OK) return s;
  const Slot &S = ev->ctx->slots[ev->slot];
  out->n_hits = S.n_hits;
  out->n_md = S.cnt[C_MD];
  out->n_ls = S.cnt[C_LS];
  out->n_t3 = S.cnt[C_T3];
  out->n_t5 = S.cnt[C_T5];
  out->n_selected = S.cnt[C_NSEL];
  out->n_tc = S.cnt[C_NTC];
  out->pairs[0] = (uint32_t)S.cnt[C_PMD];
  out->pairs[1] = (uint32_t)S.cnt[C_PLS];
  out->pairs[2] = (uint32_t)S.cnt[C_PT3];
  out->pairs[3] = (uint32_t)S.cnt[C_PT5];
  out->status = status_of(S.cnt);
  int mask = 0;
  const int f = S.cnt[C_FLAGS];
  if (f & F_OVF_MD) mask |= 1 << LST_MD;
  if (f & F_OVF_LS) mask |= 1 << LST_LS;
  if (f & F_OVF_T3) mask |= 1 << LST_T3;
  if (f & F_OVF_T5) mask |= 1 << LST_T5;
  out->overflow_mask = mask;
  return LST_OK;
}

static lst_status slot_desc_device(lst_ctx c, int si, EvDesc **dptr) {
  // one device copy of the slot descriptor in the context scratch
  const size_t need = sizeof(EvDesc);
  if (c->scratch_bytes < need) {
    cudaFree(c->scratch);
    c->scratch = nullptr;
    CU(cudaMalloc(&c->scratch, 4096));
    c->scratch_bytes = 4096;
  }
  EvDesc d = c->slots[si].d;
  CU(cudaMemcpyAsync(c->scratch, &d, sizeof d, cudaMemcpyHostToDevice, c->aux));
  CU(cudaStreamSynchronize(c->aux));
  *dptr = (EvDesc *)c->scratch;
  return LST_OK;
}

lst_status lst_get_candidates(lst_event ev, int32_t kind, int32_t *hit_idx, float *score, uint8_t *selected,
                              int64_t capacity, int64_t *n_out) {
  NvtxRange nvtx_range("lst_get_candidates");
  if (!ev || !n_out) return fail(LST_ERR_ARG, "null argument");
  if (kind < LST_MD || kind > LST_TC) return fail(LST_ERR_ARG, "bad kind");
  lst_ctx c = ev->ctx;
  DeviceGuard gd(c->device);
  lst_status s = wait_event(ev);
  if (s != LST_OK) return s;
  const Slot &S = c->slots[ev->slot];
  const int cs[5] = {C_MD, C_LS, C_T3, C_T5, C_NTC};
  const int64_t n = S.cnt[cs[kind]];
  *n_out = n;
  if (ev->status != LST_OK) return fail((lst_status)ev->status, "event has no valid results");
  if (capacity < n) return fail(LST_ERR_CAPACITY, "output capacity below object count");
  if (n == 0) return LST_OK;
  if (!hit_idx) return fail(LST_ERR_ARG, "hit_idx is NULL");
  const int width = kind == LST_MD ? 2 : kind == LST_LS ? 4 : kind == LST_T3 ? 6 : 10;
  EvDesc *dd;
  s = slot_desc_device(c, ev->slot, &dd);
  if (s != LST_OK) return s;
  if (kind == LST_TC) return gather_tc(c, dd, (int)S.cnt[C_T5], n, hit_idx, score, selected);
  const bool dev_out = is_device_ptr(hit_idx);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * c->n_sm);
  if (dev_out) {
    k_gather<<<grid, 256, 0, c->aux>>>(dd, kind, (int)n, hit_idx, kind == LST_T5 ? score : nullptr,
                                       kind == LST_T5 ? selected : nullptr);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->aux));
    return LST_OK;
  }
  const size_t bytes = (size_t)n * width * 4 + (size_t)n * 4 + (size_t)n + 1024;
  void *tmp = nullptr;
  CU(tmp_alloc(c, &tmp, bytes, c->aux));
  int32_t *d_idx = (int32_t *)tmp;
  float *d_sc = (float *)(d_idx + (size_t)n * width);
  uint8_t *d_sel = (uint8_t *)(d_sc + n);
  k_gather<<<grid, 256, 0, c->aux>>>(dd, kind, (int)n, d_idx, d_sc, d_sel);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(hit_idx, d_idx, (size_t)n * width * 4, cudaMemcpyDeviceToHost, c->aux));
  if (kind == LST_T5 && score) CU(cudaMemcpyAsync(score, d_sc, (size_t)n * 4, cudaMemcpyDeviceToHost, c->aux));
  if (kind == LST_T5 && selected) CU(cudaMemcpyAsync(selected, d_sel, (size_t)n, cudaMemcpyDeviceToHost, c->aux));
  CU(cudaFreeAsync(tmp, c->aux));
  CU(cudaStreamSynchronize(c->aux));
  return LST_OK;
}

lst_status lst_get_candidates_batch(const lst_event *evs, int32_t n, int32_t kind, int32_t *hit_idx, float *score,
                                    uint8_t *selected, int64_t capacity, int64_t *offsets) {
  NvtxRange nvtx_range("lst_get_candidates_batch");
  if (!evs || n < 1 || !offsets) return fail(LST_ERR_ARG, "null argument or n < 1");
  if (kind < LST_MD || kind > LST_TC) return fail(LST_ERR_ARG, "bad kind");
  lst_ctx c = evs[0] ? evs[0]->ctx : nullptr;
  if (!c) return fail(LST_ERR_ARG, "null event");
  for (int i = 0; i < n; i++)
    if (!evs[i] || evs[i]->ctx != c) return fail(LST_ERR_ARG, "events of one context expected");
  DeviceGuard gd(c->device);
  const int cs[5] = {C_MD, C_LS, C_T3, C_T5, C_NTC};
  std::vector<EvDesc> desc(n);
  offsets[0] = 0;
  for (int i = 0; i < n; i++) {
    lst_status s = wait_event(evs[i]);
    if (s != LST_OK) return s;
    const Slot &S = c->slots[evs[i]->slot];
    desc[i] = S.d;
    const int64_t k = evs[i]->status == LST_OK ? S.cnt[cs[kind]] : 0;
    offsets[i + 1] = offsets[i] + k;
  }
  const int64_t total = offsets[n];
  if (capacity < total) return fail(LST_ERR_CAPACITY, "output capacity below object count");
  if (total == 0) return LST_OK;
  if (!hit_idx) return fail(LST_ERR_ARG, "hit_idx is NULL");
  const int width = kind == LST_MD ? 2 : kind == LST_LS ? 4 : kind == LST_T3 ? 6 : 10;
  const bool t5like = kind == LST_T5 || kind == LST_TC;
  const bool dev_out = is_device_ptr(hit_idx);
  // device staging: descriptors, TC counters, and (host destination) the gathered arrays
  const size_t b_desc = align_up(sizeof(EvDesc) * (size_t)n, 256), b_cnt = align_up(4 * (size_t)n, 256);
  const size_t b_idx = dev_out ? 0 : align_up((size_t)total * width * 4, 256);
  const size_t b_sc = dev_out ? 0 : align_up((size_t)total * 4, 256);
  const size_t b_sel = dev_out ? 0 : align_up((size_t)total, 256);
  void *tmp = nullptr;
  CU(tmp_alloc(c, &tmp, b_desc + b_cnt + b_idx + b_sc + b_sel, c->aux));
  char *p = (char *)tmp;
  EvDesc *d_desc = (EvDesc *)p;
  int *d_cnt = (int *)(p + b_desc);
  int32_t *d_idx = dev_out ? hit_idx : (int32_t *)(p + b_desc + b_cnt);
  float *d_sc = dev_out ? score : (float *)(p + b_desc + b_cnt + b_idx);
  uint8_t *d_sel = dev_out ? selected : (uint8_t *)(p + b_desc + b_cnt + b_idx + b_sc);
  CU(cudaMemcpyAsync(d_desc, desc.data(), sizeof(EvDesc) * (size_t)n, cudaMemcpyHostToDevice, c->aux));
  CU(cudaMemsetAsync(d_cnt, 0, 4 * (size_t)n, c->aux));
  for (int i = 0; i < n; i++) {
    const int64_t k = offsets[i + 1] - offsets[i];
    if (k == 0) continue;
    int32_t *o = d_idx + offsets[i] * width;
    float *sc = t5like && d_sc ? d_sc + offsets[i] : nullptr;
    uint8_t *se = t5like && d_sel ? d_sel + offsets[i] : nullptr;
    if (kind == LST_TC) {
      const int n5 = c->slots[evs[i]->slot].cnt[C_T5];
      const int grid = (int)std::min<int64_t>((n5 + 255) / 256, 4 * c->n_sm);
      k_gather_tc<<<std::max(grid, 1), 256, 0, c->aux>>>(d_desc + i, n5, d_cnt + i, o, sc, se, k);
    } else {
      const int grid = (int)std::min<int64_t>((k + 255) / 256, 4 * c->n_sm);
      k_gather<<<grid, 256, 0, c->aux>>>(d_desc + i, kind, (int)k, o, sc, se);
    }
  }
  CU(cudaGetLastError());
  if (!dev_out) {
    CU(cudaMemcpyAsync(hit_idx, d_idx, (size_t)total * width * 4, cudaMemcpyDeviceToHost, c->aux));
    if (t5like && score) CU(cudaMemcpyAsync(score, d_sc, (size_t)total * 4, cudaMemcpyDeviceToHost, c->aux));
    if (t5like && selected) CU(cudaMemcpyAsync(selected, d_sel, (size_t)total, cudaMemcpyDeviceToHost, c->aux));
  }
  CU(cudaFreeAsync(tmp, c->aux));
  CU(cudaStreamSynchronize(c->aux));
  return LST_OK;
}

lst_status lst_get_ls_graph(lst_event ev, int32_t *row_off, int32_t *col, float *node_feat, float *edge_feat,
                           int64_t node_cap, int64_t edge_cap, int64_t *n_nodes, int64_t *n_edges) {
  NvtxRange nvtx_range("lst_get_ls_graph");
  if (!ev || !n_nodes || !n_edges) return fail(LST_ERR_ARG, "null argument");
  lst_ctx c = ev->ctx;
  DeviceGuard gd(c->device);
  lst_status s = wait_event(ev);
  if (s != LST_OK) return s;
  const Slot &S = c->slots[ev->slot];
  const int64_t nm = S.cnt[C_MD], nl = S.cnt[C_LS];
  *n_nodes = nm;
  *n_edges = nl;
  if (ev->status != LST_OK) return fail((lst_status)ev->status, "event has no valid results");
  if (node_cap < nm || edge_cap < nl) return fail(LST_ERR_CAPACITY, "graph capacity below node / edge count");
  if (!row_off) return LST_OK;                                        // size query
  if (nl > 0 && !col) return fail(LST_ERR_ARG, "col is NULL");
  EvDesc *dd;
  s = slot_desc_device(c, ev->slot, &dd);
  if (s != LST_OK) return s;
  const bool dev_out = is_device_ptr(row_off);
  const size_t b_row = 4 * (size_t)(nm + 1), b_col = 4 * (size_t)nl, b_nf = 24 * (size_t)nm, b_ef = 8 * (size_t)nl;
  void *tmp = nullptr;
  int32_t *d_row = row_off, *d_col = col;
  float *d_nf = node_feat, *d_ef = edge_feat;
  if (!dev_out) {
    CU(tmp_alloc(c, &tmp, b_row + b_col + b_nf + b_ef + 1024, c->aux));
    char *p = (char *)tmp;
    d_row = (int32_t *)p; p += align_up(b_row, 256);
    d_col = (int32_t *)p; p += align_up(b_col, 256);
    d_nf = node_feat ? (float *)p : nullptr; p += align_up(b_nf, 256);
    d_ef = edge_feat ? (float *)p : nullptr;
  }
  k_graph_rows<<<1, 1024, 0, c->aux>>>(dd, (int)nm, d_row);
  if (nm > 0) {
    const int grid = (int)std::min<int64_t>((nm + 255) / 256, 4 * c->n_sm);
    k_graph_fill<<<grid, 256, 0, c->aux>>>(dd, c->g, (int)nm, d_row, d_col, d_nf, d_ef);
  }
  CU(cudaGetLastError());
  if (!dev_out) {
    CU(cudaMemcpyAsync(row_off, d_row, b_row, cudaMemcpyDeviceToHost, c->aux));
    if (nl) CU(cudaMemcpyAsync(col, d_col, b_col, cudaMemcpyDeviceToHost, c->aux));
    if (node_feat && nm) CU(cudaMemcpyAsync(node_feat, d_nf, b_nf, cudaMemcpyDeviceToHost, c->aux));
    if (edge_feat && nl) CU(cudaMemcpyAsync(edge_feat, d_ef, b_ef, cudaMemcpyDeviceToHost, c->aux));
    CU(cudaFreeAsync(tmp, c->aux));
  }
  CU(cudaStreamSynchronize(c->aux));
  return LST_OK;
}

lst_status lst_get_t5_features(lst_event ev, float *feat, int64_t capacity, int64_t *n_out) {
  NvtxRange nvtx_range("lst_get_t5_features");
  if (!ev || !n_out) return fail(LST_ERR_ARG, "null argument");
  lst_ctx c = ev->ctx;
  DeviceGuard gd(c->device);
  lst_status s = wait_event(ev);
  if (s != LST_OK) return s;
  const int64_t n = c->slots[ev->slot].cnt[C_T5];
  *n_out = n;
  if (ev->status != LST_OK) return fail((lst_status)ev->status, "event has no valid results");
  if (capacity < n) return fail(LST_ERR_CAPACITY, "output capacity below object count");
  if (n == 0) return LST_OK;
  if (!feat) return fail(LST_ERR_ARG, "feat is NULL");
  EvDesc *dd;
  s = slot_desc_device(c, ev->slot, &dd);
  if (s != LST_OK) return s;
  const int grid = (int)std::min<int64_t>((n + 127) / 128, 4 * c->n_sm);
  if (is_device_ptr(feat)) {
    k_features<<<grid, 128, 0, c->aux>>>(dd, c->g, c->cuts.k_field, feat, (int)n);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->aux));
    return LST_OK;
  }
  void *tmp = nullptr;
  CU(tmp_alloc(c, &tmp, (size_t)n * NFEAT * 4, c->aux));
  k_features<<<grid, 128, 0, c->aux>>>(dd, c->g, c->cuts.k_field, (float *)tmp, (int)n);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(feat, tmp, (size_t)n * NFEAT * 4, cudaMemcpyDeviceToHost, c->aux));
  CU(cudaFreeAsync(tmp, c->aux));
  CU(cudaStreamSynchronize(c->aux));
  return LST_OK;
}

lst_status lst_score_t5(lst_ctx c, const float *feat, int64_t n, int32_t precision, float *score_out,
                        void *cuda_stream) {
  NvtxRange nvtx_range("lst_score_t5");
  if (!c) return fail(LST_ERR_ARG, "null ctx");
  if (n < 0) return fail(LST_ERR_ARG, "n < 0");
  if (precision != LST_FP32 && precision != LST_BF16 && precision != LST_BF16X3)
    return fail(LST_ERR_ARG, "bad precision");
  if (!c->have_geom) return fail(LST_ERR_NOT_READY, "no network loaded");
  if (n == 0) return LST_OK;
  if (!feat || !score_out) return fail(LST_ERR_ARG, "null buffer");
  DeviceGuard gd(c->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (precision != LST_FP32) {
    const bool split = precision == LST_BF16X3;
    const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)c->grid_bf[split]);
    CU(launch_score_bf16_features(grid, st, c->g, c->cuts, c->d_wpack, c->d_w, c->n_hidden, feat, n, score_out,
                                  c->d_err, c->wait_limit, split, c->skip_mma));
  } else {
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->grid_sc);
    k_score_feat_fp32<<<grid, 256, (size_t)c->n_w * 4, st>>>(feat, n, c->d_w, c->n_hidden, score_out);
  }
  CU(cudaGetLastError());
  return LST_OK;
}

// ------------------------------------------------------------------ pixel seeds (steps 5-8)
lst_status lst_match_pixel_seeds_batch(const lst_event *evs, int32_t n, const float *const *seeds,
                                       const int64_t *n_seeds, const lst_pixel_cuts *pc, lst_pixel_counts *counts) {
  NvtxRange nvtx_range("lst_match_pixel_seeds_batch");
  if (!evs || !seeds || !n_seeds || !pc || n < 1) return fail(LST_ERR_ARG, "null argument or n < 1");
  lst_ctx c = evs[0] ? evs[0]->ctx : nullptr;
  if (!c) return fail(LST_ERR_ARG, "null event");
  if (n > (int32_t)c->slots.size()) return fail(LST_ERR_ARG, "more events than the context's slots");
  for (int i = 0; i < n; i++) {
    if (!evs[i] || evs[i]->ctx != c) return fail(LST_ERR_ARG, "events of one context expected");
    for (int j = 0; j < i; j++)
      if (evs[j]->slot == evs[i]->slot) return fail(LST_ERR_ARG, "an event appears twice");
    if (n_seeds[i] < 0 || n_seeds[i] > (int64_t)1 << 26) return fail(LST_ERR_ARG, "n_seeds outside 0..2^26");
    if (n_seeds[i] > 0 && !seeds[i]) return fail(LST_ERR_ARG, "null seeds");
  }
  const float pv[7] = {pc->kappa_rel, pc->kappa_abs, pc->rz_tol, pc->dphi0, pc->dphi_cm, pc->dm_abs, pc->dm_rel};
  for (float v : pv)
    if (!(v >= 0.0f)) return fail(LST_ERR_ARG, "pixel matching parameters must be non-negative numbers");
  DeviceGuard gd(c->device);
  for (int i = 0; i < n; i++) {
    lst_status s = wait_event(evs[i]);
    if (s != LST_OK) return s;
    if (evs[i]->status != LST_OK) return fail((lst_status)evs[i]->status, "event has no valid results");
  }
  cudaStream_t st = c->aux;
  std::vector<PixDesc> P(n);
  std::vector<EvDesc> D(n);
  bool any_seeds = false;
  for (int i = 0; i < n; i++) {
    Slot &S = c->slots[evs[i]->slot];
    S.pix_rows = -1;
    const int np = (int)n_seeds[i], n5 = S.cnt[C_T5], n3 = S.cnt[C_T3], nmd = S.cnt[C_MD];
    const size_t no = (size_t)n5 + n3, npl = std::max(np, 1);
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + std::max<size_t>(b, 1), 256); return o; };
    const size_t o_hits = take(48 * npl), o_cell = take(4 * npl), o_rank = take(4 * npl);
    const size_t o_ccnt = take(4 * (size_t)PIX_NCELL), o_coff = take(4 * ((size_t)PIX_NCELL + 1));
    const size_t o_sa = take(16 * npl), o_sb = take(16 * npl), o_sm = take(4 * npl), o_sk = take(4 * npl), o_sidx = take(4 * npl);
    const size_t o_pkey = take(8 * npl), o_pcnt = take(4 * npl), o_plist = take(4 * (size_t)PIX_TIES * npl);
    const size_t o_pobj = take(4 * npl), o_pmatch = take(4 * npl);
    const size_t o_okey = take(8 * no), o_op = take(4 * no), o_omatch = take(4 * no), o_md = take((size_t)nmd);
    const size_t o_ocnt = take(4 * no), o_oseed = take(4 * (size_t)PIX_OCAP * no), o_okeys = take(8 * (size_t)PIX_OCAP * no);
    const size_t o_rows = take(12 * (no + npl)), o_ctr = take(4 * PIX_NCTR);
    if (S.pix_bytes < off) {
      CU(cudaDeviceSynchronize());
      cudaFree(S.pix_mem);
      S.pix_mem = nullptr;
      S.pix_bytes = 0;
      CU(cudaMalloc(&S.pix_mem, off));
      S.pix_bytes = off;
    }
    char *b = (char *)S.pix_mem;
    PixDesc &Q = P[i];
    Q.n_pls = np; Q.n_t5 = n5; Q.n_t3 = n3; Q.n_md = nmd;
    Q.hits = (const float *)(b + o_hits);
    Q.cell = (int *)(b + o_cell); Q.rank = (int *)(b + o_rank);
    Q.cell_cnt = (int *)(b + o_ccnt); Q.cell_off = (int *)(b + o_coff);
    Q.sa = (float4 *)(b + o_sa); Q.sb = (float4 *)(b + o_sb); Q.sm = (float *)(b + o_sm); Q.sk = (float *)(b + o_sk); Q.sidx = (int *)(b + o_sidx);
    Q.pkey = (unsigned long long *)(b + o_pkey); Q.pcnt = (int *)(b + o_pcnt); Q.plist = (int *)(b + o_plist);
    Q.pobj = (int *)(b + o_pobj); Q.pmatch = (int *)(b + o_pmatch);
    Q.okey = (unsigned long long *)(b + o_okey); Q.op = (int *)(b + o_op); Q.omatch = (int *)(b + o_omatch);
    Q.mdflag = (uint8_t *)(b + o_md); Q.rows = (int *)(b + o_rows); Q.ctr = (int *)(b + o_ctr);
    Q.ocnt = (int *)(b + o_ocnt); Q.oseed = (int *)(b + o_oseed); Q.okeys = (unsigned long long *)(b + o_okeys);
    CU(cudaMemsetAsync(Q.cell_cnt, 0, 4 * (size_t)PIX_NCELL, st));
    CU(cudaMemsetAsync(Q.omatch, 0xff, 4 * std::max<size_t>(no, 1), st));
    CU(cudaMemsetAsync(Q.ocnt, 0xff, 4 * std::max<size_t>(no, 1), st));
    CU(cudaMemsetAsync(Q.mdflag, 0, std::max(nmd, 1), st));
    CU(cudaMemsetAsync(Q.ctr, 0, 4 * PIX_NCTR, st));
    CU(cudaMemsetAsync(Q.ctr + 3, 0x7f, 4, st));          // smallest seed radius: +huge until binned
    if (np) CU(cudaMemcpyAsync(b + o_hits, seeds[i], 48 * (size_t)np, cudaMemcpyDefault, st));
    any_seeds = any_seeds || np > 0;
    D[i] = S.d;
  }
  // device copies of the descriptors and the per-event flags of the rounds
  const size_t b_p = align_up(sizeof(PixDesc) * (size_t)n, 256), b_d = align_up(sizeof(EvDesc) * (size_t)n, 256);
  void *tmp = nullptr;
  CU(tmp_alloc(c, &tmp, b_p + b_d + 4 * (size_t)n, st));
  PixDesc *dP = (PixDesc *)tmp;
  EvDesc *dD = (EvDesc *)((char *)tmp + b_p);
  int *dflags = (int *)((char *)tmp + b_p + b_d);
  CU(cudaMemcpyAsync(dP, P.data(), sizeof(PixDesc) * (size_t)n, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(dD, D.data(), sizeof(EvDesc) * (size_t)n, cudaMemcpyHostToDevice, st));
  const int grid = std::max(1, 2 * c->n_sm / n);
  lst_status res = LST_OK;
  std::vector<int> hflags(n);
  auto run = [&]() -> lst_status {
    CU(pix_launch_bin(dP, n, any_seeds, grid, st));
    for (int stage : {5, 7}) {
      if (stage == 7) {
        CU(pix_launch_mark(dD, dP, n, grid, st));
        CU(pix_launch_rebin(dP, n, any_seeds, grid, st));
      }
      CU(pix_launch_stage_begin(dP, n, stage, st));
      // rounds go out PIX_ROUNDS_PER_WAIT at a time between host waits (a stage takes about
      // three; the kernels of an event that is done return at once)
      for (int round = 0; round < 1 << 20; round += PIX_ROUNDS_PER_WAIT) {
        for (int r = 0; r < PIX_ROUNDS_PER_WAIT; r++) CU(pix_launch_round(dD, dP, n, stage, *pc, grid, dflags, st));
        CU(cudaMemcpyAsync(hflags.data(), dflags, 4 * (size_t)n, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        bool all = true;
        for (int f : hflags) {
          if (f & 2) return fail(LST_ERR_CAPACITY, "more than 8 objects tie at one seed in both ranking measures");
          all = all && (f & 1);
        }
        if (all) break;
      }
    }
    CU(pix_launch_rows(dD, dP, n, grid, st));
    return LST_OK;
  };
  res = run();
  std::vector<int> hctr((size_t)n * PIX_NCTR);
  if (res == LST_OK) {
    for (int i = 0; i < n; i++)
      CU(cudaMemcpyAsync(hctr.data() + (size_t)i * PIX_NCTR, P[i].ctr, 4 * PIX_NCTR, cudaMemcpyDeviceToHost, st));
  }
  cudaFreeAsync(tmp, st);
  CU(cudaStreamSynchronize(st));
  if (res != LST_OK) return res;
  for (int i = 0; i < n; i++) {
    const int *h = hctr.data() + (size_t)i * PIX_NCTR;
    Slot &S = c->slots[evs[i]->slot];
    S.pix_rows = h[1];
    S.pix_rows_ptr = P[i].rows;
    if (counts) {
      counts[i].n_rows = h[1];
      counts[i].n_pt5 = h[4];
      counts[i].n_t5 = h[5];
      counts[i].n_pt3 = h[6];
      counts[i].n_pls = h[7];
      counts[i].rounds_pt5 = h[PIX_ROUNDS5];
      counts[i].rounds_pt3 = h[PIX_ROUNDS7];
    }
  }
  return LST_OK;
}

lst_status lst_match_pixel_seeds(lst_event ev, const float *seeds, int64_t n_seeds, const lst_pixel_cuts *pc,
                                 lst_pixel_counts *counts) {
  if (!ev || !pc) return fail(LST_ERR_ARG, "null event or parameters");
  return lst_match_pixel_seeds_batch(&ev, 1, &seeds, &n_seeds, pc, counts);
}

lst_status lst_get_pixel_candidates(lst_event ev, int32_t *rows, int64_t capacity, int64_t *n_out) {
  NvtxRange nvtx_range("lst_get_pixel_candidates");
  if (!ev || !n_out) return fail(LST_ERR_ARG, "null argument");
  lst_ctx c = ev->ctx;
  DeviceGuard gd(c->device);
  const Slot &S = c->slots[ev->slot];
  *n_out = S.pix_rows < 0 ? 0 : S.pix_rows;
  if (S.pix_rows < 0) return fail(LST_ERR_NOT_READY, "no pixel-seed matching for this event");
  if (capacity < S.pix_rows) return fail(LST_ERR_CAPACITY, "output capacity below the candidate count");
  if (S.pix_rows == 0) return LST_OK;
  if (!rows) return fail(LST_ERR_ARG, "rows is NULL");
  CU(cudaMemcpyAsync(rows, S.pix_rows_ptr, 12 * (size_t)S.pix_rows, cudaMemcpyDefault, c->aux));
  CU(cudaStreamSynchronize(c->aux));
  return LST_OK;
}

lst_status lst_event_release(lst_event ev) {
  if (!ev) return fail(LST_ERR_ARG, "null event");
  lst_ctx c = ev->ctx;
  DeviceGuard gd(c->device);
  Slot &S = c->slots[ev->slot];
  if (!S.have_cnt && S.lane >= 0) lane_harvest(c, c->lanes[S.lane]);
  S.busy = false;
  S.pix_rows = -1;
  delete ev;
  return LST_OK;
}

lst_status lst_destroy(lst_ctx c) {
  if (!c) return fail(LST_ERR_ARG, "null ctx");
  {
    DeviceGuard gd(c->device);
    cudaDeviceSynchronize();
    for (auto &L : c->lanes) {
      for (auto &kv : L.graphs) cudaGraphExecDestroy(kv.second);
      cudaFree(L.d_desc); cudaFreeHost(L.h_desc); cudaFree(L.d_work); cudaFree(L.d_counts);
      cudaFreeHost(L.h_counts);
      if (L.done) cudaEventDestroy(L.done);
      for (auto &e : L.tev) if (e) cudaEventDestroy(e);
      if (L.cap_stream) cudaStreamDestroy(L.cap_stream);
    }
    for (auto &s : c->slots) {
      slot_buf_free(s.mem, 0, s.mem_pooled);
      slot_buf_free(s.in_mem, 0, s.in_pooled);
      cudaFree(s.pix_mem);
    }
    cudaFree(c->d_subdet); cudaFree(c->d_layer); cudaFree(c->d_map_off); cudaFree(c->d_map_tgt);
    cudaFree(c->d_ls_units);
    cudaFree(c->d_w); cudaFree(c->scratch); cudaFree(c->d_wpack); cudaFree(c->d_err);
    if (c->aux) cudaStreamDestroy(c->aux);
    cudaDeviceSynchronize();
    if (c->pool) cudaMemPoolDestroy(c->pool);
  }
  delete c;
  return LST_OK;
}

lst_status lst_get_launch(lst_ctx c, lst_launch *o) {
  if (!c || !o) return fail(LST_ERR_ARG, "null argument");
  *o = lst_launch{c->md_threads, c->md_buf, c->ls_threads, c->ls_list, c->t3_threads, c->t5_threads,
                  c->sc_threads, c->t3_mds};
  return LST_OK;
}

lst_status lst_set_launch(lst_ctx c, const lst_launch *p) {
  if (!c || !p) return fail(LST_ERR_ARG, "null argument");
  const int th[5] = {p->md_threads, p->ls_threads, p->t3_threads, p->t5_threads, p->sc_threads};
  for (int t : th)
    if (t < 32 || t > 256 || t % 32) return fail(LST_ERR_ARG, "threads must be a multiple of 32 in 32..256");
  if (p->md_buf < 1 || p->ls_list < 1) return fail(LST_ERR_ARG, "sizes must be >= 1");
  if (p->t3_mds < 0 || p->t3_mds > 32) return fail(LST_ERR_ARG, "t3_mds outside 0..32");
  DeviceGuard gd(c->device);
  CU(cudaDeviceSynchronize());
  struct { int md_threads, md_buf, ls_threads, ls_list, t3_threads, t5_threads, sc_threads; } old = {
      c->md_threads, c->md_buf, c->ls_threads, c->ls_list, c->t3_threads, c->t5_threads, c->sc_threads};
  c->md_threads = p->md_threads; c->md_buf = p->md_buf;
  c->ls_threads = p->ls_threads; c->ls_list = p->ls_list;
  c->t3_threads = p->t3_threads; c->t5_threads = p->t5_threads;
  c->sc_threads = p->sc_threads;
  c->t3_mds = p->t3_mds;
  int dev_smem = 0;
  CU(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  if (ls_smem(c) > (size_t)dev_smem - 2048 || md_smem(c) > (size_t)dev_smem || t3_smem(c) > (size_t)dev_smem - 4096) {
    c->md_threads = old.md_threads; c->md_buf = old.md_buf; c->ls_threads = old.ls_threads;
    c->ls_list = old.ls_list; c->t3_threads = old.t3_threads;
    c->t5_threads = old.t5_threads; c->sc_threads = old.sc_threads;
    return fail(LST_ERR_ARG, "shared memory of the launch shape exceeds the device limit");
  }
  lst_status s = compute_grids(c);
  if (s != LST_OK) return s;
  for (auto &L : c->lanes) {
    for (auto &kv : L.graphs) cudaGraphExecDestroy(kv.second);
    L.graphs.clear();
  }
  return LST_OK;
}

lst_status lst_device_errors(lst_ctx c) {
  if (!c) return fail(LST_ERR_ARG, "null ctx");
  DeviceGuard gd(c->device);
  int e = 0;
  CU(cudaDeviceSynchronize());
  CU(cudaMemcpy(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost));
  CU(cudaMemset(c->d_err, 0, sizeof e));
  if (e) return fail((lst_status)e, "a bounded device wait ran out (tensor-core score)");
  return LST_OK;
}

lst_status lst_test_fail_alloc(lst_ctx c, int32_t n) {
  if (!c || n < 0) return fail(LST_ERR_ARG, "null ctx or negative count");
  c->fail_allocs.store(n);
  return LST_OK;
}

lst_status lst_test_skip_mma(lst_ctx c, int32_t on) {
  if (!c) return fail(LST_ERR_ARG, "null ctx");
  DeviceGuard gd(c->device);
  CU(cudaDeviceSynchronize());
  c->skip_mma = on ? 1 : 0;
  for (auto &L : c->lanes) {                  // captured graphs hold the old kernel arguments
    for (auto &kv : L.graphs) cudaGraphExecDestroy(kv.second);
    L.graphs.clear();
  }
  return LST_OK;
}

lst_status lst_set_wait_limit(lst_ctx c, int64_t iterations) {
  if (!c || iterations < 1) return fail(LST_ERR_ARG, "null ctx or limit < 1");
  c->wait_limit = iterations;
  for (auto &L : c->lanes) {
    for (auto &kv : L.graphs) cudaGraphExecDestroy(kv.second);
    L.graphs.clear();
  }
  return LST_OK;
}

lst_status lst_set_timing(lst_ctx c, int32_t enable) {
  if (!c) return fail(LST_ERR_ARG, "null ctx");
  c->timing = enable != 0;
  for (double &v : c->stage_sum) v = 0.0;
  c->stage_n = 0;
  return LST_OK;
}

lst_status lst_stage_times(lst_ctx c, float *ms, int64_t *n_launches) {
  if (!c || !ms) return fail(LST_ERR_ARG, "null argument");
  for (int k = 0; k < LST_N_STAGES; k++) ms[k] = c->stage_n ? (float)(c->stage_sum[k] / c->stage_n) : 0.0f;
  if (n_launches) *n_launches = c->stage_n;
  return LST_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- internal accessors
namespace lstk {
// Geometry, cuts and device of a context (false while no geometry is loaded).
bool ctx_geometry(lst_ctx ctx, DevGeom *g, lst_cuts *c, int *device) {
  if (!ctx || !ctx->have_geom) return false;
  *g = ctx->g;
  *c = ctx->cuts;
  *device = ctx->device;
  return true;
}
// Sets the calling thread's lst_last_error text.
void set_last_error(const char *msg) { g_err = msg ? msg : ""; }
}  // namespace lstk

// ================================================================ serving (continuous batching)
// Two worker threads own the context while the server runs. The launcher admits requests
// (host hit arrays) in arrival order while an event slot is free and the estimated
// object-buffer memory of the admitted events stays within the budget, stages their inputs
// and sends them out in batches (one launch per stage over the batch, a CUDA graph captured
// for every batch size when the server starts) on two lanes with their own streams, so a
// batch can start while the previous one is still on the device. The completer waits for
// each launched batch, reads its counters, exports its T5 results to the host and releases
// its slots, so that this host work overlaps the launcher's. Requests that arrive
// meanwhile wait only for a slot and memory, not for the running batch.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServeReq {
  uint64_t tag = 0;
  const float *x = nullptr, *y = nullptr, *z = nullptr;
  const int32_t *sensor = nullptr;
  int64_t n = 0;
  double t_arrival = 0, t_admit = 0, t_launch = 0;
  int slot = -1;
  size_t est = 0;
  int retries = 0;
};

// estimated device bytes of one event: its slot allocation (slot_layout) plus the hit input
// buffer (16 bytes per hit)
size_t est_bytes(const lst_ctx_s *c, int64_t n) {
  int md, ls, t3, t5;
  caps_for(c, n, md, ls, t3, t5);
  const int64_t H = (int64_t)(std::max<int64_t>(n, 1024) * 1.1);
  return slot_layout(H, (size_t)c->g.n_mod, md, ls, t3, t5).total + (size_t)n * 16;
}

}  // namespace

// Pinned host staging of one finished lane batch's T5 results (one batched export). The
// polled results of the batch point into it (no copy) and it returns to the server's pool
// when the last of them has been freed (lst_serve_free_result). A stage whose results
// outlive the server is freed by the last of them.
struct ServeStage {
  int32_t *hits = nullptr;
  float *score = nullptr;
  uint8_t *sel = nullptr;
  int64_t cap = 0;
  std::mutex m;
  int pending = 0;                      // results referring to the stage; guarded by m
  bool orphan = false;                  // the server has stopped; guarded by m
};

namespace {
void stage_free(ServeStage *g) {
  cudaFreeHost(g->hits);
  cudaFreeHost(g->score);
  cudaFreeHost(g->sel);
  delete g;
}
// One result referring to g is gone; frees g if it was the last one of a stopped server.
void stage_release(ServeStage *g) {
  bool last = false;
  {
    std::lock_guard<std::mutex> lk(g->m);
    g->pending--;
    last = g->orphan && g->pending == 0;
  }
  if (last) stage_free(g);
}
}  // namespace

// A finished request: its result, and where its T5 rows sit in a stage (if anywhere).
struct ServeDone {
  lst_serve_result res;
  ServeStage *stage = nullptr;
  int64_t row = 0, n5 = 0;
};

struct lst_server_s {
  lst_ctx c = nullptr;
  lst_serve_config cfg{};
  std::thread th, th_done;              // launcher, completer
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServeReq> submitted;       // guarded by mu
  std::deque<ServeDone> done;           // guarded by mu
  std::vector<ServeStage *> stages;     // every stage; guarded by mu
  bool stop = false;                    // guarded by mu
  std::string error;                    // guarded by mu
  // state of the two workers, guarded by wm: the queues, the lanes' batches, the slots'
  // busy flags, the memory in use and the context's capacity ratios
  std::mutex wm;
  std::condition_variable wcv;
  std::deque<ServeReq> waiting;         // not yet given a slot
  std::deque<ServeReq> ready;           // holds a slot, not launched
  std::vector<ServeReq> inflight[2];    // a lane's batch, from its launch until completed
  std::deque<int> launched;             // lanes in launch order, for the completer
  bool launcher_done = false;
  cudaStream_t st[2] = {nullptr, nullptr};
  size_t mem_in_use = 0;
};

namespace {

// One finished request: its result (counts, times, and where its T5 tuples, scores and
// selection flags sit in the batch's stage, if anywhere) goes to the done queue; the slot and
// its memory budget are released. The stage's pending count was raised by the caller.
void serve_finish(lst_server_s *S, ServeReq &r, lst_status status, const int32_t *cnt, ServeStage *stage,
                  int64_t row, int64_t n5) {
  lst_ctx_s *c = S->c;
  ServeDone d;
  lst_serve_result &res = d.res;
  std::memset(&res, 0, sizeof res);
  res.tag = r.tag;
  res.status = status;
  res.counts.n_hits = r.n;
  if (cnt) {
    res.counts.n_md = cnt[C_MD]; res.counts.n_ls = cnt[C_LS]; res.counts.n_t3 = cnt[C_T3];
    res.counts.n_t5 = cnt[C_T5]; res.counts.n_selected = cnt[C_NSEL]; res.counts.n_tc = cnt[C_NTC];
    res.counts.pairs[0] = (uint32_t)cnt[C_PMD]; res.counts.pairs[1] = (uint32_t)cnt[C_PLS];
    res.counts.pairs[2] = (uint32_t)cnt[C_PT3]; res.counts.pairs[3] = (uint32_t)cnt[C_PT5];
  }
  res.counts.status = status;
  res.t_arrival = r.t_arrival;
  res.t_admit = r.t_admit;
  res.t_launch = r.t_launch;
  res.t_done = now_s();                 // the results are on the host (pinned staging)
  d.stage = stage;
  d.row = row;
  d.n5 = n5;
  {
    std::lock_guard<std::mutex> wl(S->wm);
    c->slots[r.slot].busy = false;
    S->mem_in_use -= std::min(S->mem_in_use, r.est);
  }
  S->wcv.notify_all();
  std::lock_guard<std::mutex> lk(S->mu);
  S->done.push_back(d);
  S->cv.notify_all();
}

// A pinned stage of cap T5 rows (nullptr if the host memory is not available).
ServeStage *stage_new(int64_t cap) {
  ServeStage *g = new ServeStage();
  if (cudaMallocHost(&g->hits, (size_t)cap * 10 * 4) == cudaSuccess &&
      cudaMallocHost(&g->score, (size_t)cap * 4) == cudaSuccess && cudaMallocHost(&g->sel, (size_t)cap) == cudaSuccess) {
    g->cap = cap;
    return g;
  }
  stage_free(g);
  return nullptr;
}

// A stage with room for n T5 rows and no pending results. The server starts with stages
// for full batches; should none fit, a larger one is added (with headroom) and kept: pinned
// allocations are slow and freeing pinned memory waits for the device, so neither happens
// on this path once the stages cover the batches seen.
ServeStage *serve_stage(lst_server_s *S, int64_t n) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    ServeStage *fit = nullptr;
    for (ServeStage *g : S->stages) {
      std::lock_guard<std::mutex> gl(g->m);
      if (g->pending || g->cap < n) continue;
      if (!fit || g->cap < fit->cap) fit = g;           // the smallest that fits
    }
    if (fit) return fit;
  }
  ServeStage *g = stage_new(n + n / 2 + 1024);
  if (!g) return nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  S->stages.push_back(g);
  return g;
}

// Finish the requests of one lane batch: the T5 results of every successful event are
// exported together (lst_get_candidates_batch into a pinned stage: one gather per event on
// the auxiliary stream, one copy, one synchronisation); each request's result then refers
// to its rows of the stage, which lst_serve_poll copies out on the polling thread.
void serve_finish_batch(lst_server_s *S, std::vector<ServeReq> &done, const std::vector<lst_status> &st) {
  lst_ctx_s *c = S->c;
  std::vector<lst_event_s> evs;
  std::vector<int> which;
  int64_t total = 0;
  if (S->cfg.copy_t5) {
    for (size_t k = 0; k < done.size(); k++) {
      const int32_t *cnt = c->slots[done[k].slot].cnt;
      if (st[k] == LST_OK && cnt[C_T5] > 0) {
        evs.push_back(lst_event_s{c, done[k].slot, LST_OK});
        which.push_back((int)k);
        total += cnt[C_T5];
      }
    }
  }
  std::vector<int64_t> offs(evs.size() + 1, 0);
  ServeStage *g = nullptr;
  lst_status xs = LST_OK;
  if (!evs.empty()) {
    g = serve_stage(S, total);
    std::vector<lst_event> hs(evs.size());
    for (size_t i = 0; i < evs.size(); i++) hs[i] = &evs[i];
    xs = g ? lst_get_candidates_batch(hs.data(), (int32_t)hs.size(), LST_T5, g->hits, g->score, g->sel, g->cap,
                                      offs.data())
           : LST_ERR_CUDA;
    if (xs == LST_OK) {
      std::lock_guard<std::mutex> gl(g->m);
      g->pending += (int)which.size();
    }
  }
  size_t j = 0;
  for (size_t k = 0; k < done.size(); k++) {
    const int32_t *cnt = c->slots[done[k].slot].cnt;          // the lane was harvested
    if (j < which.size() && which[j] == (int)k) {
      if (xs == LST_OK)
        serve_finish(S, done[k], st[k], cnt, g, offs[j], offs[j + 1] - offs[j]);
      else
        serve_finish(S, done[k], LST_ERR_CUDA, cnt, nullptr, 0, 0);
      j++;
    } else {
      serve_finish(S, done[k], st[k], cnt, nullptr, 0, 0);
    }
  }
}

// Launcher: admission, input staging and launches. It holds wm while it changes the shared
// state and launches (all asynchronous with pinned inputs); it never waits for the device.
void serve_loop(lst_server_s *S) {
  lst_ctx_s *c = S->c;
  cudaSetDevice(c->device);
  const int nl = std::max(1, std::min(2, S->cfg.lanes));
  for (;;) {
    bool progress = false, stop = false;
    std::vector<ServeReq> incoming, failed;
    std::vector<lst_status> failed_st;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      while (!S->submitted.empty()) {
        incoming.push_back(S->submitted.front());
        S->submitted.pop_front();
      }
      stop = S->stop;
    }
    {
      std::unique_lock<std::mutex> wl(S->wm);
      for (auto &r : incoming) S->waiting.push_back(r);
      progress = !incoming.empty();
      const bool idle = S->waiting.empty() && S->ready.empty() && S->inflight[0].empty() && S->inflight[1].empty();
      if (stop && idle) {
        S->launcher_done = true;
        wl.unlock();
        S->wcv.notify_all();
        break;
      }
      if (idle) {
        wl.unlock();
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->submitted.empty() && !S->stop) S->cv.wait_for(lk, std::chrono::microseconds(200));
        continue;
      }
      // admission: a free slot and room in the memory budget, in arrival order
      while (!S->waiting.empty()) {
        ServeReq &r = S->waiting.front();
        const size_t est = est_bytes(c, r.n);
        const bool fits = S->mem_in_use == 0 || S->mem_in_use + est <= (size_t)S->cfg.mem_budget_bytes;
        const int si = fits ? find_free_slot(c) : -1;
        if (si < 0) break;
        c->slots[si].busy = true;
        r.slot = si;
        r.est = est;
        r.t_admit = now_s();
        S->mem_in_use += est;
        S->ready.push_back(r);
        S->waiting.pop_front();
        progress = true;
      }
      // launch: every free lane takes up to max_batch ready events
      for (int li = 0; li < nl && !S->ready.empty(); li++) {
        if (!S->inflight[li].empty()) continue;
        NvtxRange nvtx_range("serve: stage inputs and launch");
        Lane &L = c->lanes[1 + li];
        std::vector<int> ids;
        std::vector<ServeReq> batch;
        while (!S->ready.empty() && (int)batch.size() < S->cfg.max_batch) {
          batch.push_back(S->ready.front());
          S->ready.pop_front();
        }
        lst_status st = LST_OK;
        for (auto &r : batch) {
          Slot &sl = c->slots[r.slot];
          if (st == LST_OK) st = slot_alloc(c, sl, r.n, S->st[li], true);
          if (st == LST_OK) st = slot_inputs(c, sl, r.x, r.y, r.z, r.sensor, r.n, S->st[li], true);
          ids.push_back(r.slot);
        }
        const double tl = now_s();
        for (auto &r : batch) r.t_launch = tl;
        if (st == LST_OK) st = run_lane(c, L, (int)batch.size(), ids.data(), S->st[li], true, false);
        if (st != LST_OK) {
          for (auto &r : batch) {
            failed.push_back(r);
            failed_st.push_back(st);
          }
          continue;
        }
        S->inflight[li] = std::move(batch);
        S->launched.push_back(li);
        progress = true;
      }
    }
    if (progress) S->wcv.notify_all();
    for (size_t k = 0; k < failed.size(); k++) serve_finish(S, failed[k], failed_st[k], nullptr, nullptr, 0, 0);
    if (!progress && failed.empty()) {
      // nothing to do until a request arrives or the completer frees a lane, a slot or memory
      std::unique_lock<std::mutex> wl(S->wm);
      S->wcv.wait_for(wl, std::chrono::microseconds(100));
    }
  }
}

// Completer: waits for the launched batches in launch order, reads their counters, exports
// their T5 results and releases their slots; events whose object buffers overflowed go back
// to the front of the ready queue with larger buffers.
void serve_complete_loop(lst_server_s *S) {
  lst_ctx_s *c = S->c;
  cudaSetDevice(c->device);
  for (;;) {
    int li;
    std::vector<ServeReq> batch;
    {
      std::unique_lock<std::mutex> wl(S->wm);
      S->wcv.wait(wl, [&] { return !S->launched.empty() || S->launcher_done; });
      if (S->launched.empty()) break;
      li = S->launched.front();
      batch = S->inflight[li];
    }
    Lane &L = c->lanes[1 + li];
    NvtxRange nvtx_range("serve: complete batch");
    const cudaError_t q = cudaEventSynchronize(L.done);
    const lst_status st = q == cudaSuccess ? lane_harvest(c, L) : LST_ERR_CUDA;
    std::vector<ServeReq> fin, retry;
    std::vector<lst_status> fst;
    for (auto &r : batch) {
      Slot &sl = c->slots[r.slot];
      const lst_status es = st != LST_OK ? st : status_of(sl.cnt);
      if (es == LST_ERR_CAPACITY && r.retries < 4) {
        {
          std::lock_guard<std::mutex> wl(S->wm);
          grow_ratios(c, sl, sl.cnt);       // run again with larger buffers
        }
        r.retries++;
        retry.push_back(r);
        continue;
      }
      fin.push_back(r);
      fst.push_back(es);
    }
    if (st != LST_OK) {
      for (auto &r : fin) serve_finish(S, r, st, nullptr, nullptr, 0, 0);
    } else {
      serve_finish_batch(S, fin, fst);
    }
    {
      std::lock_guard<std::mutex> wl(S->wm);
      for (auto it = retry.rbegin(); it != retry.rend(); ++it) S->ready.push_front(*it);
      S->inflight[li].clear();
      S->launched.pop_front();
    }
    S->wcv.notify_all();
  }
}

}  // namespace

extern "C" {

double lst_clock(void) { return now_s(); }

lst_status lst_serve_start(lst_ctx c, const lst_serve_config *cfg, lst_server *out) {
  if (!c || !cfg || !out) return fail(LST_ERR_ARG, "null argument");
  *out = nullptr;
  if (!c->have_geom) return fail(LST_ERR_NOT_READY, "no geometry loaded");
  if (cfg->max_batch < 1 || cfg->max_batch > (int)c->slots.size())
    return fail(LST_ERR_ARG, "max_batch outside 1..max_events");
  if (cfg->mem_budget_bytes <= 0) return fail(LST_ERR_ARG, "mem_budget_bytes <= 0");
  if (cfg->slot_hits < 0 || cfg->slot_hits > 1 << 30) return fail(LST_ERR_ARG, "slot_hits outside 0..2^30");
  DeviceGuard gd(c->device);
  for (auto &L : c->lanes) {
    lst_status s = lane_harvest(c, L);
    if (s != LST_OK) return s;
  }
  for (auto &sl : c->slots)
    if (sl.busy) return fail(LST_ERR_NOT_READY, "release every event before serving");
  // slot buffers of earlier plain allocations go now (freeing them waits for the device),
  // so that served slots grow within the pool only
  for (auto &sl : c->slots) {
    if (sl.mem && !sl.mem_pooled) {
      CU(slot_buf_free(sl.mem, 0, false));
      sl.mem = nullptr;
      sl.bytes = 0;
      sl.hit_cap = 0; sl.md_cap = sl.ls_cap = sl.t3_cap = sl.t5_cap = 0;
    }
    if (sl.in_mem && !sl.in_pooled) {
      CU(slot_buf_free(sl.in_mem, 0, false));
      sl.in_mem = nullptr;
      sl.in_cap = 0;
    }
  }
  if (cfg->slot_hits > 0) {
    for (auto &sl : c->slots) {
      lst_status as = slot_alloc(c, sl, cfg->slot_hits, 0, true);
      if (as != LST_OK) return as;
      if (sl.in_cap < cfg->slot_hits) {
        if (sl.in_mem) CU(slot_buf_free(sl.in_mem, 0, sl.in_pooled));
        sl.in_mem = nullptr;
        sl.in_cap = 0;
        const int64_t cap = (int64_t)(cfg->slot_hits * 1.1) + 1024;
        CU(slot_buf_alloc(c, &sl.in_mem, (size_t)cap * 16, 0, true));
        sl.in_cap = cap;
        sl.in_pooled = true;
      }
    }
    CU(cudaStreamSynchronize(0));
  }
  lst_server_s *S = new lst_server_s();
  S->c = c;
  S->cfg = *cfg;
  for (auto &s : S->st) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto &t : S->st) if (t) cudaStreamDestroy(t);
      delete S;
      return fail(LST_ERR_CUDA, "stream creation");
    }
  }
  // every batch size's graph on every lane now, so that no capture delays a request later
  if (c->cfg.use_graphs) {
    const int nl = std::max(1, std::min(2, cfg->lanes));
    for (int li = 0; li < nl; li++)
      for (int n = 1; n <= cfg->max_batch; n++) {
        cudaGraphExec_t exec;
        const lst_status gs = lane_graph(c, c->lanes[1 + li], n, false, &exec);
        if (gs != LST_OK) {
          for (auto &t : S->st) cudaStreamDestroy(t);
          delete S;
          return gs;
        }
      }
  }
  // pinned staging for the results of full batches, two per lane (batches in flight and
  // results not yet freed by the caller), sized from the PU200-like T5 count per event
  if (cfg->copy_t5) {
    const int nl = std::max(1, std::min(2, cfg->lanes));
    for (int k = 0; k < 2 * nl; k++) {
      ServeStage *g = stage_new((int64_t)cfg->max_batch * 50000);
      if (!g) break;                                   // added later as batches need them
      S->stages.push_back(g);
    }
  }
  S->th = std::thread(serve_loop, S);
  S->th_done = std::thread(serve_complete_loop, S);
  *out = S;
  return LST_OK;
}

lst_status lst_serve_submit(lst_server S, const float *x, const float *y, const float *z, const int32_t *sensor,
                            int64_t n_hits, uint64_t tag, double t_arrival) {
  if (!S) return fail(LST_ERR_ARG, "null server");
  if (n_hits < 0 || n_hits > (int64_t)1 << 30) return fail(LST_ERR_ARG, "n_hits out of range");
  if (n_hits > 0 && (!x || !y || !z || !sensor)) return fail(LST_ERR_ARG, "null hit array");
  ServeReq r;
  r.tag = tag;
  r.x = x; r.y = y; r.z = z; r.sensor = sensor;
  r.n = n_hits;
  r.t_arrival = t_arrival > 0 ? t_arrival : now_s();
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return fail(LST_ERR_NOT_READY, "server is stopping");
  S->submitted.push_back(r);
  S->cv.notify_all();
  return LST_OK;
}

lst_status lst_serve_poll(lst_server S, lst_serve_result *out, int32_t max, int32_t *n_out, int32_t wait_ms) {
  if (!S || !n_out || (max > 0 && !out)) return fail(LST_ERR_ARG, "null argument");
  std::vector<ServeDone> got;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
      S->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
    while ((int)got.size() < max && !S->done.empty()) {
      got.push_back(S->done.front());
      S->done.pop_front();
    }
  }
  // the results point into their batch's stage; lst_serve_free_result releases it
  for (size_t i = 0; i < got.size(); i++) {
    ServeDone &d = got[i];
    lst_serve_result &res = d.res;
    if (d.stage) {
      res.t5_hits = d.stage->hits + d.row * 10;
      res.t5_score = d.stage->score + d.row;
      res.t5_sel = d.stage->sel + d.row;
      res.n_t5 = d.n5;
      res.owner = d.stage;
    }
    out[i] = res;
  }
  *n_out = (int32_t)got.size();
  return LST_OK;
}

lst_status lst_serve_free_result(lst_serve_result *r) {
  if (!r) return fail(LST_ERR_ARG, "null result");
  if (r->owner) stage_release((ServeStage *)r->owner);
  r->owner = nullptr;
  r->t5_hits = nullptr; r->t5_score = nullptr; r->t5_sel = nullptr;
  r->n_t5 = 0;
  return LST_OK;
}

lst_status lst_serve_stop(lst_server S) {
  if (!S) return fail(LST_ERR_ARG, "null server");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  if (S->th_done.joinable()) S->th_done.join();
  for (auto &s : S->st) if (s) cudaStreamDestroy(s);
  // results never polled release their stages now; stages with results still held by
  // the caller are freed by the last lst_serve_free_result
  for (ServeDone &d : S->done)
    if (d.stage) stage_release(d.stage);
  S->done.clear();
  for (ServeStage *g : S->stages) {
    bool now = false;
    {
      std::lock_guard<std::mutex> lk(g->m);
      g->orphan = true;
      now = g->pending == 0;
    }
    if (now) stage_free(g);
  }
  delete S;
  return LST_OK;
}

}  // extern "C"
