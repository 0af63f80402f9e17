// lst_kernels.cu -- steps 0-4 of the LST hot path on sm_103a (arXiv 2403.13166, Section 1,
// Table 1: "each LST step is implemented as a separate kernel, where the track objects of
// interest are built in parallel").
//
// Every kernel works on a batch of events at once (one launch per stage). Stages 1-4 are
// persistent: a fixed grid of CTAs pulls work units (module, MD) from an atomic counter,
// so a launch needs no host knowledge of object counts and can be captured in a graph.
// Candidates that pass are compacted with a warp ballot + popc prefix into a per-warp
// shared-memory list and reserved in the output with ONE atomicAdd per warp and unit, so
// the objects of one unit (the MDs of a module, the LSs of an inner MD, the T3s of a first
// MD) are contiguous and the next stage can enumerate them as ranges.
// Overflow never writes out of bounds: the unit's range is dropped, the overflow flag is
// set and the counter keeps counting, so the host learns the required size.
#include "lst_internal.cuh"

namespace lstk {

// ===================================================================== step 0: hit binning
// The grouping scatters of MDs and T3s (an event has fewer of them than the grid has
// threads) walk the batch GROUP_EV events at a time, each thread taking the same index in
// all of them, so that GROUP_EV independent dependency chains (load -> dependent offset
// load -> store) are in flight per thread. The hit binning walks one event at a time: side
// by side it was slower.
constexpr int GROUP_EV = 4;
// Count hits per sensor. Sensors are keyed as (sensor & 1) * n_mod + module, so that all
// lower-sensor hits come first in the grouped order: key k < n_mod is the lower sensor of
// module k, key n_mod + k its upper sensor. The whole grid walks the batch one event at a
// time, so the sensor histogram (and in k_bin_scatter the output range) being filled is
// one event's and stays in L2. Each hit keeps the value its atomicAdd returned, its rank
// within its sensor. Only the sensor ids are read here; the coordinates are checked by
// k_bin_scatter (an invalid hit voids its event either way).
__global__ void k_bin_count(const EvDesc *__restrict__ evs, int n_events, DevGeom g) {
  const int ns = 2 * g.n_mod, tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int e = 0; e < n_events; e++) {
    const EvDesc &ev = evs[e];
    const int n = ev.n_hits;
    for (int i = tid; i < n; i += st) {
      const int s = __ldg(ev.sensor + i);
      if (s < 0 || s >= ns) {
        atomicOr(ev.cnt + C_FLAGS, F_INPUT);
        continue;
      }
      ev.hit_rank[i] = atomicAdd(ev.sens_cnt + (s & 1) * g.n_mod + (s >> 1), 1);
    }
  }
}

// Exclusive scan of the sensor histogram (one CTA per event).
__global__ void k_bin_scan(const EvDesc *__restrict__ evs, DevGeom g) {
  const EvDesc &ev = evs[blockIdx.x];
  const int ns = 2 * g.n_mod;
  const int per = (ns + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  int local = 0;
  for (int k = 0; k < per; k++)
    if (b0 + k < ns) local += ev.sens_cnt[b0 + k];
  __shared__ int s_warp[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int inc = warp_incl_scan(local);
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int v = lane < nw ? s_warp[lane] : 0;
    const int vi = warp_incl_scan(v);
    if (lane < nw) s_warp[lane] = vi - v;
  }
  __syncthreads();
  int run = s_warp[wid] + inc - local;
  for (int k = 0; k < per; k++) {
    const int s = b0 + k;
    if (s < ns) {
      const int c = ev.sens_cnt[s];
      ev.sens_off[s] = run;
      run += c;
    }
  }
  if (b0 + per >= ns && b0 < ns) ev.sens_off[ns] = run;
  if (ns == 0 && threadIdx.x == 0) ev.sens_off[0] = 0;
}

// Scatter hits into sensor order as float4 (x, y, z, r) with r = sqrtf(x*x + y*y), event
// by event like k_bin_count, each to its sensor's offset plus its rank (no atomics). A hit
// with a non-finite coordinate is placed like any other (the counts stay consistent) and
// voids its event.
__global__ void k_bin_scatter(const EvDesc *__restrict__ evs, int n_events, DevGeom g) {
  const int ns = 2 * g.n_mod, tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int e = 0; e < n_events; e++) {
    const EvDesc &ev = evs[e];
    const int n = ev.n_hits;
    for (int i = tid; i < n; i += st) {
      const int s = __ldg(ev.sensor + i);
      const float x = __ldg(ev.x + i), y = __ldg(ev.y + i), z = __ldg(ev.z + i);
      if (s < 0 || s >= ns) continue;
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(ev.cnt + C_FLAGS, F_INPUT);
      const int key = (s & 1) * g.n_mod + (s >> 1);
      const int pos = ev.sens_off[key] + ev.hit_rank[i];
      ev.hit[pos] = make_float4(x, y, z, sqrtf(x * x + y * y));
      if (s & 1)
        ev.hit_om[pos].x = i;
      else
        ev.hit_om[pos] = make_int2(i, s >> 1);         // one store: index and module
    }
  }
}

// ===================================================================== shared machinery
// The grouping scatters (k_md_scatter, k_ls_scatter, k_t3_scatter) need no atomics: the
// producer counted each object with an atomicAdd on its group's counter and kept the value
// it returned (the object's rank in its group), so the position is the group's start (an
// exclusive scan of the counts) plus the rank. k_ls_scatter walks the batch one event at a
// time with the whole grid, SCATTER_ILP LSs per thread and trip (an event has more LSs than
// the grid has threads), and writes one MD index per LS into each of two lists;
// k_md_scatter and k_t3_scatter take GROUP_EV events side by side.
constexpr int SCATTER_ILP = 8;

// Reserve n output slots: one atomicAdd per warp. Returns the base or -1 if the buffer
// would overflow (then the flag is set; the counter still records the demand).
__device__ __forceinline__ int warp_reserve(int *counter, int *flags, int flag, int n, int cap) {
  int base = 0;
  if ((threadIdx.x & 31) == 0 && n > 0) {
    base = atomicAdd(counter, n);
    if (base + n > cap) {
      atomicOr(flags, flag);
      base = -1;
    }
  }
  return __shfl_sync(FULL, base, 0);
}

// ===================================================================== step 1: mini-doublets
// One lane per lower-sensor hit. Binning puts the lower-sensor hits of all modules first,
// so warps take 32 consecutive lower hits (static striding over all events) and the pairs
// of a dense module spread over many warps. Each lane loops over the upper-sensor hits of
// its own module; pairs that pass md_prefilter are queued per warp and the exact cut runs
// on full warps of queued pairs. MDs are appended in any order (one atomicAdd per warp and
// ballot) and counted per module; a counting sort (k_md_scan, k_md_scatter) then groups
// them by module.
struct MdWarp {
  float4 L[32];
  int lo[32], mod[32], endc[32];
  int qx[64], qu[64];   // queue of (lane, upper hit) pairs that passed md_prefilter
};

__global__ void __launch_bounds__(256) k_md(const EvDesc *__restrict__ evs, int n_events, DevGeom g,
                                           lst_cuts c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  MdWarp &w = reinterpret_cast<MdWarp *>(smem_raw)[wid];
  const int nm = g.n_mod;
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return (ev.cnt[C_FLAGS] & F_INPUT) ? 0 : (ev.sens_off[nm] + 31) / 32;
  }, s_pref);
  const int total = s_pref[n_events];
  const int W = gridDim.x * nwarps;
  int cur = -1, acc = 0;
  for (int u = blockIdx.x * nwarps + wid; u < total; u += W) {
    const int e = find_event(s_pref, n_events, u);
    if (e != cur) {
      if (cur >= 0 && lane == 0 && acc) atomicAdd(evs[cur].cnt + C_PMD, acc);
      acc = 0;
      cur = e;
    }
    const EvDesc &ev = evs[e];
    const int h = (u - s_pref[e]) * 32 + lane;
    int nup = 0, up0 = 0;
    bool endcap = false;
    float4 L = make_float4(0.f, 0.f, 0.f, 1.f);
    MdLow q{};
    if (h < ev.sens_off[nm]) {
      const int m = ev.hit_om[h].y;
      up0 = ev.sens_off[nm + m];
      nup = ev.sens_off[nm + m + 1] - up0;
      endcap = g.subdet[m] != 0;
      L = ev.hit[h];
      q = md_low(L, endcap, c);
      w.L[lane] = L;
      w.lo[lane] = h;
      w.mod[lane] = m;
      w.endc[lane] = endcap;
    }
    int mx = nup, sum = nup;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      mx = max(mx, __shfl_xor_sync(FULL, mx, o));
      sum += __shfl_xor_sync(FULL, sum, o);
    }
    acc += sum;
    // exact cut on queued pairs [q0, q0 + n)
    auto run_queue = [&](int q0, int n) {
      bool pass = false;
      float kc = 0.0f, kf = 0.0f;
      int x = 0, uh = 0;
      if (lane < n) {
        x = w.qx[q0 + lane];
        uh = w.qu[q0 + lane];
        const float4 LL = w.L[x], U = ev.hit[uh];
        const bool ec = w.endc[x] != 0;
        pass = md_cut(LL, U, ec, c, kc);
        if (pass && !ec) kf = md_kappa_acc(LL, U);
      }
      const unsigned bal = __ballot_sync(FULL, pass);
      if (bal) {
        const int base = warp_reserve(ev.cnt + C_MD, ev.cnt + C_FLAGS, F_OVF_MD, __popc(bal), ev.md_cap);
        if (pass && base >= 0) {
          const int o = base + __popc(bal & lanemask_lt());
          if (chk(ev, o, ev.md_cap, 11)) {
            ev.mdu_anchor[o] = w.L[x];
            ev.mdu_kappa[o] = make_float2(kc, kf);
            ev.mdu_mod[o] = w.mod[x];
            ev.mdu_hits[o] = make_int2(ev.hit_om[w.lo[x]].x, ev.hit_om[uh].x);
            ev.mdu_rank[o] = atomicAdd(ev.md_cnt + w.mod[x], 1);
          }
        }
      }
    };
    __syncwarp();
    int qlen = 0;
    // each lane tests its lower hit against the upper hits of its module 32 at a time (the
    // next upper hit loaded while the current pair is tested), collecting the survivors as a
    // bit mask with no warp-wide step in the loop; the masks are then drained into the queue
    for (int j0 = 0; j0 < mx; j0 += 32) {
      unsigned mask = 0;
      const int jn = min(nup - j0, 32);
      if (jn > 0) {
        float4 Unext = ev.hit[up0 + j0];
        for (int j = 0; j < jn; j++) {
          const float4 U = Unext;
          if (j + 1 < jn) Unext = ev.hit[up0 + j0 + j + 1];
          mask |= (md_prefilter(L, U, endcap, q, c) ? 1u : 0u) << j;
        }
      }
      for (;;) {
        const unsigned act = __ballot_sync(FULL, mask != 0);
        if (act == 0) break;
        if (mask != 0) {
          const int j = __ffs(mask) - 1;
          mask &= mask - 1;
          const int qi = qlen + __popc(act & lanemask_lt());
          w.qx[qi] = lane;
          w.qu[qi] = up0 + j0 + j;
        }
        qlen += __popc(act);
        if (qlen >= 32) {
          __syncwarp();
          run_queue(qlen - 32, 32);
          qlen -= 32;
          __syncwarp();
        }
      }
    }
    __syncwarp();
    if (qlen > 0) run_queue(0, qlen);
    __syncwarp();
  }
  if (cur >= 0 && lane == 0 && acc) atomicAdd(evs[cur].cnt + C_PMD, acc);
}

// MDs grouped by module: exclusive scan of the per-module counts (one CTA per event) ...
__global__ void k_md_scan(const EvDesc *__restrict__ evs, DevGeom g) {
  const EvDesc &ev = evs[blockIdx.x];
  if (ev_void(ev)) return;
  const int n = g.n_mod;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  int local = 0;
  for (int k = 0; k < per && b0 + k < n; k++) local += ev.md_cnt[b0 + k];
  __shared__ int s_w[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int inc = warp_incl_scan(local);
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    const int v = lane < nw ? s_w[lane] : 0;
    const int vi = warp_incl_scan(v);
    if (lane < nw) s_w[lane] = vi - v;
  }
  __syncthreads();
  int run = s_w[wid] + inc - local;
  for (int k = 0; k < per && b0 + k < n; k++) {
    ev.md_start[b0 + k] = run;
    run += ev.md_cnt[b0 + k];
  }
}

// ... then a scatter into module order: each MD's index (as found) and key to its module's
// start plus the rank the producer drew when it counted the MD ...
__global__ void __launch_bounds__(256) k_md_scatter(const EvDesc *__restrict__ evs, int n_events) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int e0 = 0; e0 < n_events; e0 += GROUP_EV) {
    int n[GROUP_EV], nmax = 0;
#pragma unroll
    for (int k = 0; k < GROUP_EV; k++) {
      n[k] = 0;
      if (e0 + k < n_events) {
        const EvDesc &ev = evs[e0 + k];
        n[k] = ev_void(ev) ? 0 : clamp_count(ev.cnt[C_MD], ev.md_cap);
      }
      nmax = max(nmax, n[k]);
    }
    for (int o = tid; o < nmax; o += st) {
      int m[GROUP_EV], pos[GROUP_EV];
#pragma unroll
      for (int k = 0; k < GROUP_EV; k++)
        if (o < n[k]) { m[k] = evs[e0 + k].mdu_mod[o]; pos[k] = evs[e0 + k].mdu_rank[o]; }
#pragma unroll
      for (int k = 0; k < GROUP_EV; k++)
        if (o < n[k]) pos[k] += evs[e0 + k].md_start[m[k]];
#pragma unroll
      for (int k = 0; k < GROUP_EV; k++) {
        const EvDesc &ev = evs[e0 + k];
        if (o >= n[k] || !chk(ev, pos[k], ev.md_cap, 14)) continue;
        ev.md_perm[pos[k]] = o;
        ev.md_q[pos[k]] = md_key(ev.mdu_anchor[o]);
        ev.md_mod[pos[k]] = m[k];
      }
    }
  }
}

// ... and within each module the MDs in ascending md_key (ties: lower, then upper hit
// index, so the order is reproducible), moved into place. Step 2 relies on that order: its
// cut's luminous-region road, divided by rA rB, bounds |qA - qB|, so for a group of
// targets the inner MDs that can pass form one run of a module's list. A CTA takes a tile
// of MD_SORT_TILE consecutive positions of one event with their keys in shared memory;
// each thread ranks its MDs by counting the smaller keys of their module's range (keys of a
// module that crosses the tile's edge come from global memory).
constexpr int MD_SORT_TILE = 1024;
__global__ void __launch_bounds__(256) k_md_sort(const EvDesc *__restrict__ evs, int n_events) {
  __shared__ int s_pref[MAX_EVENTS + 1];
  __shared__ float s_q[MD_SORT_TILE];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void(ev) ? 0 : (clamp_count(ev.cnt[C_MD], ev.md_cap) + MD_SORT_TILE - 1) / MD_SORT_TILE;
  }, s_pref);
  const int total = s_pref[n_events];
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int e = find_event(s_pref, n_events, u);
    const EvDesc &ev = evs[e];
    const int n = clamp_count(ev.cnt[C_MD], ev.md_cap);
    const int p0 = (u - s_pref[e]) * MD_SORT_TILE, p1 = min(n, p0 + MD_SORT_TILE);
    __syncthreads();                                   // the previous tile's readers are done
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) s_q[p - p0] = ev.md_q[p];
    __syncthreads();
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const int m = ev.md_mod[p];
      const int s0 = ev.md_start[m], cn = ev.md_cnt[m];
      const int op = ev.md_perm[p];
      if (!chk(ev, op, ev.md_cap, 16) || !chk(ev, (long long)s0 + cn - 1, ev.md_cap, 15)) continue;
      const float kp = s_q[p - p0];
      const int2 hp = ev.mdu_hits[op];
      int r = 0;
      for (int j = s0; j < s0 + cn; j++) {
        const float kj = (j >= p0 && j < p1) ? s_q[j - p0] : ev.md_q[j];
        if (kj < kp) {
          r++;
        } else if (kj == kp && j != p) {
          const int oj = ev.md_perm[j];
          const int2 hj = chk(ev, oj, ev.md_cap, 17) ? ev.mdu_hits[oj] : hp;
          r += (hj.x < hp.x || (hj.x == hp.x && hj.y < hp.y)) ? 1 : 0;
        }
      }
      const int d = s0 + r;
      ev.md_anchor[d] = ev.mdu_anchor[op];
      ev.md_kappa[d] = ev.mdu_kappa[op];
      ev.md_hits[d] = hp;
    }
  }
}

// ===================================================================== step 2: line segments
// Warp minimum / maximum of finite floats in one redux each: the map from a float's bits to
// a signed integer that flips the magnitude bits of negative values preserves their order.
__device__ __forceinline__ int float_order_key(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float warp_min_float(float f) {
  return __int_as_float(float_order_key(__int_as_float(__reduce_min_sync(FULL, float_order_key(f)))));
}
__device__ __forceinline__ float warp_max_float(float f) {
  return __int_as_float(float_order_key(__int_as_float(__reduce_max_sync(FULL, float_order_key(f)))));
}

// One warp per (event, module m); the warps of a CTA never wait for one another. The
// targets (all MDs of the modules linked to m by the module map) are spread over the lanes
// 32 at a time and held in registers; the inner MDs of m sit in the warp's shared memory
// in chunks of LS_IN_CHUNK and are read as broadcasts. MDs are sorted by q = z / r within
// their module (k_md_sort), so for each group of 32 targets only a run of the chunk can pass
// the luminous-region road (a window on q);
// every (inner, target) pair of that run goes through the division-free necessary test;
// the survivors (~9% of all pairs) are queued and, 32 at a time,
// through the necessary curvature-consistency test (~1.8% of all pairs pass), whose survivors
// wait in a second queue that lives for the whole unit and run through the exact FP32 cut
// 32 at a time. LSs go out in any order, each with its ranks among the LSs of its inner and
// of its outer MD (the values of the counting atomicAdds); k_ls_scan / k_ls_scatter then
// list every LS by inner MD (its outer MD) and by outer MD (its inner MD).
constexpr int LS_IN_CHUNK = 64;
constexpr int LS_QCAP = 320;             // pairs the first queue holds (a sub-chunk's survivors at once)
constexpr int LS_WINDOW_MIN = 8;         // chunks of more inner MDs than this are windowed
constexpr int LS_TB = 160;                 // target modules per batch of the warp's table
struct LsWarp {
  float4 in[LS_IN_CHUNK];                  // inner anchors
  float2 inx[LS_IN_CHUNK];                 // rA^2, e rA + slack (ls_prefilter)
  float4 B[32];                            // the 32 targets of the current group
  int2 q2[64];                             // pairs past the curvature test: inner MD, target MD
                                           // (bit 31: target in the barrel), global indices
  float ink[LS_IN_CHUNK];                  // inner MD curvatures (cut values)
  float inq[LS_IN_CHUNK];                  // inner keys q = z / r (ascending: MDs are sorted by q)
  float kB[32];
  int md[32];
  int tpref[LS_TB + 4];                    // MD-count prefix over the target modules
  int tstart[LS_TB];
  unsigned short q[LS_QCAP];               // queued pairs: inner index << 5 | target lane
  unsigned char bB[32];
  unsigned char tbar[LS_TB];
};
static_assert(sizeof(LsWarp) == 5456, "the host sizes k_ls shared memory with 5456 bytes per warp");

// Units: with unit_off == nullptr one unit per module (all its targets); otherwise
// unit_off[m] .. unit_off[m + 1] are the units of module m, unit b taking the target
// modules [b tbu, (b + 1) tbu) of its list (upe = units per event). LSs go out unordered,
// so a module's pairs may be split over units freely.
__global__ void __launch_bounds__(256) k_ls(const EvDesc *__restrict__ evs, int n_events, DevGeom g,
                                           lst_cuts c, int *work, const int32_t *__restrict__ unit_off, int upe,
                                           int tbu) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  LsWarp &w = reinterpret_cast<LsWarp *>(smem_raw)[wid];
  const int total = n_events * upe;
  const float k0 = 1.002f * 65.0f * (c.hit_err * c.hit_err), c1 = c.z_lum + c.hit_err;
  const float Gp = 2.0f * (c.hit_err / c.sensor_gap) * 1.000001f, ce = 2.0f * c.hit_err * 1.000001f;
  for (;;) {
    // lane 0 fetches the unit and reads the event's state once for the warp (other warps
    // may set the overflow flag at any time; all lanes must take the same path)
    int u = 0, n_in = 0, m = 0, ub = 0;
    if (lane == 0) {
      u = atomicAdd(work, 1);
      if (u < total) {
        const int ee = u / upe, v = u - ee * upe;
        if (unit_off) {
          int lo = 0, hi = g.n_mod;                    // last m with unit_off[m] <= v
          while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (unit_off[mid] <= v) lo = mid; else hi = mid - 1; }
          m = lo;
          ub = v - unit_off[m];
        } else {
          m = v;
        }
        const EvDesc &evv = evs[ee];
        n_in = ev_void_before(evv, F_OVF_MD) ? 0 : evv.md_cnt[m];
      }
    }
    u = __shfl_sync(FULL, u, 0);
    n_in = __shfl_sync(FULL, n_in, 0);
    m = __shfl_sync(FULL, m, 0);
    ub = __shfl_sync(FULL, ub, 0);
    if (u >= total) break;
    if (n_in == 0) continue;
    const int e = u / upe;
    const EvDesc &ev = evs[e];
    const int in0 = ev.md_start[m];
    const bool bA = g.subdet[m] == 0;
    const int t0 = g.map_off[m], nt_all = min(g.map_off[m + 1] - t0, MAX_FANOUT);
    const int tb0 = unit_off ? ub * tbu : 0, tb1 = unit_off ? min(nt_all, tb0 + tbu) : nt_all;
    int pairs = 0;
    int q2n = 0;
    // exact cut of the first n pairs of the second queue (one per lane); LSs out in any order,
    // each with its ranks among the LSs of its inner and of its outer MD
    auto run_exact = [&](int n) {
      bool pass = false;
      int gi = 0, gm = 0;
      if (lane < n) {
        const int2 qe = w.q2[lane];
        gi = qe.x;
        gm = qe.y & 0x7fffffff;
        float k;
        pass = ls_cut(ev.md_anchor[gi], ev.md_anchor[gm], ev.md_kappa[gi].x, ev.md_kappa[gm].x, bA, qe.y < 0, c, k);
      }
      const unsigned bal = __ballot_sync(FULL, pass);
      if (bal == 0) return;
      const int base = warp_reserve(ev.cnt + C_LS, ev.cnt + C_FLAGS, F_OVF_LS, __popc(bal), ev.ls_cap);
      if (pass && base >= 0) {
        const int o = base + __popc(bal & lanemask_lt());
        ev.lsu[o] = make_int4(gi, gm, atomicAdd(ev.ls_cnt + gi, 1), atomicAdd(ev.lso_cnt + gm, 1));
      }
    };
    for (int b0 = tb0; b0 < tb1; b0 += LS_TB) {
      const int nb = min(LS_TB, tb1 - b0);
      __syncwarp();                                    // the previous batch's readers are done
      int S = 0;
      for (int b = 0; b < nb; b += 32) {
        const int t = b + lane;
        int cnt = 0, st = 0, bar = 0;
        if (t < nb) {
          const int mt = g.map_tgt[t0 + b0 + t];
          cnt = ev.md_cnt[mt];
          st = ev.md_start[mt];
          bar = g.subdet[mt] == 0;
        }
        const int inc = warp_incl_scan(cnt);
        if (t < nb) { w.tpref[t + 1] = S + inc; w.tstart[t] = st; w.tbar[t] = bar; }
        S += __shfl_sync(FULL, inc, 31);
      }
      if (lane == 0) w.tpref[0] = 0;
      __syncwarp();
      pairs += S;
      if (S == 0) continue;
      for (int c0 = 0; c0 < n_in; c0 += LS_IN_CHUNK) {
        const int nc = min(LS_IN_CHUNK, n_in - c0);
        __syncwarp();                                  // the previous chunk's readers are done
        // padded to a multiple of 4 with NaN anchors, which fail every comparison of the test
        const int nc4 = (nc + 3) & ~3;
        float rmin = 3.0e38f, rmax = 0.0f;
        for (int t = lane; t < nc4; t += 32) {
          if (t < nc) {
            const float4 A = ev.md_anchor[in0 + c0 + t];
            w.in[t] = A;
            w.inx[t] = make_float2(A.w * A.w, c.hit_err * A.w + 0.05f);
            w.ink[t] = ev.md_kappa[in0 + c0 + t].x;
            w.inq[t] = md_key(A);
            rmin = fminf(rmin, A.w);
            rmax = fmaxf(rmax, A.w);
          } else {
            const float nan = __int_as_float(0x7fc00000);
            w.in[t] = make_float4(nan, nan, nan, nan);
            w.inx[t] = make_float2(nan, nan);
            w.ink[t] = 0.0f;
            w.inq[t] = nan;
          }
        }
        rmin = warp_min_float(rmin);
        rmax = warp_max_float(rmax);
        const float irmin = __fdividef(1.0f, rmin), irmax = __fdividef(1.0f, rmax);
        __syncwarp();
        int tg = 0;                                    // target module of the group's first target
        for (int j0 = 0; j0 < S; j0 += 32) {
          const int j = j0 + lane;
          bool valid = j < S;
          float4 B = make_float4(0.f, 0.f, 0.f, 0.f);
          float kB = 0.0f, k1 = 0.0f;
          bool bB = false;
          int md = 0;
          while (w.tpref[tg + 1] <= j0) tg++;          // warp-uniform; tpref[nb] = S > j0
          if (valid) {
            int t = tg;                                // the last t with tpref[t] <= j: a group
            while (w.tpref[t + 1] <= j) t++;           // spans a few target modules
            md = w.tstart[t] + (j - w.tpref[t]);
            if (chk(ev, md, ev.md_cap, 21)) {
              B = ev.md_anchor[md];
              kB = ev.md_kappa[md].x;
              bB = w.tbar[t] != 0;
              const float X = B.w * (0.5f * c.kappa_max);
              k1 = 1.002f * 1.015625f * X * X;
            } else {
              valid = false;
            }
          }
          __syncwarp();                                // the previous group's queue readers are done
          w.B[lane] = B;
          w.kB[lane] = kB;
          w.md[lane] = md;
          w.bB[lane] = bB ? 1 : 0;
          __syncwarp();
          // curvature test of the first n queued pairs; survivors join the second queue
          auto run_kappa = [&](int off, int n) {       // the queued pairs [off, off + n)
            bool pass = false;
            int2 ent = make_int2(0, 0);
            if (lane < n) {
              const int qe = w.q[off + lane];
              const int ie = qe >> 5, le = qe & 31;
              const bool b2 = w.bB[le] != 0;
              pass = ls_kappa_prefilter(w.in[ie], w.B[le], w.ink[ie], w.kB[le], bA, b2, Gp, ce);
              ent = make_int2(in0 + c0 + ie, b2 ? (w.md[le] | (int)0x80000000u) : w.md[le]);
            }
            const unsigned bal = __ballot_sync(FULL, pass);
            if (pass) w.q2[q2n + __popc(bal & lanemask_lt())] = ent;
            q2n += __popc(bal);
            if (q2n >= 32) {
              __syncwarp();
              run_exact(32);
              __syncwarp();
              if (lane + 32 < q2n) w.q2[lane] = w.q2[lane + 32];
              __syncwarp();
              q2n -= 32;
            }
          };
          // The luminous-region road of ls_cut, |A.z rB - rA B.z| <= c1 |rB - rA| + e rA (the
          // cut's left side equals A.z rB - rA B.z in real arithmetic), divided by rA rB > 0
          // reads |qA - qB| <= c1 |1/rA - 1/rB| + e / rB with q = z / r, and |1/rA - 1/rB| is
          // largest at an end of the chunk's [rmin, rmax]. So only inner MDs whose key lies
          // in the union of the group's windows qB -+ wB can pass, one run [ilo, ihi) of the
          // sorted chunk. Slack: 0.05 / (rA rB) covers the cut's FP32 rounding of either side
          // (below 0.02: every product is below 3.2e4 in magnitude), 1e-3 wB + 1e-5 (1 + |qB|)
          // the rounding of q and of the window (approximate reciprocals and quotients, a
          // few ulp). Small chunks are taken whole.
          int ilo = 0, ihi = nc;
          if (nc > LS_WINDOW_MIN) {
            float qlo = 3.0e38f, qhi = -3.0e38f;
            if (valid) {
              const float ib = __fdividef(1.0f, B.w);
              const float qB = B.z * ib;
              const float wB = c1 * fmaxf(fabsf(irmin - ib), fabsf(irmax - ib)) + c.hit_err * ib;
              const float sl = 1e-3f * wB + 0.05f * irmin * ib + 1e-5f * (1.0f + fabsf(qB));
              qlo = qB - wB - sl;
              qhi = qB + wB + sl;
            }
            qlo = warp_min_float(qlo);
            qhi = warp_max_float(qhi);
            // positions in the sorted chunk: keys below qlo, keys up to qhi
            const float a0 = w.inq[lane];
            ilo = __popc(__ballot_sync(FULL, lane < nc && a0 < qlo));
            ihi = __popc(__ballot_sync(FULL, lane < nc && a0 <= qhi));
            if (nc > 32) {
              const float a1 = w.inq[lane + 32];
              ilo += __popc(__ballot_sync(FULL, lane + 32 < nc && a1 < qlo));
              ihi += __popc(__ballot_sync(FULL, lane + 32 < nc && a1 <= qhi));
            }
          }
          const int ib4 = ilo & ~3, ie4 = ihi > ilo ? min(nc4, (ihi + 3) & ~3) : ib4;
          // each lane tests its target against the inner MDs of the run 32 at a time,
          // collecting the survivors as a bit mask (no warp-wide step in the loop), then the
          // masks are drained into the queue, one pair per lane and round
          int qn = 0;
          for (int i0 = ib4; i0 < ie4; i0 += 32) {
            const int n4 = min(32, ie4 - i0);
            unsigned mask = 0;
            if (valid) {
              for (int i = 0; i < n4; i += 4) {
                unsigned bits = 0;
#pragma unroll
                for (int k = 0; k < 4; k++)
                  bits |= ls_prefilter(w.in[i0 + i + k], w.inx[i0 + i + k], B, k1, k0, c1) ? 1u << k : 0u;
                mask |= bits << i;
              }
            }
            // the sub-chunk's survivors into the queue at once: each lane writes its own after
            // the warp's prefix of the counts; then the curvature test on full runs of 32
            const int cntl = __popc(mask);
            const int incl = warp_incl_scan(cntl);
            const int T = __shfl_sync(FULL, incl, 31);
            if (qn + T <= LS_QCAP) {
              int pos = qn + incl - cntl;
              while (mask != 0) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1;
                w.q[pos++] = (unsigned short)(((i0 + i) << 5) | lane);
              }
              qn += T;
              __syncwarp();
              int off = 0;
              for (; qn - off >= 32; off += 32) {
                run_kappa(off, 32);
                __syncwarp();
              }
              if (off > 0) {                           // the rest (< 32) to the front
                const unsigned short v = lane < qn - off ? w.q[off + lane] : 0;
                __syncwarp();
                if (lane < qn - off) w.q[lane] = v;
                __syncwarp();
                qn -= off;
              }
            } else {                                   // too many at once: one per lane and round
              for (;;) {
                const unsigned act = __ballot_sync(FULL, mask != 0);
                if (act == 0) break;
                if (mask != 0) {
                  const int i = __ffs(mask) - 1;
                  mask &= mask - 1;
                  w.q[qn + __popc(act & lanemask_lt())] = (unsigned short)(((i0 + i) << 5) | lane);
                }
                qn += __popc(act);
                if (qn >= 32) {
                  __syncwarp();
                  run_kappa(0, 32);
                  __syncwarp();
                  if (lane + 32 < qn) w.q[lane] = w.q[lane + 32];
                  __syncwarp();
                  qn -= 32;
                }
              }
            }
          }
          if (qn > 0) {
            __syncwarp();
            run_kappa(0, qn);
          }
        }
      }
    }
    if (q2n > 0) {
      __syncwarp();
      run_exact(q2n);
    }
    if (lane == 0 && pairs) atomicAdd(ev.cnt + C_PLS, n_in * pairs);
  }
}

// LSs per inner MD and per outer MD -> ranges (two CTAs per event, one per list) ...
__global__ void k_ls_scan(const EvDesc *__restrict__ evs) {
  const EvDesc &ev = evs[blockIdx.x >> 1];
  if (ev_void(ev)) return;
  const int n = clamp_count(ev.cnt[C_MD], ev.md_cap);
  if (blockIdx.x & 1)
    block_exclusive_scan(ev.lso_cnt, ev.lso_start, n);
  else
    block_exclusive_scan(ev.ls_cnt, ev.ls_start, n);
}

// ... then each LS into both lists at the range start plus the rank k_ls drew: under its
// inner MD the outer MD's index, under its outer MD the inner MD's index.
__global__ void __launch_bounds__(256) k_ls_scatter(const EvDesc *__restrict__ evs, int n_events) {
  const int64_t tid = blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  for (int e = 0; e < n_events; e++) {
    const EvDesc &ev = evs[e];
    if (ev_void(ev)) continue;
    const int64_t n = clamp_count(ev.cnt[C_LS], ev.ls_cap);
    for (int64_t o0 = tid; o0 < n; o0 += SCATTER_ILP * st) {
      int4 r[SCATTER_ILP];
      int pi[SCATTER_ILP], po[SCATTER_ILP];
#pragma unroll
      for (int k = 0; k < SCATTER_ILP; k++)
        if (o0 + k * st < n) r[k] = ev.lsu[o0 + k * st];
#pragma unroll
      for (int k = 0; k < SCATTER_ILP; k++)
        if (o0 + k * st < n) {
          pi[k] = ev.ls_start[r[k].x] + r[k].z;
          po[k] = ev.lso_start[r[k].y] + r[k].w;
        }
#pragma unroll
      for (int k = 0; k < SCATTER_ILP; k++)
        if (o0 + k * st < n) {
          if (chk(ev, pi[k], ev.ls_cap, 24)) ev.ls_to[pi[k]] = r[k].y;
          if (chk(ev, po[k], ev.ls_cap, 25)) ev.ls_from[po[k]] = r[k].x;
        }
    }
  }
}

// ===================================================================== step 3: triplets
// A T3 is a pair (LS1, LS2) that shares its middle MD m (LS1.out == LS2.in == m), so the
// candidate pairs of m are I(m) x O(m): I(m) the LSs ending at m (their inner MDs in list
// ls_from), O(m) those starting at m (their outer MDs in list ls_to). The prefilter needs
// only the two chords P1 - P0 and P2 - P1, formed once per LS and middle MD from the MD
// anchors (the FP32 differences the cut itself forms), so no candidate pair touches global
// memory. A warp takes a unit of mdu (<= 32) consecutive middle MDs of one event (units
// pulled from a counter); MDs lacking I or O items drop out of both sides. The unit's O
// items are staged in the warp's shared memory in windows of T3_OCAP, the I items of the MDs
// meeting the window in chunks of T3_ICAP (all loads of a lane in flight at once); then each
// lane takes an I item and loops over its own MD's O items in the window. Survivors are kept
// as bit masks, drained into a warp queue of MD triples and run through the exact FP32 cut
// 32 at a time with their anchors gathered by MD index.
constexpr int T3_OCAP = 128, T3_ICAP = 96;
struct T3Warp {
  float4 O[T3_OCAP];          // window's O items: chord P2 - P1 (bx, by, bz) and |(bx, by)|
  float4 I[T3_ICAP];          // chunk's I items: chord P1 - P0 (ax, ay, az) and |(ax, ay)|
  float4 P1[32];              // anchors of the unit's middle MDs
  int omd[T3_OCAP];           // outer MD of each O item (md2)
  int imd[T3_ICAP];           // inner MD of each I item (md0)
  int ioff[33], ooff[33];     // exclusive prefixes over the unit's MDs of the I and O counts
  int ist[32], ost[32];       // each MD's start in ls_from and in ls_to
  int q0[64], q1[64], q2[64]; // queued MD triples
};
static_assert(sizeof(T3Warp) == 6288, "the host sizes k_t3 shared memory with 6288 bytes per warp");

// the last k in [0, 31] with off[k] <= f, for non-decreasing off[0..32], off[0] <= f < off[32]
__device__ __forceinline__ int t3_owner(const int *off, int f) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1)
    if (off[lo + step] <= f) lo += step;
  return lo;
}

// Stage items [f0, f1) of a unit's flat item space into shared memory: item f belongs to
// the unit's MD k = t3_owner(off, f), its far MD is list[st[k] + f - off[k]] and its chord
// runs from P1[k] to that MD's anchor (towards it when `out`, else from it). A lane takes
// two items per pass and issues both loads of each step before using either.
__device__ __forceinline__ void t3_stage(const EvDesc &ev, const int32_t *__restrict__ list, const int *off,
                                         const int *st, const float4 *P1, bool out, int f0, int f1, float4 *dst,
                                         int *dmd) {
  const int lane = threadIdx.x & 31;
  for (int fb = f0; fb < f1; fb += 64) {
    int md[2], k[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int f = fb + 32 * j + lane;
      md[j] = 0;
      k[j] = 0;
      if (f < f1) {
        k[j] = t3_owner(off, f);
        const int p = st[k[j]] + (f - off[k[j]]);
        if (chk(ev, p, ev.ls_cap, 31)) md[j] = list[p];
        if (!chk(ev, md[j], ev.md_cap, 32)) md[j] = 0;
      }
    }
    float4 Q[2];
#pragma unroll
    for (int j = 0; j < 2; j++)
      if (fb + 32 * j + lane < f1) Q[j] = ev.md_anchor[md[j]];
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int f = fb + 32 * j + lane;
      if (f < f1) {
        const float4 M = P1[k[j]];
        const float dx = out ? Q[j].x - M.x : M.x - Q[j].x;
        const float dy = out ? Q[j].y - M.y : M.y - Q[j].y;
        const float dz = out ? Q[j].z - M.z : M.z - Q[j].z;
        dst[f - f0] = make_float4(dx, dy, dz, sqrtf(dx * dx + dy * dy));
        dmd[f - f0] = md[j];
      }
    }
  }
}

// The exact cut behind a call boundary: it runs on ~2% of the candidate pairs, and its
// square roots and divisions would otherwise raise the register demand of the pair loop.
__device__ __noinline__ bool t3_cut_call(const float4 P0, const float4 P1, const float4 P2, const lst_cuts &c,
                                         float &kappa) {
  return t3_cut(P0, P1, P2, c, kappa);
}

__global__ void __launch_bounds__(256, 4) k_t3(const EvDesc *__restrict__ evs, int n_events, lst_cuts c, int *work,
                                           int mdu) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T3Warp &w = reinterpret_cast<T3Warp *>(smem_raw)[wid];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void_before(ev, F_OVF_MD | F_OVF_LS) ? 0 : (clamp_count(ev.cnt[C_MD], ev.md_cap) + mdu - 1) / mdu;
  }, s_pref);
  const int total = s_pref[n_events];
  const float tolp = c.t3_rz_tol * 1.001f + 3e-4f;
  int cur = -1, qn = 0;            // event of the queued triples, queue length
  // exact cut of the first n queued triples (one per lane) of event `cur`
  auto run_queue = [&](int n) {
    const EvDesc &ev = evs[cur];
    bool pass = false;
    float k = 0.0f;
    int md0 = 0, md1 = 0, md2 = 0;
    if (lane < n) {
      md0 = w.q0[lane];
      md1 = w.q1[lane];
      md2 = w.q2[lane];
      pass = t3_cut_call(ev.md_anchor[md0], ev.md_anchor[md1], ev.md_anchor[md2], c, k);
    }
    const unsigned bal = __ballot_sync(FULL, pass);
    if (bal) {
      const int base = warp_reserve(ev.cnt + C_T3, ev.cnt + C_FLAGS, F_OVF_T3, __popc(bal), ev.t3_cap);
      if (pass && base >= 0) {
        const int o = base + __popc(bal & lanemask_lt());
        ev.t3u_md[o] = make_int4(md0, md1, md2, atomicAdd(ev.t3_cnt + md0, 1));
        ev.t3u_kappa[o] = k;
      }
    }
  };
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(work, 1);
    u = __shfl_sync(FULL, u, 0);
    if (u >= total) break;
    const int e = find_event(s_pref, n_events, u);
    if (e != cur) {                               // the queue holds triples of one event
      if (qn > 0) {
        __syncwarp();
        run_queue(qn);
        qn = 0;
      }
      cur = e;
    }
    const EvDesc &ev = evs[e];
    const int nmd = clamp_count(ev.cnt[C_MD], ev.md_cap);
    const int m0 = (u - s_pref[e]) * mdu;
    const int m = m0 + lane;
    int nI = 0, nO = 0, sI = 0, sO = 0;
    float4 P1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < mdu && m < nmd) {                 // the anchor with the counts: one round trip
      nI = ev.lso_cnt[m];
      nO = ev.ls_cnt[m];
      sI = ev.lso_start[m];
      sO = ev.ls_start[m];
      P1 = ev.md_anchor[m];
    }
    const int np = nI * nO;
    if (np == 0) nI = nO = 0;
    const int incI = warp_incl_scan(nI), incO = warp_incl_scan(nO), incP = warp_incl_scan(np);
    __syncwarp();                                  // the previous unit's table readers are done
    w.ioff[lane] = incI - nI;
    w.ooff[lane] = incO - nO;
    w.ist[lane] = sI;
    w.ost[lane] = sO;
    w.P1[lane] = P1;
    if (lane == 31) {
      w.ioff[32] = incI;
      w.ooff[32] = incO;
      if (incP) atomicAdd(ev.cnt + C_PT3, incP);
    }
    const int TO = __shfl_sync(FULL, incO, 31);
    __syncwarp();
    for (int f0 = 0; f0 < TO; f0 += T3_OCAP) {
      const int f1 = min(TO, f0 + T3_OCAP);
      const int ka = t3_owner(w.ooff, f0), kb = t3_owner(w.ooff, f1 - 1);
      const int g1 = w.ioff[kb + 1];
      for (int c0 = w.ioff[ka]; c0 < g1; c0 += T3_ICAP) {
        const int c1 = min(g1, c0 + T3_ICAP);
        __syncwarp();                              // the previous chunk's readers are done
        if (c0 == w.ioff[ka]) t3_stage(ev, ev.ls_to, w.ooff, w.ost, w.P1, true, f0, f1, w.O, w.omd);
        t3_stage(ev, ev.ls_from, w.ioff, w.ist, w.P1, false, c0, c1, w.I, w.imd);
        __syncwarp();
        for (int gb = c0; gb < c1; gb += 32) {
          const int gi = gb + lane;
          int s = 0, len = 0, kI = 0;
          float4 A = make_float4(0.f, 0.f, 0.f, 0.f);
          if (gi < c1) {
            kI = t3_owner(w.ioff, gi);
            A = w.I[gi - c0];
            const int os = max(w.ooff[kI], f0), oe = min(w.ooff[kI + 1], f1);
            s = os - f0;
            len = max(0, oe - os);
          }
          const float a2 = __fmaf_rn(A.x, A.x, A.y * A.y), a3 = A.w * a2;
          int maxlen = len;
#pragma unroll
          for (int o = 16; o; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(FULL, maxlen, o));
          for (int k0 = 0; k0 < maxlen; k0 += 32) {
            const int kn = min(32, maxlen - k0);
            unsigned mask = 0;
            for (int k = 0; k < kn; k += 2) {      // branch-free: slots past the lane's range
#pragma unroll                                      // are read (clamped) and masked off
              for (int j = 0; j < 2; j++) {
                const int kk = k0 + k + j;
                const float4 B = w.O[min(s + kk, T3_OCAP - 1)];
                const bool p = t3_prefilter(A, a2, a3, B, tolp);
                mask |= (p && kk < len) ? 1u << (k + j) : 0u;
              }
            }
            for (;;) {                             // drain the masks into the queue
              const unsigned act = __ballot_sync(FULL, mask != 0);
              if (act == 0) break;
              if (mask != 0) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1;
                const int q = qn + __popc(act & lanemask_lt());
                w.q0[q] = w.imd[gi - c0];
                w.q1[q] = m0 + kI;
                w.q2[q] = w.omd[s + k0 + k];
              }
              qn += __popc(act);
              if (qn >= 32) {
                __syncwarp();
                run_queue(32);
                __syncwarp();
                if (lane + 32 < qn) {
                  w.q0[lane] = w.q0[lane + 32];
                  w.q1[lane] = w.q1[lane + 32];
                  w.q2[lane] = w.q2[lane + 32];
                }
                __syncwarp();
                qn -= 32;
              }
            }
          }
        }
      }
    }
  }
  if (qn > 0) {
    __syncwarp();
    run_queue(qn);
  }
}

// T3s grouped by first MD: exclusive scan of the per-MD counts (one CTA per event) ...
__global__ void k_t3_scan(const EvDesc *__restrict__ evs) {
  const EvDesc &ev = evs[blockIdx.x];
  if (ev_void(ev)) return;
  block_exclusive_scan(ev.t3_cnt, ev.t3_pos, clamp_count(ev.cnt[C_MD], ev.md_cap));
}

// ... then a scatter into that order: each T3 to the start of its first MD's range plus the
// rank the producer drew when it counted the T3.
__global__ void __launch_bounds__(256) k_t3_scatter(const EvDesc *__restrict__ evs, int n_events) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int e0 = 0; e0 < n_events; e0 += GROUP_EV) {
    int n[GROUP_EV], nmax = 0;
#pragma unroll
    for (int k = 0; k < GROUP_EV; k++) {
      n[k] = 0;
      if (e0 + k < n_events) {
        const EvDesc &ev = evs[e0 + k];
        n[k] = ev_void(ev) ? 0 : clamp_count(ev.cnt[C_T3], ev.t3_cap);
      }
      nmax = max(nmax, n[k]);
    }
    for (int o = tid; o < nmax; o += st) {
      int4 t[GROUP_EV];
      float k3[GROUP_EV];
      int pos[GROUP_EV];
#pragma unroll
      for (int k = 0; k < GROUP_EV; k++)
        if (o < n[k]) { t[k] = evs[e0 + k].t3u_md[o]; k3[k] = evs[e0 + k].t3u_kappa[o]; }
#pragma unroll
      for (int k = 0; k < GROUP_EV; k++)
        if (o < n[k]) pos[k] = evs[e0 + k].t3_pos[t[k].x] + t[k].w;
#pragma unroll
      for (int k = 0; k < GROUP_EV; k++)
        if (o < n[k]) {
          evs[e0 + k].t3_md[pos[k]] = make_int4(t[k].x, t[k].y, t[k].z, 0);
          evs[e0 + k].t3_kappa[pos[k]] = k3[k];
        }
    }
  }
}

// ===================================================================== step 4: quintuplets
// Pairs (T3a, T3b) with T3b in the list of T3s whose first MD is T3a's last MD. A warp takes
// 32 consecutive T3a with their list lengths; a warp scan of the lengths gives each T3a its
// range of flat pair indices, and a flat index maps to its T3a by a binary search in the
// warp's shared copy of the inclusive scan (32 entries). Work is spread by static striding
// over chunks of T3a of all events (no atomics); pair counts are summed per warp and
// flushed once per event.
struct T5Warp {
  int incl[32], st2[32], ta[32];
  float ka[32];
  float4 P0[32], P1[32], P2[32];
};
static_assert(sizeof(T5Warp) == 2048, "the host sizes k_t5 shared memory with 2048 bytes per warp");

__global__ void __launch_bounds__(256) k_t5(const EvDesc *__restrict__ evs, int n_events, lst_cuts c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  T5Warp &w = reinterpret_cast<T5Warp *>(smem_raw)[wid];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void_before(ev, F_OVF_MD | F_OVF_LS | F_OVF_T3) ? 0 : (clamp_count(ev.cnt[C_T3], ev.t3_cap) + 31) / 32;
  }, s_pref);
  const int total = s_pref[n_events];
  const int W = gridDim.x * nwarps;
  int cur = -1, acc = 0;
  for (int u = blockIdx.x * nwarps + wid; u < total; u += W) {
    const int e = find_event(s_pref, n_events, u);
    if (e != cur) {
      if (cur >= 0 && lane == 0 && acc) atomicAdd(evs[cur].cnt + C_PT5, acc);
      acc = 0;
      cur = e;
    }
    const EvDesc &ev = evs[e];
    const int nt3 = clamp_count(ev.cnt[C_T3], ev.t3_cap);
    const int ta = (u - s_pref[e]) * 32 + lane;
    int deg = 0;
    if (ta < nt3) {
      const int4 A3 = ev.t3_md[ta];
      deg = ev.t3_cnt[A3.z];
      if (deg > 0) {                               // most T3s start no T5: skip their anchors
        w.st2[lane] = ev.t3_pos[A3.z];
        w.ta[lane] = ta;
        w.ka[lane] = ev.t3_kappa[ta];
        w.P0[lane] = ev.md_anchor[A3.x];
        w.P1[lane] = ev.md_anchor[A3.y];
        w.P2[lane] = ev.md_anchor[A3.z];
      }
    }
    const int inc = warp_incl_scan(deg);
    w.incl[lane] = inc;
    __syncwarp();
    const int tot = __shfl_sync(FULL, inc, 31);
    acc += tot;
    for (int f0 = 0; f0 < tot; f0 += 32) {
      const int f = f0 + lane;
      bool pass = false;
      int4 a = make_int4(0, 0, 0, 0), b = make_int4(0, 0, 0, 0);
      if (f < tot) {
        int lo = 0, hi = 31;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (w.incl[mid] > f) hi = mid; else lo = mid + 1; }
        const int prev = lo ? w.incl[lo - 1] : 0;
        const int tb = w.st2[lo] + (f - prev);
        const int4 B3 = ev.t3_md[tb];
        float4 P[5];
        P[0] = w.P0[lo];
        P[1] = w.P1[lo];
        P[2] = w.P2[lo];
        P[3] = ev.md_anchor[B3.y];
        P[4] = ev.md_anchor[B3.z];
        pass = t5_cut(P, w.ka[lo], ev.t3_kappa[tb], c);
        float chi2 = 0.0f;
        if (pass) {
          // circle-fit quality: the pre-DNN mode cuts on it, the track candidates rank by it
          chi2 = t5_chi2(P, c.hit_sigma);
          if (c.t5_chi2_max > 0.0f && !(chi2 <= c.t5_chi2_max)) pass = false;
        }
        const int4 A3 = ev.t3_md[w.ta[lo]];
        a = make_int4(A3.x, A3.y, A3.z, B3.y);
        b = make_int4(B3.z, w.ta[lo], tb, __float_as_int(chi2));
      }
      const unsigned bal = __ballot_sync(FULL, pass);
      if (bal) {
        const int base = warp_reserve(ev.cnt + C_T5, ev.cnt + C_FLAGS, F_OVF_T5, __popc(bal), ev.t5_cap);
        if (pass && base >= 0) {
          const int o = base + __popc(bal & lanemask_lt());
          ev.t5_a[o] = a;
          ev.t5_b[o] = b;
        }
      }
    }
    __syncwarp();
  }
  if (cur >= 0 && lane == 0 && acc) atomicAdd(evs[cur].cnt + C_PT5, acc);
}

}  // namespace lstk
