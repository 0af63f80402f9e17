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
// Count hits per sensor (validating sensor ids and coordinates). Sensors are keyed as
// (sensor & 1) * n_mod + module, so that all lower-sensor hits come first in the grouped
// order: key k < n_mod is the lower sensor of module k, key n_mod + k its upper sensor.
__global__ void k_bin_count(const EvDesc *__restrict__ evs, DevGeom g) {
  const EvDesc &ev = evs[blockIdx.y];
  const int n = ev.n_hits, ns = 2 * g.n_mod;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = __ldg(ev.sensor + i);
    const float x = __ldg(ev.x + i), y = __ldg(ev.y + i), z = __ldg(ev.z + i);
    if (s < 0 || s >= ns || !isfinite(x) || !isfinite(y) || !isfinite(z)) {
      atomicOr(ev.cnt + C_FLAGS, F_INPUT);
      continue;
    }
    atomicAdd(ev.sens_cnt + (s & 1) * g.n_mod + (s >> 1), 1);
  }
}

// Exclusive scan of the sensor histogram (one CTA per event); re-zeroes the histogram so
// it serves as the scatter cursor.
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
      ev.sens_cnt[s] = 0;
      run += c;
    }
  }
  if (b0 + per >= ns && b0 < ns) ev.sens_off[ns] = run;
  if (ns == 0 && threadIdx.x == 0) ev.sens_off[0] = 0;
}

// Scatter hits into sensor order as float4 (x, y, z, r) with r = sqrtf(x*x + y*y).
__global__ void k_bin_scatter(const EvDesc *__restrict__ evs, DevGeom g) {
  const EvDesc &ev = evs[blockIdx.y];
  const int n = ev.n_hits, ns = 2 * g.n_mod;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = __ldg(ev.sensor + i);
    const float x = __ldg(ev.x + i), y = __ldg(ev.y + i), z = __ldg(ev.z + i);
    if (s < 0 || s >= ns || !isfinite(x) || !isfinite(y) || !isfinite(z)) continue;
    const int key = (s & 1) * g.n_mod + (s >> 1);
    const int pos = ev.sens_off[key] + atomicAdd(ev.sens_cnt + key, 1);
    ev.hit[pos] = make_float4(x, y, z, sqrtf(x * x + y * y));
    ev.hit_orig[pos] = i;
    ev.hit_mod[pos] = s >> 1;
  }
}

// ===================================================================== shared machinery
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
    float hb2r2 = 0.0f;
    if (h < ev.sens_off[nm]) {
      const int m = ev.hit_mod[h];
      up0 = ev.sens_off[nm + m];
      nup = ev.sens_off[nm + m + 1] - up0;
      endcap = g.subdet[m] != 0;
      L = ev.hit[h];
      const float hb = L.w * (0.5f * c.kappa_max) + c.hit_err / c.sensor_gap;
      hb2r2 = (L.w * hb) * (L.w * hb);
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
            ev.mdu_hits[o] = make_int2(ev.hit_orig[w.lo[x]], ev.hit_orig[uh]);
            atomicAdd(ev.md_cnt + w.mod[x], 1);
          }
        }
      }
    };
    __syncwarp();
    int qlen = 0;
    for (int j = 0; j < mx; j++) {
      bool pre = false;
      if (j < nup) pre = md_prefilter(L, ev.hit[up0 + j], endcap, hb2r2, c);
      const unsigned bal = __ballot_sync(FULL, pre);
      if (bal == 0) continue;
      if (pre) {
        const int q = qlen + __popc(bal & lanemask_lt());
        w.qx[q] = lane;
        w.qu[q] = up0 + j;
      }
      qlen += __popc(bal);
      if (qlen >= 32) {
        __syncwarp();
        run_queue(qlen - 32, 32);
        qlen -= 32;
        __syncwarp();
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
    ev.md_cur[b0 + k] = run;
    run += ev.md_cnt[b0 + k];
  }
}

// ... then a scatter into module order.
__global__ void k_md_scatter(const EvDesc *__restrict__ evs, int n_events) {
  __shared__ int s_pref[MAX_EVENTS + 1];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void(ev) ? 0 : clamp_count(ev.cnt[C_MD], ev.md_cap);
  }, s_pref);
  const int total = s_pref[n_events];
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    const int e = find_event(s_pref, n_events, u);
    const EvDesc &ev = evs[e];
    const int o = u - s_pref[e];
    const int m = ev.mdu_mod[o];
    const int pos = atomicAdd(ev.md_cur + m, 1);
    if (!chk(ev, pos, ev.md_cap, 14)) continue;
    ev.md_anchor[pos] = ev.mdu_anchor[o];
    ev.md_kappa[pos] = ev.mdu_kappa[o];
    ev.md_mod[pos] = m;
    ev.md_hits[pos] = ev.mdu_hits[o];
  }
}

// ===================================================================== step 2: line segments
// One CTA per (event, module m). The target MDs (all MDs of the modules linked to m by
// the module map, concatenated) are spread over the lanes: every lane holds one target MD
// in registers and loops over the inner MDs of m, which sit in shared memory and are read
// as broadcasts. A tile of 32 targets x IN_CHUNK inner MDs therefore costs one shared-memory
// broadcast per pair and the FP32 cut. Passing pairs go to a shared list with per-inner-MD
// counts; after the tile the CTA reserves one output range (one atomicAdd) and scatters
// the list so that the LSs of each inner MD are contiguous.
constexpr int LS_IN_CHUNK = 64;
struct LsEntry { int i; int md; float k; };

// Per-warp staging of the LS tile: the warp's 32 target MDs, and a queue of the (inner,
// target) pairs that passed ls_prefilter; the exact cut runs on 32 queued pairs at a time.
struct LsWarp {
  float4 B[32];          // target anchors
  float kB[32];          // target MD curvatures (cut values)
  int md[32];            // target MD ids
  unsigned short q[64];  // queued pairs: inner index << 5 | target lane
  unsigned char bB[32];  // target in the barrel
};
static_assert(sizeof(LsWarp) == 928, "the host sizes k_ls shared memory with 928 bytes per warp");

__global__ void __launch_bounds__(256) k_ls(const EvDesc *__restrict__ evs, int n_events, DevGeom g,
                                           lst_cuts c, int *work, int list_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  LsWarp &w = reinterpret_cast<LsWarp *>(smem_raw)[wid];                 // [nwarps]
  float4 *s_in = reinterpret_cast<float4 *>(smem_raw + nwarps * sizeof(LsWarp));  // [LS_IN_CHUNK]
  float4 *s_inx = s_in + LS_IN_CHUNK;                                    // [LS_IN_CHUNK] |A|^2, rA^2, e rA + slack
  float *s_ink = reinterpret_cast<float *>(s_inx + LS_IN_CHUNK);         // [LS_IN_CHUNK]
  int *s_cnt = reinterpret_cast<int *>(s_ink + LS_IN_CHUNK);             // [LS_IN_CHUNK]
  int *s_off = s_cnt + LS_IN_CHUNK;                                      // [LS_IN_CHUNK]
  int *s_tpref = s_off + LS_IN_CHUNK;                                    // [MAX_FANOUT + 1]
  int *s_tstart = s_tpref + MAX_FANOUT + 1;                              // [MAX_FANOUT]
  int *s_tbar = s_tstart + MAX_FANOUT;                                   // [MAX_FANOUT]
  LsEntry *s_list = reinterpret_cast<LsEntry *>(s_tbar + MAX_FANOUT);    // [list_cap]
  __shared__ int s_unit, s_nin, s_nlist, s_base;
  const int total = n_events * g.n_mod;
  const float k0 = 1.002f * 65.0f * (c.hit_err * c.hit_err), c1 = c.z_lum + c.hit_err;
  for (;;) {
    // One thread fetches the unit and reads the event's state; the whole CTA then uses
    // that one copy (the overflow flag may change under other CTAs at any time, and every
    // thread must take the same path through the barriers below).
    if (threadIdx.x == 0) {
      const int uu = atomicAdd(work, 1);
      int nin = 0;
      if (uu < total) {
        const int ee = uu / g.n_mod;
        const EvDesc &evv = evs[ee];
        nin = ev_void(evv) ? 0 : evv.md_cnt[uu - ee * g.n_mod];
      }
      s_unit = uu;
      s_nin = nin;
    }
    __syncthreads();
    const int u = s_unit;
    if (u >= total) break;
    const int e = u / g.n_mod, m = u - e * g.n_mod;
    const EvDesc &ev = evs[e];
    const int n_in = s_nin;
    if (n_in == 0) { __syncthreads(); continue; }
    const int in0 = ev.md_start[m];
    const bool bA = g.subdet[m] == 0;
    // target list: prefix of MD counts over the module map of m
    const int t0 = g.map_off[m], nt = min(g.map_off[m + 1] - t0, MAX_FANOUT);
    if (wid == 0) {
      int carry = 0;
      for (int b = 0; b < nt; b += 32) {
        const int t = b + lane;
        int cnt = 0, st = 0, bar = 0;
        if (t < nt) {
          const int mt = g.map_tgt[t0 + t];
          cnt = ev.md_cnt[mt];
          st = ev.md_start[mt];
          bar = g.subdet[mt] == 0;
        }
        const int inc = warp_incl_scan(cnt);
        if (t < nt) { s_tpref[t + 1] = carry + inc; s_tstart[t] = st; s_tbar[t] = bar; }
        carry += __shfl_sync(FULL, inc, 31);
      }
      if (lane == 0) s_tpref[0] = 0;
    }
    // the first chunk of inner MDs is loaded while warp 0 builds the target prefix
    auto load_inner = [&](int t, int i) {
      const float4 A = ev.md_anchor[i];
      s_in[t] = A;
      s_inx[t] = make_float4(A.x * A.x + A.y * A.y, A.w * A.w, c.hit_err * A.w + 0.05f, 0.0f);
      s_ink[t] = ev.md_kappa[i].x;
      s_cnt[t] = 0;
    };
    for (int t = threadIdx.x; t < min(LS_IN_CHUNK, n_in); t += blockDim.x) load_inner(t, in0 + t);
    if (threadIdx.x == 0) s_nlist = 0;
    __syncthreads();
    const int S = s_tpref[nt];
    if (threadIdx.x == 0 && S) atomicAdd(ev.cnt + C_PLS, n_in * S);
    for (int c0 = 0; c0 < n_in; c0 += LS_IN_CHUNK) {
      const int nc = min(LS_IN_CHUNK, n_in - c0);
      if (c0 > 0) {
        for (int t = threadIdx.x; t < nc; t += blockDim.x) load_inner(t, in0 + c0 + t);
        if (threadIdx.x == 0) s_nlist = 0;
        __syncthreads();
      }
      // ---- tile: lanes over targets, loop over inner MDs; the division-free necessary
      // test runs on every pair, the exact cut on full warps of queued survivors (~9%)
      for (int pass_no = 0; pass_no < 2; pass_no++) {
        const bool writing = pass_no == 1;   // second sweep only after a list overflow
        for (int j0 = wid * 32; j0 < S; j0 += nwarps * 32) {
          const int j = j0 + lane;
          bool valid = j < S;
          float4 B = make_float4(0.f, 0.f, 0.f, 0.f);
          float kB = 0.0f, k1 = 0.0f;
          bool bB = false;
          int md = 0;
          if (valid) {
            const int t = find_event(s_tpref, nt + 1, j);
            md = s_tstart[t] + (j - s_tpref[t]);
            if (chk(ev, md, ev.md_cap, 21)) {
              B = ev.md_anchor[md];
              kB = ev.md_kappa[md].x;
              bB = s_tbar[t] != 0;
              const float X = B.w * (0.5f * c.kappa_max);
              k1 = 1.002f * 1.015625f * X * X;
            } else {
              valid = false;
            }
          }
          w.B[lane] = B;
          w.kB[lane] = kB;
          w.md[lane] = md;
          w.bB[lane] = bB ? 1 : 0;
          __syncwarp();
          // exact cut of the first n queued pairs (one per lane), results to the list
          auto run_queue = [&](int n) {
            bool pass = false;
            int ie = 0, le = 0;
            float k = 0.0f;
            if (lane < n) {
              const int qe = w.q[lane];
              ie = qe >> 5;
              le = qe & 31;
              pass = ls_cut(s_in[ie], w.B[le], s_ink[ie], w.kB[le], bA, w.bB[le] != 0, c, k);
            }
            const unsigned bal = __ballot_sync(FULL, pass);
            if (bal == 0) return;
            if (!writing) {
              int pos = 0;
              if (lane == 0) pos = atomicAdd(&s_nlist, __popc(bal));
              pos = __shfl_sync(FULL, pos, 0);
              if (pass) {
                atomicAdd(&s_cnt[ie], 1);
                const int q = pos + __popc(bal & lanemask_lt());
                if (q < list_cap) s_list[q] = {ie, w.md[le], k};
              }
            } else if (pass) {
              const int o = s_base + s_off[ie] + atomicAdd(&s_cnt[ie], 1);
              if (chk(ev, o, ev.ls_cap, 23)) {
                ev.ls_in[o] = in0 + c0 + ie;
                ev.ls_out[o] = w.md[le];
                ev.ls_kappa[o] = k;
              }
            }
          };
          int qn = 0;
#pragma unroll 2
          for (int i = 0; i < nc; i++) {
            const bool cand = valid & ls_prefilter(s_in[i], s_inx[i], B, k1, k0, c1);
            const unsigned bal = __ballot_sync(FULL, cand);
            if (cand) w.q[qn + __popc(bal & lanemask_lt())] = (unsigned short)((i << 5) | lane);
            qn += __popc(bal);
            if (qn >= 32) {
              __syncwarp();
              run_queue(32);
              __syncwarp();
              if (lane + 32 < qn) w.q[lane] = w.q[lane + 32];
              __syncwarp();
              qn -= 32;
            }
          }
          if (qn > 0) {
            __syncwarp();
            run_queue(qn);
          }
          __syncwarp();
        }
        __syncthreads();
        if (writing) break;
        // ---- per-inner-MD offsets, one reservation for the tile
        if (wid == 0) {
          int carry = 0;
          for (int b = 0; b < nc; b += 32) {
            const int t = b + lane;
            const int v = t < nc ? s_cnt[t] : 0;
            const int inc = warp_incl_scan(v);
            if (t < nc) s_off[t] = carry + inc - v;
            carry += __shfl_sync(FULL, inc, 31);
          }
          int base = 0;
          if (lane == 0 && carry > 0) {
            base = atomicAdd(ev.cnt + C_LS, carry);
            if (base + carry > ev.ls_cap) { atomicOr(ev.cnt + C_FLAGS, F_OVF_LS); base = -1; }
          }
          if (lane == 0) s_base = carry > 0 ? base : -1;
        }
        __syncthreads();
        const int base = s_base;
        const int nlist = s_nlist;
        for (int t = threadIdx.x; t < nc; t += blockDim.x) {
          ev.ls_start[in0 + c0 + t] = base >= 0 ? base + s_off[t] : 0;
          ev.ls_cnt[in0 + c0 + t] = base >= 0 ? s_cnt[t] : 0;
          s_cnt[t] = 0;                    // from here on: scatter cursors (same thread, same t)
        }
        __syncthreads();
        if (base < 0) break;
        if (nlist <= list_cap) {
          for (int q = threadIdx.x; q < nlist; q += blockDim.x) {
            const LsEntry r = s_list[q];
            const int o = base + s_off[r.i] + atomicAdd(&s_cnt[r.i], 1);
            ev.ls_in[o] = in0 + c0 + r.i;
            ev.ls_out[o] = r.md;
            ev.ls_kappa[o] = r.k;
          }
          break;
        }
        // list overflow: sweep the tile again, writing in place
      }
      // the next chunk reuses s_in / s_list / s_cnt; after a unit's last chunk the barrier
      // of the next unit's fetch orders that reuse (thread 0 only writes s_unit / s_nin
      // before it, which every thread has read at this unit's start)
      if (c0 + LS_IN_CHUNK < n_in) __syncthreads();
    }
  }
}

// ===================================================================== steps 3 and 4
// Both enumerate pairs (X1, X2) where X2 ranges over a contiguous list attached to the
// middle MD of X1. A warp takes 32 (T5) or 64 (T3: two per lane) consecutive X1 with their
// list lengths;
// an inclusive warp scan of the lengths maps each flat pair index to (X1, X2) by a binary
// search in the warp's shared copy of the scan. Work is spread by static striding over
// chunks of X1 of all events (no atomics); pair counts are summed per warp and flushed
// once per event.
struct T3Warp {
  float4 P0[64], P1[64];             // 64 first LSs per warp chunk: lanes lane and 32 + lane
  int incl[64], st2[64], md0[64], md1[64];
  int qx[64], qmd[64];               // queue of pairs that passed t3_prefilter
};
static_assert(sizeof(T3Warp) == 3584, "the host sizes k_t3 shared memory with 3584 bytes per warp");

__global__ void __launch_bounds__(256) k_t3(const EvDesc *__restrict__ evs, int n_events, lst_cuts c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  T3Warp &w = reinterpret_cast<T3Warp *>(smem_raw)[wid];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void(ev) ? 0 : (clamp_count(ev.cnt[C_LS], ev.ls_cap) + 63) / 64;
  }, s_pref);
  const int total = s_pref[n_events];
  const int W = gridDim.x * nwarps;
  int cur = -1, acc = 0;
  for (int u = blockIdx.x * nwarps + wid; u < total; u += W) {
    const int e = find_event(s_pref, n_events, u);
    if (e != cur) {
      if (cur >= 0 && lane == 0 && acc) atomicAdd(evs[cur].cnt + C_PT3, acc);
      acc = 0;
      cur = e;
    }
    const EvDesc &ev = evs[e];
    const int nls = clamp_count(ev.cnt[C_LS], ev.ls_cap);
    // two first LSs per lane (slots lane and 32 + lane), their loads independent
    int deg[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int l1 = (u - s_pref[e]) * 64 + 32 * h + lane;
      if (l1 < nls) {
        const int md0 = ev.ls_in[l1], md1 = ev.ls_out[l1];
        deg[h] = ev.ls_cnt[md1];
        w.st2[32 * h + lane] = ev.ls_start[md1];
        w.md0[32 * h + lane] = md0;
        w.md1[32 * h + lane] = md1;
        w.P0[32 * h + lane] = ev.md_anchor[md0];
        w.P1[32 * h + lane] = ev.md_anchor[md1];
      }
    }
    const int inca = warp_incl_scan(deg[0]);
    const int tota = __shfl_sync(FULL, inca, 31);
    const int incb = tota + warp_incl_scan(deg[1]);
    w.incl[lane] = inca;
    w.incl[32 + lane] = incb;
    __syncwarp();
    const int tot = __shfl_sync(FULL, incb, 31);
    acc += tot;
    // exact cut on queued pairs [q0, q0 + n): (LS1 lane, outer MD)
    auto run_queue = [&](int q0, int n) {
      bool pass = false;
      float k = 0.0f;
      int x = 0, md2 = 0;
      if (lane < n) {
        x = w.qx[q0 + lane];
        md2 = w.qmd[q0 + lane];
        pass = t3_cut(w.P0[x], w.P1[x], ev.md_anchor[md2], c, k);
      }
      const unsigned bal = __ballot_sync(FULL, pass);
      if (bal) {
        const int base = warp_reserve(ev.cnt + C_T3, ev.cnt + C_FLAGS, F_OVF_T3, __popc(bal), ev.t3_cap);
        if (pass && base >= 0) {
          const int o = base + __popc(bal & lanemask_lt());
          ev.t3u_md[o] = make_int4(w.md0[x], w.md1[x], md2, 0);
          ev.t3u_kappa[o] = k;
          atomicAdd(ev.t3_cnt + w.md0[x], 1);
        }
      }
    };
    int qlen = 0;
    // flat pair index f -> (LS1 lane x, outer MD); two pairs per lane and iteration so that
    // the two dependent load chains (ls_out, then the anchor) are in flight together
    auto decode = [&](int f, int &x) {
      int lo = 0, hi = 63;
      while (lo < hi) { const int mid = (lo + hi) >> 1; if (w.incl[mid] > f) hi = mid; else lo = mid + 1; }
      x = lo;
      const int prev = lo ? w.incl[lo - 1] : 0;
      return w.st2[lo] + (f - prev);
    };
    auto enqueue = [&](bool pre, int x, int md2) {
      const unsigned bal = __ballot_sync(FULL, pre);
      if (bal == 0) return;
      if (pre) {
        const int q = qlen + __popc(bal & lanemask_lt());
        w.qx[q] = x;
        w.qmd[q] = md2;
      }
      qlen += __popc(bal);
      if (qlen >= 32) {
        __syncwarp();
        run_queue(qlen - 32, 32);
        qlen -= 32;
        __syncwarp();
      }
    };
    for (int f0 = 0; f0 < tot; f0 += 64) {
      const int fa = f0 + lane, fb = f0 + 32 + lane;
      int xa = 0, xb = 0, mda = 0, mdb = 0;
      if (fa < tot) mda = ev.ls_out[decode(fa, xa)];
      if (fb < tot) mdb = ev.ls_out[decode(fb, xb)];
      float4 Pa = make_float4(0.f, 0.f, 0.f, 0.f), Pb = Pa;
      if (fa < tot) Pa = ev.md_anchor[mda];
      if (fb < tot) Pb = ev.md_anchor[mdb];
      const bool prea = fa < tot && t3_prefilter(w.P0[xa], w.P1[xa], Pa, c);
      const bool preb = fb < tot && t3_prefilter(w.P0[xb], w.P1[xb], Pb, c);
      enqueue(prea, xa, mda);
      enqueue(preb, xb, mdb);
    }
    __syncwarp();
    if (qlen > 0) run_queue(0, qlen);
    __syncwarp();
  }
  if (cur >= 0 && lane == 0 && acc) atomicAdd(evs[cur].cnt + C_PT3, acc);
}

// T3s grouped by first MD: exclusive scan of the per-MD counts (one CTA per event) ...
__global__ void k_t3_scan(const EvDesc *__restrict__ evs) {
  const EvDesc &ev = evs[blockIdx.x];
  if (ev_void(ev)) return;
  block_exclusive_scan(ev.t3_cnt, ev.t3_pos, clamp_count(ev.cnt[C_MD], ev.md_cap));
}

// ... then a scatter into that order; afterwards t3_pos[md] holds the END of md's range.
__global__ void k_t3_scatter(const EvDesc *__restrict__ evs, int n_events) {
  __shared__ int s_pref[MAX_EVENTS + 1];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void(ev) ? 0 : clamp_count(ev.cnt[C_T3], ev.t3_cap);
  }, s_pref);
  const int total = s_pref[n_events];
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    const int e = find_event(s_pref, n_events, u);
    const EvDesc &ev = evs[e];
    const int o = u - s_pref[e];
    const int4 t = ev.t3u_md[o];
    const int pos = atomicAdd(ev.t3_pos + t.x, 1);
    ev.t3_md[pos] = t;
    ev.t3_kappa[pos] = ev.t3u_kappa[o];
  }
}

struct T5Warp {
  int incl[32], st2[32], ta[32];
  float ka[32];
  float4 P0[32], P1[32], P2[32];
  int md1[32];
};

__global__ void __launch_bounds__(256) k_t5(const EvDesc *__restrict__ evs, int n_events, lst_cuts c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  T5Warp &w = reinterpret_cast<T5Warp *>(smem_raw)[wid];
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return ev_void(ev) ? 0 : (clamp_count(ev.cnt[C_T3], ev.t3_cap) + 31) / 32;
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
      w.st2[lane] = ev.t3_pos[A3.z] - deg;
      w.ta[lane] = ta;
      w.ka[lane] = ev.t3_kappa[ta];
      w.md1[lane] = A3.y;
      w.P0[lane] = ev.md_anchor[A3.x];
      w.P1[lane] = ev.md_anchor[A3.y];
      w.P2[lane] = ev.md_anchor[A3.z];
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
