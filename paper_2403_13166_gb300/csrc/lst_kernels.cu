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
// Count hits per sensor (validating sensor ids and coordinates).
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
    atomicAdd(ev.sens_cnt + s, 1);
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
    const int pos = ev.sens_off[s] + atomicAdd(ev.sens_cnt + s, 1);
    ev.hit[pos] = make_float4(x, y, z, sqrtf(x * x + y * y));
    ev.hit_orig[pos] = i;
  }
}

// ===================================================================== shared machinery
// Fetch the next unit for a warp from a global work counter.
__device__ __forceinline__ int warp_next(int *work) {
  int u = 0;
  if ((threadIdx.x & 31) == 0) u = atomicAdd(work, 1);
  return __shfl_sync(FULL, u, 0);
}

// Reserve n output slots for a unit: one atomicAdd per warp. Returns the base or -1 if the
// buffer would overflow (then the flag is set; the counter still records the demand).
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
// One warp per (event, module): all (lower, upper) hit pairs of the module.
// smem per warp: buf_cap entries of (pair index, cut kappa, feature kappa).
struct MdBuf { int p; float kc, kf; };

__global__ void __launch_bounds__(256) k_md(const EvDesc *__restrict__ evs, int n_events, DevGeom g,
                                           lst_cuts c, int *work, int buf_cap) {
  extern __shared__ unsigned char smem_raw[];
  MdBuf *buf = reinterpret_cast<MdBuf *>(smem_raw) + (threadIdx.x >> 5) * buf_cap;
  const int lane = threadIdx.x & 31;
  const int total = n_events * g.n_mod;
  for (;;) {
    const int u = warp_next(work);
    if (u >= total) break;
    const int e = u / g.n_mod, m = u - e * g.n_mod;
    const EvDesc &ev = evs[e];
    const int flags = ev.cnt[C_FLAGS];
    const int lo0 = ev.sens_off[2 * m], lo1 = ev.sens_off[2 * m + 1], up1 = ev.sens_off[2 * m + 2];
    const int nlo = lo1 - lo0, nup = up1 - lo1;
    const long long np64 = (long long)nlo * nup;
    if (np64 > (1ll << 30)) {   // more hit pairs in one module than an int index can address
      if (lane == 0) { atomicOr(ev.cnt + C_FLAGS, F_INPUT); ev.md_start[m] = 0; ev.md_cnt[m] = 0; }
      continue;
    }
    const int np = (flags & F_INPUT) ? 0 : (int)np64;
    const bool endcap = g.subdet[m] != 0;
    if (lane == 0 && np) atomicAdd(ev.cnt + C_PMD, np);
    // pass 1: evaluate, compact into the warp's list
    int nsel = 0;
    for (int b = 0; b < np; b += 32) {
      const int p = b + lane;
      bool pass = false;
      float kc = 0.0f, kf = 0.0f;
      int i = 0, j = 0;
      if (p < np) {
        i = p / nup;
        j = p - i * nup;
        const float4 L = ev.hit[lo0 + i], U = ev.hit[lo1 + j];
        pass = md_cut(L, U, endcap, c, kc);
        if (pass && !endcap) kf = md_kappa_acc(L, U);
      }
      const unsigned bal = __ballot_sync(FULL, pass);
      const int slot = nsel + __popc(bal & lanemask_lt());
      if (pass && slot < buf_cap) buf[slot] = {p, kc, kf};
      nsel += __popc(bal);
    }
    __syncwarp();
    const int base = warp_reserve(ev.cnt + C_MD, ev.cnt + C_FLAGS, F_OVF_MD, nsel, ev.md_cap);
    if (base < 0 || nsel == 0) {
      if (lane == 0) { ev.md_start[m] = 0; ev.md_cnt[m] = 0; }
      continue;
    }
    if (nsel <= buf_cap) {
      for (int k = lane; k < nsel; k += 32) {
        const MdBuf r = buf[k];
        const int i = r.p / nup, j = r.p - (r.p / nup) * nup;
        ev.md_anchor[base + k] = ev.hit[lo0 + i];
        ev.md_kappa[base + k] = make_float2(r.kc, r.kf);
        ev.md_mod[base + k] = m;
        ev.md_hits[base + k] = make_int2(ev.hit_orig[lo0 + i], ev.hit_orig[lo1 + j]);
      }
    } else {
      // list overflow: evaluate again and write in place (same pair order)
      int w = 0;
      for (int b = 0; b < np; b += 32) {
        const int p = b + lane;
        bool pass = false;
        float kc = 0.0f, kf = 0.0f;
        int i = 0, j = 0;
        float4 L, U;
        if (p < np) {
          i = p / nup;
          j = p - i * nup;
          L = ev.hit[lo0 + i];
          U = ev.hit[lo1 + j];
          pass = md_cut(L, U, endcap, c, kc);
          if (pass && !endcap) kf = md_kappa_acc(L, U);
        }
        const unsigned bal = __ballot_sync(FULL, pass);
        if (pass) {
          const int k = base + w + __popc(bal & lanemask_lt());
          ev.md_anchor[k] = L;
          ev.md_kappa[k] = make_float2(kc, kf);
          ev.md_mod[k] = m;
          ev.md_hits[k] = make_int2(ev.hit_orig[lo0 + i], ev.hit_orig[lo1 + j]);
        }
        w += __popc(bal);
      }
    }
    if (lane == 0) { ev.md_start[m] = base; ev.md_cnt[m] = nsel; }
    __syncwarp();
  }
}

// ===================================================================== step 2: line segments
// One CTA per (event, module m). The MDs of every module linked to m by the module map are
// staged once in shared memory (anchor, cut curvature, barrel flag, MD index); each warp
// then takes one inner MD of m and tests it against all staged MDs, lanes across targets.
struct LsBuf { int j; float k; };

__global__ void __launch_bounds__(256) k_ls(const EvDesc *__restrict__ evs, int n_events, DevGeom g,
                                           lst_cuts c, int *work, int stage_cap, int buf_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *s_anc = reinterpret_cast<float4 *>(smem_raw);                 // [stage_cap]
  float *s_k = reinterpret_cast<float *>(s_anc + stage_cap);            // [stage_cap]
  int *s_idx = reinterpret_cast<int *>(s_k + stage_cap);                // [stage_cap] MD index, sign = barrel
  int *s_tpref = s_idx + stage_cap;                                     // [MAX_FANOUT + 1]
  int *s_tstart = s_tpref + MAX_FANOUT + 1;                             // [MAX_FANOUT]
  LsBuf *s_buf = reinterpret_cast<LsBuf *>(s_tstart + MAX_FANOUT);      // [warps][buf_cap]
  __shared__ int s_unit;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  LsBuf *buf = s_buf + wid * buf_cap;
  const int total = n_events * g.n_mod;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(work, 1);
    __syncthreads();
    const int u = s_unit;
    __syncthreads();
    if (u >= total) break;
    const int e = u / g.n_mod, m = u - e * g.n_mod;
    const EvDesc &ev = evs[e];
    const int n_in = ev.md_cnt[m];
    if (n_in == 0) continue;
    const int in0 = ev.md_start[m];
    // target list with prefix of MD counts
    const int t0 = g.map_off[m], nt = min(g.map_off[m + 1] - t0, MAX_FANOUT);
    if (wid == 0) {
      int carry = 0;
      for (int b = 0; b < nt; b += 32) {
        const int t = b + lane;
        int cnt = 0, st = 0;
        if (t < nt) {
          const int mt = g.map_tgt[t0 + t];
          cnt = ev.md_cnt[mt];
          st = ev.md_start[mt];
        }
        const int inc = warp_incl_scan(cnt);
        if (t < nt) { s_tpref[t + 1] = carry + inc; s_tstart[t] = st; }
        carry += __shfl_sync(FULL, inc, 31);
      }
      if (lane == 0) s_tpref[0] = 0;
    }
    __syncthreads();
    const int S = s_tpref[nt];
    const bool staged = S <= stage_cap;
    if (threadIdx.x == 0 && S) atomicAdd(ev.cnt + C_PLS, n_in * S);
    if (staged) {
      for (int q = threadIdx.x; q < S; q += blockDim.x) {
        const int t = find_event(s_tpref, nt + 1, q);
        const int md = s_tstart[t] + (q - s_tpref[t]);
        s_anc[q] = ev.md_anchor[md];
        s_k[q] = ev.md_kappa[md].x;
        const bool barrel = g.subdet[ev.md_mod[md]] == 0;
        s_idx[q] = barrel ? md : ~md;
      }
    }
    __syncthreads();
    const bool bA = g.subdet[m] == 0;
    for (int ii = wid; ii < n_in; ii += nwarps) {
      const int i = in0 + ii;
      const float4 A = ev.md_anchor[i];
      const float kA = ev.md_kappa[i].x;
      int nsel = 0;
      for (int b = 0; b < S; b += 32) {
        const int q = b + lane;
        bool pass = false;
        float k = 0.0f;
        int jm = 0;
        if (q < S) {
          float4 B;
          float kB;
          int code;
          if (staged) {
            B = s_anc[q]; kB = s_k[q]; code = s_idx[q];
          } else {
            const int t = find_event(s_tpref, nt + 1, q);
            const int md = s_tstart[t] + (q - s_tpref[t]);
            B = ev.md_anchor[md]; kB = ev.md_kappa[md].x;
            code = g.subdet[ev.md_mod[md]] == 0 ? md : ~md;
          }
          const bool bB = code >= 0;
          jm = bB ? code : ~code;
          pass = ls_cut(A, B, kA, kB, bA, bB, c, k);
        }
        const unsigned bal = __ballot_sync(FULL, pass);
        const int slot = nsel + __popc(bal & lanemask_lt());
        if (pass && slot < buf_cap) buf[slot] = {jm, k};
        nsel += __popc(bal);
      }
      __syncwarp();
      const int base = warp_reserve(ev.cnt + C_LS, ev.cnt + C_FLAGS, F_OVF_LS, nsel, ev.ls_cap);
      if (base < 0 || nsel == 0) {
        if (lane == 0) { ev.ls_start[i] = 0; ev.ls_cnt[i] = 0; }
        __syncwarp();
        continue;
      }
      if (nsel <= buf_cap) {
        for (int k = lane; k < nsel; k += 32) {
          const LsBuf r = buf[k];
          ev.ls_in[base + k] = i;
          ev.ls_out[base + k] = r.j;
          ev.ls_kappa[base + k] = r.k;
        }
      } else {
        int w = 0;
        for (int b = 0; b < S; b += 32) {
          const int q = b + lane;
          bool pass = false;
          float k = 0.0f;
          int jm = 0;
          if (q < S) {
            const int t = find_event(s_tpref, nt + 1, q);
            const int md = s_tstart[t] + (q - s_tpref[t]);
            const float4 B = ev.md_anchor[md];
            const bool bB = g.subdet[ev.md_mod[md]] == 0;
            jm = md;
            pass = ls_cut(A, B, kA, ev.md_kappa[md].x, bA, bB, c, k);
          }
          const unsigned bal = __ballot_sync(FULL, pass);
          if (pass) {
            const int o = base + w + __popc(bal & lanemask_lt());
            ev.ls_in[o] = i; ev.ls_out[o] = jm; ev.ls_kappa[o] = k;
          }
          w += __popc(bal);
        }
      }
      if (lane == 0) { ev.ls_start[i] = base; ev.ls_cnt[i] = nsel; }
      __syncwarp();
    }
    __syncthreads();
  }
}

// ===================================================================== steps 3 and 4
// Both enumerate, for one first MD (md0), all pairs (X1, X2) with X1 in out(md0) and X2 in
// out(mid(X1)) where out() is a contiguous range per MD. A warp flattens the pairs: lanes
// hold up to 32 X1 with their out-degree, an inclusive warp scan of the degrees maps each
// flat pair index to (X1, X2) by binary search in the warp's shared copy of the scan.
struct PairWarp {
  int incl[32];
  int mid[32];     // middle MD of X1
  int st2[32];     // start of out(mid)
  int x1[32];      // X1 index
};
struct T3Buf { int md1, md2; float k; };

__global__ void __launch_bounds__(256) k_t3(const EvDesc *__restrict__ evs, int n_events, lst_cuts c,
                                           int *work, int buf_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  PairWarp *pw = reinterpret_cast<PairWarp *>(smem_raw) + wid;
  T3Buf *buf = reinterpret_cast<T3Buf *>(reinterpret_cast<PairWarp *>(smem_raw) + nwarps) + wid * buf_cap;
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return (ev.cnt[C_FLAGS] & F_INPUT) ? 0 : clamp_count(ev.cnt[C_MD], ev.md_cap);
  }, s_pref);
  const int total = s_pref[n_events];
  for (;;) {
    const int u = warp_next(work);
    if (u >= total) break;
    const int e = find_event(s_pref, n_events, u);
    const EvDesc &ev = evs[e];
    const int md0 = u - s_pref[e];
    const int n1 = ev.ls_cnt[md0], s1 = ev.ls_start[md0];
    const float4 P0 = ev.md_anchor[md0];
    // count pass (with list), possibly a write pass if the list overflowed
    int nsel = 0, base = 0;
    for (int pass_no = 0; pass_no < 2; pass_no++) {
      int w = 0;
      for (int k0 = 0; k0 < n1; k0 += 32) {
        int deg = 0;
        if (k0 + lane < n1) {
          const int l1 = s1 + k0 + lane;
          const int md1 = ev.ls_out[l1];
          deg = ev.ls_cnt[md1];
          pw->mid[lane] = md1;
          pw->st2[lane] = ev.ls_start[md1];
          pw->x1[lane] = l1;
        }
        const int inc = warp_incl_scan(deg);
        pw->incl[lane] = inc;
        __syncwarp();
        const int tot = __shfl_sync(FULL, inc, 31);
        if (pass_no == 0 && lane == 0 && tot) atomicAdd(ev.cnt + C_PT3, tot);
        for (int f0 = 0; f0 < tot; f0 += 32) {
          const int f = f0 + lane;
          bool pass = false;
          float k = 0.0f;
          int md1 = 0, md2 = 0;
          if (f < tot) {
            int lo = 0, hi = 31;
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (pw->incl[mid] > f) hi = mid; else lo = mid + 1; }
            const int prev = lo ? pw->incl[lo - 1] : 0;
            md1 = pw->mid[lo];
            const int l2 = pw->st2[lo] + (f - prev);
            md2 = ev.ls_out[l2];
            pass = t3_cut(P0, ev.md_anchor[md1], ev.md_anchor[md2], c, k);
          }
          const unsigned bal = __ballot_sync(FULL, pass);
          const int slot = w + __popc(bal & lanemask_lt());
          if (pass) {
            if (pass_no == 0) {
              if (slot < buf_cap) buf[slot] = {md1, md2, k};
            } else {
              ev.t3_md[base + slot] = make_int4(md0, md1, md2, 0);
              ev.t3_kappa[base + slot] = k;
            }
          }
          w += __popc(bal);
        }
        __syncwarp();
      }
      if (pass_no == 0) {
        nsel = w;
        base = warp_reserve(ev.cnt + C_T3, ev.cnt + C_FLAGS, F_OVF_T3, nsel, ev.t3_cap);
        if (base < 0 || nsel == 0) { nsel = 0; base = 0; break; }
        if (nsel <= buf_cap) {
          for (int k = lane; k < nsel; k += 32) {
            const T3Buf r = buf[k];
            ev.t3_md[base + k] = make_int4(md0, r.md1, r.md2, 0);
            ev.t3_kappa[base + k] = r.k;
          }
          break;
        }
      }
    }
    if (lane == 0) { ev.t3_start[md0] = base; ev.t3_cnt[md0] = nsel; }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) k_t5(const EvDesc *__restrict__ evs, int n_events, lst_cuts c,
                                           int *work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pref[MAX_EVENTS + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PairWarp *pw = reinterpret_cast<PairWarp *>(smem_raw) + wid;
  block_event_prefix(n_events, [&](int e) {
    const EvDesc &ev = evs[e];
    return (ev.cnt[C_FLAGS] & F_INPUT) ? 0 : clamp_count(ev.cnt[C_MD], ev.md_cap);
  }, s_pref);
  const int total = s_pref[n_events];
  for (;;) {
    const int u = warp_next(work);
    if (u >= total) break;
    const int e = find_event(s_pref, n_events, u);
    const EvDesc &ev = evs[e];
    const int md0 = u - s_pref[e];
    const int n1 = ev.t3_cnt[md0], s1 = ev.t3_start[md0];
    if (n1 == 0) continue;
    const float4 P0 = ev.md_anchor[md0];
    for (int k0 = 0; k0 < n1; k0 += 32) {
      int deg = 0;
      if (k0 + lane < n1) {
        const int ta = s1 + k0 + lane;
        const int md2 = ev.t3_md[ta].z;
        deg = ev.t3_cnt[md2];
        pw->mid[lane] = md2;
        pw->st2[lane] = ev.t3_start[md2];
        pw->x1[lane] = ta;
      }
      const int inc = warp_incl_scan(deg);
      pw->incl[lane] = inc;
      __syncwarp();
      const int tot = __shfl_sync(FULL, inc, 31);
      if (lane == 0 && tot) atomicAdd(ev.cnt + C_PT5, tot);
      for (int f0 = 0; f0 < tot; f0 += 32) {
        const int f = f0 + lane;
        bool pass = false;
        int4 a = make_int4(0, 0, 0, 0), b = make_int4(0, 0, 0, 0);
        if (f < tot) {
          int lo = 0, hi = 31;
          while (lo < hi) { const int mid = (lo + hi) >> 1; if (pw->incl[mid] > f) hi = mid; else lo = mid + 1; }
          const int prev = lo ? pw->incl[lo - 1] : 0;
          const int ta = pw->x1[lo];
          const int tb = pw->st2[lo] + (f - prev);
          const int4 A3 = ev.t3_md[ta], B3 = ev.t3_md[tb];
          float4 P[5];
          P[0] = P0;
          P[1] = ev.md_anchor[A3.y];
          P[2] = ev.md_anchor[A3.z];
          P[3] = ev.md_anchor[B3.y];
          P[4] = ev.md_anchor[B3.z];
          pass = t5_cut(P, ev.t3_kappa[ta], ev.t3_kappa[tb], c);
          a = make_int4(md0, A3.y, A3.z, B3.y);
          b = make_int4(B3.z, ta, tb, 0);
        }
        const unsigned bal = __ballot_sync(FULL, pass);
        const int n = __popc(bal);
        if (n) {
          const int base = warp_reserve(ev.cnt + C_T5, ev.cnt + C_FLAGS, F_OVF_T5, n, ev.t5_cap);
          if (pass && base >= 0) {
            const int o = base + __popc(bal & lanemask_lt());
            ev.t5_a[o] = a;
            ev.t5_b[o] = b;
          }
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace lstk
