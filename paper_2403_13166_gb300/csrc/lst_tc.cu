// lst_tc.cu -- track candidates from the selected quintuplets (arXiv 2403.13166, Table 1
// step 6 without pixel seeds, none exist here), cleaned of duplicates (Section 2 places
// duplicate removal downstream of the T5 step).
//
// Definition (identical in the oracle): two selected T5s are duplicates when they share at
// least 3 of their 5 MDs. T5 u ranks above T5 t when rank(u) < rank(t), or the ranks are
// equal and u's 10 original hit indices (lower, upper hit of each MD in chain order) are
// lexicographically smaller; rank = the circle-fit chi2 with NaN and +inf both +inf (the
// same FP32 bits on both sides). A selected T5 is a track candidate iff no selected
// duplicate ranks above it: one pass, so a T5 removed by a better duplicate still removes
// the T5s it ranks above.
//
// GPU form: every selected T5 is listed under its 5 MDs (count, per-event scan, scatter);
// a duplicate of t shares >= 3 of t's 5 MDs, hence at least one of its middle three, so t
// compares itself with the T5s listed under md1..md3. All four kernels cover the whole
// batch in one launch each.
#include "lst_internal.cuh"

namespace lstk {

namespace {
constexpr int TC_MIN_SHARED = 3;

__device__ __forceinline__ void t5_mds(const EvDesc &ev, int t, int md[5]) {
  const int4 a = ev.t5_a[t];
  md[0] = a.x; md[1] = a.y; md[2] = a.z; md[3] = a.w;
  md[4] = ev.t5_b[t].x;
}

// u's hit tuple below t's (both 10 original hit indices in chain order)
__device__ __forceinline__ bool key_less(const EvDesc &ev, const int mu[5], const int mt[5]) {
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const int2 hu = ev.md_hits[mu[i]], ht = ev.md_hits[mt[i]];
    if (hu.x != ht.x) return hu.x < ht.x;
    if (hu.y != ht.y) return hu.y < ht.y;
  }
  return false;
}

__device__ __forceinline__ int t5_total(const EvDesc &ev) {
  return ev_void(ev) ? 0 : clamp_count(ev.cnt[C_T5], ev.t5_cap);
}
}  // namespace

// Selected T5s per MD.
__global__ void __launch_bounds__(256) k_tc_count(const EvDesc *__restrict__ evs, int n_events) {
  __shared__ int s_pref[MAX_EVENTS + 1];
  block_event_prefix(n_events, [&](int e) { return t5_total(evs[e]); }, s_pref);
  const int total = s_pref[n_events];
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    const int e = find_event(s_pref, n_events, u);
    const EvDesc &ev = evs[e];
    const int t = u - s_pref[e];
    if (!ev.t5_sel[t]) continue;
    int md[5];
    t5_mds(ev, t, md);
#pragma unroll
    for (int i = 0; i < 5; i++) atomicAdd(ev.tc_cnt + md[i], 1);
  }
}

// Exclusive scan of the per-MD counts of one event (one CTA per event): tc_pos = start.
__global__ void k_tc_scan(const EvDesc *__restrict__ evs) {
  const EvDesc &ev = evs[blockIdx.x];
  if (ev_void(ev)) return;
  block_exclusive_scan(ev.tc_cnt, ev.tc_pos, clamp_count(ev.cnt[C_MD], ev.md_cap));
}

// List every selected T5 under each of its MDs; afterwards tc_pos[md] is the END of md's range.
__global__ void __launch_bounds__(256) k_tc_scatter(const EvDesc *__restrict__ evs, int n_events) {
  __shared__ int s_pref[MAX_EVENTS + 1];
  block_event_prefix(n_events, [&](int e) { return t5_total(evs[e]); }, s_pref);
  const int total = s_pref[n_events];
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    const int e = find_event(s_pref, n_events, u);
    const EvDesc &ev = evs[e];
    const int t = u - s_pref[e];
    if (!ev.t5_sel[t]) continue;
    int md[5];
    t5_mds(ev, t, md);
#pragma unroll
    for (int i = 0; i < 5; i++) ev.tc_list[atomicAdd(ev.tc_pos + md[i], 1)] = t;
  }
}

// The track-candidate decision of every T5 of the batch, and the count per event. TC_LANES
// lanes share one T5 and walk its three lists in an interleaved way, so that a warp holds
// 32 / TC_LANES T5s and the lanes of a long list do not wait alone.
constexpr int TC_LANES = 4;
__global__ void __launch_bounds__(256) k_tc_decide(const EvDesc *__restrict__ evs, int n_events) {
  __shared__ int s_pref[MAX_EVENTS + 1];
  block_event_prefix(n_events, [&](int e) { return t5_total(evs[e]); }, s_pref);
  const int total = s_pref[n_events];
  const int lane = threadIdx.x & 31, sub = lane / TC_LANES, sl = lane % TC_LANES;
  const int stride = gridDim.x * (blockDim.x / TC_LANES);
  // warp-uniform trip count so that the votes below see the full warp
  for (int base = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / TC_LANES; base < total; base += stride) {
    const int uu = base + sub;
    bool sel = false, beaten = false;
    int e = 0, t = 0;
    if (uu < total) {
      e = find_event(s_pref, n_events, uu);
      const EvDesc &ev = evs[e];
      t = uu - s_pref[e];
      sel = ev.t5_sel[t] != 0;
      if (sel) {
        int mt[5];
        t5_mds(ev, t, mt);
        const float qt = tc_rank(__int_as_float(ev.t5_b[t].w));
        // a duplicate shares >= 3 of t's 5 MDs, so at least one of t's middle three: the
        // lists of md1..md3 (every selected T5 is listed under all 5 of its MDs) hold them all
        for (int j = 1; j <= 3 && !beaten; j++) {
          const int end = ev.tc_pos[mt[j]], beg = end - ev.tc_cnt[mt[j]];
          for (int k = beg + sl; k < end && !beaten; k += TC_LANES) {
            const int u = ev.tc_list[k];
            if (u == t) continue;
            const int4 ua = ev.t5_a[u], ub = ev.t5_b[u];
            const int mu[5] = {ua.x, ua.y, ua.z, ua.w, ub.x};
            int shared = 0;
#pragma unroll
            for (int a = 0; a < 5; a++)
#pragma unroll
              for (int b = 0; b < 5; b++) shared += mt[a] == mu[b];
            if (shared < TC_MIN_SHARED) continue;
            const float qu = tc_rank(__int_as_float(ub.w));
            if (qu < qt || (qu == qt && key_less(ev, mu, mt))) beaten = true;
          }
        }
      }
    }
    const unsigned gmask = ((1u << TC_LANES) - 1) << (sub * TC_LANES);
    const unsigned vb = __ballot_sync(FULL, beaten);        // every lane votes (not under &&)
    const bool keep = sel && (vb & gmask) == 0;
    if (uu < total && sl == 0) evs[e].t5_tc[t] = keep ? 1 : 0;
    const bool lead = uu < total && sl == 0;
    const unsigned act = __ballot_sync(FULL, lead);
    if (lead) {
      const unsigned same = __match_any_sync(act, e);
      const unsigned kb = __ballot_sync(act, keep) & same;
      if ((same & lanemask_lt()) == 0 && kb) atomicAdd(evs[e].cnt + C_NTC, __popc(kb));
    }
  }
}

}  // namespace lstk
