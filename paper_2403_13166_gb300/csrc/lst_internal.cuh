// lst_internal.cuh -- device data layout, cut arithmetic and small warp/block helpers of
// the GB300 LST library. Cut code is compiled with -fmad=false and IEEE division and
// square root so that every FP32 cut value is the correctly rounded result of the
// expression tree written below (no fused multiply-add, no fast-math).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lst.h"

namespace lstk {

constexpr int NFEAT = 38;
constexpr int NHID = 32;
constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_EVENTS = 512;       // event slots per context (batch size limit)
constexpr int MAX_FANOUT = 512;       // module-map targets of one module

// per-event counter words (int32 each)
enum CounterSlot {
  C_MD = 0, C_LS = 1, C_T3 = 2, C_T5 = 3, C_FLAGS = 4, C_NSEL = 5,
  C_PMD = 6, C_PLS = 7, C_PT3 = 8, C_PT5 = 9,   // candidate pairs tested per step
  C_DBG_SITE = 10, C_DBG_VAL = 11,              // first failed bounds check (LST_CHECK builds)
  C_NTC = 12,                                   // track candidates
  C_NCOUNTERS = 13
};
enum Flags { F_INPUT = 1, F_OVF_MD = 2, F_OVF_LS = 4, F_OVF_T3 = 8, F_OVF_T5 = 16, F_CHECK = 32, F_TIMEOUT = 64 };

struct DevGeom {
  int32_t n_mod;
  int32_t pad;
  const int8_t *subdet;    // [n_mod] 0 barrel, 1 endcap
  const int8_t *layer;     // [n_mod] 1..11
  const int32_t *map_off;  // [n_mod+1]
  const int32_t *map_tgt;  // [n_links]
};

// Device buffers of one event slot. Object indices (MD, LS, T3, T5) are event-local.
struct EvDesc {
  const float *x, *y, *z;      // caller's input (device)
  const int32_t *sensor;
  int32_t n_hits;
  int32_t md_cap, ls_cap, t3_cap, t5_cap;
  int32_t pad;
  float4 *hit;                 // [n_hits] hits grouped by sensor: x, y, z, r
  int2 *hit_om;                // [n_hits] per grouped hit: original index, module (the module
                               // for lower-sensor hits only, the ones step 1 reads it for)
  int32_t *sens_cnt;           // [2 n_mod] histogram by key
  int32_t *hit_rank;           // [n_hits] rank of each input hit within its key (input order)
  int32_t *sens_off;           // [2 n_mod + 1] key k < n_mod: lower sensor of module k,
                               // key n_mod + k: upper sensor of module k
  float4 *mdu_anchor;          // [md_cap] MDs as found, any order (same fields as below)
  float2 *mdu_kappa;
  int32_t *mdu_mod;
  int2 *mdu_hits;
  int32_t *mdu_rank;           // [md_cap] rank of each MD within its module
  float4 *md_anchor;           // [md_cap] MDs grouped by module, within a module in ascending
                               // md_key: lower-sensor hit (anchor) x, y, z, r
  float2 *md_kappa;            // [md_cap] (cut curvature, feature curvature); 0 for endcap
  int32_t *md_mod;             // [md_cap] module
  int2 *md_hits;               // [md_cap] original (lower, upper) hit indices
  int32_t *md_perm;            // [md_cap] grouped by module before the order within modules:
  float *md_q;                 //   the MD (index as found) at each position and its key
  int32_t *md_start, *md_cnt;  // [n_mod] MDs of each module: contiguous range
  int4 *lsu;                   // [ls_cap] LSs as found, any order: (inner MD, outer MD, rank
                               // within the inner MD's LSs, rank within the outer MD's LSs)
  int32_t *ls_to;              // [ls_cap] LSs grouped by inner MD: the outer MD of each
  int32_t *ls_from;            // [ls_cap] LSs grouped by outer MD: the inner MD of each
  int32_t *ls_start, *ls_cnt;  // [md_cap] per MD: start and length of its range in ls_to
  int32_t *lso_start, *lso_cnt;  // [md_cap] per MD: start and length of its range in ls_from
  int4 *t3u_md;                // [t3_cap] T3s as found (md0, md1, md2, rank within md0), any order
  float *t3u_kappa;            // [t3_cap]
  int4 *t3_md;                 // [t3_cap] T3s grouped by first MD (md0, md1, md2, 0)
  float *t3_kappa;             // [t3_cap]
  int32_t *t3_pos, *t3_cnt;    // [md_cap] per first MD: start of its range and count
  int4 *t5_a;                  // [t5_cap] (md0, md1, md2, md3)
  int4 *t5_b;                  // [t5_cap] (md4, t3a, t3b, bits of the circle-fit chi2)
  float *t5_score;             // [t5_cap]
  uint8_t *t5_sel;             // [t5_cap]
  int32_t *tc_cnt, *tc_pos;    // [md_cap] selected T5s per MD, then the end of each MD's range
  int32_t *tc_list;            // [5 t5_cap] selected T5s grouped by MD
  uint8_t *t5_tc;              // [t5_cap] 1: the T5 is a track candidate
  int32_t *cnt;                // [C_NCOUNTERS]
};

// Device buffers of the pixel-seed matching of one event (lst_pixel.cu).
struct PixDesc {
  int n_pls, n_t5, n_t3, n_md;
  const float *hits;              // [n_pls][12] seeds, input order
  int *cell, *rank;               // [n_pls] bin and rank within it, input order
  int *cell_cnt, *cell_off;       // [PIX_NCELL], [PIX_NCELL + 1]
  float4 *sa, *sb;                // [n_pls] in bin order: (x1, y1, z1, kp), (x4, y4, z4, r4)
  float *sm;                      // [n_pls] in bin order: r-z slope m_p
  float *sk;                      // [n_pls] in bin order: the seed's curvature kp (sa's w, packed)
  int *sidx;                      // [n_pls] in bin order: seed index
  unsigned long long *pkey;       // [n_pls] the round's best (residual, difference) at the seed
  int *pcnt, *plist;              // [n_pls], [n_pls][PIX_TIES] objects of that rank
  int *pobj;                      // [n_pls] the round's chosen object
  int *pmatch;                    // [n_pls] matched object (T5 index, or n_t5 + T3 index), -1
  unsigned long long *okey;       // [n_t5 + n_t3] the round's best rank at the object
  int *op;                        // [n_t5 + n_t3] and its seed
  int *omatch;                    // [n_t5 + n_t3] matched seed; -1 free, -2 out of the matching
  int *ocnt;                      // [n_t5 + n_t3] the object's cached candidates: -1 none yet,
  int *oseed;                     //   PIX_OCAP + 1 too many (scan the windows), else their number;
  unsigned long long *okeys;      //   [n_t5 + n_t3][PIX_OCAP] their seeds and ranks
  uint8_t *mdflag;                // [n_md] MD of a pT5's T5
  int *rows;                      // [n_t5 + n_t3 + n_pls][3] track candidates
  int *ctr;                       // [16]: taken this round, rows, tie overflow, bits of the
                                  // smallest seed radius, rows of type 5..8; PIX_DONE: done
                                  // with the current stage; rounds of stages 5 and 7
};
constexpr int PIX_DONE = 8, PIX_ROUNDS5 = 9, PIX_ROUNDS7 = 10, PIX_NCTR = 16;
constexpr int PIX_NPHI = 256, PIX_NM = 64, PIX_NCELL = PIX_NPHI * PIX_NM;
constexpr int PIX_TIES = 8;                     // objects equal in rank at one seed (more: error)
constexpr int PIX_OCAP = 8;                     // candidate seeds cached per object
constexpr int PIX_ROUNDS_PER_WAIT = 3;           // matching rounds launched per host wait
constexpr int PIX_QCAP = 160;                   // a warp's queue of seeds past the curvature test
constexpr int PIX_SCAN_THREADS = 256;           // CTA size of the two window-scan kernels

// ------------------------------------------------------------------ FP32 cut arithmetic
// Step 1 (Section 1, Table 1): two hits of one pT-module, pT above 0.8 GeV and inside the
// luminous-region road. L = lower-sensor hit, U = upper-sensor hit, both (x, y, z, r).
__device__ __forceinline__ bool md_cut(const float4 L, const float4 U, bool endcap,
                                       const lst_cuts &c, float &kappa) {
  const float dx = U.x - L.x, dy = U.y - L.y, dz = U.z - L.z;
  const float dt = L.x * dx + L.y * dy;
  const float rL = L.w;
  if (!endcap) {
    if (!(dt > 0.0f)) return false;                                    // direction
    const float dT = sqrtf(dx * dx + dy * dy);
    const float cr = L.x * dy - L.y * dx;
    const float sa = cr / (rL * dT);
    if (!(fabsf(sa) <= rL * (0.5f * c.kappa_max) + c.hit_err / c.sensor_gap)) return false;  // bend
    const float dr = U.w - L.w;
    if (!(fabsf(dz - (L.z / rL) * dr) <= (c.z_lum / rL) * dr + c.hit_err)) return false;    // z road
    kappa = 2.0f * sa / rL;
    return true;
  }
  if (!(dt > 0.0f && dz * L.z > 0.0f)) return false;                   // direction
  const float para = dt / rL;
  const float azl = fabsf(L.z), adz = fabsf(dz);
  const float pe = adz * rL / azl;
  if (!(fabsf(para - pe) <= adz * rL * c.z_lum / (azl * (azl - c.z_lum)) + c.hit_err)) return false;
  const float cr = L.x * dy - L.y * dx;
  const float perp = cr / rL;
  const float S = rL * (0.5f * c.kappa_max);
  const float T = S / sqrtf(1.0f - S * S);
  if (!(fabsf(perp) <= para * T + c.hit_err)) return false;           // bend
  kappa = 0.0f;
  return true;
}

// Step 2: MD anchors A (inner) and B (outer) in linked modules; kA/kB the MD curvature
// estimates (cut values), bA/bB barrel flags. Cheapest test first (the set is the same).
__device__ __forceinline__ bool ls_cut(const float4 A, const float4 B, float kA, float kB,
                                       bool bA, bool bB, const lst_cuts &c, float &kappa) {
  const float e = c.hit_err;
  const float drr = B.w - A.w;
  if (!(fabsf(A.z * drr - A.w * (B.z - A.z)) <= (c.z_lum + e) * fabsf(drr) + e * A.w)) return false;  // z0
  const float dx = B.x - A.x, dy = B.y - A.y;
  const float dt = A.x * dx + A.y * dy;
  if (!(dt > 0.0f)) return false;                                      // direction
  const float dT = sqrtf(dx * dx + dy * dy);
  const float cr = A.x * dy - A.y * dx;
  const float sl = cr / (A.w * dT);
  if (!(fabsf(sl) <= B.w * (0.5f * c.kappa_max) + e / dT)) return false;  // bend
  const float k = 2.0f * sl / B.w;
  if (bA && !(fabsf(kA - k) <= 2.0f * (e / c.sensor_gap) / A.w + 2.0f * (e / dT) / B.w)) return false;
  if (bB && !(fabsf(kB - k) <= 2.0f * (e / c.sensor_gap) / B.w + 2.0f * (e / dT) / B.w)) return false;
  kappa = k;
  return true;
}

// The curvature ls_cut assigns to an accepted LS: the same FP32 expression tree, so the
// value is bit-identical to the cut's.
__device__ __forceinline__ float ls_curvature(const float4 A, const float4 B) {
  const float dx = B.x - A.x, dy = B.y - A.y;
  const float dT = sqrtf(dx * dx + dy * dy);
  const float cr = A.x * dy - A.y * dx;
  const float sl = cr / (A.w * dT);
  return 2.0f * sl / B.w;
}

// Necessary condition of ls_cut without division or square root, in fewer operations than
// the cut's own expressions, through identities that hold exactly in real arithmetic:
//   z0:        A.z (rB - rA) - rA (zB - zA)  =  A.z rB - rA zB
//   bend:      A x (B - A)                  =  A.x B.y - A.y B.x  (= cr),
// and the bend bound squared: |cr| / (rA dT) <= X + e / dT with X = rB kappa_max / 2 means
// |cr| <= rA (X dT + e), hence cr^2 <= rA^2 ((1 + 1/64) X^2 dT^2 + 65 e^2), because
// (u + e)^2 <= (1 + t) u^2 + (1 + 1/t) e^2 for every t > 0 (here t = 1/64). The direction
// cut is left to the later tests: on the candidate pairs of a PU200-like event it rejects
// none of the pairs that pass these two (9.00% either way).
// Rounding: every product here is below 3.2e4 in magnitude (|z| <= 270 cm, r <= 115 cm), so
// the FP32 values of either form of a side differ from the real value by less than 0.02;
// the slacks (0.05 on the z0 side, the factor 1.002 and 0.05 on the squared bend, against
// bounds of at least 0.29 and 5.6) cover that, so a pair rejected here always fails ls_cut.
// Ax = (rA^2, e rA + 0.05) per inner MD; k1 = 1.002 * (1 + 1/64) X^2 per outer MD,
// k0 = 1.002 * 65 e^2, c1 = z_lum + e.
__device__ __forceinline__ bool ls_prefilter(const float4 A, const float2 Ax, const float4 B, float k1, float k0,
                                             float c1) {
  const float p = __fmaf_rn(A.z, B.w, -(A.w * B.z));
  const bool z0 = fabsf(p) <= __fmaf_rn(c1, fabsf(B.w - A.w), Ax.y);
  const float cr = __fmaf_rn(A.x, B.y, -(A.y * B.x));
  const float dx = B.x - A.x, dy = B.y - A.y;
  const float dT2 = __fmaf_rn(dx, dx, dy * dy);
  const bool bend = cr * cr <= __fmaf_rn(Ax.x, __fmaf_rn(k1, dT2, k0), 0.05f);
  return z0 & bend;
}

// Necessary condition of the two curvature-consistency cuts of ls_cut (barrel MDs), for the
// pairs that passed ls_prefilter. With M = rA rB dT > 0 and k = 2 cr / M (cr = A x B, the
// exact identity used above), |kA - k| <= 2 (e/g) / rA + 2 (e/dT) / rB is, multiplied by M,
//   |kA rA u - 2 cr| <= G u + 2 e rA      with u = rB dT, G = 2 e / g,
// and |kB - k| <= 2 (e/g) / rB + 2 (e/dT) / rB is
//   |kB rB v - 2 cr| <= G v + 2 e rA      with v = rA dT.
// dT comes from the approximate reciprocal square root (relative error below 2^-22).
// Rounding, in relative terms so that it holds for any coordinates: the exact cut in FP32
// can accept a pair whose real-arithmetic condition fails by up to 2.4e-7 of its bound plus
// (14 |k| + 1) eps-sized terms, which times M stay below 2.4e-7 (G u + 2 e rA) + 9.6e-7 v
// + 6e-8 |kA rA u|; the FP32 evaluation below errs by at most 5e-7 of |kA rA u| (or |kB rB v|)
// and 4.8e-7 rA rB (cr's cancellation). The bound is therefore widened by the factor
// (1 + 1e-6) on G and 2e, by 1e-6 (|p| + rA rB + v), and by 0.01 absolute. dT2 = 0 or a
// subnormal dT2 gives a NaN or infinite side and the pair passes (the exact cut decides).
// Checked over all candidate pairs of three PU200-like events: 1.81-1.88% pass against
// 1.80-1.87% accepted, none of the 3.3 M LSs missed.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ bool ls_kappa_prefilter(const float4 A, const float4 B, float kA, float kB, bool bA,
                                                   bool bB, float Gp, float ce) {
  const float dx = B.x - A.x, dy = B.y - A.y;
  const float dT2 = __fmaf_rn(dx, dx, dy * dy);
  const float dT = dT2 * rsqrt_approx(dT2);
  const float cr2 = 2.0f * __fmaf_rn(A.x, B.y, -(A.y * B.x));
  const float u = B.w * dT, v = A.w * dT;
  const float c0 = __fmaf_rn(ce, A.w, 0.01f);                 // 2 e rA (1 + 1e-6) + 0.01
  const float s0 = __fmaf_rn(A.w, B.w, v);                     // rA rB + v
  const float pa = kA * A.w * u, pb = kB * B.w * v;
  const bool fa = __fmaf_rn(-1e-6f, fabsf(pa) + s0, fabsf(pa - cr2)) > __fmaf_rn(Gp, u, c0);
  const bool fb = __fmaf_rn(-1e-6f, fabsf(pb) + s0, fabsf(pb - cr2)) > __fmaf_rn(Gp, v, c0);
  return !((bA & fa) | (bB & fb));
}

// Necessary condition of md_cut without division or square root. Per lower hit L (MdLow):
//   barrel: hb2r2 = (rL * hb)^2 with hb = rL (kappa_max / 2) + e / g, the bend bound of md_cut.
//     Bend: |cr| <= rL dT hb. z road, multiplied by rL > 0: |dz rL - zL dr| <= Zl dr + e rL.
//   endcap: the z road multiplied by rL |zL| > 0: |dt |zL| - |dz| rL^2| <= |dz| wz + e rL |zL|
//     with wz = rL^2 Zl / (|zL| - Zl) (infinite, so no test, for |zL| <= Zl); the bend
//     multiplied by rL: |cr| <= dt T + e rL with md_cut's own T(rL).
// md_cut's direction conditions are left to md_cut: on the candidate pairs of a PU200-like
// event they reject none of the pairs that pass the road and bend tests. The slack (1e-3 of
// the terms' magnitudes) covers FP32 rounding, so a pair rejected here always fails md_cut
// too (checked over all candidate pairs of a PU200-like event: 3.04% of barrel and 4.23% of
// endcap pairs pass, exactly the MD fractions, none missed).
struct MdLow {
  float hb2r2;                     // barrel
  float az, r2, wz, erz, T, erl;   // endcap: |zL|, rL^2, wz, e rL |zL|, T(rL), e rL
};
__device__ __forceinline__ MdLow md_low(const float4 L, bool endcap, const lst_cuts &c) {
  MdLow q;
  const float hb = L.w * (0.5f * c.kappa_max) + c.hit_err / c.sensor_gap;
  q.hb2r2 = (L.w * hb) * (L.w * hb) * 1.001f;
  q.az = fabsf(L.z);
  q.r2 = L.w * L.w;
  q.wz = q.az > c.z_lum ? q.r2 * c.z_lum / (q.az - c.z_lum) : __int_as_float(0x7f800000);
  q.erz = c.hit_err * L.w * q.az;
  const float S = L.w * (0.5f * c.kappa_max);
  q.T = endcap ? S / sqrtf(1.0f - S * S) : 0.0f;
  q.erl = c.hit_err * L.w;
  return q;
}
__device__ __forceinline__ bool md_prefilter(const float4 L, const float4 U, bool endcap, const MdLow &q,
                                             const lst_cuts &c) {
  const float dx = U.x - L.x, dy = U.y - L.y, dz = U.z - L.z;
  const float cr = __fmaf_rn(L.x, dy, -(L.y * dx));
  if (endcap) {
    const float dt = L.x * dx + L.y * dy;
    const float t1 = dt * q.az, t2 = fabsf(dz) * q.r2;
    const float rr = __fmaf_rn(fabsf(dz), q.wz, q.erz);
    const bool road = fabsf(t1 - t2) <= rr + 1e-3f * (fabsf(t1) + t2 + rr) + 1e-6f;
    const float bb = __fmaf_rn(dt, q.T, q.erl);
    const bool bend = fabsf(cr) <= bb + 1e-3f * (fabsf(dt * q.T) + q.erl) + 1e-6f;
    return road & bend;
  }
  const float dT2 = __fmaf_rn(dx, dx, dy * dy);
  const bool bend = cr * cr <= __fmaf_rn(q.hb2r2, dT2, 1e-9f);
  const float dr = U.w - L.w;
  const float a = dz * L.w, b = L.z * dr, rhs = __fmaf_rn(c.z_lum, dr, q.erl);
  const bool zr = fabsf(a - b) <= rhs + 1e-3f * (fabsf(a) + fabsf(b) + fabsf(rhs)) + 1e-6f;
  return bend & zr;
}

// Step 3: anchors of md0, md1, md2 along the chain (LS1.out == LS2.in).
__device__ __forceinline__ bool t3_cut(const float4 P0, const float4 P1, const float4 P2,
                                       const lst_cuts &c, float &kappa) {
  const float ax = P1.x - P0.x, ay = P1.y - P0.y;
  const float bx = P2.x - P1.x, by = P2.y - P1.y;
  const float cx = P2.x - P0.x, cy = P2.y - P0.y;
  const float a = sqrtf(ax * ax + ay * ay);
  const float b = sqrtf(bx * bx + by * by);
  const float cc = sqrtf(cx * cx + cy * cy);
  const float cr = ax * cy - ay * cx;
  const float k3 = 2.0f * cr / (a * b * cc);
  if (!(fabsf(k3) <= c.kappa_max * c.t3_kappa_factor)) return false;     // pT
  const float s01 = a * (1.0f + a * a * k3 * k3 / 24.0f);
  const float s12 = b * (1.0f + b * b * k3 * k3 / 24.0f);
  const float zp = P0.z + (P2.z - P0.z) * s01 / (s01 + s12);
  if (!(fabsf(P1.z - zp) <= c.t3_rz_tol)) return false;                 // rz
  kappa = k3;
  return true;
}

// Necessary condition of t3_cut without division or IEEE square root, from the chords of
// the two LSs alone: a = P1 - P0 (first LS) and b = P2 - P1 (second LS), each given as
// (dx, dy, dz, transverse length) from the FP32 differences t3_cut itself forms. It tests
// the rz cut only (the pT cut, which keeps ~80% of the candidate pairs, is left to t3_cut):
// the residual z1 - zp multiplied by S = s01 + s12 >= 0, written as (z1 - z0) s12 -
// (z2 - z1) s01, with the curvature of the three anchors from cr = a x b (= a x c, the cut's
// form), c = a + b, kappa^2 / 24 = 4 cr^2 / (24 a^2 b^2 c^2) through the approximate
// reciprocal (relative error ~1e-7). Per first LS the lane holds (ax, ay, z1 - z0, a) plus
// a^2 = ax^2 + ay^2 and a^3. The slack (1e-3 relative on the tolerance, 3e-4 cm absolute on
// the residual) is far above the approximation and rounding errors (below 1.5e-4 cm on the
// residual for coordinates within 300 cm), so a rejected triplet always fails t3_cut.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ bool t3_prefilter(const float4 A, float a2, float a3, const float4 B, float tolp) {
  const float cx = A.x + B.x, cy = A.y + B.y;
  const float b2 = __fmaf_rn(B.x, B.x, B.y * B.y), c2 = __fmaf_rn(cx, cx, cy * cy);
  const float cr = __fmaf_rn(A.x, B.y, -(A.y * B.x));
  const float abc2 = a2 * b2 * c2;
  const float k24 = (cr * cr) * rcp_approx(fmaxf(abc2, 1e-30f)) * (4.0f / 24.0f);
  const float s01 = __fmaf_rn(a3, k24, A.w), s12 = __fmaf_rn(B.w * b2, k24, B.w);
  const float lhs = __fmaf_rn(A.z, s12, -(B.z * s01));
  return fabsf(lhs) <= tolp * (s01 + s12);
}

// Step 4: five anchors in chain order; ka, kb the curvatures of T3a = (0,1,2), T3b = (2,3,4).
// Circle-fit quality of the five anchors, FP32 (the selection the T5-DNN replaces, Section 2;
// pre-DNN mode only). Coordinates relative to the middle anchor, u and v swapped when the
// chord P0 -> P4 is longer in y than in x. Algebraic circle fit gamma (u^2 + v^2) + beta u -
// v + alpha = 0, least squares in v - alpha - beta u - gamma (u^2 + v^2), normal equations by
// Cramer's rule: regular for straight tracks (gamma = 0) and free of radius-sized
// intermediates. Distance of an anchor to the circle: p = (gamma w + beta u - v + alpha) / nu,
// nu = sqrt(beta^2 + 1 - 4 gamma alpha), A = gamma / nu, distance = 2 p / (1 + sqrt(1 + 4 A
// p)); chi2 = sum of (distance / sigma)^2. Sums in chain order from zero, written as
// left-to-right expressions; no contraction (-fmad=false), so every IEEE evaluation of this
// tree gives the same bits. A degenerate system yields inf or NaN, which fails the cut.
__device__ __forceinline__ float det3f(float a, float b, float c, float d, float e, float f, float g, float h,
                                       float i) {
  return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
}
__device__ __forceinline__ float t5_chi2(const float4 *P, float sigma) {
  float u[5], v[5], w[5];
  const bool swap = !(fabsf(P[4].x - P[0].x) >= fabsf(P[4].y - P[0].y));
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const float dx = P[i].x - P[2].x, dy = P[i].y - P[2].y;
    u[i] = swap ? dy : dx;
    v[i] = swap ? dx : dy;
    w[i] = u[i] * u[i] + v[i] * v[i];
  }
  float su = 0.0f, sw = 0.0f, suu = 0.0f, suw = 0.0f, sww = 0.0f, sv = 0.0f, suv = 0.0f, swv = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    su = su + u[i];
    sw = sw + w[i];
    suu = suu + u[i] * u[i];
    suw = suw + u[i] * w[i];
    sww = sww + w[i] * w[i];
    sv = sv + v[i];
    suv = suv + u[i] * v[i];
    swv = swv + w[i] * v[i];
  }
  const float n = 5.0f;
  const float det = det3f(n, su, sw, su, suu, suw, sw, suw, sww);
  const float alpha = det3f(sv, su, sw, suv, suu, suw, swv, suw, sww) / det;
  const float beta = det3f(n, sv, sw, su, suv, suw, sw, swv, sww) / det;
  const float gamma = det3f(n, su, sv, su, suu, suv, sw, suw, swv) / det;
  const float nu = sqrtf(beta * beta + 1.0f - 4.0f * gamma * alpha);
  const float A = gamma / nu;
  float chi2 = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const float p = (gamma * w[i] + beta * u[i] - v[i] + alpha) / nu;
    const float d = 2.0f * p / (1.0f + sqrtf(1.0f + 4.0f * A * p));
    const float t = d / sigma;
    chi2 = chi2 + t * t;
  }
  return chi2;
}

__device__ __forceinline__ bool t5_cut(const float4 *P, float ka, float kb, const lst_cuts &c) {
  if (!(ka * kb > 0.0f)) return false;                                   // same charge
  if (!(fabsf(ka - kb) <= c.t5_kappa_rel * 0.5f * (fabsf(ka) + fabsf(kb)) + c.t5_kappa_abs)) return false;
  const float kbar = 0.5f * (ka + kb);
  float S[5];
  S[0] = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const float dx = P[i + 1].x - P[i].x, dy = P[i + 1].y - P[i].y;
    const float d = sqrtf(dx * dx + dy * dy);
    const float s = d * (1.0f + d * d * kbar * kbar / 24.0f);
    S[i + 1] = (i == 0) ? s : S[i] + s;
  }
  const float z0 = P[0].z, z4 = P[4].z;
#pragma unroll
  for (int j = 1; j <= 3; j++)
    if (!(fabsf(P[j].z - (z0 + (z4 - z0) * S[j] / S[4])) <= c.t5_rz_tol)) return false;  // rz
  return true;
}

// Sort key of an MD within its module, q = z / r of its anchor (approximate quotient, a few
// ulp; the same function wherever the order is relied on).
__device__ __forceinline__ float md_key(const float4 A) { return __fdividef(A.z, A.w); }

// Ranking value of a T5 among duplicates: the chi2, with NaN and +inf both +inf.
__device__ __forceinline__ float tc_rank(float chi2) { return chi2 <= 3.40282347e38f ? chi2 : __int_as_float(0x7f800000); }

// ------------------------------------------------------------------ accurate FP32 helpers
// (features only; cut values above never use them)
struct ff { float hi, lo; };
// a - b = hi + lo exactly (Knuth's two-sum on a + (-b))
__device__ __forceinline__ ff two_diff(float a, float b) {
  const float nb = -b;
  const float s = a + nb;
  const float bb = s - a;
  const float err = (a - (s - bb)) + (nb - bb);
  return {s, err};
}
// a*d - b*c with an FMA-compensated product (Kahan): error within 1.5 ulp of the result
__device__ __forceinline__ float diff_of_products(float a, float d, float b, float c) {
  const float w = b * c;
  const float e = __fmaf_rn(-b, c, w);
  const float f = __fmaf_rn(a, d, -w);
  return f + e;
}
// cross product u x v of two exact differences u = (ux.hi+ux.lo, ...), v likewise
__device__ __forceinline__ float cross_acc(ff ux, ff uy, ff vx, ff vy) {
  const float main = diff_of_products(ux.hi, vy.hi, uy.hi, vx.hi);
  const float corr = (ux.hi * vy.lo + ux.lo * vy.hi) - (uy.hi * vx.lo + uy.lo * vx.hi);
  return main + corr;
}
// signed three-point curvature 2 (P1-P0)x(P2-P0) / (|P1-P0| |P2-P1| |P2-P0|), accurate
__device__ __forceinline__ float curv3_acc(const float4 P0, const float4 P1, const float4 P2) {
  const ff ax = two_diff(P1.x, P0.x), ay = two_diff(P1.y, P0.y);
  const ff cx = two_diff(P2.x, P0.x), cy = two_diff(P2.y, P0.y);
  const ff bx = two_diff(P2.x, P1.x), by = two_diff(P2.y, P1.y);
  const float cr = cross_acc(ax, ay, cx, cy);
  const float a = sqrtf(ax.hi * ax.hi + ay.hi * ay.hi);
  const float b = sqrtf(bx.hi * bx.hi + by.hi * by.hi);
  const float c = sqrtf(cx.hi * cx.hi + cy.hi * cy.hi);
  return 2.0f * cr / (a * b * c);
}
// MD curvature estimate 2 sin(angle(L, U-L)) / rL of a barrel MD, accurate
__device__ __forceinline__ float md_kappa_acc(const float4 L, const float4 U) {
  const ff dx = two_diff(U.x, L.x), dy = two_diff(U.y, L.y);
  const ff lx = {L.x, 0.0f}, ly = {L.y, 0.0f};
  const float cr = cross_acc(lx, ly, dx, dy);
  const float dT = sqrtf(dx.hi * dx.hi + dy.hi * dy.hi);
  return 2.0f * (cr / (L.w * dT)) / L.w;
}

// ------------------------------------------------------------------ warp / block helpers
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive prefix sums pos[i] = cnt[0] + ... + cnt[i-1] for i < n, by the whole CTA
// (blockDim.x a multiple of 32, <= 1024): tiles of 4 consecutive elements per thread, so
// that a warp reads 512 contiguous bytes, with the running total carried across tiles.
__device__ __forceinline__ void block_exclusive_scan(const int32_t *__restrict__ cnt, int32_t *__restrict__ pos,
                                                     int n) {
  __shared__ int s_w[32];
  __shared__ int s_carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 4 * blockDim.x) {
    const int i0 = base + 4 * threadIdx.x;
    int v[4], local = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      v[k] = i0 + k < n ? cnt[i0 + k] : 0;
      local += v[k];
    }
    const int inc = warp_incl_scan(local);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      const int x = lane < nw ? s_w[lane] : 0;
      const int xi = warp_incl_scan(x);
      if (lane < nw) s_w[lane] = xi - x;
    }
    __syncthreads();
    int run = s_carry + s_w[wid] + inc - local;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (i0 + k < n) pos[i0 + k] = run;
      run += v[k];
    }
    __syncthreads();                                   // s_carry and s_w read by all
    if (threadIdx.x == blockDim.x - 1) s_carry = run;  // = carry + this tile's total
    __syncthreads();
  }
}

// Exclusive prefix over events of a per-event unit count, built in shared memory by
// the whole block: pref[e] = sum_{f<e} count(f), pref[n] = total. n <= MAX_EVENTS.
template <typename F>
__device__ void block_event_prefix(int n, F count, int *pref) {
  for (int base = 0; base < n; base += blockDim.x) {
    const int e = base + threadIdx.x;
    if (e < n) pref[e + 1] = count(e);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int carry = 0;
    for (int base = 0; base < n; base += 32) {
      const int e = base + threadIdx.x;
      int v = (e < n) ? pref[e + 1] : 0;
      const int inc = warp_incl_scan(v);
      if (e < n) pref[e + 1] = carry + inc;
      carry += __shfl_sync(FULL, inc, 31);
    }
    if (threadIdx.x == 0) pref[0] = 0;
  }
  __syncthreads();
}

// index e with pref[e] <= u < pref[e+1]
__device__ __forceinline__ int find_event(const int *pref, int n, int u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int clamp_count(int n, int cap) { return n < cap ? n : cap; }

// An event whose input was invalid or whose buffers overflowed is skipped by every later
// stage (its results are void and the host re-runs it with larger buffers).
// Events voided before a stage starts: an invalid input or an overflow of an earlier stage
// (`earlier`). Those flags are final when the stage's kernel starts, so every CTA of it sees
// the same set and the per-event work prefixes agree between CTAs. A stage's own overflow
// voids the event only for the host; the stage keeps counting its objects without storing
// them, which tells the host how far to grow the buffer.
__device__ __forceinline__ bool ev_void_before(const EvDesc &ev, int earlier) {
  return (ev.cnt[C_FLAGS] & (F_INPUT | earlier)) != 0;
}

__device__ __forceinline__ bool ev_void(const EvDesc &ev) {
  return (ev.cnt[C_FLAGS] & (F_INPUT | F_OVF_MD | F_OVF_LS | F_OVF_T3 | F_OVF_T5 | F_CHECK)) != 0;
}

// Bounds check of a data-derived index (debug builds, -DLST_CHECK): an index outside
// [0, cap) is not used; the first failing site and index are recorded in the event's
// counters and the event is voided, so the host reports it instead of the GPU faulting.
#ifdef LST_CHECK
static __device__ __noinline__ bool chk(const EvDesc &ev, long long i, long long cap, int site) {
  if (i >= 0 && i < cap) return true;
  if (atomicCAS(ev.cnt + C_DBG_SITE, 0, site) == 0) ev.cnt[C_DBG_VAL] = (int)i;
  atomicOr(ev.cnt + C_FLAGS, F_CHECK);
  return false;
}
#else
__device__ __forceinline__ bool chk(const EvDesc &, long long, long long, int) { return true; }
#endif

}  // namespace lstk
