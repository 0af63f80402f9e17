/*
 * lst_oracle.c -- plain, slow, single-threaded CPU reference of the LST hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code, header or constant with
 * the CUDA library; both receive the same detector, module map, hits, cut parameters
 * and network weights as inputs.
 *
 * What it computes (arXiv 2403.13166, Section 1, Table 1 steps 1-4, and Section 2-3 for
 * the T5-DNN):
 *   step 1  mini-doublets (MD): two hits in one pT-module (one per sensor) that pass the
 *           MD cuts (the pT > 0.8 GeV requirement and the luminous-region road);
 *   step 2  line segments (LS): two MDs in modules linked by the module map
 *           ("nearby modules that fulfill some geometric criteria") with consistent pT;
 *   step 3  triplets (T3): two LSs sharing the common MD (outer MD of the first is the
 *           inner MD of the second);
 *   step 4  quintuplets (T5): two T3s sharing the common MD (last MD of the first is the
 *           first MD of the second); the middle three MDs form the "bridge" T3;
 *   score   38 input features -> Linear(38,32)+ReLU -> [Linear(32,32)+ReLU]* ->
 *           Linear(32,1) -> sigmoid, binary-cross-entropy classifier (Section 2);
 *           selected iff score >= working point (Section 3).
 * The paper prints no cut formula; the cuts below are the project's specification of
 * "consistency with a continuous, helical trajectory" (Section 1). Every cut is FP32,
 * written with the parentheses of that specification and evaluated in that order; build
 * with -ffp-contract=off so that no multiply-add is fused. Features and the network are
 * FP64.
 *
 * Loops run in the plainest order: modules, then hit pairs; modules, then map targets,
 * then MD pairs; LS pairs by common MD; T3 pairs by common MD. A brute-force mode drops
 * the module indexing (all hit pairs of a module's two sensors from the raw hit list,
 * all MD pairs in layer-adjacent modules, all LS/T3 pairs tested for the shared MD).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NFEAT 38
#define NHID 32

typedef struct {
    float kappa_max, z_lum, hit_err, sensor_gap, t3_kappa_factor, t3_rz_tol, t5_kappa_rel,
        t5_kappa_abs, t5_rz_tol, t5_chi2_max, hit_sigma, k_field, wp;
} ocuts;

typedef struct {
    int32_t n_mod;
    const int32_t *layer, *subdet, *side;
    const int32_t *map_off, *map_tgt;
} ogeom;

typedef struct {
    int32_t n_hidden;      /* hidden layers, 1..4, width 32 */
    const double *w;       /* W0(32x38),b0(32),[Wh(32x32),bh(32)]*,Wout(32),bout(1) */
} omlp;

typedef struct {
    int64_t n_md, n_ls, n_t3, n_t5;
    int64_t pairs[4];                     /* candidate pairs tested per step */
    int64_t near[4];                      /* of those, tested pairs near a cut boundary */
    int32_t *md_lo, *md_up, *md_mod;       /* original hit indices, module */
    float *md_kappa;                       /* signed curvature estimate (0 for endcap) */
    int32_t *ls_in, *ls_out;               /* MD indices */
    float *ls_kappa;
    int32_t *t3_ls1, *t3_ls2, *t3_md;      /* t3_md: [n][3] */
    float *t3_kappa;
    int32_t *t5_t3a, *t5_t3b, *t5_md;      /* t5_md: [n][5] */
    double *t5_feat, *t5_score;            /* [n][38], [n] */
    uint8_t *t5_sel;
    float *t5_chi2;                        /* [n] circle-fit chi2 of the five anchors */
    uint8_t *t5_tc;                        /* [n] 1: the T5 is a track candidate */
    int64_t n_pix;                         /* pixel-seed track candidates (steps 5-8) */
    int32_t *pix_tc;                       /* [n_pix][3]: type (5 pT5, 6 T5, 7 pT3, 8 pLS),
                                              pLS index (-1 for type 6), T5 / T3 index (-1 for 8) */
    int64_t pix_ties;                      /* greedy choices between edges of equal residual */
} oresult;

typedef struct {
    float kappa_rel, kappa_abs, rz_tol, dphi0, dphi_cm, dm_abs, dm_rel;
} opcuts;

/* ------------------------------------------------------------------ growable arrays */
typedef struct { void *p; int64_t n, cap; size_t es; } vec;
static void vinit(vec *v, size_t es) { v->p = NULL; v->n = 0; v->cap = 0; v->es = es; }
static void *vpush(vec *v) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->p = realloc(v->p, (size_t)v->cap * v->es);
    }
    return (char *)v->p + (size_t)(v->n++) * v->es;
}

typedef struct { float x, y, z, r; } hit;
typedef struct { int32_t lo, up, mod; float kappa; double kfeat; } md_t;
typedef struct { int32_t in, out; float kappa; } ls_t;
typedef struct { int32_t ls1, ls2, md[3]; float kappa; } t3_t;
typedef struct { int32_t t3a, t3b, md[5]; } t5_t;

static hit mkhit(const float *x, const float *y, const float *z, int32_t i) {
    hit h;
    h.x = x[i]; h.y = y[i]; h.z = z[i];
    h.r = sqrtf(h.x * h.x + h.y * h.y);
    return h;
}

/* ------------------------------------------------------------------ near-boundary count */
/* Bookkeeping for the parity report; it decides nothing. A tolerance comparison
 * lhs <= rhs whose sides differ by at most 1e-5 of rhs marks the candidate being tested as
 * near a cut boundary, where a different rounding of the same expression could flip the
 * decision; the event driver counts such candidates per step (oresult.near). */
static _Thread_local int g_near;

static int cut_le(float lhs, float rhs)
{
    if (fabs((double)lhs - (double)rhs) <= 1e-5 * fabs((double)rhs)) g_near = 1;
    return lhs <= rhs;
}

/* ------------------------------------------------------------------ step 1: MD cuts */
/* Lower hit L, upper hit U of one module. Returns 1 if the pair is a mini-doublet. */
int oracle_md_cut(const float *Lp, const float *Up, int endcap, const ocuts *c, float *kappa)
{
    hit L = {Lp[0], Lp[1], Lp[2], Lp[3]}, U = {Up[0], Up[1], Up[2], Up[3]};
    float dx = U.x - L.x, dy = U.y - L.y, dz = U.z - L.z;
    float dT = sqrtf(dx * dx + dy * dy);
    float cr = L.x * dy - L.y * dx;
    float dt = L.x * dx + L.y * dy;
    float rL = L.r;
    if (!endcap) {
        if (!(dt > 0.0f)) return 0;                                       /* MD-dir */
        float sa = cr / (rL * dT);
        if (!cut_le(fabsf(sa), rL * (0.5f * c->kappa_max) + c->hit_err / c->sensor_gap))
            return 0;                                                      /* MD-bend */
        float dr = U.r - L.r;
        if (!cut_le(fabsf(dz - (L.z / rL) * dr), (c->z_lum / rL) * dr + c->hit_err))
            return 0;                                                      /* MD-z */
        *kappa = 2.0f * sa / rL;
        return 1;
    }
    if (!(dt > 0.0f && dz * L.z > 0.0f)) return 0;                        /* MD-dir */
    float para = dt / rL, perp = cr / rL;
    float azl = fabsf(L.z), adz = fabsf(dz);
    float pe = adz * rL / azl;
    if (!cut_le(fabsf(para - pe), adz * rL * c->z_lum / (azl * (azl - c->z_lum)) + c->hit_err))
        return 0;                                                          /* MD-z */
    float S = rL * (0.5f * c->kappa_max);
    float T = S / sqrtf(1.0f - S * S);
    if (!cut_le(fabsf(perp), para * T + c->hit_err)) return 0;            /* MD-bend */
    *kappa = 0.0f;
    return 1;
}

/* ------------------------------------------------------------------ step 2: LS cuts */
/* Anchors A (inner MD) and B (outer MD); kA/kB the MD curvatures, bA/bB barrel flags. */
int oracle_ls_cut(const float *Ap, const float *Bp, float kA, float kB, int bA, int bB,
                  const ocuts *c, float *kappa)
{
    float xa = Ap[0], ya = Ap[1], za = Ap[2], ra = Ap[3];
    float xb = Bp[0], yb = Bp[1], zb = Bp[2], rb = Bp[3];
    float e = c->hit_err;
    if (!cut_le(fabsf(za * (rb - ra) - ra * (zb - za)), (c->z_lum + e) * fabsf(rb - ra) + e * ra))
        return 0;                                                          /* LS-z0 */
    float dx = xb - xa, dy = yb - ya;
    float dT = sqrtf(dx * dx + dy * dy);
    float cr = xa * dy - ya * dx;
    float dt = xa * dx + ya * dy;
    if (!(dt > 0.0f)) return 0;                                           /* LS-dir */
    float sl = cr / (ra * dT);
    if (!cut_le(fabsf(sl), rb * (0.5f * c->kappa_max) + e / dT)) return 0; /* LS-bend */
    float k = 2.0f * sl / rb;
    if (bA && !cut_le(fabsf(kA - k), 2.0f * (e / c->sensor_gap) / ra + 2.0f * (e / dT) / rb))
        return 0;                                                          /* LS-kappa, inner */
    if (bB && !cut_le(fabsf(kB - k), 2.0f * (e / c->sensor_gap) / rb + 2.0f * (e / dT) / rb))
        return 0;                                                          /* LS-kappa, outer */
    *kappa = k;
    return 1;
}

/* ------------------------------------------------------------------ step 3: T3 cuts */
int oracle_t3_cut(const float *P0, const float *P1, const float *P2, const ocuts *c,
                  float *kappa)
{
    float x0 = P0[0], y0 = P0[1], z0 = P0[2];
    float x1 = P1[0], y1 = P1[1], z1 = P1[2];
    float x2 = P2[0], y2 = P2[1], z2 = P2[2];
    float d01x = x1 - x0, d01y = y1 - y0;
    float d12x = x2 - x1, d12y = y2 - y1;
    float d02x = x2 - x0, d02y = y2 - y0;
    float a = sqrtf(d01x * d01x + d01y * d01y);
    float b = sqrtf(d12x * d12x + d12y * d12y);
    float cc = sqrtf(d02x * d02x + d02y * d02y);
    float cr = d01x * d02y - d01y * d02x;
    float k3 = 2.0f * cr / (a * b * cc);
    if (!cut_le(fabsf(k3), c->kappa_max * c->t3_kappa_factor)) return 0;  /* T3-pT */
    float s01 = a * (1.0f + a * a * k3 * k3 / 24.0f);
    float s12 = b * (1.0f + b * b * k3 * k3 / 24.0f);
    float zp = z0 + (z2 - z0) * s01 / (s01 + s12);
    if (!cut_le(fabsf(z1 - zp), c->t3_rz_tol)) return 0;                  /* T3-rz */
    *kappa = k3;
    return 1;
}

/* ------------------------------------------------------------------ step 4: T5 cuts */
/* P: the five anchors in chain order; ka/kb the curvatures of T3a=(0,1,2), T3b=(2,3,4). */
/* Circle-fit quality of the five anchors (x, y of P[4*i]), FP32: the selection the T5-DNN
 * replaces (Section 2), applied in the pre-DNN mode only.
 *   Coordinates relative to the middle anchor: u = x - x2, v = y - y2; u and v swap when the
 *   chord P0 -> P4 is longer in y than in x, so v runs across the chord.
 *   Algebraic circle fit: gamma (u^2 + v^2) + beta u - v + alpha = 0, least squares in the
 *   residual v - alpha - beta u - gamma (u^2 + v^2); 3x3 normal equations solved by Cramer's
 *   rule. A straight track is gamma = 0, so the fit stays regular at any radius and every
 *   term stays at tracker size (no cancellation of radius-sized numbers in FP32).
 *   Distance of each anchor to that circle: with nu = sqrt(beta^2 + 1 - 4 gamma alpha) the
 *   normalised residual p = (gamma w + beta u - v + alpha) / nu and A = gamma / nu give the
 *   signed distance 2 p / (1 + sqrt(1 + 4 A p)) (exact for a circle, no subtraction of
 *   radii); chi2 = sum of (distance / sigma)^2.
 * Every sum runs over the anchors in chain order from zero. A degenerate system gives inf
 * or NaN, which fails any chi2 cut. */
static float det3f(float a, float b, float c, float d, float e, float f, float g, float h, float i)
{
    return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
}

float oracle_t5_chi2(const float *P, float sigma)
{
    float u[5], v[5], w[5];
    int swap = !(fabsf(P[16] - P[0]) >= fabsf(P[17] - P[1]));
    for (int i = 0; i < 5; i++) {
        float dx = P[4 * i] - P[8], dy = P[4 * i + 1] - P[9];
        u[i] = swap ? dy : dx;
        v[i] = swap ? dx : dy;
        w[i] = u[i] * u[i] + v[i] * v[i];
    }
    float su = 0.0f, sw = 0.0f, suu = 0.0f, suw = 0.0f, sww = 0.0f, sv = 0.0f, suv = 0.0f, swv = 0.0f;
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
    float det = det3f(n, su, sw, su, suu, suw, sw, suw, sww);
    float alpha = det3f(sv, su, sw, suv, suu, suw, swv, suw, sww) / det;
    float beta = det3f(n, sv, sw, su, suv, suw, sw, swv, sww) / det;
    float gamma = det3f(n, su, sv, su, suu, suv, sw, suw, swv) / det;
    float nu = sqrtf(beta * beta + 1.0f - 4.0f * gamma * alpha);
    float A = gamma / nu;
    float chi2 = 0.0f;
    for (int i = 0; i < 5; i++) {
        float p = (gamma * w[i] + beta * u[i] - v[i] + alpha) / nu;
        float d = 2.0f * p / (1.0f + sqrtf(1.0f + 4.0f * A * p));
        float t = d / sigma;
        chi2 = chi2 + t * t;
    }
    return chi2;
}

int oracle_t5_cut(const float *P, float ka, float kb, const ocuts *c)
{
    if (!(ka * kb > 0.0f)) return 0;                                      /* T5-q */
    if (!cut_le(fabsf(ka - kb), c->t5_kappa_rel * 0.5f * (fabsf(ka) + fabsf(kb)) + c->t5_kappa_abs))
        return 0;                                                          /* T5-kappa */
    float kbar = 0.5f * (ka + kb);
    float S[5];
    S[0] = 0.0f;
    for (int i = 0; i < 4; i++) {
        float dx = P[4 * (i + 1)] - P[4 * i], dy = P[4 * (i + 1) + 1] - P[4 * i + 1];
        float d = sqrtf(dx * dx + dy * dy);
        float s = d * (1.0f + d * d * kbar * kbar / 24.0f);
        S[i + 1] = (i == 0) ? s : S[i] + s;
    }
    float z0 = P[2], z4 = P[18];
    for (int j = 1; j <= 3; j++) {
        float zj = P[4 * j + 2];
        if (!cut_le(fabsf(zj - (z0 + (z4 - z0) * S[j] / S[4])), c->t5_rz_tol)) return 0;  /* T5-rz */
    }
    if (c->t5_chi2_max > 0.0f && !cut_le(oracle_t5_chi2(P, c->hit_sigma), c->t5_chi2_max))
        return 0;                                                          /* pre-DNN chi2 */
    return 1;
}

/* ------------------------------------------------------------------ features (FP64) */
/* Signed three-point curvature 2*cross/(a*b*c) of transverse points (Menger curvature). */
static double curv3(const double *p0, const double *p1, const double *p2)
{
    double ax = p1[0] - p0[0], ay = p1[1] - p0[1];
    double bx = p2[0] - p1[0], by = p2[1] - p1[1];
    double cx = p2[0] - p0[0], cy = p2[1] - p0[1];
    double a = sqrt(ax * ax + ay * ay), b = sqrt(bx * bx + by * by), c = sqrt(cx * cx + cy * cy);
    double cr = ax * cy - ay * cx;
    return 2.0 * cr / (a * b * c);
}

/* |kappa| floor: radii above 1e7 cm are treated as 1e7 cm in the log features. */
static double kabs(double k) { double a = fabs(k); return a < 1e-7 ? 1e-7 : a; }

/* MD curvature estimate of a barrel MD in FP64 (same definition as the MD cut). */
static double md_kappa_fp64(const double *L, const double *U)
{
    double dx = U[0] - L[0], dy = U[1] - L[1];
    double dT = sqrt(dx * dx + dy * dy);
    double rL = sqrt(L[0] * L[0] + L[1] * L[1]);
    double cr = L[0] * dy - L[1] * dx;
    double sa = cr / (rL * dT);
    return 2.0 * sa / rL;
}

/* Section 2: pT and radius of each T3's circle, anchor (r, phi, z, eta, layer) plus the
 * MD curvature estimate for each of the 5 MDs, T5 pT/eta/phi, bridge-T3 radius. */
void oracle_t5_features(const double *anc /*[5][3]*/, const int32_t *layer /*[5]*/,
                        const double *mdk /*[5] FP64 MD curvature, 0 endcap*/, double kf,
                        double *f /*[38]*/)
{
    for (int i = 0; i < 5; i++) {
        double x = anc[3 * i], y = anc[3 * i + 1], z = anc[3 * i + 2];
        double r = sqrt(x * x + y * y);
        f[6 * i + 0] = r / 100.0;
        f[6 * i + 1] = atan2(y, x) / M_PI;
        f[6 * i + 2] = z / 100.0;
        f[6 * i + 3] = asinh(z / r) / 2.5;
        f[6 * i + 4] = layer[i] / 11.0;
        f[6 * i + 5] = 100.0 * mdk[i];
    }
    double ka = curv3(anc + 0, anc + 3, anc + 6);
    double kb = curv3(anc + 6, anc + 9, anc + 12);
    f[30] = log10(kf / kabs(ka));
    f[31] = log10(1.0 / kabs(ka));
    f[32] = log10(kf / kabs(kb));
    f[33] = log10(1.0 / kabs(kb));
    double k5 = curv3(anc + 0, anc + 6, anc + 12);
    f[34] = log10(kf / kabs(k5));
    double kbar = 0.5 * (ka + kb), S4 = 0.0;
    for (int i = 0; i < 4; i++) {
        double dx = anc[3 * (i + 1)] - anc[3 * i], dy = anc[3 * (i + 1) + 1] - anc[3 * i + 1];
        double d = sqrt(dx * dx + dy * dy);
        S4 += d * (1.0 + d * d * kbar * kbar / 24.0);
    }
    f[35] = asinh((anc[14] - anc[2]) / S4) / 2.5;
    f[36] = atan2(anc[13] - anc[1], anc[12] - anc[0]) / M_PI;
    double kbr = curv3(anc + 3, anc + 6, anc + 9);
    f[37] = log10(1.0 / kabs(kbr));
}

/* Section 2: the T5-DNN forward pass, FP64, nested loops over the weight arrays. */
double oracle_mlp(const omlp *m, const double *f)
{
    double h[NHID], t[NHID];
    const double *w = m->w;
    for (int o = 0; o < NHID; o++) {
        double s = w[NHID * NFEAT + o];
        for (int i = 0; i < NFEAT; i++) s += w[o * NFEAT + i] * f[i];
        h[o] = s > 0.0 ? s : 0.0;
    }
    w += NHID * NFEAT + NHID;
    for (int l = 1; l < m->n_hidden; l++) {
        for (int o = 0; o < NHID; o++) {
            double s = w[NHID * NHID + o];
            for (int i = 0; i < NHID; i++) s += w[o * NHID + i] * h[i];
            t[o] = s > 0.0 ? s : 0.0;
        }
        memcpy(h, t, sizeof h);
        w += NHID * NHID + NHID;
    }
    double s = w[NHID];
    for (int i = 0; i < NHID; i++) s += w[i] * h[i];
    return 1.0 / (1.0 + exp(-s));
}

/* ------------------------------------------------------------------ track candidates */
/* Table 1 step 6 without pixel seeds (none exist here): the selected T5s, cleaned of
 * duplicates (Section 2 places duplicate removal downstream of the T5 step). Project
 * definition:
 *   two T5s are duplicates when they share at least 3 of their 5 MDs;
 *   T5 u ranks above T5 t when q_u < q_t, or q_u == q_t and key_u < key_t (lexicographic),
 *   where q is the circle-fit chi2 (NaN and +inf both count as +inf) and key is the 10
 *   original hit indices (lower and upper hit of each MD, in chain order);
 *   a selected T5 is a track candidate iff no selected duplicate ranks above it. This is
 *   one pass: a T5 that a better duplicate removes still removes the T5s it ranks above.
 * md [n][5] MD ids below n_md, key [n][10], q [n], sel [n] -> tc [n] (0/1). brute: test
 * every pair of selected T5s instead of the T5s listed under one of the T5's MDs. */
#define TC_MIN_SHARED 3

static int shared_mds(const int32_t *a, const int32_t *b)
{
    int s = 0;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) s += a[i] == b[j];
    return s;
}

static int ranks_above(int64_t u, int64_t t, const int32_t *key, const float *q)
{
    float qu = q[u] <= FLT_MAX ? q[u] : INFINITY, qt = q[t] <= FLT_MAX ? q[t] : INFINITY;
    if (qu < qt) return 1;
    if (qu > qt) return 0;
    for (int k = 0; k < 10; k++)
        if (key[10 * u + k] != key[10 * t + k]) return key[10 * u + k] < key[10 * t + k];
    return 0;
}

void oracle_tc_select(int64_t n, const int32_t *md, const int32_t *key, const float *q,
                      const uint8_t *sel, int64_t n_md, int brute, uint8_t *tc)
{
    int64_t *off = NULL, *list = NULL;
    if (!brute) {                     /* selected T5s listed under each of their MDs */
        off = calloc((size_t)n_md + 1, sizeof(int64_t));
        for (int64_t t = 0; t < n; t++)
            if (sel[t])
                for (int j = 0; j < 5; j++) off[md[5 * t + j] + 1]++;
        for (int64_t m = 0; m < n_md; m++) off[m + 1] += off[m];
        list = malloc(sizeof(int64_t) * (size_t)(off[n_md] ? off[n_md] : 1));
        int64_t *cur = malloc(sizeof(int64_t) * (size_t)(n_md ? n_md : 1));
        memcpy(cur, off, sizeof(int64_t) * (size_t)n_md);
        for (int64_t t = 0; t < n; t++)
            if (sel[t])
                for (int j = 0; j < 5; j++) list[cur[md[5 * t + j]]++] = t;
        free(cur);
    }
    for (int64_t t = 0; t < n; t++) {
        tc[t] = 0;
        if (!sel[t]) continue;
        int keep = 1;
        if (brute) {
            for (int64_t u = 0; u < n && keep; u++)
                if (u != t && sel[u] && shared_mds(md + 5 * t, md + 5 * u) >= TC_MIN_SHARED &&
                    ranks_above(u, t, key, q))
                    keep = 0;
        } else {
            for (int j = 0; j < 5 && keep; j++) {
                int32_t m = md[5 * t + j];
                for (int64_t k = off[m]; k < off[m + 1] && keep; k++) {
                    int64_t u = list[k];
                    if (u != t && shared_mds(md + 5 * t, md + 5 * u) >= TC_MIN_SHARED && ranks_above(u, t, key, q))
                        keep = 0;
                }
            }
        }
        tc[t] = (uint8_t)keep;
    }
    free(off);
    free(list);
}

static void fill_md_anchor(const hit *H, float *a) { a[0] = H->x; a[1] = H->y; a[2] = H->z; a[3] = H->r; }

/* ------------------------------------------------------------------ pixel seeds */
/* Table 1 steps 0 and 5-8. A pixel seed (pLS) is four inner-tracker hits H1..H4 (inner
 * first), made upstream. It is matched to an outer object (a T5 by its first T3, or a T3)
 * whose first anchors are P0, P1 and whose curvature is ko (the T3's three-point value) when
 * the two are consistent with one helix (Section 1). Project specification, FP32, only + - *
 * / sqrt, so that the GPU reaches the same decisions:
 *   window: the azimuth of P0 seen from the beamline turns from H4's by less than the bend
 *     of a track at the T3 pT limit allows over the radial distance, H4 . P0 > 0 and
 *     |H4 x P0| <= (dphi0 + dphi_cm (|P0|_T - |H4|_T)) |H4|_T |P0|_T (sine of the turn),
 *     and the r-z slopes agree, |m_p - m_o| <= dm_abs + dm_rel |m_o| with m_p = (z4 - z1) /
 *     (r4 - r1) and m_o = (z1' - z0) / (r1' - r0) (P0 -> P1);
 *   pT: |kp - ko| <= rel (|kp| + |ko|) / 2 + abs, kp the seed's curvature through H1, H3, H4;
 *   circle: the same test for kx, the curvature through H1, H4 and P0 (the seed and the
 *     object on one circle);
 *   rz: H4's z against its interpolation between H1 and P0 along the arc (the T3 form, with
 *     the mean curvature (kx + ko) / 2): |z4 - zp| <= rz_tol.
 * Matches rank by that rz residual, then by |kx - ko|, then by the seed's index, then by the
 * object's hit tuple (original hit indices, lexicographic): objects built on the same anchors
 * tie in every measure, and the tuple decides between them whatever their storage order.
 * Every curvature is the signed three-point value 2 (B - A) x (C - A) / (|B-A| |C-B| |C-A|). */
static float pix_curv3(const float *A, const float *B, const float *C)
{
    float d01x = B[0] - A[0], d01y = B[1] - A[1];
    float d12x = C[0] - B[0], d12y = C[1] - B[1];
    float d02x = C[0] - A[0], d02y = C[1] - A[1];
    float a = sqrtf(d01x * d01x + d01y * d01y);
    float b = sqrtf(d12x * d12x + d12y * d12y);
    float c = sqrtf(d02x * d02x + d02y * d02y);
    float cr = d01x * d02y - d01y * d02x;
    return 2.0f * cr / (a * b * c);
}

static int pix_kappa_ok(float k1, float k2, const opcuts *pc)
{
    return fabsf(k1 - k2) <= pc->kappa_rel * 0.5f * (fabsf(k1) + fabsf(k2)) + pc->kappa_abs;
}

/* H: the seed's hits [4][3]; P0, P1: (x, y, z, r) of the object's first two anchors.
 * Returns 1 and the ranking pair (rz residual, |kx - ko|) if the seed and the object match. */
int oracle_pixel_match(const float *H, const float *P0, const float *P1, float ko, const opcuts *pc,
                       float *resid)
{
    const float *H1 = H, *H3 = H + 6, *H4 = H + 9;
    float r1 = sqrtf(H1[0] * H1[0] + H1[1] * H1[1]);
    float r4 = sqrtf(H4[0] * H4[0] + H4[1] * H4[1]);
    if (!(H4[0] * P0[0] + H4[1] * P0[1] > 0.0f)) return 0;                        /* azimuth */
    if (!(fabsf(H4[0] * P0[1] - H4[1] * P0[0]) <= (pc->dphi0 + pc->dphi_cm * (P0[3] - r4)) * (r4 * P0[3])))
        return 0;
    float mp = (H4[2] - H1[2]) / (r4 - r1);
    float mo = (P1[2] - P0[2]) / (P1[3] - P0[3]);
    if (!(fabsf(mp - mo) <= pc->dm_abs + pc->dm_rel * fabsf(mo))) return 0;          /* slope */
    float kp = pix_curv3(H1, H3, H4);
    if (!pix_kappa_ok(kp, ko, pc)) return 0;                                        /* pT */
    float kx = pix_curv3(H1, H4, P0);
    if (!pix_kappa_ok(kx, ko, pc)) return 0;                                        /* circle */
    float kbar = 0.5f * (kx + ko);
    float ax = H4[0] - H1[0], ay = H4[1] - H1[1], bx = P0[0] - H4[0], by = P0[1] - H4[1];
    float a = sqrtf(ax * ax + ay * ay), b = sqrtf(bx * bx + by * by);
    float s14 = a * (1.0f + a * a * kbar * kbar / 24.0f);
    float s40 = b * (1.0f + b * b * kbar * kbar / 24.0f);
    float zp = H1[2] + (P0[2] - H1[2]) * s14 / (s14 + s40);
    float res = fabsf(H4[2] - zp);
    if (!(res <= pc->rz_tol)) return 0;                                             /* rz */
    resid[0] = res;
    resid[1] = fabsf(kx - ko);
    return 1;
}

typedef struct { float res, dk; int32_t p, o, rank; } pedge;

static int pedge_cmp(const void *a, const void *b)
{
    const pedge *x = a, *y = b;
    if (x->res != y->res) return x->res < y->res ? -1 : 1;
    if (x->dk != y->dk) return x->dk < y->dk ? -1 : 1;
    if (x->p != y->p) return x->p < y->p ? -1 : 1;
    return (x->rank > y->rank) - (x->rank < y->rank);
}

typedef struct { int32_t key[10]; int32_t o; } pobj;

static int pobj_cmp(const void *a, const void *b)
{
    const pobj *x = a, *y = b;
    for (int k = 0; k < 10; k++)
        if (x->key[k] != y->key[k]) return x->key[k] < y->key[k] ? -1 : 1;
    return 0;
}

/* rank[o] = position of object o in the lexicographic order of its hit tuple key[o][0..w) */
static void pix_ranks(const int32_t *key, int w, int64_t n, int32_t *rank)
{
    pobj *v = malloc(sizeof(pobj) * (size_t)(n ? n : 1));
    for (int64_t o = 0; o < n; o++) {
        for (int k = 0; k < 10; k++) v[o].key[k] = k < w ? key[(size_t)w * o + k] : 0;
        v[o].o = (int32_t)o;
    }
    qsort(v, (size_t)n, sizeof(pobj), pobj_cmp);
    for (int64_t i = 0; i < n; i++) rank[v[i].o] = (int32_t)i;
    free(v);
}

/* One-to-one matching of seeds and objects, preferring the better rank: the edges in
 * ascending (rz residual, |kx - ko|, seed, object hit tuple) order, each taken when both its
 * ends are still free. Objects with elig[o] == 0 and seeds with pused[p] != 0 take part in no
 * edge. obj_p[o] receives the seed taken by object o (or stays -1); pused marks taken seeds.
 * Counts in *ties the edges taken while an edge equal in (residual, |kx - ko|) and sharing an
 * end was left, i.e. where the seed index or the hit tuple decided. */
static void pix_greedy(const float *pls, int64_t n_pls, int64_t n_obj, const uint8_t *elig,
                       const float *P0s, const float *P1s, const float *kos, const int32_t *rank,
                       const opcuts *pc, int32_t *obj_p, uint8_t *pused, int64_t *ties)
{
    vec E; vinit(&E, sizeof(pedge));
    for (int64_t p = 0; p < n_pls; p++) {
        if (pused[p]) continue;
        for (int64_t o = 0; o < n_obj; o++) {
            if (!elig[o]) continue;
            float r[2];
            if (oracle_pixel_match(pls + 12 * p, P0s + 4 * o, P1s + 4 * o, kos[o], pc, r)) {
                pedge *e = vpush(&E);
                e->res = r[0]; e->dk = r[1]; e->p = (int32_t)p; e->o = (int32_t)o; e->rank = rank[o];
            }
        }
    }
    pedge *ed = E.p;
    qsort(ed, (size_t)E.n, sizeof(pedge), pedge_cmp);
    uint8_t *otaken = calloc((size_t)(n_obj ? n_obj : 1), 1);
    for (int64_t i = 0; i < E.n; i++) {
        if (pused[ed[i].p] || otaken[ed[i].o]) continue;
        pused[ed[i].p] = 1;
        otaken[ed[i].o] = 1;
        obj_p[ed[i].o] = ed[i].p;
        for (int64_t j = i + 1; j < E.n && ed[j].res == ed[i].res && ed[j].dk == ed[i].dk; j++)
            if (ed[j].p == ed[i].p || ed[j].o == ed[i].o) (*ties)++;
    }
    free(otaken);
    free(E.p);
}

/* Table 1 steps 5-8 from the event's track-candidate T5s (t5_tc), all T3s and the seeds:
 *   5 pT5: seeds matched one-to-one to track-candidate T5s (by the T5's first T3);
 *   6 T5: track-candidate T5s left without a seed;
 *   7 pT3: the remaining seeds matched one-to-one to T3s not in a pT5 (a T3 is in a pT5
 *     when each of its three MDs belongs to a pT5's T5);
 *   8 pLS: seeds used by neither. */
static void pix_tcs(const float *pls, int64_t n_pls, const opcuts *pc, const hit *H, const md_t *MD,
                    int64_t n_md, const t3_t *T3, int64_t n_t3, const t5_t *T5, int64_t n_t5,
                    const uint8_t *t5_tc, oresult *out)
{
    uint8_t *pused = calloc((size_t)(n_pls ? n_pls : 1), 1);
    int64_t nt5 = n_t5 ? n_t5 : 1, nt3 = n_t3 ? n_t3 : 1;
    float *P0 = malloc(16 * (size_t)(nt5 > nt3 ? nt5 : nt3)), *P1 = malloc(16 * (size_t)(nt5 > nt3 ? nt5 : nt3));
    float *ko = malloc(4 * (size_t)(nt5 > nt3 ? nt5 : nt3));
    int32_t *t5p = malloc(4 * (size_t)nt5), *t3p = malloc(4 * (size_t)nt3);
    uint8_t *elig = malloc((size_t)(nt5 > nt3 ? nt5 : nt3));
    int32_t *key = malloc(40 * (size_t)(nt5 > nt3 ? nt5 : nt3)), *rank = malloc(4 * (size_t)(nt5 > nt3 ? nt5 : nt3));
    for (int64_t t = 0; t < n_t5; t++)
        for (int j = 0; j < 5; j++) {
            key[10 * t + 2 * j] = MD[T5[t].md[j]].lo;
            key[10 * t + 2 * j + 1] = MD[T5[t].md[j]].up;
        }
    pix_ranks(key, 10, n_t5, rank);
    for (int64_t t = 0; t < n_t5; t++) {
        fill_md_anchor(&H[MD[T5[t].md[0]].lo], P0 + 4 * t);
        fill_md_anchor(&H[MD[T5[t].md[1]].lo], P1 + 4 * t);
        ko[t] = T3[T5[t].t3a].kappa;
        elig[t] = t5_tc[t];
        t5p[t] = -1;
    }
    pix_greedy(pls, n_pls, n_t5, elig, P0, P1, ko, rank, pc, t5p, pused, &out->pix_ties);
    uint8_t *mdin = calloc((size_t)(n_md ? n_md : 1), 1);
    for (int64_t t = 0; t < n_t5; t++)
        if (t5p[t] >= 0)
            for (int j = 0; j < 5; j++) mdin[T5[t].md[j]] = 1;
    for (int64_t u = 0; u < n_t3; u++)
        for (int j = 0; j < 3; j++) {
            key[6 * u + 2 * j] = MD[T3[u].md[j]].lo;
            key[6 * u + 2 * j + 1] = MD[T3[u].md[j]].up;
        }
    pix_ranks(key, 6, n_t3, rank);
    for (int64_t u = 0; u < n_t3; u++) {
        fill_md_anchor(&H[MD[T3[u].md[0]].lo], P0 + 4 * u);
        fill_md_anchor(&H[MD[T3[u].md[1]].lo], P1 + 4 * u);
        ko[u] = T3[u].kappa;
        elig[u] = !(mdin[T3[u].md[0]] && mdin[T3[u].md[1]] && mdin[T3[u].md[2]]);
        t3p[u] = -1;
    }
    pix_greedy(pls, n_pls, n_t3, elig, P0, P1, ko, rank, pc, t3p, pused, &out->pix_ties);
    vec R; vinit(&R, 12);
    for (int64_t t = 0; t < n_t5; t++) {
        if (!t5_tc[t]) continue;
        int32_t *row = vpush(&R);
        row[0] = t5p[t] >= 0 ? 5 : 6; row[1] = t5p[t]; row[2] = (int32_t)t;
    }
    for (int64_t u = 0; u < n_t3; u++)
        if (t3p[u] >= 0) { int32_t *row = vpush(&R); row[0] = 7; row[1] = t3p[u]; row[2] = (int32_t)u; }
    for (int64_t p = 0; p < n_pls; p++)
        if (!pused[p]) { int32_t *row = vpush(&R); row[0] = 8; row[1] = (int32_t)p; row[2] = -1; }
    out->n_pix = R.n;
    out->pix_tc = R.p ? R.p : malloc(12);
    free(pused); free(P0); free(P1); free(ko); free(t5p); free(t3p); free(elig); free(mdin);
    free(key); free(rank);
}

/* ------------------------------------------------------------------ event driver */
static int layer_adjacent(int la, int sa, int lb, int sb)
{
    if (la <= 5 && lb == la + 1) return 1;          /* barrel l -> l+1 */
    if (la <= 6 && lb == 7) return 1;               /* barrel -> first disk */
    if (la >= 7 && la <= 10 && lb == la + 1 && sa == sb) return 1;  /* disk d -> d+1 */
    return 0;
}


int oracle_run(const ogeom *g, const float *x, const float *y, const float *z,
               const int32_t *sensor, int64_t n_hits, const ocuts *c, const omlp *mlp,
               int brute, const float *pls, int64_t n_pls, const opcuts *pc, oresult *out)
{
    memset(out, 0, sizeof *out);
    int32_t nm = g->n_mod;
    for (int64_t i = 0; i < n_hits; i++)
        if (sensor[i] < 0 || sensor[i] >= 2 * nm || !isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i]))
            return 1;
    hit *H = malloc(sizeof(hit) * (size_t)(n_hits ? n_hits : 1));
    for (int64_t i = 0; i < n_hits; i++) H[i] = mkhit(x, y, z, (int32_t)i);

    /* hits of each sensor, ascending original index (stable counting sort) */
    int64_t ns = 2 * (int64_t)nm;
    int64_t *soff = calloc((size_t)ns + 1, sizeof(int64_t));
    int32_t *sidx = malloc(sizeof(int32_t) * (size_t)(n_hits ? n_hits : 1));
    for (int64_t i = 0; i < n_hits; i++) soff[sensor[i] + 1]++;
    for (int64_t s = 0; s < ns; s++) soff[s + 1] += soff[s];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)ns);
    memcpy(fill, soff, sizeof(int64_t) * (size_t)ns);
    for (int64_t i = 0; i < n_hits; i++) sidx[fill[sensor[i]]++] = (int32_t)i;
    free(fill);

    /* ---- step 1: mini-doublets, module by module ---- */
    vec mds; vinit(&mds, sizeof(md_t));
    int64_t *mdoff = calloc((size_t)nm + 1, sizeof(int64_t));
    for (int32_t m = 0; m < nm; m++) {
        int endcap = g->subdet[m] != 0;
        if (!brute) {
            for (int64_t a = soff[2 * m]; a < soff[2 * m + 1]; a++)
                for (int64_t b = soff[2 * m + 1]; b < soff[2 * m + 2]; b++) {
                    out->pairs[0]++;
                    float L[4], U[4], k;
                    fill_md_anchor(&H[sidx[a]], L);
                    fill_md_anchor(&H[sidx[b]], U);
                    g_near = 0;
                    int ok = oracle_md_cut(L, U, endcap, c, &k);
                    out->near[0] += g_near;
                    if (ok) {
                        md_t *d = vpush(&mds);
                        d->lo = sidx[a]; d->up = sidx[b]; d->mod = m; d->kappa = k;
                    }
                }
        } else {
            for (int64_t i = 0; i < n_hits; i++) {
                if (sensor[i] != 2 * m) continue;
                for (int64_t j = 0; j < n_hits; j++) {
                    if (sensor[j] != 2 * m + 1) continue;
                    out->pairs[0]++;
                    float L[4], U[4], k;
                    fill_md_anchor(&H[i], L);
                    fill_md_anchor(&H[j], U);
                    g_near = 0;
                    int ok = oracle_md_cut(L, U, endcap, c, &k);
                    out->near[0] += g_near;
                    if (ok) {
                        md_t *d = vpush(&mds);
                        d->lo = (int32_t)i; d->up = (int32_t)j; d->mod = m; d->kappa = k;
                    }
                }
            }
        }
        mdoff[m + 1] = mds.n;
    }
    md_t *MD = mds.p;
    for (int64_t i = 0; i < mds.n; i++) {
        if (g->subdet[MD[i].mod] != 0) { MD[i].kfeat = 0.0; continue; }
        double L[2] = {x[MD[i].lo], y[MD[i].lo]}, U[2] = {x[MD[i].up], y[MD[i].up]};
        MD[i].kfeat = md_kappa_fp64(L, U);
    }

    /* ---- step 2: line segments, MD pairs across linked modules ---- */
    vec lss; vinit(&lss, sizeof(ls_t));
    for (int32_t m = 0; m < nm; m++) {
        for (int64_t i = mdoff[m]; i < mdoff[m + 1]; i++) {
            float A[4]; fill_md_anchor(&H[MD[i].lo], A);
            int bA = g->subdet[m] == 0;
            if (!brute) {
                for (int32_t t = g->map_off[m]; t < g->map_off[m + 1]; t++) {
                    int32_t mt = g->map_tgt[t];
                    for (int64_t j = mdoff[mt]; j < mdoff[mt + 1]; j++) {
                        out->pairs[1]++;
                        float B[4], k; fill_md_anchor(&H[MD[j].lo], B);
                        g_near = 0;
                        int ok = oracle_ls_cut(A, B, MD[i].kappa, MD[j].kappa, bA, g->subdet[mt] == 0, c, &k);
                        out->near[1] += g_near;
                        if (ok) {
                            ls_t *s = vpush(&lss); s->in = (int32_t)i; s->out = (int32_t)j; s->kappa = k;
                        }
                    }
                }
            } else {
                for (int64_t j = 0; j < mds.n; j++) {
                    int32_t mt = MD[j].mod;
                    if (!layer_adjacent(g->layer[m], g->side[m], g->layer[mt], g->side[mt])) continue;
                    out->pairs[1]++;
                    float B[4], k; fill_md_anchor(&H[MD[j].lo], B);
                    g_near = 0;
                    int ok = oracle_ls_cut(A, B, MD[i].kappa, MD[j].kappa, bA, g->subdet[mt] == 0, c, &k);
                    out->near[1] += g_near;
                    if (ok) {
                        ls_t *s = vpush(&lss); s->in = (int32_t)i; s->out = (int32_t)j; s->kappa = k;
                    }
                }
            }
        }
    }
    ls_t *LS = lss.p;
    /* LS list of every MD as inner MD (LSs are already ordered by inner MD) */
    int64_t *lsoff = calloc((size_t)mds.n + 1, sizeof(int64_t));
    for (int64_t s = 0; s < lss.n; s++) lsoff[LS[s].in + 1]++;
    for (int64_t i = 0; i < mds.n; i++) lsoff[i + 1] += lsoff[i];

    /* ---- step 3: triplets, LS pairs sharing the middle MD ---- */
    vec t3s; vinit(&t3s, sizeof(t3_t));
    for (int64_t s1 = 0; s1 < lss.n; s1++) {
        int64_t lo = brute ? 0 : lsoff[LS[s1].out], hi = brute ? lss.n : lsoff[LS[s1].out + 1];
        for (int64_t s2 = lo; s2 < hi; s2++) {
            if (LS[s2].in != LS[s1].out) continue;
            out->pairs[2]++;
            float P0[4], P1[4], P2[4], k;
            fill_md_anchor(&H[MD[LS[s1].in].lo], P0);
            fill_md_anchor(&H[MD[LS[s1].out].lo], P1);
            fill_md_anchor(&H[MD[LS[s2].out].lo], P2);
            g_near = 0;
            int ok = oracle_t3_cut(P0, P1, P2, c, &k);
            out->near[2] += g_near;
            if (ok) {
                t3_t *t = vpush(&t3s);
                t->ls1 = (int32_t)s1; t->ls2 = (int32_t)s2;
                t->md[0] = LS[s1].in; t->md[1] = LS[s1].out; t->md[2] = LS[s2].out;
                t->kappa = k;
            }
        }
    }
    t3_t *T3 = t3s.p;
    /* T3 list of every MD as first MD (T3s are ordered by their first LS, hence first MD) */
    int64_t *t3off = calloc((size_t)mds.n + 1, sizeof(int64_t));
    for (int64_t t = 0; t < t3s.n; t++) t3off[T3[t].md[0] + 1]++;
    for (int64_t i = 0; i < mds.n; i++) t3off[i + 1] += t3off[i];

    /* ---- step 4: quintuplets, T3 pairs sharing the joint MD, then the score ---- */
    vec t5s; vinit(&t5s, sizeof(t5_t));
    for (int64_t a = 0; a < t3s.n; a++) {
        int64_t lo = brute ? 0 : t3off[T3[a].md[2]], hi = brute ? t3s.n : t3off[T3[a].md[2] + 1];
        for (int64_t b = lo; b < hi; b++) {
            if (T3[b].md[0] != T3[a].md[2]) continue;
            out->pairs[3]++;
            int32_t md5[5] = {T3[a].md[0], T3[a].md[1], T3[a].md[2], T3[b].md[1], T3[b].md[2]};
            float P[20];
            for (int i = 0; i < 5; i++) fill_md_anchor(&H[MD[md5[i]].lo], P + 4 * i);
            g_near = 0;
            int ok = oracle_t5_cut(P, T3[a].kappa, T3[b].kappa, c);
            out->near[3] += g_near;
            if (ok) {
                t5_t *q = vpush(&t5s);
                q->t3a = (int32_t)a; q->t3b = (int32_t)b;
                memcpy(q->md, md5, sizeof md5);
            }
        }
    }
    t5_t *T5 = t5s.p;

    /* ---- outputs ---- */
    out->n_md = mds.n; out->n_ls = lss.n; out->n_t3 = t3s.n; out->n_t5 = t5s.n;
    size_t nmd = (size_t)(mds.n ? mds.n : 1), nls = (size_t)(lss.n ? lss.n : 1);
    size_t nt3 = (size_t)(t3s.n ? t3s.n : 1), nt5 = (size_t)(t5s.n ? t5s.n : 1);
    out->md_lo = malloc(4 * nmd); out->md_up = malloc(4 * nmd); out->md_mod = malloc(4 * nmd);
    out->md_kappa = malloc(4 * nmd);
    for (int64_t i = 0; i < mds.n; i++) {
        out->md_lo[i] = MD[i].lo; out->md_up[i] = MD[i].up; out->md_mod[i] = MD[i].mod;
        out->md_kappa[i] = MD[i].kappa;
    }
    out->ls_in = malloc(4 * nls); out->ls_out = malloc(4 * nls); out->ls_kappa = malloc(4 * nls);
    for (int64_t i = 0; i < lss.n; i++) {
        out->ls_in[i] = LS[i].in; out->ls_out[i] = LS[i].out; out->ls_kappa[i] = LS[i].kappa;
    }
    out->t3_ls1 = malloc(4 * nt3); out->t3_ls2 = malloc(4 * nt3); out->t3_md = malloc(12 * nt3);
    out->t3_kappa = malloc(4 * nt3);
    for (int64_t i = 0; i < t3s.n; i++) {
        out->t3_ls1[i] = T3[i].ls1; out->t3_ls2[i] = T3[i].ls2;
        memcpy(out->t3_md + 3 * i, T3[i].md, 12); out->t3_kappa[i] = T3[i].kappa;
    }
    out->t5_t3a = malloc(4 * nt5); out->t5_t3b = malloc(4 * nt5); out->t5_md = malloc(20 * nt5);
    out->t5_feat = malloc(sizeof(double) * NFEAT * nt5); out->t5_score = malloc(sizeof(double) * nt5);
    out->t5_sel = malloc(nt5);
    out->t5_chi2 = malloc(4 * nt5);
    for (int64_t i = 0; i < t5s.n; i++) {
        out->t5_t3a[i] = T5[i].t3a; out->t5_t3b[i] = T5[i].t3b;
        memcpy(out->t5_md + 5 * i, T5[i].md, 20);
        double anc[15], mdk[5];
        int32_t lay[5];
        for (int j = 0; j < 5; j++) {
            const md_t *d = &MD[T5[i].md[j]];
            anc[3 * j] = x[d->lo]; anc[3 * j + 1] = y[d->lo]; anc[3 * j + 2] = z[d->lo];
            lay[j] = g->layer[d->mod];
            mdk[j] = d->kfeat;
        }
        float P[20];
        for (int j = 0; j < 5; j++) fill_md_anchor(&H[MD[T5[i].md[j]].lo], P + 4 * j);
        out->t5_chi2[i] = oracle_t5_chi2(P, c->hit_sigma);
        double *f = out->t5_feat + (size_t)NFEAT * i;
        oracle_t5_features(anc, lay, mdk, (double)c->k_field, f);
        double s = mlp ? oracle_mlp(mlp, f) : 0.0;
        out->t5_score[i] = s;
        /* pre-DNN mode: the chi2 cut already selected the T5; DNN mode: the working point */
        out->t5_sel[i] = c->t5_chi2_max > 0.0f ? 1 : s >= (double)c->wp;
    }

    /* ---- track candidates from the selected T5s ---- */
    out->t5_tc = malloc(nt5);
    {
        int32_t *key = malloc(40 * nt5);
        for (int64_t i = 0; i < t5s.n; i++)
            for (int j = 0; j < 5; j++) {
                key[10 * i + 2 * j] = MD[T5[i].md[j]].lo;
                key[10 * i + 2 * j + 1] = MD[T5[i].md[j]].up;
            }
        oracle_tc_select(t5s.n, out->t5_md, key, out->t5_chi2, out->t5_sel, mds.n, brute, out->t5_tc);
        free(key);
    }

    /* ---- pixel seeds: track candidates of steps 5-8 ---- */
    if (pls && pc) pix_tcs(pls, n_pls, pc, H, MD, mds.n, T3, t3s.n, T5, t5s.n, out->t5_tc, out);
    free(H); free(soff); free(sidx); free(mdoff); free(lsoff); free(t3off);
    free(mds.p); free(lss.p); free(t3s.p); free(t5s.p);
    return 0;
}

void oracle_free(oresult *r)
{
    void *ps[] = {r->md_lo, r->md_up, r->md_mod, r->md_kappa, r->ls_in, r->ls_out, r->ls_kappa,
                  r->t3_ls1, r->t3_ls2, r->t3_md, r->t3_kappa, r->t5_t3a, r->t5_t3b, r->t5_md,
                  r->t5_feat, r->t5_score, r->t5_sel, r->t5_chi2, r->t5_tc, r->pix_tc};
    for (size_t i = 0; i < sizeof ps / sizeof ps[0]; i++) free(ps[i]);
    memset(r, 0, sizeof *r);
}
