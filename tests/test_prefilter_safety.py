"""The necessary tests that the CUDA kernels run before the exact FP32 cuts (md_prefilter,
ls_prefilter + ls_kappa_prefilter, t3_prefilter in csrc/lst_internal.cuh) must never
reject an object the exact cut accepts; their rounding slacks are argued in the header
comments. Here each test is restated in float32 numpy (a fused multiply-add as an exact
float64 product plus a sum rounded once to float32; the approximate reciprocal and
reciprocal square root perturbed by +-2e-7 relative, above their documented error) and
evaluated on every MD, LS and T3 the oracle accepts in one PU200-like event: none may fail.
A sample of candidate pairs also checks that the LS tests are selective. CPU only."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import synth

f32, f64 = np.float32, np.float64
APPROX = (1.0 - 2e-7, 1.0 + 2e-7)


def fma(a, b, c):
    return (np.asarray(a, f64) * np.asarray(b, f64) + np.asarray(c, f64)).astype(f32)


def full(shape, v):
    return np.full(shape, f32(v), f32)


@pytest.fixture(scope="module")
def event(geom_full, cuts):
    e = synth.pileup_event(geom_full, 11, pileup=200, mean_per_vertex=96)
    r = oracle.run_event(geom_full, e, cuts, None)
    x, y, z = (a.astype(f32) for a in (e.x, e.y, e.z))
    r_ = np.sqrt(x * x + y * y).astype(f32)
    return e, r, (x, y, z, r_)


def md_prefilter(L, U, endcap, c):
    """md_prefilter / md_low of csrc/lst_internal.cuh, float32."""
    Lx, Ly, Lz, Lr = L
    Ux, Uy, Uz, Ur = U
    km, e, gap, zl = (f32(c[k]) for k in ("kappa_max", "hit_err", "sensor_gap", "z_lum"))
    with np.errstate(all="ignore"):
        dx, dy, dz = Ux - Lx, Uy - Ly, Uz - Lz
        dt = Lx * dx + Ly * dy
        cr = fma(Lx, dy, -(Ly * dx))
        # endcap
        az, r2 = np.abs(Lz), Lr * Lr
        wz = np.where(az > zl, r2 * zl / (az - zl), f32(np.inf)).astype(f32)
        erz, erl = e * Lr * az, e * Lr
        S = Lr * (f32(0.5) * km)
        T = (S / np.sqrt(f32(1.0) - S * S)).astype(f32)
        t1, t2 = dt * az, np.abs(dz) * r2
        rr = fma(np.abs(dz), wz, erz)
        road = np.abs(t1 - t2) <= rr + f32(1e-3) * (np.abs(t1) + t2 + rr) + f32(1e-6)
        bb = fma(dt, T, erl)
        bend_e = np.abs(cr) <= bb + f32(1e-3) * (np.abs(dt * T) + erl) + f32(1e-6)
        ec = road & bend_e
        # barrel
        hb = Lr * (f32(0.5) * km) + e / gap
        hb2r2 = (Lr * hb) * (Lr * hb) * f32(1.001)
        dT2 = fma(dx, dx, dy * dy)
        bend = cr * cr <= fma(hb2r2, dT2, full(dT2.shape, 1e-9))
        dr = Ur - Lr
        a, b = dz * Lr, Lz * dr
        rhs = fma(full(dr.shape, zl), dr, erl)
        zr = np.abs(a - b) <= rhs + f32(1e-3) * (np.abs(a) + np.abs(b) + np.abs(rhs)) + f32(1e-6)
        br = bend & zr
    return np.where(endcap, ec, br)


def ls_prefilters(A, B, kA, kB, bA, bB, c, rel):
    """ls_prefilter and ls_kappa_prefilter, float32 (rel: the rsqrt approximation)."""
    Ax, Ay, Az, Ar = A
    Bx, By, Bz, Br = B
    km, e, gap, zl = (f32(c[k]) for k in ("kappa_max", "hit_err", "sensor_gap", "z_lum"))
    with np.errstate(all="ignore"):
        # first test
        X = Br * (f32(0.5) * km)
        k1 = f32(1.002) * f32(1.015625) * X * X
        k0 = f32(1.002) * f32(65.0) * (e * e)
        p = fma(Az, Br, -(Ar * Bz))
        z0 = np.abs(p) <= fma(full(p.shape, zl + e), np.abs(Br - Ar), e * Ar + f32(0.05))
        cr = fma(Ax, By, -(Ay * Bx))
        dx, dy = Bx - Ax, By - Ay
        dT2 = fma(dx, dx, dy * dy)
        bend = cr * cr <= fma(Ar * Ar, fma(k1, dT2, full(dT2.shape, k0)), full(dT2.shape, 0.05))
        first = z0 & bend
        # curvature test
        Gp = f32(f32(2.0) * (e / gap) * f32(1.000001))
        ce = f32(f32(2.0) * e * f32(1.000001))
        dT = (dT2 * (f32(1.0) / np.sqrt(dT2)) * f32(rel)).astype(f32)
        cr2 = f32(2.0) * cr
        u, v = Br * dT, Ar * dT
        c0 = fma(full(Ar.shape, ce), Ar, full(Ar.shape, 0.01))
        s0 = fma(Ar, Br, v)
        pa, pb = kA * Ar * u, kB * Br * v
        fa = fma(full(pa.shape, -1e-6), np.abs(pa) + s0, np.abs(pa - cr2)) > fma(full(u.shape, Gp), u, c0)
        fb = fma(full(pb.shape, -1e-6), np.abs(pb) + s0, np.abs(pb - cr2)) > fma(full(v.shape, Gp), v, c0)
        second = ~((bA & fa) | (bB & fb))
    return first, second


def t3_prefilter(P0, P1, P2, c, rel):
    """t3_prefilter (rz test) from the two LS chords (a = P1 - P0, b = P2 - P1 with their
    transverse lengths sqrtf(dx*dx + dy*dy), correctly rounded), float32."""
    tolp = f32(f32(c["t3_rz_tol"]) * f32(1.001) + f32(3e-4))
    with np.errstate(all="ignore"):
        ax, ay, az = P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]
        bx, by, bz = P2[0] - P1[0], P2[1] - P1[1], P2[2] - P1[2]
        a = np.sqrt(ax * ax + ay * ay).astype(f32)
        b = np.sqrt(bx * bx + by * by).astype(f32)
        a2 = fma(ax, ax, ay * ay)
        a3 = a * a2
        cx, cy = ax + bx, ay + by
        b2, c2 = fma(bx, bx, by * by), fma(cx, cx, cy * cy)
        cr = fma(ax, by, -(ay * bx))
        abc2 = a2 * b2 * c2
        k24 = ((cr * cr) * ((f32(1.0) / np.maximum(abc2, f32(1e-30))) * f32(rel)).astype(f32)) * f32(4.0 / 24.0)
        s01, s12 = fma(a3, k24, a), fma(b * b2, k24, b)
        lhs = fma(az, s12, -(bz * s01))
    return np.abs(lhs) <= tolp * (s01 + s12)


def test_md_prefilter_keeps_every_mini_doublet(event, geom_full, cuts):
    e, r, H = event
    lo, up = r.md_lo, r.md_up
    endcap = geom_full.subdet[r.md_mod] != 0
    ok = md_prefilter(tuple(h[lo] for h in H), tuple(h[up] for h in H), endcap, cuts)
    assert len(lo) > 100_000 and ok.all(), int((~ok).sum())


def test_ls_prefilters_keep_every_line_segment(event, geom_full, cuts):
    e, r, H = event
    anchors = tuple(h[r.md_lo] for h in H)
    A = tuple(a[r.ls_in] for a in anchors)
    B = tuple(a[r.ls_out] for a in anchors)
    kA, kB = r.md_kappa[r.ls_in].astype(f32), r.md_kappa[r.ls_out].astype(f32)
    bA, bB = geom_full.subdet[r.md_mod[r.ls_in]] == 0, geom_full.subdet[r.md_mod[r.ls_out]] == 0
    assert len(r.ls_in) > 1_000_000
    for rel in APPROX:
        first, second = ls_prefilters(A, B, kA, kB, bA, bB, cuts, rel)
        assert first.all(), int((~first).sum())
        assert second.all(), int((~second).sum())


def test_ls_prefilters_are_selective(event, geom_full, cuts):
    """Over all candidate pairs of 300 modules: the first test keeps about a tenth, the
    curvature test brings it close to the accepted fraction."""
    e, r, H = event
    g = geom_full
    anchors = tuple(h[r.md_lo] for h in H)
    kap = r.md_kappa.astype(f32)
    order = np.argsort(r.md_mod, kind="stable")
    cnt = np.bincount(r.md_mod, minlength=g.n_mod)
    start = np.concatenate([[0], np.cumsum(cnt)])
    acc = set(zip(r.ls_in.tolist(), r.ls_out.tolist()))
    n = n1 = n2 = n_acc = 0
    for m in np.flatnonzero(cnt)[::max(1, len(np.flatnonzero(cnt)) // 300)]:
        ia = order[start[m]:start[m + 1]]
        tg = g.map_tgt[g.map_off[m]:g.map_off[m + 1]]
        ib = np.concatenate([order[start[t]:start[t + 1]] for t in tg]) if len(tg) else np.zeros(0, int)
        if len(ib) == 0:
            continue
        ii, jj = np.repeat(ia, len(ib)), np.tile(ib, len(ia))
        first, second = ls_prefilters(tuple(a[ii] for a in anchors), tuple(a[jj] for a in anchors), kap[ii],
                                      kap[jj], np.full(len(ii), g.subdet[m] == 0),
                                      g.subdet[r.md_mod[jj]] == 0, cuts, 1.0)
        n += len(ii)
        n1 += int(first.sum())
        n2 += int((first & second).sum())
        n_acc += sum((a, b) in acc for a, b in zip(ii.tolist(), jj.tolist()))
    assert n > 1_000_000
    assert n_acc <= n2 <= 1.05 * n_acc + 10
    assert n2 < 0.3 * n1 < 0.05 * n


def test_t3_prefilter_keeps_every_triplet(event, cuts):
    e, r, H = event
    anchors = tuple(h[r.md_lo] for h in H)
    P = [tuple(a[r.t3_md[:, k]] for a in anchors) for k in range(3)]
    assert len(r.t3_md) > 100_000
    for rel in APPROX:
        ok = t3_prefilter(P[0], P[1], P[2], cuts, rel)
        assert ok.all(), int((~ok).sum())


def q_window(zB, rB, rmin, rmax, c, rel=1.0):
    """The window of k_ls on an inner key for target anchor (zB, rB) and a chunk of inner MDs
    with radii in [rmin, rmax], float32 (no contraction); the approximate reciprocals
    (__fdividef, within 2 ulp) are scaled by `rel`."""
    e = f32(c["hit_err"])
    c1 = f32(f32(c["z_lum"]) + e)
    rel = f32(rel)
    ib = (f32(1.0) / rB) * rel
    irmin, irmax = (f32(1.0) / rmin) * rel, (f32(1.0) / rmax) * rel
    qB = zB * ib
    wB = c1 * np.maximum(np.abs(irmin - ib), np.abs(irmax - ib)) + e * ib
    sl = f32(1e-3) * wB + f32(0.05) * irmin * ib + f32(1e-5) * (f32(1.0) + np.abs(qB))
    return (qB - wB) - sl, (qB + wB) + sl


def test_ls_q_window_keeps_every_line_segment(event, geom_full, cuts):
    """Every LS the oracle accepts has its inner MD's key q = z / r inside the window k_ls
    computes for its target. The window only widens when the chunk's radius range [rmin,
    rmax] grows, so the check takes the narrowest case, a chunk holding the inner MD alone
    (rmin = rmax = its own radius): then it holds for every chunk the MD can sit in, and
    skipping the inner MDs outside the union of a group's windows drops no LS."""
    e, r, H = event
    x, y, z, rr = H
    q = z[r.md_lo] * (f32(1.0) / rr[r.md_lo])
    i, j = r.ls_in, r.ls_out
    ra = rr[r.md_lo[i]]
    assert len(i) > 1_000_000
    for rel in (1.0 - 3e-7, 1.0, 1.0 + 3e-7):
        lo, hi = q_window(z[r.md_lo[j]], rr[r.md_lo[j]], ra, ra, cuts, rel)
        qi = q[i] * f32(rel)
        inside = (qi >= lo) & (qi <= hi)
        assert inside.all(), (rel, int((~inside).sum()))


def test_ls_q_window_prunes(event, geom_full, cuts):
    """Over 300 modules, with groups of 32 consecutive targets and chunks of 64 inner MDs (in
    the order the MDs were found): the inner MDs inside the union of a group's windows make
    well under the full count of lane steps."""
    e, r, H = event
    g = geom_full
    x, y, z, rr = H
    q = z[r.md_lo] * (f32(1.0) / rr[r.md_lo])
    order = np.argsort(r.md_mod, kind="stable")
    cnt = np.bincount(r.md_mod, minlength=g.n_mod)
    start = np.concatenate([[0], np.cumsum(cnt)])
    full_steps = run_steps = 0
    mods = np.flatnonzero(cnt)
    for m in mods[::max(1, len(mods) // 300)]:
        ia = order[start[m]:start[m + 1]]
        tg = g.map_tgt[g.map_off[m]:g.map_off[m + 1]]
        T = np.concatenate([order[start[t]:start[t + 1]] for t in tg]) if len(tg) else np.zeros(0, int)
        if len(T) == 0:
            continue
        for c0 in range(0, len(ia), 64):
            ch = ia[c0:c0 + 64]
            qa, ra = q[ch], rr[r.md_lo[ch]]
            lo, hi = q_window(z[r.md_lo[T]], rr[r.md_lo[T]], ra.min(), ra.max(), cuts)
            n4 = (len(ch) + 3) // 4 * 4
            for j0 in range(0, len(T), 32):
                k = int(((qa >= lo[j0:j0 + 32].min()) & (qa <= hi[j0:j0 + 32].max())).sum())
                full_steps += 32 * n4
                run_steps += 32 * (n4 if len(ch) <= 8 else (k + 3) // 4 * 4)
    assert full_steps > 1_000_000 and run_steps < 0.75 * full_steps, run_steps / full_steps

