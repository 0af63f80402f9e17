"""Seeded synthetic inputs for line-segment tracking: detector, module map, events, parameters.

This module produces INPUT DATA only. It holds none of the tracking method's
arithmetic (no mini-doublet, segment, triplet or quintuplet cut, no feature, no
network evaluation); both the CUDA library and the CPU oracle consume what it
makes, and neither is imported here.

What it models (all lengths in cm, momenta in GeV, field 3.8 T along +z):

* The outer tracker is built from pT-modules: two parallel sensors a few mm apart
  (Section 1 of the paper: 2S = two strip sensors, PS = macro-pixel + strip).
  Here every module is a flat 10 x 10 cm square pair with a 0.26 cm gap. The
  "lower" sensor (s = 0) is the one closer to the interaction point; it plays the
  macro-pixel / inner-strip role, so its hit is the anchor hit (Section 2).
* Barrel: 6 layers at r = 23, 36, 51, 68, 88, 110 cm, 24 modules in z covering
  |z| < 120, ceil(2 pi r / 10) modules in phi (full coverage) -> 5760 modules.
* Endcap: 5 disks per side at |z| = 130, 160, 190, 225, 265 cm, 9 rings centred at
  r = 28 + 10 k cm with ceil(2 pi r_c / 10) modules each -> 389 modules per disk.
* Module map (Section 1: segments are built only across adjacent modules that pass
  geometric criteria): a module A is linked to module B of the next layer (barrel
  l -> l+1, barrel -> first disk, disk d -> d+1 on the same side, no layer
  skipping) when some pair of points on the two lower sensors could satisfy the
  segment's luminous-region road and maximal-bend window with generous margins.
  It is a conservative geometric superset; the oracle's brute-force mode checks
  that it drops nothing.
* Events: charged helices from a vertex, closed-form crossings with sensor planes,
  isotropic Gaussian smearing in the sensor plane, optional uniform noise hits.
  Hits are shuffled so that the input order carries no structure.

Sensor id convention: sensor = 2 * module + s, s = 0 lower / 1 upper.
Layer numbering: 1..6 barrel, 7..11 disks 1..5 (either side).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

B_FIELD_T = 3.8
#: pT [GeV] = K_FIELD * R [cm]  (0.299792458 * B / 100)
K_FIELD = 0.299792458 * B_FIELD_T / 100.0

BARREL_R = (23.0, 36.0, 51.0, 68.0, 88.0, 110.0)
BARREL_NZ = 24
BARREL_ZMAX = 120.0
DISK_Z = (130.0, 160.0, 190.0, 225.0, 265.0)
RING_RC = tuple(28.0 + 10.0 * k for k in range(9))
MOD_HALF = 5.0
SENSOR_GAP = 0.26
HIT_SIGMA = 0.003
PS_LAYERS = (1, 2, 3)
PS_RING_RMAX = 60.0

SUBDET_BARREL = 0
SUBDET_ENDCAP = 1


# --------------------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------------------
@dataclass
class Geometry:
    """Module table (one row per pT-module) plus the module map in CSR form."""

    layer: np.ndarray      # int32 [n]  1..6 barrel, 7..11 disks
    subdet: np.ndarray     # int32 [n]  0 barrel, 1 endcap
    side: np.ndarray       # int32 [n]  0 barrel, -1/+1 endcap
    ps: np.ndarray         # int32 [n]  1 = PS module, 0 = 2S
    centre: np.ndarray     # f64 [n,3]  module mid-plane centre
    normal: np.ndarray     # f64 [n,3]  unit normal pointing away from the IP
    uax: np.ndarray        # f64 [n,3]  in-plane axis 1 (tangential)
    vax: np.ndarray        # f64 [n,3]  in-plane axis 2 (z for barrel, radial for disks)
    with_endcap: bool
    map_off: np.ndarray = field(default=None)   # int32 [n+1]
    map_tgt: np.ndarray = field(default=None)   # int32 [n_links]
    # bookkeeping for hit generation
    barrel_first: tuple = ()   # first module id of each barrel layer
    barrel_nphi: tuple = ()
    disk_first: dict = field(default_factory=dict)  # (side, disk, ring) -> (first id, nphi)

    @property
    def n_mod(self) -> int:
        return int(self.layer.shape[0])

    @property
    def n_sensor(self) -> int:
        return 2 * self.n_mod

    def sensor_centre(self, sensor: np.ndarray) -> np.ndarray:
        m = sensor // 2
        s = sensor % 2
        off = np.where(s == 0, -0.5 * SENSOR_GAP, 0.5 * SENSOR_GAP)
        return self.centre[m] + off[:, None] * self.normal[m]


def build_geometry(with_endcap: bool = True) -> Geometry:
    layer, subdet, side, ps = [], [], [], []
    centre, normal, uax, vax = [], [], [], []
    barrel_first, barrel_nphi = [], []
    for li, r in enumerate(BARREL_R):
        nphi = int(math.ceil(2.0 * math.pi * r / (2 * MOD_HALF)))
        barrel_first.append(len(layer))
        barrel_nphi.append(nphi)
        for iz in range(BARREL_NZ):
            zc = -BARREL_ZMAX + (iz + 0.5) * (2 * MOD_HALF)
            for ip in range(nphi):
                ph = 2.0 * math.pi * ip / nphi
                c, s = math.cos(ph), math.sin(ph)
                layer.append(li + 1)
                subdet.append(SUBDET_BARREL)
                side.append(0)
                ps.append(1 if (li + 1) in PS_LAYERS else 0)
                centre.append((r * c, r * s, zc))
                normal.append((c, s, 0.0))
                uax.append((-s, c, 0.0))
                vax.append((0.0, 0.0, 1.0))
    disk_first = {}
    if with_endcap:
        for sd in (-1, 1):
            for di, zd in enumerate(DISK_Z):
                for ri, rc in enumerate(RING_RC):
                    nphi = int(math.ceil(2.0 * math.pi * rc / (2 * MOD_HALF)))
                    disk_first[(sd, di, ri)] = (len(layer), nphi)
                    for ip in range(nphi):
                        ph = 2.0 * math.pi * ip / nphi
                        c, s = math.cos(ph), math.sin(ph)
                        layer.append(7 + di)
                        subdet.append(SUBDET_ENDCAP)
                        side.append(sd)
                        ps.append(1 if rc < PS_RING_RMAX else 0)
                        centre.append((rc * c, rc * s, sd * zd))
                        normal.append((0.0, 0.0, float(sd)))
                        uax.append((-s, c, 0.0))
                        vax.append((c, s, 0.0))
    g = Geometry(
        layer=np.asarray(layer, np.int32), subdet=np.asarray(subdet, np.int32),
        side=np.asarray(side, np.int32), ps=np.asarray(ps, np.int32),
        centre=np.asarray(centre, np.float64), normal=np.asarray(normal, np.float64),
        uax=np.asarray(uax, np.float64), vax=np.asarray(vax, np.float64),
        with_endcap=with_endcap, barrel_first=tuple(barrel_first),
        barrel_nphi=tuple(barrel_nphi), disk_first=disk_first)
    g.map_off, g.map_tgt = build_module_map(g)
    return g


def layers_adjacent(la, sa, lb, sb):
    """Layer relation of the module map: barrel l->l+1, barrel->disk 1, disk d->d+1 (same side)."""
    la = np.asarray(la)
    lb = np.asarray(lb)
    bb = (la <= 5) & (lb == la + 1)
    bd = (la <= 6) & (lb == 7)
    dd = (la >= 7) & (la <= 10) & (lb == la + 1) & (np.asarray(sa) == np.asarray(sb))
    return bb | bd | dd


def _lower_sensor_boxes(g: Geometry):
    """(r, z, phi) extents of every module's lower sensor (plus smearing margin)."""
    n = g.n_mod
    rlo = np.empty(n)
    rhi = np.empty(n)
    zlo = np.empty(n)
    zhi = np.empty(n)
    hw = np.empty(n)
    cr = np.hypot(g.centre[:, 0], g.centre[:, 1])
    phc = np.arctan2(g.centre[:, 1], g.centre[:, 0])
    bar = g.subdet == SUBDET_BARREL
    d = cr[bar] - 0.5 * SENSOR_GAP
    rlo[bar] = d
    rhi[bar] = np.sqrt(d * d + MOD_HALF ** 2)
    zlo[bar] = g.centre[bar, 2] - MOD_HALF
    zhi[bar] = g.centre[bar, 2] + MOD_HALF
    hw[bar] = np.arctan(MOD_HALF / d)
    ec = ~bar
    zs = g.centre[ec, 2] - 0.5 * SENSOR_GAP * g.side[ec]
    rlo[ec] = cr[ec] - MOD_HALF
    rhi[ec] = np.sqrt((cr[ec] + MOD_HALF) ** 2 + MOD_HALF ** 2)
    zlo[ec] = zs
    zhi[ec] = zs
    hw[ec] = np.arctan(MOD_HALF / (cr[ec] - MOD_HALF))
    m = 0.05  # smearing / rounding margin [cm]
    return rlo - m, rhi + m, zlo - m, zhi + m, phc, hw + m / np.maximum(rlo, 1.0)


def build_module_map(g: Geometry, z_lum: float = 20.0, kappa_max: float = K_FIELD / 0.8,
                     hit_err: float = 3.0 * 1.41421356 * HIT_SIGMA):
    """Conservative module map as CSR (map_off, map_tgt), targets sorted per source."""
    rlo, rhi, zlo, zhi, phc, hw = _lower_sensor_boxes(g)
    n = g.n_mod
    src_all, tgt_all = [], []
    layers = np.unique(g.layer)
    for la in layers:
        for sa in np.unique(g.side[g.layer == la]):
            A = np.nonzero((g.layer == la) & (g.side == sa))[0]
            for lb in layers:
                for sb in np.unique(g.side[g.layer == lb]):
                    if not layers_adjacent(la, sa, lb, sb):
                        continue
                    B = np.nonzero((g.layer == lb) & (g.side == sb))[0]
                    ok = _map_pairs_ok(A, B, rlo, rhi, zlo, zhi, phc, hw,
                                       z_lum, kappa_max, hit_err)
                    ia, ib = np.nonzero(ok)
                    src_all.append(A[ia])
                    tgt_all.append(B[ib])
    src = np.concatenate(src_all) if src_all else np.zeros(0, np.int64)
    tgt = np.concatenate(tgt_all) if tgt_all else np.zeros(0, np.int64)
    order = np.lexsort((tgt, src))
    src, tgt = src[order], tgt[order]
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off)
    return off.astype(np.int32), tgt.astype(np.int32)


def _map_pairs_ok(A, B, rlo, rhi, zlo, zhi, phc, hw, z_lum, kappa_max, hit_err):
    ra0, ra1 = rlo[A][:, None], rhi[A][:, None]
    za0, za1 = zlo[A][:, None], zhi[A][:, None]
    rb0, rb1 = rlo[B][None, :], rhi[B][None, :]
    zb0, zb1 = zlo[B][None, :], zhi[B][None, :]
    # luminous-region road: F = za*rb - ra*zb must be small (|z0| <= z_lum); the interval
    # evaluation is exact because each variable occurs once.
    p1 = np.stack([za0 * rb0, za0 * rb1, za1 * rb0, za1 * rb1])
    p2 = np.stack([ra0 * zb0, ra0 * zb1, ra1 * zb0, ra1 * zb1])
    flo = p1.min(0) - p2.max(0)
    fhi = p1.max(0) - p2.min(0)
    fmin = np.where((flo <= 0) & (fhi >= 0), 0.0, np.minimum(np.abs(flo), np.abs(fhi)))
    dr_max = np.maximum(np.abs(rb1 - ra0), np.abs(rb0 - ra1))
    rhs = (z_lum + hit_err) * dr_max + hit_err * ra1
    road = fmin <= rhs * 1.02 + 0.5
    # bend window: |dphi| <= asin(rb*kappa_max/2 + e/dT) for a chord leaving A outward.
    dz_min = np.maximum(0.0, np.maximum(zb0 - za1, za0 - zb1))
    zabs = np.maximum(np.abs(za0), np.abs(za1))
    dt_min = np.maximum(np.maximum(rb0 - ra1, ra0 * (dz_min - hit_err) / (zabs + z_lum + hit_err)), 0.1)
    sarg = np.minimum(1.0, rb1 * 0.5 * kappa_max + hit_err / dt_min)
    amax = np.arcsin(sarg) + 0.02
    dphi = np.abs(np.angle(np.exp(1j * (phc[A][:, None] - phc[B][None, :]))))
    gap = dphi - hw[A][:, None] - hw[B][None, :]
    return road & (gap <= amax)


# --------------------------------------------------------------------------------------
# events
# --------------------------------------------------------------------------------------
@dataclass
class Event:
    x: np.ndarray        # float32 [n]
    y: np.ndarray
    z: np.ndarray
    sensor: np.ndarray   # int32 [n]
    pid: np.ndarray      # int32 [n]  particle index, -1 for noise
    particles: dict      # per particle: pt, eta, phi, q, vx, vy, vz, displaced
    seed: int = 0

    @property
    def n_hits(self) -> int:
        return int(self.x.shape[0])


def _wrap2pi(a):
    return np.mod(a, 2.0 * np.pi)


def _helix_point(C, qR, phi0, q, psi):
    ph = phi0 - q * psi
    return C[:, 0] - qR * np.sin(ph), C[:, 1] + qR * np.cos(ph)


def _plane_crossing(C, R, q, phi0, alpha, dpl):
    """Smallest positive turning angle where the transverse circle meets n.p = dpl."""
    qR = q * R
    w = (dpl - (np.cos(alpha) * C[:, 0] + np.sin(alpha) * C[:, 1])) / qR
    ok = np.abs(w) <= 1.0
    aw = np.arcsin(np.clip(w, -1.0, 1.0))
    ph1 = alpha - aw
    ph2 = alpha - np.pi + aw
    p1 = _wrap2pi(q * (phi0 - ph1))
    p2 = _wrap2pi(q * (phi0 - ph2))
    psi = np.minimum(p1, p2)
    return psi, ok


def _gen_hits(g: Geometry, parts: dict, rng: np.random.Generator):
    pt, eta, phi0, q = parts["pt"], parts["eta"], parts["phi"], parts["q"]
    vx, vy, vz = parts["vx"], parts["vy"], parts["vz"]
    npart = pt.shape[0]
    R = pt / K_FIELD
    C = np.stack([vx + q * R * np.sin(phi0), vy - q * R * np.cos(phi0)], axis=1)
    sh = np.sinh(eta)
    pidx = np.arange(npart)
    out_pos, out_sensor, out_pid = [], [], []

    def emit(sel_p, mods, sens, px, py, pz):
        out_pos.append(np.stack([px, py, pz], axis=1))
        out_sensor.append(2 * mods + sens)
        out_pid.append(sel_p)

    # --- barrel layers ---
    for li, rl in enumerate(BARREL_R):
        first, nphi = g.barrel_first[li], g.barrel_nphi[li]
        d = np.hypot(C[:, 0], C[:, 1])
        ok = (np.abs(R - rl) <= d) & (d <= R + rl) & (d > 0)
        a = (rl * rl - R * R + d * d) / (2.0 * np.where(d > 0, d, 1.0))
        h = np.sqrt(np.maximum(rl * rl - a * a, 0.0))
        ux, uy = C[:, 0] / np.where(d > 0, d, 1.0), C[:, 1] / np.where(d > 0, d, 1.0)
        best_psi = np.full(npart, np.inf)
        best_x = np.zeros(npart)
        best_y = np.zeros(npart)
        for sgn in (-1.0, 1.0):
            px = a * ux - sgn * h * uy
            py = a * uy + sgn * h * ux
            ph = np.arctan2(-(px - C[:, 0]) / (q * R), (py - C[:, 1]) / (q * R))
            psi = _wrap2pi(q * (phi0 - ph))
            better = psi < best_psi
            best_psi = np.where(better, psi, best_psi)
            best_x = np.where(better, px, best_x)
            best_y = np.where(better, py, best_y)
        zc = vz + R * best_psi * sh
        ok &= (best_psi <= np.pi) & (np.abs(zc) < BARREL_ZMAX + 2 * MOD_HALF)
        sel = pidx[ok]
        if sel.size == 0:
            continue
        phc = np.arctan2(best_y[sel], best_x[sel])
        ip0 = np.rint(phc / (2 * np.pi / nphi)).astype(np.int64)
        iz0 = np.floor((zc[sel] + BARREL_ZMAX) / (2 * MOD_HALF)).astype(np.int64)
        for dip in (-1, 0, 1):
            for diz in (-1, 0, 1):
                ip = np.mod(ip0 + dip, nphi)
                iz = iz0 + diz
                zok = (iz >= 0) & (iz < BARREL_NZ)
                mods = first + np.clip(iz, 0, BARREL_NZ - 1) * nphi + ip
                alpha = 2 * np.pi * ip / nphi
                for s, off in ((0, -0.5 * SENSOR_GAP), (1, 0.5 * SENSOR_GAP)):
                    dpl = rl + off
                    p = sel
                    psi, pok = _plane_crossing(C[p], R[p], q[p], phi0[p], alpha, dpl)
                    px, py = _helix_point(C[p], q[p] * R[p], phi0[p], q[p], psi)
                    pz = vz[p] + R[p] * psi * sh[p]
                    cen = g.centre[mods] + off * g.normal[mods]
                    rel = np.stack([px, py, pz], 1) - cen
                    u = np.einsum("ij,ij->i", rel, g.uax[mods])
                    v = np.einsum("ij,ij->i", rel, g.vax[mods])
                    keep = (zok & pok & (psi <= np.pi) & (np.abs(u) <= MOD_HALF)
                            & (np.abs(v) <= MOD_HALF))
                    if keep.any():
                        emit(p[keep], mods[keep], np.full(keep.sum(), s), px[keep], py[keep], pz[keep])
    # --- endcap disks ---
    if g.with_endcap:
        for sd in (-1, 1):
            for di, zd in enumerate(DISK_Z):
                zmid = sd * zd
                with np.errstate(divide="ignore", invalid="ignore"):
                    psi_c = (zmid - vz) / (R * sh)
                ok = np.isfinite(psi_c) & (psi_c > 0) & (psi_c <= np.pi)
                sel = pidx[ok]
                if sel.size == 0:
                    continue
                px, py = _helix_point(C[sel], q[sel] * R[sel], phi0[sel], q[sel], psi_c[sel])
                rr = np.hypot(px, py)
                phc = np.arctan2(py, px)
                ri0 = np.rint((rr - RING_RC[0]) / 10.0).astype(np.int64)
                for dri in (-1, 0, 1):
                    ri = ri0 + dri
                    rok = (ri >= 0) & (ri < len(RING_RC))
                    ric = np.clip(ri, 0, len(RING_RC) - 1)
                    firsts = np.array([g.disk_first[(sd, di, k)][0] for k in range(len(RING_RC))])
                    nphis = np.array([g.disk_first[(sd, di, k)][1] for k in range(len(RING_RC))])
                    f0, npp = firsts[ric], nphis[ric]
                    ip0 = np.rint(phc / (2 * np.pi / npp)).astype(np.int64)
                    for dip in (-1, 0, 1):
                        ip = np.mod(ip0 + dip, npp)
                        mods = f0 + ip
                        for s, off in ((0, -0.5 * SENSOR_GAP), (1, 0.5 * SENSOR_GAP)):
                            zs = sd * (zd + off)
                            p = sel
                            psi = (zs - vz[p]) / (R[p] * sh[p])
                            qx, qy = _helix_point(C[p], q[p] * R[p], phi0[p], q[p], psi)
                            cen = g.centre[mods]
                            u = (qx - cen[:, 0]) * g.uax[mods, 0] + (qy - cen[:, 1]) * g.uax[mods, 1]
                            v = (qx - cen[:, 0]) * g.vax[mods, 0] + (qy - cen[:, 1]) * g.vax[mods, 1]
                            keep = (rok & (psi > 0) & (psi <= np.pi) & (np.abs(u) <= MOD_HALF)
                                    & (np.abs(v) <= MOD_HALF))
                            if keep.any():
                                emit(p[keep], mods[keep], np.full(keep.sum(), s), qx[keep], qy[keep],
                                     np.full(keep.sum(), zs))
    if out_pos:
        pos = np.concatenate(out_pos)
        sensor = np.concatenate(out_sensor).astype(np.int64)
        pid = np.concatenate(out_pid).astype(np.int64)
    else:
        pos = np.zeros((0, 3))
        sensor = np.zeros(0, np.int64)
        pid = np.zeros(0, np.int64)
    return pos, sensor, pid


def _smear(g: Geometry, pos, sensor, rng, sigma):
    if sigma <= 0 or pos.shape[0] == 0:
        return pos
    m = sensor // 2
    n1 = rng.normal(0.0, sigma, pos.shape[0])
    n2 = rng.normal(0.0, sigma, pos.shape[0])
    return pos + n1[:, None] * g.uax[m] + n2[:, None] * g.vax[m]


def _noise_hits(g: Geometry, n, rng):
    sens = rng.integers(0, g.n_sensor, n)
    u = rng.uniform(-MOD_HALF, MOD_HALF, n)
    v = rng.uniform(-MOD_HALF, MOD_HALF, n)
    cen = g.sensor_centre(sens)
    m = sens // 2
    pos = cen + u[:, None] * g.uax[m] + v[:, None] * g.vax[m]
    return pos, sens


def make_event(g: Geometry, parts: dict, rng: np.random.Generator, sigma=HIT_SIGMA,
               noise_frac=0.0, shuffle=True, seed=0) -> Event:
    pos, sensor, pid = _gen_hits(g, parts, rng)
    pos = _smear(g, pos, sensor, rng, sigma)
    if noise_frac > 0:
        nn = int(round(noise_frac * pos.shape[0]))
        npos, nsens = _noise_hits(g, nn, rng)
        pos = np.concatenate([pos, npos])
        sensor = np.concatenate([sensor, nsens])
        pid = np.concatenate([pid, np.full(nn, -1)])
    if shuffle:
        perm = rng.permutation(pos.shape[0])
        pos, sensor, pid = pos[perm], sensor[perm], pid[perm]
    return Event(x=pos[:, 0].astype(np.float32), y=pos[:, 1].astype(np.float32),
                 z=pos[:, 2].astype(np.float32), sensor=sensor.astype(np.int32),
                 pid=pid.astype(np.int32), particles=parts, seed=seed)


def _particles(pt, eta, phi, q, vx, vy, vz, displaced=None):
    n = pt.shape[0]
    return dict(pt=pt.astype(np.float64), eta=eta.astype(np.float64), phi=phi.astype(np.float64),
                q=q.astype(np.float64), vx=vx.astype(np.float64), vy=vy.astype(np.float64),
                vz=vz.astype(np.float64),
                displaced=(np.zeros(n, bool) if displaced is None else displaced))


def toy_event(g: Geometry, index: int = 0, n_muons: int = 50, sigma=HIT_SIGMA) -> Event:
    """50 prompt muons, pT log-uniform 1-10 GeV, |eta| < 1, no pile-up, no noise."""
    seed = 1000 * 1 + index
    rng = np.random.Generator(np.random.PCG64(seed))
    pt = np.exp(rng.uniform(np.log(1.0), np.log(10.0), n_muons))
    eta = rng.uniform(-1.0, 1.0, n_muons)
    phi = rng.uniform(-np.pi, np.pi, n_muons)
    q = rng.choice([-1.0, 1.0], n_muons)
    zero = np.zeros(n_muons)
    parts = _particles(pt, eta, phi, q, zero, zero, zero)
    return make_event(g, parts, rng, sigma=sigma, noise_frac=0.0, seed=seed)


def pileup_event(g: Geometry, index: int = 0, pileup: int = 200, config: int = 2,
                 mean_per_vertex: float = 50.0, noise_frac: float = 0.03,
                 displaced_frac: float = 0.05, sigma=HIT_SIGMA) -> Event:
    """HL-LHC-like event: `pileup` vertices (sigma_z 5 cm), Poisson(50) particles each,
    pT = 0.8 + Exp(1) GeV, |eta| < 2.4, 5% displaced by up to 10 cm, 3% noise hits."""
    seed = 1000 * config + index
    rng = np.random.Generator(np.random.PCG64(seed))
    vz_v = rng.normal(0.0, 5.0, pileup)
    vx_v = rng.normal(0.0, 0.001, pileup)
    vy_v = rng.normal(0.0, 0.001, pileup)
    mult = rng.poisson(mean_per_vertex, pileup)
    vid = np.repeat(np.arange(pileup), mult)
    n = vid.shape[0]
    pt = 0.8 + rng.exponential(1.0, n)
    eta = rng.uniform(-2.4, 2.4, n)
    phi = rng.uniform(-np.pi, np.pi, n)
    q = rng.choice([-1.0, 1.0], n)
    vx, vy, vz = vx_v[vid].copy(), vy_v[vid].copy(), vz_v[vid].copy()
    disp = rng.uniform(0, 1, n) < displaced_frac
    dd = rng.uniform(0.0, 10.0, n)
    da = rng.uniform(-np.pi, np.pi, n)
    vx = np.where(disp, vx + dd * np.cos(da), vx)
    vy = np.where(disp, vy + dd * np.sin(da), vy)
    parts = _particles(pt, eta, phi, q, vx, vy, vz, disp)
    return make_event(g, parts, rng, sigma=sigma, noise_frac=noise_frac, seed=seed)


def muon_cube_event(g: Geometry, index: int = 0, n_muons: int = 20, config: int = 6,
                    half: float = 2.5, sigma=HIT_SIGMA) -> Event:
    """Section 3's displaced-track sample: muons produced at points uniform in a cube of
    side 2 * half cm (5 cm) around the origin; pT log-uniform 1-20 GeV, |eta| < 2.4, no
    pile-up, no noise."""
    seed = 1000 * config + index
    rng = np.random.Generator(np.random.PCG64(seed))
    pt = np.exp(rng.uniform(np.log(1.0), np.log(20.0), n_muons))
    eta = rng.uniform(-2.4, 2.4, n_muons)
    phi = rng.uniform(-np.pi, np.pi, n_muons)
    q = rng.choice([-1.0, 1.0], n_muons)
    v = rng.uniform(-half, half, (3, n_muons))
    parts = _particles(pt, eta, phi, q, v[0], v[1], v[2], np.hypot(v[0], v[1]) > 0.0)
    return make_event(g, parts, rng, sigma=sigma, noise_frac=0.0, seed=seed)


def muon_event(g: Geometry, pts, etas, phis, qs, vertex=(0.0, 0.0, 0.0), sigma=0.0,
               seed=0) -> Event:
    """Explicit list of tracks (for closed-form and threshold tests)."""
    pts = np.asarray(pts, np.float64)
    n = pts.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = _particles(pts, np.asarray(etas, np.float64), np.asarray(phis, np.float64),
                       np.asarray(qs, np.float64), np.full(n, vertex[0]), np.full(n, vertex[1]),
                       np.full(n, vertex[2]))
    return make_event(g, parts, rng, sigma=sigma, noise_frac=0.0, shuffle=False, seed=seed)


# --------------------------------------------------------------------------------------
# pixel seeds (Table 1 step 0: track segments from the inner tracker)
# --------------------------------------------------------------------------------------
#: barrel pixel layers (cylinders) of the synthetic inner tracker
PIXEL_R = (3.0, 6.8, 10.9, 16.0)
PIXEL_ZMAX = 100.0
PIXEL_SIGMA_RPHI = 0.001
PIXEL_SIGMA_Z = 0.002


@dataclass
class PixelSeeds:
    hits: np.ndarray     # float32 [n, 4, 3]: (x, y, z) on the four pixel layers, inner first
    pid: np.ndarray      # int32 [n]: particle index, -1 for a fake seed

    @property
    def n(self) -> int:
        return int(self.hits.shape[0])


def _cylinder_crossing(C, R, q, phi0, rho):
    """First crossing (smallest turning angle) of each transverse circle with the cylinder
    of radius rho around the beamline: (x, y, psi, ok)."""
    n = C.shape[0]
    d = np.hypot(C[:, 0], C[:, 1])
    ok = (np.abs(R - rho) <= d) & (d <= R + rho) & (d > 0)
    dd = np.where(d > 0, d, 1.0)
    a = (rho * rho - R * R + d * d) / (2.0 * dd)
    h = np.sqrt(np.maximum(rho * rho - a * a, 0.0))
    ux, uy = C[:, 0] / dd, C[:, 1] / dd
    best_psi = np.full(n, np.inf)
    best_x = np.zeros(n)
    best_y = np.zeros(n)
    for sgn in (-1.0, 1.0):
        px = a * ux - sgn * h * uy
        py = a * uy + sgn * h * ux
        ph = np.arctan2(-(px - C[:, 0]) / (q * R), (py - C[:, 1]) / (q * R))
        psi = _wrap2pi(q * (phi0 - ph))
        better = psi < best_psi
        best_psi = np.where(better, psi, best_psi)
        best_x = np.where(better, px, best_x)
        best_y = np.where(better, py, best_y)
    return best_x, best_y, best_psi, ok & (best_psi <= np.pi)


def pixel_seeds(ev: Event, fake_frac: float = 0.05, sigma_rphi: float = PIXEL_SIGMA_RPHI,
                sigma_z: float = PIXEL_SIGMA_Z) -> PixelSeeds:
    """Pixel seeds (pLS) of an event, standing in for the upstream iteration of the paper's
    Section 1 that runs on the inner-tracker hits: every particle of the event whose helix
    crosses all four pixel cylinders (PIXEL_R, |z| < PIXEL_ZMAX) before turning back gives
    one seed of four hits, smeared by sigma_rphi along the cylinder and sigma_z in z. Fake
    seeds (fake_frac of the real count) join the inner two hits of one seed to the outer
    two of the seed nearest in azimuth at the third layer. Seeds come in random order. The
    random stream is the event's own seed offset by 500000, so the hits are unchanged."""
    P = ev.particles
    rng = np.random.Generator(np.random.PCG64(int(ev.seed) + 500_000))
    pt, eta, phi0, q = P["pt"], P["eta"], P["phi"], P["q"]
    n = pt.shape[0]
    R = pt / K_FIELD
    C = np.stack([P["vx"] + q * R * np.sin(phi0), P["vy"] - q * R * np.cos(phi0)], axis=1)
    sh = np.sinh(eta)
    ok = np.ones(n, bool)
    H = np.zeros((n, 4, 3))
    for k, rho in enumerate(PIXEL_R):
        x, y, psi, okk = _cylinder_crossing(C, R, q, phi0, rho)
        z = P["vz"] + R * psi * sh
        ok &= okk & (np.abs(z) < PIXEL_ZMAX)
        H[:, k] = np.stack([x, y, z], axis=1)
    sel = np.flatnonzero(ok)
    H = H[sel]
    r = np.hypot(H[..., 0], H[..., 1])
    e1 = rng.normal(0.0, sigma_rphi, r.shape) if sigma_rphi > 0 else np.zeros(r.shape)
    e2 = rng.normal(0.0, sigma_z, r.shape) if sigma_z > 0 else np.zeros(r.shape)
    tx, ty = -H[..., 1] / r, H[..., 0] / r
    H[..., 0] += tx * e1
    H[..., 1] += ty * e1
    H[..., 2] += e2
    pid = sel.astype(np.int64)
    nf = int(round(fake_frac * len(sel)))
    if nf > 0 and len(sel) > 1:
        ph3 = np.arctan2(H[:, 2, 1], H[:, 2, 0])
        order = np.argsort(ph3, kind="stable")
        pos = np.empty(len(sel), np.int64)
        pos[order] = np.arange(len(sel))
        a = rng.choice(len(sel), nf, replace=False)
        b = order[(pos[a] + 1) % len(sel)]
        F = np.concatenate([H[a, :2], H[b, 2:]], axis=1)
        H = np.concatenate([H, F])
        pid = np.concatenate([pid, np.full(nf, -1)])
    perm = rng.permutation(H.shape[0])
    return PixelSeeds(hits=H[perm].astype(np.float32), pid=pid[perm].astype(np.int32))


# --------------------------------------------------------------------------------------
# parameters passed to both implementations
# --------------------------------------------------------------------------------------
def default_cuts() -> dict:
    """Cut parameters (float32 values) for the mini-doublet .. quintuplet selections.

    kappa_max is the curvature of a 0.8 GeV track (Section 1's MD threshold), z_lum the
    half-length of the luminous-region road, hit_err the 3-sigma error of a two-hit
    difference with 30 um hits."""
    return dict(
        kappa_max=np.float32(K_FIELD / 0.8),
        z_lum=np.float32(20.0),
        hit_err=np.float32(3.0 * 1.41421356 * HIT_SIGMA),
        sensor_gap=np.float32(SENSOR_GAP),
        t3_kappa_factor=np.float32(1.25),
        t3_rz_tol=np.float32(0.02),
        t5_kappa_rel=np.float32(0.3),
        t5_kappa_abs=np.float32(0.001),
        t5_rz_tol=np.float32(0.03),
        t5_chi2_max=np.float32(0.0),       # DNN mode: no circle-fit selection
        hit_sigma=np.float32(HIT_SIGMA),
        k_field=np.float32(K_FIELD),
        wp=np.float32(0.5),
    )


#: parameter order of the pixel-seed matching (lst_pixel_cuts)
PIXEL_CUT_FIELDS = ("kappa_rel", "kappa_abs", "rz_tol", "dphi0", "dphi_cm", "dm_abs", "dm_rel")


def default_pixel_cuts() -> dict:
    """Matching of pixel seeds to T5s and T3s (float32 values): curvature consistency (the
    relative and absolute tolerances, for the seed's own curvature and for the circle through
    the seed's end hits and the object's first anchor), the rz interpolation tolerance at
    the seed's outer hit, and the search window: the turn of the azimuth from the seed's
    outer hit to the object's first anchor (a constant plus a rate per cm of radius; 0.0125
    per cm bounds the half-curvature of a T3 at its pT limit, 1.25 x 0.8 GeV / 0.64 GeV) and
    the r-z slope (absolute and relative)."""
    return dict(kappa_rel=np.float32(0.2), kappa_abs=np.float32(0.0005), rz_tol=np.float32(0.05),
                dphi0=np.float32(0.05), dphi_cm=np.float32(0.0125), dm_abs=np.float32(0.05),
                dm_rel=np.float32(0.5))


def open_cuts() -> dict:
    """Cut parameters with the fit-quality tolerances of steps 3-4 opened up (Section 2: the
    selections correlated with the quality of the r-phi circle fit are removed when the
    T5-DNN decides instead). Used to build the DNN's training sample: ~95k T5s per
    PU200-like event, ~64% of them real."""
    c = default_cuts()
    c.update(t3_rz_tol=np.float32(0.2), t5_rz_tol=np.float32(2.0), t5_kappa_rel=np.float32(2.0),
             t5_kappa_abs=np.float32(0.01))
    return c


def pre_dnn_cuts(chi2_max: float = 20.0) -> dict:
    """The pre-DNN mode (Section 2): the open-cut quintuplets that also pass a circle-fit
    chi2 selection (five anchors, sigma = hit_sigma), instead of the T5-DNN score."""
    c = open_cuts()
    c["t5_chi2_max"] = np.float32(chi2_max)
    return c


CUT_FIELDS = ("kappa_max", "z_lum", "hit_err", "sensor_gap", "t3_kappa_factor", "t3_rz_tol",
              "t5_kappa_rel", "t5_kappa_abs", "t5_rz_tol", "t5_chi2_max", "hit_sigma",
              "k_field", "wp")

N_FEATURES = 38
HIDDEN = 32


def xavier_mlp(n_hidden_layers: int = 2, seed: int = 2403) -> dict:
    """Xavier-uniform weights (biases zero) from a seeded PCG64 stream, PyTorch
    Linear layout: W[l] has shape (out, in)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = [N_FEATURES] + [HIDDEN] * n_hidden_layers + [1]
    Ws, bs = [], []
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        Ws.append(rng.uniform(-lim, lim, (fan_out, fan_in)))
        bs.append(np.zeros(fan_out))
    return dict(W=Ws, b=bs)


def mlp_flat(mlp: dict, dtype=np.float64) -> np.ndarray:
    """Flatten weights as W0,b0,W1,b1,...,Wout,bout (row-major (out,in))."""
    parts = []
    for W, b in zip(mlp["W"], mlp["b"]):
        parts.append(np.asarray(W, dtype).ravel())
        parts.append(np.asarray(b, dtype).ravel())
    return np.concatenate(parts)


def mlp_hidden_layers(mlp: dict) -> int:
    return len(mlp["W"]) - 1
