"""Input generator pins: hits lie on their sensor planes and on the helix of the Lorentz force."""
import numpy as np
import pytest

from paper_2403_13166_gb300 import synth


def _rk4_track(p, q, R, phi0, vx, vy, ds=0.05, smax=800.0):
    """Integrate d(x,y)/ds = u, du/ds = (q/R) * (u_y, -u_x) (positive charge turns clockwise
    in a field along +z, F = q v x B) in FP64; return the sampled transverse path."""
    def f(s):
        x, y, ux, uy = s
        return np.array([ux, uy, (q / R) * uy, -(q / R) * ux])
    st = np.array([vx, vy, np.cos(phi0), np.sin(phi0)])
    pts = [st[:2].copy()]
    for _ in range(int(smax / ds)):
        k1 = f(st); k2 = f(st + 0.5 * ds * k1); k3 = f(st + 0.5 * ds * k2); k4 = f(st + ds * k3)
        st = st + ds / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        pts.append(st[:2].copy())
    return np.array(pts)


def test_toy_geometry_and_hit_count(geom_toy):
    assert geom_toy.n_mod == 5760
    e = synth.toy_event(geom_toy, 0)
    assert 500 <= e.n_hits <= 700          # ~600 hits: 50 muons x 6 layers x 2 sensors


def test_full_geometry_module_count(geom_full):
    # 6 barrel layers (5760 modules) + 2 x 5 disks x 389 modules
    assert geom_full.n_mod == 5760 + 10 * 389
    assert set(np.unique(geom_full.layer)) == set(range(1, 12))


@pytest.mark.parametrize("q", [-1.0, 1.0])
def test_hits_on_sensor_plane_and_helix(geom_full, q):
    pts = [0.9, 1.7, 4.0, 12.0]
    etas = [0.1, 0.8, 1.6, 2.2]
    phis = [0.3, -2.0, 2.5, -0.7]
    e = synth.muon_event(geom_full, pts, etas, phis, [q] * 4, sigma=0.0)
    assert e.n_hits > 0
    pos = np.stack([e.x, e.y, e.z], 1).astype(np.float64)
    cen = geom_full.sensor_centre(e.sensor)
    nrm = geom_full.normal[e.sensor // 2]
    assert np.max(np.abs(np.einsum("ij,ij->i", pos - cen, nrm))) < 2e-4
    for p in range(4):
        sel = e.pid == p
        R = pts[p] / synth.K_FIELD
        path = _rk4_track(pts[p], q, R, phis[p], 0.0, 0.0, smax=min(400.0, np.pi * R))
        # transverse distance of each hit to the numerically integrated trajectory
        d = np.min(np.hypot(path[None, :, 0] - pos[sel, 0, None], path[None, :, 1] - pos[sel, 1, None]), 1)
        assert np.max(d) < 0.03  # sampling step 0.05 cm bounds the distance
        # z grows linearly with transverse arc length at rate sinh(eta)
        idx = np.argmin(np.hypot(path[None, :, 0] - pos[sel, 0, None], path[None, :, 1] - pos[sel, 1, None]), 1)
        s = idx * 0.05
        assert np.max(np.abs(pos[sel, 2] - s * np.sinh(etas[p]))) < 0.05 * abs(np.sinh(etas[p])) + 1e-3


def test_disk_crossing_matches_stepping(geom_full):
    e = synth.muon_event(geom_full, [3.0], [2.0], [1.0], [1.0], sigma=0.0)
    disk = geom_full.subdet[e.sensor // 2] == 1
    assert disk.sum() >= 8
    R = 3.0 / synth.K_FIELD
    path = _rk4_track(3.0, 1.0, R, 1.0, 0.0, 0.0, ds=0.01, smax=120.0)
    for x, y, z in zip(e.x[disk], e.y[disk], e.z[disk]):
        s_t = z / np.sinh(2.0)
        i = int(round(s_t / 0.01))
        assert np.hypot(path[i, 0] - x, path[i, 1] - y) < 0.02


def test_pileup_event_shape(geom_full):
    e = synth.pileup_event(geom_full, 0, pileup=20)
    assert e.x.dtype == np.float32 and e.sensor.dtype == np.int32
    assert e.sensor.min() >= 0 and e.sensor.max() < geom_full.n_sensor
    noise = (e.pid < 0).mean()
    assert 0.02 < noise < 0.04
    assert 0.03 < e.particles["displaced"].mean() < 0.08


def test_module_map_respects_layer_relation(geom_full):
    g = geom_full
    src = np.repeat(np.arange(g.n_mod), np.diff(g.map_off))
    tgt = g.map_tgt
    ok = synth.layers_adjacent(g.layer[src], g.side[src], g.layer[tgt], g.side[tgt])
    assert ok.all()
    assert (np.diff(g.map_off) > 0).sum() > 0.8 * (g.layer < 11).sum() * 0.5
