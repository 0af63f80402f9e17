"""The threshold pins catch plausible mistakes in the oracle's cut code, and the pixel-seed
pins those in its pixel-seed steps.

Each case edits one expression of a private copy of the oracle's C source (a dropped term,
a removed branch, a loosened or mis-scaled tolerance, a wrong radius, sign or order), rebuilds
it and runs `test_oracle_thresholds.py` (cuts) or `test_oracle_pixel.py` (pixel seeds)
against the copy: every edit must turn at least one of those tests red, and the unedited copy
must stay green. The one edit that no test can
catch, removing the barrel MD direction test, is left out on purpose: within the tracker
(r <= 110 cm, 2.6 mm sensor gap) an upper hit on the beamline side of the lower hit always
fails the MD bend or road test as well, so that branch changes no decision.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "LS kappa, inner MD check removed": ("if (bA && !cut_le(", "if (0 && bA && !cut_le("),
    "LS kappa, outer MD check removed": ("if (bB && !cut_le(", "if (0 && bB && !cut_le("),
    "LS kappa, outer bound doubled": (
        "2.0f * (e / c->sensor_gap) / rb + 2.0f * (e / dT) / rb",
        "2.0f * (2.0f * (e / c->sensor_gap) / rb + 2.0f * (e / dT) / rb)"),
    "LS kappa, inner bound at the outer radius": (
        "2.0f * (e / c->sensor_gap) / ra", "2.0f * (e / c->sensor_gap) / rb"),
    "endcap MD bend removed": (
        "if (!cut_le(fabsf(perp), para * T + c->hit_err)) return 0;",
        "if (0 && !cut_le(fabsf(perp), para * T + c->hit_err)) return 0;"),
    "endcap MD bend uses sin for tan": ("float T = S / sqrtf(1.0f - S * S);", "float T = S;"),
    "endcap MD road x3": ("adz * rL * c->z_lum / (azl", "3.0f * adz * rL * c->z_lum / (azl"),
    "barrel MD bend error dropped": (
        "rL * (0.5f * c->kappa_max) + c->hit_err / c->sensor_gap", "rL * (0.5f * c->kappa_max)"),
    "barrel MD road x3": ("(c->z_lum / rL) * dr + c->hit_err", "3.0f * (c->z_lum / rL) * dr + c->hit_err"),
    "endcap MD z direction removed": ("if (!(dt > 0.0f && dz * L.z > 0.0f))", "if (!(dt > 0.0f))"),
    "LS bend error dropped": ("rb * (0.5f * c->kappa_max) + e / dT", "rb * (0.5f * c->kappa_max)"),
    "LS road error over the lever arm dropped": ("fabsf(rb - ra) + e * ra))", "fabsf(rb - ra)))"),
    "LS curvature without the factor 2": ("float k = 2.0f * sl / rb;", "float k = sl / rb;"),
    "T3 pT removed": (
        "if (!cut_le(fabsf(k3), c->kappa_max * c->t3_kappa_factor)) return 0;",
        "if (0 && !cut_le(fabsf(k3), c->kappa_max * c->t3_kappa_factor)) return 0;"),
    "T3 arc-length series dropped": ("float s01 = a * (1.0f + a * a * k3 * k3 / 24.0f);", "float s01 = a;"),
    "T5 charge test removed": ("if (!(ka * kb > 0.0f)) return 0;", "if (0) return 0;"),
    "T5 kappa relative tolerance x3": ("c->t5_kappa_rel * 0.5f", "3.0f * c->t5_kappa_rel * 0.5f"),
    "T5 kappa absolute tolerance dropped": (" + c->t5_kappa_abs))", "))"),
    "T5 arc-length series dropped": ("float s = d * (1.0f + d * d * kbar * kbar / 24.0f);", "float s = d;"),
}

# edits of the pixel-seed steps, caught by test_oracle_pixel.py
PIXEL_MUTANTS = {
    "pixel azimuth hemisphere test removed": ("if (!(H4[0] * P0[0] + H4[1] * P0[1] > 0.0f)) return 0;",
                                              "if (0) return 0;"),
    "pixel azimuth turn unbounded": ("(pc->dphi0 + pc->dphi_cm * (P0[3] - r4))", "(2.0f + pc->dphi_cm * (P0[3] - r4))"),
    "pixel azimuth turn per cm dropped": ("(pc->dphi0 + pc->dphi_cm * (P0[3] - r4))", "(pc->dphi0)"),
    "pixel slope window removed": ("if (!(fabsf(mp - mo) <= pc->dm_abs + pc->dm_rel * fabsf(mo))) return 0;",
                                   "if (0) return 0;"),
    "pixel pT test removed": ("if (!pix_kappa_ok(kp, ko, pc)) return 0;", "if (0) return 0;"),
    "pixel circle test removed": ("if (!pix_kappa_ok(kx, ko, pc)) return 0;", "if (0) return 0;"),
    "pixel circle through H3": ("float kx = pix_curv3(H1, H4, P0);", "float kx = pix_curv3(H3, H4, P0);"),
    "pixel rz tolerance x3": ("if (!(res <= pc->rz_tol)) return 0;", "if (!(res <= 3.0f * pc->rz_tol)) return 0;"),
    "pixel greedy prefers the worse match": ("if (x->res != y->res) return x->res < y->res ? -1 : 1;",
                                             "if (x->res != y->res) return x->res > y->res ? -1 : 1;"),
    "pixel T3s of pT5s stay eligible": ("elig[u] = !(mdin[T3[u].md[0]] && mdin[T3[u].md[1]] && mdin[T3[u].md[2]]);",
                                        "elig[u] = 1;"),
    "pixel step 6 dropped": ("row[0] = t5p[t] >= 0 ? 5 : 6;", "if (t5p[t] < 0) { R.n--; continue; } row[0] = 5;"),
}


def _copy(dst):
    os.makedirs(dst)
    for d in ("oracle", "paper_2403_13166_gb300"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d),
                        ignore=shutil.ignore_patterns("*.so", "_lib", "_tuned", "__pycache__", "weights", "csrc"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle_thresholds.py", "test_oracle_pixel.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))


def _run(dst, edit, test_file):
    _copy(dst)
    if edit is not None:
        src = os.path.join(dst, "oracle", "lst_oracle.c")
        text = open(src).read()
        a, b = edit
        assert text.count(a) == 1, a
        open(src, "w").write(text.replace(a, b))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/" + test_file], cwd=dst, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


@pytest.mark.parametrize("mutants,test_file", [(MUTANTS, "test_oracle_thresholds.py"),
                                               (PIXEL_MUTANTS, "test_oracle_pixel.py")])
def test_every_mutant_is_caught(tmp_path, mutants, test_file):
    jobs = {"unedited": None, **mutants}
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {k: ex.submit(_run, str(tmp_path / f"m{i}"), v, test_file) for i, (k, v) in enumerate(jobs.items())}
        res = {k: f.result() for k, f in futs.items()}
    rc, out = res.pop("unedited")
    assert rc == 0, out
    survivors = [k for k, (rc, out) in res.items() if rc != 1 or "CalledProcessError" in out]
    assert not survivors, {k: res[k][1] for k in survivors}
