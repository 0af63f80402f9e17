"""GPU: the launch-shape autotuner keeps results identical, never slows its own stage
down, and its cache round-trips."""
import numpy as np
import pytest

from paper_2403_13166_gb300 import autotune, lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tuning_keeps_results_and_caches(geom_full, cuts, tmp_path):
    evs = [synth.pileup_event(geom_full, i, pileup=pu, mean_per_vertex=96, config=4)
           for i, pu in enumerate((60, 140, 100, 30))]
    d = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (e.x, e.y, e.z, e.sensor)] for e in evs]
    c = lst.Context(0, max_events=8, use_graphs=1)
    c.load_geometry(geom_full, cuts, synth.mlp_flat(synth.xavier_mlp()), 2)

    def results():
        hs = c.run_batch(d)
        out = [np.sort(h.candidates(lst.LST_TC)[0], axis=0) for h in hs] + \
              [np.sort(h.candidates(lst.LST_LS), axis=0) for h in hs]
        for h in hs:
            h.release()
        return out

    before = results()
    start = c.get_launch()
    space = {"ls_threads": (64, 128, 256), "ls_list": (512, 2048), "t3_threads": (128, 256)}
    path = str(tmp_path / "cache.json")
    r = autotune.tune_or_load(c, d, path=path, reps=2, space=space)
    assert r["cached"] is False and len(r["trials"]) >= 3
    after = results()
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    c.set_launch(**start)
    r2 = autotune.tune_or_load(c, d, path=path)
    assert r2["cached"] is True and c.get_launch() == r["launch"]
    c.close()
