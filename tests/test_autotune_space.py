"""Host logic of the autotuner (CPU): every tunable is a field of lst_launch and is judged
by the stage its kernel runs in."""
from paper_2403_13166_gb300 import autotune, lst

EXPECTED_STAGE = {"md_threads": "md", "ls_threads": "ls", "ls_list": "ls", "t3_threads": "t3",
                  "t5_threads": "t5", "sc_threads": "score"}


def test_space_parameters_are_launch_fields_with_their_stage():
    fields = {f for f, _ in lst.lst_launch._fields_}
    assert set(autotune.SPACE) <= set(autotune.STAGE) <= fields
    for p, k in autotune.STAGE.items():
        assert 0 <= k < lst.N_STAGES
        assert lst.STAGES[k] == EXPECTED_STAGE[p], p
    for p, values in autotune.SPACE.items():
        assert len(values) >= 2 and all(v % 32 == 0 and 32 <= v <= 256 for v in values), p


def test_workload_key_rounds_hits():
    class T:
        def __init__(self, n):
            self.shape = (n,)
    assert autotune.workload_key([(T(249_276),)] * 64) == "batch64|hits250000"
