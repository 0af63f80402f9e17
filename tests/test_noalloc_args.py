"""Host-side checks of lst_find_minidoublets_noalloc's buffers (no GPU needed): its kernels
trust the sizes they are given, so the binding rejects any buffer of the wrong kind, type,
shape, length or device before anything reaches the library."""
import numpy as np
import pytest

from paper_2403_13166_gb300 import lst

torch = pytest.importorskip("torch")

DEV = torch.device("cpu")   # stands in for the context's CUDA device


def _good(n=10, cap=6):
    f = lambda: torch.zeros(n, dtype=torch.float32)
    return dict(x=f(), y=f(), z=f(), sensor=torch.zeros(n, dtype=torch.int32),
                md_hits=torch.zeros((cap, 2), dtype=torch.int32),
                md_kappa=torch.zeros(cap, dtype=torch.float32), md_count=torch.zeros(1, dtype=torch.int64))


def _call(device=DEV, **kw):
    a = _good()
    a.update(kw)
    return lst.noalloc_arguments(device, a["x"], a["y"], a["z"], a["sensor"], a["md_hits"], a["md_kappa"],
                                 a["md_count"])


def test_good_buffers_pass():
    assert _call() == (10, 6)
    assert _call(md_kappa=None) == (10, 6)
    assert _call(md_kappa=torch.zeros(9, dtype=torch.float32)) == (10, 6)
    z = torch.zeros(0, dtype=torch.float32)
    assert _call(x=z, y=z, z=z, sensor=torch.zeros(0, dtype=torch.int32)) == (0, 6)


@pytest.mark.parametrize("kw,what", [
    (dict(x=np.zeros(10, np.float32)), "x: expected a torch tensor"),
    (dict(md_hits=np.zeros((6, 2), np.int32)), "md_hits: expected a torch tensor"),
    (dict(y=torch.zeros(10, dtype=torch.float64)), "y: dtype"),
    (dict(sensor=torch.zeros(10, dtype=torch.int64)), "sensor: dtype"),
    (dict(z=torch.zeros(9, dtype=torch.float32)), "z: length 9"),
    (dict(sensor=torch.zeros(11, dtype=torch.int32)), "sensor: length 11"),
    (dict(x=torch.zeros((5, 2), dtype=torch.float32)), "x: expected one dimension"),
    (dict(x=torch.zeros(20, dtype=torch.float32)[::2]), "x: not contiguous"),
    (dict(md_hits=torch.zeros(12, dtype=torch.int32)), "md_hits: expected shape"),
    (dict(md_hits=torch.zeros((6, 3), dtype=torch.int32)), "md_hits: expected shape"),
    (dict(md_hits=torch.zeros((6, 2), dtype=torch.int64)), "md_hits: dtype"),
    (dict(md_hits=torch.zeros((2, 6), dtype=torch.int32).t()), "md_hits: not contiguous"),
    (dict(md_kappa=torch.zeros(5, dtype=torch.float32)), "md_kappa: 5 elements"),
    (dict(md_kappa=torch.zeros(6, dtype=torch.float64)), "md_kappa: dtype"),
    (dict(md_count=torch.zeros(1, dtype=torch.int32)), "md_count: dtype"),
    (dict(md_count=torch.zeros(0, dtype=torch.int64)), "md_count: empty"),
])
def test_bad_buffer_rejected(kw, what):
    with pytest.raises(ValueError, match=what):
        _call(**kw)


def test_wrong_device_rejected():
    with pytest.raises(ValueError, match="x: on cpu"):
        _call(device=torch.device("cuda", 0))
