"""Helpers shared by the GPU parity tests (test infrastructure, imported by tests only)."""
import numpy as np

import oracle


def canon_order(a):
    return np.lexsort(a.T[::-1]) if len(a) else np.zeros(0, np.int64)


def expected_tc(ref, sel_gpu, og, oe):
    """The oracle's track candidates for the GPU's own selection flags: the duplicate
    removal (oracle_tc_select) run on the oracle's T5s, keys and circle-fit chi2 with the
    flags the GPU produced (rows og of the GPU's T5s match rows oe of the oracle's). A
    selection flip near the working point then changes both sides alike, so the duplicate
    removal is compared exactly on every event."""
    sel = np.zeros(len(ref.t5_score), np.uint8)
    sel[oe] = np.asarray(sel_gpu)[og]
    tc = oracle.tc_select(ref.t5_md, ref.t5_hits(), ref.t5_chi2, sel, len(ref.md_lo))
    return ref.t5_hits()[tc.astype(bool)]


def near_boundary(ref, label=""):
    """Tested candidate pairs with a cut comparison within 1e-5 relative of its bound, per
    step (MD, LS, T3, T5); the parity bar wants them under 1e-4 of all tested pairs. The
    sets compare exactly whatever this count, so it is reported, and the bound asserted."""
    near, pairs = ref.near, ref.pairs
    frac = float(near.sum()) / max(1, int(pairs.sum()))
    print(f"near-boundary {label}: {near.tolist()} of {pairs.tolist()} tested pairs ({frac:.2e})")
    assert frac < 1e-4, (near, pairs)
    return frac
