"""CPU oracle of the LST hot path (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may import
this package. It never calls, and is never called by, the CUDA library; both read the
same inputs (detector module table, module map, hits, cut parameters, network
weights).

Parity status per function (pins live in tests/test_oracle_*.py):
  oracle_md_cut / oracle_ls_cut / oracle_t3_cut / oracle_t5_cut  pinned: closed-form
      helices (pT threshold scans, straight lines, charge sign), brute force on tiny events,
      truth-matched efficiency on isolated muons.
  oracle_t5_features  pinned: analytic helix quantities (pT, R, eta, phi, layer) of
      noiseless tracks.
  oracle_mlp          pinned: hand-solvable networks (zero weights, single paths,
      asymmetric weights that detect a transposed operand), sigmoid identities.
  oracle_t5_chi2      pinned: exact circles of any radius give ~0, one displaced anchor gives the
      linearised least-squares value (leverage from an FP64 hat matrix), invariance under
      rotation/translation, and the chi-square law with 2 degrees of freedom on
      single-particle quintuplets of smeared events.
  oracle_tc_select    pinned: hand-built T5 sets (3 shared MDs vs 2, one-pass semantics on
      a chain of three, ties, NaN chi2, unselected T5s), index == brute force, the kept set
      holds no duplicates, one track candidate per isolated muon.
"""
from .oracle import (OracleResult, build_oracle, md_cut, ls_cut, t3_cut, t5_cut, t5_chi2,
                     tc_select, t5_features, mlp_forward, pixel_match, run_event)

__all__ = ["OracleResult", "build_oracle", "md_cut", "ls_cut", "t3_cut", "t5_cut", "t5_chi2",
           "tc_select", "t5_features", "mlp_forward", "pixel_match", "run_event"]
