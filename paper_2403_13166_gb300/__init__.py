"""GB300-native line-segment tracking (LST) hot path: mini-doublets, line segments,
triplets, quintuplets and the quintuplet DNN score, as hand-written sm_103a CUDA
behind a C-ABI library. Submodules load lazily: importing the package does not
load the CUDA library."""
