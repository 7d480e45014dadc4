"""GB300 (sm_103a) implementation of the Hermite 6th-order direct N-body hot
path with block time steps: prediction, pairwise acceleration/jerk/snap/
potential evaluation, j-split reduction, correction and time stepping, in
FP64, float-float ("EX") and FP32-with-split-coordinates precisions."""
