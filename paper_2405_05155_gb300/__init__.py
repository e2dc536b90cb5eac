"""GB300 (sm_103a) implementation of the truncated-kernel SPH hot path of arXiv 2405.05155."""
