"""GB300 (sm_103a) CUDA library for multidimensional included and excluded sums."""
