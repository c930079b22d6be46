// Explicit instantiations of the colour-pass and fused-step kernels:
// 2D, double, n = 2, 3, 4 (split across translation units so
// that they compile in parallel).
#include "smoother_impl.cuh"

SIPG_SMOOTH_INST(2, double, 2)
SIPG_SMOOTH_INST(2, double, 3)
SIPG_SMOOTH_INST(2, double, 4)
