// Explicit instantiations of the colour-pass and fused-step kernels:
// 2D, double, n = 7, 8 (split across translation units so
// that they compile in parallel).
#include "smoother_impl.cuh"

SIPG_SMOOTH_INST(2, double, 7)
SIPG_SMOOTH_INST(2, double, 8)
