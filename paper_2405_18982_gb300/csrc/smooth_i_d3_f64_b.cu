// Explicit instantiations of the colour-pass and fused-step kernels:
// 3D, double, n = 5, 6 (split across translation units so
// that they compile in parallel).
#include "smoother_impl.cuh"

SIPG_SMOOTH_INST(3, double, 5)
SIPG_SMOOTH_INST(3, double, 6)
