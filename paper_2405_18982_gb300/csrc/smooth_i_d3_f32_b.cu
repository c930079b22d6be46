// Explicit instantiations of the colour-pass and fused-step kernels:
// 3D, float, n = 5, 6 (split across translation units so
// that they compile in parallel).
#include "smoother_impl.cuh"

SIPG_SMOOTH_INST(3, float, 5)
SIPG_CLAMPED_INST(5)
SIPG_FULL3_INST(5)
SIPG_SMOOTH_INST(3, float, 6)
SIPG_CLAMPED_INST(6)
SIPG_FULL3_INST(6)
