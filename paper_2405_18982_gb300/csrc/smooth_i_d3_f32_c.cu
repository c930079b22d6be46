// Explicit instantiations of the colour-pass and fused-step kernels:
// 3D, float, n = 7, 8 (split across translation units so
// that they compile in parallel).
#include "smoother_impl.cuh"

SIPG_SMOOTH_INST(3, float, 7)
SIPG_CLAMPED_INST(7)
SIPG_FULL3_INST(7)
SIPG_SMOOTH_INST(3, float, 8)
SIPG_CLAMPED_INST(8)
SIPG_FULL3_INST(8)
