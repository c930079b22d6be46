// Explicit instantiations of the colour-pass and fused-step kernels:
// 3D, float, n = 2, 3, 4 (split across translation units so
// that they compile in parallel).
#include "smoother_impl.cuh"

SIPG_SMOOTH_INST(3, float, 2)
SIPG_CLAMPED_INST(2)
SIPG_FULL3_INST(2)
SIPG_SMOOTH_INST(3, float, 3)
SIPG_CLAMPED_INST(3)
SIPG_FULL3_INST(3)
SIPG_SMOOTH_INST(3, float, 4)
SIPG_CLAMPED_INST(4)
SIPG_FULL3_INST(4)

cudaError_t launch_barrier_selftest(const sipg_handle* h, int extra, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  unsigned int* bar = reinterpret_cast<unsigned int*>(h->ws + h->off_sync);
  int* status = reinterpret_cast<int*>(h->ws + h->off_sync + 2 * sizeof(unsigned int));
  return cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, bar, status, extra);
}
