// Public launchers of the smoother (declared in sipg_internal.cuh): dispatch
// on dimension and degree to the instantiations in smooth_i_*.cu.
#include "sipg_internal.cuh"

template <int DIM, typename T, int NN>
cudaError_t smooth_colour_n(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s);
template <int DIM, typename T, int NN>
cudaError_t smooth_step_n(const sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s);
template <int NN>
cudaError_t clamped_colour3_n(const sipg_handle* h, int level, int colour, const float* b, float* x,
                              cudaStream_t s);

namespace {

template <int DIM, typename T>
cudaError_t colour_dim(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s) {
  switch (h->n) {
    case 2: return smooth_colour_n<DIM, T, 2>(h, level, colour, b, x, s);
    case 3: return smooth_colour_n<DIM, T, 3>(h, level, colour, b, x, s);
    case 4: return smooth_colour_n<DIM, T, 4>(h, level, colour, b, x, s);
    case 5: return smooth_colour_n<DIM, T, 5>(h, level, colour, b, x, s);
    case 6: return smooth_colour_n<DIM, T, 6>(h, level, colour, b, x, s);
    case 7: return smooth_colour_n<DIM, T, 7>(h, level, colour, b, x, s);
    case 8: return smooth_colour_n<DIM, T, 8>(h, level, colour, b, x, s);
  }
  return cudaErrorInvalidValue;
}

template <int DIM, typename T>
cudaError_t step_dim(const sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s) {
  switch (h->n) {
    case 2: return smooth_step_n<DIM, T, 2>(h, level, reverse, b, x, s);
    case 3: return smooth_step_n<DIM, T, 3>(h, level, reverse, b, x, s);
    case 4: return smooth_step_n<DIM, T, 4>(h, level, reverse, b, x, s);
    case 5: return smooth_step_n<DIM, T, 5>(h, level, reverse, b, x, s);
    case 6: return smooth_step_n<DIM, T, 6>(h, level, reverse, b, x, s);
    case 7: return smooth_step_n<DIM, T, 7>(h, level, reverse, b, x, s);
    case 8: return smooth_step_n<DIM, T, 8>(h, level, reverse, b, x, s);
  }
  return cudaErrorInvalidValue;
}

// The clamped kernel's fused colour pass (3D FP32); cudaErrorNotSupported
// elsewhere (the caller then runs the residual-per-colour path).
template <typename T>
cudaError_t clamped_fused(const sipg_handle* h, int level, int colour, const T* b, T* x, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (h->prm.dim != 3) return cudaErrorNotSupported;
    switch (h->n) {
      case 3: return clamped_colour3_n<3>(h, level, colour, b, x, s);
      case 4: return clamped_colour3_n<4>(h, level, colour, b, x, s);
      case 5: return clamped_colour3_n<5>(h, level, colour, b, x, s);
      case 6: return clamped_colour3_n<6>(h, level, colour, b, x, s);
      case 7: return clamped_colour3_n<7>(h, level, colour, b, x, s);
      case 8: return clamped_colour3_n<8>(h, level, colour, b, x, s);
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace

// Kernels one colour pass launches: one for the interior patches and one for
// the patches on the domain boundary, where the colour has any (the patch
// enumeration of make_grid: per direction m in [0, cnt), interior box
// [lo, hi)).
int colour_kernels(int dim, int N, int colour) {
  long long tot = 1, inner = 1;
  for (int e = 0; e < dim; ++e) {
    const int par = (colour >> e) & 1;
    const int cnt = par ? N / 2 : N / 2 - 1;
    const int lo = par ? 1 : 0;
    int hi = N / 2 - 1;
    if (hi < lo) hi = lo;
    tot *= cnt > 0 ? cnt : 0;
    inner *= hi - lo;
  }
  if (tot <= 0) return 0;
  return (inner > 0 ? 1 : 0) + (tot - inner > 0 ? 1 : 0);
}

template <typename T>
cudaError_t launch_smooth_colour(const sipg_handle* h, int level, int colour, const T* b, T* x,
                                 cudaStream_t s) {
  if (h->prm.smoother == SIPG_SMOOTHER_CLAMPED) {
    const cudaError_t e = clamped_fused<T>(h, level, colour, b, x, s);
    if (e != cudaErrorNotSupported) return e;
  }
  if (h->prm.smoother == SIPG_SMOOTHER_FULL || h->prm.smoother == SIPG_SMOOTHER_CLAMPED) {
    int nl = 0;
    return launch_full_colour<T>(h, level, colour, b, x, s, &nl);
  }
  return h->prm.dim == 2 ? colour_dim<2, T>(h, level, colour, b, x, s) : colour_dim<3, T>(h, level, colour, b, x, s);
}
template cudaError_t launch_smooth_colour<double>(const sipg_handle*, int, int, const double*, double*,
                                                  cudaStream_t);
template cudaError_t launch_smooth_colour<float>(const sipg_handle*, int, int, const float*, float*,
                                                 cudaStream_t);

template <typename T>
cudaError_t launch_smooth_step(const sipg_handle* h, int level, int reverse, const T* b, T* x, cudaStream_t s,
                               int* launches) {
  const int nc = 1 << h->prm.dim;
  if (h->prm.smoother == SIPG_SMOOTHER_FULL || h->prm.smoother == SIPG_SMOOTHER_CLAMPED) {
    *launches = 0;
    for (int i = 0; i < nc; ++i) {
      const int c = reverse ? nc - 1 - i : i;
      int nl = colour_kernels(h->prm.dim, h->lv[level].N, c);
      cudaError_t e = cudaErrorNotSupported;
      if (h->prm.smoother == SIPG_SMOOTHER_CLAMPED) e = clamped_fused<T>(h, level, c, b, x, s);
      if (e == cudaErrorNotSupported) e = launch_full_colour<T>(h, level, c, b, x, s, &nl);
      *launches += nl;
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (h->fuse_small_levels && h->tuned_path(sizeof(T) == 4 ? 1 : 0, level) != 1) {
    cudaError_t e = h->prm.dim == 2 ? step_dim<2, T>(h, level, reverse, b, x, s)
                                    : step_dim<3, T>(h, level, reverse, b, x, s);
    if (e == cudaSuccess) {
      *launches = 1;
      return cudaSuccess;
    }
    if (e != cudaErrorNotSupported) return e;
  }
  *launches = 0;
  for (int i = 0; i < nc; ++i) {
    const int c = reverse ? nc - 1 - i : i;
    cudaError_t e = launch_smooth_colour<T>(h, level, c, b, x, s);
    if (e != cudaSuccess) return e;
    *launches += colour_kernels(h->prm.dim, h->lv[level].N, c);
  }
  return cudaSuccess;
}
template cudaError_t launch_smooth_step<double>(const sipg_handle*, int, int, const double*, double*, cudaStream_t,
                                                int*);
template cudaError_t launch_smooth_step<float>(const sipg_handle*, int, int, const float*, float*, cudaStream_t,
                                               int*);
