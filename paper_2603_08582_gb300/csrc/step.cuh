// Complex soft thresholding of Algorithm 1, S_alpha(u) = u max(0, 1 -
// alpha / |u|), as the factor that multiplies u, shared by the stored-Gram
// step (k_fista.cu) and the pixel-space Gram form (k_pixgram.cu).
#pragma once

namespace osar {
namespace {

// Shrink factor max(0, 1 - alpha/|u|) from |u|^2: FP64 on the FP64 path; on
// the FP32-Gram paths (whose matvec is FP32 anyway) an FP32 reciprocal
// square root, since GB300's FP64 pipes are ~1/64 of its FP32 rate.
template <typename T2>
__device__ __forceinline__ double shrink_keep(double mag2, double alpha);
template <>
__device__ __forceinline__ double shrink_keep<double2>(double mag2, double alpha) {
  const double mag = sqrt(mag2);
  return mag > alpha ? 1.0 - alpha / mag : 0.0;
}
template <>
__device__ __forceinline__ double shrink_keep<float2>(double mag2, double alpha) {
  if (!(mag2 > alpha * alpha)) return 0.0;
  return (double)(1.0f - (float)alpha * rsqrtf((float)mag2));
}

}  // namespace
}  // namespace osar
