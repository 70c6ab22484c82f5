// Complex soft thresholding of Algorithm 1, S_alpha(u) = u max(0, 1 -
// alpha / |u|), as the factor that multiplies u, shared by the stored-Gram
// step (k_fista.cu) and the pixel-space Gram form (k_pixgram.cu).
#pragma once

namespace osar {
namespace {

// Shrink factor max(0, 1 - alpha/|u|) from |u|^2, to FP64 accuracy on every
// path: near the threshold 1 - alpha/|u| cancels, so a factor with an FP32
// error would leave a small surviving coefficient with a large relative
// error.  The zero / non-zero decision is |u|^2 > alpha^2 in FP64.  The FP64
// path takes a square root and a division.  The FP32-Gram paths avoid the
// long FP64 division and square-root sequences on a part whose FP64 rate is
// ~1/64 of its FP32 rate: 1/|u| starts from the FP32 reciprocal square root
// (relative error below 2^-22) and takes one Newton-Raphson step for
// y = 1/sqrt(x), y' = y (3 - x y^2) / 2, in FP64, which squares the relative
// error (below 2^-43); magnitudes outside FP32's normal range take the
// square root and division instead.
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
  if (!(mag2 > 1e-36 && mag2 < 1e36)) return 1.0 - alpha / sqrt(mag2);
  const double y0 = (double)rsqrtf((float)mag2);
  const double y1 = y0 * (1.5 - 0.5 * mag2 * y0 * y0);
  return fmax(0.0, 1.0 - alpha * y1);
}

}  // namespace
}  // namespace osar
