// Complex soft thresholding of Algorithm 1, S_alpha(u) = u max(0, 1 -
// alpha / |u|), as the factor that multiplies u, shared by the stored-Gram
// step (k_fista.cu) and the pixel-space Gram form (k_pixgram.cu).
#pragma once

namespace osar {
namespace {

// Shrink factor max(0, 1 - alpha/|u|) from |u|^2, in FP64 on every path: near
// the threshold 1 - alpha/|u| cancels, and an FP32 factor would leave a small
// surviving coefficient with a large relative error.  It costs one FP64
// square root and division per coefficient and step (the step's partial sums
// stay in the matvec's precision).  The template parameter is the matvec's
// working type and no longer changes the arithmetic.
template <typename T2>
__device__ __forceinline__ double shrink_keep(double mag2, double alpha) {
  const double mag = sqrt(mag2);
  return mag > alpha ? 1.0 - alpha / mag : 0.0;
}

}  // namespace
}  // namespace osar
