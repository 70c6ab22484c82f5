// Consumers of the matvec's partial sums and the block reductions shared by
// the finalize kernels (Algorithm 1's step, the power iteration of Eq. 11,
// the adjoint and the pixel-space form): the per-output-block gather, the
// FP64 block sum, the last-CTA ticket and the fixed-order sum of per-block
// results.  Included by several .cu files; everything has internal linkage.
#pragma once

#include "matvec.cuh"

namespace osar {
namespace {

constexpr int FIN_GROUPS = 8;                  // partial-list splits per block
constexpr int FIN_THREADS = FIN_GROUPS * BLK;  // 1024

// y_K = sum of the segment partials of block column K and the block partials
// of (K, J), J > K, accumulated in Acc (FP32 on the FP32-Gram paths).  The
// partial list is split over FIN_GROUPS thread groups and the group sums are
// combined in a fixed order; a deferred Gram update's term (corr, FP32
// paths) is added last.  Called by every thread; threads < BLK get the sum
// for coefficient threadIdx.x.
template <typename T2, typename Acc>
__device__ __forceinline__ double2 gather_row(const T2* __restrict__ segpart,
                                              const T2* __restrict__ tilepart,
                                              const int* __restrict__ seg_begin,
                                              int nb, int K,
                                              const float2* __restrict__ corr = nullptr) {
  __shared__ Acc red_r[FIN_GROUPS][BLK], red_i[FIN_GROUPS][BLK];
  const int g = threadIdx.x / BLK, i = threadIdx.x % BLK;
  const int s0 = seg_begin[K], nseg = seg_begin[K + 1] - s0;
  const int total = nseg + (nb - 1 - K);
  const int64_t t0 = packed_block(K, K, nb) + 1;  // block (K, K+1)
  Acc yr = 0, yi = 0;
  // q = g, g + FIN_GROUPS, ... over the segment partials, then on over the
  // block partials (two loops: no select in the load stream)
  int q = g;
#pragma unroll 4
  for (; q < nseg; q += FIN_GROUPS) {
    const T2 v = segpart[(int64_t)(s0 + q) * BLK + i];
    yr += (Acc)v.x;
    yi += (Acc)v.y;
  }
#pragma unroll 8
  for (; q < total; q += FIN_GROUPS) {
    const T2 v = tilepart[(t0 + (q - nseg)) * BLK + i];
    yr += (Acc)v.x;
    yi += (Acc)v.y;
  }
  red_r[g][i] = yr;
  red_i[g][i] = yi;
  __syncthreads();
  double2 y = make_double2(0.0, 0.0);
  if (threadIdx.x < BLK) {
    Acc sr = 0, si = 0;
#pragma unroll
    for (int k = 0; k < FIN_GROUPS; ++k) {
      sr += red_r[k][i];
      si += red_i[k][i];
    }
    if (corr) {
      const float2 cv = corr[K * BLK + i];
      sr += (Acc)cv.x;
      si += (Acc)cv.y;
    }
    y = make_double2((double)sr, (double)si);
  }
  return y;
}

// Sum (a, b) over the threads of the block's first nw warps (every other
// thread of the block holds zeros: the total is the block's); thread 0 gets
// the total.  GB300 issues FP64 arithmetic at about 1/64 of its FP32 rate,
// one pipe per SM for all its warps, so the 1024-thread finalizes reduce
// only the 4 warps that hold their block's 128 coefficients: the tree over
// all 32 warps took 5-7 us of a 29 us step finalize.
__device__ __forceinline__ double2 block_sum(double a, double b, int nw) {
  __shared__ double2 red[32];
  __syncthreads();
  const int w = threadIdx.x >> 5;
  if (w < nw) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) red[w] = make_double2(a, b);
  }
  __syncthreads();
  double2 t = make_double2(0, 0);
  if (threadIdx.x == 0) {
    for (int k = 0; k < nw; ++k) {
      t.x += red[k].x;
      t.y += red[k].y;
    }
  }
  return t;
}

// Ticket for the last CTA of a grid: thread 0 fences this CTA's published
// results and takes a ticket; returns true (block-uniform) in the CTA that
// finishes last, which then sees every other CTA's published result.
__device__ __forceinline__ bool last_block(unsigned* counter, unsigned nblocks) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(counter, 1u) == nblocks - 1;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// Sum of the per-block (x, y) partials in a fixed order, by one block.
__device__ __forceinline__ double2 sum_parts(const double2* part, int n) {
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double2 v = __ldcg(part + k);
    a += v.x;
    b += v.y;
  }
  const int used = n < (int)blockDim.x ? n : (int)blockDim.x;
  return block_sum(a, b, (used + 31) >> 5);
}

}  // namespace
}  // namespace osar
