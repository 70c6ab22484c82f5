// The packed-Gram matvec kernel and the partial-sum helpers shared by the
// FISTA, power-iteration and adjoint kernels.  Included by several .cu files;
// everything has internal linkage.
//
// Gram storage: the upper 128 x 128 blocks T_IJ = A[I-rows, J-cols], I <= J,
// each stored column-major: entry (r, c) of the block sits at c * 128 + r.
//
// Matvec: y = A x needs, for every stored block,
//     y_I += T_IJ x_J      and, when I < J,      y_J += T_IJ^H x_I.
// Work items ("segments") are runs of blocks I0..I1-1 of one block column J.
// A CTA streams each block once from HBM; each warp owns 16 stored columns c,
// each lane 4 consecutive rows r (one 32-byte sector per column):
//   * y_J[c] = sum_r conj(T[r][c]) x_I[r] accumulates over the whole segment
//     in registers and is reduced across lanes once at the end (segment
//     partial); on a diagonal block (T Hermitian, stored in full) this alone
//     is the block's product;
//   * y_I[r] = sum_c T[r][c] x_J[c] is reduced across the 8 warps through
//     shared memory per off-diagonal block (block partial).
// The consumer (gather_row) sums, per output block K, the segment partials
// of column K and the block partials of (K, J), J > K, which are contiguous
// in the packed order.  No floating-point atomics: results are deterministic.
#pragma once

#include "ctx.h"

namespace osar {
namespace {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using T2 = float2;
};
template <>
struct Vec<double> {
  using T2 = double2;
};

// Four consecutive complex entries of one stored column (streamed once).
__device__ __forceinline__ void load4(const float2* p, float2 (&g)[4]) {
  const float4* q = reinterpret_cast<const float4*>(p);
  float4 a = __ldcs(q), b = __ldcs(q + 1);
  g[0] = make_float2(a.x, a.y);
  g[1] = make_float2(a.z, a.w);
  g[2] = make_float2(b.x, b.y);
  g[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const double2* p, double2 (&g)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) g[c] = __ldcs(p + c);
}

template <typename T>
__global__ void __launch_bounds__(256, 2)
    k_matvec(const typename Vec<T>::T2* __restrict__ G,
             const typename Vec<T>::T2* __restrict__ x,
             typename Vec<T>::T2* __restrict__ segpart,
             typename Vec<T>::T2* __restrict__ tilepart,
             const int4* __restrict__ segs, int nseg, int nb,
             const DevScalars* __restrict__ sc, int gated) {
  using T2 = typename Vec<T>::T2;
  constexpr int RB = sizeof(T) == 4 ? 8 : 4;  // stored columns per load batch
  if (gated && sc->converged) return;
  __shared__ T2 xs[BLK];
  __shared__ T2 red[8][BLK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const int4 sg = segs[s];
    const int J = sg.x;
    __syncthreads();
    if (threadIdx.x < BLK) xs[threadIdx.x] = x[J * BLK + threadIdx.x];
    __syncthreads();
    T br[16], bi[16];  // y_J partials of this warp's 16 columns
#pragma unroll
    for (int c = 0; c < 16; ++c) br[c] = bi[c] = T(0);
    for (int I = sg.y; I < sg.z; ++I) {
      const T2* blk = G + packed_block(I, J, nb) * (int64_t)(BLK * BLK) +
                      (int64_t)(warp * 16) * BLK + lane * 4;
      T2 xi[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) xi[q] = x[I * BLK + lane * 4 + q];
      T ar[4], ai[4];  // y_I partials of this lane's 4 rows
#pragma unroll
      for (int q = 0; q < 4; ++q) ar[q] = ai[q] = T(0);
#pragma unroll
      for (int c0 = 0; c0 < 16; c0 += RB) {
        T2 g[RB][4];
#pragma unroll
        for (int c = 0; c < RB; ++c) load4(blk + (int64_t)(c0 + c) * BLK, g[c]);
#pragma unroll
        for (int c = 0; c < RB; ++c) {
          const T2 xj = xs[warp * 16 + c0 + c];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const T2 e = g[c][q];
            // y_J[c] += conj(e) x_I[r]
            br[c0 + c] = fma(e.x, xi[q].x, br[c0 + c]);
            br[c0 + c] = fma(e.y, xi[q].y, br[c0 + c]);
            bi[c0 + c] = fma(e.x, xi[q].y, bi[c0 + c]);
            bi[c0 + c] = fma(-e.y, xi[q].x, bi[c0 + c]);
            // y_I[r] += e x_J[c]
            ar[q] = fma(e.x, xj.x, ar[q]);
            ar[q] = fma(-e.y, xj.y, ar[q]);
            ai[q] = fma(e.x, xj.y, ai[q]);
            ai[q] = fma(e.y, xj.x, ai[q]);
          }
        }
      }
      if (I != J) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T2 v;
          v.x = ar[q];
          v.y = ai[q];
          red[warp][lane * 4 + q] = v;
        }
        __syncthreads();
        if (threadIdx.x < BLK) {
          T sr = 0, si = 0;
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            sr += red[w][threadIdx.x].x;
            si += red[w][threadIdx.x].y;
          }
          T2 v;
          v.x = sr;
          v.y = si;
          tilepart[packed_block(I, J, nb) * BLK + threadIdx.x] = v;
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      T vr = br[c], vi = bi[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (lane == c) {
        T2 v;
        v.x = vr;
        v.y = vi;
        segpart[(int64_t)sg.w * BLK + warp * 16 + c] = v;
      }
    }
  }
}

constexpr int FIN_GROUPS = 8;                  // partial-list splits per block
constexpr int FIN_THREADS = FIN_GROUPS * BLK;  // 1024

// y_K = sum of the segment partials of block column K and the block partials
// of (K, J), J > K, accumulated in Acc (FP32 on the FP32-Gram paths).  The
// partial list is split over FIN_GROUPS thread groups and the group sums are
// combined in a fixed order.  Called by every thread; threads < BLK get the
// sum for coefficient threadIdx.x.
template <typename T2, typename Acc>
__device__ __forceinline__ double2 gather_row(const T2* __restrict__ segpart,
                                              const T2* __restrict__ tilepart,
                                              const int* __restrict__ seg_begin,
                                              int nb, int K) {
  __shared__ Acc red_r[FIN_GROUPS][BLK], red_i[FIN_GROUPS][BLK];
  const int g = threadIdx.x / BLK, i = threadIdx.x % BLK;
  const int s0 = seg_begin[K], nseg = seg_begin[K + 1] - s0;
  const int total = nseg + (nb - 1 - K);
  const int64_t t0 = packed_block(K, K, nb) + 1;  // block (K, K+1)
  Acc yr = 0, yi = 0;
#pragma unroll 4
  for (int q = g; q < total; q += FIN_GROUPS) {
    const T2 v = q < nseg ? segpart[(int64_t)(s0 + q) * BLK + i]
                          : tilepart[(t0 + (q - nseg)) * BLK + i];
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
    y = make_double2((double)sr, (double)si);
  }
  return y;
}

// Sum (a, b) over all threads of the block; thread 0 gets the total.
__device__ __forceinline__ double2 block_sum(double a, double b) {
  __shared__ double2 red[32];
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(a, b);
  __syncthreads();
  double2 t = make_double2(0, 0);
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t.x += red[w].x;
      t.y += red[w].y;
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
  return block_sum(a, b);
}

}  // namespace
}  // namespace osar
