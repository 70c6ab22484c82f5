// Deferred Gram update: the pending block's term of a Gram pass.
//
// With defer_gram the Gram update G_n = G_{n-1} + A_n^H A_n runs on the side
// stream while the power steps and FISTA steps of pulse n read G_{n-1}.  Each
// of their passes adds A_n^H (A_n x), which the two kernels here form from
// the pulse's forward block, kept as split-BF16 planes (hi + lo of the FP32
// dictionary product, atom-major: plane p, atom m, frequency k at
// p * Mp * Kp + m * Kp + k; planes 0 / 1 hold the real / imaginary hi parts,
// 3 / 4 the lo parts).  The matvec's finalize adds the result to the
// partial sums of the G_{n-1} pass, so that y = G_{n-1} x + A_n^H A_n x,
// which is G_n x (Eq. 12: G_n = G_{n-1} + A_n^H A_n) evaluated in another
// order.  Each kernel reads the block once (two planes of each part: 8 bytes
// per entry, Mp x Kp entries, in 16-byte loads) and runs its sums in a fixed
// order; Kp <= 2048.
#include "ctx.h"
#include "finalize.cuh"

namespace osar {
namespace {

constexpr int CORR_THREADS = 256;
constexpr int CORR_MAX_KP = 2048;  // frequencies (8 per thread and row)

// Eight consecutive entries (re, im) of one atom row: hi + lo of each part,
// in FP32, from four 16-byte loads.
__device__ __forceinline__ void row8(const __nv_bfloat16* __restrict__ pl,
                                     int64_t plane, int64_t off, float (&re)[8],
                                     float (&im)[8]) {
  const uint4 rh = *reinterpret_cast<const uint4*>(pl + off);
  const uint4 ih = *reinterpret_cast<const uint4*>(pl + plane + off);
  const uint4 rl = *reinterpret_cast<const uint4*>(pl + 3 * plane + off);
  const uint4 il = *reinterpret_cast<const uint4*>(pl + 4 * plane + off);
  const __nv_bfloat16* a = reinterpret_cast<const __nv_bfloat16*>(&rh);
  const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&ih);
  const __nv_bfloat16* c = reinterpret_cast<const __nv_bfloat16*>(&rl);
  const __nv_bfloat16* d = reinterpret_cast<const __nv_bfloat16*>(&il);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    re[q] = __bfloat162float(a[q]) + __bfloat162float(c[q]);
    im[q] = __bfloat162float(b[q]) + __bfloat162float(d[q]);
  }
}

// u = A x over frequencies k: CTA K sums the atoms of block K, thread
// (g, j) frequencies 8j..8j+7 over rows g, g + RG, ...; the RG row groups
// are added in order, then the last CTA adds the nb block partials in
// block order into u.
__global__ void __launch_bounds__(CORR_THREADS)
    k_corr_u(const __nv_bfloat16* __restrict__ pl, int Mp, int Kp,
             const float2* __restrict__ x, float2* __restrict__ part,
             float2* __restrict__ u, unsigned* __restrict__ tick,
             const int32_t* __restrict__ gate) {
  if (gate && *gate) return;  // the solution has met the stop rule
  const int K = blockIdx.x, nb = gridDim.x;
  const int64_t plane = (int64_t)Mp * Kp;
  const int tk = Kp / 8, rg = CORR_THREADS / tk;  // threads per row, row groups
  __shared__ float2 xs[BLK];
  __shared__ float2 red[CORR_MAX_KP];
  if (threadIdx.x < BLK) xs[threadIdx.x] = x[K * BLK + threadIdx.x];
  __syncthreads();
  const int g = threadIdx.x / tk, j = threadIdx.x % tk;
  float ur[8], ui[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) ur[q] = ui[q] = 0.f;
  if (g < rg) {
#pragma unroll 4
    for (int r = g; r < BLK; r += rg) {
      float re[8], im[8];
      row8(pl, plane, (int64_t)(K * BLK + r) * Kp + 8 * j, re, im);
      const float2 xv = xs[r];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        ur[q] = fmaf(re[q], xv.x, ur[q]);
        ur[q] = fmaf(-im[q], xv.y, ur[q]);
        ui[q] = fmaf(re[q], xv.y, ui[q]);
        ui[q] = fmaf(im[q], xv.x, ui[q]);
      }
    }
  }
  // row groups in order: group 0 writes, then 1, 2, ... add
  for (int h = 0; h < rg; ++h) {
    if (g == h) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float2 v = make_float2(ur[q], ui[q]);
        if (h > 0) {
          const float2 o = red[8 * j + q];
          v = make_float2(o.x + v.x, o.y + v.y);
        }
        red[8 * j + q] = v;
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < Kp; k += CORR_THREADS)
    part[(int64_t)K * Kp + k] = red[k];
  if (!last_block(tick, nb)) return;
  for (int k = threadIdx.x; k < Kp; k += CORR_THREADS) {
    float sr = 0.f, si = 0.f;
    for (int b = 0; b < nb; ++b) {
      const float2 v = part[(int64_t)b * Kp + k];
      sr += v.x;
      si += v.y;
    }
    u[k] = make_float2(sr, si);
  }
  if (threadIdx.x == 0) *tick = 0;
}

// corr_m = sum_k conj(A[k, m]) u_k: one warp per atom, lane l frequencies
// 8l..8l+7, 8(l + 32).., the lane sums combined by a fixed shuffle tree.
__global__ void __launch_bounds__(CORR_THREADS)
    k_corr_y(const __nv_bfloat16* __restrict__ pl, int Mp, int Kp,
             const float2* __restrict__ u, float2* __restrict__ corr,
             const int32_t* __restrict__ gate) {
  if (gate && *gate) return;
  __shared__ float2 us[CORR_MAX_KP];
  for (int k = threadIdx.x; k < Kp; k += CORR_THREADS) us[k] = u[k];
  __syncthreads();
  const int64_t plane = (int64_t)Mp * Kp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int WARPS = CORR_THREADS / 32;
  for (int r = warp; r < BLK; r += WARPS) {
    const int m = blockIdx.x * BLK + r;
    float yr = 0.f, yi = 0.f;
    for (int k0 = 8 * lane; k0 < Kp; k0 += 256) {
      float re[8], im[8];
      row8(pl, plane, (int64_t)m * Kp + k0, re, im);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 uv = us[k0 + q];
        // conj(a) u = (a.re u.re + a.im u.im, a.re u.im - a.im u.re)
        yr = fmaf(re[q], uv.x, yr);
        yr = fmaf(im[q], uv.y, yr);
        yi = fmaf(re[q], uv.y, yi);
        yi = fmaf(-im[q], uv.x, yi);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      yr += __shfl_xor_sync(0xffffffffu, yr, o);
      yi += __shfl_xor_sync(0xffffffffu, yi, o);
    }
    if (lane == 0) corr[m] = make_float2(yr, yi);
  }
}

}  // namespace

const float2* corr_set(const osar_ctx* ctx, int set) {
  return ctx->gram_pending ? ctx->corr + (int64_t)set * ctx->Mp : nullptr;
}

cudaError_t launch_corr(osar_ctx* ctx, const void* xt, int set,
                        const int32_t* gate) {
  if (!ctx->gram_pending) return cudaSuccess;
  const unsigned nb = (unsigned)ctx->nb;
  float2* u = ctx->corr_u + (int64_t)ctx->nb * ctx->Kp;
  ProfEvent ev;
  prof_begin(ctx, KCL_CORR, &ev);
  k_corr_u<<<nb, CORR_THREADS, 0, ctx->stream>>>(
      ctx->Apl, ctx->Mp, ctx->Kp, (const float2*)xt, ctx->corr_u, u,
      ctx->corr_tick, gate);
  k_corr_y<<<nb, CORR_THREADS, 0, ctx->stream>>>(
      ctx->Apl, ctx->Mp, ctx->Kp, u, ctx->corr + (int64_t)set * ctx->Mp, gate);
  prof_end(ctx, &ev);
  ctx->launches += 2;
  return cudaGetLastError();
}

}  // namespace osar
