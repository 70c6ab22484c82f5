// SIMT complex GEMMs for the FP64 (plain) and FP32 paths.
//
//  dictionary apply (Eq. 6):  A[j][m] = sum_p H^T[j][p] F[m][p]
//  Gram update (Eqs. 12-13):  G[i][j] += sum_m conj(A[i][m]) A[j][m]
//
// Both operands are stored K-contiguous ("row i holds the K values of
// operand row i"), so one kernel serves both.  A CTA computes a 64 x 64
// complex tile with 256 threads, each owning a 4 x 4 register tile at a
// 16-element stride, with 16-deep k chunks staged through shared memory.
// The Gram variant accumulates into the packed upper-triangular 128 x 128
// blocks, which are stored column-major (entry (r, c) at c * 128 + r).
#include "ctx.h"

namespace osar {
namespace {

constexpr int ST = 64;   // output tile edge
constexpr int SK = 16;   // k chunk

template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using T2 = double2;
};
template <>
struct Cx<float> {
  using T2 = float2;
};

template <typename T, bool CONJ_A, bool PACKED>
__global__ void __launch_bounds__(256)
    k_cgemm_tn(const typename Cx<T>::T2* __restrict__ P, int ldp,
               const typename Cx<T>::T2* __restrict__ Q, int ldq, int kdim,
               typename Cx<T>::T2* __restrict__ C, int ldc,
               const int4* __restrict__ blocks) {
  using T2 = typename Cx<T>::T2;
  __shared__ T2 As[SK][ST + 1];
  __shared__ T2 Bs[SK][ST + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  int row0, col0;
  T2* out;
  int ldo;
  if (PACKED) {
    int4 blk = blocks[blockIdx.x];  // (row block, column block, packed block)
    int sub = blockIdx.y;  // 4 sub-tiles per 128 x 128 block
    row0 = blk.x * BLK + (sub >> 1) * ST;
    col0 = blk.y * BLK + (sub & 1) * ST;
    // column-major block: entry (r, c) at c * BLK + r
    out = C + (int64_t)blk.z * (BLK * BLK) +
          (int64_t)((sub & 1) * ST) * BLK + (sub >> 1) * ST;
    ldo = BLK;
  } else {
    row0 = blockIdx.x * ST;
    col0 = blockIdx.y * ST;
    out = C + (int64_t)row0 * ldc + col0;
    ldo = ldc;
  }

  T accr[4][4], acci[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) accr[a][b] = acci[a][b] = T(0);

  const int lr = tid >> 2;        // 0..63 operand row of the tile
  const int lk = (tid & 3) * 4;   // 0, 4, 8, 12
  for (int k0 = 0; k0 < kdim; k0 += SK) {
    const T2* pa = P + (int64_t)(row0 + lr) * ldp + k0 + lk;
    const T2* pb = Q + (int64_t)(col0 + lr) * ldq + k0 + lk;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[lk + q][lr] = pa[q];
      Bs[lk + q][lr] = pb[q];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SK; ++k) {
      T2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T ar = av[a].x, ai = CONJ_A ? -av[a].y : av[a].y;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          accr[a][b] = fma(ar, bv[b].x, accr[a][b]);
          accr[a][b] = fma(-ai, bv[b].y, accr[a][b]);
          acci[a][b] = fma(ar, bv[b].y, acci[a][b]);
          acci[a][b] = fma(ai, bv[b].x, acci[a][b]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      T2* dst = PACKED ? out + (int64_t)(tx + 16 * b) * ldo + ty + 16 * a
                       : out + (int64_t)(ty + 16 * a) * ldo + tx + 16 * b;
      if (PACKED) {
        T2 g = *dst;
        g.x += accr[a][b];
        g.y += acci[a][b];
        *dst = g;
      } else {
        T2 g;
        g.x = accr[a][b];
        g.y = acci[a][b];
        *dst = g;
      }
    }
}

}  // namespace

cudaError_t launch_dict_simt(osar_ctx* ctx) {
  ProfEvent ev;
  prof_begin(ctx, KCL_DICT, &ev);
  dim3 grid(ctx->Mp / ST, ctx->Kp / ST);
  if (ctx->prec == OSAR_FP64)
    k_cgemm_tn<double, false, false><<<grid, 256, 0, ctx->stream>>>(
        (const double2*)ctx->D, ctx->Np, (const double2*)ctx->F, ctx->Np,
        ctx->Np, (double2*)ctx->A, ctx->Kp, nullptr);
  else
    k_cgemm_tn<float, false, false><<<grid, 256, 0, ctx->stream>>>(
        (const float2*)ctx->D, ctx->Np, (const float2*)ctx->F, ctx->Np,
        ctx->Np, (float2*)ctx->A, ctx->Kp, nullptr);
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_gram_simt(osar_ctx* ctx) {
  ProfEvent ev;
  prof_begin(ctx, KCL_GRAM, &ev);
  dim3 grid((unsigned)ctx->nblk, 4);
  if (ctx->prec == OSAR_FP64)
    k_cgemm_tn<double, true, true><<<grid, 256, 0, ctx->stream>>>(
        (const double2*)ctx->A, ctx->Kp, (const double2*)ctx->A, ctx->Kp,
        ctx->Kp, (double2*)ctx->g_hi, 0, ctx->gram_tiles);
  else
    k_cgemm_tn<float, true, true><<<grid, 256, 0, ctx->stream>>>(
        (const float2*)ctx->A, ctx->Kp, (const float2*)ctx->A, ctx->Kp,
        ctx->Kp, (float2*)ctx->g_hi, 0, ctx->gram_tiles);
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_gram_simt_tiles(cudaStream_t st, int prec, const void* A,
                                   int kp, void* g_hi, const int4* tiles,
                                   int n_tiles) {
  if (n_tiles <= 0) return cudaSuccess;
  dim3 grid((unsigned)n_tiles, 4);
  if (prec == OSAR_FP64)
    k_cgemm_tn<double, true, true><<<grid, 256, 0, st>>>(
        (const double2*)A, kp, (const double2*)A, kp, kp, (double2*)g_hi, 0,
        tiles);
  else
    k_cgemm_tn<float, true, true><<<grid, 256, 0, st>>>(
        (const float2*)A, kp, (const float2*)A, kp, kp, (float2*)g_hi, 0,
        tiles);
  return cudaGetLastError();
}

}  // namespace osar
