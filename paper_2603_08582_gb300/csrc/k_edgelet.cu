// Forward block for the binary edgelet dictionary (§III-A, Eq. 6).
//
// H is binary, so A_s = F_s H needs no GEMM: the row of atom m is the sum of
// the phase rows F_s[:, p] over the atom's pixels p (at most 64 of them).
// The phases are formed pixel-major (row p holds F_s[k, p] for k = 0 .. Kp-1,
// in FP32 for the split-BF16 and FP32 paths, FP64 on the plain path) by the
// phase kernel; here each thread takes one atom and eight consecutive
// frequencies, adds the atom's pixel rows with 16- or 32-byte loads, and
// writes the atom-major block: six bf16 planes (re, im, -re) x (hi, lo) for
// the tensor-core Gram update, or complex words for the SIMT paths.  Every
// sum runs in pixel-list order, so results do not depend on the grid.
#include "ctx.h"

namespace osar {
namespace {

__device__ __forceinline__ void split_bf16_pair(float x, __nv_bfloat16& hi,
                                                __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// A (split planes) from FP32 pixel-major phases.
__global__ void k_edgelet_planes(const float2* __restrict__ f, int Kp,
                                 const int* __restrict__ atom_ptr,
                                 const int* __restrict__ atom_pix, int M, int Mp,
                                 __nv_bfloat16* __restrict__ planes) {
  const int groups = Kp / 8;
  const int64_t plane = (int64_t)Mp * Kp;
  for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       gid < (int64_t)Mp * groups; gid += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(gid / groups);
    const int k0 = (int)(gid - (int64_t)m * groups) * 8;
    float re[8], im[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) re[q] = im[q] = 0.f;
    if (m < M) {
      for (int t = atom_ptr[m]; t < atom_ptr[m + 1]; ++t) {
        const float4* row =
            reinterpret_cast<const float4*>(f + (int64_t)atom_pix[t] * Kp + k0);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float4 v = row[h];
          re[2 * h] += v.x;
          im[2 * h] += v.y;
          re[2 * h + 1] += v.z;
          im[2 * h + 1] += v.w;
        }
      }
    }
    __align__(16) __nv_bfloat16 v[6][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      split_bf16_pair(re[q], v[0][q], v[3][q]);
      split_bf16_pair(im[q], v[1][q], v[4][q]);
      split_bf16_pair(-re[q], v[2][q], v[5][q]);
    }
    const int64_t off = (int64_t)m * Kp + k0;
#pragma unroll
    for (int pl = 0; pl < 6; ++pl)
      *reinterpret_cast<uint4*>(planes + pl * plane + off) =
          *reinterpret_cast<const uint4*>(v[pl]);
  }
}

// A (complex, atom-major) from pixel-major phases of the same type.
template <typename T2>
__global__ void k_edgelet_complex(const T2* __restrict__ f, int Kp,
                                  const int* __restrict__ atom_ptr,
                                  const int* __restrict__ atom_pix, int M, int Mp,
                                  T2* __restrict__ a) {
  for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       gid < (int64_t)Mp * Kp; gid += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(gid / Kp);
    const int k = (int)(gid - (int64_t)m * Kp);
    T2 s;
    s.x = 0;
    s.y = 0;
    if (m < M)
      for (int t = atom_ptr[m]; t < atom_ptr[m + 1]; ++t) {
        const T2 v = f[(int64_t)atom_pix[t] * Kp + k];
        s.x += v.x;
        s.y += v.y;
      }
    a[gid] = s;
  }
}

// rho_p = sum over the nonzero coefficients q of [p in atom idx_q] val_q
// (the image H c of a sparse c), in coefficient order, FP64.
__global__ void k_sim_rho_edgelet(int Np, int nnz, const int* __restrict__ idx,
                                  const double2* __restrict__ val,
                                  const int* __restrict__ atom_ptr,
                                  const int* __restrict__ atom_pix, double2* rho) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Np) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int q = 0; q < nnz; ++q) {
    const int m = idx[q];
    for (int t = atom_ptr[m]; t < atom_ptr[m + 1]; ++t)
      if (atom_pix[t] == p) {
        acc.x += val[q].x;
        acc.y += val[q].y;
      }
  }
  rho[p] = acc;
}

unsigned grid_for(int64_t n, int t, int grid_cap) {
  int64_t g = (n + t - 1) / t;
  if (grid_cap > 0 && g > 4 * (int64_t)grid_cap) g = 4 * (int64_t)grid_cap;
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_edgelet(osar_ctx* ctx, int grid_cap) {
  ProfEvent ev;
  prof_begin(ctx, KCL_DICT, &ev);
  if (ctx->prec == OSAR_SPLIT_BF16) {
    const int64_t n = (int64_t)ctx->Mp * (ctx->Kp / 8);
    k_edgelet_planes<<<grid_for(n, 256, grid_cap), 256, 0, ctx->stream>>>(
        (const float2*)ctx->F, ctx->Kp, ctx->atom_ptr, ctx->atom_pix, ctx->M,
        ctx->Mp, ctx->Apl);
  } else if (ctx->prec == OSAR_FP64) {
    const int64_t n = (int64_t)ctx->Mp * ctx->Kp;
    k_edgelet_complex<double2><<<grid_for(n, 256, grid_cap), 256, 0, ctx->stream>>>(
        (const double2*)ctx->F, ctx->Kp, ctx->atom_ptr, ctx->atom_pix, ctx->M,
        ctx->Mp, (double2*)ctx->A);
  } else {
    const int64_t n = (int64_t)ctx->Mp * ctx->Kp;
    k_edgelet_complex<float2><<<grid_for(n, 256, grid_cap), 256, 0, ctx->stream>>>(
        (const float2*)ctx->F, ctx->Kp, ctx->atom_ptr, ctx->atom_pix, ctx->M,
        ctx->Mp, (float2*)ctx->A);
  }
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_sim_rho_edgelet(osar_ctx* ctx, int nnz) {
  k_sim_rho_edgelet<<<(unsigned)((ctx->Np + 255) / 256), 256, 0, ctx->stream>>>(
      ctx->Np, nnz, ctx->sim_idx, ctx->sim_nz, ctx->atom_ptr, ctx->atom_pix,
      ctx->sim_rho);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace osar
