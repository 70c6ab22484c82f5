// Batched kernels for the batching form: every launch covers all scenes
// through (scene, work item) lists; per-scene constants come from SceneDesc
// and per-scene scalars from one DevScalars per scene.  The arithmetic of
// each step is that of the single-scene kernels (Eqs. 2-4, 12-13, Eq. 11,
// Algorithm 1); only the indexing differs.  A scene whose `active` flag is
// clear (no pulse in the last push) is skipped by every kernel.
#include "batch.h"
#include "finalize.cuh"
#include "step.cuh"

namespace osar {
namespace {

constexpr double TWO64 = 18446744073709551616.0;

__device__ __forceinline__ uint64_t frac_q64(double t) {
  return __double2ull_rz(ldexp(t, 63)) << 1;
}

__global__ void k_b_turns(const SceneDesc* __restrict__ desc,
                          const int* __restrict__ row_scene,
                          const double* __restrict__ gam, int rows,
                          ulonglong2* __restrict__ turns) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int s = row_scene[r];
  const SceneDesc& d = desc[s];
  const int p = r - d.row;
  if (!d.active || p >= d.M) {
    turns[r] = make_ulonglong2(0, 0);
    return;
  }
  const int i = p / d.nx, j = p - (p / d.nx) * d.nx;
  const double x = ((double)j - d.cx_half) * d.pixel_m;
  const double y = ((double)i - d.cy_half) * d.pixel_m;
  const double dx = gam[3 * s] - x, dy = gam[3 * s + 1] - y, dz = gam[3 * s + 2];
  const double rr = sqrt(dx * dx + dy * dy + dz * dz);  // Eq. 3
  double a = d.two_flo_c * rr, e = d.two_df_c * rr;
  a -= floor(a);
  e -= floor(e);
  turns[r] = make_ulonglong2(frac_q64(a), frac_q64(e));
}

__device__ __forceinline__ float2 phase_f32(uint64_t turn) {
  const float x = (float)(int)(turn >> 32) * 2.3283064365386963e-10f;
  float s, c;
  sincospif(2.0f * x, &s, &c);
  return make_float2(c, -s);
}
__device__ __forceinline__ double2 phase_f64(uint64_t turn) {
  const double x = (double)(long long)turn * (1.0 / TWO64);
  double s, c;
  sincospi(2.0 * x, &s, &c);
  return make_double2(c, -s);
}

// Stacked pixel-major forward blocks: split-BF16 planes.
__global__ void k_b_phase_planes(const SceneDesc* __restrict__ desc,
                                 const int* __restrict__ row_scene,
                                 const ulonglong2* __restrict__ turns, int rows,
                                 int Kp, __nv_bfloat16* __restrict__ planes) {
  const int groups = Kp / 8;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)rows * groups) return;
  const int r = (int)(gid / groups);
  const int m0 = (int)(gid - (int64_t)r * groups) * 8;
  const SceneDesc& d = desc[row_scene[r]];
  const bool live = d.active && (r - d.row) < d.M;
  const ulonglong2 tp = turns[r];
  const int64_t plane = (int64_t)rows * Kp;
  __align__(16) __nv_bfloat16 v[6][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float2 e = make_float2(0.f, 0.f);
    if (live && m0 + q < d.K) e = phase_f32(tp.x + (uint64_t)(m0 + q) * tp.y);
    split_bf16(e.x, v[0][q], v[3][q]);
    split_bf16(e.y, v[1][q], v[4][q]);
    split_bf16(-e.x, v[2][q], v[5][q]);
  }
  const int64_t off = (int64_t)r * Kp + m0;
#pragma unroll
  for (int pl = 0; pl < 6; ++pl)
    *reinterpret_cast<uint4*>(planes + pl * plane + off) =
        *reinterpret_cast<const uint4*>(v[pl]);
}

template <typename T2>
__device__ __forceinline__ T2 phase_t(uint64_t turn);
template <>
__device__ __forceinline__ float2 phase_t<float2>(uint64_t turn) {
  return phase_f32(turn);
}
template <>
__device__ __forceinline__ double2 phase_t<double2>(uint64_t turn) {
  return phase_f64(turn);
}

template <typename T2>
__global__ void k_b_phase_complex(const SceneDesc* __restrict__ desc,
                                  const int* __restrict__ row_scene,
                                  const ulonglong2* __restrict__ turns, int rows,
                                  int Kp, T2* __restrict__ out) {
  const int groups = Kp / 8;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)rows * groups) return;
  const int r = (int)(gid / groups);
  const int m0 = (int)(gid - (int64_t)r * groups) * 8;
  const SceneDesc& d = desc[row_scene[r]];
  const bool live = d.active && (r - d.row) < d.M;
  const ulonglong2 tp = turns[r];
  T2* dst = out + (int64_t)r * Kp + m0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    T2 e;
    e.x = 0;
    e.y = 0;
    if (live && m0 + q < d.K) e = phase_t<T2>(tp.x + (uint64_t)(m0 + q) * tp.y);
    dst[q] = e;
  }
}

// b_j += sum_m conj(A[j][m]) d_m per stacked row (warp per row).
__global__ void __launch_bounds__(256)
    k_b_data_update_planes(const SceneDesc* __restrict__ desc,
                           const int* __restrict__ row_scene,
                           const __nv_bfloat16* __restrict__ Ap, int rows, int Kp,
                           const float2* __restrict__ d, double2* __restrict__ b) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const int s = row_scene[r];
  if (!desc[s].active) return;
  const int64_t plane = (int64_t)rows * Kp;
  const __nv_bfloat16* rh = Ap + (int64_t)r * Kp;
  const float2* ds = d + (int64_t)s * Kp;
  float sr = 0.f, si = 0.f;
  for (int m0 = lane * 8; m0 < Kp; m0 += 256) {
    const uint4 vrh = *reinterpret_cast<const uint4*>(rh + m0);
    const uint4 vih = *reinterpret_cast<const uint4*>(rh + plane + m0);
    const uint4 vrl = *reinterpret_cast<const uint4*>(rh + 3 * plane + m0);
    const uint4 vil = *reinterpret_cast<const uint4*>(rh + 4 * plane + m0);
    const __nv_bfloat16* prh = reinterpret_cast<const __nv_bfloat16*>(&vrh);
    const __nv_bfloat16* pih = reinterpret_cast<const __nv_bfloat16*>(&vih);
    const __nv_bfloat16* prl = reinterpret_cast<const __nv_bfloat16*>(&vrl);
    const __nv_bfloat16* pil = reinterpret_cast<const __nv_bfloat16*>(&vil);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float ar = __bfloat162float(prh[q]) + __bfloat162float(prl[q]);
      const float ai = __bfloat162float(pih[q]) + __bfloat162float(pil[q]);
      const float2 dm = ds[m0 + q];
      sr = fmaf(ar, dm.x, fmaf(ai, dm.y, sr));
      si = fmaf(ar, dm.y, fmaf(-ai, dm.x, si));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    const double2 bj = b[r];
    b[r] = make_double2(bj.x + (double)sr, bj.y + (double)si);
  }
}

template <typename T2>
__global__ void __launch_bounds__(256)
    k_b_data_update_complex(const SceneDesc* __restrict__ desc,
                            const int* __restrict__ row_scene,
                            const T2* __restrict__ A, int rows, int Kp,
                            const double2* __restrict__ d,
                            double2* __restrict__ b) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const int s = row_scene[r];
  if (!desc[s].active) return;
  const T2* row = A + (int64_t)r * Kp;
  const double2* ds = d + (int64_t)s * Kp;
  double sr = 0.0, si = 0.0;
  for (int m = lane; m < Kp; m += 32) {
    const T2 a = row[m];
    const double2 dm = ds[m];
    sr += (double)a.x * dm.x + (double)a.y * dm.y;
    si += (double)a.x * dm.y - (double)a.y * dm.x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) {
    const double2 bj = b[r];
    b[r] = make_double2(bj.x + sr, bj.y + si);
  }
}

// lambda_n per scene (one block per scene) and the pulse count.
__global__ void __launch_bounds__(256)
    k_b_lambda(const SceneDesc* __restrict__ desc, const double2* __restrict__ b,
               DevScalars* sc) {
  const int s = blockIdx.x;
  const SceneDesc& d = desc[s];
  if (!d.active) return;
  double m = 0.0;
  for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
    const double2 v = b[d.row + j];
    m = fmax(m, v.x * v.x + v.y * v.y);
  }
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t = fmax(t, red[w]);
    sc[s].lambda = d.relative ? d.lam * sqrt(t) : d.lam;
    sc[s].n += 1;
  }
}

// Gather for item (scene, K): the scene's column-K segment partials and its
// block partials (K, J), J > K.
template <typename T2, typename Acc>
__device__ __forceinline__ double2 b_gather(const T2* __restrict__ segpart,
                                            const T2* __restrict__ tilepart,
                                            const int* __restrict__ seg_begin,
                                            const SceneDesc& d, int K) {
  __shared__ Acc red_r[FIN_GROUPS][BLK], red_i[FIN_GROUPS][BLK];
  const int g = threadIdx.x / BLK, i = threadIdx.x % BLK;
  const int s0 = seg_begin[d.seg0 + K], nseg = seg_begin[d.seg0 + K + 1] - s0;
  const int total = nseg + (d.nb - 1 - K);
  const int64_t t0 = d.gblk + packed_block(K, K, d.nb) + 1;
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

// Algorithm 1 step for item (scene, K); the scene's last block updates its
// t, step count and stop flag.
template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS)
    k_b_fista_finalize(const T2* __restrict__ segpart,
                       const T2* __restrict__ tilepart,
                       const int* __restrict__ seg_begin,
                       const int2* __restrict__ items,
                       const SceneDesc* __restrict__ desc,
                       const double2* __restrict__ b, double2* __restrict__ c,
                       double2* __restrict__ z, T2* __restrict__ zt,
                       double2* __restrict__ part, DevScalars* sc) {
  const int2 it = items[blockIdx.x];
  const int s = it.x, K = it.y;
  const SceneDesc& d = desc[s];
  if (!d.active || sc[s].converged) return;
  // the scene's scalars once per CTA (FP64 square root and division: slow
  // on GB300's FP64 pipe), visible after the gather's barrier
  __shared__ double sh[3];  // tau, alpha, beta
  if (threadIdx.x == 0) {
    const double tau = sc[s].tau, t = sc[s].t;
    const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sh[0] = tau;
    sh[1] = sc[s].lambda * tau;
    sh[2] = (t - 1.0) / t_next;
  }
  const double2 y = b_gather<T2, Acc>(segpart, tilepart, seg_begin, d, K);
  const int i = threadIdx.x, idx = d.row + K * BLK + i;
  double p0 = 0.0, p1 = 0.0;
  if (i < BLK) {
    const double tau = sh[0], alpha = sh[1], beta = sh[2];
    const double2 zk = z[idx], bk = b[idx], cprev = c[idx];
    const double ur = zk.x - tau * (y.x - bk.x);
    const double ui = zk.y - tau * (y.y - bk.y);
    const double keep = shrink_keep<T2>(ur * ur + ui * ui, alpha);
    const double cr = ur * keep, ci = ui * keep;
    const double2 zn = make_double2(cr + beta * (cr - cprev.x),
                                    ci + beta * (ci - cprev.y));
    c[idx] = make_double2(cr, ci);
    z[idx] = zn;
    T2 znt;
    znt.x = zn.x;
    znt.y = zn.y;
    zt[idx] = znt;
    const double dr = cr - zk.x, di = ci - zk.y;
    p0 = dr * dr + di * di;
    p1 = cr * cr + ci * ci;
  }
  const double2 ps = block_sum(p0, p1, BLK / 32);
  if (i == 0) part[blockIdx.x] = ps;
  if (!last_block(&sc[s].done, d.nb)) return;
  const double2 tot = sum_parts(part + d.item0, d.nb);
  if (i == 0) {
    const double t = sc[s].t;
    sc[s].t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc[s].iters += 1;
    if (sc[s].tol > 0.0 && sqrt(tot.x) <= sc[s].tol * sqrt(tot.y)) sc[s].converged = 1;
    sc[s].done = 0;
  }
}

// Power step for item (scene, K); the scene's last block forms mu, the
// normalised v and (last step) L and tau.
template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS)
    k_b_power_finalize(const T2* __restrict__ segpart,
                       const T2* __restrict__ tilepart,
                       const int* __restrict__ seg_begin,
                       const int2* __restrict__ items,
                       const SceneDesc* __restrict__ desc,
                       double2* __restrict__ v, T2* __restrict__ vt,
                       double2* __restrict__ w, double2* __restrict__ part,
                       DevScalars* sc, int pstep) {
  const int2 it = items[blockIdx.x];
  const int s = it.x, K = it.y;
  const SceneDesc& d = desc[s];
  if (!d.active || pstep >= d.psteps) return;
  const int last_step = pstep == d.psteps - 1;
  const double2 y = b_gather<T2, Acc>(segpart, tilepart, seg_begin, d, K);
  const int i = threadIdx.x, idx = d.row + K * BLK + i;
  double p0 = 0.0, p1 = 0.0;
  if (i < BLK) {
    w[idx] = y;
    const double2 vk = v[idx];
    p0 = vk.x * y.x + vk.y * y.y;
    p1 = y.x * y.x + y.y * y.y;
  }
  const double2 ps = block_sum(p0, p1, BLK / 32);
  if (i == 0) part[blockIdx.x] = ps;
  if (!last_block(&sc[s].done, d.nb)) return;
  const double2 tot = sum_parts(part + d.item0, d.nb);
  __shared__ double inv_s;
  if (i == 0) {
    const double mu = tot.x;
    sc[s].mu = mu;
    inv_s = tot.y > 0.0 ? 1.0 / sqrt(tot.y) : 0.0;
    sc[s].inv_norm = inv_s;
    if (last_step) {
      const double l = (1.0 + d.margin) * mu;
      if (l > sc[s].lip) sc[s].lip = l;
      sc[s].tau = sc[s].lip > 0.0 ? 1.0 / sc[s].lip : 0.0;
    }
    sc[s].done = 0;
  }
  __syncthreads();
  const double inv = inv_s;
  if (inv > 0.0) {
    for (int k = i; k < d.nb * BLK; k += blockDim.x) {
      const double2 yw = __ldcg(w + d.row + k);
      const double2 nv = make_double2(yw.x * inv, yw.y * inv);
      v[d.row + k] = nv;
      T2 t;
      t.x = nv.x;
      t.y = nv.y;
      vt[d.row + k] = t;
    }
  }
}

template <typename T2>
__global__ void k_b_burst_begin(const SceneDesc* __restrict__ desc,
                                const int* __restrict__ row_scene,
                                double2* __restrict__ z, T2* __restrict__ zt,
                                const double2* __restrict__ c, int rows,
                                DevScalars* sc) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int s = row_scene[r];
  const SceneDesc& d = desc[s];
  if (!d.active) return;
  const double2 v = c[r];
  z[r] = v;
  T2 t;
  t.x = v.x;
  t.y = v.y;
  zt[r] = t;
  if (r == d.row) {
    if (sc[s].n == 1 || d.restart) sc[s].t = 1.0;
    sc[s].converged = 0;
  }
}

__global__ void k_b_iter_begin(const SceneDesc* __restrict__ desc, int S,
                               DevScalars* sc, double tol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  sc[s].iters = 0;
  sc[s].tol = tol;
}

__global__ void k_b_stage(const double2* __restrict__ d, float2* __restrict__ d32,
                          int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d32[i] = make_float2((float)d[i].x, (float)d[i].y);
}

unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t batch_launch_phase(osar_batch* B) {
  k_b_turns<<<grid_for(B->rows, 256), 256, 0, B->stream>>>(
      B->desc, B->row_scene, B->gam, B->rows, B->turns);
  const unsigned g = grid_for((int64_t)B->rows * (B->Kp / 8), 256);
  if (B->prec == OSAR_SPLIT_BF16)
    k_b_phase_planes<<<g, 256, 0, B->stream>>>(B->desc, B->row_scene, B->turns,
                                               B->rows, B->Kp, B->Apl);
  else if (B->prec == OSAR_FP64)
    k_b_phase_complex<double2><<<g, 256, 0, B->stream>>>(
        B->desc, B->row_scene, B->turns, B->rows, B->Kp, (double2*)B->A);
  else
    k_b_phase_complex<float2><<<g, 256, 0, B->stream>>>(
        B->desc, B->row_scene, B->turns, B->rows, B->Kp, (float2*)B->A);
  B->launches += 2;
  return cudaGetLastError();
}

cudaError_t batch_launch_gram(osar_batch* B) {
  if (B->n_gram_tiles == 0) return cudaSuccess;
  B->launches++;
  if (B->prec == OSAR_SPLIT_BF16)
    return launch_gram_tc_tiles(B->stream, B->sm_count, B->map1, B->map2,
                                B->gram_tiles, B->n_gram_tiles,
                                (float2*)B->g_hi, B->g_lo, B->Kp, &B->sc[0].error);
  return launch_gram_simt_tiles(B->stream, B->prec, B->A, B->Kp, B->g_hi,
                                B->gram_tiles, B->n_gram_tiles);
}

cudaError_t batch_launch_data_update(osar_batch* B) {
  const unsigned g = grid_for(B->rows, 8);
  if (B->prec == OSAR_SPLIT_BF16) {
    k_b_stage<<<grid_for((int64_t)B->S * B->Kp, 256), 256, 0, B->stream>>>(
        B->d, B->d32, B->S * B->Kp);
    k_b_data_update_planes<<<g, 256, 0, B->stream>>>(
        B->desc, B->row_scene, B->Apl, B->rows, B->Kp, B->d32, B->b);
    B->launches++;
  } else if (B->prec == OSAR_FP64) {
    k_b_data_update_complex<double2><<<g, 256, 0, B->stream>>>(
        B->desc, B->row_scene, (const double2*)B->A, B->rows, B->Kp, B->d, B->b);
  } else {
    k_b_data_update_complex<float2><<<g, 256, 0, B->stream>>>(
        B->desc, B->row_scene, (const float2*)B->A, B->rows, B->Kp, B->d, B->b);
  }
  k_b_lambda<<<B->S, 256, 0, B->stream>>>(B->desc, B->b, B->sc);
  B->launches += 2;
  return cudaGetLastError();
}

cudaError_t batch_launch_matvec(osar_batch* B, const void* xt, int gated,
                                int pstep) {
  if (B->nseg <= 0) return cudaSuccess;
  const MvBatch mb{B->seg_scene, B->desc, B->sc, gated, pstep};
  auto go = [&](auto zero) {
    using T = decltype(zero);
    using T2 = typename Vec<T>::T2;
    using C = Mv<T, 1>;
    const int grid = std::min(B->nseg, C::CTAS * B->sm_count);
    MvArgs<T, 1> a = {};
    a.x[0] = (const T2*)xt;
    a.segpart[0] = (T2*)B->segpart;
    a.tilepart[0] = (T2*)B->tilepart;
    cudaFuncSetAttribute(k_matvec<T, 1, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    k_matvec<T, 1, true><<<grid, C::THREADS, C::SMEM, B->stream>>>(
        (const T2*)B->g_hi, a, B->segs, B->nseg, 0, B->sc, 0,
        matvec_queue(B->sc), mb, nullptr);
  };
  if (B->prec == OSAR_FP64)
    go(0.0);
  else
    go(0.0f);
  B->launches++;
  return cudaGetLastError();
}

// Power steps: each active scene runs its own count (SceneDesc::psteps, more
// at its first pulse); the launches cover the largest count and skip scenes
// that are done.
cudaError_t batch_launch_power(osar_batch* B, int max_steps) {
  for (int k = 0; k < max_steps; ++k) {
    cudaError_t e = batch_launch_matvec(B, B->vt, 0, k);
    if (e != cudaSuccess) return e;
    if (B->prec == OSAR_FP64)
      k_b_power_finalize<double2, double><<<B->items, FIN_THREADS, 0, B->stream>>>(
          (const double2*)B->segpart, (const double2*)B->tilepart, B->seg_begin,
          B->items_dev, B->desc, B->v, (double2*)B->vt, B->w, B->part, B->sc, k);
    else
      k_b_power_finalize<float2, float><<<B->items, FIN_THREADS, 0, B->stream>>>(
          (const float2*)B->segpart, (const float2*)B->tilepart, B->seg_begin,
          B->items_dev, B->desc, B->v, (float2*)B->vt, B->w, B->part, B->sc, k);
    B->launches++;
  }
  return cudaGetLastError();
}

cudaError_t batch_launch_burst_begin(osar_batch* B) {
  const unsigned g = grid_for(B->rows, 256);
  if (B->prec == OSAR_FP64)
    k_b_burst_begin<double2><<<g, 256, 0, B->stream>>>(
        B->desc, B->row_scene, B->z, (double2*)B->zt, B->c, B->rows, B->sc);
  else
    k_b_burst_begin<float2><<<g, 256, 0, B->stream>>>(
        B->desc, B->row_scene, B->z, (float2*)B->zt, B->c, B->rows, B->sc);
  B->launches++;
  return cudaGetLastError();
}

cudaError_t batch_launch_iter_begin(osar_batch* B, double tol) {
  k_b_iter_begin<<<grid_for(B->S, 128), 128, 0, B->stream>>>(B->desc, B->S, B->sc, tol);
  B->launches++;
  return cudaGetLastError();
}

cudaError_t batch_launch_fista_step(osar_batch* B) {
  cudaError_t e = batch_launch_matvec(B, B->zt, 1, -1);
  if (e != cudaSuccess) return e;
  if (B->prec == OSAR_FP64)
    k_b_fista_finalize<double2, double><<<B->items, FIN_THREADS, 0, B->stream>>>(
        (const double2*)B->segpart, (const double2*)B->tilepart, B->seg_begin,
        B->items_dev, B->desc, B->b, B->c, B->z, (double2*)B->zt, B->part, B->sc);
  else
    k_b_fista_finalize<float2, float><<<B->items, FIN_THREADS, 0, B->stream>>>(
        (const float2*)B->segpart, (const float2*)B->tilepart, B->seg_begin,
        B->items_dev, B->desc, B->b, B->c, B->z, (float2*)B->zt, B->part, B->sc);
  B->launches++;
  return cudaGetLastError();
}

bool batch_make_tensor_maps(osar_batch* B, std::string* err) {
  return encode_plane_map(&B->map1, B->Apl, B->Kp, B->rows, 6, 1, err) &&
         encode_plane_map(&B->map2, B->Apl, B->Kp, B->rows, 6, 2, err);
}

}  // namespace osar
