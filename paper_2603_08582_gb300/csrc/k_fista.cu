// Bandwidth-bound part of Online FISTA: the Hermitian Gram matvec on the
// packed upper triangle, the fused Algorithm-1 step (gradient, step,
// complex shrinkage, momentum, stop rule), the power iteration for L
// (Eq. 11), the data-vector update of Eqs. 12-13 and lambda_n.
//
// Gram storage: the upper 128 x 128 blocks T_IJ = A[I-rows, J-cols], I <= J,
// each stored column-major: entry (r, c) of the block sits at c * 128 + r.
// Column-major blocks make the tensor-core epilogue (one TMEM lane = one row
// per thread) write 256 contiguous bytes per warp instruction.
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
// A second kernel sums, per output block K, the segment partials of column K
// and the block partials of (K, J), J > K (contiguous in the packed order),
// then applies the elementwise step.  The partial traffic is ~1/64 of the
// Gram's.  The last CTA of that grid (an atomic ticket after a fence) does
// the scalar bookkeeping, so an inner step is two launches.  No floating-point
// atomics: results are deterministic and checkpoints resume bit-for-bit.
//
// GB300 has very little FP64 throughput, so on the split-BF16 and FP32 paths
// the partial sums stay in FP32 and only the per-coefficient step (and the
// scalars t, L, lambda) run in FP64.
#include "ctx.h"

#include "finalize.cuh"
#include "step.cuh"

namespace osar {
namespace {

// One step of Algorithm 1 for the 128 coefficients of block K:
//   g = A z - b,  u = z - tau g,  c = S_{lambda tau}(u),
//   t' = (1 + sqrt(1 + 4 t^2)) / 2,  z' = c + (t - 1)/t' (c - c_prev).
// The last CTA then sets t <- t', counts the step and applies the stop rule
// |c - z|_2 <= tol |c|_2 to the whole vector.
// The complex shrinkage factor is shrink_keep (step.cuh).

// Two CTAs per SM (32 registers a thread): the nb blocks of the 128 x 128
// workload (256) then run as one wave over the 152 SMs instead of two.
template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS, 2)
    k_fista_finalize(const T2* __restrict__ segpart,
                     const T2* __restrict__ tilepart,
                     const int* __restrict__ seg_begin, int nb,
                     const double2* __restrict__ b, double2* __restrict__ c,
                     double2* __restrict__ z, T2* __restrict__ zt,
                     double2* __restrict__ part, DevScalars* sc,
                     DevScalars* gs, int count_pass,
                     const float2* __restrict__ corr) {
  // sc: this solution's scalars; gs: the shared ones (tau, tol, passes)
  const int K = blockIdx.x, i = threadIdx.x, idx = K * BLK + i;
  // The step's inputs z, b, c_prev go to shared memory by asynchronous
  // copies issued first, so that their round trip overlaps the converged
  // check and the partial gather instead of following them.
  __shared__ double2 in[3][BLK];
  if (i < BLK) {
    async_copy16(&in[0][i], z + idx);
    async_copy16(&in[1][i], b + idx);
    async_copy16(&in[2][i], c + idx);
  }
  if (sc->converged) {
    async_copy_wait_all();
    return;
  }
  __shared__ double sh[3];  // tau, alpha, beta
  if (threadIdx.x == 0) {
    const double t = sc->t, tau = gs->tau;
    const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sh[0] = tau;
    sh[1] = sc->lambda * tau;
    sh[2] = (t - 1.0) / t_next;
  }
  const double2 y = gather_row<T2, Acc>(segpart, tilepart, seg_begin, nb, K, corr);
  double p0 = 0.0, p1 = 0.0;
  if (i < BLK) {
    const double tau = sh[0], alpha = sh[1], beta = sh[2];
    async_copy_wait_all();
    const double2 zk = in[0][i], bk = in[1][i], cprev = in[2][i];
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
  const double2 s = block_sum(p0, p1, BLK / 32);
  if (i == 0) part[K] = s;
  if (!last_block(&sc->done, gridDim.x)) return;
  const double2 tot = sum_parts(part, nb);
  if (i == 0) {
    const double t = sc->t;
    sc->t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc->iters += 1;
    gs->passes += count_pass;
    if (gs->tol > 0.0 && sqrt(tot.x) <= gs->tol * sqrt(tot.y)) sc->converged = 1;
    sc->done = 0;
  }
}

// y_K from the partials a Gram update's fused power step wrote: the column
// partials of the stored blocks (I, K), I <= K, then the two half-row
// partials of each block (K, J), J > K (contiguous in the packed order),
// split over FIN_GROUPS thread groups and combined in a fixed order.
__device__ __forceinline__ double2 gather_gram_row(const float2* __restrict__ pcol,
                                                   const float2* __restrict__ prow,
                                                   int nb, int K) {
  __shared__ float red_r[FIN_GROUPS][BLK], red_i[FIN_GROUPS][BLK];
  const int g = threadIdx.x / BLK, i = threadIdx.x % BLK;
  const int ncol = K + 1;
  const int total = ncol + 2 * (nb - 1 - K);
  const int64_t r0 = 2 * (packed_block(K, K, nb) + 1);  // block (K, K+1), half 0
  float yr = 0.f, yi = 0.f;
#pragma unroll 4
  for (int q = g; q < total; q += FIN_GROUPS) {
    const float2 v = q < ncol ? pcol[packed_block(q, K, nb) * BLK + i]
                              : prow[(r0 + (q - ncol)) * BLK + i];
    yr += v.x;
    yi += v.y;
  }
  red_r[g][i] = yr;
  red_i[g][i] = yi;
  __syncthreads();
  double2 y = make_double2(0.0, 0.0);
  if (threadIdx.x < BLK) {
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int k = 0; k < FIN_GROUPS; ++k) {
      sr += red_r[k][i];
      si += red_i[k][i];
    }
    y = make_double2((double)sr, (double)si);
  }
  return y;
}

// Power step: w = A v; the last CTA forms mu = Re(v^H A v) (v has unit
// norm) and 1/|w|, and on the last step of a pulse sets
// L_n = max(L_{n-1}, (1 + margin) mu) and tau = 1/L_n.  FROM_GRAM: A v
// comes from the Gram update's fused power step (segpart / tilepart are
// its column / half-row partials; no Gram pass is counted).
template <typename T2, typename Acc, bool FROM_GRAM = false>
__global__ void __launch_bounds__(FIN_THREADS)
    k_power_finalize(const T2* __restrict__ segpart,
                     const T2* __restrict__ tilepart,
                     const int* __restrict__ seg_begin, int nb,
                     const double2* __restrict__ v, double2* __restrict__ w,
                     double2* __restrict__ part, DevScalars* sc, int last_step,
                     double margin, const float2* __restrict__ corr) {
  const int K = blockIdx.x, i = threadIdx.x, idx = K * BLK + i;
  double2 y;
  if constexpr (FROM_GRAM)
    y = gather_gram_row(segpart, tilepart, nb, K);
  else
    y = gather_row<T2, Acc>(segpart, tilepart, seg_begin, nb, K, corr);
  double p0 = 0.0, p1 = 0.0;
  if (i < BLK) {
    w[idx] = y;
    const double2 vk = v[idx];
    p0 = vk.x * y.x + vk.y * y.y;
    p1 = y.x * y.x + y.y * y.y;
  }
  const double2 s = block_sum(p0, p1, BLK / 32);
  if (i == 0) part[K] = s;
  if (!last_block(&sc->done, gridDim.x)) return;
  const double2 tot = sum_parts(part, nb);
  if (i == 0) {
    const double mu = tot.x;
    sc->mu = mu;
    sc->inv_norm = tot.y > 0.0 ? 1.0 / sqrt(tot.y) : 0.0;
    if (last_step) {
      const double l = (1.0 + margin) * mu;
      if (l > sc->lip) sc->lip = l;
      sc->tau = sc->lip > 0.0 ? 1.0 / sc->lip : 0.0;
    }
    if (!FROM_GRAM) sc->passes += 1;
    sc->done = 0;
  }
}

// v <- w / |w| and its working-precision copy (v kept when |w| = 0).
template <typename T2>
__global__ void k_power_normalize(const double2* __restrict__ w,
                                  double2* __restrict__ v, T2* __restrict__ vt,
                                  int n, const DevScalars* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double s = sc->inv_norm;
  if (i >= n || s == 0.0) return;
  const double2 y = w[i];
  const double2 nv = make_double2(y.x * s, y.y * s);
  v[i] = nv;
  T2 t;
  t.x = nv.x;
  t.y = nv.y;
  vt[i] = t;
}

// y = A x for osar_gram_apply.
template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS)
    k_apply_finalize(const T2* __restrict__ segpart,
                     const T2* __restrict__ tilepart,
                     const int* __restrict__ seg_begin, int nb,
                     double2* __restrict__ y) {
  const int K = blockIdx.x, i = threadIdx.x;
  const double2 v = gather_row<T2, Acc>(segpart, tilepart, seg_begin, nb, K);
  if (i < BLK) y[K * BLK + i] = v;
}

// y = A x of a pass whose result is needed as a vector (the pixel-space Gram
// form); gated: nothing once solution 0 has met the stop rule.
template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS)
    k_pass_finalize(const T2* __restrict__ segpart,
                    const T2* __restrict__ tilepart,
                    const int* __restrict__ seg_begin, int nb,
                    double2* __restrict__ y, const DevScalars* sc, int gated) {
  if (gated && sc->converged) return;
  const int K = blockIdx.x, i = threadIdx.x;
  const double2 v = gather_row<T2, Acc>(segpart, tilepart, seg_begin, nb, K);
  if (i < BLK) y[K * BLK + i] = v;
}

// ------------------------------------------------------- data vector, lambda
// The last CTA of a data-update grid sets lambda_n = rel * max_j |b_j| (or
// the absolute value) and counts the pulse.  Each thread brings the bit
// pattern of its largest |b_j|^2 (0 if none): non-negative doubles order as
// their bit patterns, so the maximum is taken with 64-bit integer compares
// instead of FP64 ones, of which GB300 issues about 1/64 as many.
__device__ __forceinline__ void lambda_tail(unsigned long long bits,
                                            double* bmax, DevScalars* sc,
                                            const LamSet& lam, int relative) {
  __shared__ unsigned long long red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = v > bits ? v : bits;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t = red[w2] > t ? red[w2] : t;
    bmax[blockIdx.x] = __longlong_as_double((long long)t);
  }
  if (!last_block(&sc->done, gridDim.x)) return;
  unsigned long long mx = 0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    const unsigned long long v =
        (unsigned long long)__double_as_longlong(__ldcg(bmax + k));
    mx = v > mx ? v : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t = red[w2] > t ? red[w2] : t;
    const double m2 = __longlong_as_double((long long)t);
    // every solution of the lambda path: lambda_n = factor x ||b_n||_inf
    // (Eq. 11's lambda, relative) or the absolute value
    for (int l = 0; l < lam.n; ++l)
      sc[l].lambda = relative ? lam.v[l] * sqrt(m2) : lam.v[l];
    sc->n += 1;
    sc->done = 0;
  }
}

// b_j += sum_m conj(A[j][m]) d_m (Eqs. 12-13), one warp per atom j.
template <typename T2>
__global__ void __launch_bounds__(256)
    k_data_update_complex(const T2* __restrict__ A, int Mp, int Kp,
                          const double2* __restrict__ d, double2* __restrict__ b,
                          double* bmax, DevScalars* sc, LamSet lam,
                          int relative) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  unsigned long long m2b = 0;
  if (j < Mp) {
    const T2* row = A + (int64_t)j * Kp;
    double sr = 0.0, si = 0.0;
    for (int m = lane; m < Kp; m += 32) {
      const T2 a = row[m];
      const double2 dm = d[m];
      sr += (double)a.x * dm.x + (double)a.y * dm.y;
      si += (double)a.x * dm.y - (double)a.y * dm.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      const double2 bj = b[j];
      const double2 nb2 = make_double2(bj.x + sr, bj.y + si);
      b[j] = nb2;
      m2b = (unsigned long long)__double_as_longlong(nb2.x * nb2.x + nb2.y * nb2.y);
    }
  }
  lambda_tail(m2b, bmax, sc, lam, relative);
}

// Split-BF16 planes: A = (re_hi + re_lo) + i (im_hi + im_lo), FP32 products
// and sums.  A CTA takes DU_ATOMS consecutive atoms: each warp forms the
// dot products of DU_ATOMS / DU_WARPS of them (8 entries per lane per load,
// one xor tree per atom) into shared memory, then one lane per atom adds the
// sum into b_j in FP64 and forms |b_j|^2.  One warp instruction of that FP64
// tail covers 32 atoms; issued by one lane per warp and atom, the tail and
// the lambda reduction's FP64 compares held the kernel at 72 us for the
// 134 MB of planes of the 128 x 128 workload.
constexpr int DU_WARPS = 16, DU_ATOMS = 128;
__global__ void __launch_bounds__(DU_WARPS * 32)
    k_data_update_planes(const __nv_bfloat16* __restrict__ Ap, int Mp, int Kp,
                         const float2* __restrict__ d, double2* __restrict__ b,
                         double* bmax, DevScalars* sc, LamSet lam,
                         int relative) {
  __shared__ float2 sums[DU_ATOMS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.x * DU_ATOMS;
  const int64_t plane = (int64_t)Mp * Kp;
  for (int a = warp; a < DU_ATOMS; a += DU_WARPS) {
    const int j = j0 + a;
    float sr = 0.f, si = 0.f;
    if (j < Mp) {
      const __nv_bfloat16* rh = Ap + (int64_t)j * Kp;
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
          const float2 dm = d[m0 + q];
          sr = fmaf(ar, dm.x, fmaf(ai, dm.y, sr));
          si = fmaf(ar, dm.y, fmaf(-ai, dm.x, si));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
    }
    if (lane == 0) sums[a] = make_float2(sr, si);
  }
  __syncthreads();
  unsigned long long m2b = 0;
  const int j = j0 + (int)threadIdx.x;
  if (threadIdx.x < DU_ATOMS && j < Mp) {
    const float2 s = sums[threadIdx.x];
    const double2 bj = b[j];
    const double2 nb2 = make_double2(bj.x + (double)s.x, bj.y + (double)s.y);
    b[j] = nb2;
    m2b = (unsigned long long)__double_as_longlong(nb2.x * nb2.x + nb2.y * nb2.y);
  }
  lambda_tail(m2b, bmax, sc, lam, relative);
}

__global__ void k_stage_data(const double2* __restrict__ d,
                             float2* __restrict__ d32, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d32[i] = make_float2((float)d[i].x, (float)d[i].y);
}

// Start of a burst (Algorithm 1 initialisation): z^(1) = c^(0) = c_hat_{n-1},
// t_1 = 1 at the first pulse (or always, with restart), else t_{n-1}.
template <typename T2>
__global__ void k_burst_begin(double2* __restrict__ z, T2* __restrict__ zt,
                              const double2* __restrict__ c, int n,
                              DevScalars* sc, int reset_t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 v = c[i];
    z[i] = v;
    T2 t;
    t.x = v.x;
    t.y = v.y;
    zt[i] = t;
  }
  if (i == 0) {
    if (reset_t) sc->t = 1.0;
    sc->converged = 0;
  }
}

__global__ void k_iter_begin(DevScalars* sc, int n_lam, double tol) {
  for (int l = 0; l < n_lam; ++l) sc[l].iters = 0;
  sc->tol = tol;
}

template <typename T2>
__global__ void k_to_working(const double2* __restrict__ x, T2* __restrict__ xt,
                             int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    T2 t;
    t.x = x[i].x;
    t.y = x[i].y;
    xt[i] = t;
  }
}

// Offset of Gram entry (i, j) in the packed, column-major blocks; entries
// below the diagonal are read from their mirror (upper = false: conjugate).
__device__ __forceinline__ int64_t stored_index(int i, int j, int nb,
                                                bool* upper) {
  *upper = i <= j;
  const int a = *upper ? i : j, c = *upper ? j : i;
  return packed_block(a / BLK, c / BLK, nb) * (int64_t)(BLK * BLK) +
         (int64_t)(c % BLK) * BLK + (a % BLK);
}

// Dense rows [r0, r0 + rows) of the Hermitian Gram (M columns), from the
// packed upper blocks plus the optional compensation word.
template <typename T2>
__global__ void k_gram_expand(const T2* __restrict__ G,
                              const __nv_bfloat162* __restrict__ Glo, int nb, int M,
                              int r0, int rows, double2* __restrict__ out) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)rows * M) return;
  const int i = r0 + (int)(gid / M);
  const int j = (int)(gid - (int64_t)(gid / M) * M);
  bool upper;
  const int64_t o = stored_index(i, j, nb, &upper);
  double re = (double)G[o].x, im = (double)G[o].y;
  if (Glo) {
    const float2 lo = __bfloat1622float2(Glo[o]);
    re += (double)lo.x;
    im += (double)lo.y;
  }
  out[gid] = make_double2(re, upper ? im : -im);
}

template <typename T2>
__global__ void k_gram_entries(const T2* __restrict__ G,
                               const __nv_bfloat162* __restrict__ Glo, int nb,
                               const int2* __restrict__ rc, int count,
                               double2* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  bool upper;
  const int64_t o = stored_index(rc[q].x, rc[q].y, nb, &upper);
  double re = (double)G[o].x, im = (double)G[o].y;
  if (Glo) {
    const float2 lo = __bfloat1622float2(Glo[o]);
    re += (double)lo.x;
    im += (double)lo.y;
  }
  out[q] = make_double2(re, upper ? im : -im);
}

// Working-precision copy of a caller vector that holds only n_valid entries
// (zero beyond), and y = A x written only for the first m_valid entries:
// used when x and y are caller buffers of length M rather than Mp.
template <typename T2>
__global__ void k_to_working_bounded(const double2* __restrict__ x,
                                     T2* __restrict__ xt, int n_valid, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = i < n_valid ? x[i] : make_double2(0.0, 0.0);
  T2 t;
  t.x = v.x;
  t.y = v.y;
  xt[i] = t;
}

template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS)
    k_apply_finalize_bounded(const T2* __restrict__ segpart,
                             const T2* __restrict__ tilepart,
                             const int* __restrict__ seg_begin, int nb,
                             double2* __restrict__ y, int m_valid) {
  const int K = blockIdx.x, i = threadIdx.x;
  const double2 v = gather_row<T2, Acc>(segpart, tilepart, seg_begin, nb, K);
  if (i < BLK && K * BLK + i < m_valid) y[K * BLK + i] = v;
}

// One matvec launch over R vectors: one CTA per SM (the shared-memory ring
// fills an SM), at most one per segment.
// Packed Grams up to this size stay in L2 (129 MB on GB300) across passes.
constexpr int64_t KEEP_L2_BYTES = 80ll << 20;

template <typename T, int R>
void launch_mv(osar_ctx* ctx, MvArgs<T, R> a, int gated) {
  using C = Mv<T, R>;
  a.keep_l2 = ctx->nblk * BLK * BLK * (int64_t)sizeof(typename Vec<T>::T2) <=
              KEEP_L2_BYTES;
  cudaFuncSetAttribute(k_matvec<T, R, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  const int slots = C::CTAS * ctx->sm_count;
  const unsigned grid = (unsigned)(ctx->nseg < slots ? ctx->nseg : slots);
  k_matvec<T, R, false><<<grid, C::THREADS, C::SMEM, ctx->stream>>>(
      (const typename Vec<T>::T2*)ctx->g_hi, a, ctx->segs, ctx->nseg, ctx->nb,
      ctx->scal, gated, matvec_queue(ctx->scal), MvBatch{},
      (const void* const*)ctx->gram_ref);
}

// Device address of solution l's stop flag (pointer arithmetic only).
const int32_t* stop_flag(const osar_ctx* ctx, int l) {
  return reinterpret_cast<const int32_t*>(
      reinterpret_cast<const char*>(ctx->scal + l) +
      offsetof(DevScalars, converged));
}

// Partial-sum buffers for vector slot l of a pass: 0 the main ones, 1 the
// second vector's, 2.. the lambda path's further solutions.
void* seg_set(const osar_ctx* ctx, int l) {
  if (l == 0) return ctx->segpart;
  if (l == 1) return ctx->segpart2;
  const size_t cplx = ctx->prec == OSAR_FP64 ? 16 : 8;
  return static_cast<char*>(ctx->segpart_x) +
         (size_t)(l - 2) * cplx * BLK * (size_t)ctx->nseg;
}
void* tile_set(const osar_ctx* ctx, int l) {
  if (l == 0) return ctx->tilepart;
  if (l == 1) return ctx->tilepart2;
  const size_t cplx = ctx->prec == OSAR_FP64 ? 16 : 8;
  return static_cast<char*>(ctx->tilepart_x) +
         (size_t)(l - 2) * cplx * BLK * (size_t)ctx->nblk;
}

template <typename T>
void launch_mv(osar_ctx* ctx, const void* xt, void* segp, void* tilep,
               int gated) {
  using T2 = typename Vec<T>::T2;
  MvArgs<T, 1> a;
  a.x[0] = (const T2*)xt;
  a.segpart[0] = (T2*)segp;
  a.tilepart[0] = (T2*)tilep;
  a.gate[0] = stop_flag(ctx, 0);
  launch_mv<T, 1>(ctx, a, gated);
}

// Launch the matvec on the working-precision copy of a vector (and, with a
// deferred Gram update pending, the pending block's term into set 0).
void matvec(osar_ctx* ctx, const void* xt, int gated) {
  launch_corr(ctx, xt, 0, gated ? stop_flag(ctx, 0) : nullptr);
  ProfEvent ev;
  prof_begin(ctx, KCL_MATVEC, &ev);
  if (ctx->prec == OSAR_FP64)
    launch_mv<double>(ctx, xt, ctx->segpart, ctx->tilepart, gated);
  else
    launch_mv<float>(ctx, xt, ctx->segpart, ctx->tilepart, gated);
  prof_end(ctx, &ev);
  ctx->launches++;
}

// Gated pass applying the Gram to the iterates of solutions l and l + 1
// (both when l + 1 < n_lam) into their partial-sum sets.
template <typename T>
void matvec_solutions(osar_ctx* ctx, int l) {
  using T2 = typename Vec<T>::T2;
  const size_t wv = sizeof(T2) * (size_t)ctx->Mp;
  const char* zt = static_cast<const char*>(ctx->zt);
  if (l + 1 < ctx->n_lam) {
    MvArgs<T, 2> a;
    for (int r = 0; r < 2; ++r) {
      a.x[r] = reinterpret_cast<const T2*>(zt + (l + r) * wv);
      a.segpart[r] = (T2*)seg_set(ctx, l + r);
      a.tilepart[r] = (T2*)tile_set(ctx, l + r);
      a.gate[r] = stop_flag(ctx, l + r);
    }
    launch_mv<T, 2>(ctx, a, 1);
  } else {
    MvArgs<T, 1> a;
    a.x[0] = reinterpret_cast<const T2*>(zt + l * wv);
    a.segpart[0] = (T2*)seg_set(ctx, l);
    a.tilepart[0] = (T2*)tile_set(ctx, l);
    a.gate[0] = stop_flag(ctx, l);
    launch_mv<T, 1>(ctx, a, 1);
  }
}

}  // namespace

cudaError_t launch_data_update(osar_ctx* ctx) {
  ProfEvent ev;
  prof_begin(ctx, KCL_BUPD, &ev);
  const unsigned g = (unsigned)((ctx->Mp + 7) / 8);
  const LamSet lam = ctx->lam;
  const int rel = ctx->cfg.lambda_relative;
  if (ctx->prec == OSAR_SPLIT_BF16) {
    k_stage_data<<<(unsigned)((ctx->Kp + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->d_dev, ctx->d32, ctx->Kp);
    k_data_update_planes<<<(unsigned)((ctx->Mp + DU_ATOMS - 1) / DU_ATOMS),
                           DU_WARPS * 32, 0, ctx->stream>>>(
        ctx->Apl, ctx->Mp, ctx->Kp, ctx->d32, ctx->b, ctx->bmax, ctx->scal,
        lam, rel);
    ctx->launches++;
  } else if (ctx->prec == OSAR_FP64) {
    k_data_update_complex<double2><<<g, 256, 0, ctx->stream>>>(
        (const double2*)ctx->A, ctx->Mp, ctx->Kp, ctx->d_dev, ctx->b, ctx->bmax,
        ctx->scal, lam, rel);
  } else {
    k_data_update_complex<float2><<<g, 256, 0, ctx->stream>>>(
        (const float2*)ctx->A, ctx->Mp, ctx->Kp, ctx->d_dev, ctx->b, ctx->bmax,
        ctx->scal, lam, rel);
  }
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_power_steps(osar_ctx* ctx, int steps, bool fuse) {
  const unsigned nb = (unsigned)ctx->nb;
  // the FP64 path keeps separate passes: two FP64 vectors' partial sums do
  // not fit the matvec's registers; a lambda path pairs its own solutions
  fuse = fuse && ctx->prec != OSAR_FP64 && ctx->n_lam == 1;
  // the Gram update just formed G_n v (first step, no pass of its own)
  const bool from_gram = ctx->gp_ready;
  ctx->gp_ready = false;
  bool fused_last = false;
  for (int s = 0; s < steps; ++s) {
    const int last = s == steps - 1 ? 1 : 0;
    if (s == 0 && from_gram) {
      ProfEvent ev;
      prof_begin(ctx, KCL_POWFIN, &ev);
      k_power_finalize<float2, float, true><<<nb, FIN_THREADS, 0, ctx->stream>>>(
          ctx->gp_col, ctx->gp_row, nullptr, ctx->nb, ctx->v, ctx->w,
          ctx->part, ctx->scal, last, ctx->cfg.lipschitz_margin, nullptr);
      k_power_normalize<float2><<<nb, BLK, 0, ctx->stream>>>(
          ctx->w, ctx->v, (float2*)ctx->vt, ctx->Mp, ctx->scal);
      prof_end(ctx, &ev);
      ctx->launches += 2;
      continue;
    }
    if (last && fuse) {
      fused_last = true;
      // the burst that follows starts from z = c_hat: apply the Gram to it
      // in the same pass as the last power step
      cudaError_t e = launch_burst_begin(ctx);
      if (e == cudaSuccess) e = launch_corr(ctx, ctx->vt, 0, nullptr);
      if (e == cudaSuccess) e = launch_corr(ctx, ctx->zt, 1, nullptr);
      if (e != cudaSuccess) return e;
      ProfEvent ev;
      prof_begin(ctx, KCL_MATVEC, &ev);
      MvArgs<float, 2> a;
      a.x[0] = (const float2*)ctx->vt;
      a.x[1] = (const float2*)ctx->zt;
      a.segpart[0] = (float2*)ctx->segpart;
      a.segpart[1] = (float2*)ctx->segpart2;
      a.tilepart[0] = (float2*)ctx->tilepart;
      a.tilepart[1] = (float2*)ctx->tilepart2;
      a.gate[0] = a.gate[1] = stop_flag(ctx, 0);  // ungated pass
      launch_mv<float, 2>(ctx, a, 0);
      prof_end(ctx, &ev);
      ctx->launches++;
    } else {
      matvec(ctx, ctx->vt, 0);
    }
    ProfEvent ev;
    prof_begin(ctx, KCL_POWFIN, &ev);
    if (ctx->prec == OSAR_FP64) {
      k_power_finalize<double2, double><<<nb, FIN_THREADS, 0, ctx->stream>>>(
          (const double2*)ctx->segpart, (const double2*)ctx->tilepart,
          ctx->seg_begin, ctx->nb, ctx->v, ctx->w, ctx->part, ctx->scal, last,
          ctx->cfg.lipschitz_margin, nullptr);
      k_power_normalize<double2><<<nb, BLK, 0, ctx->stream>>>(
          ctx->w, ctx->v, (double2*)ctx->vt, ctx->Mp, ctx->scal);
    } else {
      k_power_finalize<float2, float><<<nb, FIN_THREADS, 0, ctx->stream>>>(
          (const float2*)ctx->segpart, (const float2*)ctx->tilepart,
          ctx->seg_begin, ctx->nb, ctx->v, ctx->w, ctx->part, ctx->scal, last,
          ctx->cfg.lipschitz_margin, corr_set(ctx, 0));
      k_power_normalize<float2><<<nb, BLK, 0, ctx->stream>>>(
          ctx->w, ctx->v, (float2*)ctx->vt, ctx->Mp, ctx->scal);
    }
    prof_end(ctx, &ev);
    ctx->launches += 2;
  }
  if (fused_last) {
    ctx->first_ready = true;
    ctx->fresh = false;
  }
  return cudaGetLastError();
}

cudaError_t launch_burst_begin(osar_ctx* ctx) {
  const bool reset = ctx->n == 1 || ctx->cfg.restart_momentum;
  const int64_t Mp = ctx->Mp;
  for (int l = 0; l < ctx->n_lam; ++l) {
    if (ctx->prec == OSAR_FP64)
      k_burst_begin<double2><<<(unsigned)ctx->nb, 128, 0, ctx->stream>>>(
          ctx->z + l * Mp, (double2*)ctx->zt + l * Mp, ctx->c + l * Mp, ctx->Mp,
          ctx->scal + l, reset ? 1 : 0);
    else
      k_burst_begin<float2><<<(unsigned)ctx->nb, 128, 0, ctx->stream>>>(
          ctx->z + l * Mp, (float2*)ctx->zt + l * Mp, ctx->c + l * Mp, ctx->Mp,
          ctx->scal + l, reset ? 1 : 0);
    ctx->launches++;
  }
  return cudaGetLastError();
}

// The matvec runs with the largest shared-memory carve-out; the small
// kernels between its passes ask for the same one, so that the SMs need not
// switch their L1 / shared-memory split at every launch of a burst.
cudaError_t prepare_burst_kernels() {
  const int v = cudaSharedmemCarveoutMaxShared;
  const cudaFuncAttribute a = cudaFuncAttributePreferredSharedMemoryCarveout;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, a, v);
  };
  set((const void*)k_fista_finalize<float2, float>);
  set((const void*)k_fista_finalize<double2, double>);
  set((const void*)k_power_finalize<float2, float>);
  set((const void*)k_power_finalize<float2, float, true>);
  set((const void*)k_power_finalize<double2, double>);
  set((const void*)k_pass_finalize<float2, float>);
  set((const void*)k_pass_finalize<double2, double>);
  set((const void*)k_power_normalize<float2>);
  set((const void*)k_power_normalize<double2>);
  set((const void*)k_burst_begin<float2>);
  set((const void*)k_burst_begin<double2>);
  set((const void*)k_iter_begin);
  return e;
}

__global__ void k_set_gram_ref(void** ref, void* p) { *ref = p; }

cudaError_t launch_set_gram_ref(osar_ctx* ctx) {
  if (!ctx->gram_ref) return cudaSuccess;
  k_set_gram_ref<<<1, 1, 0, ctx->stream>>>(ctx->gram_ref, ctx->g_hi);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_iter_begin(osar_ctx* ctx, double tol) {
  k_iter_begin<<<1, 1, 0, ctx->stream>>>(ctx->scal, ctx->n_lam, tol);
  ctx->launches++;
  return cudaGetLastError();
}

namespace {

// Algorithm 1's step (after the Gram pass) for solution l from partial set s.
template <typename T2, typename Acc>
void fista_finalize(osar_ctx* ctx, int l, int s, int count_pass) {
  const int64_t Mp = ctx->Mp;
  k_fista_finalize<T2, Acc><<<(unsigned)ctx->nb, FIN_THREADS, 0, ctx->stream>>>(
      (const T2*)seg_set(ctx, s), (const T2*)tile_set(ctx, s), ctx->seg_begin,
      ctx->nb, ctx->b, ctx->c + l * Mp, ctx->z + l * Mp, (T2*)ctx->zt + l * Mp,
      ctx->part, ctx->scal + l, ctx->scal, count_pass,
      ctx->n_lam == 1 ? corr_set(ctx, s) : nullptr);
}

}  // namespace

cudaError_t launch_fista_step(osar_ctx* ctx) {
  const bool fp64 = ctx->prec == OSAR_FP64;
  if (ctx->n_lam > 1) {
    // lambda path: one pass per two solutions, then each solution's step
    // (a solution past the stop rule skips both; a pass of two runs while
    // either still steps, and counts once)
    for (int l = 0; l < ctx->n_lam; l += 2) {
      ProfEvent ev;
      prof_begin(ctx, KCL_MATVEC, &ev);
      if (fp64)
        matvec_solutions<double>(ctx, l);
      else
        matvec_solutions<float>(ctx, l);
      prof_end(ctx, &ev);
      ctx->launches++;
    }
    ProfEvent ev;
    prof_begin(ctx, KCL_FIN, &ev);
    for (int l = 0; l < ctx->n_lam; ++l) {
      // the pair's pass is counted with its first solution's step
      const int count = l % 2 == 0 ? 1 : 0;
      if (fp64)
        fista_finalize<double2, double>(ctx, l, l, count);
      else
        fista_finalize<float2, float>(ctx, l, l, count);
      ctx->launches++;
    }
    prof_end(ctx, &ev);
    return cudaGetLastError();
  }
  // the first step after a fused push reuses the pass made with the last
  // power step (already counted as a Gram pass)
  const bool pre = ctx->first_ready;
  ctx->first_ready = false;
  if (!pre) matvec(ctx, ctx->zt, 1);
  ProfEvent ev;
  prof_begin(ctx, KCL_FIN, &ev);
  if (fp64)
    fista_finalize<double2, double>(ctx, 0, pre ? 1 : 0, pre ? 0 : 1);
  else
    fista_finalize<float2, float>(ctx, 0, pre ? 1 : 0, pre ? 0 : 1);
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_gram_apply(osar_ctx* ctx, const double2* x, double2* y) {
  const unsigned g = (unsigned)((ctx->Mp + 255) / 256);
  if (ctx->prec == OSAR_FP64)
    k_to_working<double2><<<g, 256, 0, ctx->stream>>>(x, (double2*)ctx->xt, ctx->Mp);
  else
    k_to_working<float2><<<g, 256, 0, ctx->stream>>>(x, (float2*)ctx->xt, ctx->Mp);
  matvec(ctx, ctx->xt, 0);
  if (ctx->prec == OSAR_FP64)
    k_apply_finalize<double2, double><<<(unsigned)ctx->nb, FIN_THREADS, 0, ctx->stream>>>(
        (const double2*)ctx->segpart, (const double2*)ctx->tilepart,
        ctx->seg_begin, ctx->nb, y);
  else
    k_apply_finalize<float2, float><<<(unsigned)ctx->nb, FIN_THREADS, 0, ctx->stream>>>(
        (const float2*)ctx->segpart, (const float2*)ctx->tilepart,
        ctx->seg_begin, ctx->nb, y);
  ctx->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_set_working(osar_ctx* ctx) {
  // working-precision copies of every solution's z and of v (after a
  // checkpoint load)
  const int nz = ctx->n_lam * ctx->Mp;
  const unsigned gz = (unsigned)((nz + 255) / 256);
  const unsigned g = (unsigned)((ctx->Mp + 255) / 256);
  if (ctx->prec == OSAR_FP64) {
    k_to_working<double2><<<gz, 256, 0, ctx->stream>>>(ctx->z, (double2*)ctx->zt, nz);
    k_to_working<double2><<<g, 256, 0, ctx->stream>>>(ctx->v, (double2*)ctx->vt, ctx->Mp);
  } else {
    k_to_working<float2><<<gz, 256, 0, ctx->stream>>>(ctx->z, (float2*)ctx->zt, nz);
    k_to_working<float2><<<g, 256, 0, ctx->stream>>>(ctx->v, (float2*)ctx->vt, ctx->Mp);
  }
  ctx->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_gram_expand(osar_ctx* ctx, int r0, int rows, double2* dense) {
  const int64_t n = (int64_t)rows * ctx->M;
  const unsigned g = (unsigned)((n + 255) / 256);
  if (ctx->prec == OSAR_FP64)
    k_gram_expand<double2><<<g, 256, 0, ctx->stream>>>(
        (const double2*)ctx->g_hi, nullptr, ctx->nb, ctx->M, r0, rows, dense);
  else
    k_gram_expand<float2><<<g, 256, 0, ctx->stream>>>(
        (const float2*)ctx->g_hi, ctx->g_lo, ctx->nb, ctx->M, r0, rows, dense);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_gram_entries(osar_ctx* ctx, const int2* rc, int count,
                                double2* out) {
  const unsigned g = (unsigned)((count + 255) / 256);
  if (ctx->prec == OSAR_FP64)
    k_gram_entries<double2><<<g, 256, 0, ctx->stream>>>(
        (const double2*)ctx->g_hi, nullptr, ctx->nb, rc, count, out);
  else
    k_gram_entries<float2><<<g, 256, 0, ctx->stream>>>(
        (const float2*)ctx->g_hi, ctx->g_lo, ctx->nb, rc, count, out);
  ctx->launches++;
  return cudaGetLastError();
}

size_t gram_apply_scratch_bytes(const osar_ctx* ctx) {
  const size_t cplx = ctx->prec == OSAR_FP64 ? 16 : 8;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  return al(cplx * ctx->Mp) + al(cplx * BLK * (size_t)ctx->nseg) +
         al(cplx * BLK * (size_t)ctx->nblk);
}

// y = A x with caller-provided scratch (working copy of x, segment and block
// partials carved from `scratch`, which must hold gram_apply_scratch_bytes);
// x and y are device vectors of M entries.  Every scratch byte read is
// written earlier in the same call, so the scratch needs no clearing.
cudaError_t launch_gram_apply_scratch(osar_ctx* ctx, const double2* x,
                                      double2* y, void* scratch) {
  const size_t cplx = ctx->prec == OSAR_FP64 ? 16 : 8;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  char* base = static_cast<char*>(scratch);
  void* xt = base;
  void* segp = base + al(cplx * ctx->Mp);
  void* tilep = base + al(cplx * ctx->Mp) + al(cplx * BLK * (size_t)ctx->nseg);
  const unsigned g = (unsigned)((ctx->Mp + 255) / 256);
  if (ctx->prec == OSAR_FP64) {
    k_to_working_bounded<double2><<<g, 256, 0, ctx->stream>>>(
        x, (double2*)xt, ctx->M, ctx->Mp);
    launch_mv<double>(ctx, xt, segp, tilep, 0);
    k_apply_finalize_bounded<double2, double>
        <<<(unsigned)ctx->nb, FIN_THREADS, 0, ctx->stream>>>(
            (const double2*)segp, (const double2*)tilep, ctx->seg_begin,
            ctx->nb, y, ctx->M);
  } else {
    k_to_working_bounded<float2><<<g, 256, 0, ctx->stream>>>(
        x, (float2*)xt, ctx->M, ctx->Mp);
    launch_mv<float>(ctx, xt, segp, tilep, 0);
    k_apply_finalize_bounded<float2, float>
        <<<(unsigned)ctx->nb, FIN_THREADS, 0, ctx->stream>>>(
            (const float2*)segp, (const float2*)tilep, ctx->seg_begin, ctx->nb,
            y, ctx->M);
  }
  ctx->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_matvec(osar_ctx* ctx, const void* xt) {
  matvec(ctx, xt, 0);
  return cudaGetLastError();
}

cudaError_t launch_gram_pass(osar_ctx* ctx, const void* xt, int gated,
                             double2* y, int kind) {
  matvec(ctx, xt, gated);
  ProfEvent ev;
  prof_begin(ctx, kind, &ev);
  if (ctx->prec == OSAR_FP64)
    k_pass_finalize<double2, double><<<(unsigned)ctx->nb, FIN_THREADS, 0, ctx->stream>>>(
        (const double2*)ctx->segpart, (const double2*)ctx->tilepart,
        ctx->seg_begin, ctx->nb, y, ctx->scal, gated);
  else
    k_pass_finalize<float2, float><<<(unsigned)ctx->nb, FIN_THREADS, 0, ctx->stream>>>(
        (const float2*)ctx->segpart, (const float2*)ctx->tilepart,
        ctx->seg_begin, ctx->nb, y, ctx->scal, gated);
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace osar
