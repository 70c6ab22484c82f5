// Pixel-space Gram form of Online FISTA for a binary edgelet dictionary H
// (config pixel_gram; the dense dictionaries' products are in
// k_pixgram_dense.cu).
//
// Eqs. 12-13 accumulate G_n = sum_s A_s^H A_s and b_n = sum_s A_s^H d_s with
// A_s = F_s H (Eq. 6), so G_n = H^H P_n H and b_n = H^H b_pix with
// P_n = sum_s F_s^H F_s (N x N) and b_pix = sum_s F_s^H d_s: the pixel-basis
// statistics, which the context keeps with its pixel-basis kernels (phase
// synthesis, data update, Gram update, packed Gram matvec).  Algorithm 1 and
// the power iteration of Eq. 11 then run on the M coefficients with G_n
// applied as three steps: u = H x (per pixel, the sum of x over the atoms
// that cover it), w = P_n u (one pass over the packed P_n), and
// (G_n x)_m = sum of w over atom m's pixels.  P_n holds N^2 entries where
// G_n holds M^2 (a quarter for M = 2N), and the forward block A_s is never
// formed.  The iterates are those of the stored-Gram form up to the order of
// summation.
#include "ctx.h"

#include "finalize.cuh"
#include "step.cuh"

namespace osar {
namespace {

constexpr int PG_THREADS = 256;

// u_p = sum of x_m over the atoms m covering pixel p (list order), in the
// matvec's working precision; 0 on the padding pixels.  gated: nothing once
// the stop rule has been met.
template <typename T2>
__global__ void k_pg_scatter(const double2* __restrict__ x,
                             const int* __restrict__ pix_ptr,
                             const int* __restrict__ pix_atom, int N, int Np,
                             T2* __restrict__ u, const DevScalars* sc,
                             int gated) {
  if (gated && sc->converged) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Np) return;
  double sr = 0.0, si = 0.0;
  if (p < N)
    for (int t = pix_ptr[p]; t < pix_ptr[p + 1]; ++t) {
      const double2 v = x[pix_atom[t]];
      sr += v.x;
      si += v.y;
    }
  T2 o;
  o.x = sr;
  o.y = si;
  u[p] = o;
}

// (H^H w)_m: the sum of w over the pixels of atom m (list order).
__device__ __forceinline__ double2 atom_sum(const double2* __restrict__ w,
                                           const int* __restrict__ atom_ptr,
                                           const int* __restrict__ atom_pix,
                                           int m) {
  double sr = 0.0, si = 0.0;
  for (int t = atom_ptr[m]; t < atom_ptr[m + 1]; ++t) {
    const double2 v = w[atom_pix[t]];
    sr += v.x;
    si += v.y;
  }
  return make_double2(sr, si);
}

// b_n = H^H b_pix; the last CTA sets lambda_n = rel max_m |b_m| (Eq. 11's
// relative rule) or the absolute value.
__global__ void __launch_bounds__(PG_THREADS)
    k_pg_bvec(const double2* __restrict__ bpix, const int* __restrict__ atom_ptr,
              const int* __restrict__ atom_pix, int M, double2* __restrict__ b,
              double* __restrict__ bmax, DevScalars* sc, double lam, int relative) {
  __shared__ double red[PG_THREADS / 32];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double m2 = 0.0;
  if (m < M) {
    const double2 v = atom_sum(bpix, atom_ptr, atom_pix, m);
    b[m] = v;
    m2 = v.x * v.x + v.y * v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < PG_THREADS / 32; ++k) t = fmax(t, red[k]);
    bmax[blockIdx.x] = t;
  }
  if (!last_block(&sc->done, gridDim.x)) return;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) t = fmax(t, __ldcg(bmax + k));
    sc->lambda = relative ? lam * sqrt(t) : lam;
    sc->done = 0;
  }
}

// Power step on the coefficients: w = G_n v from the pass's pixel vector;
// the last CTA forms mu = Re(v^H w), 1/|w| and, on the pulse's last step,
// L_n = max(L_{n-1}, (1 + margin) mu) and tau = 1/L_n.
__global__ void __launch_bounds__(BLK)
    k_pg_power_finalize(const double2* __restrict__ wpix,
                        const int* __restrict__ atom_ptr,
                        const int* __restrict__ atom_pix, int M,
                        const double2* __restrict__ v, double2* __restrict__ w,
                        double2* __restrict__ part, DevScalars* sc,
                        int last_step, double margin) {
  const int idx = blockIdx.x * BLK + threadIdx.x;
  double p0 = 0.0, p1 = 0.0;
  if (idx < M) {
    const double2 y = atom_sum(wpix, atom_ptr, atom_pix, idx);
    w[idx] = y;
    const double2 vk = v[idx];
    p0 = vk.x * y.x + vk.y * y.y;
    p1 = y.x * y.x + y.y * y.y;
  }
  const double2 s = block_sum(p0, p1, BLK / 32);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(&sc->done, gridDim.x)) return;
  const double2 tot = sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    const double mu = tot.x;
    sc->mu = mu;
    sc->inv_norm = tot.y > 0.0 ? 1.0 / sqrt(tot.y) : 0.0;
    if (last_step) {
      const double l = (1.0 + margin) * mu;
      if (l > sc->lip) sc->lip = l;
      sc->tau = sc->lip > 0.0 ? 1.0 / sc->lip : 0.0;
    }
    sc->passes += 1;
    sc->done = 0;
  }
}

// v <- w / |w| (v kept when |w| = 0).
__global__ void k_pg_normalize(const double2* __restrict__ w,
                               double2* __restrict__ v, int n,
                               const DevScalars* __restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double s = sc->inv_norm;
  if (i >= n || s == 0.0) return;
  const double2 y = w[i];
  v[i] = make_double2(y.x * s, y.y * s);
}

// One step of Algorithm 1 on the coefficients, with g = G_n z - b_n formed
// from the pass's pixel vector w = P_n H z:
//   u = z - tau g,  c = S_{lambda tau}(u),  z' = c + (t - 1)/t' (c - c_prev);
// the last CTA advances t, counts the step and applies the stop rule
// |c - z|_2 <= tol |c|_2.
template <typename T2>
__global__ void __launch_bounds__(BLK)
    k_pg_fista_finalize(const double2* __restrict__ wpix,
                        const int* __restrict__ atom_ptr,
                        const int* __restrict__ atom_pix, int M,
                        const double2* __restrict__ b, double2* __restrict__ c,
                        double2* __restrict__ z, double2* __restrict__ part,
                        DevScalars* sc) {
  if (sc->converged) return;
  __shared__ double sh[3];  // tau, alpha, beta
  if (threadIdx.x == 0) {
    const double t = sc->t, tau = sc->tau;
    const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sh[0] = tau;
    sh[1] = sc->lambda * tau;
    sh[2] = (t - 1.0) / t_next;
  }
  __syncthreads();
  const int idx = blockIdx.x * BLK + threadIdx.x;
  double p0 = 0.0, p1 = 0.0;
  if (idx < M) {
    const double tau = sh[0], alpha = sh[1], beta = sh[2];
    const double2 y = atom_sum(wpix, atom_ptr, atom_pix, idx);
    const double2 zk = z[idx], bk = b[idx], cprev = c[idx];
    const double ur = zk.x - tau * (y.x - bk.x);
    const double ui = zk.y - tau * (y.y - bk.y);
    const double keep = shrink_keep<T2>(ur * ur + ui * ui, alpha);
    const double cr = ur * keep, ci = ui * keep;
    c[idx] = make_double2(cr, ci);
    z[idx] = make_double2(cr + beta * (cr - cprev.x), ci + beta * (ci - cprev.y));
    const double dr = cr - zk.x, di = ci - zk.y;
    p0 = dr * dr + di * di;
    p1 = cr * cr + ci * ci;
  }
  const double2 s = block_sum(p0, p1, BLK / 32);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(&sc->done, gridDim.x)) return;
  const double2 tot = sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    const double t = sc->t;
    sc->t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc->iters += 1;
    sc->passes += 1;
    if (sc->tol > 0.0 && sqrt(tot.x) <= sc->tol * sqrt(tot.y)) sc->converged = 1;
    sc->done = 0;
  }
}

// Start of a burst: z = c_hat_{n-1}; t = 1 at the first pulse (or always,
// with restart); the stop flag cleared.
__global__ void k_pg_burst_begin(double2* __restrict__ z,
                                 const double2* __restrict__ c, int n,
                                 DevScalars* sc, int reset_t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = c[i];
  if (i == 0) {
    if (reset_t) sc->t = 1.0;
    sc->converged = 0;
  }
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// u = H x into the matvec's input (the context's pixel working vector);
// u = D x for a dense dictionary.
cudaError_t scatter(osar_ctx* ctx, const double2* x, int gated) {
  const PixGram& g = *ctx->pg;
  if (g.dense) return pgd_forward(ctx, x, gated);
  if (ctx->prec == OSAR_FP64)
    k_pg_scatter<double2><<<blocks(ctx->Np, PG_THREADS), PG_THREADS, 0, ctx->stream>>>(
        x, g.pix_ptr, g.pix_atom, ctx->N, ctx->Np, (double2*)ctx->zt, ctx->scal,
        gated);
  else
    k_pg_scatter<float2><<<blocks(ctx->Np, PG_THREADS), PG_THREADS, 0, ctx->stream>>>(
        x, g.pix_ptr, g.pix_atom, ctx->N, ctx->Np, (float2*)ctx->zt, ctx->scal,
        gated);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_pixgram_kernels() {
  // the burst's matvec runs with the largest shared-memory carve-out; the
  // kernels between its passes ask for the same one (no L1 / shared
  // reconfiguration between launches)
  const int v = cudaSharedmemCarveoutMaxShared;
  const cudaFuncAttribute a = cudaFuncAttributePreferredSharedMemoryCarveout;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, a, v);
  };
  set((const void*)k_pg_scatter<float2>);
  set((const void*)k_pg_scatter<double2>);
  set((const void*)k_pg_fista_finalize<float2>);
  set((const void*)k_pg_fista_finalize<double2>);
  set((const void*)k_pg_power_finalize);
  set((const void*)k_pg_normalize);
  set((const void*)k_pg_bvec);
  set((const void*)k_pg_burst_begin);
  return e;
}

cudaError_t pg_after_push(osar_ctx* ctx) {
  const PixGram& g = *ctx->pg;
  if (g.dense) {
    cudaError_t e = pgd_adjoint(ctx, 0, 0);  // b_n = D^H b_pix, lambda_n
    if (e != cudaSuccess) return e;
  } else {
    k_pg_bvec<<<blocks(g.M, PG_THREADS), PG_THREADS, 0, ctx->stream>>>(
        ctx->b, ctx->atom_ptr, ctx->atom_pix, g.M, g.b, g.bmax, ctx->scal,
        ctx->lam.v[0], ctx->cfg.lambda_relative);
    ctx->launches++;
  }
  const int steps = ctx->n == 1 ? ctx->cfg.power_iters_first : ctx->cfg.power_iters;
  for (int s = 0; s < steps; ++s) {
    cudaError_t e = scatter(ctx, g.v, 0);
    if (e == cudaSuccess) e = launch_gram_pass(ctx, ctx->zt, 0, ctx->w, KCL_POWFIN);
    if (e != cudaSuccess) return e;
    if (g.dense) {
      // D^H w with the power step (profiled as a dictionary product)
      e = pgd_adjoint(ctx, 1, s == steps - 1 ? 1 : 0);
      if (e != cudaSuccess) return e;
      ctx->launches--;  // counted below with the normalisation
    }
    ProfEvent ev;
    prof_begin(ctx, KCL_POWFIN, &ev);
    if (!g.dense) {
      k_pg_power_finalize<<<(unsigned)g.nb, BLK, 0, ctx->stream>>>(
          ctx->w, ctx->atom_ptr, ctx->atom_pix, g.M, g.v, g.w, g.part, ctx->scal,
          s == steps - 1 ? 1 : 0, ctx->cfg.lipschitz_margin);
    }
    k_pg_normalize<<<blocks(g.Mp, PG_THREADS), PG_THREADS, 0, ctx->stream>>>(
        g.w, g.v, g.Mp, ctx->scal);
    prof_end(ctx, &ev);
    ctx->launches += 2;
  }
  return cudaGetLastError();
}

cudaError_t pg_burst_begin(osar_ctx* ctx) {
  const PixGram& g = *ctx->pg;
  const bool reset = ctx->n == 1 || ctx->cfg.restart_momentum;
  k_pg_burst_begin<<<blocks(g.Mp, PG_THREADS), PG_THREADS, 0, ctx->stream>>>(
      g.z, g.c, g.Mp, ctx->scal, reset ? 1 : 0);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t pg_fista_step(osar_ctx* ctx) {
  const PixGram& g = *ctx->pg;
  cudaError_t e = scatter(ctx, g.z, 1);
  if (e == cudaSuccess) e = launch_gram_pass(ctx, ctx->zt, 1, ctx->w, KCL_FIN);
  if (e != cudaSuccess) return e;
  // D^H w with the step (profiled as a dictionary product)
  if (g.dense) return pgd_adjoint(ctx, 2, 0);
  ProfEvent ev;
  prof_begin(ctx, KCL_FIN, &ev);
  if (ctx->prec == OSAR_FP64)
    k_pg_fista_finalize<double2><<<(unsigned)g.nb, BLK, 0, ctx->stream>>>(
        ctx->w, ctx->atom_ptr, ctx->atom_pix, g.M, g.b, g.c, g.z, g.part,
        ctx->scal);
  else
    k_pg_fista_finalize<float2><<<(unsigned)g.nb, BLK, 0, ctx->stream>>>(
        ctx->w, ctx->atom_ptr, ctx->atom_pix, g.M, g.b, g.c, g.z, g.part,
        ctx->scal);
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace osar
