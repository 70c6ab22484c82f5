// Pixel-space Gram form for a dense dictionary D (the Gaussian or a host
// dictionary; config pixel_gram).
//
// As for the edgelets (k_pixgram.cu), Eqs. 12-13 with A_s = F_s D (Eq. 6)
// give G_n = D^H P_n D and b_n = D^H b_pix, with P_n = sum_s F_s^H F_s
// (N x N) and b_pix = sum_s F_s^H d_s kept by the context's pixel-basis
// kernels.  G_n x is applied as u = D x, w = P_n u (one pass over the packed
// P_n) and (D^H w)_m.  P_n has N^2 entries where G_n has M^2 (a quarter for
// M = 2N) and no forward block A_s or dictionary product is formed; each
// application of G_n reads D twice (u = D x and D^H w) besides P_n, so a
// step streams 2 |D| + |P_n| bytes where the stored form streams |G_n|.
//
// Both dictionary products are matrix-vector products: bound by HBM
// bandwidth, so they run on the SIMT pipes with 16-byte loads, not on the
// tensor cores.  D is the context's dictionary in its stored form: split
// planes (re_hi, im_hi, re_lo, im_lo; bf16, re = re_hi + re_lo exactly in
// FP32) for split-BF16, FP32 or FP64 complex otherwise; atom-major rows of
// Np pixels.  Sums run in FP32 on the FP32-Gram paths and in FP64 on the
// FP64 path, each in a fixed order (results do not depend on the grid).
#include "ctx.h"

#include "finalize.cuh"
#include "step.cuh"

namespace osar {
namespace {

constexpr int PD_THREADS = 256;
constexpr int PD_FWD_PIX = PD_THREADS * 8;   // pixels of a forward CTA (8 a thread)
constexpr int PD_FWD_ATOMS = 256;            // most atoms of a forward CTA
constexpr int PD_ATOMS = 64;                 // atoms of an adjoint CTA (8 a warp)
constexpr int PD_CHUNK = 2048;               // pixels of w staged at a time

// Eight consecutive entries D[m][p0 .. p0 + 7] (p0 a multiple of 8) as
// (re, im) in T.
struct DSplit {
  const __nv_bfloat16* d;
  int64_t plane;  // Mp_atoms x Np
  template <typename T>
  __device__ __forceinline__ void load8(int m, int p0, int64_t np, T* er, T* ei) const {
    const int64_t o = (int64_t)m * np + p0;
    const uint4 rh = __ldg(reinterpret_cast<const uint4*>(d + o));
    const uint4 ih = __ldg(reinterpret_cast<const uint4*>(d + plane + o));
    const uint4 rl = __ldg(reinterpret_cast<const uint4*>(d + 2 * plane + o));
    const uint4 il = __ldg(reinterpret_cast<const uint4*>(d + 3 * plane + o));
    const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(&rh);
    const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&ih);
    const __nv_bfloat162* c = reinterpret_cast<const __nv_bfloat162*>(&rl);
    const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&il);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 r0 = __bfloat1622float2(a[k]), r1 = __bfloat1622float2(c[k]);
      const float2 i0 = __bfloat1622float2(b[k]), i1 = __bfloat1622float2(e[k]);
      er[2 * k] = (T)(r0.x + r1.x);
      er[2 * k + 1] = (T)(r0.y + r1.y);
      ei[2 * k] = (T)(i0.x + i1.x);
      ei[2 * k + 1] = (T)(i0.y + i1.y);
    }
  }
};

struct DF32 {
  const float2* d;
  template <typename T>
  __device__ __forceinline__ void load8(int m, int p0, int64_t np, T* er, T* ei) const {
    const float4* q = reinterpret_cast<const float4*>(d + (int64_t)m * np + p0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 v = __ldg(q + k);
      er[2 * k] = (T)v.x;
      ei[2 * k] = (T)v.y;
      er[2 * k + 1] = (T)v.z;
      ei[2 * k + 1] = (T)v.w;
    }
  }
};

struct DF64 {
  const double2* d;
  template <typename T>
  __device__ __forceinline__ void load8(int m, int p0, int64_t np, T* er, T* ei) const {
    const double2* q = d + (int64_t)m * np + p0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double2 v = __ldg(q + k);
      er[k] = (T)v.x;
      ei[k] = (T)v.y;
    }
  }
};

// u = D x, first as partial sums over chunks of `chunk` atoms (at most
// PD_FWD_ATOMS; fewer for small scenes, so that the grid still fills the
// GPU): part[c][p] = sum over chunk c's atoms m (in order) of D[m][p] x_m.
// Padding atoms have zero rows and zero x.  gated: nothing once the stop
// rule has been met.
template <typename S, typename T>
__global__ void __launch_bounds__(PD_THREADS)
    k_pgd_forward(S d, int Mp, int Np, int chunk, const double2* __restrict__ x,
                  typename Vec<T>::T2* __restrict__ part,
                  const DevScalars* sc, int gated) {
  using T2 = typename Vec<T>::T2;
  if (gated && sc->converged) return;
  __shared__ T2 xs[PD_FWD_ATOMS];
  const int a0 = blockIdx.y * chunk;
  const int na = min(chunk, Mp - a0);
  for (int i = threadIdx.x; i < PD_FWD_ATOMS; i += PD_THREADS) {
    T2 v;
    v.x = 0;
    v.y = 0;
    if (i < na) {
      const double2 xv = x[a0 + i];
      v.x = (T)xv.x;
      v.y = (T)xv.y;
    }
    xs[i] = v;
  }
  __syncthreads();
  const int p0 = blockIdx.x * PD_FWD_PIX + threadIdx.x * 8;
  if (p0 >= Np) return;
  T ar[8], ai[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) ar[i] = ai[i] = T(0);
#pragma unroll 4
  for (int k = 0; k < na; ++k) {
    T er[8], ei[8];
    d.template load8<T>(a0 + k, p0, Np, er, ei);
    const T2 xv = xs[k];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      ar[i] = fma(er[i], xv.x, fma(-ei[i], xv.y, ar[i]));
      ai[i] = fma(er[i], xv.y, fma(ei[i], xv.x, ai[i]));
    }
  }
  T2* out = part + (int64_t)blockIdx.y * Np + p0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    T2 v;
    v.x = ar[i];
    v.y = ai[i];
    out[i] = v;
  }
}

// u_p = the chunk partials summed, into the matvec's input vector (working
// precision).  A CTA takes 32 pixels with 8 threads each: thread group g
// sums chunks g, g + 8, ... in order, then the 8 group sums are added in
// group order (a fixed order, independent of the grid).
constexpr int PD_RED_PIX = 32, PD_RED_GROUPS = 8;

template <typename T, typename TW2>
__global__ void __launch_bounds__(PD_RED_PIX * PD_RED_GROUPS)
    k_pgd_reduce(const typename Vec<T>::T2* __restrict__ part, int nchunk,
                 int Np, TW2* __restrict__ u, const DevScalars* sc, int gated) {
  if (gated && sc->converged) return;
  __shared__ T rs[PD_RED_GROUPS][PD_RED_PIX], is[PD_RED_GROUPS][PD_RED_PIX];
  const int px = threadIdx.x % PD_RED_PIX, grp = threadIdx.x / PD_RED_PIX;
  const int p = blockIdx.x * PD_RED_PIX + px;
  T sr = 0, si = 0;
  if (p < Np)
    for (int k = grp; k < nchunk; k += PD_RED_GROUPS) {
      const typename Vec<T>::T2 v = part[(int64_t)k * Np + p];
      sr += v.x;
      si += v.y;
    }
  rs[grp][px] = sr;
  is[grp][px] = si;
  __syncthreads();
  if (grp == 0 && p < Np) {
    T tr = 0, ti = 0;
#pragma unroll
    for (int q = 0; q < PD_RED_GROUPS; ++q) {
      tr += rs[q][px];
      ti += is[q][px];
    }
    TW2 o;
    o.x = tr;
    o.y = ti;
    u[p] = o;
  }
}

enum { PD_BVEC = 0, PD_POWER = 1, PD_FISTA = 2 };

struct PdArgs {
  int M;                      // atoms
  const double2* b;           // b_n (FISTA)
  double2* out;               // b_n (BVEC), w = G v (POWER)
  double2* c;                 // FISTA: c^(k-1) in, c^(k) out
  double2* z;                 // FISTA: z^(k) in, z^(k+1) out
  const double2* v;           // POWER: the unit vector v
  double2* part;              // per-CTA partial sums
  double* bmax;               // BVEC: per-CTA max |b_m|^2
  DevScalars* sc;
  double lam;                 // BVEC: lambda setting
  int relative;
  int last_step;              // POWER: the pulse's last power step
  double margin;
};

// Partial sums of y_m = (D^H w)_m over one chunk of PD_CHUNK pixels for
// the PD_ATOMS atoms of this CTA (8 warps, 8 atoms each; each lane sums its
// pixels in order, then a butterfly over the warp): part[chunk][m].  Tiles
// of (atoms, pixels) keep the grid many waves deep, so no SM idles at the
// end of a pass over D.
template <typename S, typename T>
__global__ void __launch_bounds__(PD_THREADS)
    k_pgd_adjoint(S d, int Np, const double2* __restrict__ w,
                  typename Vec<T>::T2* __restrict__ part, const DevScalars* sc,
                  int gated) {
  using T2 = typename Vec<T>::T2;
  if (gated && sc->converged) return;
  // w staged with PADW padding entries after every 8 pixels: a lane reads
  // its 8 consecutive pixels with 16-byte loads, and the padding puts the 8
  // lanes of each shared-memory wavefront on distinct banks
  constexpr int PADW = sizeof(T) == 4 ? 2 : 1;
  __shared__ __align__(16) T2 ws[PD_CHUNK / 8 * (8 + PADW)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * PD_ATOMS + warp * 8;
  const int c0 = blockIdx.y * PD_CHUNK;
  const int cl = min(PD_CHUNK, Np - c0);
  for (int i = threadIdx.x; i < cl; i += PD_THREADS) {
    const double2 v = w[c0 + i];
    T2 t;
    t.x = (T)v.x;
    t.y = (T)v.y;
    ws[i + (i >> 3) * PADW] = t;
  }
  __syncthreads();
  T ar[8], ai[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) ar[j] = ai[j] = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
#pragma unroll 1
    for (int q = lane * 8; q < cl; q += 256) {
      T er[8], ei[8];
      d.template load8<T>(m0 + j, c0 + q, Np, er, ei);
      const T2* wq = ws + q + (q >> 3) * PADW;
      T2 wl[8];
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 v = reinterpret_cast<const float4*>(wq)[k];
          wl[2 * k].x = v.x;
          wl[2 * k].y = v.y;
          wl[2 * k + 1].x = v.z;
          wl[2 * k + 1].y = v.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) wl[k] = wq[k];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const T2 wv = wl[i];
        // conj(D) w
        ar[j] = fma(er[i], wv.x, fma(ei[i], wv.y, ar[j]));
        ai[j] = fma(er[i], wv.y, fma(-ei[i], wv.x, ai[j]));
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar[j] += __shfl_xor_sync(0xffffffffu, ar[j], o);
      ai[j] += __shfl_xor_sync(0xffffffffu, ai[j], o);
    }
  }
  if (lane == 0) {
    T2* out = part + (int64_t)blockIdx.y * gridDim.x * PD_ATOMS + m0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      T2 v;
      v.x = ar[j];
      v.y = ai[j];
      out[j] = v;
    }
  }
}

// y_m = the chunk partials summed in chunk order (FP64 from here), then per
// MODE: b_n and lambda_n (BVEC), a power step (POWER) or Algorithm 1's step
// (FISTA), each finished by the grid's last CTA as the edgelet form's
// kernels do.  One CTA per 128 atoms.
template <typename T, int MODE>
__global__ void __launch_bounds__(BLK)
    k_pgd_finish(const typename Vec<T>::T2* __restrict__ part, int nchunk,
                 int mp, PdArgs a) {
  if (MODE == PD_FISTA && a.sc->converged) return;
  __shared__ double sh[3];
  if (MODE == PD_FISTA && threadIdx.x == 0) {
    const double t = a.sc->t, tau = a.sc->tau;
    const double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sh[0] = tau;
    sh[1] = a.sc->lambda * tau;
    sh[2] = (t - 1.0) / t_next;
  }
  __syncthreads();
  const int idx = blockIdx.x * BLK + threadIdx.x;
  const bool mine = idx < a.M;
  double2 y = make_double2(0.0, 0.0);
  if (mine) {
    T sr = 0, si = 0;
    for (int k = 0; k < nchunk; ++k) {
      const typename Vec<T>::T2 v = part[(int64_t)k * mp + idx];
      sr += v.x;
      si += v.y;
    }
    y = make_double2((double)sr, (double)si);
  }
  if constexpr (MODE == PD_BVEC) {
    double m2 = 0.0;
    if (mine) {
      a.out[idx] = y;
      m2 = y.x * y.x + y.y * y.y;
    }
    __shared__ double red[BLK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < BLK / 32; ++k) t = fmax(t, red[k]);
      a.bmax[blockIdx.x] = t;
    }
    if (!last_block(&a.sc->done, gridDim.x)) return;
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)gridDim.x; ++k) t = fmax(t, __ldcg(a.bmax + k));
      a.sc->lambda = a.relative ? a.lam * sqrt(t) : a.lam;
      a.sc->done = 0;
    }
  } else if constexpr (MODE == PD_POWER) {
    double p0 = 0.0, p1 = 0.0;
    if (mine) {
      a.out[idx] = y;
      const double2 vk = a.v[idx];
      p0 = vk.x * y.x + vk.y * y.y;
      p1 = y.x * y.x + y.y * y.y;
    }
    const double2 s = block_sum(p0, p1, blockDim.x / 32);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
    if (!last_block(&a.sc->done, gridDim.x)) return;
    const double2 tot = sum_parts(a.part, gridDim.x);
    if (threadIdx.x == 0) {
      DevScalars* sc = a.sc;
      const double mu = tot.x;
      sc->mu = mu;
      sc->inv_norm = tot.y > 0.0 ? 1.0 / sqrt(tot.y) : 0.0;
      if (a.last_step) {
        const double l = (1.0 + a.margin) * mu;
        if (l > sc->lip) sc->lip = l;
        sc->tau = sc->lip > 0.0 ? 1.0 / sc->lip : 0.0;
      }
      sc->passes += 1;
      sc->done = 0;
    }
  } else {
    double p0 = 0.0, p1 = 0.0;
    if (mine) {
      const double tau = sh[0], alpha = sh[1], beta = sh[2];
      const double2 zk = a.z[idx], bk = a.b[idx], cprev = a.c[idx];
      const double ur = zk.x - tau * (y.x - bk.x);
      const double ui = zk.y - tau * (y.y - bk.y);
      const double keep = shrink_keep<typename Vec<T>::T2>(ur * ur + ui * ui, alpha);
      const double cr = ur * keep, ci = ui * keep;
      a.c[idx] = make_double2(cr, ci);
      a.z[idx] = make_double2(cr + beta * (cr - cprev.x), ci + beta * (ci - cprev.y));
      const double dr = cr - zk.x, di = ci - zk.y;
      p0 = dr * dr + di * di;
      p1 = cr * cr + ci * ci;
    }
    const double2 s = block_sum(p0, p1, blockDim.x / 32);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s;
    if (!last_block(&a.sc->done, gridDim.x)) return;
    const double2 tot = sum_parts(a.part, gridDim.x);
    if (threadIdx.x == 0) {
      DevScalars* sc = a.sc;
      const double t = sc->t;
      sc->t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      sc->iters += 1;
      sc->passes += 1;
      if (sc->tol > 0.0 && sqrt(tot.x) <= sc->tol * sqrt(tot.y)) sc->converged = 1;
      sc->done = 0;
    }
  }
}

unsigned cdiv(int64_t n, int64_t t) { return (unsigned)((n + t - 1) / t); }

template <typename F>
cudaError_t with_dict(const osar_ctx* ctx, F&& f) {
  const PixGram& g = *ctx->pg;
  if (ctx->prec == OSAR_SPLIT_BF16)
    return f(DSplit{ctx->Dpl, (int64_t)g.Mp * ctx->Np}, 0.0f);
  if (ctx->prec == OSAR_FP32) return f(DF32{(const float2*)ctx->D}, 0.0f);
  return f(DF64{(const double2*)ctx->D}, 0.0);
}

}  // namespace

// Atoms per forward CTA: the largest of 256, 128, 64, 32 that still gives
// at least four CTAs per SM.
int pgd_fwd_atoms(const osar_ctx* ctx) {
  int a = PD_FWD_ATOMS;
  const int64_t px_tiles = cdiv(ctx->Np, PD_FWD_PIX);
  while (a > 32 && px_tiles * cdiv(ctx->pg->Mp, a) < 4 * (int64_t)ctx->sm_count)
    a /= 2;
  return a;
}

int pgd_chunks(const osar_ctx* ctx) {
  return (int)cdiv(ctx->pg->Mp, pgd_fwd_atoms(ctx));
}

int pgd_adjoint_chunks(const osar_ctx* ctx) {
  return (int)cdiv(ctx->Np, PD_CHUNK);
}

// u = D x into the context's pixel working vector (zt).
cudaError_t pgd_forward(osar_ctx* ctx, const double2* x, int gated) {
  const PixGram& g = *ctx->pg;
  const int nch = pgd_chunks(ctx);
  ProfEvent ev;
  prof_begin(ctx, KCL_DAPPLY, &ev);
  cudaError_t e = with_dict(ctx, [&](auto d, auto zero) {
    using T = decltype(zero);
    using T2 = typename Vec<T>::T2;
    const dim3 grid(cdiv(ctx->Np, PD_FWD_PIX), (unsigned)nch);
    k_pgd_forward<decltype(d), T><<<grid, PD_THREADS, 0, ctx->stream>>>(
        d, g.Mp, ctx->Np, pgd_fwd_atoms(ctx), x, (T2*)g.upart, ctx->scal, gated);
    const unsigned rg = cdiv(ctx->Np, PD_RED_PIX);
    const int rt = PD_RED_PIX * PD_RED_GROUPS;
    if (ctx->prec == OSAR_FP64)
      k_pgd_reduce<T, double2><<<rg, rt, 0, ctx->stream>>>(
          (const T2*)g.upart, nch, ctx->Np, (double2*)ctx->zt, ctx->scal, gated);
    else
      k_pgd_reduce<T, float2><<<rg, rt, 0, ctx->stream>>>(
          (const T2*)g.upart, nch, ctx->Np, (float2*)ctx->zt, ctx->scal, gated);
    return cudaGetLastError();
  });
  prof_end(ctx, &ev);
  ctx->launches += 2;
  return e;
}

// (D^H w)_m and the MODE's work, w the pass's pixel vector (ctx->w).
cudaError_t pgd_adjoint(osar_ctx* ctx, int mode, int last_step) {
  PixGram& g = *ctx->pg;
  PdArgs a;
  a.M = g.M;
  a.b = g.b;
  a.out = mode == PD_BVEC ? g.b : g.w;
  a.c = g.c;
  a.z = g.z;
  a.v = g.v;
  a.part = g.part;
  a.bmax = g.bmax;
  a.sc = ctx->scal;
  a.lam = ctx->lam.v[0];
  a.relative = ctx->cfg.lambda_relative;
  a.last_step = last_step;
  a.margin = ctx->cfg.lipschitz_margin;
  const double2* w = mode == PD_BVEC ? ctx->b : ctx->w;
  const dim3 grid(cdiv(g.Mp, PD_ATOMS), cdiv(ctx->Np, PD_CHUNK));
  const int gated = mode == PD_FISTA ? 1 : 0;
  ProfEvent ev;
  prof_begin(ctx, KCL_DAPPLY, &ev);
  cudaError_t e = with_dict(ctx, [&](auto d, auto zero) {
    using T = decltype(zero);
    using T2 = typename Vec<T>::T2;
    k_pgd_adjoint<decltype(d), T><<<grid, PD_THREADS, 0, ctx->stream>>>(
        d, ctx->Np, w, (T2*)g.apart, ctx->scal, gated);
    const unsigned fg = (unsigned)g.nb;
    const int nch = (int)grid.y, mp = (int)grid.x * PD_ATOMS;
    if (mode == PD_BVEC)
      k_pgd_finish<T, PD_BVEC><<<fg, BLK, 0, ctx->stream>>>((const T2*)g.apart, nch, mp, a);
    else if (mode == PD_POWER)
      k_pgd_finish<T, PD_POWER><<<fg, BLK, 0, ctx->stream>>>((const T2*)g.apart, nch, mp, a);
    else
      k_pgd_finish<T, PD_FISTA><<<fg, BLK, 0, ctx->stream>>>((const T2*)g.apart, nch, mp, a);
    return cudaGetLastError();
  });
  prof_end(ctx, &ev);
  ctx->launches += 2;
  return e;
}

}  // namespace osar
