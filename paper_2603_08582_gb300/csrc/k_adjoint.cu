// Differentiation form: reverse-mode adjoint of T unrolled steps of
// Algorithm 1's inner loop on the context's Gram A_n and data vector b_n.
//
// Forward map (z_1 = c_0, t_1 = t0):
//   g_k = A z_k - b,  u_k = z_k - tau g_k,  c_k = S_alpha(u_k), alpha = lambda tau,
//   z_{k+1} = (1 + beta_k) c_k - beta_k c_{k-1},  beta_k = (t_k - 1) / t_{k+1},
// loss L = |c_T - c_true|^2.  Complex adjoints use the convention
// dL/dRe + i dL/dIm.  With cbar_T = 2 (c_T - c_true) the reverse step k is
//   ubar_k = J_S(u_k)^T cbar_k   (J_S = (1 - alpha/|u|) I + (alpha/|u|) uhat uhat^T
//                                 for |u| > alpha, else 0; J_S is symmetric)
//   alphabar += -<uhat, cbar_k>,  taubar += -<g_k, ubar_k>,  bbar += tau ubar_k,
//   zbar_k = ubar_k - tau A ubar_k                     (A Hermitian)
//   cbar_{k-1} = carry + (1 + beta_{k-1}) zbar_k,  carry <- -beta_{k-1} zbar_k,
// and finally dL/dlambda = alphabar tau, dL/dtau = taubar + alphabar lambda.
// <x, y> is the real inner product Re(sum conj(x) y).
//
// Memory: every `ckpt` steps the forward pass stores (z_k, c_{k-1}); the
// reverse sweep recomputes each segment from its checkpoint while recording
// (u_k, g_k), then walks it backwards.  Each step costs three Gram passes in
// all (forward, recompute, adjoint), the matvec being the same bandwidth-bound
// kernel as the FISTA step; the elementwise kernels below are the adjoint.
#include <cmath>
#include <vector>

#include "finalize.cuh"

namespace osar {
namespace {

struct AdjScalars {
  double alphabar;
  double taubar;
  double loss;
  unsigned done;
  unsigned pad;
};

// Forward step with optional recording of (u_k, g_k).
template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS)
    k_unroll_fwd(const T2* __restrict__ segpart, const T2* __restrict__ tilepart,
                 const int* __restrict__ seg_begin, int nb,
                 const double2* __restrict__ b, double2* __restrict__ z,
                 T2* __restrict__ zt, double2* __restrict__ cprev,
                 double2* __restrict__ u_rec, double2* __restrict__ g_rec,
                 const double* __restrict__ prm, int k) {
  const int K = blockIdx.x, i = threadIdx.x, idx = K * BLK + i;
  const double2 y = gather_row<T2, Acc>(segpart, tilepart, seg_begin, nb, K);
  if (i >= BLK) return;
  const double tau = prm[0], alpha = prm[1], beta = prm[2 + k];
  const double2 zk = z[idx], bk = b[idx], cp = cprev[idx];
  const double gr = y.x - bk.x, gi = y.y - bk.y;
  const double ur = zk.x - tau * gr, ui = zk.y - tau * gi;
  const double mag = hypot(ur, ui);
  const double keep = mag > alpha ? 1.0 - alpha / mag : 0.0;
  const double cr = ur * keep, ci = ui * keep;
  const double2 zn = make_double2(cr + beta * (cr - cp.x), ci + beta * (ci - cp.y));
  if (u_rec) {
    u_rec[idx] = make_double2(ur, ui);
    g_rec[idx] = make_double2(gr, gi);
  }
  cprev[idx] = make_double2(cr, ci);
  z[idx] = zn;
  T2 t;
  t.x = zn.x;
  t.y = zn.y;
  zt[idx] = t;
}

// Loss |c_T - c_true|^2 and cbar_T = 2 (c_T - c_true).
__global__ void __launch_bounds__(256)
    k_unroll_loss(const double2* __restrict__ c, const double2* __restrict__ ct,
                  double2* __restrict__ cbar, int n, double2* __restrict__ part,
                  AdjScalars* as) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    const double dr = c[i].x - ct[i].x, di = c[i].y - ct[i].y;
    cbar[i] = make_double2(2.0 * dr, 2.0 * di);
    s += dr * dr + di * di;
  }
  const double2 bs = block_sum(s, 0.0, blockDim.x / 32);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
  if (!last_block(&as->done, gridDim.x)) return;
  const double2 tot = sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    as->loss = tot.x;
    as->done = 0;
  }
}

// Adjoint of the shrinkage and of the gradient step (first half of reverse
// step k): ubar = J_S(u)^T cbar, the alpha and tau partials, bbar += tau ubar.
template <typename T2>
__global__ void __launch_bounds__(256)
    k_adj_shrink(const double2* __restrict__ u, const double2* __restrict__ g,
                 const double2* __restrict__ cbar, double2* __restrict__ ubar,
                 T2* __restrict__ ubar_t, double2* __restrict__ bbar, int n,
                 const double* __restrict__ prm, double2* __restrict__ part,
                 AdjScalars* as) {
  const double tau = prm[0], alpha = prm[1];
  double pa = 0.0, pt = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    const double2 uk = u[i], cb = cbar[i];
    const double mag = hypot(uk.x, uk.y);
    double2 ub = make_double2(0.0, 0.0);
    if (mag > alpha) {
      const double hr = uk.x / mag, hi = uk.y / mag;
      const double proj = hr * cb.x + hi * cb.y;  // <uhat, cbar>
      const double s = alpha / mag;
      ub = make_double2((1.0 - s) * cb.x + s * hr * proj,
                        (1.0 - s) * cb.y + s * hi * proj);
      pa -= proj;
    }
    const double2 gk = g[i];
    pt -= gk.x * ub.x + gk.y * ub.y;
    ubar[i] = ub;
    T2 t;
    t.x = ub.x;
    t.y = ub.y;
    ubar_t[i] = t;
    const double2 bb = bbar[i];
    bbar[i] = make_double2(bb.x + tau * ub.x, bb.y + tau * ub.y);
  }
  const double2 s = block_sum(pa, pt, blockDim.x / 32);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!last_block(&as->done, gridDim.x)) return;
  const double2 tot = sum_parts(part, gridDim.x);
  if (threadIdx.x == 0) {
    as->alphabar += tot.x;
    as->taubar += tot.y;
    as->done = 0;
  }
}

// Second half of reverse step k: zbar = ubar - tau A ubar, then the momentum
// adjoint cbar_{k-1} = carry + (1 + beta_{k-1}) zbar, carry = -beta_{k-1} zbar.
template <typename T2, typename Acc>
__global__ void __launch_bounds__(FIN_THREADS)
    k_adj_momentum(const T2* __restrict__ segpart, const T2* __restrict__ tilepart,
                   const int* __restrict__ seg_begin, int nb,
                   const double2* __restrict__ ubar, double2* __restrict__ cbar,
                   double2* __restrict__ carry, const double* __restrict__ prm,
                   int k) {
  const int K = blockIdx.x, i = threadIdx.x, idx = K * BLK + i;
  const double2 y = gather_row<T2, Acc>(segpart, tilepart, seg_begin, nb, K);
  if (i >= BLK) return;
  const double tau = prm[0], beta_prev = prm[2 + k - 1];
  const double2 ub = ubar[idx], cr = carry[idx];
  const double zr = ub.x - tau * y.x, zi = ub.y - tau * y.y;
  cbar[idx] = make_double2(cr.x + (1.0 + beta_prev) * zr, cr.y + (1.0 + beta_prev) * zi);
  carry[idx] = make_double2(-beta_prev * zr, -beta_prev * zi);
}

template <typename T2>
__global__ void k_copy_working(const double2* __restrict__ x, T2* __restrict__ xt,
                               int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    T2 t;
    t.x = x[i].x;
    t.y = x[i].y;
    xt[i] = t;
  }
}

constexpr int ADJ_BLOCKS = 256;

struct Buffers {
  double2 *z, *cprev, *ck_z, *ck_c, *urec, *grec, *cbar, *carry, *ubar, *bbar,
      *ctr, *part, *cT;
  void *zt, *ubar_t;
  AdjScalars* as;
  double* prm;  // tau, alpha = lambda tau, beta_0 .. beta_{T+1}
};

// The whole device sequence of one gradient: forward pass with checkpoints,
// loss, reverse sweep.  Only device work (kernels and device-to-device
// copies) on ctx->stream, every scalar read from B.prm, so that it can be
// captured once into a CUDA graph and replayed for later gradients.
template <typename T2, typename Acc>
cudaError_t unroll_impl(osar_ctx* ctx, const Buffers& B, int T, int C) {
  const int64_t Mp = ctx->Mp;
  const size_t vec = sizeof(double2) * Mp;
  const int nck = (T + C - 1) / C;
  const unsigned g = (unsigned)((Mp + 255) / 256);
  cudaStream_t st = ctx->stream;
  T2* zt = (T2*)B.zt;
  T2* ubar_t = (T2*)B.ubar_t;
  cudaError_t e;
  auto fwd = [&](int k, double2* u, double2* gg) -> cudaError_t {
    cudaError_t x = launch_matvec(ctx, zt);
    if (x != cudaSuccess) return x;
    k_unroll_fwd<T2, Acc><<<(unsigned)ctx->nb, FIN_THREADS, 0, st>>>(
        (const T2*)ctx->segpart, (const T2*)ctx->tilepart, ctx->seg_begin,
        ctx->nb, ctx->b, B.z, zt, B.cprev, u, gg, B.prm, k);
    ctx->launches++;
    return cudaGetLastError();
  };
  k_copy_working<T2><<<g, 256, 0, st>>>(B.z, zt, (int)Mp);
  ctx->launches++;
  // forward pass with checkpoints every C steps
  for (int k = 1; k <= T; ++k) {
    if ((k - 1) % C == 0) {
      const int j = (k - 1) / C;
      if ((e = cudaMemcpyAsync(B.ck_z + j * Mp, B.z, vec, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(B.ck_c + j * Mp, B.cprev, vec, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    }
    if ((e = fwd(k, nullptr, nullptr)) != cudaSuccess) return e;
  }
  if ((e = cudaMemcpyAsync(B.cT, B.cprev, vec, cudaMemcpyDeviceToDevice, st)) !=
      cudaSuccess)
    return e;
  k_unroll_loss<<<ADJ_BLOCKS, 256, 0, st>>>(B.cprev, B.ctr, B.cbar, (int)Mp,
                                            B.part, B.as);
  ctx->launches++;
  // reverse sweep, one checkpointed segment at a time
  for (int j = nck - 1; j >= 0; --j) {
    const int k0 = j * C + 1, k1 = std::min(k0 + C - 1, T);
    if ((e = cudaMemcpyAsync(B.z, B.ck_z + j * Mp, vec, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(B.cprev, B.ck_c + j * Mp, vec, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    k_copy_working<T2><<<g, 256, 0, st>>>(B.z, zt, (int)Mp);
    ctx->launches++;
    for (int k = k0; k <= k1; ++k)
      if ((e = fwd(k, B.urec + (k - k0) * Mp, B.grec + (k - k0) * Mp)) != cudaSuccess)
        return e;
    for (int k = k1; k >= k0; --k) {
      k_adj_shrink<T2><<<ADJ_BLOCKS, 256, 0, st>>>(
          B.urec + (k - k0) * Mp, B.grec + (k - k0) * Mp, B.cbar, B.ubar, ubar_t,
          B.bbar, (int)Mp, B.prm, B.part, B.as);
      ctx->launches++;
      if (k == 1) break;  // z_1 = c_0: nothing earlier depends on lambda, tau, b
      if ((e = launch_matvec(ctx, ubar_t)) != cudaSuccess) return e;
      k_adj_momentum<T2, Acc><<<(unsigned)ctx->nb, FIN_THREADS, 0, st>>>(
          (const T2*)ctx->segpart, (const T2*)ctx->tilepart, ctx->seg_begin,
          ctx->nb, B.ubar, B.cbar, B.carry, B.prm, k);
      ctx->launches++;
    }
  }
  return cudaGetLastError();
}

// Runs the gradient's device sequence.  The sequence depends only on
// (T, C, the precision, the scratch buffer) and reads every scalar from the
// device, so it is captured once into a CUDA graph and replayed: one launch
// instead of some 8 per step (T = 64: ~470 kernels and 30 copies).  A stream
// that is already being captured runs the sequence as it is.
cudaError_t run_sequence(osar_ctx* ctx, const Buffers& B, int T, int C,
                         size_t buf_bytes) {
  auto eager = [&]() {
    return ctx->prec == OSAR_FP64 ? unroll_impl<double2, double>(ctx, B, T, C)
                                  : unroll_impl<float2, float>(ctx, B, T, C);
  };
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(ctx->stream, &cs);
  if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return eager();
  AdjGraph& g = ctx->adj_graph;
  if (!g.exec || g.T != T || g.C != C || g.buf != ctx->adj_buf ||
      g.bytes != buf_bytes) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    const bool prof = ctx->prof_on;
    ctx->prof_on = false;  // no profiling events inside the graph
    const int64_t l0 = ctx->launches;
    e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
    cudaError_t ei = e == cudaSuccess ? eager() : e;
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamEndCapture(ctx->stream, &graph);
    if (e == cudaSuccess) e = ei;
    ctx->prof_on = prof;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return e;
    }
    g.kernels = ctx->launches - l0;
    ctx->launches = l0;
    g.T = T;
    g.C = C;
    g.buf = ctx->adj_buf;
    g.bytes = buf_bytes;
  }
  ctx->launches += g.kernels;
  return cudaGraphLaunch(g.exec, ctx->stream);
}

}  // namespace

cudaError_t run_unroll_grad(osar_ctx* ctx, int T, int C, double lambda,
                            double tau, double t0, const double* c0,
                            const double* ctrue, double* loss, double* dlam,
                            double* dtau, double* db, double* cT) {
  const int64_t Mp = ctx->Mp;
  const int nck = (T + C - 1) / C;
  const size_t vec = sizeof(double2) * Mp;
  const size_t wvec = (ctx->prec == OSAR_FP64 ? 16 : 8) * Mp;
  const size_t need = (vec + 256) * (2 * (size_t)nck + 2 * (size_t)C + 10) +
                      2 * (wvec + 256) + sizeof(double2) * ADJ_BLOCKS + 1024 +
                      sizeof(double) * ((size_t)T + 4) + 256;
  if (ctx->adj_bytes < need) {
    if (ctx->adj_buf) {
      cudaFree(ctx->adj_buf);
      auto& rg = ctx->guards.regions;  // the freed buffer's guard goes too
      for (size_t i = 0; i < rg.size(); ++i)
        if (rg[i].name == "ctx->adj_buf") {
          rg.erase(rg.begin() + (std::ptrdiff_t)i);
          break;
        }
    }
    ctx->adj_buf = nullptr;
    ctx->adj_bytes = 0;
    cudaError_t e = guarded_malloc(ctx->guards, &ctx->adj_buf, need, "ctx->adj_buf",
                                   ctx->stream, nullptr);
    if (e != cudaSuccess) return e;
    ctx->adj_bytes = need;
  }
  char* p = static_cast<char*>(ctx->adj_buf);
  auto take = [&](size_t b) {
    char* r = p;
    p += (b + 255) / 256 * 256;
    return r;
  };
  Buffers B;
  B.z = (double2*)take(vec);
  B.cprev = (double2*)take(vec);
  B.ck_z = (double2*)take(vec * nck);
  B.ck_c = (double2*)take(vec * nck);
  B.urec = (double2*)take(vec * C);
  B.grec = (double2*)take(vec * C);
  B.cbar = (double2*)take(vec);
  B.carry = (double2*)take(vec);
  B.ubar = (double2*)take(vec);
  B.bbar = (double2*)take(vec);
  B.ctr = (double2*)take(vec);
  B.zt = take(wvec);
  B.ubar_t = take(wvec);
  B.part = (double2*)take(sizeof(double2) * ADJ_BLOCKS);
  B.as = (AdjScalars*)take(sizeof(AdjScalars));
  B.cT = (double2*)take(vec);
  B.prm = (double*)take(sizeof(double) * ((size_t)T + 4));

  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  ok(cudaMemsetAsync(B.z, 0, vec, st));
  ok(cudaMemsetAsync(B.ctr, 0, vec, st));
  ok(cudaMemcpyAsync(B.z, c0, sizeof(double2) * ctx->M, cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(B.ctr, ctrue, sizeof(double2) * ctx->M, cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(B.cprev, B.z, vec, cudaMemcpyDeviceToDevice, st));
  ok(cudaMemsetAsync(B.carry, 0, vec, st));
  ok(cudaMemsetAsync(B.bbar, 0, vec, st));
  ok(cudaMemsetAsync(B.as, 0, sizeof(AdjScalars), st));
  if (e != cudaSuccess) return e;

  // the step's scalars on the host: tau, alpha = lambda tau, and the
  // momentum weights from t_1 = t0, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
  std::vector<double> prm((size_t)T + 4, 0.0);
  prm[0] = tau;
  prm[1] = lambda * tau;
  double t = t0;
  for (int k = 1; k <= T; ++k) {
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    prm[2 + k] = (t - 1.0) / tn;  // beta_k
    t = tn;
  }
  ok(cudaMemcpyAsync(B.prm, prm.data(), sizeof(double) * prm.size(),
                     cudaMemcpyHostToDevice, st));
  if (e != cudaSuccess) return e;
  e = run_sequence(ctx, B, T, C, need);
  if (e != cudaSuccess) return e;
  AdjScalars hs;
  ok(cudaMemcpyAsync(&hs, B.as, sizeof(hs), cudaMemcpyDeviceToHost, st));
  if (cT) ok(cudaMemcpyAsync(cT, B.cT, sizeof(double2) * ctx->M, cudaMemcpyDeviceToHost, st));
  if (db) ok(cudaMemcpyAsync(db, B.bbar, sizeof(double2) * ctx->M, cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return e;
  if (loss) *loss = hs.loss;
  if (dlam) *dlam = hs.alphabar * tau;
  if (dtau) *dtau = hs.taubar + hs.alphabar * lambda;
  return cudaSuccess;
}

}  // namespace osar
