// libosar C ABI: context management and the per-pulse / per-burst call
// sequences of Online FISTA (Eqs. 12-13 and Algorithm 1).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ctx.h"
#include "trace.h"

using namespace osar;

namespace {

constexpr int RING = osar_ctx::RING;

thread_local std::string g_create_error;

osar_status fail(osar_ctx* ctx, osar_status st, const std::string& msg) {
  if (ctx) {
    ctx->last_error = msg;
    if (st == OSAR_E_CUDA) ctx->sticky = OSAR_E_CUDA;
  } else {
    g_create_error = msg;
  }
  return st;
}

osar_status cuda_fail(osar_ctx* ctx, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
  return fail(ctx, e == cudaErrorMemoryAllocation ? OSAR_E_OOM : OSAR_E_CUDA,
              msg);
}

#define CK(ctx, expr)                                    \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
  } while (0)

int64_t roundup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

bool is_finite(double v) { return std::isfinite(v); }

template <typename T>
osar_status dev_alloc(osar_ctx* ctx, T** p, size_t bytes, const char* name) {
  size_t total = 0;
  cudaError_t e = guarded_malloc(ctx->guards, (void**)p, bytes, name,
                                 ctx->stream, &total);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
  ctx->dev_bytes += (int64_t)total;
  return OSAR_OK;
}

void free_all(osar_ctx* ctx) {
  void* ptrs[] = {ctx->scal, ctx->b, ctx->c, ctx->z, ctx->v, ctx->w, ctx->xtmp,
                  ctx->part, ctx->d_dev, ctx->turns, ctx->g_hi, ctx->g_lo,
                  ctx->segpart, ctx->tilepart, ctx->segs, ctx->seg_begin,
                  ctx->zt, ctx->vt, ctx->xt, ctx->bmax, ctx->d32,
                  ctx->gram_tiles, ctx->dict_tiles, ctx->A, ctx->F, ctx->D,
                  ctx->Apl, ctx->Fpl, ctx->Dpl, ctx->sim_rho, ctx->sim_nz,
                  ctx->sim_idx, ctx->sim_d, ctx->dict_part, ctx->gram_pairs,
                  ctx->dict_pairs, ctx->segpart2, ctx->tilepart2,
                  ctx->segpart_x, ctx->tilepart_x, ctx->gn_hi, ctx->gn_lo,
                  ctx->Apl_alt, ctx->corr, ctx->corr_u, ctx->corr_tick,
                  ctx->atom_ptr, ctx->atom_pix, ctx->wk_dev, ctx->gp_col,
                  ctx->gp_row, ctx->metrics_buf, ctx->gram_ref};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->pg) {
    const PixGram& g = *ctx->pg;
    for (void* p : {(void*)g.pix_ptr, (void*)g.pix_atom, (void*)g.c, (void*)g.z,
                    (void*)g.b, (void*)g.v, (void*)g.w, (void*)g.part,
                    (void*)g.bmax, g.upart, g.apart})
      if (p) cudaFree(p);
    delete ctx->pg;
    ctx->pg = nullptr;
  }
  if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
  if (ctx->h_wring) cudaFreeHost(ctx->h_wring);
  for (cudaEvent_t ev : ctx->w_ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->adj_graph.exec) cudaGraphExecDestroy(ctx->adj_graph.exec);
  if (ctx->adj_buf) cudaFree(ctx->adj_buf);
  for (int i = 0; i < RING; ++i)
    if (ctx->ring_ev[i]) cudaEventDestroy(ctx->ring_ev[i]);
  if (ctx->h_iters) cudaFreeHost(ctx->h_iters);
  for (cudaEvent_t ev : {ctx->ev_free, ctx->ev_synth, ctx->ev_gram, ctx->ev_steps,
                         ctx->ev_mark[0], ctx->ev_mark[1]})
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : ctx->ev_iters)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : ctx->copy_ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  for (auto& pe : ctx->prof_pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (auto ev : ctx->ev_pool) cudaEventDestroy(ev);
}

osar_status check_usable(osar_ctx* ctx) {
  if (!ctx) return OSAR_E_INVALID;
  if (ctx->sticky != OSAR_OK) return ctx->sticky;
  return OSAR_OK;
}

osar_status validate(const osar_config* c, std::string* why) {
  if (!c) return *why = "config is NULL", OSAR_E_INVALID;
  if (c->nx < 1 || c->ny < 1) return *why = "nx, ny must be >= 1", OSAR_E_INVALID;
  if ((int64_t)c->nx * c->ny > (1 << 20))
    return *why = "nx * ny exceeds 2^20 pixels", OSAR_E_INVALID;
  if (!is_finite(c->pixel_m) || c->pixel_m <= 0)
    return *why = "pixel_m must be finite and > 0", OSAR_E_INVALID;
  if (c->n_freq < 1 || c->n_freq > 16384)
    return *why = "n_freq must be in [1, 16384]", OSAR_E_INVALID;
  if (!is_finite(c->f_lo_hz) || !is_finite(c->f_hi_hz) || c->f_lo_hz <= 0 ||
      c->f_hi_hz < c->f_lo_hz)
    return *why = "need 0 < f_lo_hz <= f_hi_hz", OSAR_E_INVALID;
  if (c->precision < OSAR_FP64 || c->precision > OSAR_SPLIT_BF16)
    return *why = "unknown precision", OSAR_E_INVALID;
  if (c->dict_kind < OSAR_DICT_IDENTITY || c->dict_kind > OSAR_DICT_EDGELET)
    return *why = "unknown dict_kind", OSAR_E_INVALID;
  if (c->dict_kind == OSAR_DICT_EDGELET) {
    const int nl = c->n_edgelet_lengths, na = c->n_edgelet_angles;
    if (nl < 1 || nl > 16 || na < 1 || na > 16 || !c->edgelet_lengths ||
        !c->edgelet_angles_deg)
      return *why = "edgelets need 1..16 lengths and 1..16 angles", OSAR_E_INVALID;
    for (int i = 0; i < nl; ++i)
      if (c->edgelet_lengths[i] < 1 || c->edgelet_lengths[i] > 64)
        return *why = "edgelet lengths must be in [1, 64]", OSAR_E_INVALID;
    for (int i = 0; i < na; ++i) {
      const double a = c->edgelet_angles_deg[i];
      if (!is_finite(a) || a < 0 || a >= 360 || std::fmod(a, 45.0) != 0.0)
        return *why = "edgelet angles must be multiples of 45 in [0, 360)",
               OSAR_E_INVALID;
    }
    const int64_t m = (int64_t)nl * na * c->nx * c->ny;
    if ((int64_t)c->nx * c->ny > 131072 || m > 262144)
      return *why = "edgelet dictionaries are limited to 131072 pixels and "
                    "262144 atoms", OSAR_E_INVALID;
    if (c->n_atoms != 0 && c->n_atoms != m)
      return *why = "edgelets: n_atoms must be 0 or lengths x angles x pixels",
             OSAR_E_INVALID;
  } else if (c->dict_kind != OSAR_DICT_IDENTITY) {
    if (c->n_atoms < 1 || c->n_atoms > 131072)
      return *why = "n_atoms must be in [1, 131072]", OSAR_E_INVALID;
    if (c->dict_kind == OSAR_DICT_HOST && !c->dict_c128)
      return *why = "dict_c128 is NULL", OSAR_E_INVALID;
  } else if ((int64_t)c->nx * c->ny > 131072) {
    return *why = "pixel-basis scenes are limited to 131072 pixels", OSAR_E_INVALID;
  }
  if (!is_finite(c->lambda) || c->lambda < 0)
    return *why = "lambda must be finite and >= 0", OSAR_E_INVALID;
  if (c->power_iters_first < 1 || c->power_iters < 0)
    return *why = "need power_iters_first >= 1 and power_iters >= 0", OSAR_E_INVALID;
  if (!is_finite(c->lipschitz_margin) || c->lipschitz_margin < 0)
    return *why = "lipschitz_margin must be finite and >= 0", OSAR_E_INVALID;
  if (c->overlap_synthesis != 0 && c->overlap_synthesis != 1)
    return *why = "overlap_synthesis must be 0 or 1", OSAR_E_INVALID;
  if (c->synth_ctas < 0) return *why = "synth_ctas must be >= 0", OSAR_E_INVALID;
  if (c->tc_pairs < 0 || c->tc_pairs > 3)
    return *why = "tc_pairs must be in [0, 3]", OSAR_E_INVALID;
  if (c->fuse_first_step != 0 && c->fuse_first_step != 1)
    return *why = "fuse_first_step must be 0 or 1", OSAR_E_INVALID;
  if (c->fuse_power_gram != 0 && c->fuse_power_gram != 1)
    return *why = "fuse_power_gram must be 0 or 1", OSAR_E_INVALID;
  if (c->pixel_gram != 0 && c->pixel_gram != 1)
    return *why = "pixel_gram must be 0 or 1", OSAR_E_INVALID;
  if (c->gram_superblock < 0 || c->gram_superblock > 64)
    return *why = "gram_superblock must be in [0, 64]", OSAR_E_INVALID;
  if (c->pixel_gram &&
      (c->dict_kind == OSAR_DICT_IDENTITY || c->n_lambdas != 1 || c->defer_gram))
    return *why = "pixel_gram needs a dictionary (edgelet, Gaussian or host), "
                  "one lambda and defer_gram = 0", OSAR_E_INVALID;
  if (c->n_lambdas < 1 || c->n_lambdas > MAX_LAMBDAS)
    return *why = "n_lambdas must be in [1, 8]", OSAR_E_INVALID;
  if (c->n_lambdas > 1) {
    if (!c->lambda_list) return *why = "lambda_list is NULL", OSAR_E_INVALID;
    for (int l = 0; l < c->n_lambdas; ++l)
      if (!is_finite(c->lambda_list[l]) || c->lambda_list[l] < 0)
        return *why = "lambda_list values must be finite and >= 0", OSAR_E_INVALID;
  }
  if (c->guard_bytes < 0 || c->guard_bytes > (1 << 20) || c->guard_bytes % 256)
    return *why = "guard_bytes must be a multiple of 256 in [0, 1 MiB]", OSAR_E_INVALID;
  if (c->defer_gram != 0 && c->defer_gram != 1)
    return *why = "defer_gram must be 0 or 1", OSAR_E_INVALID;
  if (c->defer_gram &&
      (c->precision != OSAR_SPLIT_BF16 || c->dict_kind == OSAR_DICT_IDENTITY ||
       !c->overlap_synthesis || c->n_lambdas != 1 || c->n_freq > 2048))
    return *why = "defer_gram needs SPLIT_BF16, a dictionary, overlap_synthesis, "
                  "one lambda and n_freq <= 2048", OSAR_E_INVALID;
  if (c->gram_ahead < 0 || c->gram_ahead > 2)
    return *why = "gram_ahead must be 0, 1 or 2", OSAR_E_INVALID;
  if (c->gram_ahead &&
      (c->precision != OSAR_SPLIT_BF16 || !c->overlap_synthesis || c->defer_gram ||
       c->pixel_gram))
    return *why = "gram_ahead needs SPLIT_BF16, overlap_synthesis, defer_gram = 0 "
                  "and pixel_gram = 0", OSAR_E_INVALID;
  return OSAR_OK;
}

void build_tables(osar_ctx* ctx, std::vector<int4>& segs,
                  std::vector<int>& seg_begin, std::vector<int4>& gram_tiles,
                  std::vector<int4>& dict_tiles, std::vector<int4>& gram_pairs,
                  std::vector<int4>& dict_pairs) {
  const int nb = ctx->nb;
  // matvec segments: runs of S blocks of one block column
  int64_t target = (int64_t)ctx->sm_count * 2 * 12;
  int S = (int)(ctx->nblk / (target > 0 ? target : 1));
  if (S < 1) S = 1;
  if (S > 16) S = 16;
  seg_begin.assign(nb + 1, 0);
  for (int J = 0; J < nb; ++J) {
    seg_begin[J] = (int)segs.size();
    for (int I0 = 0; I0 <= J; I0 += S) {
      int I1 = I0 + S < J + 1 ? I0 + S : J + 1;
      segs.push_back(make_int4(J, I0, I1, (int)segs.size()));
    }
  }
  seg_begin[nb] = (int)segs.size();
  // Hand the segments out from the last block column down: the longest
  // columns go first and the one-block columns last, which evens out the
  // pass's tail.  The partial slots (.w) keep the column order that
  // seg_begin indexes.
  std::reverse(segs.begin(), segs.end());
  // Gram tiles: upper blocks grouped in SB x SB super-blocks so that the
  // CTAs running at the same time share operand rows in L2.  The default is
  // 32 for the update on the whole GPU, 16 when it runs ahead on part of it
  // beside a burst (128 x 128 / M = 32768 on 84 SMs: 8.5-8.7 ms per update
  // against 8.8-8.9 with 32 and 9.1-9.3 with 64).
  const int SB = ctx->cfg.gram_superblock > 0 ? ctx->cfg.gram_superblock
                                              : (ctx->cfg.gram_ahead ? 16 : 32);
  for (int bi = 0; bi < nb; bi += SB)
    for (int bj = bi; bj < nb; bj += SB)
      for (int I = bi; I < bi + SB && I < nb; ++I)
        for (int J = (bj > I ? bj : I); J < bj + SB && J < nb; ++J)
          gram_tiles.push_back(
              make_int4(I, J, (int)packed_block(I, J, nb), 0));
  // The same super-blocks for CTA pairs: rows I0 and I0 + 1 of one block
  // column J share B; on the diagonal an even I0 == J has no partner.
  for (int bi = 0; bi < nb; bi += SB)
    for (int bj = bi; bj < nb; bj += SB)
      for (int J = bj; J < bj + SB && J < nb; ++J)
        for (int I0 = bi; I0 < bi + SB && I0 <= J; I0 += 2) {
          const bool single = I0 + 1 > J;
          gram_pairs.push_back(
              make_int4(I0, J, single ? I0 : I0 + 1, single ? 1 : 0));
        }
  if (ctx->dict) {
    // Split-K slices (tensor-core path only) one after another: the tiles
    // in flight together share one slice of the phase operand F (6 planes x
    // Kp x 4096 pixels, 25 MB at K = 512), which stays in L2 however many
    // SMs the product gets; the frequency tiles of one atom block are
    // adjacent, so its dictionary rows come from HBM once.
    const int S = ctx->prec == OSAR_SPLIT_BF16 ? ctx->dict_slices : 1;
    for (int sl = 0; sl < S; ++sl)
      for (int I = 0; I < nb; ++I)
        for (int J = 0; J < ctx->Kp / BLK; ++J)
          dict_tiles.push_back(make_int4(I, J | (sl << 16), 0, 0));
    for (int sl = 0; sl < S; ++sl)
      for (int I0 = 0; I0 < nb; I0 += 2)
        for (int J = 0; J < ctx->Kp / BLK; ++J) {
          const bool single = I0 + 1 >= nb;
          dict_pairs.push_back(make_int4(I0, J | (sl << 16),
                                         single ? I0 : I0 + 1, single ? 1 : 0));
        }
  }
}

// Pixel lists of the edgelet atoms (§III-A): atom m = (length index x
// angles + angle index) x N + y x nx + x covers the centre (x, y) plus
// j - (l - 1) / 2 steps of (dx, dy) for j = 0 .. l - 1, pixels off the grid
// dropped; (dx, dy) = (round(cos psi), round(sin psi)) for psi = 45 s.
void build_edgelets(const osar_config& c, std::vector<int>& ptr,
                    std::vector<int>& pix) {
  static const int DX[8] = {1, 1, 0, -1, -1, -1, 0, 1};
  static const int DY[8] = {0, 1, 1, 1, 0, -1, -1, -1};
  ptr.assign(1, 0);
  pix.clear();
  for (int li = 0; li < c.n_edgelet_lengths; ++li) {
    const int l = c.edgelet_lengths[li];
    for (int ai = 0; ai < c.n_edgelet_angles; ++ai) {
      const int s = (int)std::lround(c.edgelet_angles_deg[ai] / 45.0) % 8;
      for (int y = 0; y < c.ny; ++y)
        for (int x = 0; x < c.nx; ++x) {
          for (int j = 0; j < l; ++j) {
            const int o = j - (l - 1) / 2;
            const int px = x + o * DX[s], py = y + o * DY[s];
            if (px >= 0 && px < c.nx && py >= 0 && py < c.ny)
              pix.push_back(py * c.nx + px);
          }
          ptr.push_back((int)pix.size());
        }
    }
  }
}

osar_status create_impl(const osar_config* cfg, osar_ctx** out) {
  std::string why;
  osar_status st = validate(cfg, &why);
  if (st != OSAR_OK) return fail(nullptr, st, why);
  osar_ctx* ctx = new osar_ctx();
  ctx->cfg = *cfg;
  ctx->cfg.dict_c128 = nullptr;
  ctx->cfg.lambda_list = nullptr;  // copied below
  ctx->n_lam = cfg->n_lambdas;
  ctx->lam.n = ctx->n_lam;
  for (int l = 0; l < MAX_LAMBDAS; ++l)
    ctx->lam.v[l] = l < ctx->n_lam && ctx->n_lam > 1 ? cfg->lambda_list[l]
                                                     : cfg->lambda;
  ctx->prec = cfg->precision;
  // the pixel-space Gram form runs the context as a pixel-basis one and
  // keeps the edgelet coefficients beside it (PixGram)
  const bool pixgram = cfg->pixel_gram != 0;
  ctx->dict = cfg->dict_kind != OSAR_DICT_IDENTITY && !pixgram;
  ctx->edgelet = cfg->dict_kind == OSAR_DICT_EDGELET && !pixgram;
  ctx->N = cfg->nx * cfg->ny;
  ctx->M = ctx->edgelet ? cfg->n_edgelet_lengths * cfg->n_edgelet_angles * ctx->N
           : ctx->dict  ? cfg->n_atoms
                        : ctx->N;
  if (pixgram) {
    ctx->pg = new PixGram();
    ctx->pg->dense = cfg->dict_kind != OSAR_DICT_EDGELET;
    ctx->pg->M = ctx->pg->dense ? cfg->n_atoms
                                : cfg->n_edgelet_lengths * cfg->n_edgelet_angles * ctx->N;
    ctx->pg->Mp = (int)roundup(ctx->pg->M, BLK);
    ctx->pg->nb = ctx->pg->Mp / BLK;
  }
  ctx->cfg.n_atoms = ctx->dict ? ctx->M : pixgram ? ctx->pg->M : cfg->n_atoms;
  ctx->cfg.edgelet_lengths = nullptr;     // the atom lists are built below
  ctx->cfg.edgelet_angles_deg = nullptr;
  ctx->K = cfg->n_freq;
  ctx->Mp = (int)roundup(ctx->M, BLK);
  ctx->Np = (int)roundup(ctx->N, BLK);
  ctx->Kp = (int)roundup(ctx->K, BLK);
  ctx->nb = ctx->Mp / BLK;
  ctx->nblk = packed_count(ctx->nb);
  ctx->dict_slices = dict_slices(ctx->Np);

  auto bail = [&](osar_status s) {
    g_create_error = ctx->last_error;
    free_all(ctx);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return s;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = prepare_burst_kernels();
  if (e == cudaSuccess && ctx->pg) e = prepare_pixgram_kernels();
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaGetDevice"));
  if (cfg->cuda_stream) {
    ctx->stream = (cudaStream_t)cfg->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaStreamCreate"));
    ctx->own_stream = true;
  }

  std::vector<int4> segs;
  std::vector<int> seg_begin;
  std::vector<int4> gtiles, dtiles, gpairs, dpairs;
  build_tables(ctx, segs, seg_begin, gtiles, dtiles, gpairs, dpairs);
  ctx->nseg = (int)segs.size();
  ctx->n_dict_tiles = (int)dtiles.size();
  ctx->n_gram_pairs = (int)gpairs.size();
  ctx->n_dict_pairs = (int)dpairs.size();

  const size_t cplx = ctx->prec == OSAR_FP64 ? 16 : 8;
  const int64_t Mp = ctx->Mp, Np = ctx->Np, Kp = ctx->Kp;
  const int64_t bb = (int64_t)BLK * BLK;
#define AL(p, bytes)                                 \
  do {                                               \
    osar_status _s = dev_alloc(ctx, &(p), (bytes), #p);  \
    if (_s != OSAR_OK) return bail(_s);              \
  } while (0)
  const int L = ctx->n_lam;
  ctx->guards.bytes = (size_t)cfg->guard_bytes;
  AL(ctx->scal, sizeof(DevScalars) * L);
  AL(ctx->b, 16 * Mp);
  AL(ctx->c, 16 * Mp * L);
  AL(ctx->z, 16 * Mp * L);
  AL(ctx->v, 16 * Mp);
  AL(ctx->w, 16 * Mp);
  AL(ctx->xtmp, 16 * Mp);
  AL(ctx->part, 16 * (int64_t)ctx->nb);
  AL(ctx->d_dev, 16 * Kp);
  AL(ctx->turns, 16 * Np);
  AL(ctx->g_hi, cplx * bb * ctx->nblk);
  if (ctx->prec == OSAR_SPLIT_BF16 && cfg->compensated)
    AL(ctx->g_lo, 4 * bb * ctx->nblk);
  AL(ctx->segpart, cplx * BLK * (int64_t)ctx->nseg);
  AL(ctx->tilepart, cplx * BLK * ctx->nblk);
  if (ctx->prec == OSAR_SPLIT_BF16 && (cfg->tc_pairs & 2) &&
      cfg->fuse_power_gram && !cfg->defer_gram && !ctx->pg) {
    AL(ctx->gp_col, 8 * BLK * ctx->nblk);
    AL(ctx->gp_row, 16 * BLK * ctx->nblk);
  }
  if (cfg->fuse_first_step || L > 1) {
    AL(ctx->segpart2, cplx * BLK * (int64_t)ctx->nseg);
    AL(ctx->tilepart2, cplx * BLK * ctx->nblk);
  }
  if (L > 2) {
    AL(ctx->segpart_x, cplx * BLK * (int64_t)ctx->nseg * (L - 2));
    AL(ctx->tilepart_x, cplx * BLK * ctx->nblk * (L - 2));
  }
  AL(ctx->zt, cplx * Mp * L);
  AL(ctx->vt, cplx * Mp);
  AL(ctx->xt, cplx * Mp);
  AL(ctx->bmax, 8 * ((Mp + 7) / 8));
  AL(ctx->d32, 8 * Kp);
  AL(ctx->segs, sizeof(int4) * segs.size());
  AL(ctx->seg_begin, sizeof(int) * seg_begin.size());
  AL(ctx->gram_tiles, sizeof(int4) * gtiles.size());
  if (ctx->dict) AL(ctx->dict_tiles, sizeof(int4) * (dtiles.size() ? dtiles.size() : 1));
  AL(ctx->gram_pairs, sizeof(int4) * gpairs.size());
  if (ctx->dict) AL(ctx->dict_pairs, sizeof(int4) * (dpairs.size() ? dpairs.size() : 1));
  std::vector<int> atom_ptr, atom_pix;
  if (ctx->edgelet) {
    // edgelets: pixel-major phases (FP32 for the split and FP32 paths) and
    // the atoms' pixel lists instead of a dictionary in device memory
    build_edgelets(*cfg, atom_ptr, atom_pix);
    AL(ctx->F, (ctx->prec == OSAR_FP64 ? 16 : 8) * Np * Kp);
    AL(ctx->atom_ptr, sizeof(int) * atom_ptr.size());
    AL(ctx->atom_pix, sizeof(int) * (atom_pix.empty() ? 1 : atom_pix.size()));
    if (ctx->prec == OSAR_SPLIT_BF16)
      AL(ctx->Apl, 2 * 6 * Mp * Kp);
    else
      AL(ctx->A, cplx * Mp * Kp);
  } else if (ctx->prec == OSAR_SPLIT_BF16) {
    AL(ctx->Apl, 2 * 6 * Mp * Kp);
    if (ctx->dict) {
      AL(ctx->Fpl, 2 * 6 * Kp * Np);
      AL(ctx->Dpl, 2 * 4 * Mp * Np);
      AL(ctx->dict_part, 8 * (int64_t)ctx->dict_slices * Mp * Kp);
    }
  } else {
    AL(ctx->A, cplx * Mp * Kp);
    if (ctx->dict) {
      AL(ctx->F, cplx * Kp * Np);
      AL(ctx->D, cplx * Mp * Np);
    }
  }
  if (cfg->gram_ahead) {
    // the second Gram buffer the update runs ahead into
    AL(ctx->gn_hi, cplx * bb * ctx->nblk);
    if (ctx->g_lo) AL(ctx->gn_lo, 4 * bb * ctx->nblk);
  }
  if (cfg->gram_ahead || cfg->defer_gram) AL(ctx->gram_ref, sizeof(void*));
  if (cfg->defer_gram) {
    // second Gram and forward-block buffers, the pending block's term
    AL(ctx->gn_hi, cplx * bb * ctx->nblk);
    if (ctx->g_lo) AL(ctx->gn_lo, 4 * bb * ctx->nblk);
    AL(ctx->Apl_alt, 2 * 6 * Mp * Kp);
    AL(ctx->corr, 8 * 2 * Mp);
    AL(ctx->corr_u, 8 * ((int64_t)ctx->nb + 1) * Kp);
    AL(ctx->corr_tick, sizeof(unsigned));
  }
  std::vector<int> pix_ptr, pix_atom;
  if (ctx->pg && ctx->pg->dense) {
    // a dense dictionary in its stored form for the two dictionary products
    // of every Gram application, and the coefficient-side vectors
    PixGram& g = *ctx->pg;
    const int64_t gm = g.Mp;
    if (ctx->prec == OSAR_SPLIT_BF16)
      AL(ctx->Dpl, 2 * 4 * gm * Np);
    else
      AL(ctx->D, cplx * gm * Np);
    AL(g.upart, cplx * (int64_t)pgd_chunks(ctx) * Np);
    AL(g.apart, cplx * (int64_t)pgd_adjoint_chunks(ctx) * gm);
    AL(g.c, 16 * gm);
    AL(g.z, 16 * gm);
    AL(g.b, 16 * gm);
    AL(g.v, 16 * gm);
    AL(g.w, 16 * gm);
    AL(g.part, 16 * (int64_t)g.nb);
    AL(g.bmax, 8 * (int64_t)g.nb);
  } else if (ctx->pg) {
    // H both ways: the atoms' pixel lists and, per pixel, its atoms
    PixGram& g = *ctx->pg;
    build_edgelets(*cfg, atom_ptr, atom_pix);
    pix_ptr.assign((size_t)ctx->N + 1, 0);
    for (int p : atom_pix) pix_ptr[p + 1]++;
    for (int p = 0; p < ctx->N; ++p) pix_ptr[p + 1] += pix_ptr[p];
    pix_atom.resize(atom_pix.size());
    std::vector<int> fill(pix_ptr.begin(), pix_ptr.end() - 1);
    for (int m = 0; m < g.M; ++m)
      for (int t = atom_ptr[m]; t < atom_ptr[m + 1]; ++t)
        pix_atom[fill[atom_pix[t]]++] = m;
    const size_t lists = atom_pix.empty() ? 1 : atom_pix.size();
    AL(ctx->atom_ptr, sizeof(int) * atom_ptr.size());
    AL(ctx->atom_pix, sizeof(int) * lists);
    AL(g.pix_ptr, sizeof(int) * pix_ptr.size());
    AL(g.pix_atom, sizeof(int) * lists);
    AL(g.c, 16 * (int64_t)g.Mp);
    AL(g.z, 16 * (int64_t)g.Mp);
    AL(g.b, 16 * (int64_t)g.Mp);
    AL(g.v, 16 * (int64_t)g.Mp);
    AL(g.w, 16 * (int64_t)g.Mp);
    AL(g.part, 16 * (int64_t)g.nb);
    AL(g.bmax, 8 * (int64_t)((g.M + 255) / 256));
  }
  const int64_t coef_p = ctx->pg ? std::max<int64_t>(Mp, ctx->pg->Mp) : Mp;
  AL(ctx->wk_dev, 8 * 2 * Kp);
  AL(ctx->sim_rho, 16 * Np);
  AL(ctx->sim_nz, 16 * coef_p);
  AL(ctx->sim_idx, 4 * coef_p);
  AL(ctx->sim_d, 16 * Kp);
#undef AL
  e = cudaMallocHost((void**)&ctx->h_ring, sizeof(double2) * RING * Kp);
  if (e == cudaSuccess)
    e = cudaMallocHost((void**)&ctx->h_wring, sizeof(double) * RING * Kp);
  for (int i = 0; i < RING && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&ctx->w_ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaMallocHost"));
  for (int i = 0; i < RING; ++i) {
    e = cudaEventCreateWithFlags(&ctx->ring_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaEventCreate"));
  }
  for (cudaEvent_t& ev : ctx->copy_ev) {
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaEventCreate"));
  }
  // the side stream: the next pulse's forward block beside the burst (a
  // dictionary), and the Gram update run ahead (gram_ahead, any basis)
  if ((ctx->dict || cfg->gram_ahead) && cfg->overlap_synthesis) {
    e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&ctx->ev_free, &ctx->ev_synth})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (cudaEvent_t& ev : ctx->ev_iters)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = cudaMallocHost((void**)&ctx->h_iters, sizeof(int32_t) * osar_ctx::ITERS_RING);
    if (cfg->defer_gram)
      for (cudaEvent_t* ev : {&ctx->ev_gram, &ctx->ev_mark[0], &ctx->ev_mark[1]}) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(*ev, ctx->stream);
      }
    if (cfg->gram_ahead)
      for (cudaEvent_t* ev : {&ctx->ev_gram, &ctx->ev_steps}) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(*ev, ctx->stream);
      }
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "side stream"));
  }
  e = launch_set_gram_ref(ctx);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "Gram address slot"));

  e = cudaMemcpyAsync(ctx->segs, segs.data(), sizeof(int4) * segs.size(),
                      cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->seg_begin, seg_begin.data(),
                        sizeof(int) * seg_begin.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->gram_tiles, gtiles.data(),
                        sizeof(int4) * gtiles.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess && ctx->dict && !dtiles.empty())
    e = cudaMemcpyAsync(ctx->dict_tiles, dtiles.data(),
                        sizeof(int4) * dtiles.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->gram_pairs, gpairs.data(),
                        sizeof(int4) * gpairs.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess && ctx->dict && !dpairs.empty())
    e = cudaMemcpyAsync(ctx->dict_pairs, dpairs.data(),
                        sizeof(int4) * dpairs.size(), cudaMemcpyHostToDevice,
                        ctx->stream);
  // initial scalars and power vector v = 1/sqrt(M) on the M real atoms
  std::vector<DevScalars> s0(L);
  std::memset(s0.data(), 0, sizeof(DevScalars) * L);
  for (auto& s : s0) s.t = 1.0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->scal, s0.data(), sizeof(DevScalars) * L,
                        cudaMemcpyHostToDevice, ctx->stream);
  std::vector<double2> v0((size_t)Mp, make_double2(0.0, 0.0));
  for (int i = 0; i < ctx->M; ++i) v0[i].x = 1.0 / std::sqrt((double)ctx->M);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->v, v0.data(), 16 * Mp, cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess) e = launch_set_working(ctx);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "upload tables"));

  if (ctx->edgelet) {
    e = cudaMemcpyAsync(ctx->atom_ptr, atom_ptr.data(), sizeof(int) * atom_ptr.size(),
                        cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && !atom_pix.empty())
      e = cudaMemcpyAsync(ctx->atom_pix, atom_pix.data(),
                          sizeof(int) * atom_pix.size(), cudaMemcpyHostToDevice,
                          ctx->stream);
    // the host lists leave scope below: the copies complete first
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "edgelet atoms"));
  } else if (ctx->pg && ctx->pg->dense) {
    // the coefficient power vector v = 1/sqrt(M) on the M atoms, and D
    const PixGram& g = *ctx->pg;
    std::vector<double2> vc((size_t)g.Mp, make_double2(0.0, 0.0));
    for (int i = 0; i < g.M; ++i) vc[i].x = 1.0 / std::sqrt((double)g.M);
    e = cudaMemcpyAsync(g.v, vc.data(), 16 * (size_t)g.Mp, cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e == cudaSuccess)
      e = launch_dictionary_build(
          ctx, cfg->dict_kind == OSAR_DICT_HOST ? cfg->dict_c128 : nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "dictionary build"));
  } else if (ctx->pg) {
    // both lists, and the coefficient power vector v = 1/sqrt(M) on the
    // M atoms (the stored-Gram form's start)
    const PixGram& g = *ctx->pg;
    std::vector<double2> vc((size_t)g.Mp, make_double2(0.0, 0.0));
    for (int i = 0; i < g.M; ++i) vc[i].x = 1.0 / std::sqrt((double)g.M);
    e = cudaMemcpyAsync(ctx->atom_ptr, atom_ptr.data(), sizeof(int) * atom_ptr.size(),
                        cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.pix_ptr, pix_ptr.data(), sizeof(int) * pix_ptr.size(),
                          cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && !atom_pix.empty())
      e = cudaMemcpyAsync(ctx->atom_pix, atom_pix.data(),
                          sizeof(int) * atom_pix.size(), cudaMemcpyHostToDevice,
                          ctx->stream);
    if (e == cudaSuccess && !pix_atom.empty())
      e = cudaMemcpyAsync(g.pix_atom, pix_atom.data(),
                          sizeof(int) * pix_atom.size(), cudaMemcpyHostToDevice,
                          ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.v, vc.data(), 16 * (size_t)g.Mp, cudaMemcpyHostToDevice,
                          ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "edgelet atoms"));
  } else if (ctx->dict) {
    e = launch_dictionary_build(
        ctx, cfg->dict_kind == OSAR_DICT_HOST ? cfg->dict_c128 : nullptr);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "dictionary build"));
  }
  if (ctx->prec == OSAR_SPLIT_BF16) {
    std::string err;
    if (!make_tensor_maps(ctx, &err))
      return bail(fail(ctx, OSAR_E_CUDA, err));
  }
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "create synchronize"));
  *out = ctx;
  return OSAR_OK;
}

osar_status read_scalars(osar_ctx* ctx, DevScalars* s) {
  CK(ctx, cudaMemcpyAsync(s, ctx->scal, sizeof(*s), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (s->error)
    return fail(ctx, OSAR_E_TIMEOUT, "a bounded device wait gave up");
  return OSAR_OK;
}

// The launchers issue on ctx->stream and record their profiling events there;
// this points ctx->stream at another stream for one scope.
struct LaunchOn {
  osar_ctx* ctx;
  cudaStream_t saved;
  LaunchOn(osar_ctx* c, cudaStream_t s) : ctx(c), saved(c->stream) { c->stream = s; }
  ~LaunchOn() { ctx->stream = saved; }
};

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) != cudaSuccess ||
         cs != cudaStreamCaptureStatusNone;
}

// Forward block of a pulse (Eq. 4 with the dictionary of Eq. 5): per-pixel
// phase terms, phase matrix, then A_s = F_s D for dictionary models.
cudaError_t synthesize_phase(osar_ctx* ctx, const double gamma[3], int grid_cap) {
  cudaError_t e = cudaSuccess;
  ctx->synth_w = nullptr;
  if (ctx->w_slot >= 0) {
    // a non-white pulse: its weights, on the stream of its phases
    double* dev = ctx->wk_dev + (int64_t)(ctx->n & 1) * ctx->Kp;
    e = cudaMemcpyAsync(dev, ctx->h_wring + (int64_t)ctx->w_slot * ctx->Kp,
                        sizeof(double) * ctx->Kp, cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->w_ev[ctx->w_slot], ctx->stream);
    ctx->synth_w = dev;
  }
  if (e == cudaSuccess) e = launch_pixel_turns(ctx, gamma);
  if (e == cudaSuccess) e = launch_phase(ctx, grid_cap);
  ctx->synth_w = nullptr;
  return e;
}
cudaError_t synthesize_dict(osar_ctx* ctx, int grid_cap) {
  if (!ctx->dict) return cudaSuccess;
  if (ctx->edgelet) return launch_edgelet(ctx, grid_cap);
  return ctx->prec == OSAR_SPLIT_BF16 ? launch_dict_tc(ctx, grid_cap)
                                      : launch_dict_simt(ctx);
}
cudaError_t synthesize(osar_ctx* ctx, const double gamma[3], int grid_cap) {
  cudaError_t e = synthesize_phase(ctx, gamma, grid_cap);
  if (e == cudaSuccess) e = synthesize_dict(ctx, grid_cap);
  return e;
}

// Step count of a recent burst, for synth_grid.  The host may run ahead of
// the device; here it waits for the burst before the last one queued, so it
// stays about two pulses ahead and the estimate at most one burst old, and
// it takes the last burst's count when that one has finished already.
void refresh_iters_estimate(osar_ctx* ctx) {
  const int64_t q = ctx->iters_seq;
  constexpr int R = osar_ctx::ITERS_RING;
  if (q == 0) return;
  const int last = (int)((q - 1) % R);
  if (cudaEventQuery(ctx->ev_iters[last]) == cudaSuccess) {
    ctx->iters_est = ctx->h_iters[last];
    return;
  }
  cudaGetLastError();  // cudaErrorNotReady is not an error here
  if (q >= 2) {
    const int prev = (int)((q - 2) % R);
    if (cudaEventSynchronize(ctx->ev_iters[prev]) == cudaSuccess)
      ctx->iters_est = ctx->h_iters[prev];
  }
}

// CTAs for the overlapped dictionary product, which runs beside the previous
// pulse's power steps and FISTA burst: the product keeps the tensor cores
// busy while the burst streams the FP32 Gram from HBM.  A small model picks
// the grid.  On g SMs the product takes D / g (D = its tensor flops over
// the split-BF16 rate one SM sustains beside the burst); meanwhile a Gram
// pass takes max(bytes / HBM bandwidth, bytes / ((S - g) x per-SM
// bandwidth)) x contention (per-SM bandwidth fitted at 84 GB/s, below the
// 105 GB/s one SM pulls alone: beside the product the pass also shares HBM
// with it; 105 gave the product more SMs and measured 13.35 against 13.30
// ms per pulse), and the rest of the
// burst runs at full speed.  The g that finishes both soonest is compared
// with running the product alone on the whole GPU after the burst (0).  The
// constants were measured on GB300 with the 128 x 128 workload (one SM:
// 1.23e13 f/s alone, about 1.2e13 beside the burst).
int synth_grid(const osar_ctx* ctx, bool main_idle, double* t_model = nullptr) {
  if (t_model) *t_model = 0.0;
  if (ctx->cfg.synth_ctas > 0) return std::min(ctx->cfg.synth_ctas, ctx->sm_count);
  // an edgelet block is a gather of phase rows, too short to overlap; the
  // pixel basis has no product (its side stream serves gram_ahead)
  if (ctx->edgelet || !ctx->dict) return 0;
  // nothing in flight on the main stream (the caller waited for the last
  // burst): the product has the GPU to itself
  if (main_idle) return 0;
  constexpr double kSmRateAlone = 1.23e13, kSmRateBeside = 1.2e13;  // f/s
  constexpr double kHbm = 6.8e12, kSmBw = 84e9, kContention = 1.08;  // B/s
  const double flops = 24.0 * ctx->Kp * (double)ctx->Np * ctx->Mp;
  const double bytes = (double)ctx->nblk * BLK * BLK * 8.0;
  const double pass = bytes / kHbm;
  const int power = ctx->n <= 1 ? ctx->cfg.power_iters_first : ctx->cfg.power_iters;
  // the first power step rides on the Gram update when fuse_power_gram holds
  const double passes = power - (ctx->gp_col && power > 0 ? 1 : 0) + ctx->iters_est;
  const int S = ctx->sm_count;
  double best = flops / (kSmRateAlone * S) + passes * pass;
  int best_g = 0;
  for (int g = 8; g <= S - 16; g += 4) {
    const double t_dict = flops / (kSmRateBeside * g);
    const double t_pass = std::max(pass, bytes / ((S - g) * kSmBw)) * kContention;
    const double beside = t_dict / t_pass;  // passes made while the product runs
    const double t = passes <= beside ? t_dict : t_dict + (passes - beside) * pass;
    if (t < best) {
      best = t;
      best_g = g;
    }
  }
  if (t_model) *t_model = best;
  return best_g;
}

// gram_ahead: SMs for the side stream when the pushed pulse's forward block
// and its Gram update both run there beside the previous pulse's burst, or
// 0 when the in-order schedule is expected to finish the pulse sooner.  The
// in-order time is synth_grid's (the product beside the burst) plus the
// update alone on the whole GPU; ahead, both products share g SMs (the
// update at 1.05e13 f/s per SM, its measured rate) while the burst's passes
// run on the rest and share HBM with the update's read-modify-write, the
// model of defer_grid.  A burst too short to hide the update keeps the
// in-order schedule.  gram_ahead = 2 always runs ahead (on synth_ctas SMs
// when set; on half the GPU when nothing is in flight to model).
int ahead_grid(const osar_ctx* ctx, bool main_idle) {
  const int S = ctx->sm_count;
  if (ctx->cfg.gram_ahead == 2) {
    if (ctx->cfg.synth_ctas > 0) return std::min(ctx->cfg.synth_ctas, S);
    if (main_idle) return S / 2;
  } else if (main_idle) {
    return 0;
  }
  constexpr double kDictRate = 1.2e13, kGramRate = 1.05e13;  // f/s per SM
  constexpr double kHbm = 6.8e12, kSmBw = 105e9, kContention = 1.15;  // B/s
  const double dict_f =
      ctx->edgelet || !ctx->dict ? 0.0 : 24.0 * ctx->Kp * (double)ctx->Np * ctx->Mp;
  const double gram_f = 3.0 * 2.0 * BLK * 2.0 * BLK * 2.0 * ctx->Kp * (double)ctx->nblk;
  const double bytes = (double)ctx->nblk * BLK * BLK * 8.0;
  const double pass = bytes / kHbm;
  const int power = ctx->n <= 1 ? ctx->cfg.power_iters_first : ctx->cfg.power_iters;
  const double passes = power - (ctx->gp_col && power > 0 ? 1 : 0) + ctx->iters_est;
  double t_inorder = 0.0;
  if (synth_grid(ctx, false, &t_inorder) == 0 || t_inorder <= 0.0)
    t_inorder = dict_f / (1.23e13 * S) + passes * pass;
  t_inorder += gram_f / (kGramRate * S);
  const double side = dict_f / kDictRate + gram_f / kGramRate;  // SM-seconds
  double best = 0.0;
  int best_g = 0;
  for (int g = 16; g <= S - 16; g += 4) {
    const double t_side = side / g;
    const double t_pass = std::max(pass, bytes / ((S - g) * kSmBw)) * kContention;
    const double beside = t_side / t_pass;  // passes made while the side works
    const double t = passes <= beside ? t_side : t_side + (passes - beside) * pass;
    if (best_g == 0 || t < best) {
      best = t;
      best_g = g;
    }
  }
  if (ctx->cfg.gram_ahead == 2) return best_g;
  return best < t_inorder ? best_g : 0;
}

// SMs for the side stream in the deferred mode, where this pulse's Gram
// update and the next pulse's synthesis run there beside this pulse's power
// steps and burst: the model of synth_grid with both products on the side
// (the Gram update at 1.05e13 f/s per SM, its measured rate), the pass
// reading the pending block twice besides the Gram, and no option of running
// the products alone.
int defer_grid(const osar_ctx* ctx) {
  if (ctx->cfg.synth_ctas > 0) return std::min(ctx->cfg.synth_ctas, ctx->sm_count);
  constexpr double kDictRate = 1.2e13, kGramRate = 1.05e13;  // f/s per SM
  constexpr double kHbm = 6.8e12, kSmBw = 105e9, kContention = 1.15;  // B/s
  const double dict_f = 24.0 * ctx->Kp * (double)ctx->Np * ctx->Mp;
  const double gram_f = 3.0 * 2.0 * BLK * 2.0 * BLK * 2.0 * ctx->Kp * (double)ctx->nblk;
  const double side = dict_f / kDictRate + gram_f / kGramRate;  // SM-seconds
  const double bytes =
      (double)ctx->nblk * BLK * BLK * 8.0 + 2.0 * 8.0 * ctx->Mp * ctx->Kp;
  const double pass = bytes / kHbm;
  const int power = ctx->n <= 1 ? ctx->cfg.power_iters_first : ctx->cfg.power_iters;
  const double passes = power + ctx->iters_est;
  const int S = ctx->sm_count;
  double best = 0.0;
  int best_g = S / 2;
  for (int g = 16; g <= S - 16; g += 4) {
    const double t_side = side / g;
    const double t_pass = std::max(pass, bytes / ((S - g) * kSmBw)) * kContention;
    const double beside = t_side / t_pass;  // passes made while the side works
    const double t = passes <= beside ? t_side : t_side + (passes - beside) * pass;
    if (best == 0.0 || t < best) {
      best = t;
      best_g = g;
    }
  }
  return best_g;
}

// Deferred push (defer_gram).  Pulse n's passes read G_{n-1} plus the term
// of A_n; the side stream forms A_n (after the main stream is done with the
// block buffer's previous content, A_{n-2}) and then G_n = G_{n-1} + A_n^H
// A_n into the other Gram buffer (after the main stream is done with pulse
// n-1's passes, the last readers of G_{n-2} there).  The next push makes
// the main stream wait for G_n and swaps the buffers.
osar_status push_deferred(osar_ctx* ctx, const double gamma[3]) {
  refresh_iters_estimate(ctx);
  const int par = ctx->n & 1;
  cudaError_t e = settle_gram(ctx);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_mark[par], ctx->stream);
  std::swap(ctx->Apl, ctx->Apl_alt);
  std::swap(ctx->map_a_rows1, ctx->map_alt_rows1);
  std::swap(ctx->map_a_rows2, ctx->map_alt_rows2);
  const int grid = defer_grid(ctx);
  if (e == cudaSuccess) {
    LaunchOn on(ctx, ctx->side);
    e = cudaStreamWaitEvent(ctx->side, ctx->ev_mark[par ^ 1], 0);
    if (e == cudaSuccess) e = synthesize(ctx, gamma, grid);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_synth, ctx->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_mark[par], 0);
    if (e == cudaSuccess) e = launch_gram_tc(ctx, ctx->gn_hi, ctx->gn_lo, grid);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_gram, ctx->side);
  }
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_synth, 0);
  if (e == cudaSuccess) e = launch_data_update(ctx);
  ctx->gram_pending = true;
  ctx->synth_side = true;
  ctx->n += 1;
  ctx->fresh = true;
  ctx->first_ready = false;
  if (e == cudaSuccess)
    e = ctx->pg ? pg_after_push(ctx)
                : launch_power_steps(ctx,
                                     ctx->n == 1 ? ctx->cfg.power_iters_first
                                                 : ctx->cfg.power_iters,
                                     ctx->cfg.fuse_first_step != 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "osar_push_pulse");
  return OSAR_OK;
}

// Push with the Gram update run ahead (gram_ahead) on `grid` SMs of the side
// stream: the forward block A_n (after the main stream's last reader of the
// block buffer, ev_free) and then G_n = G_{n-1} + A_n^H A_n into the second
// Gram buffer (after the previous push's power steps, ev_steps: the last
// main-stream reads of the Gram, of the power vector and of the fused power
// step's partials that the update reads or writes); both run beside the
// previous pulse's burst, which reads G_{n-1} in the other buffer.  The main
// stream waits for G_n, takes the buffer that holds it, and runs the data
// update and the power steps.  The arithmetic is the in-order push's.
osar_status push_ahead(osar_ctx* ctx, const double gamma[3], int grid) {
  cudaError_t e = cudaSuccess;
  const bool early = ctx->dict && ctx->synth_side;
  if (early) {
    LaunchOn on(ctx, ctx->side);
    e = synthesize_phase(ctx, gamma, grid);
  }
  if (ctx->free_stale && e == cudaSuccess)
    e = cudaEventRecord(ctx->ev_free, ctx->stream);
  ctx->free_stale = false;
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_free, 0);
  if (e == cudaSuccess) {
    LaunchOn on(ctx, ctx->side);
    e = early ? synthesize_dict(ctx, grid) : synthesize(ctx, gamma, grid);
  }
  ctx->synth_side = true;
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_steps, 0);
  if (e == cudaSuccess) {
    LaunchOn on(ctx, ctx->side);
    e = launch_gram_tc(ctx, ctx->gn_hi, ctx->gn_lo, grid, true);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_gram, ctx->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_gram, 0);
  std::swap(ctx->g_hi, ctx->gn_hi);
  std::swap(ctx->g_lo, ctx->gn_lo);
  if (e == cudaSuccess) e = launch_set_gram_ref(ctx);
  ctx->pushes_ahead++;
  ctx->ahead_grid_last = grid;
  if (e == cudaSuccess) e = launch_data_update(ctx);
  // the data update was the block buffer's last main-stream reader
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_free, ctx->stream);
  ctx->n += 1;
  ctx->fresh = true;
  ctx->first_ready = false;
  if (e == cudaSuccess)
    e = launch_power_steps(ctx,
                           ctx->n == 1 ? ctx->cfg.power_iters_first
                                       : ctx->cfg.power_iters,
                           ctx->cfg.fuse_first_step != 0);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_steps, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "osar_push_pulse");
  return OSAR_OK;
}

// True when every launch on the main stream has finished (the caller waited
// for the last burst before pushing).
bool main_idle(osar_ctx* ctx) {
  if (cudaStreamQuery(ctx->stream) == cudaSuccess) return true;
  cudaGetLastError();  // cudaErrorNotReady: work in flight
  return false;
}

// idle: main_idle() taken before the pulse's data copy was queued.
osar_status push_impl(osar_ctx* ctx, const double gamma[3], bool idle) {
  cudaError_t e = cudaSuccess;
  if (ctx->cfg.gram_ahead && capturing(ctx->stream))
    return fail(ctx, OSAR_E_STATE,
                "gram_ahead: a push cannot be captured into a CUDA graph (the "
                "Gram it updates alternates between two buffers)");
  if (ctx->cfg.defer_gram) {
    if (capturing(ctx->stream))
      return fail(ctx, OSAR_E_STATE,
                  "defer_gram: a push cannot be captured into a CUDA graph");
    return push_deferred(ctx, gamma);
  }
  if (ctx->side && !capturing(ctx->stream)) {
    refresh_iters_estimate(ctx);
    if (ctx->cfg.gram_ahead) {
      const int ahead = ahead_grid(ctx, idle);
      if (ahead > 0) return push_ahead(ctx, gamma, ahead);
    }
    const int grid = synth_grid(ctx, idle);
    if (grid > 0) {
      // With a dictionary the phase operand F is read only by the product:
      // when the previous product ran earlier on the side stream, the phases
      // go first.  The product's output (and, without a dictionary, the
      // phase planes themselves) is free once the previous pulse's Gram
      // update, its last reader, is done (ev_free); so are the phase
      // buffers when the previous synthesis ran on the main stream.  The
      // burst after the Gram update only reads the Gram, b and the
      // coefficient vectors.
      const bool early = ctx->dict && ctx->synth_side;
      if (early) {
        LaunchOn on(ctx, ctx->side);
        e = synthesize_phase(ctx, gamma, grid);
      }
      if (ctx->free_stale && e == cudaSuccess)
        e = cudaEventRecord(ctx->ev_free, ctx->stream);
      ctx->free_stale = false;
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_free, 0);
      if (e == cudaSuccess) {
        LaunchOn on(ctx, ctx->side);
        e = early ? synthesize_dict(ctx, grid) : synthesize(ctx, gamma, grid);
      }
      ctx->synth_side = true;
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_synth, ctx->side);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_synth, 0);
    } else {
      // the product is best run alone on the whole GPU: in order on the
      // main stream, after the burst (on the side stream its persistent
      // CTAs would hold SMs that the burst's launches wait for)
      e = synthesize(ctx, gamma, 0);
      ctx->synth_side = false;
    }
  } else {
    // a captured push leaves no usable ev_free behind
    if (ctx->side) ctx->free_stale = true;
    e = synthesize(ctx, gamma, 0);
    ctx->synth_side = false;
  }
  if (e == cudaSuccess) e = launch_data_update(ctx);
  if (e == cudaSuccess)
    e = ctx->prec == OSAR_SPLIT_BF16 ? launch_gram_tc(ctx, nullptr, nullptr, 0, true)
                                     : launch_gram_simt(ctx);
  if (e == cudaSuccess && ctx->side && !ctx->free_stale)
    e = cudaEventRecord(ctx->ev_free, ctx->stream);
  ctx->n += 1;
  ctx->fresh = true;
  ctx->first_ready = false;
  if (e == cudaSuccess)
    e = ctx->pg ? pg_after_push(ctx)
                : launch_power_steps(ctx,
                                     ctx->n == 1 ? ctx->cfg.power_iters_first
                                                 : ctx->cfg.power_iters,
                                     ctx->cfg.fuse_first_step != 0);
  // (with gram_ahead; a push is then never captured)
  if (e == cudaSuccess && ctx->ev_steps) e = cudaEventRecord(ctx->ev_steps, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "osar_push_pulse");
  return OSAR_OK;
}

}  // namespace

namespace osar {

cudaError_t settle_gram(osar_ctx* ctx) {
  if (!ctx->gram_pending) return cudaSuccess;
  const cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->ev_gram, 0);
  if (e != cudaSuccess) return e;
  std::swap(ctx->g_hi, ctx->gn_hi);
  std::swap(ctx->g_lo, ctx->gn_lo);
  ctx->gram_pending = false;
  const cudaError_t e2 = launch_set_gram_ref(ctx);
  if (e2 != cudaSuccess) return e2;
  // a fused first step's pass lacks the block's term: the step runs its own
  ctx->first_ready = false;
  return cudaSuccess;
}

void prof_begin(osar_ctx* ctx, int kind, ProfEvent* ev) {
  ev->kind = -1;
  if (!ctx->prof_on || !((ctx->prof_mask >> kind) & 1u)) return;
  if (ctx->prof_seq[kind]++ % ctx->prof_every[kind] != 0) return;
  for (int i = 0; i < 2; ++i) {
    cudaEvent_t x;
    if (!ctx->ev_pool.empty()) {
      x = ctx->ev_pool.back();
      ctx->ev_pool.pop_back();
    } else if (cudaEventCreate(&x) != cudaSuccess) {
      return;
    }
    (i == 0 ? ev->a : ev->b) = x;
  }
  ev->kind = kind;
  cudaEventRecord(ev->a, ctx->stream);
}

void prof_end(osar_ctx* ctx, ProfEvent* ev) {
  if (ev->kind < 0) return;
  cudaEventRecord(ev->b, ctx->stream);
  ctx->prof_pending.push_back(*ev);
}

}  // namespace osar

extern "C" {

void osar_config_default(osar_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = 32;
  c->ny = 32;
  c->pixel_m = 1.0;
  c->n_freq = 128;
  c->f_lo_hz = 9.9e9;
  c->f_hi_hz = 10.1e9;
  c->dict_kind = OSAR_DICT_IDENTITY;
  c->n_atoms = 0;
  c->dict_c128 = nullptr;
  c->dict_seed = 0;
  c->precision = OSAR_FP64;
  c->lambda = 0.05;
  c->lambda_relative = 1;
  c->power_iters_first = 30;
  c->power_iters = 4;
  c->lipschitz_margin = 0.01;
  c->restart_momentum = 0;
  c->compensated = 1;
  c->cuda_stream = nullptr;
  c->overlap_synthesis = 1;
  c->synth_ctas = 0;
  c->tc_pairs = 3;
  c->fuse_first_step = 1;
  c->n_lambdas = 1;
  c->lambda_list = nullptr;
  c->defer_gram = 0;
  c->guard_bytes = 0;
  c->fuse_power_gram = 1;
  c->pixel_gram = 0;
}

namespace {
// The coefficient vector c_hat and its length (the atoms' side in the
// pixel-space Gram form).
const double2* coef_c(const osar_ctx* ctx) { return ctx->pg ? ctx->pg->c : ctx->c; }
int coef_m(const osar_ctx* ctx) { return ctx->pg ? ctx->pg->M : ctx->M; }
osar_status no_pixgram(osar_ctx* ctx, const char* what) {
  return fail(ctx, OSAR_E_STATE,
              std::string(what) + ": not available in the pixel-space Gram form");
}
}  // namespace

osar_status osar_create(const osar_config* cfg, osar_ctx** out) {
  osar::TraceRange trace_("osar_create");
  if (!out) return fail(nullptr, OSAR_E_INVALID, "out is NULL");
  *out = nullptr;
  const osar_status st = create_impl(cfg, out);
  // the allocation-free Gram apply's static array: looked up now, on the
  // context's device, so that its first call loads nothing
  if (st == OSAR_OK) osar::prepare_static_scratch();
  return st;
}

osar_status osar_destroy(osar_ctx* ctx) {
  if (!ctx) return OSAR_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  free_all(ctx);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return OSAR_OK;
}

osar_status osar_push_pulse(osar_ctx* ctx, const double gamma_xyz[3],
                            const double* d_c128) {
  osar::TraceRange trace_("osar_push_pulse");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!gamma_xyz || !d_c128)
    return fail(ctx, OSAR_E_INVALID, "osar_push_pulse: NULL argument");
  for (int i = 0; i < 3; ++i)
    if (!is_finite(gamma_xyz[i]))
      return fail(ctx, OSAR_E_INVALID, "osar_push_pulse: non-finite gamma");
  const bool idle = main_idle(ctx);
  const int slot = ctx->ring_pos;
  ctx->ring_pos = (ctx->ring_pos + 1) % RING;
  CK(ctx, cudaEventSynchronize(ctx->ring_ev[slot]));
  double2* h = ctx->h_ring + (size_t)slot * ctx->Kp;
  std::memcpy(h, d_c128, sizeof(double2) * ctx->K);
  CK(ctx, cudaMemcpyAsync(ctx->d_dev, h, sizeof(double2) * ctx->K,
                          cudaMemcpyHostToDevice, ctx->stream));
  CK(ctx, cudaEventRecord(ctx->ring_ev[slot], ctx->stream));
  return push_impl(ctx, gamma_xyz, idle);
}

osar_status osar_push_pulse_var(osar_ctx* ctx, const double gamma_xyz[3],
                                const double* d_c128, const double* noise_var) {
  osar::TraceRange trace_("osar_push_pulse_var");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!gamma_xyz || !d_c128)
    return fail(ctx, OSAR_E_INVALID, "osar_push_pulse_var: NULL argument");
  if (!noise_var) return osar_push_pulse(ctx, gamma_xyz, d_c128);
  for (int i = 0; i < 3; ++i)
    if (!is_finite(gamma_xyz[i]))
      return fail(ctx, OSAR_E_INVALID, "osar_push_pulse_var: non-finite gamma");
  for (int k = 0; k < ctx->K; ++k)
    if (!is_finite(noise_var[k]) || !(noise_var[k] > 0.0))
      return fail(ctx, OSAR_E_INVALID,
                  "osar_push_pulse_var: noise variances must be finite and > 0");
  const bool idle = main_idle(ctx);
  // weights 1 / sigma_k for the phases (host ring slot)
  const int ws = ctx->w_pos;
  ctx->w_pos = (ctx->w_pos + 1) % RING;
  CK(ctx, cudaEventSynchronize(ctx->w_ev[ws]));
  double* w = ctx->h_wring + (size_t)ws * ctx->Kp;
  for (int k = 0; k < ctx->Kp; ++k)
    w[k] = k < ctx->K ? 1.0 / std::sqrt(noise_var[k]) : 0.0;
  // the whitened data R_n^{-1/2} d
  const int slot = ctx->ring_pos;
  ctx->ring_pos = (ctx->ring_pos + 1) % RING;
  CK(ctx, cudaEventSynchronize(ctx->ring_ev[slot]));
  double2* h = ctx->h_ring + (size_t)slot * ctx->Kp;
  for (int k = 0; k < ctx->K; ++k)
    h[k] = make_double2(d_c128[2 * k] * w[k], d_c128[2 * k + 1] * w[k]);
  CK(ctx, cudaMemcpyAsync(ctx->d_dev, h, sizeof(double2) * ctx->K,
                          cudaMemcpyHostToDevice, ctx->stream));
  CK(ctx, cudaEventRecord(ctx->ring_ev[slot], ctx->stream));
  ctx->w_slot = ws;
  st = push_impl(ctx, gamma_xyz, idle);
  ctx->w_slot = -1;
  return st;
}

osar_status osar_push_pulse_dev(osar_ctx* ctx, const double gamma_xyz[3],
                                const void* d_dev_c128) {
  osar::TraceRange trace_("osar_push_pulse_dev");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!gamma_xyz || !d_dev_c128)
    return fail(ctx, OSAR_E_INVALID, "osar_push_pulse_dev: NULL argument");
  for (int i = 0; i < 3; ++i)
    if (!is_finite(gamma_xyz[i]))
      return fail(ctx, OSAR_E_INVALID, "osar_push_pulse_dev: non-finite gamma");
  const bool idle = main_idle(ctx);
  CK(ctx, cudaMemcpyAsync(ctx->d_dev, d_dev_c128, sizeof(double2) * ctx->K,
                          cudaMemcpyDeviceToDevice, ctx->stream));
  return push_impl(ctx, gamma_xyz, idle);
}

osar_status osar_iterate(osar_ctx* ctx, int32_t max_iters, double tol,
                         int32_t* iters_done) {
  osar::TraceRange trace_("osar_iterate");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (max_iters < 0 || !is_finite(tol) || tol < 0)
    return fail(ctx, OSAR_E_INVALID, "osar_iterate: bad max_iters or tol");
  if (ctx->n == 0)
    return fail(ctx, OSAR_E_STATE, "osar_iterate before the first pulse");
  cudaError_t e = cudaSuccess;
  if (ctx->fresh) {
    e = ctx->pg ? pg_burst_begin(ctx) : launch_burst_begin(ctx);
    ctx->fresh = false;
  }
  if (e == cudaSuccess) e = launch_iter_begin(ctx, tol);
  for (int k = 0; e == cudaSuccess && k < max_iters; ++k)
    e = ctx->pg ? pg_fista_step(ctx) : launch_fista_step(ctx);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "osar_iterate");
  if (iters_done) {
    DevScalars s;
    st = read_scalars(ctx, &s);
    if (st != OSAR_OK) return st;
    *iters_done = s.iters;
    ctx->iters_est = s.iters;
  } else if (ctx->side && !capturing(ctx->stream)) {
    // the step count reaches the host without a wait, for synth_grid
    const int slot = (int)(ctx->iters_seq % osar_ctx::ITERS_RING);
    const char* src = reinterpret_cast<const char*>(ctx->scal) +
                      offsetof(DevScalars, iters);
    CK(ctx, cudaMemcpyAsync(ctx->h_iters + slot, src, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->ev_iters[slot], ctx->stream));
    ctx->iters_seq += 1;
  }
  return OSAR_OK;
}

osar_status osar_get_coeffs(osar_ctx* ctx, double* out_c128) {
  osar::TraceRange trace_("osar_get_coeffs");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!out_c128) return fail(ctx, OSAR_E_INVALID, "osar_get_coeffs: NULL");
  CK(ctx, cudaMemcpyAsync(out_c128, coef_c(ctx), sizeof(double2) * coef_m(ctx),
                          cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return OSAR_OK;
}

osar_status osar_get_coeffs_dev(osar_ctx* ctx, void* out_dev_c128) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!out_dev_c128) return fail(ctx, OSAR_E_INVALID, "osar_get_coeffs_dev: NULL");
  CK(ctx, cudaMemcpyAsync(out_dev_c128, coef_c(ctx), sizeof(double2) * coef_m(ctx),
                          cudaMemcpyDeviceToDevice, ctx->stream));
  return OSAR_OK;
}

osar_status osar_get_coeffs_async(osar_ctx* ctx, double* out_c128,
                                  int32_t slot) {
  osar::TraceRange trace_("osar_get_coeffs_async");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!out_c128 || slot < 0 || slot >= OSAR_COPY_SLOTS)
    return fail(ctx, OSAR_E_INVALID, "osar_get_coeffs_async: bad buffer or slot");
  CK(ctx, cudaMemcpyAsync(out_c128, coef_c(ctx), sizeof(double2) * coef_m(ctx),
                          cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaEventRecord(ctx->copy_ev[slot], ctx->stream));
  return OSAR_OK;
}

osar_status osar_wait_coeffs(osar_ctx* ctx, int32_t slot) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (slot < 0 || slot >= OSAR_COPY_SLOTS)
    return fail(ctx, OSAR_E_INVALID, "osar_wait_coeffs: slot out of range");
  CK(ctx, cudaEventSynchronize(ctx->copy_ev[slot]));
  return OSAR_OK;
}

osar_status osar_get_state(osar_ctx* ctx, int32_t* n, double* lipschitz,
                           double* lambda, double* t) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  DevScalars s;
  st = read_scalars(ctx, &s);
  if (st != OSAR_OK) return st;
  if (n) *n = ctx->n;
  if (lipschitz) *lipschitz = s.lip;
  if (lambda) *lambda = s.lambda;
  if (t) *t = s.t;
  return OSAR_OK;
}

osar_status osar_get_lambda_state(osar_ctx* ctx, int32_t l, double* out_c128,
                                  double* lambda, double* t, int32_t* iters) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (ctx->pg) return no_pixgram(ctx, "osar_get_lambda_state");
  if (l < 0 || l >= ctx->n_lam)
    return fail(ctx, OSAR_E_INVALID, "osar_get_lambda_state: no such solution");
  DevScalars s;
  CK(ctx, cudaMemcpyAsync(&s, ctx->scal + l, sizeof(s), cudaMemcpyDeviceToHost,
                          ctx->stream));
  if (out_c128)
    CK(ctx, cudaMemcpyAsync(out_c128, ctx->c + (int64_t)l * ctx->Mp,
                            sizeof(double2) * ctx->M, cudaMemcpyDeviceToHost,
                            ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (lambda) *lambda = s.lambda;
  if (t) *t = s.t;
  if (iters) *iters = s.iters;
  return OSAR_OK;
}

osar_status osar_get_dims(const osar_ctx* ctx, int32_t* m_atoms,
                          int32_t* n_pixels, int32_t* n_freq) {
  if (!ctx) return OSAR_E_INVALID;
  if (m_atoms) *m_atoms = coef_m(ctx);
  if (n_pixels) *n_pixels = ctx->N;
  if (n_freq) *n_freq = ctx->K;
  return OSAR_OK;
}

osar_status osar_get_gram(osar_ctx* ctx, double* out_c128) {
  osar::TraceRange trace_("osar_get_gram");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!out_c128) return fail(ctx, OSAR_E_INVALID, "osar_get_gram: NULL");
  CK(ctx, settle_gram(ctx));
  const int64_t M = ctx->M;
  int64_t rows = (int64_t)(256ll << 20) / (16 * M);
  if (rows < 1) rows = 1;
  if (rows > M) rows = M;
  double2* tmp = nullptr;
  CK(ctx, cudaMalloc(&tmp, sizeof(double2) * rows * M));
  for (int64_t r0 = 0; r0 < M; r0 += rows) {
    int64_t nr = r0 + rows <= M ? rows : M - r0;
    cudaError_t e = launch_gram_expand(ctx, (int)r0, (int)nr, tmp);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out_c128 + 2 * r0 * M, tmp, sizeof(double2) * nr * M,
                          cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(ctx, e, "osar_get_gram");
    }
  }
  cudaFree(tmp);
  return OSAR_OK;
}

osar_status osar_get_gram_entries(osar_ctx* ctx, const int32_t* rows,
                                  const int32_t* cols, int32_t count,
                                  double* out_c128) {
  osar::TraceRange trace_("osar_get_gram_entries");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (count < 0 || (count > 0 && (!rows || !cols || !out_c128)))
    return fail(ctx, OSAR_E_INVALID, "osar_get_gram_entries: bad arguments");
  if (count == 0) return OSAR_OK;
  CK(ctx, settle_gram(ctx));
  std::vector<int2> rc(count);
  for (int q = 0; q < count; ++q) {
    if (rows[q] < 0 || rows[q] >= ctx->M || cols[q] < 0 || cols[q] >= ctx->M)
      return fail(ctx, OSAR_E_INVALID, "osar_get_gram_entries: index out of range");
    rc[q] = make_int2(rows[q], cols[q]);
  }
  int2* drc = nullptr;
  double2* dout = nullptr;
  CK(ctx, cudaMalloc(&drc, sizeof(int2) * count));
  cudaError_t e = cudaMalloc(&dout, sizeof(double2) * count);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(drc, rc.data(), sizeof(int2) * count,
                        cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_gram_entries(ctx, drc, count, dout);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_c128, dout, sizeof(double2) * count,
                        cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(drc);
  if (dout) cudaFree(dout);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "osar_get_gram_entries");
  return OSAR_OK;
}

osar_status osar_get_b(osar_ctx* ctx, double* out_c128) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!out_c128) return fail(ctx, OSAR_E_INVALID, "osar_get_b: NULL");
  CK(ctx, cudaMemcpyAsync(out_c128, ctx->pg ? ctx->pg->b : ctx->b,
                          sizeof(double2) * coef_m(ctx),
                          cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return OSAR_OK;
}

osar_status osar_gram_apply(osar_ctx* ctx, const double* x_c128,
                            double* y_c128) {
  osar::TraceRange trace_("osar_gram_apply");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!x_c128 || !y_c128) return fail(ctx, OSAR_E_INVALID, "osar_gram_apply: NULL");
  CK(ctx, settle_gram(ctx));
  CK(ctx, cudaMemsetAsync(ctx->xtmp, 0, sizeof(double2) * ctx->Mp, ctx->stream));
  CK(ctx, cudaMemcpyAsync(ctx->xtmp, x_c128, sizeof(double2) * ctx->M,
                          cudaMemcpyHostToDevice, ctx->stream));
  CK(ctx, launch_gram_apply(ctx, ctx->xtmp, ctx->w));
  CK(ctx, cudaMemcpyAsync(y_c128, ctx->w, sizeof(double2) * ctx->M,
                          cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return OSAR_OK;
}

osar_status osar_simulate_pulse(osar_ctx* ctx, const double gamma_xyz[3],
                                const double* coeffs_c128, double* d_c128) {
  osar::TraceRange trace_("osar_simulate_pulse");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!gamma_xyz || !coeffs_c128 || !d_c128)
    return fail(ctx, OSAR_E_INVALID, "osar_simulate_pulse: NULL argument");
  std::vector<int> idx;
  std::vector<double2> val;
  for (int j = 0; j < coef_m(ctx); ++j) {
    double re = coeffs_c128[2 * j], im = coeffs_c128[2 * j + 1];
    if (re != 0.0 || im != 0.0) {
      idx.push_back(j);
      val.push_back(make_double2(re, im));
    }
  }
  const int nnz = (int)idx.size();
  if (nnz) {
    CK(ctx, cudaMemcpyAsync(ctx->sim_idx, idx.data(), sizeof(int) * nnz,
                            cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->sim_nz, val.data(), sizeof(double2) * nnz,
                            cudaMemcpyHostToDevice, ctx->stream));
  }
  CK(ctx, launch_pixel_turns(ctx, gamma_xyz));
  CK(ctx, launch_simulate(ctx, nnz, ctx->sim_d));
  CK(ctx, cudaMemcpyAsync(d_c128, ctx->sim_d, sizeof(double2) * ctx->K,
                          cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return OSAR_OK;
}

osar_status osar_unroll_grad(osar_ctx* ctx, int32_t steps, int32_t ckpt_every,
                             double lambda, double tau, double t0,
                             const double* c0_c128, const double* c_true_c128,
                             double* loss, double* d_lambda, double* d_tau,
                             double* d_b_c128, double* c_T_c128) {
  osar::TraceRange trace_("osar_unroll_grad");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (ctx->pg) return no_pixgram(ctx, "osar_unroll_grad");
  if (ctx->n == 0)
    return fail(ctx, OSAR_E_STATE, "osar_unroll_grad before the first pulse");
  CK(ctx, settle_gram(ctx));
  if (steps < 1 || ckpt_every < 1 || !is_finite(tau) || tau <= 0 ||
      !is_finite(lambda) || lambda < 0 || !is_finite(t0) || t0 < 1 ||
      !c0_c128 || !c_true_c128)
    return fail(ctx, OSAR_E_INVALID, "osar_unroll_grad: bad arguments");
  cudaError_t e = run_unroll_grad(ctx, steps, ckpt_every, lambda, tau, t0,
                                  c0_c128, c_true_c128, loss, d_lambda, d_tau,
                                  d_b_c128, c_T_c128);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "osar_unroll_grad");
  return OSAR_OK;
}

osar_status osar_set_lambda(osar_ctx* ctx, int32_t l, double lambda) {
  osar::TraceRange trace_("osar_set_lambda");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (l < 0 || l >= ctx->n_lam || !is_finite(lambda) || lambda < 0)
    return fail(ctx, OSAR_E_INVALID, "osar_set_lambda: bad solution index or lambda");
  ctx->lam.v[l] = lambda;
  if (ctx->n_lam == 1) ctx->cfg.lambda = lambda;
  return OSAR_OK;
}

osar_status osar_set_gram_ahead(osar_ctx* ctx, int32_t mode) {
  osar::TraceRange trace_("osar_set_gram_ahead");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (mode < 0 || mode > 2)
    return fail(ctx, OSAR_E_INVALID, "osar_set_gram_ahead: mode must be 0, 1 or 2");
  if (!ctx->gn_hi || !ctx->ev_steps)
    return fail(ctx, OSAR_E_STATE,
                "osar_set_gram_ahead: the context was created with gram_ahead = 0");
  ctx->cfg.gram_ahead = mode;
  return OSAR_OK;
}

osar_status osar_synchronize(osar_ctx* ctx) {
  osar::TraceRange trace_("osar_synchronize");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->side) CK(ctx, cudaStreamSynchronize(ctx->side));
  return OSAR_OK;
}

osar_status osar_check_guards(osar_ctx* ctx, int32_t* corrupted) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!corrupted) return fail(ctx, OSAR_E_INVALID, "osar_check_guards: NULL");
  if (ctx->side) CK(ctx, cudaStreamSynchronize(ctx->side));
  int bad = 0;
  std::string first;
  CK(ctx, check_guards(ctx->guards, ctx->stream, &bad, &first));
  *corrupted = bad;
  if (bad) ctx->last_error = "guard overwritten behind " + first;
  return OSAR_OK;
}

osar_status osar_poke_guard(osar_ctx* ctx, int32_t index) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (index < 0 || index >= (int32_t)ctx->guards.regions.size())
    return fail(ctx, OSAR_E_INVALID, "osar_poke_guard: no such guard");
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  CK(ctx, cudaMemset(ctx->guards.regions[index].addr + ctx->guards.bytes / 2, 0, 1));
  return OSAR_OK;
}

osar_status osar_profile_enable(osar_ctx* ctx, int32_t on) {
  if (!ctx) return OSAR_E_INVALID;
  ctx->prof_on = on != 0;
  return OSAR_OK;
}

osar_status osar_profile_select(osar_ctx* ctx, uint32_t mask) {
  if (!ctx) return OSAR_E_INVALID;
  if (mask >> KCL_COUNT)
    return fail(ctx, OSAR_E_INVALID, "osar_profile_select: mask has bits past the last kernel class");
  ctx->prof_mask = mask;
  return OSAR_OK;
}

osar_status osar_profile_sample(osar_ctx* ctx, int32_t kernel, int32_t every) {
  if (!ctx) return OSAR_E_INVALID;
  if (kernel < 0 || kernel >= KCL_COUNT || every < 1)
    return fail(ctx, OSAR_E_INVALID, "osar_profile_sample: kernel class or every out of range");
  ctx->prof_every[kernel] = every;
  ctx->prof_seq[kernel] = 0;
  return OSAR_OK;
}

static osar_status profile_collect(osar_ctx* ctx) {
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto& pe : ctx->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
      ctx->prof_ms[pe.kind] += ms;
      ctx->prof_launches[pe.kind] += 1;
    }
    ctx->ev_pool.push_back(pe.a);
    ctx->ev_pool.push_back(pe.b);
  }
  ctx->prof_pending.clear();
  return OSAR_OK;
}

osar_status osar_profile_read(osar_ctx* ctx, int32_t kernel, int64_t* launches,
                              double* total_ms) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (kernel < 0 || kernel >= KCL_COUNT)
    return fail(ctx, OSAR_E_INVALID, "osar_profile_read: unknown kernel class");
  st = profile_collect(ctx);
  if (st != OSAR_OK) return st;
  if (launches) *launches = ctx->prof_launches[kernel];
  if (total_ms) *total_ms = ctx->prof_ms[kernel];
  return OSAR_OK;
}

osar_status osar_profile_reset(osar_ctx* ctx) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  st = profile_collect(ctx);
  if (st != OSAR_OK) return st;
  for (int k = 0; k < KCL_COUNT; ++k) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_launches[k] = 0;
    ctx->prof_seq[k] = 0;
  }
  ctx->launches = 0;
  ctx->pushes_ahead = 0;
  CK(ctx, cudaMemsetAsync(reinterpret_cast<char*>(ctx->scal) +
                              offsetof(DevScalars, passes),
                          0, sizeof(unsigned long long), ctx->stream));
  return OSAR_OK;
}

osar_status osar_profile_passes(osar_ctx* ctx, int64_t* passes) {
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!passes) return fail(ctx, OSAR_E_INVALID, "osar_profile_passes: NULL");
  DevScalars s;
  st = read_scalars(ctx, &s);
  if (st != OSAR_OK) return st;
  *passes = (int64_t)s.passes;
  return OSAR_OK;
}

osar_status osar_profile_ahead(const osar_ctx* ctx, int64_t* pushes,
                               int32_t* last_grid) {
  if (!ctx || !pushes) return OSAR_E_INVALID;
  *pushes = ctx->pushes_ahead;
  if (last_grid) *last_grid = ctx->ahead_grid_last;
  return OSAR_OK;
}

osar_status osar_launch_count(const osar_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return OSAR_E_INVALID;
  *launches = ctx->launches;
  return OSAR_OK;
}

osar_status osar_device_bytes(const osar_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return OSAR_E_INVALID;
  *bytes = ctx->dev_bytes;
  return OSAR_OK;
}

// ------------------------------------------------------------ checkpoints --
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version;
  int32_t M, N, K, prec, dict_kind, compensated, n, fresh;
  int64_t nblk;
  int32_t entry_bytes, has_lo;
  int32_t n_lambdas, pad;
};

osar_status write_dev(osar_ctx* ctx, FILE* f, const void* dev, size_t bytes) {
  std::vector<char> buf(bytes);
  CK(ctx, cudaMemcpyAsync(buf.data(), dev, bytes, cudaMemcpyDeviceToHost,
                          ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (fwrite(buf.data(), 1, bytes, f) != bytes)
    return fail(ctx, OSAR_E_IO, "checkpoint write failed");
  return OSAR_OK;
}

osar_status read_dev(osar_ctx* ctx, FILE* f, void* dev, size_t bytes) {
  std::vector<char> buf(bytes);
  if (fread(buf.data(), 1, bytes, f) != bytes)
    return fail(ctx, OSAR_E_IO, "checkpoint truncated");
  CK(ctx, cudaMemcpyAsync(dev, buf.data(), bytes, cudaMemcpyHostToDevice,
                          ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return OSAR_OK;
}
}  // namespace

osar_status osar_save(osar_ctx* ctx, const char* path) {
  osar::TraceRange trace_("osar_save");
  osar_status st = check_usable(ctx);
  if (st != OSAR_OK) return st;
  if (!path) return fail(ctx, OSAR_E_INVALID, "osar_save: NULL path");
  if (ctx->pg) return no_pixgram(ctx, "osar_save");
  CK(ctx, settle_gram(ctx));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, OSAR_E_IO, std::string("cannot open ") + path);
  CkptHeader h = {};
  std::memcpy(h.magic, "OSARCKP", 8);
  h.version = 5;
  h.M = ctx->M;
  h.N = ctx->N;
  h.K = ctx->K;
  h.prec = ctx->prec;
  h.dict_kind = ctx->cfg.dict_kind;
  h.compensated = ctx->cfg.compensated;
  h.n = ctx->n;
  h.fresh = ctx->fresh ? 1 : 0;
  h.nblk = ctx->nblk;
  h.entry_bytes = ctx->prec == OSAR_FP64 ? 16 : 8;
  h.has_lo = ctx->g_lo ? 1 : 0;
  h.n_lambdas = ctx->n_lam;
  const size_t vec = sizeof(double2) * ctx->Mp;
  const size_t lvec = vec * ctx->n_lam;
  const size_t gb = (size_t)h.entry_bytes * BLK * BLK * ctx->nblk;
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1;
  if (!ok) {
    fclose(f);
    return fail(ctx, OSAR_E_IO, "checkpoint write failed");
  }
  st = write_dev(ctx, f, ctx->scal, sizeof(DevScalars) * ctx->n_lam);
  if (st == OSAR_OK) st = write_dev(ctx, f, ctx->b, vec);
  if (st == OSAR_OK) st = write_dev(ctx, f, ctx->c, lvec);
  if (st == OSAR_OK) st = write_dev(ctx, f, ctx->z, lvec);
  if (st == OSAR_OK) st = write_dev(ctx, f, ctx->v, vec);
  if (st == OSAR_OK) st = write_dev(ctx, f, ctx->g_hi, gb);
  if (st == OSAR_OK && ctx->g_lo) st = write_dev(ctx, f, ctx->g_lo, (size_t)4 * BLK * BLK * ctx->nblk);
  if (fclose(f) != 0 && st == OSAR_OK) st = fail(ctx, OSAR_E_IO, "checkpoint close failed");
  return st;
}

osar_status osar_load(const char* path, const osar_config* cfg, osar_ctx** out) {
  osar::TraceRange trace_("osar_load");
  if (!out) return fail(nullptr, OSAR_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!path || !cfg) return fail(nullptr, OSAR_E_INVALID, "osar_load: NULL argument");
  if (cfg->pixel_gram)
    return fail(nullptr, OSAR_E_STATE,
                "osar_load: not available in the pixel-space Gram form");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(nullptr, OSAR_E_IO, std::string("cannot open ") + path);
  CkptHeader h;
  if (fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "OSARCKP", 8) != 0 ||
      h.version != 5) {
    fclose(f);
    return fail(nullptr, OSAR_E_IO, "not an osar checkpoint");
  }
  osar_ctx* ctx = nullptr;
  osar_status st = osar_create(cfg, &ctx);
  if (st != OSAR_OK) {
    fclose(f);
    return st;
  }
  if (h.M != ctx->M || h.N != ctx->N || h.K != ctx->K || h.prec != ctx->prec ||
      h.dict_kind != ctx->cfg.dict_kind || h.nblk != ctx->nblk ||
      h.has_lo != (ctx->g_lo ? 1 : 0) || h.n_lambdas != ctx->n_lam) {
    fclose(f);
    osar_destroy(ctx);
    return fail(nullptr, OSAR_E_INVALID, "checkpoint does not match the config");
  }
  const size_t vec = sizeof(double2) * ctx->Mp;
  const size_t lvec = vec * ctx->n_lam;
  const size_t gb = (size_t)h.entry_bytes * BLK * BLK * ctx->nblk;
  st = read_dev(ctx, f, ctx->scal, sizeof(DevScalars) * ctx->n_lam);
  if (st == OSAR_OK) st = read_dev(ctx, f, ctx->b, vec);
  if (st == OSAR_OK) st = read_dev(ctx, f, ctx->c, lvec);
  if (st == OSAR_OK) st = read_dev(ctx, f, ctx->z, lvec);
  if (st == OSAR_OK) st = read_dev(ctx, f, ctx->v, vec);
  if (st == OSAR_OK) st = read_dev(ctx, f, ctx->g_hi, gb);
  if (st == OSAR_OK && ctx->g_lo)
    st = read_dev(ctx, f, ctx->g_lo, (size_t)4 * BLK * BLK * ctx->nblk);
  fclose(f);
  if (st == OSAR_OK) {
    cudaError_t e = launch_set_working(ctx);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "osar_load");
  }
  if (st != OSAR_OK) {
    g_create_error = ctx->last_error;
    osar_destroy(ctx);
    return st;
  }
  ctx->n = h.n;
  ctx->fresh = h.fresh != 0;
  *out = ctx;
  return OSAR_OK;
}

const char* osar_last_error(const osar_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->last_error.c_str();
}

const char* osar_version(void) { return "libosar 0.1 (sm_103a)"; }

}  // extern "C"
