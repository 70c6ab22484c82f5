// C ABI of the batching form (osar_batch_*): many independent online
// reconstructions of uneven size in one context, each with its own Gram,
// data vector, warm start and scalars.
//
// Layout: the scenes' atoms are stacked (each scene padded to a multiple of
// 128 rows), their packed Gram blocks are concatenated, and one tile list
// (A row block, B row block, output block) covers every scene's upper Gram
// blocks, so a pulse's Gram update for all scenes is one persistent tcgen05
// launch; a FISTA step for all scenes is one matvec launch over (scene,
// segment) items and one finalize launch over (scene, block) items.  Bursts
// are captured once per step count as CUDA graphs and replayed.  The matvec
// segment length (blocks per work item) is chosen by a small autotuner that
// times the candidates on the device and caches the choice in the file named
// by OSAR_TUNE_CACHE.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "batch.h"
#include "trace.h"

using namespace osar;

namespace {

thread_local std::string g_batch_error;

osar_status bfail(osar_batch* B, osar_status st, const std::string& msg) {
  if (B) {
    B->last_error = msg;
    if (st == OSAR_E_CUDA) B->sticky = OSAR_E_CUDA;
  } else {
    g_batch_error = msg;
  }
  return st;
}

osar_status bcuda(osar_batch* B, cudaError_t e, const char* where) {
  return bfail(B, e == cudaErrorMemoryAllocation ? OSAR_E_OOM : OSAR_E_CUDA,
               std::string(where) + ": " + cudaGetErrorName(e));
}

#define BCK(B, expr)                                   \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return bcuda(B, _e, #expr); \
  } while (0)

int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

template <typename T>
cudaError_t balloc(osar_batch* B, T** p, size_t bytes, const char* name) {
  size_t total = 0;
  cudaError_t e = guarded_malloc(B->guards, (void**)p, bytes, name, B->stream, &total);
  if (e == cudaSuccess) B->dev_bytes += (int64_t)total;
  return e;
}

void free_batch(osar_batch* B) {
  void* ptrs[] = {B->desc, B->sc, B->row_scene, B->gam, B->d, B->d32, B->turns,
                  B->b, B->c, B->z, B->v, B->w, B->zt, B->vt, B->part, B->bmax,
                  B->g_hi, B->g_lo, B->segpart, B->tilepart, B->segs,
                  B->seg_scene, B->seg_begin, B->items_dev, B->gram_tiles,
                  B->Apl, B->A};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (B->h_pinned) cudaFreeHost(B->h_pinned);
  if (B->h_gam) cudaFreeHost(B->h_gam);
  if (B->h_active) cudaFreeHost(B->h_active);
  if (B->stage_ev) cudaEventDestroy(B->stage_ev);
  for (auto& g : B->graphs) cudaGraphExecDestroy(g.second);
  B->graphs.clear();
}

// Matvec segments: per scene, per block column J, runs of `len` blocks.
void build_segments(const osar_batch* B, int len, std::vector<int4>& segs,
                    std::vector<int>& seg_scene, std::vector<int>& seg_begin) {
  segs.clear();
  seg_scene.clear();
  seg_begin.clear();
  for (int s = 0; s < B->S; ++s) {
    const int nb = B->desc_h[s].nb;
    for (int J = 0; J < nb; ++J) {
      seg_begin.push_back((int)segs.size());
      for (int I0 = 0; I0 <= J; I0 += len) {
        const int I1 = I0 + len < J + 1 ? I0 + len : J + 1;
        segs.push_back(make_int4(J, I0, I1, (int)segs.size()));
        seg_scene.push_back(s);
      }
    }
    seg_begin.push_back((int)segs.size());
  }
}

cudaError_t upload_segments(osar_batch* B, int len) {
  std::vector<int4> segs;
  std::vector<int> seg_scene, seg_begin;
  build_segments(B, len, segs, seg_scene, seg_begin);
  cudaError_t e = cudaMemcpyAsync(B->segs, segs.data(), sizeof(int4) * segs.size(),
                                  cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->seg_scene, seg_scene.data(),
                        sizeof(int) * seg_scene.size(), cudaMemcpyHostToDevice,
                        B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->seg_begin, seg_begin.data(),
                        sizeof(int) * seg_begin.size(), cudaMemcpyHostToDevice,
                        B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  B->nseg = (int)segs.size();
  B->seg_len = len;
  for (auto& g : B->graphs) cudaGraphExecDestroy(g.second);
  B->graphs.clear();
  return e;
}

cudaError_t upload_desc(osar_batch* B) {
  return cudaMemcpyAsync(B->desc, B->desc_h.data(),
                         sizeof(SceneDesc) * B->S, cudaMemcpyHostToDevice,
                         B->stream);
}

// Every scene's Gram tiles (global operand row blocks, global packed output
// block, scene), each scene's upper blocks in gram_sb x gram_sb super-blocks
// (the tiles running together share operand rows in L2), the scenes in
// index order or, with gram_lpt, the largest first (their long tile runs
// start early and the small scenes fill the tail).  Each output block is
// one tile's, so the order never changes a result.
void build_gram_tiles(osar_batch* B) {
  std::vector<int> order(B->S);
  for (int s = 0; s < B->S; ++s) order[s] = s;
  if (B->gram_lpt)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return B->desc_h[a].nb > B->desc_h[b].nb;
    });
  const int SB = B->gram_sb;
  B->gram_tiles_all.clear();
  for (int s : order) {
    const SceneDesc& d = B->desc_h[s];
    const int rb = d.row / BLK;
    for (int bi = 0; bi < d.nb; bi += SB)
      for (int bj = bi; bj < d.nb; bj += SB)
        for (int I = bi; I < bi + SB && I < d.nb; ++I)
          for (int J = (bj > I ? bj : I); J < bj + SB && J < d.nb; ++J)
            B->gram_tiles_all.push_back(make_int4(
                rb + I, rb + J, (int)(d.gblk + packed_block(I, J, d.nb)), s));
  }
  B->n_gram_tiles = 0;  // the next push uploads its active scenes' tiles
}

std::string tune_key(const osar_batch* B) {
  std::ostringstream k;
  k << "batch_tune2 prec" << B->prec << " sm" << B->sm_count << " S" << B->S
    << " K" << B->Kp;
  uint64_t h = 1469598103934665603ull;
  for (int s = 0; s < B->S; ++s) {
    h ^= (uint64_t)B->desc_h[s].nb;
    h *= 1099511628211ull;
  }
  k << " nb" << std::hex << h;
  return k.str();
}

// Tuning cache ($OSAR_TUNE_CACHE): lines "key=seg_len sb lpt"; the last
// line for a key wins.  Returns false when the key is absent.
bool cache_lookup(const std::string& key, int* seg, int* sb, int* lpt) {
  const char* path = std::getenv("OSAR_TUNE_CACHE");
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    const size_t eq = line.rfind('=');
    if (eq == std::string::npos || line.substr(0, eq) != key) continue;
    std::istringstream v(line.substr(eq + 1));
    int a = 0, b = 0, c = -1;
    if (v >> a >> b >> c && a > 0 && b > 0 && (c == 0 || c == 1)) {
      *seg = a;
      *sb = b;
      *lpt = c;
      found = true;
    }
  }
  return found;
}

void cache_store(const std::string& key, int seg, int sb, int lpt) {
  const char* path = std::getenv("OSAR_TUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << "=" << seg << " " << sb << " " << lpt << "\n";
}

// Two timing events, destroyed on every path.
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&a);
    return e == cudaSuccess ? cudaEventCreate(&b) : e;
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" {

osar_status osar_batch_create(const osar_config* cfgs, int32_t n_scenes,
                              void* cuda_stream, osar_batch** out) {
  osar::TraceRange trace_("osar_batch_create");
  if (!out) return bfail(nullptr, OSAR_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfgs || n_scenes < 1 || n_scenes > 4096)
    return bfail(nullptr, OSAR_E_INVALID, "need 1..4096 scene configs");
  const int prec = cfgs[0].precision;
  int kmax = 0;
  for (int s = 0; s < n_scenes; ++s) {
    const osar_config& c = cfgs[s];
    if (c.dict_kind != OSAR_DICT_IDENTITY)
      return bfail(nullptr, OSAR_E_INVALID, "batched scenes use the pixel basis");
    if (c.precision != prec)
      return bfail(nullptr, OSAR_E_INVALID, "all scenes share one precision");
    if (c.n_lambdas > 1)
      return bfail(nullptr, OSAR_E_INVALID,
                   "batched scenes have one lambda each (a lambda path is a "
                   "single-context feature)");
    if (c.nx < 1 || c.ny < 1 || (int64_t)c.nx * c.ny > 131072 || c.n_freq < 1 ||
        c.n_freq > 16384 || !(c.pixel_m > 0) || !(c.f_lo_hz > 0) ||
        !(c.f_hi_hz >= c.f_lo_hz) || !(c.lambda >= 0) ||
        c.power_iters_first < 1 || c.power_iters < 0 || !(c.lipschitz_margin >= 0))
      return bfail(nullptr, OSAR_E_INVALID, "invalid scene config");
    if (c.n_freq > kmax) kmax = c.n_freq;
  }
  if (prec < OSAR_FP64 || prec > OSAR_SPLIT_BF16)
    return bfail(nullptr, OSAR_E_INVALID, "unknown precision");
  const int gb = cfgs[0].guard_bytes;
  if (gb < 0 || gb > (1 << 20) || gb % 256)
    return bfail(nullptr, OSAR_E_INVALID,
                 "guard_bytes must be a multiple of 256 in [0, 1 MiB]");

  osar_batch* B = new osar_batch();
  B->guards.bytes = (size_t)gb;
  B->S = n_scenes;
  B->prec = prec;
  B->Kp = (int)rup(kmax, BLK);
  B->cfg.assign(cfgs, cfgs + n_scenes);
  B->n_h.assign(n_scenes, 0);
  B->active_h.assign(n_scenes, 0);
  auto bail = [&](osar_status st) {
    g_batch_error = B->last_error;
    free_batch(B);
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    delete B;
    return st;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bail(bcuda(B, e, "cudaGetDevice"));
  if (cuda_stream) {
    B->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(bcuda(B, e, "cudaStreamCreate"));
    B->own_stream = true;
  }

  // scene layout
  B->desc_h.resize(n_scenes);
  int rows = 0, items = 0;
  int64_t blocks = 0;
  std::vector<int> row_scene;
  std::vector<int2> items_h;
  for (int s = 0; s < n_scenes; ++s) {
    const osar_config& c = cfgs[s];
    SceneDesc& d = B->desc_h[s];
    std::memset(&d, 0, sizeof(d));
    d.M = c.nx * c.ny;
    d.K = c.n_freq;
    d.nx = c.nx;
    const int mp = (int)rup(d.M, BLK);
    d.nb = mp / BLK;
    d.row = rows;
    d.gblk = blocks;
    d.item0 = items;
    d.seg0 = 0;
    d.relative = c.lambda_relative;
    d.restart = c.restart_momentum;
    d.pixel_m = c.pixel_m;
    d.cx_half = 0.5 * (c.nx - 1);
    d.cy_half = 0.5 * (c.ny - 1);
    const double df = c.n_freq > 1 ? (c.f_hi_hz - c.f_lo_hz) / (c.n_freq - 1) : 0.0;
    d.two_flo_c = 2.0 * c.f_lo_hz / C_LIGHT;
    d.two_df_c = 2.0 * df / C_LIGHT;
    d.lam = c.lambda;
    d.margin = c.lipschitz_margin;
    for (int r = 0; r < mp; ++r) row_scene.push_back(s);
    for (int K = 0; K < d.nb; ++K) items_h.push_back(make_int2(s, K));
    rows += mp;
    blocks += packed_count(d.nb);
    items += d.nb;
  }
  // seg_begin runs: scene s owns entries [seg0, seg0 + nb]
  int off = 0;
  for (int s = 0; s < n_scenes; ++s) {
    B->desc_h[s].seg0 = off;
    off += B->desc_h[s].nb + 1;
  }
  B->rows = rows;
  B->blocks = blocks;
  B->items = items;
  build_gram_tiles(B);
  const size_t cplx = prec == OSAR_FP64 ? 16 : 8;
  const int64_t R = rows, Kp = B->Kp;
#define BA(p, bytes)                                        \
  do {                                                      \
    cudaError_t _e = balloc(B, &(p), (bytes), #p);          \
    if (_e != cudaSuccess) return bail(bcuda(B, _e, "cudaMalloc")); \
  } while (0)
  BA(B->desc, sizeof(SceneDesc) * n_scenes);
  BA(B->sc, sizeof(DevScalars) * n_scenes);
  BA(B->row_scene, sizeof(int) * R);
  BA(B->gam, sizeof(double) * 3 * n_scenes);
  BA(B->d, sizeof(double2) * n_scenes * Kp);
  BA(B->d32, sizeof(float2) * n_scenes * Kp);
  BA(B->turns, sizeof(ulonglong2) * R);
  BA(B->b, 16 * R);
  BA(B->c, 16 * R);
  BA(B->z, 16 * R);
  BA(B->v, 16 * R);
  BA(B->w, 16 * R);
  BA(B->zt, cplx * R);
  BA(B->vt, cplx * R);
  BA(B->part, sizeof(double2) * items);
  BA(B->bmax, sizeof(double) * items);
  BA(B->g_hi, cplx * BLK * BLK * blocks);
  if (prec == OSAR_SPLIT_BF16 && cfgs[0].compensated)
    BA(B->g_lo, 4 * (size_t)BLK * BLK * blocks);
  BA(B->segpart, cplx * BLK * blocks);   // enough for 1-block segments
  BA(B->tilepart, cplx * BLK * blocks);
  BA(B->segs, sizeof(int4) * blocks);
  BA(B->seg_scene, sizeof(int) * blocks);
  BA(B->seg_begin, sizeof(int) * (items + n_scenes));
  BA(B->items_dev, sizeof(int2) * items);
  BA(B->gram_tiles, sizeof(int4) * B->gram_tiles_all.size());
  if (prec == OSAR_SPLIT_BF16)
    BA(B->Apl, 2 * 6 * R * Kp);
  else
    BA(B->A, cplx * R * Kp);
#undef BA
  e = cudaMallocHost((void**)&B->h_pinned, sizeof(double2) * n_scenes * Kp);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&B->h_gam, sizeof(double) * 3 * n_scenes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->stage_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(bcuda(B, e, "host staging"));

  e = cudaMemcpyAsync(B->row_scene, row_scene.data(), sizeof(int) * R,
                      cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->items_dev, items_h.data(), sizeof(int2) * items,
                        cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) e = upload_desc(B);
  // scalars: t = 1; power vectors v = 1/sqrt(M) on each scene's atoms
  std::vector<DevScalars> sc0(n_scenes);
  std::memset(sc0.data(), 0, sizeof(DevScalars) * n_scenes);
  for (auto& x : sc0) x.t = 1.0;
  std::vector<double2> v0((size_t)R, make_double2(0.0, 0.0));
  for (int s = 0; s < n_scenes; ++s)
    for (int j = 0; j < B->desc_h[s].M; ++j)
      v0[B->desc_h[s].row + j].x = 1.0 / std::sqrt((double)B->desc_h[s].M);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->sc, sc0.data(), sizeof(DevScalars) * n_scenes,
                        cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->v, v0.data(), 16 * R, cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) {
    if (prec == OSAR_FP64) {
      e = cudaMemcpyAsync(B->vt, v0.data(), 16 * R, cudaMemcpyHostToDevice, B->stream);
    } else {
      std::vector<float2> vf((size_t)R);
      for (int64_t r = 0; r < R; ++r) vf[r] = make_float2((float)v0[r].x, 0.f);
      e = cudaMemcpyAsync(B->vt, vf.data(), 8 * R, cudaMemcpyHostToDevice, B->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    }
  }
  if (e != cudaSuccess) return bail(bcuda(B, e, "upload tables"));
  int len = (int)(blocks / ((int64_t)B->sm_count * 2 * 12));
  if (len < 1) len = 1;
  if (len > 16) len = 16;
  int c_seg = 0, c_sb = 0, c_lpt = 0;
  if (cache_lookup(tune_key(B), &c_seg, &c_sb, &c_lpt)) {
    len = c_seg;
    B->gram_sb = c_sb;
    B->gram_lpt = c_lpt;
    build_gram_tiles(B);
  }
  e = upload_segments(B, len);
  if (e != cudaSuccess) return bail(bcuda(B, e, "segments"));
  if (prec == OSAR_SPLIT_BF16) {
    std::string err;
    if (!batch_make_tensor_maps(B, &err)) return bail(bfail(B, OSAR_E_CUDA, err));
  }
  e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return bail(bcuda(B, e, "create synchronize"));
  *out = B;
  return OSAR_OK;
}

osar_status osar_batch_destroy(osar_batch* B) {
  if (!B) return OSAR_OK;
  cudaStreamSynchronize(B->stream);
  free_batch(B);
  if (B->own_stream) cudaStreamDestroy(B->stream);
  delete B;
  return OSAR_OK;
}

osar_status osar_batch_push(osar_batch* B, const int32_t* active,
                            const double* gammas_xyz, const double* d_c128,
                            int32_t d_stride) {
  osar::TraceRange trace_("osar_batch_push");
  if (!B) return OSAR_E_INVALID;
  if (B->sticky != OSAR_OK) return B->sticky;
  if (!active || !gammas_xyz || !d_c128 || d_stride < 1)
    return bfail(B, OSAR_E_INVALID, "osar_batch_push: bad arguments");
  bool changed = false;
  int max_steps = 0;
  for (int s = 0; s < B->S; ++s) {
    const int a = active[s] ? 1 : 0;
    if (a && d_stride < B->cfg[s].n_freq)
      return bfail(B, OSAR_E_INVALID, "osar_batch_push: d_stride < n_freq");
    for (int q = 0; q < 3 && a; ++q)
      if (!std::isfinite(gammas_xyz[3 * s + q]))
        return bfail(B, OSAR_E_INVALID, "osar_batch_push: non-finite gamma");
    changed |= a != B->desc_h[s].active;
    B->desc_h[s].active = a;
    B->desc_h[s].psteps = a ? (B->n_h[s] == 0 ? B->cfg[s].power_iters_first
                                              : B->cfg[s].power_iters)
                            : 0;
    if (B->desc_h[s].psteps > max_steps) max_steps = B->desc_h[s].psteps;
  }
  // staging: wait until the previous push's copies have read the buffers
  BCK(B, cudaEventSynchronize(B->stage_ev));
  std::memset(B->h_pinned, 0, sizeof(double2) * B->S * B->Kp);
  for (int s = 0; s < B->S; ++s) {
    if (!active[s]) continue;
    std::memcpy(B->h_pinned + (size_t)s * B->Kp, d_c128 + 2 * (size_t)s * d_stride,
                sizeof(double2) * B->cfg[s].n_freq);
    std::memcpy(B->h_gam + 3 * s, gammas_xyz + 3 * s, 3 * sizeof(double));
  }
  BCK(B, cudaMemcpyAsync(B->d, B->h_pinned, sizeof(double2) * B->S * B->Kp,
                         cudaMemcpyHostToDevice, B->stream));
  BCK(B, cudaMemcpyAsync(B->gam, B->h_gam, sizeof(double) * 3 * B->S,
                         cudaMemcpyHostToDevice, B->stream));
  BCK(B, upload_desc(B));
  BCK(B, cudaEventRecord(B->stage_ev, B->stream));
  if (changed || B->n_gram_tiles == 0) {
    std::vector<int4> t;
    for (const int4& x : B->gram_tiles_all)
      if (B->desc_h[x.w].active) t.push_back(x);
    B->n_gram_tiles = (int)t.size();
    if (!t.empty()) {
      BCK(B, cudaMemcpyAsync(B->gram_tiles, t.data(), sizeof(int4) * t.size(),
                             cudaMemcpyHostToDevice, B->stream));
      BCK(B, cudaStreamSynchronize(B->stream));
    }
  }
  BCK(B, batch_launch_phase(B));
  BCK(B, batch_launch_data_update(B));
  BCK(B, batch_launch_gram(B));
  BCK(B, batch_launch_power(B, max_steps));
  for (int s = 0; s < B->S; ++s)
    if (active[s]) B->n_h[s]++;
  B->fresh = true;
  return OSAR_OK;
}

osar_status osar_batch_iterate(osar_batch* B, int32_t max_iters, double tol,
                               int32_t* iters) {
  osar::TraceRange trace_("osar_batch_iterate");
  if (!B) return OSAR_E_INVALID;
  if (B->sticky != OSAR_OK) return B->sticky;
  if (max_iters < 0 || !std::isfinite(tol) || tol < 0)
    return bfail(B, OSAR_E_INVALID, "osar_batch_iterate: bad max_iters or tol");
  bool any = false;
  for (int s = 0; s < B->S; ++s) any |= B->desc_h[s].active && B->n_h[s] > 0;
  if (!any) return bfail(B, OSAR_E_STATE, "osar_batch_iterate before a push");
  if (B->fresh) {
    BCK(B, batch_launch_burst_begin(B));
    B->fresh = false;
  }
  BCK(B, batch_launch_iter_begin(B, tol));
  if (max_iters > 0) {
    cudaGraphExec_t exec = nullptr;
    for (auto& g : B->graphs)
      if (g.first == max_iters) exec = g.second;
    if (!exec) {
      const int64_t saved = B->launches;
      cudaGraph_t graph = nullptr;
      BCK(B, cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < max_iters && e == cudaSuccess; ++k)
        e = batch_launch_fista_step(B);
      cudaError_t e2 = cudaStreamEndCapture(B->stream, &graph);
      if (e != cudaSuccess) return bcuda(B, e, "burst capture");
      if (e2 != cudaSuccess) return bcuda(B, e2, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return bcuda(B, e, "cudaGraphInstantiate");
      B->graphs.emplace_back(max_iters, exec);
      B->launches = saved;
    }
    BCK(B, cudaGraphLaunch(exec, B->stream));
    B->launches += 2 * (int64_t)max_iters;
  }
  if (iters) {
    std::vector<DevScalars> h(B->S);
    BCK(B, cudaMemcpyAsync(h.data(), B->sc, sizeof(DevScalars) * B->S,
                           cudaMemcpyDeviceToHost, B->stream));
    BCK(B, cudaStreamSynchronize(B->stream));
    for (int s = 0; s < B->S; ++s) iters[s] = B->desc_h[s].active ? h[s].iters : 0;
  }
  return OSAR_OK;
}

osar_status osar_batch_get_coeffs(osar_batch* B, int32_t scene, double* out_c128) {
  osar::TraceRange trace_("osar_batch_get_coeffs");
  if (!B) return OSAR_E_INVALID;
  if (B->sticky != OSAR_OK) return B->sticky;
  if (scene < 0 || scene >= B->S || !out_c128)
    return bfail(B, OSAR_E_INVALID, "osar_batch_get_coeffs: bad arguments");
  const SceneDesc& d = B->desc_h[scene];
  BCK(B, cudaMemcpyAsync(out_c128, B->c + d.row, sizeof(double2) * d.M,
                         cudaMemcpyDeviceToHost, B->stream));
  BCK(B, cudaStreamSynchronize(B->stream));
  return OSAR_OK;
}

osar_status osar_batch_get_state(osar_batch* B, int32_t scene, int32_t* n,
                                 double* lipschitz, double* lambda, double* t) {
  if (!B) return OSAR_E_INVALID;
  if (B->sticky != OSAR_OK) return B->sticky;
  if (scene < 0 || scene >= B->S)
    return bfail(B, OSAR_E_INVALID, "osar_batch_get_state: bad scene");
  DevScalars h;
  BCK(B, cudaMemcpyAsync(&h, B->sc + scene, sizeof(h), cudaMemcpyDeviceToHost,
                         B->stream));
  BCK(B, cudaStreamSynchronize(B->stream));
  if (h.error) return bfail(B, OSAR_E_TIMEOUT, "a bounded device wait gave up");
  if (n) *n = B->n_h[scene];
  if (lipschitz) *lipschitz = h.lip;
  if (lambda) *lambda = h.lambda;
  if (t) *t = h.t;
  return OSAR_OK;
}

osar_status osar_batch_autotune(osar_batch* B, int32_t* chosen) {
  if (!B) return OSAR_E_INVALID;
  if (B->sticky != OSAR_OK) return B->sticky;
  const std::string key = tune_key(B);
  int seg = 0, sb = 0, lpt = 0;
  if (!cache_lookup(key, &seg, &sb, &lpt)) {
    std::vector<int> saved(B->S);
    for (int s = 0; s < B->S; ++s) {
      saved[s] = B->desc_h[s].active;
      B->desc_h[s].active = 1;
    }
    BCK(B, upload_desc(B));
    EventPair ev;
    BCK(B, ev.create());
    auto time_it = [&](auto&& launch, int reps, float* ms) -> cudaError_t {
      cudaError_t e = launch();  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(ev.a, B->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
      if (e == cudaSuccess) e = cudaEventRecord(ev.b, B->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ev.a, ev.b);
      return e;
    };
    // 1. The Gram update's tile order: super-block size and scene order.
    // Timed only before the first pulse: the statistics and the operand
    // planes are still zero, so each timed update adds exact zeros and
    // leaves every Gram as it was.  Afterwards the order is kept.
    bool pushed = false;
    for (int s = 0; s < B->S; ++s) pushed |= B->n_h[s] > 0;
    sb = B->gram_sb;
    lpt = B->gram_lpt;
    if (!pushed) {
      float best_ms = 1e30f;
      for (int cand_lpt : {0, 1})
        for (int cand_sb : {4, 8, 16, 32}) {
          B->gram_sb = cand_sb;
          B->gram_lpt = cand_lpt;
          build_gram_tiles(B);
          B->n_gram_tiles = (int)B->gram_tiles_all.size();
          BCK(B, cudaMemcpyAsync(B->gram_tiles, B->gram_tiles_all.data(),
                                 sizeof(int4) * B->gram_tiles_all.size(),
                                 cudaMemcpyHostToDevice, B->stream));
          float ms = 0.f;
          BCK(B, time_it([&] { return batch_launch_gram(B); }, 3, &ms));
          if (cand_sb == 8 && cand_lpt == 0) B->tune_gram_ms[0] = ms / 3;
          if (ms < best_ms) {
            best_ms = ms;
            sb = cand_sb;
            lpt = cand_lpt;
          }
        }
      B->tune_gram_ms[1] = best_ms / 3;
    }
    // 2. The matvec's work-item size (blocks per segment).
    float best_ms = 1e30f;
    for (int len : {1, 2, 4, 8, 16}) {
      BCK(B, upload_segments(B, len));
      float ms = 0.f;
      BCK(B, time_it([&] { return batch_launch_matvec(B, B->zt, 0, -1); }, 5, &ms));
      if (ms < best_ms) {
        best_ms = ms;
        seg = len;
      }
    }
    for (int s = 0; s < B->S; ++s) B->desc_h[s].active = saved[s];
    BCK(B, upload_desc(B));
    cache_store(key, seg, sb, lpt);
  }
  B->gram_sb = sb;
  B->gram_lpt = lpt;
  build_gram_tiles(B);
  BCK(B, upload_segments(B, seg));
  if (chosen) *chosen = seg;
  return OSAR_OK;
}

osar_status osar_batch_get_tuning(const osar_batch* B, int32_t* segment_blocks,
                                  int32_t* gram_superblock,
                                  int32_t* gram_largest_first,
                                  double* gram_ms_default, double* gram_ms_chosen) {
  if (!B) return OSAR_E_INVALID;
  if (segment_blocks) *segment_blocks = B->seg_len;
  if (gram_superblock) *gram_superblock = B->gram_sb;
  if (gram_largest_first) *gram_largest_first = B->gram_lpt;
  if (gram_ms_default) *gram_ms_default = B->tune_gram_ms[0];
  if (gram_ms_chosen) *gram_ms_chosen = B->tune_gram_ms[1];
  return OSAR_OK;
}

osar_status osar_batch_info(const osar_batch* B, int32_t* n_scenes,
                            int64_t* device_bytes, int64_t* launches,
                            int32_t* segment_blocks) {
  if (!B) return OSAR_E_INVALID;
  if (n_scenes) *n_scenes = B->S;
  if (device_bytes) *device_bytes = B->dev_bytes;
  if (launches) *launches = B->launches;
  if (segment_blocks) *segment_blocks = B->seg_len;
  return OSAR_OK;
}

osar_status osar_batch_synchronize(osar_batch* B) {
  if (!B) return OSAR_E_INVALID;
  if (B->sticky != OSAR_OK) return B->sticky;
  BCK(B, cudaStreamSynchronize(B->stream));
  return OSAR_OK;
}

osar_status osar_batch_check_guards(osar_batch* B, int32_t* corrupted) {
  if (!B || !corrupted) return OSAR_E_INVALID;
  if (B->sticky != OSAR_OK) return B->sticky;
  int bad = 0;
  std::string first;
  BCK(B, check_guards(B->guards, B->stream, &bad, &first));
  *corrupted = bad;
  if (bad) B->last_error = "guard overwritten behind " + first;
  return OSAR_OK;
}

const char* osar_batch_last_error(const osar_batch* B) {
  if (!B) return g_batch_error.c_str();
  return B->last_error.c_str();
}

}  // extern "C"
