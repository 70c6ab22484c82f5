// Batching form: many independent online reconstructions of uneven size in
// one context.  Each scene keeps its own Gram, data vector, coefficients,
// warm start and scalars; per-pulse work and FISTA bursts for all scenes run
// as single launches over (scene, work item) lists, and bursts are replayed
// from captured CUDA graphs.
#pragma once

#include <string>
#include <vector>

#include "ctx.h"

namespace osar {

// Per-scene constants read by the batched kernels.
struct SceneDesc {
  int64_t gblk;       // first packed Gram block of the scene
  int row;            // first stacked atom row (multiple of 128)
  int nb;             // Gram blocks per side
  int M;              // atoms = pixels (pixel basis)
  int K;              // frequencies
  int nx;
  int seg0;           // first entry of the scene's seg_begin run (nb + 1 entries)
  int item0;          // first (scene, block) finalize item of the scene
  int active;         // received a pulse in the last push (gates all work)
  int relative;       // lambda relative to ||b||_inf
  int restart;        // restart momentum per pulse
  int psteps;         // power-iteration steps for this push
  double pixel_m, cx_half, cy_half, two_flo_c, two_df_c;
  double lam, margin;
};

}  // namespace osar

struct osar_batch {
  osar::Guards guards;  // guard regions behind device buffers (guard_bytes)
  int S = 0;
  int prec = OSAR_FP32;
  int Kp = 0;
  int rows = 0;          // sum of Mp over scenes
  int64_t blocks = 0;    // sum of packed blocks
  int nseg = 0;
  int items = 0;         // sum of nb (finalize items)
  int seg_len = 0;       // blocks per matvec segment (autotuned)
  int gram_sb = 8;       // Gram tile order: super-blocks of sb x sb blocks
  int gram_lpt = 0;      // 1: the largest scenes' tiles first (autotuned)
  double tune_gram_ms[2] = {0.0, 0.0};  // Gram update: default order, chosen
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  osar_status sticky = OSAR_OK;
  std::string last_error;

  std::vector<osar_config> cfg;
  std::vector<osar::SceneDesc> desc_h;
  std::vector<int> n_h;          // pulses per scene (host mirror)
  std::vector<int> active_h;
  std::vector<int> power_first_h, power_iters_h;
  bool fresh = true;

  // device
  osar::SceneDesc* desc = nullptr;
  osar::DevScalars* sc = nullptr;   // one per scene
  int* row_scene = nullptr;         // scene of each stacked row
  double* gam = nullptr;            // S x 3 platform positions of the push
  double2* d = nullptr;             // S x Kp pulse data of the push
  float2* d32 = nullptr;
  ulonglong2* turns = nullptr;      // stacked rows
  double2 *b = nullptr, *c = nullptr, *z = nullptr, *v = nullptr, *w = nullptr;
  void *zt = nullptr, *vt = nullptr;
  double2* part = nullptr;          // per finalize item
  double* bmax = nullptr;
  void* g_hi = nullptr;
  __nv_bfloat162* g_lo = nullptr;
  void* segpart = nullptr;
  void* tilepart = nullptr;
  int4* segs = nullptr;             // (J, I0, I1, slot), scene-local J, I
  int* seg_scene = nullptr;
  int* seg_begin = nullptr;         // per scene: nb + 1 global segment indices
  int2* items_dev = nullptr;        // (scene, K)
  int4* gram_tiles = nullptr;       // (A rows, B rows, out block, scene)
  int n_gram_tiles = 0;
  std::vector<int4> gram_tiles_all; // every scene's tiles (host)
  __nv_bfloat16* Apl = nullptr;     // split: 6 x rows x Kp
  void* A = nullptr;                // FP32 / FP64: rows x Kp complex
  CUtensorMap map1, map2;
  double2* h_pinned = nullptr;      // S x Kp staging
  double* h_gam = nullptr;
  int* h_active = nullptr;
  cudaEvent_t stage_ev = nullptr;

  // captured bursts: one graph per step count
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;

  int64_t launches = 0;
  int64_t dev_bytes = 0;
};

namespace osar {

// k_batch.cu launchers
cudaError_t batch_launch_phase(osar_batch* B);
cudaError_t batch_launch_gram(osar_batch* B);
cudaError_t batch_launch_data_update(osar_batch* B);
cudaError_t batch_launch_power(osar_batch* B, int max_steps);
cudaError_t batch_launch_burst_begin(osar_batch* B);
cudaError_t batch_launch_iter_begin(osar_batch* B, double tol);
cudaError_t batch_launch_fista_step(osar_batch* B);
cudaError_t batch_launch_matvec(osar_batch* B, const void* xt, int gated,
                                int pstep);
bool batch_make_tensor_maps(osar_batch* B, std::string* err);

// k_gemm_tc.cu / k_gemm_simt.cu entry points shared with the batch
cudaError_t launch_gram_tc_tiles(cudaStream_t st, int sm_count,
                                 const CUtensorMap& m1, const CUtensorMap& m2,
                                 const int4* tiles, int n_tiles, float2* g_hi,
                                 __nv_bfloat162* g_lo, int kp, int* err);
cudaError_t launch_gram_simt_tiles(cudaStream_t st, int prec, const void* A,
                                   int kp, void* g_hi, const int4* tiles,
                                   int n_tiles);
bool encode_plane_map(CUtensorMap* m, void* base, int cols, int rows,
                      int planes, int box_planes, std::string* err);

}  // namespace osar
