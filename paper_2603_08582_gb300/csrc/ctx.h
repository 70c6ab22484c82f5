// Host-side context of libosar and the launchers each kernel file exports.
#pragma once

#include <cstddef>

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "osar.h"
#include "common.cuh"
#include "guard.h"

namespace osar {

constexpr double C_LIGHT = 299792458.0;
constexpr int MAX_LAMBDAS = 8;  // solutions of a lambda path

// lambda settings of the path's solutions (relative factors or absolute)
struct LamSet {
  double v[MAX_LAMBDAS];
  int n;
};

// Scalars of the online state that live on the device so that no step of a
// pulse or a FISTA burst needs a host round trip.  A lambda path keeps one
// per solution: entry 0 holds the shared fields (L_n, tau, mu, tol, error,
// queue, pass count) and solution 0's; entry l > 0 only solution l's (t,
// lambda, converged, iters, done).
struct DevScalars {
  double t;         // momentum scalar t_k of Algorithm 1
  double t_next;    // t_{k+1} of the step in flight
  double lip;       // L_n
  double tau;       // 1 / L_n
  double lambda;    // lambda_n
  double mu;        // last Rayleigh quotient of the power iteration
  double inv_norm;  // 1 / |G v| of the last power step
  double tol;       // stop tolerance of the current burst call
  int32_t converged;
  int32_t iters;    // steps taken in the current osar_iterate call
  int32_t n;        // pulses pushed
  int32_t error;    // device-side error code (bounded waits)
  uint32_t done;    // blocks finished in the current grid (last-block steps)
  uint32_t pad;
  uint32_t mvq[2];  // matvec work queue: next item, CTAs finished
  unsigned long long passes;  // Gram passes that did work (instrumentation)
};

// Device address of the matvec work queue inside a device-resident
// DevScalars (pointer arithmetic only; the host never reads it).
inline unsigned* matvec_queue(DevScalars* s) {
  return reinterpret_cast<unsigned*>(reinterpret_cast<char*>(s) +
                                     offsetof(DevScalars, mvq));
}

enum KernelClass {
  KCL_PHASE = 0, KCL_DICT = 1, KCL_GRAM = 2, KCL_BUPD = 3, KCL_MATVEC = 4,
  KCL_FIN = 5, KCL_POWFIN = 6, KCL_CORR = 7, KCL_DAPPLY = 8, KCL_COUNT = 9
};

// A captured unrolled-gradient sequence and what it was captured for.
struct AdjGraph {
  cudaGraphExec_t exec = nullptr;
  int T = 0, C = 0;
  void* buf = nullptr;
  size_t bytes = 0;
  int64_t kernels = 0;  // launches one replay stands for
};

struct ProfEvent {
  int kind;
  cudaEvent_t a, b;
};

// Pixel-space Gram form (config pixel_gram, binary edgelet dictionary H):
// the context runs as a pixel-basis one (its Gram is P_n = sum_s F_s^H F_s,
// N x N, its data vector b_pix = sum_s F_s^H d_s) and this holds the
// coefficient side: G_n = H^H P_n H and b_n = H^H b_pix are applied, never
// stored.
struct PixGram {
  bool dense = false;         // a dense dictionary D (Gaussian or host) in
                              // the context's D / Dpl, not edgelet lists
  void* upart = nullptr;      // dense: partial sums of u = D x (chunks x Np)
  void* apart = nullptr;      // dense: partial sums of D^H w (chunks x Mp)
  int M = 0;                  // atoms
  int Mp = 0;                 // atoms padded to BLK
  int nb = 0;                 // Mp / BLK
  int* pix_ptr = nullptr;     // first entry of pixel p in pix_atom (N + 1)
  int* pix_atom = nullptr;    // atoms covering each pixel, ascending
  double2* c = nullptr;       // c_hat (Mp)
  double2* z = nullptr;       // z of Algorithm 1 (Mp)
  double2* b = nullptr;       // H^H b_pix (Mp)
  double2* v = nullptr;       // power vector (Mp)
  double2* w = nullptr;       // G v (Mp)
  double2* part = nullptr;    // per-block partial sums (nb)
  double* bmax = nullptr;     // per-block max |b_m|^2 (blocks of the b grid)
};

}  // namespace osar

struct osar_ctx {
  osar_config cfg;
  osar::PixGram* pg = nullptr;  // pixel-space Gram form, or NULL
  int prec = OSAR_FP64;
  bool dict = false;  // overcomplete / explicit dictionary present
  bool edgelet = false;  // binary edgelet dictionary (atom pixel lists)
  int M = 0, N = 0, K = 0;
  int Mp = 0, Np = 0, Kp = 0;
  int nb = 0;          // Mp / BLK
  int64_t nblk = 0;    // packed upper blocks
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;

  osar_status sticky = OSAR_OK;
  std::string last_error;

  // device state
  osar::DevScalars* scal = nullptr;  // n_lam entries (lambda path)
  int n_lam = 1;                     // solutions of the lambda path
  osar::LamSet lam;                  // their lambda settings
  double2* b = nullptr;        // data vector b_n (Mp)
  double2* c = nullptr;        // c^(k) == c_hat after a burst (n_lam x Mp)
  double2* z = nullptr;        // z^(k) (n_lam x Mp)
  double2* v = nullptr;        // power-iteration vector, unit norm (Mp)
  double2* w = nullptr;        // G v scratch (Mp)
  double2* xtmp = nullptr;     // scratch vector for osar_gram_apply (Mp)
  void* zt = nullptr;          // z in the matvec's precision (n_lam x Mp)
  void* vt = nullptr;          // v in the matvec's precision (Mp)
  void* xt = nullptr;          // osar_gram_apply input, matvec precision (Mp)
  double2* part = nullptr;     // per-block partial sums (nb)
  double2* d_dev = nullptr;    // staged pulse data (Kp)
  ulonglong2* turns = nullptr; // per-pixel fixed-point phase terms (Np)
  void* g_hi = nullptr;        // packed Gram, float2 or double2 per entry
  __nv_bfloat162* g_lo = nullptr;  // TwoSum compensation word (split-BF16),
                                   // bf16 (re, im) per entry
  void* segpart = nullptr;     // matvec segment partials (nseg x BLK)
  void* tilepart = nullptr;    // matvec per-block partials (nblk x BLK)
  void* segpart2 = nullptr;    // partials of a second vector: the fused
  void* tilepart2 = nullptr;   // first step's G z_1, or solution 1's G z
  void* segpart_x = nullptr;   // lambda path: partials of solutions 2..
  void* tilepart_x = nullptr;
  bool first_ready = false;    // segpart2 / tilepart2 hold G z_1 for the burst
  float2* gp_col = nullptr;    // Gram update's fused power step: column
  float2* gp_row = nullptr;    // partials (nblk x BLK), half-row partials
                               // (nblk x 2 x BLK)
  bool gp_ready = false;       // gp_col / gp_row hold G_n v for the first power step
  int4* segs = nullptr;        // matvec work items (J, I0, I1, slot)
  int* seg_begin = nullptr;    // first segment of block column J (nb + 1)
  double* bmax = nullptr;      // per-block max |b_j|^2 (data update)
  float2* d32 = nullptr;       // staged pulse data in FP32 (Kp)
  int nseg = 0;
  int4* gram_tiles = nullptr;  // (I, J, packed block, 0), L2-friendly order
  // tile pairs for CTA-pair tcgen05 launches: (I0, J | slice << 16, I1,
  // 1 if the second block is missing (I1 = I0 then))
  int4* gram_pairs = nullptr;
  int n_gram_pairs = 0;
  int4* dict_pairs = nullptr;
  int n_dict_pairs = 0;
  int tc_pair_limit = 0;       // co-resident CTA pairs (0 = not queried yet)
  int4* dict_tiles = nullptr;  // (atom block, frequency block | slice << 16, 0, 0)
  int n_dict_tiles = 0;
  int dict_slices = 1;         // split-K slices of the dictionary product
  float2* dict_part = nullptr; // split: FP32 slice partials (slices x Mp x Kp)
  // per-pulse operands
  void* A = nullptr;           // FP64/FP32: Mp x Kp complex, atom-major
  void* F = nullptr;           // FP64/FP32 + dictionary: Kp x Np complex
  void* D = nullptr;           // FP64/FP32 + dictionary: Mp x Np complex
  __nv_bfloat16* Apl = nullptr;  // split: 6 planes x Mp x Kp
  __nv_bfloat16* Fpl = nullptr;  // split + dictionary: 6 planes x Kp x Np
  __nv_bfloat16* Dpl = nullptr;  // split + dictionary: 4 planes x Mp x Np
  int* atom_ptr = nullptr;       // edgelets: first entry of atom m (M + 1)
  int* atom_pix = nullptr;       // edgelets: pixels of the atoms, in order
  CUtensorMap map_a_rows1;     // Apl, box (KC, 128, 1)
  CUtensorMap map_a_rows2;     // Apl, box (KC, 128, 2)
  CUtensorMap map_d_rows1;     // Dpl, box (KC, 128, 1)
  CUtensorMap map_f_rows1;     // Fpl, box (KC, 128, 1)
  CUtensorMap map_f_rows2;     // Fpl, box (KC, 128, 2)
  // overlapped synthesis (dictionary models): the next pulse's phase and
  // dictionary product on a side stream while the current burst runs
  cudaStream_t side = nullptr;
  cudaEvent_t ev_free = nullptr;   // main: last reader of the synthesis buffers done
  cudaEvent_t ev_synth = nullptr;  // side: synthesis of the pushed pulse done
  // step counts of recent bursts, copied to pinned memory without a wait
  static constexpr int ITERS_RING = 4;
  cudaEvent_t ev_iters[ITERS_RING] = {};
  int32_t* h_iters = nullptr;      // ITERS_RING pinned counts
  int64_t iters_seq = 0;           // counts queued so far
  int iters_est = 20;              // FISTA steps expected in a burst
  bool free_stale = false;         // ev_free predates a captured push
  bool synth_side = false;         // the last push synthesised on `side`
  // deferred Gram update (defer_gram): G_n forms on `side` into the second
  // buffer while pulse n's passes read G_{n-1} and add A_n^H A_n x
  void* gn_hi = nullptr;               // the other Gram buffer
  // with two Gram buffers: a device slot holding g_hi's address, rewritten
  // in stream order at each swap, which the matvec reads (so that a burst
  // captured in a CUDA graph follows the swaps)
  void** gram_ref = nullptr;
  __nv_bfloat162* gn_lo = nullptr;
  __nv_bfloat16* Apl_alt = nullptr;    // the other forward-block buffer
  CUtensorMap map_alt_rows1;           // Apl_alt, box (KC, 128, 1)
  CUtensorMap map_alt_rows2;           // Apl_alt, box (KC, 128, 2)
  cudaEvent_t ev_gram = nullptr;       // side: the pending Gram update done
  // gram_ahead: main stream past the last push's power steps (their reads of
  // the Gram, of v and of the fused power step's partials are done)
  cudaEvent_t ev_steps = nullptr;
  cudaEvent_t ev_mark[2] = {};         // main: all work before push n (n % 2)
  bool gram_pending = false;           // g_hi holds G_{n-1}, gn_hi gets G_n
  float2* corr = nullptr;              // A_n^H A_n x per partial set (2 x Mp)
  float2* corr_u = nullptr;            // A_n x: nb block partials, then the sum
  unsigned* corr_tick = nullptr;       // last-CTA ticket of the A_n x sums
  // non-white pulses (osar_push_pulse_var): weights 1 / sigma_k in a pinned
  // host ring, copied on the synthesis stream into a device slot by pulse
  // parity; synth_w is the slot the phase kernels of the synthesis being
  // queued scale their rows by (nullptr: white)
  double* h_wring = nullptr;          // RING x Kp pinned
  cudaEvent_t w_ev[8] = {};
  int w_pos = 0;
  int w_slot = -1;                    // host slot of the push in progress
  double* wk_dev = nullptr;           // 2 x Kp device
  const double* synth_w = nullptr;
  // osar_get_coeffs_async completion events (OSAR_COPY_SLOTS)
  cudaEvent_t copy_ev[4] = {};
  // pinned staging ring for pulse data (slots of Kp complex)
  static constexpr int RING = 8;
  double2* h_ring = nullptr;
  cudaEvent_t ring_ev[RING] = {};
  int ring_pos = 0;
  // simulate scratch
  double2* sim_rho = nullptr;  // Np
  double2* sim_nz = nullptr;   // nonzero coefficient values (Mp)
  int* sim_idx = nullptr;      // nonzero coefficient indices (Mp)
  double2* sim_d = nullptr;    // simulated pulse (Kp)

  osar::Guards guards;  // guard regions behind device buffers (guard_bytes)

  // osar_get_metrics scratch (allocated by its first call): sums + mask
  void* metrics_buf = nullptr;

  // differentiation-form scratch (allocated by the first unrolled gradient)
  void* adj_buf = nullptr;
  size_t adj_bytes = 0;
  osar::AdjGraph adj_graph;  // the gradient's device sequence, captured

  // host mirror
  int n = 0;
  bool fresh = true;
  int64_t launches = 0;
  int64_t pushes_ahead = 0;     // pushes whose Gram update ran ahead (gram_ahead)
  int32_t ahead_grid_last = 0;  // side-stream SMs of the last such push
  int64_t dev_bytes = 0;

  // profiling
  bool prof_on = false;
  uint32_t prof_mask = ~0u;  // kernel classes bracketed while prof_on
  int32_t prof_every[osar::KCL_COUNT] = {1, 1, 1, 1, 1, 1, 1, 1, 1};  // stride
  int64_t prof_seq[osar::KCL_COUNT] = {0};  // launches seen per class
  std::vector<osar::ProfEvent> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[osar::KCL_COUNT] = {0};
  int64_t prof_launches[osar::KCL_COUNT] = {0};
};

namespace osar {

// ---- deferred Gram update ---------------------------------------------------
// the main stream waits for a pending Gram update, whose result its passes
// then read directly (no-op when none is pending)
cudaError_t settle_gram(osar_ctx* ctx);
// writes g_hi's address into gram_ref on the context's stream (no-op
// without a second Gram buffer)
cudaError_t launch_set_gram_ref(osar_ctx* ctx);

// ---- launch bracketing for the per-kernel profile -------------------------
void prof_begin(osar_ctx* ctx, int kind, ProfEvent* ev);
void prof_end(osar_ctx* ctx, ProfEvent* ev);

// ---- k_edgelet.cu -----------------------------------------------------------
// A_s = F_s H for the binary edgelet dictionary (sums of pixel phase rows)
cudaError_t launch_edgelet(osar_ctx* ctx, int grid_cap);
// the image H c of the simulation's sparse coefficients (sim_idx / sim_nz)
cudaError_t launch_sim_rho_edgelet(osar_ctx* ctx, int nnz);

// ---- k_pixgram.cu ------------------------------------------------------------
// b_n = H^H b_pix, lambda_n and the pulse's power steps on G_n = H^H P_n H
cudaError_t pg_after_push(osar_ctx* ctx);
cudaError_t prepare_pixgram_kernels();  // shared-memory carve-out, as the burst's
cudaError_t pg_burst_begin(osar_ctx* ctx);
cudaError_t pg_fista_step(osar_ctx* ctx);

// ---- k_pixgram_dense.cu -----------------------------------------------------
// the pixel-space form with a dense dictionary: u = D x into the pass's input
// vector (zt), and (D^H w)_m with b_n / lambda_n (mode 0), a power step
// (mode 1) or Algorithm 1's step (mode 2)
int pgd_chunks(const osar_ctx* ctx);
int pgd_adjoint_chunks(const osar_ctx* ctx);
cudaError_t pgd_forward(osar_ctx* ctx, const double2* x, int gated);
cudaError_t pgd_adjoint(osar_ctx* ctx, int mode, int last_step);

// ---- k_defer.cu -------------------------------------------------------------
// corr[set] = A_n^H (A_n x) for the pending forward block (nothing when no
// Gram update is pending); gate: skip when that flag is set
cudaError_t launch_corr(osar_ctx* ctx, const void* xt, int set,
                        const int32_t* gate);
// the correction a finalize adds for partial set `set`, or nullptr
const float2* corr_set(const osar_ctx* ctx, int set);

// ---- k_phase.cu -------------------------------------------------------------
cudaError_t launch_pixel_turns(osar_ctx* ctx, const double gamma[3]);
// grid_cap > 0: grid-stride over at most 4 x grid_cap CTAs (split-BF16)
cudaError_t launch_phase(osar_ctx* ctx, int grid_cap);
cudaError_t launch_dictionary_build(osar_ctx* ctx, const double* host_dict);
cudaError_t launch_simulate(osar_ctx* ctx, int nnz, double2* d_out);

// ---- k_gemm_simt.cu --------------------------------------------------------
cudaError_t launch_dict_simt(osar_ctx* ctx);
cudaError_t launch_gram_simt(osar_ctx* ctx);

// ---- k_gemm_tc.cu ----------------------------------------------------------
bool make_tensor_maps(osar_ctx* ctx, std::string* err);
// grid_cap > 0: at most that many CTAs for the product (the reduction that
// follows is a short full-grid kernel)
cudaError_t launch_dict_tc(osar_ctx* ctx, int grid_cap);
int dict_slices(int np);
// G += A^H A in place, or, with dst_hi set, dst = G + A^H A (G unchanged);
// grid_cap > 0: at most that many SMs.  power: where the context holds the
// buffers (gp_col), the update also forms the partials of G_n v for the
// pulse's first power step and sets gp_ready.
cudaError_t launch_gram_tc(osar_ctx* ctx, void* dst_hi = nullptr,
                           __nv_bfloat162* dst_lo = nullptr, int grid_cap = 0,
                           bool power = false);

// ---- k_fista.cu ------------------------------------------------------------
cudaError_t launch_data_update(osar_ctx* ctx);
// fuse: the last step also applies the Gram to the next burst's z_1 = c_hat
// (burst started here; its first FISTA step reuses that pass)
cudaError_t launch_power_steps(osar_ctx* ctx, int steps, bool fuse);
cudaError_t prepare_burst_kernels();  // shared-memory carve-out of the burst kernels
cudaError_t launch_set_working(osar_ctx* ctx);
cudaError_t launch_burst_begin(osar_ctx* ctx);
cudaError_t launch_iter_begin(osar_ctx* ctx, double tol);
cudaError_t launch_fista_step(osar_ctx* ctx);
cudaError_t launch_gram_apply(osar_ctx* ctx, const double2* x, double2* y);
cudaError_t launch_gram_expand(osar_ctx* ctx, int r0, int rows, double2* dense);
cudaError_t launch_gram_entries(osar_ctx* ctx, const int2* rc, int count,
                                double2* out);
size_t gram_apply_scratch_bytes(const osar_ctx* ctx);
// k_static.cu: look up the allocation-free apply's static array on the
// current device (errors are left to that entry point to report)
void prepare_static_scratch();
cudaError_t launch_matvec(osar_ctx* ctx, const void* xt);
// One Gram pass y = G x over the working-precision vector xt (Mp), into the
// FP64 vector y; gated: the pass and its finalize skip once solution 0 has
// met the stop rule.  kind: the profile class of the finalize.
cudaError_t launch_gram_pass(osar_ctx* ctx, const void* xt, int gated,
                             double2* y, int kind);

// ---- k_adjoint.cu ----------------------------------------------------------
cudaError_t run_unroll_grad(osar_ctx* ctx, int T, int C, double lambda,
                            double tau, double t0, const double* c0,
                            const double* ctrue, double* loss, double* dlam,
                            double* dtau, double* db, double* cT);
cudaError_t launch_gram_apply_scratch(osar_ctx* ctx, const double2* x,
                                      double2* y, void* scratch);

}  // namespace osar
