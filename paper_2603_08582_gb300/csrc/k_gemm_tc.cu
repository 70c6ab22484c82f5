// Split-BF16 complex GEMM on tcgen05 tensor cores (sm_103a), used for the
// dictionary apply (Eq. 6) and the Gram update (Eqs. 12-13).
//
// Each complex operand is stored as bf16 planes [plane][row][k]:
//   block / Gram operand (6 planes): re_hi, im_hi, -re_hi, re_lo, im_lo, -re_lo
//   dictionary operand   (4 planes): re_hi, im_hi, re_lo, im_lo
// with x = hi + lo, hi = rn_bf16(x), lo = rn_bf16(x - hi).  A 128 x 128
// complex output tile C = sum_k op(P)[i][k] Q[j][k] is one real GEMM of
// M = 128, N = 256, K = 2 Kc whose N axis stacks [real part | imaginary part]:
//
//   first half of K  (A = P_re):  B rows = [Q_re ; Q_im]
//   second half of K (A = P_im):  B rows = [Q_im ; -Q_re]
//
// which accumulates  [Re | Im] = [P_re Q_re + P_im Q_im | P_re Q_im - P_im Q_re]
// = conj(P) Q  (Gram), or, with the A operand negated in the second half,
// [P_re Q_re - P_im Q_im | P_re Q_im + P_im Q_re] = P Q  (dictionary).  The
// B operand of each half is one 3-D TMA box spanning two adjacent planes.
// Three products per chunk (hi*hi, hi*lo, lo*hi) run on the tensor pipe with
// FP32 accumulation in tensor memory.
//
// Kernel structure (persistent, one CTA per SM, 320 threads):
//   warp 0  TMA producer: 4-stage ring of 48 KB stages (A hi/lo, B hi/lo).
//   warp 1  TMEM allocation and the single-thread MMA issuer.
//   warps 2-9  epilogue: two warps per TMEM lane quarter, each owning 64 of
//           the 128 output columns, read the 128 x 256 fp32 accumulator in
//           16-column pieces (tcgen05.ld) and either store an FP32 partial
//           (dictionary) or apply a TwoSum read-modify-write to the packed
//           Gram block (hi, lo), which is stored column-major so that a warp
//           (32 consecutive rows) reads and writes 256 contiguous bytes per
//           access.  The Gram words of the next piece are loaded before the
//           current one is processed (~64 KB in flight per SM).
// The accumulator is double-buffered (2 x 256 TMEM columns) so the epilogue
// of tile t overlaps the MMAs of tile t+1.
// CTA-pair variant (clusters of two, cta_group::2): two tiles that share
// their B rows run as one M = 256 MMA on two SMs, each SM loading its own A
// rows and one of the two B planes (32 KB per ring slot instead of 48 KB, 7
// slots); in Gram mode the ring keeps 5 slots and the Gram read-modify-write
// is staged through the rest of the shared memory by bulk copies in
// 8-column pieces; see k_tc_cgemm<true>.  There the epilogue can also apply
// each updated block of G_n to the power vector (the pulse's first power
// step, Eq. 11): row partials T x_J and column partials T^H x_I per block,
// which a finalize kernel sums per output block, so that step reads no Gram.
//
// Accumulation in the tensor pipe rounds its FP32 partial sums toward zero,
// which biases long reductions (|A| shrinks by ~(steps) 2^-24).  The
// dictionary reduction runs over N = 16384 pixels, so it is split into
// slices of at most 4096 pixels (split-K); each slice writes an FP32 partial
// and a small kernel sums the slices with round-to-nearest before the bf16
// split.  The Gram reduction (2K <= 2048 terms) stays in one accumulator.  Every mbarrier wait is bounded
// (2 s); a timeout sets the device error word, stops the other roles, drains
// in-flight TMA loads and MMAs, and frees TMEM before the kernel returns.
#include <cudaTypedefs.h>

#include <algorithm>

#include "ctx.h"

namespace osar {
namespace {

constexpr int TILE_A_BYTES = BLK * KC * 2;        // 128 rows x 64 B
constexpr int TC_THREADS = 320;
constexpr int EPI_THREADS = 256;
constexpr uint32_t TMEM_COLS = 512;

// Ring geometry: one CTA per tile (B = 256 rows, two planes) or CTA pairs
// (B = this CTA's 128 rows, one plane).
// Gram epilogue of the pair kernel: per 64-column half of the tile, a
// G_COLS-column piece of the block (hi 8 KB + lo 4 KB, contiguous in the
// column-major block) is staged by a bulk copy; two slots per half.  The
// narrower the pieces, the deeper the operand ring beside them: 16-column
// pieces left 4 ring slots, 8-column pieces leave 5 (3.8 against 4.2 ms per
// update; a 3-slot ring ran 12 % slower than 4).  4-column pieces leave 6
// but cost more in per-piece barriers and copies (4.2 ms).
constexpr int G_COLS = 8;
constexpr int G_PIECES = 64 / G_COLS;            // per half and tile
constexpr int G_PIECE_HI = G_COLS * BLK * 8;
constexpr int G_PIECE_LO = G_COLS * BLK * 4;
constexpr int G_SLOT = G_PIECE_HI + G_PIECE_LO;  // 12 KB
constexpr int PAIR_GRAM_STAGES =  // operand ring beside the four slots
    G_COLS == 16 ? 4 : G_COLS == 8 ? 5 : 6;

template <bool PAIR>
struct TcCfg {
  static constexpr int STAGES = PAIR ? 7 : 4;
  static constexpr int B_BYTES = (PAIR ? 1 : 2) * BLK * KC * 2;
  static constexpr int STAGE_BYTES = 2 * TILE_A_BYTES + 2 * B_BYTES;  // 32 / 48 KB
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};
static_assert(TcCfg<true>::SMEM <= 227 * 1024 && TcCfg<false>::SMEM <= 227 * 1024,
              "tcgen05 ring exceeds shared memory");
// Fused power step (TcParams::pv): per tile parity and half, the 4 warps'
// column sums of their 32 rows (128 floats each), combined after the tile,
// and the half's 64 entries of x_J.
constexpr int PW_RED_BYTES = 2 * 2 * 4 * BLK * 4;  // 8 KB
constexpr int PW_X_BYTES = 2 * 2 * 64 * 8;         // 2 KB
static_assert(PAIR_GRAM_STAGES * TcCfg<true>::STAGE_BYTES + 4 * G_SLOT +
                      PW_RED_BYTES + PW_X_BYTES <=
                  TcCfg<true>::STAGES * TcCfg<true>::STAGE_BYTES,
              "staged Gram epilogue does not fit beside the operand ring");
static_assert(G_COLS == 8, "the fused power step reduces 8-column pieces");
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

struct TcParams {
  // (A row block, B row block | slice << 16, output block, 0); row blocks
  // index the operand tensors' rows in units of 128, the output block is the
  // packed Gram block to update (Gram mode)
  const int4* tiles;
  int n_tiles;
  int k_chunks;    // KC chunks per half of the reduction (whole K)
  int k_slice;     // KC chunks per half handled by one tile
  int a_lo;        // plane offset of the lo part on the A side
  int b_lo;        // plane offset of the lo part on the B side
  int neg_second;  // negate A in the second half (plain product P Q)
  int mode;        // 0: FP32 partial output, 1: packed Gram update
  float2* part;    // mode 0: [slice][rows][part_ld] partial sums
  int part_ld;
  int64_t part_slice;
  float2* g_hi;          // the Gram written
  __nv_bfloat162* g_lo;  // compensation word, bf16 (re, im), or NULL
  const float2* gs_hi;   // the Gram read (g_hi for an update in place)
  const __nv_bfloat162* gs_lo;
  // Fused power step on the updated Gram (pair kernel, Gram mode), or NULL:
  // w = G x for x = pv (FP32, Mp entries).  Per stored block (I, J):
  //   pcol[blk][c]        = sum_r conj(T[r][c]) x_I[r]   (all 128 columns;
  //                         on a diagonal block the block's whole product)
  //   prow[blk][h][r]     = sum over the 64 columns c of half h of T[r][c] x_J[c]
  //                         (off-diagonal blocks only)
  const float2* pv;
  float2* pcol;
  float2* prow;
  int nb;
  int* err;
};

// One W-column piece of the Gram read-modify-write for this thread's row:
// hi + lo += delta with an error-free TwoSum, the new rounding error kept as
// the bf16 compensation word.  (Keeping 8 bits of an error that is at most
// half an FP32 ulp of hi still leaves the pair 2^-33-accurate, far below the
// 2^-17 of the split-BF16 products, and saves a quarter of the traffic.)
// Blocks are column-major, so entry (row, c) is at c * 128 + row and the 32
// lanes of a warp (32 consecutive rows) touch contiguous bytes per access.
template <int W, bool KEEP = false>
__device__ __forceinline__ void gram_piece(float2* gh, __nv_bfloat162* gl,
                                           float2 (&h)[W],
                                           const __nv_bfloat162 (&l)[W],
                                           const float* re, const float* im,
                                           bool comp) {
#pragma unroll
  for (int q = 0; q < W; ++q) {
    float2 hv = h[q];
    if (comp) {
      const float2 lv = __bfloat1622float2(l[q]);
      float s0, e0, s1, e1;
      two_sum(hv.x, __fadd_rn(re[q], lv.x), s0, e0);
      two_sum(hv.y, __fadd_rn(im[q], lv.y), s1, e1);
      hv = make_float2(s0, s1);
      gl[q * BLK] = __floats2bfloat162_rn(e0, e1);
    } else {
      hv.x += re[q];
      hv.y += im[q];
    }
    gh[q * BLK] = hv;
    if (KEEP) h[q] = hv;  // the updated entry, for a fused power step
  }
}

// One 8-column piece of the fused power step for this thread's row r of
// block (I, J), h = the updated entries T[r][c0 .. c0+7]:
//   racc += sum_c T[r][c] x_J[c]                        (row partial)
//   red[j] = sum over the warp's 32 rows of conj(T[r][c]) x_I[r]
// for the piece's 16 floats j = 2 c + (0: re, 1: im).  The column sums are
// a butterfly reduce-scatter: after halving over lane bits 4..1 and a final
// exchange over bit 0, lanes 2j and 2j + 1 both hold float j.
__device__ __forceinline__ void power_piece(const float2 (&h)[8], float2 xi,
                                            const float2* xj_src, int lane,
                                            float2& racc, float* red) {
  float2 xj[8];  // x_J[c0 .. c0+7], from shared memory (one broadcast each)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = reinterpret_cast<const float4*>(xj_src)[k];
    xj[2 * k] = make_float2(v.x, v.y);
    xj[2 * k + 1] = make_float2(v.z, v.w);
  }
  float v[16];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    racc.x = fmaf(h[c].x, xj[c].x, racc.x);
    racc.x = fmaf(-h[c].y, xj[c].y, racc.x);
    racc.y = fmaf(h[c].x, xj[c].y, racc.y);
    racc.y = fmaf(h[c].y, xj[c].x, racc.y);
    v[2 * c] = fmaf(h[c].x, xi.x, h[c].y * xi.y);
    v[2 * c + 1] = fmaf(h[c].x, xi.y, -(h[c].y * xi.x));
  }
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1) {
    const int bit = w * 2;  // lane bit 4, 3, 2, 1
    const bool up = (lane & bit) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const float send = up ? v[k] : v[k + w];
      const float keep = up ? v[k + w] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  if ((lane & 1) == 0) red[lane >> 1] = v[0];
}

__device__ __forceinline__ void load_piece(const float2* gh,
                                           const __nv_bfloat162* gl,
                                           float2 (&h)[16], __nv_bfloat162 (&l)[16],
                                           bool comp) {
#pragma unroll
  for (int q = 0; q < 16; ++q) h[q] = gh[q * BLK];
  if (comp) {
#pragma unroll
    for (int q = 0; q < 16; ++q) l[q] = gl[q * BLK];
  }
}

// PAIR = false: one CTA per tile (the layout described at the top).
// PAIR = true: clusters of two CTAs on two SMs compute two tiles that share
// the B rows (blocks (I0, J) and (I1, J)) with one M = 256 tcgen05 MMA: each
// CTA loads its own 128 A rows and one of the two B planes of the N = 256
// axis ([Q_re | Q_im] or [Q_im | -Q_re]), i.e. 32 KB per k-chunk instead of
// 48 KB, and keeps its own 128 x 256 accumulator in its TMEM.  The even CTA
// issues the MMAs; both CTAs' loads complete on the even CTA's stage
// barrier, the MMA commits release the stage in both CTAs, and the odd
// CTA's epilogue warps release the accumulator through the even CTA's
// barrier.  A tile pair whose second block is missing (odd count) marks it
// so; the odd CTA then computes a copy and stores nothing.
template <bool PAIR>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_cgemm(const __grid_constant__ CUtensorMap mapA,
               const __grid_constant__ CUtensorMap mapB, const TcParams p) {
  using C = TcCfg<PAIR>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* tfull = empty + C::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint64_t* gfull = drain + 1;    // staged Gram pieces: slot landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gfull + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  // pair kernel, Gram mode: shorter operand ring, Gram pieces staged after it
  const bool staged = PAIR && p.mode == 1;
  const int nst = staged ? PAIR_GRAM_STAGES : C::STAGES;
  const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int units = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  // a failed wait stops the peer CTA too
  auto stop_peer = [&]() {
    if (PAIR) st_cluster_u32((const void*)abort_flag, rank ^ 1u, 1u);
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], PAIR ? 2 * (EPI_THREADS / 32) : EPI_THREADS);
    }
    for (int b = 0; b < 4; ++b) mbar_init(&gfull[b], 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
    fence_proxy_async();
    tma_prefetch_desc(&mapA);
    tma_prefetch_desc(&mapB);
  }
  if (warp == 1) {
    if (PAIR) {
      tmem_alloc_pair(tmem_slot, TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(tmem_slot, TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  if (PAIR)
    cluster_sync();  // both CTAs' barriers exist before any remote arrive
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int total_k = 2 * p.k_slice;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------ TMA producer
      uint32_t issued[C::STAGES];
      for (int s = 0; s < C::STAGES; ++s) issued[s] = 0;
      int stage = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = unit; ok && t < p.n_tiles; t += units) {
        const int4 tile = p.tiles[t];
        const int ra = (PAIR && rank ? tile.z : tile.x) * BLK;
        const int rb = (tile.y & 0xFFFF) * BLK;
        const int k0 = (tile.y >> 16) * p.k_slice;
        for (int kc = 0; kc < total_k; ++kc) {
          if (!mbar_wait_bounded(&empty[stage], ph ^ 1, abort_flag, p.err,
                                 WAIT_LIMIT_NS)) {
            ok = false;
            stop_peer();
            break;
          }
          const int half = kc >= p.k_slice ? 1 : 0;
          const int k = (k0 + kc - half * p.k_slice) * KC;
          uint8_t* sb = smem + stage * C::STAGE_BYTES;
          // B: both planes of the N axis here, or this CTA's one plane
          const int bp = half + (PAIR ? (int)rank : 0);
          if (PAIR && rank) {
            // the pair's bytes all complete on the even CTA's barrier
            const uint32_t bar = cluster_addr(&full[stage], 0u);
            tma_load_3d_peer(sb, &mapA, bar, k, ra, half);
            tma_load_3d_peer(sb + TILE_A_BYTES, &mapA, bar, k, ra, half + p.a_lo);
            tma_load_3d_peer(sb + 2 * TILE_A_BYTES, &mapB, bar, k, rb, bp);
            tma_load_3d_peer(sb + 2 * TILE_A_BYTES + C::B_BYTES, &mapB, bar, k,
                             rb, bp + p.b_lo);
          } else {
            mbar_expect_tx(&full[stage], (PAIR ? 2 : 1) * C::STAGE_BYTES);
            tma_load_3d(sb, &mapA, &full[stage], k, ra, half);
            tma_load_3d(sb + TILE_A_BYTES, &mapA, &full[stage], k, ra,
                        half + p.a_lo);
            tma_load_3d(sb + 2 * TILE_A_BYTES, &mapB, &full[stage], k, rb, bp);
            tma_load_3d(sb + 2 * TILE_A_BYTES + C::B_BYTES, &mapB,
                        &full[stage], k, rb, bp + p.b_lo);
          }
          issued[stage]++;
          if (++stage == nst) {
            stage = 0;
            ph ^= 1;
          }
        }
      }
      // Drain: every load this thread issued must land before the CTA exits:
      // its own barrier says so, or (odd CTA of a pair, whose loads complete
      // on the even CTA's barrier) the MMA commit that released the stage.
      volatile int no_abort = 0;
      for (int s = 0; s < nst; ++s)
        if (issued[s]) {
          if (PAIR && rank)
            mbar_wait_bounded(&empty[s], (issued[s] - 1) & 1, &no_abort, p.err,
                              WAIT_LIMIT_NS);
          else
            mbar_wait_bounded(&full[s], (issued[s] - 1) & 1, &no_abort, p.err,
                              WAIT_LIMIT_NS);
        }
    }
  } else if (warp == 1) {
    if (lane == 0 && (!PAIR || rank == 0)) {
      // -------------------------------------------------------- MMA issuer
      const int m = PAIR ? 2 * BLK : BLK;
      const uint32_t id_pos = idesc_bf16_f32(m, 256, false);
      const uint32_t id_neg = idesc_bf16_f32(m, 256, true);
      int stage = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      for (int t = unit; ok && t < p.n_tiles; t += units) {
        const bool got =
            PAIR ? mbar_wait_bounded_cluster(&tempty[acc], aph ^ 1, abort_flag,
                                             p.err, WAIT_LIMIT_NS)
                 : mbar_wait_bounded(&tempty[acc], aph ^ 1, abort_flag, p.err,
                                     WAIT_LIMIT_NS);
        if (!got) {
          ok = false;
          stop_peer();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)acc * 256u;
        for (int kc = 0; kc < total_k; ++kc) {
          if (!mbar_wait_bounded(&full[stage], ph, abort_flag, p.err,
                                 WAIT_LIMIT_NS)) {
            ok = false;
            stop_peer();
            break;
          }
          tc_fence_after();
          const int half = kc >= p.k_slice ? 1 : 0;
          const uint32_t id = (half && p.neg_second) ? id_neg : id_pos;
          const uint32_t a_hi = smem_u32(smem + stage * C::STAGE_BYTES);
          const uint32_t a_lo = a_hi + TILE_A_BYTES;
          const uint32_t b_hi = a_hi + 2 * TILE_A_BYTES;
          const uint32_t b_lo = b_hi + C::B_BYTES;
#pragma unroll
          for (int k16 = 0; k16 < KC / 16; ++k16) {
            const uint32_t o = (uint32_t)k16 * 32u;
            const uint64_t dah = smem_desc_sw64(a_hi + o);
            const uint64_t dal = smem_desc_sw64(a_lo + o);
            const uint64_t dbh = smem_desc_sw64(b_hi + o);
            const uint64_t dbl = smem_desc_sw64(b_lo + o);
            const uint32_t first = (kc | k16) != 0 ? 1u : 0u;
            if (PAIR) {
              tc_mma_f16_pair(d, dah, dbh, id, first);
              tc_mma_f16_pair(d, dah, dbl, id, 1u);
              tc_mma_f16_pair(d, dal, dbh, id, 1u);
            } else {
              tc_mma_f16(d, dah, dbh, id, first);
              tc_mma_f16(d, dah, dbl, id, 1u);
              tc_mma_f16(d, dal, dbh, id, 1u);
            }
          }
          if (PAIR)
            tc_commit_pair(&empty[stage], 0x3);
          else
            tc_commit(&empty[stage]);
          if (++stage == nst) {
            stage = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        if (PAIR)
          tc_commit_pair(&tfull[acc], 0x3);
        else
          tc_commit(&tfull[acc]);
        acc ^= 1;
        if (acc == 0) aph ^= 1;
      }
      // Drain: all MMAs issued by this thread complete before TMEM is freed.
      if (PAIR)
        tc_commit_pair(drain, 0x1);
      else
        tc_commit(drain);
      volatile int no_abort = 0;
      mbar_wait_bounded(drain, 0, &no_abort, p.err, WAIT_LIMIT_NS);
    }
  } else if (staged) {
    // ------------------------------------- epilogue, Gram, staged pieces
    // Each 64-column half (4 warps) walks its G_COLS-column pieces of every
    // tile in order; piece n sits in slot n & 1 of its half.  One thread per
    // half bulk-loads a piece into its slot, the 4 warps update it there
    // (TwoSum, in place), and the same thread bulk-stores it back and then
    // loads piece n + 2 into the slot.  Two pieces per half are in flight
    // each way without holding registers, and the next tile's first pieces
    // load while this tile's MMAs run.
    const int q = warp & 3;
    const int colh = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const bool comp = p.g_lo != nullptr;
    const bool loader = lane == 0 && (warp - 2) % 4 == 0;
    uint8_t* slots = smem + PAIR_GRAM_STAGES * C::STAGE_BYTES + colh * 2 * G_SLOT;
    uint64_t* gf = gfull + colh * 2;
    const uint32_t bytes = G_PIECE_HI + (comp ? G_PIECE_LO : 0);
    // offset of piece pc (G_COLS columns) of the block this CTA updates for tile t
    auto piece_off = [&](int t, int pc) {
      const int4 tile = p.tiles[t];
      const int ti = rank ? tile.z : tile.x;
      return packed_block(ti, tile.y & 0xFFFF, p.nb) * (BLK * BLK) +
             (int64_t)(colh * 64 + pc * G_COLS) * BLK;
    };
    auto issue = [&](int t, int pc, int b) {
      const int64_t off = piece_off(t, pc);
      uint8_t* dst = slots + b * G_SLOT;
      mbar_expect_tx(&gf[b], bytes);
      bulk_load(dst, p.gs_hi + off, G_PIECE_HI, &gf[b]);
      if (comp) bulk_load(dst + G_PIECE_HI, p.gs_lo + off, G_PIECE_LO, &gf[b]);
    };
    // fused power step: this half's column-sum buffers (one per tile parity)
    const bool pw = p.pv != nullptr;
    float* pw_red = reinterpret_cast<float*>(
        smem + PAIR_GRAM_STAGES * C::STAGE_BYTES + 4 * G_SLOT);
    float2* pw_x = reinterpret_cast<float2*>(
        smem + PAIR_GRAM_STAGES * C::STAGE_BYTES + 4 * G_SLOT + PW_RED_BYTES);
    int tcount = 0;
    uint32_t issued[2] = {0, 0};
    if (loader && unit < p.n_tiles) {
      issue(unit, 0, 0);
      issue(unit, 1, 1);
      issued[0] = issued[1] = 1;
    }
    int acc = 0;
    uint32_t aph = 0;
    bool fail = false;
    int n = 0;  // pieces of this half processed so far
    // The 4 warps of a half pass the same barriers: every tile they enter
    // has G_PIECES barriers (one more with the power step), and whether to
    // stop is the OR over the half, taken at a barrier, so all of them leave
    // together.
    for (int t = unit; t < p.n_tiles; t += units, ++tcount) {
      const int4 tl = p.tiles[t];
      const bool store = !(rank && (tl.w & 1));
      const int ti = rank ? tl.z : tl.x, tj = tl.y & 0xFFFF;
      float* red = pw_red + ((tcount & 1) * 2 + colh) * 4 * BLK;
      float2* xs = pw_x + ((tcount & 1) * 2 + colh) * 64;
      float2 xi = make_float2(0.f, 0.f), racc = make_float2(0.f, 0.f);
      if (pw && store) {
        // x_I for this row; the half's x_J to shared memory, seen by its
        // 4 warps after the first piece's barrier
        xi = p.pv[ti * BLK + row];
        if (row < 64) xs[row] = p.pv[tj * BLK + colh * 64 + row];
      }
      if (!mbar_wait_bounded(&tfull[acc], aph, abort_flag, p.err,
                             WAIT_LIMIT_NS))
        fail = true;
      fail = __any_sync(0xffffffffu, fail);
      if (fail) stop_peer();
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) +
                            (uint32_t)acc * 256u + (uint32_t)colh * 64u;
      float2 h[G_COLS];  // the piece's updated entries of this thread's row
      for (int pc = 0; pc < G_PIECES; ++pc, ++n) {
        const int b = n & 1;
        const uint32_t gph = (uint32_t)(n >> 1) & 1u;
        float re[G_COLS], im[G_COLS];
        if (!fail) {
          if constexpr (G_COLS == 16) {
            tmem_ld16(base + (uint32_t)(pc * 16), re);
            tmem_ld16(base + 128u + (uint32_t)(pc * 16), im);
          } else if constexpr (G_COLS == 8) {
            tmem_ld8(base + (uint32_t)(pc * 8), re);
            tmem_ld8(base + 128u + (uint32_t)(pc * 8), im);
          } else {
            tmem_ld4(base + (uint32_t)(pc * 4), re);
            tmem_ld4(base + 128u + (uint32_t)(pc * 4), im);
          }
          tmem_wait_ld();
          if (!mbar_wait_bounded(&gf[b], gph, abort_flag, p.err, WAIT_LIMIT_NS))
            fail = true;
          fail = __any_sync(0xffffffffu, fail);
          if (fail) stop_peer();
        }
        uint8_t* sl = slots + b * G_SLOT;
        if (!fail && store) {
          float2* hs = reinterpret_cast<float2*>(sl) + row;
          __nv_bfloat162* ls =
              reinterpret_cast<__nv_bfloat162*>(sl + G_PIECE_HI) + row;
          __nv_bfloat162 l[G_COLS];
#pragma unroll
          for (int c = 0; c < G_COLS; ++c) h[c] = hs[c * BLK];
          if (comp) {
#pragma unroll
            for (int c = 0; c < G_COLS; ++c) l[c] = ls[c * BLK];
          }
          gram_piece<G_COLS, true>(hs, comp ? ls : nullptr, h, l, re, im, comp);
          fence_proxy_async();  // the bulk store reads what was written here
        }
        // all 4 warps of the half have updated the piece (or given up)
        if (named_barrier_or(1 + colh, EPI_THREADS / 2, fail || *abort_flag)) {
          fail = true;
          break;
        }
        if (loader) {
          if (store) {
            const int64_t off = piece_off(t, pc);
            bulk_store(p.g_hi + off, sl, G_PIECE_HI);
            if (comp) bulk_store(p.g_lo + off, sl + G_PIECE_HI, G_PIECE_LO);
            bulk_commit();
          }
          // next piece for this slot: n + 2 (this tile, or the next one's)
          const int m = pc + 2;
          const int tn = m < G_PIECES ? t : t + units;
          if (tn < p.n_tiles) {
            bulk_wait_read();
            issue(tn, m % G_PIECES, b);
            issued[b]++;
          }
        }
        __syncwarp();
        // the power step's share of the piece, after the copies are issued
        if (pw && store)
          power_piece(h, xi, xs + pc * G_COLS, lane, racc,
                      red + q * BLK + pc * 2 * G_COLS);
      }
      if (fail) break;
      if (pw && store) {
        // every warp's column sums are in; the buffers of this parity are
        // next written two tiles on, after this half's barriers of the tile
        // between
        named_barrier(1 + colh, EPI_THREADS / 2);
        const int64_t blk = packed_block(ti, tj, p.nb);
        const float s = ((red[row] + red[BLK + row]) + red[2 * BLK + row]) +
                        red[3 * BLK + row];
        reinterpret_cast<float*>(p.pcol + blk * BLK + colh * 64)[row] = s;
        if (ti != tj) p.prow[(blk * 2 + colh) * BLK + row] = racc;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(&tempty[acc], 0u);
      acc ^= 1;
      if (acc == 0) aph ^= 1;
    }
    // every piece this thread loaded or stored completes before the CTA exits
    if (loader) {
      volatile int no_abort = 0;
      for (int b = 0; b < 2; ++b)
        if (issued[b])
          mbar_wait_bounded(&gf[b], (issued[b] - 1) & 1, &no_abort, p.err,
                            WAIT_LIMIT_NS);
      bulk_wait_all();
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;             // TMEM lane quarter this warp may access
    const int colh = (warp - 2) >> 2;   // which 64-column half of the tile
    const int row = q * 32 + lane;
    const bool comp = p.g_lo != nullptr;
    int acc = 0;
    uint32_t aph = 0;
    for (int t = unit; t < p.n_tiles; t += units) {
      const int4 tile = p.tiles[t];
      const int tj = tile.y & 0xFFFF, slice = tile.y >> 16;
      const int ti = PAIR && rank ? tile.z : tile.x;    // this CTA's A rows
      const bool store = !(PAIR && rank && (tile.w & 1));
      float2 h0[16], h1[16];
      __nv_bfloat162 l0[16], l1[16];
      float2* gh = nullptr;
      __nv_bfloat162* gl = nullptr;
      const float2* src_hi = nullptr;
      const __nv_bfloat162* src_lo = nullptr;
      if (p.mode == 1 && store) {
        const int64_t blk = PAIR ? packed_block(ti, tj, p.nb) : (int64_t)tile.z;
        const int64_t off = blk * (BLK * BLK) + (int64_t)(colh * 64) * BLK + row;
        gh = p.g_hi + off;
        gl = comp ? p.g_lo + off : nullptr;
        src_hi = p.gs_hi + off;
        src_lo = comp ? p.gs_lo + off : nullptr;
        load_piece(src_hi, src_lo, h0, l0, comp);  // prefetch before the MMAs finish
      }
      if (!mbar_wait_bounded(&tfull[acc], aph, abort_flag, p.err,
                             WAIT_LIMIT_NS)) {
        stop_peer();
        break;
      }
      __syncwarp();
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) +
                            (uint32_t)acc * 256u + (uint32_t)colh * 64u;
#pragma unroll
      for (int pc = 0; pc < 4; ++pc) {
        float re[16], im[16];
        tmem_ld16(base + (uint32_t)(pc * 16), re);
        tmem_ld16(base + 128u + (uint32_t)(pc * 16), im);
        if (p.mode == 1 && store && pc < 3) {
          const int64_t nxt = (int64_t)(16 * (pc + 1)) * BLK;
          if (pc & 1)
            load_piece(src_hi + nxt, comp ? src_lo + nxt : nullptr, h0, l0, comp);
          else
            load_piece(src_hi + nxt, comp ? src_lo + nxt : nullptr, h1, l1, comp);
        }
        tmem_wait_ld();
        if (!store) continue;
        if (p.mode == 1) {
          const int64_t cur = (int64_t)(16 * pc) * BLK;
          if (pc & 1)
            gram_piece<16>(gh + cur, comp ? gl + cur : nullptr, h1, l1, re, im, comp);
          else
            gram_piece<16>(gh + cur, comp ? gl + cur : nullptr, h0, l0, re, im, comp);
        } else {
          float4* dst = reinterpret_cast<float4*>(
              p.part + slice * p.part_slice +
              (int64_t)(ti * BLK + row) * p.part_ld + tj * BLK + colh * 64 +
              pc * 16);
#pragma unroll
          for (int c = 0; c < 8; ++c)
            dst[c] = make_float4(re[2 * c], im[2 * c], re[2 * c + 1], im[2 * c + 1]);
        }
      }
      tc_fence_before();
      if (PAIR) {
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(&tempty[acc], 0u);
      } else {
        mbar_arrive(&tempty[acc]);
      }
      acc ^= 1;
      if (acc == 0) aph ^= 1;
    }
  }
  tc_fence_before();
  if (PAIR)
    cluster_sync();  // no CTA leaves while its peer may still touch it
  else
    __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem, TMEM_COLS);
    else
      tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Sum the split-K slices of the dictionary product (round-to-nearest FP32,
// fixed order) and write the six bf16 planes of the forward block.
__global__ void k_dict_reduce(const float2* __restrict__ part, int slices,
                              int64_t slice_stride, int64_t groups,
                              __nv_bfloat16* __restrict__ planes,
                              int64_t plane) {
  // grid-stride: a capped grid leaves SMs to the burst running beside it
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t off = g * 8;
    float re[8], im[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) re[q] = im[q] = 0.f;
    for (int s = 0; s < slices; ++s) {
      const float4* src = reinterpret_cast<const float4*>(part + s * slice_stride + off);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float4 v = __ldcs(src + c);
        re[2 * c] += v.x;
        im[2 * c] += v.y;
        re[2 * c + 1] += v.z;
        im[2 * c + 1] += v.w;
      }
    }
    __align__(16) __nv_bfloat16 v[6][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      split_bf16(re[q], v[0][q], v[3][q]);
      split_bf16(im[q], v[1][q], v[4][q]);
      split_bf16(-re[q], v[2][q], v[5][q]);
    }
#pragma unroll
    for (int pl = 0; pl < 6; ++pl)
      *reinterpret_cast<uint4*>(planes + pl * plane + off) =
          *reinterpret_cast<const uint4*>(v[pl]);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                         cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

bool encode_planes(CUtensorMap* m, void* base, int cols, int rows, int planes,
                   int box_planes, std::string* err) {
  auto fn = encode_fn();
  if (!fn) {
    *err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)cols * 2,
                           (cuuint64_t)cols * (cuuint64_t)rows * 2};
  cuuint32_t box[3] = {(cuuint32_t)KC, (cuuint32_t)BLK, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *err = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
    return false;
  }
  return true;
}

// Launch one persistent tcgen05 grid over p.n_tiles work items (tiles, or
// tile pairs on CTA pairs) with at most grid_cap CTAs (0: one per SM).
// Tiles are dealt round-robin (unit u takes tiles u, u + units, ...).  With
// a capped grid (beside a burst) the unit count is rounded down to a
// multiple of `group` (the dictionary's frequency tiles per atom block):
// every unit then keeps one frequency tile, and the tiles that read the same
// dictionary rows run in the same round on different units at about the
// same time, so that most of those rows come from HBM once.  128 x 128 /
// M = 32768, one-pass DRAM counters of the product alone: 34 pairs read
// 6.5-6.7 GB, 32 pairs 5.4-5.7 GB, for a 4.3 GB dictionary.
template <bool PAIR>
cudaError_t launch_tc_grid(cudaStream_t st, int sm_count, int pair_limit,
                           const CUtensorMap& ma, const CUtensorMap& mb,
                           const TcParams& p, int grid_cap, int group) {
  cudaError_t e = cudaFuncSetAttribute(
      k_tc_cgemm<PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      TcCfg<PAIR>::SMEM);
  if (e != cudaSuccess) return e;
  const int cap = grid_cap > 0 && grid_cap < sm_count ? grid_cap : sm_count;
  if (p.n_tiles <= 0) return cudaSuccess;
  if (!PAIR) {
    int grid = p.n_tiles < cap ? p.n_tiles : cap;
    if (grid_cap > 0 && group > 1 && grid > group) grid -= grid % group;
    k_tc_cgemm<PAIR><<<grid, TC_THREADS, TcCfg<PAIR>::SMEM, st>>>(ma, mb, p);
    return cudaGetLastError();
  }
  int pairs = std::min(p.n_tiles, std::max(1, cap / 2));
  if (pair_limit > 0) pairs = std::min(pairs, pair_limit);
  if (grid_cap > 0 && group > 1 && pairs > group) pairs -= pairs % group;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * pairs));
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = TcCfg<PAIR>::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tc_cgemm<PAIR>, ma, mb, p);
}

// Clusters of two of k_tc_cgemm<true> that fit on the device at once.
int pair_limit(osar_ctx* ctx) {
  if (ctx->tc_pair_limit == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ctx->sm_count & ~1));
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = TcCfg<true>::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaFuncSetAttribute(k_tc_cgemm<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcCfg<true>::SMEM) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&n, k_tc_cgemm<true>, &cfg) == cudaSuccess &&
        n > 0)
      ctx->tc_pair_limit = n;
    else
      ctx->tc_pair_limit = -1;  // unknown: one pair per two SMs
    cudaGetLastError();
  }
  return ctx->tc_pair_limit > 0 ? ctx->tc_pair_limit : 0;
}

cudaError_t launch_tc(osar_ctx* ctx, const CUtensorMap& ma,
                      const CUtensorMap& mb, const TcParams& p, int kind,
                      bool pairs, int grid_cap, int group) {
  ProfEvent ev;
  prof_begin(ctx, kind, &ev);
  const cudaError_t e =
      pairs ? launch_tc_grid<true>(ctx->stream, ctx->sm_count, pair_limit(ctx),
                                   ma, mb, p, grid_cap, group)
            : launch_tc_grid<false>(ctx->stream, ctx->sm_count, 0, ma, mb, p,
                                    grid_cap, group);
  prof_end(ctx, &ev);
  ctx->launches++;
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

bool make_tensor_maps(osar_ctx* ctx, std::string* err) {
  if (!encode_planes(&ctx->map_a_rows1, ctx->Apl, ctx->Kp, ctx->Mp, 6, 1, err))
    return false;
  if (!encode_planes(&ctx->map_a_rows2, ctx->Apl, ctx->Kp, ctx->Mp, 6, 2, err))
    return false;
  if (ctx->Apl_alt &&
      (!encode_planes(&ctx->map_alt_rows1, ctx->Apl_alt, ctx->Kp, ctx->Mp, 6, 1, err) ||
       !encode_planes(&ctx->map_alt_rows2, ctx->Apl_alt, ctx->Kp, ctx->Mp, 6, 2, err)))
    return false;
  if (ctx->dict && !ctx->edgelet) {
    if (!encode_planes(&ctx->map_d_rows1, ctx->Dpl, ctx->Np, ctx->Mp, 4, 1, err))
      return false;
    if (!encode_planes(&ctx->map_f_rows1, ctx->Fpl, ctx->Np, ctx->Kp, 6, 1, err))
      return false;
    if (!encode_planes(&ctx->map_f_rows2, ctx->Fpl, ctx->Np, ctx->Kp, 6, 2, err))
      return false;
  }
  return true;
}

int dict_slices(int np) {
  const int chunks = np / KC;
  int s = 1;
  while (chunks % (2 * s) == 0 && chunks / (2 * s) >= 4096 / KC) s *= 2;
  return s;
}

cudaError_t launch_dict_tc(osar_ctx* ctx, int grid_cap) {
  const bool pairs = (ctx->cfg.tc_pairs & 1) != 0;
  TcParams p = {};
  p.tiles = pairs ? ctx->dict_pairs : ctx->dict_tiles;
  p.n_tiles = pairs ? ctx->n_dict_pairs : ctx->n_dict_tiles;
  p.k_chunks = ctx->Np / KC;
  p.k_slice = p.k_chunks / ctx->dict_slices;
  p.a_lo = 2;
  p.b_lo = 3;
  p.neg_second = 1;
  p.mode = 0;
  p.part = ctx->dict_part;
  p.part_ld = ctx->Kp;
  p.part_slice = (int64_t)ctx->Mp * ctx->Kp;
  p.nb = ctx->nb;
  p.err = &ctx->scal->error;
  cudaError_t e = launch_tc(ctx, ctx->map_d_rows1,
                            pairs ? ctx->map_f_rows1 : ctx->map_f_rows2, p,
                            KCL_DICT, pairs, grid_cap, ctx->Kp / BLK);
  if (e != cudaSuccess) return e;
  const int64_t groups = (int64_t)ctx->Mp * ctx->Kp / 8;
  int64_t rg = (groups + 255) / 256;
  if (grid_cap > 0 && rg > 4 * grid_cap) rg = 4 * grid_cap;  // beside a burst
  ProfEvent ev;
  prof_begin(ctx, KCL_DICT, &ev);
  k_dict_reduce<<<(unsigned)rg, 256, 0, ctx->stream>>>(
      ctx->dict_part, ctx->dict_slices, p.part_slice, groups, ctx->Apl,
      p.part_slice);
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(osar_ctx* ctx, void* dst_hi, __nv_bfloat162* dst_lo,
                           int grid_cap, bool power) {
  const bool pairs = (ctx->cfg.tc_pairs & 2) != 0;
  TcParams p = {};
  p.tiles = pairs ? ctx->gram_pairs : ctx->gram_tiles;
  p.n_tiles = pairs ? ctx->n_gram_pairs : (int)ctx->nblk;
  p.k_chunks = ctx->Kp / KC;
  p.k_slice = p.k_chunks;
  p.a_lo = 3;
  p.b_lo = 3;
  p.neg_second = 0;
  p.mode = 1;
  p.gs_hi = (const float2*)ctx->g_hi;
  p.gs_lo = ctx->g_lo;
  p.g_hi = dst_hi ? (float2*)dst_hi : (float2*)ctx->g_hi;
  p.g_lo = dst_hi ? dst_lo : ctx->g_lo;
  p.nb = ctx->nb;
  p.err = &ctx->scal->error;
  ctx->gp_ready = false;
  if (power && pairs && ctx->gp_col) {
    p.pv = (const float2*)ctx->vt;
    p.pcol = ctx->gp_col;
    p.prow = ctx->gp_row;
    ctx->gp_ready = true;
  }
  return launch_tc(ctx, ctx->map_a_rows1,
                   pairs ? ctx->map_a_rows1 : ctx->map_a_rows2, p, KCL_GRAM,
                   pairs, grid_cap, 1);
}

bool encode_plane_map(CUtensorMap* m, void* base, int cols, int rows,
                      int planes, int box_planes, std::string* err) {
  return encode_planes(m, base, cols, rows, planes, box_planes, err);
}

// Gram update over an explicit tile list (used by the batching form, whose
// tiles span many scenes' stacked operand rows and packed Gram blocks).
cudaError_t launch_gram_tc_tiles(cudaStream_t st, int sm_count,
                                 const CUtensorMap& m1, const CUtensorMap& m2,
                                 const int4* tiles, int n_tiles, float2* g_hi,
                                 __nv_bfloat162* g_lo, int kp, int* err) {
  TcParams p = {};
  p.tiles = tiles;
  p.n_tiles = n_tiles;
  p.k_chunks = kp / KC;
  p.k_slice = p.k_chunks;
  p.a_lo = 3;
  p.b_lo = 3;
  p.neg_second = 0;
  p.mode = 1;
  p.g_hi = g_hi;
  p.g_lo = g_lo;
  p.gs_hi = g_hi;
  p.gs_lo = g_lo;
  p.err = err;
  return launch_tc_grid<false>(st, sm_count, 0, m1, m2, p, 0, 1);
}

}  // namespace osar
