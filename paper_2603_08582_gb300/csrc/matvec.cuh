// The packed-Gram matvec kernel.  Included by several .cu files (through
// finalize.cuh, which adds the consumers of its partial sums); everything
// has internal linkage.
//
// Gram storage: the upper 128 x 128 blocks T_IJ = A[I-rows, J-cols], I <= J,
// each stored column-major: entry (r, c) of the block sits at c * 128 + r.
//
// Matvec: y = A x needs, for every stored block,
//     y_I += T_IJ x_J      and, when I < J,      y_J += T_IJ^H x_I.
// Work items ("segments") are runs of blocks I0..I1-1 of one block column J
// (of one scene, in the batching form).  A CTA's producer thread streams each
// block once from HBM into a shared-memory ring, in 32 KB chunks of stored
// columns; each consumer warp owns WC columns of every chunk (16 of each
// block), each lane 4 rows r of them (mv_row):
//   * y_J[c] = sum_r conj(T[r][c]) x_I[r]: each lane's 4-row sum per block is
//     added to a register accumulator that runs over the whole segment and
//     is reduced across lanes once at the end (segment partial); on a
//     diagonal block (T Hermitian, stored in full) this alone is the block's
//     product;
//   * y_I[r] = sum_c T[r][c] x_J[c] is reduced across the 8 warps through
//     shared memory per off-diagonal block (block partial).
// The consumer (gather_row, finalize.cuh) sums, per output block K, the
// segment partials of column K and the block partials of (K, J), J > K,
// which are contiguous in the packed order.  No floating-point atomics:
// results are deterministic.
#pragma once

#include "batch.h"

namespace osar {
namespace {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using T2 = float2;
};
template <>
struct Vec<double> {
  using T2 = double2;
};

// Rows of a block that consumer lane `lane` handles (q = 0..3).  FP32: rows
// 2 lane, 2 lane + 1, 64 + 2 lane, 64 + 2 lane + 1, so that each 16-byte
// load of a stored column covers 512 contiguous bytes across the warp (four
// shared-memory wavefronts, no bank conflict).  FP64: four consecutive rows
// (the FP64 pass is bound by the FP64 pipe, not by shared memory).
template <typename T>
__device__ __forceinline__ int mv_row(int lane, int q);
template <>
__device__ __forceinline__ int mv_row<float>(int lane, int q) {
  return (q >> 1) * 64 + 2 * lane + (q & 1);
}
template <>
__device__ __forceinline__ int mv_row<double>(int lane, int q) {
  return lane * 4 + q;
}

// The lane's four entries of one stored column, from shared memory.
__device__ __forceinline__ void load4_smem(const float2* col, int lane,
                                           float2 (&g)[4]) {
  const float4 a = reinterpret_cast<const float4*>(col + 2 * lane)[0];
  const float4 b = reinterpret_cast<const float4*>(col + 64 + 2 * lane)[0];
  g[0] = make_float2(a.x, a.y);
  g[1] = make_float2(a.z, a.w);
  g[2] = make_float2(b.x, b.y);
  g[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4_smem(const double2* col, int lane,
                                           double2 (&g)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) g[c] = col[lane * 4 + c];
}

// acc += a * b on both components (FP64: two scalar FMAs).
__device__ __forceinline__ void mac2(double2& acc, double a, double2 b) {
  acc.x = fma(a, b.x, acc.x);
  acc.y = fma(a, b.y, acc.y);
}

// acc += a * b componentwise: one packed FP32x2 FMA (FFMA2), rounding as two
// scalar FMAs.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 acc) {
  return __ffma2_rn(a, b, acc);
}

// Shared-memory pipeline of the matvec.  A stage holds one chunk of CC
// stored columns of a block (32 KB) and, for each of the R right-hand sides,
// the block's x_I (128 entries) and the chunk's x_J entries, all brought in
// by TMA bulk copies issued by one producer thread; CW consumer warps work
// on every chunk, WC columns each.  R = 2 applies the Gram to two vectors
// in one pass (the last power step of a pulse and the first FISTA step).
// The one-vector FP32 pass runs two CTAs per SM (16 consumer warps per SM
// to hide the latency of the packed-FMA chains), each with a 3-stage ring
// and one block-partial buffer; the others run one CTA per SM with a ring of
// up to 6 stages.  The chunking, the warps per CTA and every sum's order
// are the same in all of them.
template <typename T, int R>
struct Mv {
  using T2 = typename Vec<T>::T2;
  static constexpr int CW = 8;                                 // consumer warps
  static constexpr int CC = 32768 / (BLK * (int)sizeof(T2));  // 32 f32 / 16 f64
  static constexpr int CHUNKS = BLK / CC;                      // per block
  static constexpr int WC = CC / CW;                           // columns per warp and chunk
  static constexpr int NACC = CHUNKS * WC;                     // y_J columns per thread
  static constexpr int G_BYTES = CC * BLK * (int)sizeof(T2);
  static constexpr int XI_BYTES = BLK * (int)sizeof(T2);
  static constexpr int XJ_BYTES = CC * (int)sizeof(T2);
  static constexpr int STAGE = G_BYTES + R * (XI_BYTES + XJ_BYTES);
  static constexpr int CTAS = sizeof(T) == 4 && R == 1 ? 2 : 1;  // per SM
  static constexpr int RB = CTAS == 2 ? 1 : 2;  // block-partial buffers
  static constexpr int RED_BYTES = RB * R * CW * BLK * (int)sizeof(T2);
  static constexpr int FIXED = RED_BYTES + 16;
  static constexpr int PER_STAGE = STAGE + 2 * 8 + 16;         // + barriers, meta
  // shared memory of one CTA: 228 KB per SM, 1 KB of it reserved per CTA
  static constexpr int BUDGET = CTAS == 2 ? 228 * 1024 / 2 - 1024 : 227 * 1024;
  static constexpr int NST = (BUDGET - FIXED) / PER_STAGE > 6
                                 ? 6 : (BUDGET - FIXED) / PER_STAGE;  // ring depth
  static constexpr int SMEM = NST * STAGE + RED_BYTES + 2 * NST * 8 +
                              NST * 16 + 16;
  static constexpr int THREADS = 32 * (CW + 1);  // producer warp + consumers
};
static_assert(Mv<float, 1>::NST >= 3 && Mv<float, 2>::NST >= 4 &&
                  Mv<double, 1>::NST >= 4,
              "matvec ring too shallow");
static_assert(Mv<float, 1>::SMEM <= Mv<float, 1>::BUDGET &&
                  Mv<float, 2>::SMEM <= Mv<float, 2>::BUDGET &&
                  Mv<double, 1>::SMEM <= Mv<double, 1>::BUDGET,
              "matvec ring exceeds shared memory");

// The R right-hand sides of one pass and their partial-sum outputs.
template <typename T, int R>
struct MvArgs {
  const typename Vec<T>::T2* x[R];
  typename Vec<T>::T2* segpart[R];
  typename Vec<T>::T2* tilepart[R];
  const int32_t* gate[R];  // gated passes: skipped when every flag is set
  int keep_l2;  // the Gram fits in L2: keep it there between passes
};

// Batching form: a segment's scene gives its Gram's first packed block, its
// block count per side and its first stacked row, and whether it takes part
// in this pass (active scene, stop rule not met, power steps left).
struct MvBatch {
  const int* seg_scene;
  const SceneDesc* desc;
  const DevScalars* sc;
  int gated;
  int pstep;  // power step of the pass, or -1 for a FISTA pass
};

constexpr uint64_t MV_WAIT_LIMIT_NS = 2000000000ull;

// One Gram pass.  Each thread accumulates y_J over NACC of the block's stored
// columns (chunk k, warp w: columns k*CC + w*WC + j) for the whole segment
// and y_I over its 4 rows for one block; the same sums as the definition at
// the top, in a fixed order, so the result does not depend on the grid, on
// which CTA takes which segment, or on R.  Segments are handed out
// dynamically (first by block index, then from an atomic ticket), so the
// kernel spreads over whatever SMs are free, e.g. beside the next pulse's
// dictionary product.  Every wait is bounded; on a timeout the CTA records
// the error, stops at the next per-block barrier and drains its copies.
// gref (nullable): a device slot holding the Gram's address, which then
// replaces G; a context whose Gram alternates between two buffers rewrites
// the slot in stream order at each swap, so that a launch captured in a CUDA
// graph reads the Gram current when it runs.
template <typename T, int R, bool BATCH>
__global__ void __launch_bounds__(Mv<T, R>::THREADS, Mv<T, R>::CTAS)
    k_matvec(const typename Vec<T>::T2* __restrict__ G, const MvArgs<T, R> a,
             const int4* __restrict__ segs, int nseg, int nb,
             DevScalars* __restrict__ sc, int gated,
             unsigned* __restrict__ queue, const MvBatch mb,
             const void* const* __restrict__ gref) {
  using C = Mv<T, R>;
  using T2 = typename Vec<T>::T2;
  if (!BATCH && gated) {
    bool all = true;
#pragma unroll
    for (int r = 0; r < R; ++r) all = all && *a.gate[r] != 0;
    if (all) return;  // every vector's solution has met the stop rule
  }
  extern __shared__ __align__(128) uint8_t mv_smem[];
  T2* red = reinterpret_cast<T2*>(mv_smem + C::NST * C::STAGE);  // [RB][R][CW][BLK]
  uint64_t* full = reinterpret_cast<uint64_t*>(mv_smem + C::NST * C::STAGE +
                                               C::RED_BYTES);
  uint64_t* empty = full + C::NST;
  // per stage: (packed block of the Gram, diagonal?, segment slot, flags)
  int4* meta = reinterpret_cast<int4*>(empty + C::NST);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(meta + C::NST);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < C::NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], C::CW);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == 0) {
    if (lane != 0) return;
    // ------------------------------------------------------------ producer
    // a Gram larger than L2 streams through it once per pass; a small one
    // stays resident for the next pass
    const uint64_t stream_policy =
        a.keep_l2 ? l2_policy_evict_last() : l2_policy_evict_first();
    if (gref) G = reinterpret_cast<const T2*>(*gref);
    uint32_t issued[C::NST];
    for (int i = 0; i < C::NST; ++i) issued[i] = 0;
    int stage = 0;
    uint32_t ph = 0;
    bool ok = true;
    int s = blockIdx.x;
    int s_next = nseg;
    if (s < nseg) s_next = (int)gridDim.x + (int)atomicAdd(&queue[0], 1u);
    while (ok && s < nseg) {
      const int4 sg = segs[s];
      int64_t gbase = 0, xrow = 0;
      int nbs = nb;
      bool take = true;
      if (BATCH) {
        const int scene = mb.seg_scene[s];
        const SceneDesc& d = mb.desc[scene];
        take = d.active && !(mb.gated && mb.sc[scene].converged) &&
               !(mb.pstep >= 0 && mb.pstep >= d.psteps);
        gbase = d.gblk;
        nbs = d.nb;
        xrow = d.row;
      }
      for (int I = sg.y; take && ok && I < sg.z; ++I) {
        const int64_t pb = gbase + packed_block(I, sg.x, nbs);
        const T2* blk = G + pb * (int64_t)(BLK * BLK);
        for (int k = 0; k < C::CHUNKS; ++k) {
          if (!mbar_wait_bounded(&empty[stage], ph ^ 1, abort_flag, &sc->error,
                                 MV_WAIT_LIMIT_NS)) {
            ok = false;
            break;
          }
          if (k == 0)
            meta[stage] = make_int4((int)pb, I == sg.x ? 1 : 0, sg.w,
                                    (I == sg.y ? 1 : 0) | (I == sg.z - 1 ? 2 : 0));
          uint8_t* st = mv_smem + stage * C::STAGE;
          mbar_expect_tx(&full[stage], C::STAGE);
          bulk_load_hint(st, blk + (int64_t)k * C::CC * BLK, C::G_BYTES,
                         &full[stage], stream_policy);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            bulk_load(st + C::G_BYTES + r * C::XI_BYTES,
                      a.x[r] + xrow + (int64_t)I * BLK, C::XI_BYTES, &full[stage]);
            bulk_load(st + C::G_BYTES + R * C::XI_BYTES + r * C::XJ_BYTES,
                      a.x[r] + xrow + (int64_t)sg.x * BLK + k * C::CC, C::XJ_BYTES,
                      &full[stage]);
          }
          issued[stage]++;
          if (++stage == C::NST) {
            stage = 0;
            ph ^= 1;
          }
        }
      }
      s = s_next;
      if (s < nseg) s_next = (int)gridDim.x + (int)atomicAdd(&queue[0], 1u);
    }
    // end of work: a stage whose meta says so (no copy); its earlier copies
    // have landed, since the consumers released it
    int sentinel = -1;
    if (ok && mbar_wait_bounded(&empty[stage], ph ^ 1, abort_flag, &sc->error,
                                MV_WAIT_LIMIT_NS)) {
      meta[stage] = make_int4(-1, 0, 0, 0);
      mbar_arrive(&full[stage]);
      sentinel = stage;
    }
    // the last CTA to leave resets the ticket counter for the next launch
    __threadfence();
    if (atomicAdd(&queue[1], 1u) == gridDim.x - 1) {
      queue[0] = 0;
      queue[1] = 0;
      __threadfence();
    }
    // every copy this thread issued lands before the CTA exits
    volatile int no_abort = 0;
    for (int i = 0; i < C::NST; ++i)
      if (issued[i] && i != sentinel)
        mbar_wait_bounded(&full[i], (issued[i] - 1) & 1, &no_abort, &sc->error,
                          MV_WAIT_LIMIT_NS);
    return;
  }

  // -------------------------------------------------------------- consumers
  const int cw = warp - 1;
  int stage = 0, rp = 0;
  uint32_t ph = 0;
  T2 yj[R][C::NACC];  // y_J partials (re, im) of this thread's columns
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < C::NACC; ++c) yj[r][c].x = yj[r][c].y = T(0);
  for (;;) {
    bool ok = !*abort_flag && mbar_wait_bounded(&full[stage], ph, abort_flag,
                                                &sc->error, MV_WAIT_LIMIT_NS);
    const int4 m = ok ? meta[stage] : make_int4(-1, 0, 0, 0);
    const bool work = ok && m.x >= 0;
    if (work) {
      const bool diag = m.y != 0;
      if (m.w & 1) {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int c = 0; c < C::NACC; ++c) yj[r][c].x = yj[r][c].y = T(0);
      }
      // x_I of this lane's 4 rows as (re, im) and (im, -re)
      T2 xa[R][4], xb[R][4];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const T2* xis = reinterpret_cast<const T2*>(
            mv_smem + stage * C::STAGE + C::G_BYTES + r * C::XI_BYTES);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xa[r][q] = xis[mv_row<T>(lane, q)];
          xb[r][q].x = xa[r][q].y;
          xb[r][q].y = -xa[r][q].x;
        }
      }
      // y_I partials of this lane's 4 rows.  FP32 keeps two packed sums per
      // row, u = sum e (x.re, -x.im) and v = sum e (x.im, x.re) over the
      // entries e = (re, im) of the row and x = x_J[c], so that every entry
      // enters an FFMA2 as loaded: y_I = (u.x + u.y, v.x + v.y).  FP64 keeps
      // (re, im) in yu.
      T2 yu[R][4], yv[R][4];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) yu[r][q].x = yu[r][q].y = yv[r][q].x = yv[r][q].y = T(0);
#pragma unroll
      for (int k = 0; k < C::CHUNKS; ++k) {
        if (k > 0 && ok)
          ok = !*abort_flag && mbar_wait_bounded(&full[stage], ph, abort_flag,
                                                 &sc->error, MV_WAIT_LIMIT_NS);
        if (ok) {
          const uint8_t* st = mv_smem + stage * C::STAGE;
          const T2* gs = reinterpret_cast<const T2*>(st);
#pragma unroll
          for (int j = 0; j < C::WC; ++j) {
            const int col = cw * C::WC + j;
            T2 g[4];
            load4_smem(gs + col * BLK, lane, g);
            const int aa = k * C::WC + j;
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const T2 ja = reinterpret_cast<const T2*>(
                  st + C::G_BYTES + R * C::XI_BYTES + r * C::XJ_BYTES)[col];
              if constexpr (sizeof(T) == 4) {
                // y_J[c] += sum_r conj(e) x_I[r]: p = sum e (x.re, x.im),
                // q = sum e (x.im, -x.re), folded once per column
                const float2 cj = make_float2(ja.x, -ja.y);
                const float2 sj = make_float2(ja.y, ja.x);
                float2 p = make_float2(0.f, 0.f), qs = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const float2 e = g[q];
                  p = fma2(e, xa[r][q], p);
                  qs = fma2(e, xb[r][q], qs);
                  yu[r][q] = fma2(e, cj, yu[r][q]);
                  yv[r][q] = fma2(e, sj, yv[r][q]);
                }
                yj[r][aa].x += p.x + p.y;
                yj[r][aa].y += qs.x + qs.y;
              } else {
                T2 jb;  // (-im, re) of x_J[c]
                jb.x = -ja.y;
                jb.y = ja.x;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const T2 e = g[q];
                  // y_J[c] += conj(e) x_I[r] = e.re (x.re, x.im) + e.im (x.im, -x.re)
                  mac2(yj[r][aa], e.x, xa[r][q]);
                  mac2(yj[r][aa], e.y, xb[r][q]);
                  // y_I[r] += e x_J[c] = e.re (x.re, x.im) + e.im (-x.im, x.re)
                  mac2(yu[r][q], e.x, ja);
                  mac2(yu[r][q], e.y, jb);
                }
              }
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[stage]);
        }
        if (++stage == C::NST) {
          stage = 0;
          ph ^= 1;
        }
      }
      if (ok && !diag) {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            T2 v = yu[r][q];
            if constexpr (sizeof(T) == 4) {
              v.x = yu[r][q].x + yu[r][q].y;
              v.y = yv[r][q].x + yv[r][q].y;
            }
            red[((rp * R + r) * C::CW + cw) * BLK + mv_row<T>(lane, q)] = v;
          }
      }
      if (ok && (m.w & 2)) {
        // segment done: y_J over all rows of its blocks, one lane per column
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int aa = 0; aa < C::NACC; ++aa) {
            T vr = yj[r][aa].x, vi = yj[r][aa].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              vr += __shfl_xor_sync(0xffffffffu, vr, o);
              vi += __shfl_xor_sync(0xffffffffu, vi, o);
            }
            if (lane == aa) {
              T2 v;
              v.x = vr;
              v.y = vi;
              const int col = (aa / C::WC) * C::CC + cw * C::WC + (aa % C::WC);
              a.segpart[r][(int64_t)m.z * BLK + col] = v;
            }
          }
      }
    }
    // Per-block barrier of the consumer warps: the block partial is summed
    // over the warps in a fixed order, and the loop ends here for everyone
    // at once (end of work, or an abort any warp saw before the barrier: the
    // decision is the barrier's OR over all consumer threads).
    if (named_barrier_or(1, 32 * C::CW, !work || *abort_flag)) break;
    const int rr = (int)threadIdx.x - 32;
    if (!m.y && rr < R * BLK) {
      const int r = rr / BLK, row = rr % BLK;
      T sr = 0, si = 0;
#pragma unroll
      for (int w = 0; w < C::CW; ++w) {
        sr += red[((rp * R + r) * C::CW + w) * BLK + row].x;
        si += red[((rp * R + r) * C::CW + w) * BLK + row].y;
      }
      T2 v;
      v.x = sr;
      v.y = si;
      a.tilepart[r][(int64_t)m.x * BLK + row] = v;
    }
    if (C::RB == 2)
      rp ^= 1;
    else
      named_barrier(1, 32 * C::CW);  // one buffer: read before the next block's writes
  }
}

}  // namespace
}  // namespace osar
