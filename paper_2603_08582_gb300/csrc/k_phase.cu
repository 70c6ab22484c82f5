// Phase synthesis (Eqs. 2-4), dictionary construction (Sec. III-A) and the
// forward simulator of Eq. 5.
//
// The phase of F[m, p] = exp(-i 2 k_m R_p), k_m = 2 pi f_m / c, reaches
// ~5e5 rad, so it is never formed in floating point.  Per pixel the kernel
// computes R_p = |gamma - x_p| in FP64 and the two turn counts
//     a_p = 2 f_lo R_p / c,     e_p = 2 df R_p / c,    df = (f_hi - f_lo)/(K-1)
// keeps only their fractional parts as 64-bit fixed-point numbers A_p, E_p
// (units of 2^-64 turn), and then forms every entry's phase exactly modulo one
// turn with integer arithmetic:  turn(m, p) = A_p + m E_p  (mod 2^64).
// The only rounding is in a_p and e_p (~1e-11 turn); the sin/cos that follows
// runs in FP32 (split-BF16 and FP32 paths) or FP64 (plain path).
#include "ctx.h"

namespace osar {

namespace {

constexpr double TWO64 = 18446744073709551616.0;

__device__ __forceinline__ uint64_t frac_to_q64(double t) {
  // t in [0, 1): t * 2^63 is exactly representable below 2^63.
  double s = ldexp(t, 63);
  uint64_t u = __double2ull_rz(s);
  return u << 1;
}

__global__ void k_pixel_turns(int nx, int N, int Np, double pixel_m,
                              double cx_half, double cy_half, double gx,
                              double gy, double gz, double two_flo_over_c,
                              double two_df_over_c, ulonglong2* out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Np) return;
  if (p >= N) {
    out[p] = make_ulonglong2(0ull, 0ull);
    return;
  }
  int i = p / nx, j = p - (p / nx) * nx;
  double x = ((double)j - cx_half) * pixel_m;
  double y = ((double)i - cy_half) * pixel_m;
  double dx = gx - x, dy = gy - y, dz = gz;
  double r = sqrt(dx * dx + dy * dy + dz * dz);  // Eq. 3, FP64
  double a = two_flo_over_c * r;
  double e = two_df_over_c * r;
  a -= floor(a);
  e -= floor(e);
  out[p] = make_ulonglong2(frac_to_q64(a), frac_to_q64(e));
}

// exp(-2 pi i turn) for a 64-bit turn fraction.
__device__ __forceinline__ double2 unit_phase_f64(uint64_t turn) {
  double x = (double)(long long)turn * (1.0 / TWO64);  // [-1/2, 1/2)
  double s, c;
  sincospi(2.0 * x, &s, &c);
  return make_double2(c, -s);
}
__device__ __forceinline__ float2 unit_phase_f32(uint64_t turn) {
  float x = (float)(int)(turn >> 32) * 2.3283064365386963e-10f;  // 2^-32
  float s, c;
  sincospif(2.0f * x, &s, &c);
  return make_float2(c, -s);
}

template <typename T2>
__device__ __forceinline__ T2 phase_entry(uint64_t turn);
template <>
__device__ __forceinline__ double2 phase_entry<double2>(uint64_t turn) {
  return unit_phase_f64(turn);
}
template <>
__device__ __forceinline__ float2 phase_entry<float2>(uint64_t turn) {
  return unit_phase_f32(turn);
}

// Complex output.  PIXEL_MAJOR: out[p][m] (ld = Kp, rows Mp), used when the
// dictionary is the identity so that the block is written in the K-contiguous
// layout the Gram update reads.  Otherwise out[m][p] (ld = Np, rows Kp).
// Each thread writes 8 consecutive entries along the contiguous axis.
// wk (nullable): per-frequency weights 1 / sigma_k of a non-white pulse, the
// rows of R_n^{-1/2} F (Eq. 12 with R_n = diag(sigma_k^2)).
template <typename T2, bool PIXEL_MAJOR>
__global__ void k_phase_complex(const ulonglong2* __restrict__ turns, int N,
                                int K, int rows, int ld, T2* __restrict__ out,
                                const double* __restrict__ wk) {
  const int groups = ld / 8;
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)rows * groups) return;
  int row = (int)(gid / groups);
  int col0 = (int)(gid - (int64_t)row * groups) * 8;
  T2* dst = out + (int64_t)row * ld + col0;
  if (PIXEL_MAJOR) {
    const int p = row;
    ulonglong2 tp = p < N ? turns[p] : make_ulonglong2(0, 0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int m = col0 + q;
      T2 v;
      if (p < N && m < K) {
        v = phase_entry<T2>(tp.x + (uint64_t)m * tp.y);
        if (wk) {
          v.x *= wk[m];
          v.y *= wk[m];
        }
      } else {
        v.x = 0; v.y = 0;
      }
      dst[q] = v;
    }
  } else {
    const int m = row;
    const double w = wk && m < K ? wk[m] : 1.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int p = col0 + q;
      T2 v;
      if (p < N && m < K) {
        ulonglong2 tp = turns[p];
        v = phase_entry<T2>(tp.x + (uint64_t)m * tp.y);
        if (wk) {
          v.x *= w;
          v.y *= w;
        }
      } else {
        v.x = 0; v.y = 0;
      }
      dst[q] = v;
    }
  }
}

// Split-BF16 output: six planes (re, im, -re) x (hi, lo), each rows x ld.
template <bool PIXEL_MAJOR>
__global__ void k_phase_planes(const ulonglong2* __restrict__ turns, int N,
                               int K, int rows, int ld,
                               __nv_bfloat16* __restrict__ planes,
                               const double* __restrict__ wk) {
  const int groups = ld / 8;
  const int64_t plane = (int64_t)rows * ld;
  // grid-stride: a capped grid leaves SMs to the burst running beside it
  for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
       gid < (int64_t)rows * groups; gid += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)(gid / groups);
    int col0 = (int)(gid - (int64_t)row * groups) * 8;
    __align__(16) __nv_bfloat16 v[6][8];
    ulonglong2 tp_row = make_ulonglong2(0, 0);
    if (PIXEL_MAJOR && row < N) tp_row = turns[row];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int p = PIXEL_MAJOR ? row : col0 + q;
      int m = PIXEL_MAJOR ? col0 + q : row;
      float2 e = make_float2(0.f, 0.f);
      if (p < N && m < K) {
        ulonglong2 tp = PIXEL_MAJOR ? tp_row : turns[p];
        e = unit_phase_f32(tp.x + (uint64_t)m * tp.y);
        if (wk) {
          const float w = (float)wk[m];
          e.x *= w;
          e.y *= w;
        }
      }
      split_bf16(e.x, v[0][q], v[3][q]);
      split_bf16(e.y, v[1][q], v[4][q]);
      split_bf16(-e.x, v[2][q], v[5][q]);
    }
    const int64_t off = (int64_t)row * ld + col0;
#pragma unroll
    for (int pl = 0; pl < 6; ++pl)
      *reinterpret_cast<uint4*>(planes + pl * plane + off) =
          *reinterpret_cast<const uint4*>(v[pl]);
  }
}

// ---------------------------------------------------------------- dictionary
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x), lo0 = 0xD2511F53u * ctr.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z), lo1 = 0xCD9E8D57u * ctr.z;
    ctr = make_uint4(hi1 ^ ctr.y ^ k0, lo1, hi0 ^ ctr.w ^ k1, lo0);
  }
  return ctr;
}

// Unnormalised Gaussian atom entry (pixel p, atom j) by Box-Muller.
__device__ __forceinline__ double2 gauss_entry(int p, int j, uint64_t seed) {
  uint4 r = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)j, 0x5A5D1C7u, 0u),
                          (uint32_t)(seed & 0xFFFFFFFFull),
                          (uint32_t)(seed >> 32));
  uint64_t w1 = ((uint64_t)r.y << 32) | r.x;
  uint64_t w2 = ((uint64_t)r.w << 32) | r.z;
  double u1 = ((double)(w1 >> 11) + 0.5) * 1.1102230246251565e-16;  // 2^-53
  double u2 = ((double)(w2 >> 11) + 0.5) * 1.1102230246251565e-16;
  double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return make_double2(rad * c, rad * s);
}

// Column 2-norms (FP64) of the Gaussian dictionary: one block per atom.
__global__ void k_gauss_norms(int N, int M, uint64_t seed, double* inv_norm) {
  int j = blockIdx.x;
  if (j >= M) return;
  double acc = 0.0;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    double2 zv = gauss_entry(p, j, seed);
    acc += zv.x * zv.x + zv.y * zv.y;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) inv_norm[j] = 1.0 / sqrt(acc);
  }
}

// Host-provided dictionary column norms are not recomputed: inv_norm = 1.
// Source of entry (p, j): the Gaussian generator or a staged host copy
// (atom-major, N entries per atom).
__device__ __forceinline__ double2 dict_entry(int p, int j, int N, int M,
                                              uint64_t seed,
                                              const double2* host_copy,
                                              const double* inv_norm) {
  if (p >= N || j >= M) return make_double2(0.0, 0.0);
  if (host_copy) return host_copy[(int64_t)j * N + p];
  double2 zv = gauss_entry(p, j, seed);
  double s = inv_norm[j];
  return make_double2(zv.x * s, zv.y * s);
}

template <typename T2>
__global__ void k_dict_complex(int N, int M, int Mp, int Np, uint64_t seed,
                               const double2* host_copy, const double* inv_norm,
                               T2* __restrict__ out) {
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)Mp * Np) return;
  int j = (int)(gid / Np);
  int p = (int)(gid - (int64_t)j * Np);
  double2 e = dict_entry(p, j, N, M, seed, host_copy, inv_norm);
  T2 v;
  v.x = e.x;
  v.y = e.y;
  out[gid] = v;
}

// Dictionary planes for the split-BF16 path: (re, im) x (hi, lo), atom-major.
__global__ void k_dict_planes(int N, int M, int Mp, int Np, uint64_t seed,
                              const double2* host_copy, const double* inv_norm,
                              __nv_bfloat16* __restrict__ planes) {
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)Mp * Np) return;
  int j = (int)(gid / Np);
  int p = (int)(gid - (int64_t)j * Np);
  double2 e = dict_entry(p, j, N, M, seed, host_copy, inv_norm);
  const int64_t plane = (int64_t)Mp * Np;
  // hi from the FP64 value, lo from the FP64 remainder
  __nv_bfloat16 rh = __double2bfloat16(e.x);
  __nv_bfloat16 ih = __double2bfloat16(e.y);
  __nv_bfloat16 rl = __double2bfloat16(e.x - (double)__bfloat162float(rh));
  __nv_bfloat16 il = __double2bfloat16(e.y - (double)__bfloat162float(ih));
  planes[gid] = rh;
  planes[plane + gid] = ih;
  planes[2 * plane + gid] = rl;
  planes[3 * plane + gid] = il;
}

// ------------------------------------------------------------- simulation ---
// rho_p = sum over nonzero j of H[p, j] c_j (FP64 arithmetic).
template <typename T2>
__global__ void k_sim_rho_complex(const T2* __restrict__ D, int Np, int nnz,
                                  const int* __restrict__ idx,
                                  const double2* __restrict__ val, double2* rho) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Np) return;
  double2 acc = make_double2(0, 0);
  for (int q = 0; q < nnz; ++q) {
    T2 e = D[(int64_t)idx[q] * Np + p];
    acc.x += (double)e.x * val[q].x - (double)e.y * val[q].y;
    acc.y += (double)e.x * val[q].y + (double)e.y * val[q].x;
  }
  rho[p] = acc;
}

__global__ void k_sim_rho_planes(const __nv_bfloat16* __restrict__ Dp, int Mp,
                                 int Np, int nnz, const int* __restrict__ idx,
                                 const double2* __restrict__ val, double2* rho) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Np) return;
  const int64_t plane = (int64_t)Mp * Np;
  double2 acc = make_double2(0, 0);
  for (int q = 0; q < nnz; ++q) {
    int64_t o = (int64_t)idx[q] * Np + p;
    double er = (double)__bfloat162float(Dp[o]) +
                (double)__bfloat162float(Dp[2 * plane + o]);
    double ei = (double)__bfloat162float(Dp[plane + o]) +
                (double)__bfloat162float(Dp[3 * plane + o]);
    acc.x += er * val[q].x - ei * val[q].y;
    acc.y += er * val[q].y + ei * val[q].x;
  }
  rho[p] = acc;
}

__global__ void k_sim_scatter(int nnz, const int* idx, const double2* val,
                              double2* rho) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nnz) rho[idx[q]] = val[q];
}

// d_m = sum_p F[m, p] rho_p, one block per frequency, FP64.
__global__ void k_sim_data(const ulonglong2* __restrict__ turns, int N,
                           const double2* __restrict__ rho, double2* d) {
  const int m = blockIdx.x;
  double2 acc = make_double2(0, 0);
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    ulonglong2 tp = turns[p];
    double2 e = unit_phase_f64(tp.x + (uint64_t)m * tp.y);
    double2 r = rho[p];
    acc.x += e.x * r.x - e.y * r.y;
    acc.y += e.x * r.y + e.y * r.x;
  }
  __shared__ double2 red[32];
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : make_double2(0, 0);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (threadIdx.x == 0) d[m] = acc;
  }
}

inline unsigned blocks_for(int64_t n, int t) {
  return (unsigned)((n + t - 1) / t);
}

}  // namespace

cudaError_t launch_pixel_turns(osar_ctx* ctx, const double gamma[3]) {
  const osar_config& c = ctx->cfg;
  double df = ctx->K > 1 ? (c.f_hi_hz - c.f_lo_hz) / (double)(ctx->K - 1) : 0.0;
  ProfEvent ev;
  prof_begin(ctx, KCL_PHASE, &ev);
  k_pixel_turns<<<blocks_for(ctx->Np, 256), 256, 0, ctx->stream>>>(
      c.nx, ctx->N, ctx->Np, c.pixel_m, 0.5 * (c.nx - 1), 0.5 * (c.ny - 1),
      gamma[0], gamma[1], gamma[2], 2.0 * c.f_lo_hz / C_LIGHT,
      2.0 * df / C_LIGHT, ctx->turns);
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_phase(osar_ctx* ctx, int grid_cap) {
  ProfEvent ev;
  prof_begin(ctx, KCL_PHASE, &ev);
  // pixel-major rows (p, k) for the pixel basis (they are the block itself)
  // and for edgelets (whose atoms sum pixel rows); frequency-major for the
  // dictionary GEMM
  const bool pix = !ctx->dict || ctx->edgelet;
  const int rows = !ctx->dict ? ctx->Mp : ctx->edgelet ? ctx->Np : ctx->Kp;
  const int ld = pix ? ctx->Kp : ctx->Np;
  const int64_t work = (int64_t)rows * (ld / 8);
  unsigned g = blocks_for(work, 256);
  // beside a burst: at most 4 CTAs per SM the side work was given (the
  // split-BF16 kernel strides over its rows)
  if (grid_cap > 0 && ctx->prec == OSAR_SPLIT_BF16 && g > (unsigned)(4 * grid_cap))
    g = (unsigned)(4 * grid_cap);
  if (ctx->edgelet) {
    // FP32 phases for the split and FP32 paths, FP64 on the plain path
    const unsigned gc = blocks_for(work, 256);  // one thread per 8 entries
    if (ctx->prec == OSAR_FP64)
      k_phase_complex<double2, true><<<gc, 256, 0, ctx->stream>>>(
          ctx->turns, ctx->N, ctx->K, rows, ld, (double2*)ctx->F, ctx->synth_w);
    else
      k_phase_complex<float2, true><<<gc, 256, 0, ctx->stream>>>(
          ctx->turns, ctx->N, ctx->K, rows, ld, (float2*)ctx->F, ctx->synth_w);
  } else if (ctx->prec == OSAR_SPLIT_BF16) {
    __nv_bfloat16* out = pix ? ctx->Apl : ctx->Fpl;
    if (pix)
      k_phase_planes<true><<<g, 256, 0, ctx->stream>>>(ctx->turns, ctx->N,
                                                       ctx->K, rows, ld, out,
                                                       ctx->synth_w);
    else
      k_phase_planes<false><<<g, 256, 0, ctx->stream>>>(ctx->turns, ctx->N,
                                                        ctx->K, rows, ld, out,
                                                        ctx->synth_w);
  } else if (ctx->prec == OSAR_FP64) {
    double2* out = (double2*)(pix ? ctx->A : ctx->F);
    if (pix)
      k_phase_complex<double2, true><<<g, 256, 0, ctx->stream>>>(
          ctx->turns, ctx->N, ctx->K, rows, ld, out, ctx->synth_w);
    else
      k_phase_complex<double2, false><<<g, 256, 0, ctx->stream>>>(
          ctx->turns, ctx->N, ctx->K, rows, ld, out, ctx->synth_w);
  } else {
    float2* out = (float2*)(pix ? ctx->A : ctx->F);
    if (pix)
      k_phase_complex<float2, true><<<g, 256, 0, ctx->stream>>>(
          ctx->turns, ctx->N, ctx->K, rows, ld, out, ctx->synth_w);
    else
      k_phase_complex<float2, false><<<g, 256, 0, ctx->stream>>>(
          ctx->turns, ctx->N, ctx->K, rows, ld, out, ctx->synth_w);
  }
  prof_end(ctx, &ev);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t launch_dictionary_build(osar_ctx* ctx, const double* host_dict) {
  // the atoms: the context's own, or the coefficient side of a pixel-space
  // Gram form with a dense dictionary
  const int N = ctx->N, Np = ctx->Np;
  const int M = ctx->pg ? ctx->pg->M : ctx->M;
  const int Mp = ctx->pg ? ctx->pg->Mp : ctx->Mp;
  cudaError_t e;
  double* inv_norm = nullptr;
  double2* host_copy = nullptr;
  e = cudaMallocAsync(&inv_norm, sizeof(double) * Mp, ctx->stream);
  if (e != cudaSuccess) return e;
  if (host_dict) {
    size_t bytes = sizeof(double2) * (size_t)N * M;
    e = cudaMallocAsync(&host_copy, bytes, ctx->stream);
    if (e != cudaSuccess) {
      cudaFreeAsync(inv_norm, ctx->stream);
      return e;
    }
    e = cudaMemcpyAsync(host_copy, host_dict, bytes, cudaMemcpyHostToDevice,
                        ctx->stream);
    if (e != cudaSuccess) return e;
  } else {
    k_gauss_norms<<<M, 256, 0, ctx->stream>>>(N, M, ctx->cfg.dict_seed,
                                              inv_norm);
    ctx->launches++;
  }
  const unsigned g = blocks_for((int64_t)Mp * Np, 256);
  if (ctx->prec == OSAR_SPLIT_BF16) {
    k_dict_planes<<<g, 256, 0, ctx->stream>>>(N, M, Mp, Np, ctx->cfg.dict_seed,
                                              host_copy, inv_norm, ctx->Dpl);
  } else if (ctx->prec == OSAR_FP64) {
    k_dict_complex<double2><<<g, 256, 0, ctx->stream>>>(
        N, M, Mp, Np, ctx->cfg.dict_seed, host_copy, inv_norm,
        (double2*)ctx->D);
  } else {
    k_dict_complex<float2><<<g, 256, 0, ctx->stream>>>(
        N, M, Mp, Np, ctx->cfg.dict_seed, host_copy, inv_norm, (float2*)ctx->D);
  }
  ctx->launches++;
  e = cudaGetLastError();
  cudaFreeAsync(inv_norm, ctx->stream);
  if (host_copy) cudaFreeAsync(host_copy, ctx->stream);
  return e;
}

cudaError_t launch_simulate(osar_ctx* ctx, int nnz, double2* d_out) {
  const int Np = ctx->Np;
  const int Mpd = ctx->pg ? ctx->pg->Mp : ctx->Mp;  // atoms of the dictionary rows
  if (ctx->edgelet || (ctx->pg && !ctx->pg->dense)) {
    // the image H c (the pixel-space Gram form keeps H's lists too)
    cudaError_t e = launch_sim_rho_edgelet(ctx, nnz);
    if (e != cudaSuccess) return e;
  } else if (!ctx->dict && !ctx->pg) {
    cudaMemsetAsync(ctx->sim_rho, 0, sizeof(double2) * Np, ctx->stream);
    if (nnz > 0)
      k_sim_scatter<<<blocks_for(nnz, 256), 256, 0, ctx->stream>>>(
          nnz, ctx->sim_idx, ctx->sim_nz, ctx->sim_rho);
  } else if (ctx->prec == OSAR_SPLIT_BF16) {
    k_sim_rho_planes<<<blocks_for(Np, 256), 256, 0, ctx->stream>>>(
        ctx->Dpl, Mpd, Np, nnz, ctx->sim_idx, ctx->sim_nz, ctx->sim_rho);
  } else if (ctx->prec == OSAR_FP64) {
    k_sim_rho_complex<double2><<<blocks_for(Np, 256), 256, 0, ctx->stream>>>(
        (const double2*)ctx->D, Np, nnz, ctx->sim_idx, ctx->sim_nz,
        ctx->sim_rho);
  } else {
    k_sim_rho_complex<float2><<<blocks_for(Np, 256), 256, 0, ctx->stream>>>(
        (const float2*)ctx->D, Np, nnz, ctx->sim_idx, ctx->sim_nz,
        ctx->sim_rho);
  }
  k_sim_data<<<ctx->K, 256, 0, ctx->stream>>>(ctx->turns, ctx->N, ctx->sim_rho,
                                              d_out);
  ctx->launches += 2;
  return cudaGetLastError();
}

}  // namespace osar
