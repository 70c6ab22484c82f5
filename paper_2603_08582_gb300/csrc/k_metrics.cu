// Reconstruction-quality figures of the current estimate c_hat_n (Sec. IV-B):
// the count of "large" coefficients (|c_m| above a threshold; the
// experiments use 2e-2) and the SNR of Eq. 18, read in the coefficient
// domain: 20 log10 of the RMS of |c_m| over a reference support (the
// scene's true atoms) over the RMS of |c_m| off it.  One CTA reduces the
// whole vector in a fixed order, so the figures are deterministic.
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "ctx.h"

namespace osar {
namespace {

constexpr int MT_THREADS = 1024;

struct MetricSums {
  double l1, max_abs, s_on, s_off;
  int32_t n_large, n_nonzero, n_on, large_off;
};

__global__ void __launch_bounds__(MT_THREADS)
    k_metrics(const double2* __restrict__ c, const uint8_t* __restrict__ mask,
              int m, double threshold, MetricSums* __restrict__ out) {
  double l1 = 0.0, mx = 0.0, son = 0.0, soff = 0.0;
  int nl = 0, nz = 0, non = 0, loff = 0;
  for (int i = threadIdx.x; i < m; i += MT_THREADS) {
    const double2 v = c[i];
    const double a = hypot(v.x, v.y);
    const bool on = mask && mask[i];
    l1 += a;
    mx = fmax(mx, a);
    nz += a > 0.0;
    const bool large = a > threshold;
    nl += large;
    if (on) {
      son += a * a;
      ++non;
    } else {
      soff += a * a;
      loff += large;
    }
  }
  __shared__ double sd[4][MT_THREADS / 32];
  __shared__ int si[4][MT_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    son += __shfl_xor_sync(0xffffffffu, son, o);
    soff += __shfl_xor_sync(0xffffffffu, soff, o);
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
    non += __shfl_xor_sync(0xffffffffu, non, o);
    loff += __shfl_xor_sync(0xffffffffu, loff, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sd[0][w] = l1;
    sd[1][w] = mx;
    sd[2][w] = son;
    sd[3][w] = soff;
    si[0][w] = nl;
    si[1][w] = nz;
    si[2][w] = non;
    si[3][w] = loff;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    MetricSums r{0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0};
    for (int k = 0; k < MT_THREADS / 32; ++k) {
      r.l1 += sd[0][k];
      r.max_abs = fmax(r.max_abs, sd[1][k]);
      r.s_on += sd[2][k];
      r.s_off += sd[3][k];
      r.n_large += si[0][k];
      r.n_nonzero += si[1][k];
      r.n_on += si[2][k];
      r.large_off += si[3][k];
    }
    *out = r;
  }
}

}  // namespace
}  // namespace osar

extern "C" osar_status osar_get_metrics(osar_ctx* ctx, double threshold,
                                        const int32_t* support,
                                        int32_t n_support,
                                        osar_metrics* out) {
  using namespace osar;
  if (!ctx) return OSAR_E_INVALID;
  if (ctx->sticky != OSAR_OK) return ctx->sticky;
  if (!out || !std::isfinite(threshold) || threshold < 0.0 || n_support < 0 ||
      (n_support > 0 && !support)) {
    ctx->last_error = "osar_get_metrics: bad arguments";
    return OSAR_E_INVALID;
  }
  const int m = ctx->pg ? ctx->pg->M : ctx->M;
  const double2* c = ctx->pg ? ctx->pg->c : ctx->c;
  std::vector<uint8_t> mask;
  if (n_support > 0) {
    mask.assign((size_t)m, 0);
    for (int32_t q = 0; q < n_support; ++q) {
      if (support[q] < 0 || support[q] >= m) {
        ctx->last_error = "osar_get_metrics: support index out of range";
        return OSAR_E_INVALID;
      }
      mask[(size_t)support[q]] = 1;
    }
  }
  auto cuda_err = [&](cudaError_t e) {
    ctx->last_error = std::string("osar_get_metrics: ") + cudaGetErrorName(e) +
                      " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return OSAR_E_OOM;
    ctx->sticky = OSAR_E_CUDA;
    return OSAR_E_CUDA;
  };
  // scratch (kept until destroy): the sums, then an M-byte support mask
  const size_t need = 256 + (size_t)m;
  if (!ctx->metrics_buf) {
    size_t total = 0;
    cudaError_t e = guarded_malloc(ctx->guards, &ctx->metrics_buf, need,
                                   "metrics_buf", ctx->stream, &total);
    if (e != cudaSuccess) return cuda_err(e);
    ctx->dev_bytes += (int64_t)total;
  }
  MetricSums* d_sums = static_cast<MetricSums*>(ctx->metrics_buf);
  uint8_t* d_mask = static_cast<uint8_t*>(ctx->metrics_buf) + 256;
  cudaError_t e = cudaSuccess;
  if (n_support > 0)
    e = cudaMemcpyAsync(d_mask, mask.data(), (size_t)m, cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess) {
    k_metrics<<<1, MT_THREADS, 0, ctx->stream>>>(
        c, n_support > 0 ? d_mask : nullptr, m, threshold, d_sums);
    ctx->launches++;
    e = cudaGetLastError();
  }
  MetricSums h{};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, d_sums, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(e);
  out->n_large = h.n_large;
  out->n_nonzero = h.n_nonzero;
  out->n_support = n_support > 0 ? h.n_on : 0;
  out->large_outside_support = n_support > 0 ? h.large_off : h.n_large;
  out->l1 = h.l1;
  out->max_abs = h.max_abs;
  const int n_off = m - (n_support > 0 ? h.n_on : 0);
  out->rms_signal = h.n_on > 0 ? std::sqrt(h.s_on / h.n_on) : 0.0;
  out->rms_noise = n_off > 0 ? std::sqrt(h.s_off / n_off) : 0.0;
  if (n_support == 0 || h.n_on == 0)
    out->snr_db = std::numeric_limits<double>::quiet_NaN();
  else if (out->rms_noise == 0.0)
    out->snr_db = out->rms_signal > 0.0 ? std::numeric_limits<double>::infinity()
                                        : std::numeric_limits<double>::quiet_NaN();
  else
    out->snr_db = 20.0 * std::log10(out->rms_signal / out->rms_noise);
  return OSAR_OK;
}
