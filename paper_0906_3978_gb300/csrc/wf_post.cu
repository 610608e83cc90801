// wf_post.cu -- the steps around the solve (Kitaura et al. 2009): the redshift-distortion factor
// and the deconvolution B^-1 Z^-1 of Sec. 3.3.2 (Eq. eq:DEC), and the evaluation of a reconstruction of
// Sec. 4.1 "Statistical correlation measures" and Sec. 5.5 "Statistics of the density field": Gaussian
// smoothing (both Fourier multipliers dispatch to the per-size FP64 transform passes), the
// correlation coefficient, Euclidean and normalised
// Kullback-Leibler distances, and binned density statistics per radial shell and observed /
// unobserved region with their moments.
//
// Decisions taken in floating point (the bin of 1 + delta, the shell of a node) use explicitly
// rounded FP64 operations in the order of the plain definition, so they are the ones the
// definition gives; counts are integer atomics (exact whatever the order); every sum is
// per-block partials plus a fixed-order single-CTA finisher (deterministic).
#include <cmath>
#include <vector>

#include "wf_ctx.h"
#include "wf_solver_group.h"
#include "wf_spectral.cuh"

namespace wf {

constexpr int kPostBlocks = 152 * 4;  // grid of the sweeps (per-block partials)

// ------------------------------------------------------------------------------------------
// Sec. 4.1: sums of t r, t^2, r^2, (r - t)^2, (1 + r) log((1 + r) / (1 + t)) (where both
// 1 + delta > 0) and the count of the cells left out of the last one.  6 partials per block.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_compare(const double* __restrict__ rec, const double* __restrict__ tru, size_t n, double* __restrict__ partials) {
  __shared__ double red[32];
  AccD tr, tt, rr, d2, kl;
  double excl = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double r = rec[e], t = tru[e];
    tr.add_prod(t, r);
    tt.add_prod(t, t);
    rr.add_prod(r, r);
    const double d = r - t;
    d2.add_prod(d, d);
    const double a = 1.0 + r, b = 1.0 + t;
    if (a > 0.0 && b > 0.0) kl.add(a * log(a / b));
    else excl += 1.0;
  }
  const double v[6] = {tr.get(), tt.get(), rr.get(), d2.get(), kl.get(), excl};
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const double s = block_sum(v[j], red);
    if (threadIdx.x == 0) partials[6 * blockIdx.x + j] = s;
  }
}

// res[0..3] = r, D_Euc, D_KL, excluded cells
__global__ void k_compare_fin(const double* __restrict__ partials, int nblk, double n_cells, double* __restrict__ res) {
  __shared__ double red[32];
  double s[6];
  for (int j = 0; j < 6; ++j) s[j] = sum_partials(partials, nblk, 6, j, red);
  if (threadIdx.x == 0) {
    res[0] = s[0] / (sqrt(s[1]) * sqrt(s[2]));
    res[1] = sqrt(s[3] / n_cells);
    res[2] = s[4] / n_cells;
    res[3] = s[5];
  }
}

// ------------------------------------------------------------------------------------------
// Sec. 5.5: counts of 1 + delta per (shell, region, bin); slot n_bins holds the values below the
// bins, slot n_bins + 1 those above.  Shared-memory counters per block, flushed with 64-bit
// atomics.  grid-stride over the n^3 nodes (n^3 < 2^31).
// ------------------------------------------------------------------------------------------
struct DensArgs {
  int n, n_shells, n_bins;
  double H, ox, oy, oz, lo, width;
  double shells[16];
};

__global__ void __launch_bounds__(256)
k_density_hist(const double* __restrict__ delta, const double* __restrict__ w, DensArgs a,
               unsigned long long* __restrict__ hist) {
  extern __shared__ unsigned int cnt[];  // [n_shells][2][n_bins + 2]
  const int nb2 = a.n_bins + 2, tot = a.n_shells * 2 * nb2;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) cnt[i] = 0u;
  __syncthreads();
  const unsigned un = (unsigned)a.n, V = un * un * un;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < V; e += gridDim.x * blockDim.x) {
    const double q = floor(__ddiv_rn(__dsub_rn(__dadd_rn(1.0, delta[e]), a.lo), a.width));
    int slot;
    if (q < 0.0) slot = a.n_bins;
    else if (q >= (double)a.n_bins) slot = a.n_bins + 1;
    else if (q >= 0.0) slot = (int)q;
    else continue;  // NaN: in no bin
    const unsigned row = e / un;
    const int iz = (int)(e - row * un), iy = (int)(row % un), ix = (int)(row / un);
    const double dx = __dsub_rn(__dmul_rn((double)ix, a.H), a.ox);
    const double dy = __dsub_rn(__dmul_rn((double)iy, a.H), a.oy);
    const double dz = __dsub_rn(__dmul_rn((double)iz, a.H), a.oz);
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const int g = w[e] > 0.0 ? 0 : 1;
    for (int s = 0; s < a.n_shells; ++s)
      if (r >= a.shells[2 * s] && r < a.shells[2 * s + 1]) atomicAdd(&cnt[(s * 2 + g) * nb2 + slot], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tot; i += blockDim.x)
    if (cnt[i]) atomicAdd(&hist[i], (unsigned long long)cnt[i]);
}

// One CTA per (shell, region): N, mean, mu2..mu4, skewness, kurtosis, Pearson's skewness from the
// bin centres lo + (i + 1/2) width - 1; the mode is the first bin of largest count.
__global__ void __launch_bounds__(256)
k_density_moments(const unsigned long long* __restrict__ hist, int n_bins, double lo, double width,
                  double* __restrict__ mom) {
  __shared__ double red[32];
  __shared__ double bc[2];
  __shared__ unsigned long long bmax[256];
  __shared__ int bidx[256];
  const unsigned long long* f = hist + (size_t)blockIdx.x * (n_bins + 2);
  const int tid = threadIdx.x;
  auto centre = [&](int i) { return __dsub_rn(__dadd_rn(lo, __dmul_rn((double)i + 0.5, width)), 1.0); };
  double sn = 0.0, sc = 0.0;
  unsigned long long mx = 0;
  int mi = 0x7fffffff;
  for (int i = tid; i < n_bins; i += blockDim.x) {
    const double fi = (double)f[i];
    sn += fi;
    sc += fi * centre(i);
    if (f[i] > mx) {  // i increases within a thread: the first of equal counts is kept
      mx = f[i];
      mi = i;
    }
  }
  bmax[tid] = mx;
  bidx[tid] = mi;
  const double N = block_sum(sn, red);
  const double SC = block_sum(sc, red);
  if (tid == 0) {
    bc[0] = N;
    bc[1] = N > 0.0 ? SC / N : 0.0;
  }
  __syncthreads();
  const double mean = bc[1];
  double s2 = 0.0, s3 = 0.0, s4 = 0.0;
  for (int i = tid; i < n_bins; i += blockDim.x) {
    const double fi = (double)f[i], d = centre(i) - mean, d2 = d * d;
    s2 += fi * d2;
    s3 += fi * d2 * d;
    s4 += fi * d2 * d2;
  }
  const double S2 = block_sum(s2, red), S3 = block_sum(s3, red), S4 = block_sum(s4, red);
  // mode: the largest count, ties to the smallest index (fixed-order tree)
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    __syncthreads();
    if (tid < o) {
      const unsigned long long c2 = bmax[tid + o];
      const int i2 = bidx[tid + o];
      if (c2 > bmax[tid] || (c2 == bmax[tid] && i2 < bidx[tid])) {
        bmax[tid] = c2;
        bidx[tid] = i2;
      }
    }
  }
  if (tid == 0) {
    double* m = mom + (size_t)blockIdx.x * 8;
    m[0] = N;
    if (N > 0.0) {
      const double mu2 = S2 / N, mu3 = S3 / N, mu4 = S4 / N, sig = sqrt(mu2);
      m[1] = mean;
      m[2] = mu2;
      m[3] = mu3;
      m[4] = mu4;
      m[5] = mu3 / (sig * sig * sig);
      m[6] = mu4 / (mu2 * mu2) - 3.0;
      m[7] = (mean - centre(bidx[0])) / sig;
    } else {
      for (int j = 1; j < 8; ++j) m[j] = NAN;
    }
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
wf_status multiply_fourier(Ctx& c, int n, const double* in, double* out, const std::vector<double>& table,
                           cudaStream_t st) {
  switch (n) {
#define WF_CASE(N) \
  case N:          \
    return fourier_multiply_n<N>(c, in, out, table, st);
    WF_SIZES(WF_CASE)
#undef WF_CASE
    default:
      return WF_ERR_UNSUPPORTED;
  }
}

// table index n2 = |m|^2 of the signed DFT index m, up to 3 (n/2)^2; |k| = 2 pi sqrt(n2) / box
static inline size_t n2_entries(int n) { return (size_t)3 * (n / 2) * (n / 2) + 1; }

wf_status smooth_run(Ctx& c, const wf_grid& g, const double* in, double r_s, double* out, cudaStream_t st) {
  if (!in || !out || !(r_s >= 0.0) || !std::isfinite(r_s)) return WF_ERR_ARG;
  std::vector<double> t(n2_entries(g.n));
  const double kf = 2.0 * 3.14159265358979323846 / g.box;
  for (size_t n2 = 0; n2 < t.size(); ++n2) t[n2] = std::exp(-0.5 * kf * kf * (double)n2 * r_s * r_s);
  return multiply_fourier(c, g.n, in, out, t, st);
}

// <K D>_mu of Sec. 3.3.3 ("Redshift distortion operator"): the mean over mu in [0, 1] of
// (1 + beta mu^2)^2 / (1 + a mu^2), a = k^2 sigma_v^2 / 2.  Dividing the numerator by 1 + a mu^2
// gives beta^2 / (3a) + 2 beta / a - beta^2 / a^2 + (1 - beta / a)^2 atan(sqrt a) / sqrt a; for
// a < 1/2, where those terms cancel, the power series sum_j (-a)^j (1/(2j+1) + 2 beta/(2j+3) +
// beta^2/(2j+5)) is summed instead.
double rsd_factor(double k, double beta, double sigma_v) {
  const double a = 0.5 * (k * sigma_v) * (k * sigma_v);
  if (a < 0.5) {
    double sum = 0.0, p = 1.0;
    for (int j = 0; j < 200; ++j) {
      const double term = p * (1.0 / (2 * j + 1) + 2.0 * beta / (2 * j + 3) + beta * beta / (2 * j + 5));
      sum += term;
      if (std::fabs(term) <= 1e-18 * std::fabs(sum)) break;
      p *= -a;
    }
    return sum;
  }
  const double sa = std::sqrt(a), u = 1.0 - beta / a;
  return beta * beta / (3.0 * a) + 2.0 * beta / a - beta * beta / (a * a) + u * u * std::atan(sa) / sa;
}

wf_status deconvolve_run(Ctx& c, const wf_grid& g, const double* in, double beta, double sigma_v, double bias,
                         double* out, cudaStream_t st) {
  if (!in || !out || !std::isfinite(beta) || !(sigma_v >= 0.0) || !std::isfinite(sigma_v) || !(bias > 0.0) ||
      !std::isfinite(bias))
    return WF_ERR_ARG;
  std::vector<double> t(n2_entries(g.n));
  const double kf = 2.0 * 3.14159265358979323846 / g.box;
  for (size_t n2 = 0; n2 < t.size(); ++n2) {
    const double f = rsd_factor(kf * std::sqrt((double)n2), beta, sigma_v);
    if (!(f > 0.0)) return WF_ERR_ARG;  // (1 + beta mu^2)^2 vanishing on all of [0, 1] is impossible;
                                        // a non-positive mean only comes from a non-finite input
    t[n2] = 1.0 / (bias * std::sqrt(f));
  }
  return multiply_fourier(c, g.n, in, out, t, st);
}

wf_status response_tables(const wf_grid& g, const wf_response* r, std::vector<double>& sinv,
                          std::vector<double>& ginv) {
  if (!r || !(r->bias > 0.0) || !std::isfinite(r->bias) || !std::isfinite(r->beta) || !(r->sigma_v >= 0.0) ||
      !std::isfinite(r->sigma_v))
    return WF_ERR_ARG;
  ginv.assign(n2_entries(g.n), 0.0);
  if (sinv.size() != ginv.size()) return WF_ERR_ARG;
  const double kf = 2.0 * 3.14159265358979323846 / g.box;
  for (size_t n2 = 0; n2 < ginv.size(); ++n2) {
    const double f = rsd_factor(kf * std::sqrt((double)n2), r->beta, r->sigma_v);
    if (!(f > 0.0)) return WF_ERR_ARG;
    const double g2 = r->bias * r->bias * f;  // g(k)^2
    sinv[n2] /= g2;
    ginv[n2] = 1.0 / (r->bias * std::sqrt(f));
  }
  return WF_OK;
}

wf_status compare_run(Ctx& c, int64_t n_cells, const double* rec, const double* truth, wf_compare_result* out,
                      cudaStream_t st) {
  if (n_cells <= 0 || !rec || !truth || !out) return WF_ERR_ARG;
  double *part, *res, *hres;
  WF_TRY(c.get("post_part", (size_t)kPostBlocks * 6 * sizeof(double), (void**)&part));
  WF_TRY(c.get("post_res", 4 * sizeof(double), (void**)&res));
  WF_TRY(c.get_pinned("post_res_h", 4 * sizeof(double), (void**)&hres));
  c.launch("compare", 16.0 * (double)n_cells, st,
           [&] { k_compare<<<kPostBlocks, 256, 0, st>>>(rec, truth, (size_t)n_cells, part); });
  c.launch("fin", 0, st, [&] { k_compare_fin<<<1, 1024, 0, st>>>(part, kPostBlocks, (double)n_cells, res); });
  WF_CUDA(cudaMemcpyAsync(hres, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  out->r = hres[0];
  out->d_euc = hres[1];
  out->d_kl = hres[2];
  out->kl_excluded = (int64_t)hres[3];
  return WF_OK;
}

wf_status density_run(Ctx& c, const wf_grid& g, const double* delta, const double* w, const double* observer,
                      int n_shells, const double* shells, double lo, double width, int n_bins, int64_t* hist,
                      wf_density_moments* moments, cudaStream_t st) {
  if (!delta || !w || !observer || !shells || !hist || !moments || n_shells < 1 || n_shells > 8 || n_bins < 1 ||
      (int64_t)n_shells * (n_bins + 2) > 6144 || !(width > 0.0) || !std::isfinite(width) || !std::isfinite(lo))
    return WF_ERR_ARG;
  DensArgs a;
  a.n = g.n;
  a.n_shells = n_shells;
  a.n_bins = n_bins;
  a.H = g.box / (double)g.n;
  a.ox = observer[0];
  a.oy = observer[1];
  a.oz = observer[2];
  a.lo = lo;
  a.width = width;
  for (int i = 0; i < 16; ++i) a.shells[i] = i < 2 * n_shells ? shells[i] : 0.0;
  for (int i = 0; i < 2 * n_shells; ++i)
    if (std::isnan(shells[i])) return WF_ERR_ARG;
  const int nb2 = n_bins + 2, slots = n_shells * 2 * nb2;
  unsigned long long *dh, *hh;
  double *dm, *hm;
  WF_TRY(c.get("post_hist", (size_t)slots * sizeof(unsigned long long), (void**)&dh));
  WF_TRY(c.get("post_mom", (size_t)n_shells * 2 * 8 * sizeof(double), (void**)&dm));
  WF_TRY(c.get_pinned("post_hist_h", (size_t)slots * sizeof(unsigned long long), (void**)&hh));
  WF_TRY(c.get_pinned("post_mom_h", (size_t)n_shells * 2 * 8 * sizeof(double), (void**)&hm));
  WF_CUDA(cudaMemsetAsync(dh, 0, (size_t)slots * sizeof(unsigned long long), st));
  const size_t V = (size_t)g.n * g.n * g.n;
  const size_t smem = (size_t)slots * sizeof(unsigned int);
  c.launch("density_hist", 16.0 * (double)V, st,
           [&] { k_density_hist<<<kPostBlocks, 256, smem, st>>>(delta, w, a, dh); });
  c.launch("fin", 0, st, [&] { k_density_moments<<<n_shells * 2, 256, 0, st>>>(dh, n_bins, lo, width, dm); });
  WF_CUDA(cudaMemcpyAsync(hh, dh, (size_t)slots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaMemcpyAsync(hm, dm, (size_t)n_shells * 2 * 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < slots; ++i) hist[i] = (int64_t)hh[i];
  for (int j = 0; j < n_shells * 2; ++j) {
    const double* m = hm + 8 * j;
    moments[j] = wf_density_moments{m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7]};
  }
  return WF_OK;
}

}  // namespace wf

// ==========================================================================================
// FP64 FMA throughput of the device (a measurement for reporting the FP64-bound kernels against
// a measured peak): every thread runs 8 independent FMA chains; 2 flops per FMA.
// ==========================================================================================
namespace wf {
static __global__ void __launch_bounds__(256) k_fma_rate(double* __restrict__ out, int iters, double a, double b) {
  double v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = fma(v[j], a, b);
  double t = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) t += v[j];
  if (t == 12345.678) out[0] = t;  // keeps the chains live; practically never stores
}
}  // namespace wf

extern "C" wf_status wf_fp64_rate(wf_ctx* ctx, double* flops_per_s) {
  using namespace wf;
  if (!ctx || !flops_per_s) return WF_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  int sms = 0;
  WF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  double* out;
  WF_TRY(c->get("fma_rate", 64, (void**)&out));
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  cudaEvent_t e0, e1;
  WF_CUDA(cudaEventCreate(&e0));
  WF_CUDA(cudaEventCreate(&e1));
  k_fma_rate<<<blocks, threads>>>(out, iters / 8, 0.999999, 1e-7);  // warm-up
  WF_CUDA(cudaEventRecord(e0));
  k_fma_rate<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  WF_CUDA(cudaEventRecord(e1));
  WF_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  WF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return WF_OK;
}
