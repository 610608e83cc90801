// wf_assign.cu -- supersampled mass assignment (Sec. 3.1.2 of Kitaura et al. 2009, Eq. def:ngrid).
//
// Step 1: each galaxy is placed on the fine grid (s n)^3 with CIC or TSC weights in fixed
//         point (Q16 per axis, product Q48) by 64-bit integer atomics, so the fine grid is
//         exact and independent of the order in which galaxies land.
// Step 2: the ideal discrete low-pass filter (keep modes with every |k_i| < n/2, drop the
//         coarse Nyquist planes) and sampling at n^3.  The filter is a box in k and therefore
//         separable: per axis, a line of 2n samples is transformed (real FFT of length 2n,
//         computed as a complex FFT of length n), the n/2 lowest modes are kept, and the line
//         is transformed back at length n (complex FFT of length n/2) and divided by n.
//         Three passes (z, y, x) each halve one axis: (2n)^3 -> (2n)^2 n -> 2n n^2 -> n^3.
#include "wf_ctx.h"
#include "wf_spectral.cuh"

namespace wf {

// ------------------------------------------------------------------------------------------
// step 1: fixed-point CIC / TSC atomics
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int axis_nodes(double x, double scale, long long nf, int scheme,
                                          long long* node, unsigned long long* wt) {
  const double u = __dmul_rn(x, scale);
  if (!(fabs(u) < 4503599627370496.0)) return -1;  // 2^52: floor exact, non-finite rejected
  const long long m = nf * 65536LL;
  long long q = (long long)floor(u);
  q %= m;
  if (q < 0) q += m;
  if (scheme == WF_CIC) {
    const long long i = q >> 16;
    const unsigned long long f = (unsigned long long)(q & 0xFFFF);
    node[0] = i % nf;
    node[1] = (i + 1) % nf;
    wt[0] = 65536ULL - f;
    wt[1] = f;
    return 2;
  }
  const long long qp = q + 32768;
  const long long j = qp >> 16;
  const long long D = (qp & 0xFFFF) - 32768;  // offset from node j, [-2^15, 2^15)
  const unsigned long long a = (unsigned long long)(32768 - D), b = (unsigned long long)(32768 + D);
  const unsigned long long wm = (a * a) >> 17, wp = (b * b) >> 17;
  node[0] = ((j - 1) % nf + nf) % nf;
  node[1] = j % nf;
  node[2] = (j + 1) % nf;
  wt[0] = wm;
  wt[1] = 65536ULL - wm - wp;
  wt[2] = wp;
  return 3;
}

__global__ void __launch_bounds__(256)
k_assign(const double* __restrict__ pos, long long n_gal, long long nf, double scale, int scheme,
         unsigned long long* __restrict__ fine, int* __restrict__ err) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= n_gal) return;
  long long nd[3][3];
  unsigned long long wt[3][3];
  int cnt = 0;
  for (int a = 0; a < 3; ++a) {
    cnt = axis_nodes(pos[3 * g + a], scale, nf, scheme, nd[a], wt[a]);
    if (cnt < 0) {
      atomicOr(err, 1);
      return;
    }
  }
  for (int i = 0; i < cnt; ++i)
    for (int j = 0; j < cnt; ++j) {
      const size_t rowb = ((size_t)nd[0][i] * nf + (size_t)nd[1][j]) * nf;
      const unsigned long long wij = wt[0][i] * wt[1][j];
      for (int k = 0; k < cnt; ++k) {
        const unsigned long long add = wij * wt[2][k];
        if (add == 0) continue;
        const unsigned long long old = atomicAdd(fine + rowb + nd[2][k], add);
        if (old + add < old) atomicOr(err, 2);
      }
    }
}

// Weighted assignment for the inverse-weighting estimator (Sec. 4, Eq. def:ngrid with galaxy
// mass wgt[g], e.g. 1 / w): each node contribution is the Q48 weight times wgt[g], rounded once
// to the nearest Q32 unit, so the grid is exact and independent of the order of the atomics.
__global__ void __launch_bounds__(256)
k_assign_weighted(const double* __restrict__ pos, const double* __restrict__ wgt, long long n_gal, long long nf,
                  double scale, int scheme, unsigned long long* __restrict__ fine, int* __restrict__ err) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= n_gal) return;
  const double wg = wgt[g];
  if (!(wg >= 0.0) || !(wg < 4294967296.0)) {  // [0, 2^32): a contribution stays below 2^64
    atomicOr(err, 1);
    return;
  }
  long long nd[3][3];
  unsigned long long wt[3][3];
  int cnt = 0;
  for (int a = 0; a < 3; ++a) {
    cnt = axis_nodes(pos[3 * g + a], scale, nf, scheme, nd[a], wt[a]);
    if (cnt < 0) {
      atomicOr(err, 1);
      return;
    }
  }
  for (int i = 0; i < cnt; ++i)
    for (int j = 0; j < cnt; ++j) {
      const size_t rowb = ((size_t)nd[0][i] * nf + (size_t)nd[1][j]) * nf;
      const unsigned long long wij = wt[0][i] * wt[1][j];
      for (int k = 0; k < cnt; ++k) {
        const double q = __ull2double_rn(wij * wt[2][k]);  // exact: < 2^49
        const unsigned long long add = __double2ull_rn(__dmul_rn(__dmul_rn(q, wg), 1.0 / 65536.0));
        if (add == 0) continue;
        const unsigned long long old = atomicAdd(fine + rowb + nd[2][k], add);
        if (old + add < old) atomicOr(err, 2);
      }
    }
}

// fine grid in fixed-point units (2^-48 galaxies, 2^-32 weighted galaxies) -> FP64 counts
__global__ void k_q48_to_double(const unsigned long long* __restrict__ fine, double* __restrict__ out, size_t n,
                                double unit) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __ull2double_rn(fine[i]) * unit;
}

// ------------------------------------------------------------------------------------------
// step 2: one axis of the ideal low-pass: line of 2N reals -> N reals.
// AXIS 0: lines along z (contiguous rows), input rows of 2N, (2N)^2 rows.
// AXIS 1: lines along y of [2N][2N][N]  -> [2N][N][N]; tile = NL consecutive z, fixed x.
// AXIS 2: lines along x of [2N][N][N]   -> [N][N][N];  tile = NL consecutive z, fixed y.
// ------------------------------------------------------------------------------------------
template <class IN> WF_D double to_real(IN v, double s);
template <> WF_D double to_real<unsigned long long>(unsigned long long v, double s) { return __ull2double_rn(v) * s; }
template <> WF_D double to_real<double>(double v, double s) { return v * s; }

// lines per CTA: a divisor of N (the y and x passes tile N consecutive z values)
template <class R, int N> constexpr int lp_lines() { return div_le(N, tile_lines<R>()); }
template <class R, int N>
constexpr int lp_threads() { return lp_lines<R, N>() * tpl<R, N>(); }

template <class R, int N, int AXIS, class IN>
__global__ void __launch_bounds__(lp_threads<R, N>())
k_lowpass(const IN* __restrict__ in, double* __restrict__ out, double in_scale,
          const double2* __restrict__ twtab) {
  constexpr int M = N, NL = lp_lines<R, N>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = NL * TPL;
  static_assert(N % NL == 0, "tile width must divide N");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;  // exp(-2 pi i e/(2N)), e < 2N
  const int tid = threadIdx.x;
  for (int e = tid; e < 2 * N; e += NT) tw[e] = ld_c<R>(twtab + e);
  // ---- load 2N reals per line as N complex
  if constexpr (AXIS == 0) {
    const size_t r0 = (size_t)blockIdx.x * NL;
    int nonzero = 0;
    for (int idx = tid; idx < M * NL; idx += NT) {
      const int l = idx / M, m = idx % M;
      const IN* src = in + (r0 + l) * (2 * N) + 2 * m;
      nonzero |= (src[0] != 0) | (src[1] != 0);
      tile[m * LD + l] = cx<R>{RT<R>::from_d(to_real(src[0], in_scale)), RT<R>::from_d(to_real(src[1], in_scale))};
    }
    // rows the survey never reaches are all zero: their filtered output is exactly zero
    if (!__syncthreads_or(nonzero)) {
      double2* o2 = reinterpret_cast<double2*>(out);
      for (int idx = tid; idx < (M / 2) * NL; idx += NT)
        o2[(r0 + idx / (M / 2)) * (N / 2) + idx % (M / 2)] = make_double2(0.0, 0.0);
      return;
    }
  } else {
    const int z0 = blockIdx.x * NL, c = blockIdx.y;
    for (int idx = tid; idx < M * NL; idx += NT) {
      const int m = idx / NL, l = idx % NL;
      size_t e0, e1;
      if constexpr (AXIS == 1) {
        e0 = ((size_t)c * 2 * N + 2 * m) * N + z0 + l;
        e1 = e0 + N;
      } else {
        e0 = ((size_t)(2 * m) * N + c) * N + z0 + l;
        e1 = e0 + (size_t)N * N;
      }
      tile[m * LD + l] = cx<R>{RT<R>::from_d(to_real(in[e0], in_scale)), RT<R>::from_d(to_real(in[e1], in_scale))};
    }
  }
  __syncthreads();
  const int l = tid % NL, t = tid / NL;
  cx<R>* col = tile + l;
  // forward complex FFT of length N (real FFT of length 2N, packed)
  fft_line<R, M, TPL, LD, -1, 2>(col, t, tw);
  // real-2N spectrum X_k, k < N/2, then the length-N C2R pre-step with X_{N/2} = 0
  const R half = RT<R>::c(0.5);
  for (int k = t; k <= N / 4; k += TPL) {
    if (k == 0) {
      const cx<R> z = col[0];
      const R x0 = z.x + z.y;
      col[0] = cx<R>{x0, x0};
    } else {
      const int k2 = N / 2 - k;
      const cx<R> za = col[k * LD], zb = col[(N - k) * LD];
      const cx<R> zc = col[k2 * LD], zd = col[(N - k2) * LD];
      // X_k = (Z_k + conj Z_{N-k})/2 - (i/2) W_2N^k (Z_k - conj Z_{N-k})
      const cx<R> Xa = scale((za + conj(zb)) - mul_i(tw[k] * (za - conj(zb))), half);
      const cx<R> Xc = scale((zc + conj(zd)) - mul_i(tw[k2] * (zc - conj(zd))), half);
      // Z'_k = (X_k + conj X_{N/2-k}) + i W_N^{-k}* (X_k - conj X_{N/2-k})
      col[k * LD] = (Xa + conj(Xc)) + mul_i(conj(tw[2 * k]) * (Xa - conj(Xc)));
      if (k2 != k) col[k2 * LD] = (Xc + conj(Xa)) + mul_i(conj(tw[2 * k2]) * (Xc - conj(Xa)));
    }
  }
  __syncthreads();
  fft_line<R, M / 2, TPL, LD, +1, 4>(col, t, tw);
  // ---- store N reals per line (N/2 complex), divided by N
  const double inv_n = 1.0 / (double)N;
  if constexpr (AXIS == 0) {
    const size_t r0 = (size_t)blockIdx.x * NL;
    double2* o2 = reinterpret_cast<double2*>(out);
    for (int idx = tid; idx < (M / 2) * NL; idx += NT) {
      const int ll = idx / (M / 2), m = idx % (M / 2);
      const cx<R> v = tile[m * LD + ll];
      o2[(r0 + ll) * (N / 2) + m] = make_double2(RT<R>::to_d(v.x) * inv_n, RT<R>::to_d(v.y) * inv_n);
    }
  } else {
    const int z0 = blockIdx.x * NL, c = blockIdx.y;
    for (int idx = tid; idx < (M / 2) * NL; idx += NT) {
      const int m = idx / NL, ll = idx % NL;
      const cx<R> v = tile[m * LD + ll];
      size_t e0, e1;
      if constexpr (AXIS == 1) {
        e0 = ((size_t)c * N + 2 * m) * N + z0 + ll;
        e1 = e0 + N;
      } else {
        e0 = ((size_t)(2 * m) * N + c) * N + z0 + ll;
        e1 = e0 + (size_t)N * N;
      }
      out[e0] = RT<R>::to_d(v.x) * inv_n;
      out[e1] = RT<R>::to_d(v.y) * inv_n;
    }
  }
}

template <class K>
static cudaError_t smem_attr(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class R, int N>
static wf_status lowpass_sized(Ctx& c, const unsigned long long* fine, double* n_obs, double unit,
                               cudaStream_t st) {
  constexpr int NL = lp_lines<R, N>();
  const size_t smem = (size_t)(N * (NL + 1) + 2 * N) * sizeof(cx<R>);
  const int nt = lp_threads<R, N>();
  const double2* tw;
  WF_TRY(c.tw(N, &tw));
  double *t1, *t2;
  WF_TRY(c.get("lp_t1", (size_t)4 * N * N * N * sizeof(double), (void**)&t1));
  WF_TRY(c.get("lp_t2", (size_t)2 * N * N * N * sizeof(double), (void**)&t2));
  WF_CUDA(smem_attr(k_lowpass<R, N, 0, unsigned long long>, smem));
  WF_CUDA(smem_attr(k_lowpass<R, N, 1, double>, smem));
  WF_CUDA(smem_attr(k_lowpass<R, N, 2, double>, smem));
  const double q48 = unit;
  const double V = (double)N * N * N;
  c.launch("lowpass_z", 8 * (8 * V + 4 * V), st, [&] {
    k_lowpass<R, N, 0, unsigned long long><<<(unsigned)((size_t)4 * N * N / NL), nt, smem, st>>>(fine, t1, q48, tw);
  });
  WF_CUDA(cudaGetLastError());
  c.launch("lowpass_y", 8 * (4 * V + 2 * V), st,
           [&] { k_lowpass<R, N, 1, double><<<dim3(N / NL, 2 * N), nt, smem, st>>>(t1, t2, 1.0, tw); });
  WF_CUDA(cudaGetLastError());
  c.launch("lowpass_x", 8 * (2 * V + V), st,
           [&] { k_lowpass<R, N, 2, double><<<dim3(N / NL, N), nt, smem, st>>>(t2, n_obs, 1.0, tw); });
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

static wf_status assign_any(Ctx& c, const wf_grid& g, int scheme, const double* pos, const double* wgt,
                            int64_t n_gal, uint64_t* fine_out, double* n_obs, cudaStream_t st);

wf_status assign_run(Ctx& c, const wf_grid& g, int scheme, const double* pos, int64_t n_gal,
                     uint64_t* fine_out, double* n_obs, cudaStream_t st) {
  return assign_any(c, g, scheme, pos, nullptr, n_gal, fine_out, n_obs, st);
}

wf_status assign_weighted_run(Ctx& c, const wf_grid& g, int scheme, const double* pos, const double* wgt,
                              int64_t n_gal, uint64_t* fine_out, double* n_obs, cudaStream_t st) {
  if (n_gal > 0 && !wgt) return WF_ERR_ARG;
  return assign_any(c, g, scheme, pos, wgt, n_gal, fine_out, n_obs, st);
}

// wgt == nullptr: unit masses in Q48; else masses wgt[g] in Q32.
static wf_status assign_any(Ctx& c, const wf_grid& g, int scheme, const double* pos, const double* wgt,
                            int64_t n_gal, uint64_t* fine_out, double* n_obs, cudaStream_t st) {
  const int n = g.n, ss = g.supersample;
  if (!supported_size(n)) return WF_ERR_UNSUPPORTED;
  if (!(g.box > 0.0) || !(g.box < 1e300) || (ss != 1 && ss != 2) || (scheme != WF_CIC && scheme != WF_TSC) ||
      n_gal < 0 || (n_gal > 0 && !pos) || !n_obs)
    return WF_ERR_ARG;
  const long long nf = (long long)ss * n;
  const size_t nfine = (size_t)nf * nf * nf;
  unsigned long long* fine = reinterpret_cast<unsigned long long*>(fine_out);
  if (!fine) WF_TRY(c.get("fine", nfine * sizeof(uint64_t), (void**)&fine));
  int* err;
  WF_TRY(c.get("assign_err", 64, (void**)&err));
  WF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  WF_CUDA(cudaMemsetAsync(fine, 0, nfine * sizeof(uint64_t), st));  // counted as a launch below
  c.prof.launches += 1;
  const double scale = ((double)nf * 65536.0) / g.box;
  const double unit = wgt ? 2.3283064365386963e-10 /* 2^-32 */ : 3.5527136788005009e-15 /* 2^-48 */;
  if (n_gal > 0) {
    c.launch("assign", 24.0 * n_gal + 16.0 * 27 * n_gal, st, [&] {
      if (wgt)
        k_assign_weighted<<<(unsigned)((n_gal + 255) / 256), 256, 0, st>>>(pos, wgt, (long long)n_gal, nf, scale,
                                                                           scheme, fine, err);
      else
        k_assign<<<(unsigned)((n_gal + 255) / 256), 256, 0, st>>>(pos, (long long)n_gal, nf, scale, scheme, fine, err);
    });
    WF_CUDA(cudaGetLastError());
  }
  if (ss == 1) {
    c.launch("q48", 16.0 * nfine, st, [&] { k_q48_to_double<<<1216, 256, 0, st>>>(fine, n_obs, nfine, unit); });
    WF_CUDA(cudaGetLastError());
  } else {
    wf_status s = WF_ERR_UNSUPPORTED;
    switch (n) {
#define WF_CASE(N) \
  case N:          \
    s = lowpass_sized<double, N>(c, fine, n_obs, unit, st); \
    break;
      WF_SIZES(WF_CASE)
#undef WF_CASE
    }
    if (s != WF_OK) return s;
  }
  int* h = reinterpret_cast<int*>(c.host_pinned);
  WF_CUDA(cudaMemcpyAsync(h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (h[0] & 1) return WF_ERR_ARG;
  if (h[0] & 2) return WF_ERR_OVERFLOW;
  return WF_OK;
}

}  // namespace wf
