// wf_noise.cu -- 3D window, mean density, data and noise diagonals
// (Kitaura et al. 2009, Sec. 3.1.3 and Sec. 3.2: Eqs. eq:datamodel, eq:nmean, eq:noiseav).
//
//   w    = [in cone] * [outside every hole] * f(r) at node x = i H (no periodic wrap)
//   nbar = N_gal / sum(w)               (galaxies per cell; the observed volume in cells)
//   d    = n_obs / nbar - w
//   b    = R^T N^-1 d = nbar d  (w > 0),  0 (w = 0)     with R = diag(w), N = diag(w / nbar)
// The cone and hole tests are decisions taken in floating point; they are evaluated with
// explicitly rounded IEEE operations in a fixed order (no contraction), so the decision is the
// one the plain definition gives.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "wf_ctx.h"
#include "wf_spectral.cuh"

namespace wf {

struct SelParams {
  double ox, oy, oz;
  double ax, ay, az;
  double cos_half;
  double H;
  double p0, p1;
  int kind;
  int n_holes;
};

// The selection at offset (dx, dy, dz) from the observer: cone x holes x radial law, w = 0 at
// the observer; every operation explicitly rounded, in the order of the definition.
WF_D double sel_value(const SelParams& s, const double4* __restrict__ holes, double dx, double dy, double dz) {
  const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  double val = 0.0;
  if (r > 0.0) {
    bool inside = __dadd_rn(__dadd_rn(__dmul_rn(dx, s.ax), __dmul_rn(dy, s.ay)), __dmul_rn(dz, s.az)) >=
                  __dmul_rn(s.cos_half, r);
    for (int h = 0; h < s.n_holes && inside; ++h) {
      const double4 hv = holes[h];
      if (__dadd_rn(__dadd_rn(__dmul_rn(dx, hv.x), __dmul_rn(dy, hv.y)), __dmul_rn(dz, hv.z)) > __dmul_rn(hv.w, r))
        inside = false;
    }
    if (inside) {
      if (s.kind == 0) {
        val = 1.0;
      } else if (s.kind == 1) {
        const double t = __ddiv_rn(r, s.p0);
        val = exp(-__dmul_rn(t, t));
      } else {
        // t^p1 exp(p1 (1 - t)) as one exponential, exp(p1 (log t + 1 - t))
        const double t = __ddiv_rn(r, s.p0);
        val = exp(__dmul_rn(s.p1, __dadd_rn(log(t), __dsub_rn(1.0, t))));
      }
    }
  }
  return val;
}

__global__ void __launch_bounds__(256)
k_window(int n, SelParams s, const double4* __restrict__ holes, double* __restrict__ w,
         double* __restrict__ partials) {
  __shared__ double red[32];
  const size_t V = (size_t)n * n * n;
  AccD acc;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < V; e += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)(e % n), iy = (int)((e / n) % n), ix = (int)(e / ((size_t)n * n));
    const double val = sel_value(s, holes, __dsub_rn(__dmul_rn((double)ix, s.H), s.ox),
                                 __dsub_rn(__dmul_rn((double)iy, s.H), s.oy),
                                 __dsub_rn(__dmul_rn((double)iz, s.H), s.oz));
    w[e] = val;
    acc.add(val);
  }
  const double sum = block_sum(acc.get(), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

// The selection at arbitrary positions pos[3 i] (the completeness at a galaxy), or its
// reciprocal (0 where w = 0), the galaxy mass of the inverse-weighting estimator.
__global__ void __launch_bounds__(256)
k_window_at(const double* __restrict__ pos, long long n_pts, SelParams s, const double4* __restrict__ holes,
            bool reciprocal, double* __restrict__ w) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pts; i += (long long)gridDim.x * blockDim.x) {
    const double v = sel_value(s, holes, __dsub_rn(pos[3 * i], s.ox), __dsub_rn(pos[3 * i + 1], s.oy),
                               __dsub_rn(pos[3 * i + 2], s.oz));
    w[i] = reciprocal ? (v > 0.0 ? __drcp_rn(v) : 0.0) : v;
  }
}

// scal[0] = sum(w), scal[1] = nbar, scal[2] = 1/nbar
__global__ void k_nbar(const double* __restrict__ partials, int np, double n_gal, double* scal) {
  __shared__ double red[32];
  const double s = sum_partials(partials, np, 1, 0, red);
  if (threadIdx.x == 0) {
    scal[0] = s;
    const double nb = s > 0.0 ? n_gal / s : 0.0;
    scal[1] = nb;
    scal[2] = nb > 0.0 ? 1.0 / nb : 0.0;
  }
}

__global__ void __launch_bounds__(256)
k_data(const double* __restrict__ n_obs, const double* __restrict__ w, const double* __restrict__ scal,
       double* __restrict__ d, double* __restrict__ b, size_t V) {
  const double nb = scal[1], inb = scal[2];
  const double2* no2 = reinterpret_cast<const double2*>(n_obs);
  const double2* w2 = reinterpret_cast<const double2*>(w);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < V / 2; e += (size_t)gridDim.x * blockDim.x) {
    const double2 nv = no2[e], wv = w2[e];
    double2 dv, bv;
    dv.x = nv.x * inb - wv.x;
    dv.y = nv.y * inb - wv.y;
    bv.x = wv.x > 0.0 ? nb * dv.x : 0.0;
    bv.y = wv.y > 0.0 ? nb * dv.y : 0.0;
    if (d) reinterpret_cast<double2*>(d)[e] = dv;
    reinterpret_cast<double2*>(b)[e] = bv;
  }
}

// ------------------------------------------------------------------------------------------
// Signal-dependent noise (Eq. eq:noisecov, N^SD = w lambda / nbar^2): the solve's diagonal
// nbar^2 w / lambda and right-hand side nbar^2 d / lambda, d = n_obs / nbar - w; lambda given, or
// the flat-prior mean (n_obs + 1) / w.  Cells with w = 0 or lambda <= 0 carry no data term.
// Every operation explicitly rounded in the order of the definition.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_sd_noise(const double* __restrict__ n_obs, const double* __restrict__ w, const double* __restrict__ lam,
           double nbar, size_t n, double* __restrict__ D, double* __restrict__ b) {
  const double nb2 = __dmul_rn(nbar, nbar);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double nv = n_obs[e], wv = w[e];
    const double l = lam ? lam[e] : (wv > 0.0 ? __ddiv_rn(__dadd_rn(nv, 1.0), wv) : 0.0);
    if (wv > 0.0 && l > 0.0) {
      const double d = __dsub_rn(__ddiv_rn(nv, nbar), wv);
      D[e] = __ddiv_rn(__dmul_rn(nb2, wv), l);
      b[e] = __ddiv_rn(__dmul_rn(nb2, d), l);
    } else {
      D[e] = 0.0;
      b[e] = 0.0;
    }
  }
}

// Eq. eq:selfunc: galaxy g kept when u_g < alpha / w_g, then mass 1 / alpha (else 0).
__global__ void __launch_bounds__(256)
k_jackknife_masses(const double* __restrict__ w, const double* __restrict__ u, double alpha, long long n,
                   double* __restrict__ out) {
  const double inv = __drcp_rn(alpha);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double wv = w[i];
    out[i] = (wv > 0.0 && u[i] < __ddiv_rn(alpha, wv)) ? inv : 0.0;
  }
}

wf_status sd_noise_run(Ctx& c, int64_t n_cells, const double* n_obs, const double* w, const double* lambda,
                       double nbar, double* D, double* b, cudaStream_t st) {
  if (n_cells <= 0 || !n_obs || !w || !D || !b || !(nbar > 0.0) || !std::isfinite(nbar)) return WF_ERR_ARG;
  c.launch("sd_noise", (lambda ? 40.0 : 32.0) * (double)n_cells, st, [&] {
    k_sd_noise<<<152 * 4, 256, 0, st>>>(n_obs, w, lambda, nbar, (size_t)n_cells, D, b);
  });
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status jackknife_run(Ctx& c, int64_t n_gal, const double* w_gal, const double* u, double alpha, double* out,
                        cudaStream_t st) {
  if (n_gal < 0 || (n_gal > 0 && (!w_gal || !u || !out)) || !(alpha > 0.0) || !(alpha <= 1.0)) return WF_ERR_ARG;
  if (n_gal == 0) return WF_OK;
  const unsigned grid = (unsigned)std::min<int64_t>((n_gal + 255) / 256, 152 * 16);
  c.launch("jackknife", 24.0 * (double)n_gal, st,
           [&] { k_jackknife_masses<<<grid, 256, 0, st>>>(w_gal, u, alpha, (long long)n_gal, out); });
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// acc += f s, element by element (the mean of the Jackknife reconstructions, added in subsample order)
__global__ void __launch_bounds__(256)
k_add_scaled(double* __restrict__ acc, const double* __restrict__ s, double f, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc[i] = __dadd_rn(acc[i], __dmul_rn(f, s[i]));
}

wf_status add_scaled_run(Ctx& c, int64_t n, const double* s, double f, double* acc, cudaStream_t st) {
  if (n <= 0 || !s || !acc) return WF_ERR_ARG;
  c.launch("add_scaled", 24.0 * (double)n, st,
           [&] { k_add_scaled<<<152 * 4, 256, 0, st>>>(acc, s, f, (size_t)n); });
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// ------------------------------------------------------------------------------------------
// Projection of a sky completeness map along rays (Sec. 3.1.3, Eq. eq:transf): sample (j, i, k) is
// the point o + r_k u_ij, r_k = (k + 1/2) dr, u = (cos d cos a, cos d sin a, sin d) with the
// pixel-centre cosines and sines from the host; its nearest-grid-point cell receives the pixel's
// sky value and the radial table's value in Q32 fixed point (integer atomics: exact, any order)
// and one count.  Every operation explicitly rounded in the order of the definition.
// ------------------------------------------------------------------------------------------
struct MaskArgs {
  int n, n_r, kc;  // kc = ceil(n_r / 32): 32-sample chunks per ray
  long long npix;
  double step;     // dr / H
  float ox, oy, oz;  // observer in cell units, fl32(o / H)
};

// Per sky pixel: the ray step in cell units g = fl32(u dr / H), u = (cos d cos a, cos d sin a,
// sin d), and the sky value in Q32 (rint(v 2^32)); a value outside [0, 1] sets the error flag.
__global__ void __launch_bounds__(256)
k_mask_pix(const double* __restrict__ sky, const double* __restrict__ ca, const double* __restrict__ sa,
           const double* __restrict__ cd, const double* __restrict__ sd, int n_alpha, long long npix, double step,
           float4* __restrict__ pix, unsigned long long* __restrict__ qsky, int* __restrict__ err) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % n_alpha), j = (int)(p / n_alpha);
    const double v = sky[p];
    unsigned long long q = 0;
    if (v >= 0.0 && v <= 1.0) q = __double2ull_rn(__dmul_rn(v, 4294967296.0));
    else atomicOr(err, 1);
    qsky[p] = q;
    pix[p] = make_float4(__double2float_rn(__dmul_rn(__dmul_rn(cd[j], ca[i]), step)),
                         __double2float_rn(__dmul_rn(__dmul_rn(cd[j], sa[i]), step)),
                         __double2float_rn(__dmul_rn(sd[j], step)), 0.0f);
  }
}

// One warp per (pixel, 32 consecutive radial samples).  The cell of sample k is decided in FP32 in
// cell units, X = O + (k + 1/2) g, each operation rounded once.  A ray never re-enters a cell it
// left, so equal cells form runs of neighbouring lanes; the last lane of a run adds the run's sums
// (Q32 sky value x run length, Q32 radial values, count) with one atomic each.
__global__ void __launch_bounds__(256)
k_project_mask(const float4* __restrict__ pix, const unsigned long long* __restrict__ qsky,
               const unsigned long long* __restrict__ qr, MaskArgs a, unsigned long long* __restrict__ ss,
               unsigned long long* __restrict__ sr, unsigned long long* __restrict__ cnt) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long ntask = a.npix * a.kc;
  const float nf = (float)a.n;
  for (long long t = warp; t < ntask; t += nwarp) {  // warp-uniform loop
    const long long p = t / a.kc;
    const int k = (int)(t - p * a.kc) * 32 + lane;
    const float4 g = pix[p];
    bool valid = k < a.n_r;
    unsigned long long key = ~0ull, qv = 0;
    if (valid) {
      const float tk = __fadd_rn((float)k, 0.5f);
      const float fx = floorf(__fadd_rn(a.ox, __fmul_rn(tk, g.x)));
      const float fy = floorf(__fadd_rn(a.oy, __fmul_rn(tk, g.y)));
      const float fz = floorf(__fadd_rn(a.oz, __fmul_rn(tk, g.z)));
      valid = fx >= 0.0f && fx < nf && fy >= 0.0f && fy < nf && fz >= 0.0f && fz < nf;
      if (valid) {
        key = ((unsigned long long)(unsigned)fx * a.n + (unsigned)fy) * a.n + (unsigned)fz;
        qv = qr[k];
      }
    }
    // runs of equal keys: heads, the run start of each lane, and the tails
    const unsigned long long prev = __shfl_up_sync(FULL, key, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0 || prev != key);
    const int start = 31 - __clz(heads & (FULL >> (31 - lane)));
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    // inclusive prefix sum of the radial values across the warp
    unsigned long long pre = qv;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(FULL, pre, d);
      if (lane >= d) pre += o;
    }
    const unsigned long long before = __shfl_sync(FULL, pre, start > 0 ? start - 1 : 0);
    if (valid && tail) {
      const unsigned long long len = (unsigned long long)(lane - start + 1);
      atomicAdd(ss + key, qsky[p] * len);
      atomicAdd(sr + key, start > 0 ? pre - before : pre);
      atomicAdd(cnt + key, len);
    }
  }
}

// w = (S_sky 2^-32 rc) (S_r 2^-32 rc) with rc = fl(1 / count), 0 where no sample fell; rc from
// the host table rtab for count < kMaskRcp, else the correctly rounded reciprocal
constexpr int kMaskRcp = 4096;
__global__ void __launch_bounds__(256)
k_mask_finish(const unsigned long long* __restrict__ ss, const unsigned long long* __restrict__ sr,
              const unsigned long long* __restrict__ cnt, const double* __restrict__ rtab, size_t V,
              double* __restrict__ w, long long* __restrict__ counts) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < V; c += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long nc = cnt[c];
    double v = 0.0;
    if (nc) {
      const double rc = nc < (unsigned long long)kMaskRcp ? rtab[nc] : __drcp_rn(__ull2double_rn(nc));
      v = __dmul_rn(__dmul_rn(__dmul_rn(__ull2double_rn(ss[c]), 0x1p-32), rc),
                    __dmul_rn(__dmul_rn(__ull2double_rn(sr[c]), 0x1p-32), rc));
    }
    w[c] = v;
    if (counts) counts[c] = (long long)nc;
  }
}

wf_status project_mask_run(Ctx& c, const wf_grid& g, const double* sky, int n_alpha, int n_delta, double alpha0,
                           double dalpha, double delta0, double ddelta, const double* obs, double dr, int n_r,
                           const double* wr, double* w, int64_t* counts, cudaStream_t st) {
  if (!sky || !obs || !wr || !w || n_alpha <= 0 || n_delta <= 0 || n_r <= 0 || !(dr > 0.0) || !std::isfinite(dr) ||
      !std::isfinite(alpha0) || !std::isfinite(dalpha) || !std::isfinite(delta0) || !std::isfinite(ddelta) ||
      !std::isfinite(obs[0]) || !std::isfinite(obs[1]) || !std::isfinite(obs[2]))
    return WF_ERR_ARG;
  for (int k = 0; k < n_r; ++k)
    if (!(wr[k] >= 0.0 && wr[k] <= 1.0)) return WF_ERR_ARG;
  // pixel-centre cosines and sines (libm on the host, as the definition takes them) and the radial
  // values in Q32
  const size_t nd = (size_t)2 * n_alpha + 2 * n_delta;
  std::vector<double> h(nd + n_r + kMaskRcp);
  double *ca = h.data(), *sa = ca + n_alpha, *cd = sa + n_alpha, *sd = cd + n_delta;
  unsigned long long* qr = reinterpret_cast<unsigned long long*>(sd + n_delta);
  for (int i = 0; i < n_alpha; ++i) {
    const double al = alpha0 + ((double)i + 0.5) * dalpha;
    ca[i] = std::cos(al);
    sa[i] = std::sin(al);
  }
  for (int j = 0; j < n_delta; ++j) {
    const double de = delta0 + ((double)j + 0.5) * ddelta;
    cd[j] = std::cos(de);
    sd[j] = std::sin(de);
  }
  for (int k = 0; k < n_r; ++k) qr[k] = (unsigned long long)std::nearbyint(wr[k] * 4294967296.0);
  double* rtab = h.data() + nd + n_r;
  rtab[0] = 0.0;
  for (int m = 1; m < kMaskRcp; ++m) rtab[m] = 1.0 / (double)m;
  const size_t V = (size_t)g.n * g.n * g.n;
  const long long npix = (long long)n_alpha * n_delta;
  const double H = g.box / (double)g.n;
  double* dtab;
  float4* pix;
  unsigned long long *qsky, *acc;
  int* err;
  WF_TRY(c.get("mask_tab", h.size() * sizeof(double), (void**)&dtab));
  WF_TRY(c.get("mask_pix", (size_t)npix * sizeof(float4), (void**)&pix));
  WF_TRY(c.get("mask_qsky", (size_t)npix * sizeof(unsigned long long), (void**)&qsky));
  WF_TRY(c.get("mask_acc", 3 * V * sizeof(unsigned long long), (void**)&acc));
  WF_TRY(c.get("mask_err", 64, (void**)&err));
  WF_CUDA(cudaMemcpyAsync(dtab, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  WF_CUDA(cudaMemsetAsync(acc, 0, 3 * V * sizeof(unsigned long long), st));
  WF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const double* dca = dtab;
  const double* dsa = dca + n_alpha;
  const double* dcd = dsa + n_alpha;
  const double* dsd = dcd + n_delta;
  const unsigned long long* dqr = reinterpret_cast<const unsigned long long*>(dsd + n_delta);
  const double* drtab = dtab + nd + n_r;
  const double step = dr / H;
  const unsigned pgrid = (unsigned)std::min<long long>((npix + 255) / 256, 152 * 8);
  c.launch("mask_pix", 56.0 * (double)npix, st,
           [&] { k_mask_pix<<<pgrid, 256, 0, st>>>(sky, dca, dsa, dcd, dsd, n_alpha, npix, step, pix, qsky, err); });
  MaskArgs a{g.n, n_r, (n_r + 31) / 32, npix, step, (float)(obs[0] / H), (float)(obs[1] / H), (float)(obs[2] / H)};
  const double samples = (double)npix * n_r;
  c.launch("project_mask", 8.0 * samples, st, [&] {
    k_project_mask<<<152 * 16, 256, 0, st>>>(pix, qsky, dqr, a, acc, acc + V, acc + 2 * V);
  });
  c.launch("mask_finish", 32.0 * (double)V, st, [&] {
    k_mask_finish<<<152 * 4, 256, 0, st>>>(acc, acc + V, acc + 2 * V, drtab, V, w,
                                           reinterpret_cast<long long*>(counts));
  });
  WF_CUDA(cudaGetLastError());
  int* hp = reinterpret_cast<int*>(c.host_pinned);
  WF_CUDA(cudaMemcpyAsync(hp, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));  // also keeps h alive until the copy is done
  return hp[0] ? WF_ERR_ARG : WF_OK;
}

wf_status selection_at_run(Ctx& c, const wf_selection& sel, const double* pos, int64_t n_pts, bool reciprocal,
                          double* w, cudaStream_t st) {
  if (n_pts < 0 || (n_pts > 0 && (!pos || !w)) || sel.n_holes < 0 || (sel.n_holes > 0 && !sel.holes) ||
      sel.radial_kind < 0 || sel.radial_kind > 2)
    return WF_ERR_ARG;
  if (sel.radial_kind > 0 && !(sel.radial_params[0] > 0.0)) return WF_ERR_ARG;
  if (n_pts == 0) return WF_OK;
  SelParams s;
  s.ox = sel.observer[0];
  s.oy = sel.observer[1];
  s.oz = sel.observer[2];
  s.ax = sel.axis[0];
  s.ay = sel.axis[1];
  s.az = sel.axis[2];
  s.cos_half = cos(sel.half_angle);
  s.H = 0.0;
  s.p0 = sel.radial_params[0];
  s.p1 = sel.radial_params[1];
  s.kind = sel.radial_kind;
  s.n_holes = sel.n_holes;
  std::vector<double4> hh((size_t)(sel.n_holes > 0 ? sel.n_holes : 1));
  for (int h = 0; h < sel.n_holes; ++h)
    hh[h] = make_double4(sel.holes[4 * h], sel.holes[4 * h + 1], sel.holes[4 * h + 2], cos(sel.holes[4 * h + 3]));
  double4* dh;
  WF_TRY(c.get("holes_at", hh.size() * sizeof(double4), (void**)&dh));
  WF_CUDA(cudaMemcpyAsync(dh, hh.data(), hh.size() * sizeof(double4), cudaMemcpyHostToDevice, st));
  const unsigned grid = (unsigned)std::min<int64_t>((n_pts + 255) / 256, 152 * 16);
  c.launch("window_at", 32.0 * (double)n_pts, st, [&] { k_window_at<<<grid, 256, 0, st>>>(pos, (long long)n_pts, s, dh, reciprocal, w); });
  WF_CUDA(cudaGetLastError());
  // the host copy of the hole table must outlive the copy
  WF_CUDA(cudaStreamSynchronize(st));
  return WF_OK;
}

wf_status noise_run(Ctx& c, const wf_grid& g, const wf_selection& sel, const double* n_obs, int64_t n_gal,
                    double* w, double* d, double* b, double* nbar, cudaStream_t st) {
  const int n = g.n;
  if (!supported_size(n)) return WF_ERR_UNSUPPORTED;
  if (!(g.box > 0.0) || !n_obs || !w || !b || !nbar || n_gal <= 0 || sel.n_holes < 0 ||
      (sel.n_holes > 0 && !sel.holes) || sel.radial_kind < 0 || sel.radial_kind > 2)
    return WF_ERR_ARG;
  if (sel.radial_kind > 0 && !(sel.radial_params[0] > 0.0)) return WF_ERR_ARG;
  SelParams s;
  s.ox = sel.observer[0];
  s.oy = sel.observer[1];
  s.oz = sel.observer[2];
  s.ax = sel.axis[0];
  s.ay = sel.axis[1];
  s.az = sel.axis[2];
  s.cos_half = cos(sel.half_angle);
  s.H = g.box / (double)n;
  s.p0 = sel.radial_params[0];
  s.p1 = sel.radial_params[1];
  s.kind = sel.radial_kind;
  s.n_holes = sel.n_holes;
  std::vector<double4> hh((size_t)(sel.n_holes > 0 ? sel.n_holes : 1));
  for (int h = 0; h < sel.n_holes; ++h)
    hh[h] = make_double4(sel.holes[4 * h], sel.holes[4 * h + 1], sel.holes[4 * h + 2], cos(sel.holes[4 * h + 3]));
  double4* dh;
  WF_TRY(c.get("holes", hh.size() * sizeof(double4), (void**)&dh));
  WF_CUDA(cudaMemcpyAsync(dh, hh.data(), hh.size() * sizeof(double4), cudaMemcpyHostToDevice, st));
  const int grid = 152 * 8;
  double *part, *scal;
  WF_TRY(c.get("noise_part", grid * sizeof(double), (void**)&part));
  WF_TRY(c.get("noise_scal", 4 * sizeof(double), (void**)&scal));
  const size_t V = (size_t)n * n * n;
  c.launch("window", 8.0 * V, st, [&] { k_window<<<grid, 256, 0, st>>>(n, s, dh, w, part); });
  WF_CUDA(cudaGetLastError());
  c.launch("fin", 0, st, [&] { k_nbar<<<1, 1024, 0, st>>>(part, grid, (double)n_gal, scal); });
  WF_CUDA(cudaGetLastError());
  c.launch("data", 8.0 * V * (d ? 4 : 3), st, [&] { k_data<<<grid, 256, 0, st>>>(n_obs, w, scal, d, b, V); });
  WF_CUDA(cudaGetLastError());
  double* h = reinterpret_cast<double*>(c.host_pinned);
  WF_CUDA(cudaMemcpyAsync(h, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (!(h[0] > 0.0)) return WF_ERR_ARG;
  *nbar = h[1];
  return WF_OK;
}

}  // namespace wf

// ==========================================================================================
// wf_build_noise_noalloc: the same window / nbar / data computation for callers that must not
// allocate device memory.  Some embedders cannot let a library call cudaMalloc: a simulation
// code that owns the whole device through its own pool and runs at its memory limit, or a
// real-time pipeline where cudaMalloc's implicit device synchronisation would stall other
// streams.  This variant takes only the caller's buffers; its scratch (per-block partial sums
// of w, the nbar scalars, the hole table) is a fixed array in the library's device image,
// which every GPU that loads the library holds until the process exits.
// ==========================================================================================
namespace wf {

constexpr int kNoallocParts = 152 * 8;   // blocks of the window kernel = partial sums
constexpr int kNoallocMaxHoles = 256;    // largest hole table the scratch can hold
// layout (doubles): [0, kNoallocParts) partials | 4 scalars | 4 * kNoallocMaxHoles hole rows
constexpr int kNoallocDoubles = kNoallocParts + 4 + 4 * kNoallocMaxHoles;  // 2244 doubles
constexpr size_t kNoallocBytes = sizeof(double) * kNoallocDoubles;           // 17,952 bytes

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];
static_assert(sizeof(g_noalloc_scratch) == 17952, "the header states the scratch size");
static_assert(kNoallocBytes == 17952, "the header states the scratch size");

// Device addresses of g_noalloc_scratch, looked up once per (device, context) -- host code must
// not use the symbol itself: on the host it is only a stand-in, not a device address.  The key
// includes the driver's unique context id, so a context created after cudaDeviceReset (whose
// copy of the array may sit elsewhere) gets its own lookup instead of a stale address.
static std::mutex g_noalloc_mu;
static std::map<std::pair<int, unsigned long long>, double*> g_noalloc_addr;

// The current context's unique id (0 if the driver cannot tell), through the runtime's driver
// entry points, so the library does not link libcuda itself.
static unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (PFN_cuCtxGetCurrent_v4000)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (PFN_cuCtxGetId_v12000)f;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx) get_id(ctx, &id);
  return id;
}

static wf_status noalloc_scratch(int device, double** out) {
  // (before the runtime's first call on this device there is no context yet: id 0, and the
  // next call, with the context made, looks the address up once more)
  const std::pair<int, unsigned long long> key(device, current_context_id());
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_addr.find(key);
  if (it != g_noalloc_addr.end()) {
    *out = it->second;
    return WF_OK;
  }
  double* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_last_error("cudaGetSymbolAddress(g_noalloc_scratch)", e);
    return WF_ERR_CUDA;
  }
  g_noalloc_addr[key] = p;
  *out = p;
  return WF_OK;
}

}  // namespace wf

extern "C" wf_status wf_build_noise_noalloc(const wf_grid* grid, const wf_selection* sel, const double* n_obs,
                                            int64_t n_gal, double* w, double* d, double* b, double* nbar,
                                            void* stream) {
  using namespace wf;
  if (!grid || !sel) return WF_ERR_ARG;
  const int n = grid->n;
  if (!supported_size(n)) return WF_ERR_UNSUPPORTED;
  if (!(grid->box > 0.0) || !n_obs || !w || !b || !nbar || n_gal <= 0 || sel->n_holes < 0 ||
      (sel->n_holes > 0 && !sel->holes) || sel->radial_kind < 0 || sel->radial_kind > 2)
    return WF_ERR_ARG;
  if (sel->radial_kind > 0 && !(sel->radial_params[0] > 0.0)) return WF_ERR_ARG;
  if (sel->n_holes > kNoallocMaxHoles) {
    set_last_error("wf_build_noise_noalloc: more than 256 holes do not fit the fixed scratch", cudaSuccess);
    return WF_ERR_ARG;
  }
  int dev = 0;
  WF_CUDA(cudaGetDevice(&dev));
  double* scratch = nullptr;
  WF_TRY(noalloc_scratch(dev, &scratch));
  double* part = scratch;
  double* scal = scratch + kNoallocParts;
  double4* dh = reinterpret_cast<double4*>(scratch + kNoallocParts + 4);
  cudaStream_t st = (cudaStream_t)stream;
  SelParams s;
  s.ox = sel->observer[0];
  s.oy = sel->observer[1];
  s.oz = sel->observer[2];
  s.ax = sel->axis[0];
  s.ay = sel->axis[1];
  s.az = sel->axis[2];
  s.cos_half = cos(sel->half_angle);
  s.H = grid->box / (double)n;
  s.p0 = sel->radial_params[0];
  s.p1 = sel->radial_params[1];
  s.kind = sel->radial_kind;
  s.n_holes = sel->n_holes;
  double4 hh[kNoallocMaxHoles];
  for (int h = 0; h < sel->n_holes; ++h)
    hh[h] = make_double4(sel->holes[4 * h], sel->holes[4 * h + 1], sel->holes[4 * h + 2], cos(sel->holes[4 * h + 3]));
  if (sel->n_holes > 0)
    WF_CUDA(cudaMemcpyAsync(dh, hh, sizeof(double4) * sel->n_holes, cudaMemcpyHostToDevice, st));
  // every partial and scalar below is written before it is read: nothing in the scratch
  // needs clearing between calls
  const size_t V = (size_t)n * n * n;
  k_window<<<kNoallocParts, 256, 0, st>>>(n, s, dh, w, part);
  WF_CUDA(cudaGetLastError());
  k_nbar<<<1, 1024, 0, st>>>(part, kNoallocParts, (double)n_gal, scal);
  WF_CUDA(cudaGetLastError());
  k_data<<<kNoallocParts, 256, 0, st>>>(n_obs, w, scal, d, b, V);
  WF_CUDA(cudaGetLastError());
  double h3[3];
  WF_CUDA(cudaMemcpyAsync(h3, scal, sizeof(h3), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  if (!(h3[0] > 0.0)) return WF_ERR_ARG;
  *nbar = h3[1];
  return WF_OK;
}
