/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the Wiener-reconstruction hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path calls this file: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * What it computes (Kitaura et al. 2009, "Cosmic cartography of the large-scale
 * structure with SDSS DR6", arXiv:0906.3978):
 *   - supersampled gridding, step 1 (Sec. 3.1.2 "Supersampling step", Eq. def:ngrid):
 *     CIC / TSC assignment of point galaxies onto a grid s times finer than the target,
 *     in a fixed-point rule (Q16 per axis, Q48 per galaxy) so the fine grid is exact;
 *   - supersampled gridding, step 2 (Sec. 3.1.2): the ideal discrete low-pass filter on the
 *     fine grid, then sampling at the target grid;
 *   - the 3D window w (Sec. 3.1.3 "Calculation of the three-dimensional mask"), here
 *     an analytic cone x holes x radial law evaluated at the nodes;
 *   - the data and noise model (Sec. 3.2, Eqs. eq:datamodel, eq:nmean, eq:noiseav):
 *     nbar = N_gal / sum(w), d = n_obs/nbar - w, N = w/nbar, R = diag(w);
 *   - the signal-space Wiener filter (Sec. 3.3.1, Eq. eq:WF), i.e. the linear system
 *     (S^-1 + R^T N^-1 R) s = R^T N^-1 d with S diagonal in Fourier space, solved by
 *     textbook conjugate gradients (the paper names a Krylov-space inversion, Sec. 1).
 *
 * Every transform is a plain complex DFT done by the textbook recursive mixed-radix
 * Cooley-Tukey algorithm below; real fields are carried as complex arrays with zero
 * imaginary part.  No real-to-complex packing, no fusion, no blocking.
 *
 * Conventions: grids are cubic, N cells per axis, row-major [x][y][z] (z fastest); node
 * i sits at i*H with H = L/N; forward DFT X_k = sum_j x_j exp(-2 pi i j.k/N), inverse
 * without normalisation; frequencies are taken with signed indices in (-N/2, N/2].
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC oracle.c -lm.  Floating-point
 * contraction is switched off so that every decision taken in floating point (cone and
 * hole membership, floor of positions) follows the plain IEEE operation order written here.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum {
  OR_OK = 0,
  OR_ERR_ARG = -1,
  OR_ERR_OOM = -2,
  OR_ERR_NOT_CONVERGED = -4,
  OR_ERR_BREAKDOWN = -5,
  OR_ERR_OVERFLOW = -7
};

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------ */
/* 1. Fixed-point mass assignment (Sec. 3.1.2, Eq. def:ngrid; CIC/TSC kernels named there) */
/* ------------------------------------------------------------------------------------ */

/* Per-axis nodes and Q16 weights of one galaxy coordinate.
 * u = x * (Nf * 2^16 / L) is rounded down to an integer q (one FP64 multiply, then
 * floor) and wrapped into [0, Nf*2^16).  q/2^16 is the position in fine-cell units.
 * CIC: nodes (i, i+1) with weights (2^16 - f, f), i = q >> 16, f = q & 0xFFFF.
 * TSC: j = round(u), D = offset from node j in Q16 in [-2^15, 2^15); the quadratic
 * spline weights (1/2)(1/2 -+ d)^2 are floored in Q16 and the centre weight takes the
 * remainder so the three weights sum to exactly 2^16.
 * Returns the number of nodes (2 or 3), or -1 for a non-finite / out-of-range value. */
static int axis_weights(double x, double scale, int64_t nf, int scheme, int64_t node[3],
                        uint64_t wt[3]) {
  double u = x * scale;
  if (!(fabs(u) < 4503599627370496.0)) return -1; /* 2^52: floor must stay exact */
  int64_t m = nf * 65536;
  int64_t q = (int64_t)floor(u);
  q %= m;
  if (q < 0) q += m;
  if (scheme == 1) { /* CIC */
    int64_t i = q >> 16;
    uint64_t f = (uint64_t)(q & 0xFFFF);
    node[0] = i % nf;
    node[1] = (i + 1) % nf;
    wt[0] = 65536u - f;
    wt[1] = f;
    return 2;
  }
  /* TSC */
  int64_t qp = q + 32768;
  int64_t j = qp >> 16;
  int64_t D = (qp & 0xFFFF) - 32768; /* in [-2^15, 2^15) */
  uint64_t a = (uint64_t)(32768 - D), b = (uint64_t)(32768 + D);
  uint64_t wm = (a * a) >> 17, wp = (b * b) >> 17;
  node[0] = ((j - 1) % nf + nf) % nf;
  node[1] = j % nf;
  node[2] = (j + 1) % nf;
  wt[0] = wm;
  wt[1] = 65536u - wm - wp;
  wt[2] = wp;
  return 3;
}

/* fine[(Nf)^3], Nf = ss*n, is overwritten with the Q48 mass of the galaxies.
 * scheme: 1 = CIC, 2 = TSC.  Returns OR_ERR_OVERFLOW if a cell would exceed 2^64-1. */
int oracle_assign(int n, double box, int ss, int scheme, const double* pos, int64_t n_gal,
                  uint64_t* fine) {
  if (n <= 0 || ss < 1 || !(box > 0) || (scheme != 1 && scheme != 2) || n_gal < 0)
    return OR_ERR_ARG;
  int64_t nf = (int64_t)ss * n;
  size_t nfine = (size_t)nf * nf * nf;
  memset(fine, 0, nfine * sizeof(uint64_t));
  double scale = ((double)nf * 65536.0) / box;
  int overflow = 0;
  for (int64_t g = 0; g < n_gal; ++g) {
    int64_t nd[3][3];
    uint64_t wt[3][3];
    int cnt = 0;
    for (int a = 0; a < 3; ++a) {
      cnt = axis_weights(pos[3 * g + a], scale, nf, scheme, nd[a], wt[a]);
      if (cnt < 0) return OR_ERR_ARG;
    }
    for (int i = 0; i < cnt; ++i)
      for (int j = 0; j < cnt; ++j)
        for (int k = 0; k < cnt; ++k) {
          uint64_t add = wt[0][i] * wt[1][j] * wt[2][k];
          size_t idx = ((size_t)nd[0][i] * nf + (size_t)nd[1][j]) * nf + (size_t)nd[2][k];
          uint64_t old = fine[idx];
          fine[idx] = old + add;
          if (fine[idx] < old) overflow = 1;
        }
  }
  return overflow ? OR_ERR_OVERFLOW : OR_OK;
}

/* Weighted assignment for the inverse-weighting estimator (Sec. 4, Eq. def:ngrid with the
 * galaxy mass 1/w): galaxy g carries weight wgt[g] >= 0.  Each node's contribution is its Q48
 * fixed-point weight (as in oracle_assign) times wgt[g], rounded once to the nearest Q32 unit:
 * rint(double(q48) * wgt[g] * 2^-16).  The grid is then exact and independent of the order of
 * the galaxies; a cell holds fine[i] * 2^-32 weighted galaxies. */
int oracle_assign_weighted(int n, double box, int ss, int scheme, const double* pos, const double* wgt,
                           int64_t n_gal, uint64_t* fine) {
  if (n <= 0 || ss < 1 || !(box > 0) || (scheme != 1 && scheme != 2) || n_gal < 0) return OR_ERR_ARG;
  int64_t nf = (int64_t)ss * n;
  size_t nfine = (size_t)nf * nf * nf;
  memset(fine, 0, nfine * sizeof(uint64_t));
  double scale = ((double)nf * 65536.0) / box;
  int overflow = 0;
  for (int64_t g = 0; g < n_gal; ++g) {
    if (!(wgt[g] >= 0.0) || !(wgt[g] < 4294967296.0)) return OR_ERR_ARG; /* < 2^32 */
    int64_t nd[3][3];
    uint64_t wt[3][3];
    int cnt = 0;
    for (int a = 0; a < 3; ++a) {
      cnt = axis_weights(pos[3 * g + a], scale, nf, scheme, nd[a], wt[a]);
      if (cnt < 0) return OR_ERR_ARG;
    }
    for (int i = 0; i < cnt; ++i)
      for (int j = 0; j < cnt; ++j)
        for (int k = 0; k < cnt; ++k) {
          double q = (double)(wt[0][i] * wt[1][j] * wt[2][k]);
          uint64_t add = (uint64_t)rint(q * wgt[g] * (1.0 / 65536.0));
          size_t idx = ((size_t)nd[0][i] * nf + (size_t)nd[1][j]) * nf + (size_t)nd[2][k];
          uint64_t old = fine[idx];
          fine[idx] = old + add;
          if (fine[idx] < old) overflow = 1;
        }
  }
  return overflow ? OR_ERR_OVERFLOW : OR_OK;
}

/* ------------------------------------------------------------------------------------ */
/* 2. Plain complex DFT: recursive decimation in time, radix = smallest prime factor    */
/* ------------------------------------------------------------------------------------ */

static size_t smallest_factor(size_t n) {
  for (size_t p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

/* out[k] = sum_j in[j*stride] W^(j k), W = exp(sign 2 pi i / n).  tw[e] = exp(sign 2 pi i e / tw_n)
 * for the top-level length tw_n (a multiple of n). */
static void dft_rec(const cplx* in, size_t stride, cplx* out, size_t n, const cplx* tw,
                    size_t tw_n) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  size_t p = smallest_factor(n), m = n / p;
  for (size_t r = 0; r < p; ++r) dft_rec(in + r * stride, stride * p, out + r * m, m, tw, tw_n);
  size_t step = tw_n / n;
  cplx y[p];
  for (size_t k = 0; k < m; ++k) {
    for (size_t r = 0; r < p; ++r) y[r] = out[k + r * m] * tw[(r * k * step) % tw_n];
    for (size_t q = 0; q < p; ++q) {
      cplx acc = 0;
      for (size_t r = 0; r < p; ++r) acc += y[r] * tw[((r * q) % p) * m * step];
      out[k + q * m] = acc;
    }
  }
}

static cplx* make_twiddles(size_t n, int sign) {
  cplx* tw = (cplx*)malloc(n * sizeof(cplx));
  if (!tw) return NULL;
  for (size_t e = 0; e < n; ++e) {
    double ang = 2.0 * OR_PI * (double)e / (double)n;
    tw[e] = cos(ang) + I * (sign * sin(ang));
  }
  return tw;
}

/* In-place unnormalised 1D DFT of a contiguous complex array of length n. */
int oracle_fft1d(cplx* a, int n, int sign) {
  cplx* tw = make_twiddles((size_t)n, sign);
  cplx* tmp = (cplx*)malloc((size_t)n * sizeof(cplx));
  if (!tw || !tmp) {
    free(tw);
    free(tmp);
    return OR_ERR_OOM;
  }
  dft_rec(a, 1, tmp, (size_t)n, tw, (size_t)n);
  memcpy(a, tmp, (size_t)n * sizeof(cplx));
  free(tw);
  free(tmp);
  return OR_OK;
}

/* In-place unnormalised 3D DFT of an n^3 complex array: 1D DFTs along z, then y, then x. */
int oracle_fft3d(cplx* a, int n, int sign) {
  size_t N = (size_t)n;
  cplx* tw = make_twiddles(N, sign);
  if (!tw) return OR_ERR_OOM;
  int err = 0;
  for (int axis = 0; axis < 3; ++axis) {
    size_t stride = axis == 0 ? 1 : (axis == 1 ? N : N * N);
#pragma omp parallel
    {
      cplx* line = (cplx*)malloc(N * sizeof(cplx));
      cplx* res = (cplx*)malloc(N * sizeof(cplx));
      if (!line || !res) {
#pragma omp atomic write
        err = 1;
      } else {
#pragma omp for schedule(static)
        for (long long l = 0; l < (long long)(N * N); ++l) {
          /* the line index l enumerates the two other coordinates */
          size_t base;
          if (axis == 0)
            base = (size_t)l * N;
          else if (axis == 1)
            base = ((size_t)l / N) * N * N + ((size_t)l % N);
          else
            base = (size_t)l;
          for (size_t j = 0; j < N; ++j) line[j] = a[base + j * stride];
          dft_rec(line, 1, res, N, tw, N);
          for (size_t j = 0; j < N; ++j) a[base + j * stride] = res[j];
        }
      }
      free(line);
      free(res);
    }
  }
  free(tw);
  return err ? OR_ERR_OOM : OR_OK;
}

/* ------------------------------------------------------------------------------------ */
/* 3. Ideal low-pass + downsample (Sec. 3.1.2, supersampling step 2)                       */
/* ------------------------------------------------------------------------------------ */

/* signed frequency of index j on an axis of length n; the Nyquist index n/2 maps to n/2 */
static long sfreq(long j, long n) { return j <= n / 2 ? j : j - n; }

/* n_obs[n^3] from the fine Q48 grid (ss*n)^3.
 * ss == 1: n_obs = fine / 2^48 (plain gridding).
 * ss >= 2: F = DFT of fine/2^48 on the fine grid; keep the modes whose three signed
 * coarse indices satisfy |k| < n/2 (the coarse Nyquist planes are dropped, which keeps
 * the result real and alias-free); place them in an n^3 spectrum and return
 * (1/n^3) * inverse DFT.  The k = 0 mode is kept, so sum(n_obs) = sum(fine)/2^48. */
int oracle_lowpass_scaled(int n, int ss, const uint64_t* fine, double unit, double* n_obs);
int oracle_lowpass(int n, int ss, const uint64_t* fine, double* n_obs) {
  return oracle_lowpass_scaled(n, ss, fine, 1.0 / 281474976710656.0 /* 2^-48 */, n_obs);
}
/* The same for a fine grid in other fixed-point units: a cell holds fine[i] * unit galaxies
 * (2^-48 for oracle_assign, 2^-32 for oracle_assign_weighted). */
int oracle_lowpass_scaled(int n, int ss, const uint64_t* fine, double unit, double* n_obs) {
  if (n <= 0 || ss < 1 || (n % 2) != 0) return OR_ERR_ARG;
  size_t N = (size_t)n, V = N * N * N;
  const double q48 = unit;
  if (ss == 1) {
    for (size_t i = 0; i < V; ++i) n_obs[i] = (double)fine[i] * q48;
    return OR_OK;
  }
  size_t NF = (size_t)ss * N, VF = NF * NF * NF;
  cplx* F = (cplx*)malloc(VF * sizeof(cplx));
  cplx* C = (cplx*)malloc(V * sizeof(cplx));
  if (!F || !C) {
    free(F);
    free(C);
    return OR_ERR_OOM;
  }
  for (size_t i = 0; i < VF; ++i) F[i] = (double)fine[i] * q48;
  int st = oracle_fft3d(F, (int)NF, -1);
  if (st == OR_OK) {
    for (size_t jx = 0; jx < N; ++jx)
      for (size_t jy = 0; jy < N; ++jy)
        for (size_t jz = 0; jz < N; ++jz) {
          size_t c = (jx * N + jy) * N + jz;
          if (jx == N / 2 || jy == N / 2 || jz == N / 2) {
            C[c] = 0;
            continue;
          }
          long kx = sfreq((long)jx, (long)N), ky = sfreq((long)jy, (long)N),
               kz = sfreq((long)jz, (long)N);
          size_t fx = (size_t)((kx + (long)NF) % (long)NF), fy = (size_t)((ky + (long)NF) % (long)NF),
                 fz = (size_t)((kz + (long)NF) % (long)NF);
          C[c] = F[(fx * NF + fy) * NF + fz];
        }
    st = oracle_fft3d(C, n, +1);
    if (st == OR_OK)
      for (size_t i = 0; i < V; ++i) n_obs[i] = creal(C[i]) / (double)V;
  }
  free(F);
  free(C);
  return st;
}

/* The same low-pass written as the direct sum over the (sparse) fine grid for one output
 * node: n_obs[j] = sum_i fine_i/2^48 * prod_axes D(ss*j_a - i_a), with
 * D(m) = (1/n) sum_{|k|<n/2} exp(2 pi i k m /(ss*n)).  Used to check sampled outputs of
 * large grids one by one. */
double oracle_lowpass_point(int n, int ss, const uint64_t* fine, int jx, int jy, int jz) {
  size_t N = (size_t)n, NF = (size_t)ss * N;
  const double q48 = 1.0 / 281474976710656.0;
  double* D = (double*)malloc(NF * sizeof(double));
  if (!D) return NAN;
  for (size_t m = 0; m < NF; ++m) {
    double acc = 1.0;
    for (long k = 1; k < n / 2; ++k) acc += 2.0 * cos(2.0 * OR_PI * (double)k * (double)m / (double)NF);
    D[m] = acc / (double)n;
  }
  double sum = 0.0;
  long j[3] = {jx, jy, jz};
  for (size_t ix = 0; ix < NF; ++ix)
    for (size_t iy = 0; iy < NF; ++iy)
      for (size_t iz = 0; iz < NF; ++iz) {
        uint64_t f = fine[(ix * NF + iy) * NF + iz];
        if (!f) continue;
        size_t mx = (size_t)((((long)ss * j[0] - (long)ix) % (long)NF + (long)NF) % (long)NF);
        size_t my = (size_t)((((long)ss * j[1] - (long)iy) % (long)NF + (long)NF) % (long)NF);
        size_t mz = (size_t)((((long)ss * j[2] - (long)iz) % (long)NF + (long)NF) % (long)NF);
        sum += (double)f * q48 * D[mx] * D[my] * D[mz];
      }
  free(D);
  return sum;
}

/* ------------------------------------------------------------------------------------ */
/* 4. Window w at the nodes (Sec. 3.1.3; w <= 1)                                            */
/* ------------------------------------------------------------------------------------ */

/* w(x) = [angle(x - o, axis) <= half_angle] * prod_h [angle(x - o, h) >= rho_h] * f(r),
 * r = |x - o|, evaluated at node positions x = i*H (no periodic wrap), w = 0 at r = 0.
 * The membership tests compare dot products with cos(angle)*r, in the operation order
 * written here.  axis and the hole directions must be unit vectors.
 * holes[4*h] = (hx, hy, hz, rho_h).  radial_kind 0: f = 1; 1: f = exp(-(r/p0)^2);
 * 2: f = (r/p0)^p1 * exp(p1 * (1 - r/p0)) (peak 1 at r = p0). */
static double window_value(double dx, double dy, double dz, const double* axis, double cos_half,
                           int n_holes, const double* holes, const double* cos_h, int radial_kind,
                           const double* rp) {
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  double val = 0.0;
  if (r > 0.0) {
    int inside = (dx * axis[0] + dy * axis[1] + dz * axis[2]) >= cos_half * r;
    for (int h = 0; h < n_holes && inside; ++h) {
      const double* hv = holes + 4 * h;
      if ((dx * hv[0] + dy * hv[1] + dz * hv[2]) > cos_h[h] * r) inside = 0;
    }
    if (inside) {
      if (radial_kind == 0) {
        val = 1.0;
      } else if (radial_kind == 1) {
        double t = r / rp[0];
        val = exp(-(t * t));
      } else {
        double t = r / rp[0];
        val = pow(t, rp[1]) * exp(rp[1] * (1.0 - t));
      }
    }
  }
  return val;
}

/* The same selection at arbitrary positions pts[3 i] (the completeness at a galaxy, for the
 * inverse-weighting estimator of Sec. 4). */
int oracle_window_at(int64_t n_pts, const double* pts, const double* obs, const double* axis,
                     double half_angle, int n_holes, const double* holes, int radial_kind,
                     const double* rp, double* w) {
  if (n_pts < 0 || n_holes < 0 || radial_kind < 0 || radial_kind > 2) return OR_ERR_ARG;
  double cos_half = cos(half_angle);
  double* cos_h = (double*)malloc((size_t)(n_holes > 0 ? n_holes : 1) * sizeof(double));
  if (!cos_h) return OR_ERR_OOM;
  for (int h = 0; h < n_holes; ++h) cos_h[h] = cos(holes[4 * h + 3]);
  for (int64_t i = 0; i < n_pts; ++i)
    w[i] = window_value(pts[3 * i] - obs[0], pts[3 * i + 1] - obs[1], pts[3 * i + 2] - obs[2], axis, cos_half,
                        n_holes, holes, cos_h, radial_kind, rp);
  free(cos_h);
  return OR_OK;
}

int oracle_window(int n, double box, const double* obs, const double* axis, double half_angle,
                  int n_holes, const double* holes, int radial_kind, const double* rp,
                  double* w) {
  if (n <= 0 || !(box > 0) || n_holes < 0 || radial_kind < 0 || radial_kind > 2) return OR_ERR_ARG;
  double H = box / (double)n;
  double cos_half = cos(half_angle);
  double* cos_h = (double*)malloc((size_t)(n_holes > 0 ? n_holes : 1) * sizeof(double));
  if (!cos_h) return OR_ERR_OOM;
  for (int h = 0; h < n_holes; ++h) cos_h[h] = cos(holes[4 * h + 3]);
  size_t N = (size_t)n;
  for (size_t ix = 0; ix < N; ++ix)
    for (size_t iy = 0; iy < N; ++iy)
      for (size_t iz = 0; iz < N; ++iz) {
        double dx = (double)ix * H - obs[0];
        double dy = (double)iy * H - obs[1];
        double dz = (double)iz * H - obs[2];
        w[(ix * N + iy) * N + iz] =
            window_value(dx, dy, dz, axis, cos_half, n_holes, holes, cos_h, radial_kind, rp);
      }
  free(cos_h);
  return OR_OK;
}

/* Projection of a sky completeness map onto the grid (Sec. 3.1.3): sky pixel (i, j) of an
 * equidistant alpha x delta map has centre alpha_i = alpha0 + (i + 1/2) dalpha, delta_j =
 * delta0 + (j + 1/2) ddelta; its ray from the observer is sampled at r_k = (k + 1/2) dr, k < n_r,
 * at x = o + r_k u with u = (cos delta cos alpha, cos delta sin alpha, sin delta) (Eq. eq:transf);
 * each sample inside the box goes to its nearest-grid-point cell floor(x / H) (exact geometry in
 * FP64).  Per cell the sky values and the radial completeness values wr[k] of the samples are
 * summed in Q32 fixed point (rint(v 2^32), exact and order-independent) and counted; each
 * projection is normalised by the number of samples ("mask counts") and the two are multiplied:
 * w = (S_sky 2^-32 / count) * (S_r 2^-32 / count), 0 where no sample fell.  sky[j * n_alpha + i],
 * values in [0, 1]; counts may be NULL.
 * near (may be NULL) reports how close the decisions came to a cell face: with face_margin > 0, a
 * sample whose position x / H lies within face_margin (cell units) of a cell face on some axis adds
 * 1 to near[] at its own cell and at the cell across each such face (those inside the box).  A
 * computation of x / H with an error below face_margin can move only those samples, and only
 * between those cells. */
int oracle_project_mask(int n, double box, const double* sky, int n_alpha, int n_delta, double alpha0,
                        double dalpha, double delta0, double ddelta, const double* obs, double dr, int n_r,
                        const double* wr, double* w, int64_t* counts, double face_margin, int64_t* near) {
  if (n <= 0 || !(box > 0) || n_alpha <= 0 || n_delta <= 0 || !(dr > 0) || n_r <= 0) return OR_ERR_ARG;
  for (int k = 0; k < n_r; ++k)
    if (!(wr[k] >= 0.0 && wr[k] <= 1.0)) return OR_ERR_ARG;
  for (size_t p = 0; p < (size_t)n_alpha * n_delta; ++p)
    if (!(sky[p] >= 0.0 && sky[p] <= 1.0)) return OR_ERR_ARG;
  size_t V = (size_t)n * n * n;
  uint64_t* ss = (uint64_t*)calloc(V, sizeof(uint64_t));
  uint64_t* sr = (uint64_t*)calloc(V, sizeof(uint64_t));
  int64_t* cnt = (int64_t*)calloc(V, sizeof(int64_t));
  if (!ss || !sr || !cnt) {
    free(ss);
    free(sr);
    free(cnt);
    return OR_ERR_OOM;
  }
  if (near)
    for (size_t c = 0; c < V; ++c) near[c] = 0;
  const double H = box / (double)n, q32 = 4294967296.0;
  for (int j = 0; j < n_delta; ++j) {
    const double de = delta0 + ((double)j + 0.5) * ddelta;
    for (int i = 0; i < n_alpha; ++i) {
      const double v = sky[(size_t)j * n_alpha + i];
      const double al = alpha0 + ((double)i + 0.5) * dalpha;
      const double u[3] = {cos(de) * cos(al), cos(de) * sin(al), sin(de)};
      const uint64_t qs = (uint64_t)rint(v * q32);
      for (int k = 0; k < n_r; ++k) {
        const double r = ((double)k + 0.5) * dr;
        double X[3];
        long f[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
          X[a] = (obs[a] + r * u[a]) / H;
          const double fa = floor(X[a]);
          f[a] = (fa >= 0.0 && fa < (double)n) ? (long)fa : -1;
          if (f[a] < 0) inside = 0;
        }
        if (inside) {
          const size_t c = ((size_t)f[0] * n + (size_t)f[1]) * n + (size_t)f[2];
          ss[c] += qs;
          sr[c] += (uint64_t)rint(wr[k] * q32);
          cnt[c] += 1;
        }
        if (near && face_margin > 0.0) {
          /* the cell and its neighbours across every face within the margin */
          long lo[3], hi[3];
          int any = 0;
          for (int a = 0; a < 3; ++a) {
            const double fa = floor(X[a]);
            lo[a] = (long)fa;
            hi[a] = (long)fa;
            if (X[a] - fa < face_margin) { lo[a] -= 1; any = 1; }
            if (fa + 1.0 - X[a] < face_margin) { hi[a] += 1; any = 1; }
          }
          if (any)
            for (long ax = lo[0]; ax <= hi[0]; ++ax)
              for (long ay = lo[1]; ay <= hi[1]; ++ay)
                for (long az = lo[2]; az <= hi[2]; ++az)
                  if (ax >= 0 && ax < n && ay >= 0 && ay < n && az >= 0 && az < n)
                    near[((size_t)ax * n + (size_t)ay) * n + (size_t)az] += 1;
        }
      }
    }
  }
  for (size_t c = 0; c < V; ++c) {
    const double cn = (double)cnt[c];
    w[c] = cnt[c] ? ((double)ss[c] / q32 / cn) * ((double)sr[c] / q32 / cn) : 0.0;
    if (counts) counts[c] = cnt[c];
  }
  free(ss);
  free(sr);
  free(cnt);
  return OR_OK;
}

/* ------------------------------------------------------------------------------------ */
/* 5. Data and noise (Sec. 3.2: eq:datamodel, eq:nmean, eq:noiseav)                     */
/* ------------------------------------------------------------------------------------ */

/* nbar = N_gal / sum_i w_i (galaxies per cell; the fair-sample mean of eq:nmean with the
 * observed volume counted in cells); d = n_obs/nbar - w; b = R^T N^-1 d = nbar*d where
 * w > 0 and 0 where w = 0 (no data term in unobserved cells, Sec. 5.4 "Cluster prediction").
 * diag(R^T N^-1 R) = nbar*w is not stored: the solver forms it from w and nbar. */
int oracle_build_noise(int n, const double* n_obs, const double* w, int64_t n_gal, double* d,
                       double* b, double* nbar_out) {
  size_t V = (size_t)n * n * n;
  double sumw = 0.0;
  for (size_t i = 0; i < V; ++i) sumw += w[i];
  if (!(sumw > 0.0) || n_gal <= 0) return OR_ERR_ARG;
  double nbar = (double)n_gal / sumw;
  for (size_t i = 0; i < V; ++i) {
    d[i] = n_obs[i] / nbar - w[i];
    b[i] = w[i] > 0.0 ? nbar * d[i] : 0.0;
  }
  *nbar_out = nbar;
  return OR_OK;
}

/* ------------------------------------------------------------------------------------ */
/* 6. Prior S^-1 in Fourier space (Sec. 3.3.1: S-hat = (2 pi)^3 P(k) delta_D)            */
/* ------------------------------------------------------------------------------------ */

/* Power spectrum at k by log-log linear interpolation in the table (extrapolated with the
 * end segments outside it). */
static double pk_interp(double k, const double* pk_k, const double* pk_p, int n_pk) {
  int i = 0;
  while (i < n_pk - 2 && k > pk_k[i + 1]) ++i;
  double t = (log(k) - log(pk_k[i])) / (log(pk_k[i + 1]) - log(pk_k[i]));
  return exp(log(pk_p[i]) + t * (log(pk_p[i + 1]) - log(pk_p[i])));
}

/* table[n2] = dV / P(k) with k = (2 pi / L) sqrt(n2), n2 = kx^2+ky^2+kz^2 over signed integer
 * indices, for n2 = 0 .. 3(n/2)^2; table[0] = 0 (flat prior on the mean mode).
 * For cell-averaged fields and an unnormalised DFT the covariance of the DFT coefficients
 * is V_c * P(k)/dV, so S^-1 = F^-1 diag(dV/P) F. */
int oracle_sinv_table(int n, double box, const double* pk_k, const double* pk_p, int n_pk,
                      double* table) {
  if (n <= 0 || !(box > 0) || n_pk < 2) return OR_ERR_ARG;
  for (int i = 0; i < n_pk; ++i)
    if (!(pk_k[i] > 0) || !(pk_p[i] > 0) || (i > 0 && !(pk_k[i] > pk_k[i - 1]))) return OR_ERR_ARG;
  double H = box / (double)n, dV = H * H * H;
  long half = n / 2, len = 3 * half * half + 1;
  table[0] = 0.0;
  for (long n2 = 1; n2 < len; ++n2) {
    double k = (2.0 * OR_PI / box) * sqrt((double)n2);
    table[n2] = dV / pk_interp(k, pk_k, pk_p, n_pk);
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------------------ */
/* 7. The Wiener operator and textbook CG (Sec. 3.3.1, Eq. eq:WF; Krylov inversion)       */
/* ------------------------------------------------------------------------------------ */

/* q = A p = F^-1[ S^-1(k) F p ] / V_c + nbar * w * p. */
int oracle_matvec(int n, const double* table, double nbar, const double* w, const double* p,
                  double* q) {
  size_t N = (size_t)n, V = N * N * N;
  cplx* a = (cplx*)malloc(V * sizeof(cplx));
  if (!a) return OR_ERR_OOM;
  for (size_t i = 0; i < V; ++i) a[i] = p[i];
  int st = oracle_fft3d(a, n, -1);
  if (st == OR_OK) {
    for (size_t ix = 0; ix < N; ++ix)
      for (size_t iy = 0; iy < N; ++iy)
        for (size_t iz = 0; iz < N; ++iz) {
          long kx = sfreq((long)ix, (long)N), ky = sfreq((long)iy, (long)N), kz = sfreq((long)iz, (long)N);
          a[(ix * N + iy) * N + iz] *= table[kx * kx + ky * ky + kz * kz];
        }
    st = oracle_fft3d(a, n, +1);
  }
  if (st == OR_OK)
    for (size_t i = 0; i < V; ++i) q[i] = creal(a[i]) / (double)V + nbar * w[i] * p[i];
  free(a);
  return st;
}

static double dot(const double* u, const double* v, size_t V) {
  double s = 0.0;
  for (size_t i = 0; i < V; ++i) s += u[i] * v[i];
  return s;
}

/* Textbook (Hestenes-Stiefel) CG on A x = b from x0 = 0.  Stop test: the relative residual
 * ||b - A x|| / ||b|| recomputed from x (not the recurrence) must be <= tol; it is
 * recomputed whenever the recurrence residual reaches tol, and if the recomputed one has not,
 * r is replaced by it and the search direction restarted.  b = 0 gives x = 0 at 0 iterations. */
int oracle_cg(int n, const double* table, double nbar, const double* w, const double* b, double tol,
              int max_iter, double* x, int* iters_out, double* rel_res_out) {
  size_t V = (size_t)n * n * n;
  double *r = (double*)malloc(V * sizeof(double)), *p = (double*)malloc(V * sizeof(double)),
         *q = (double*)malloc(V * sizeof(double));
  int st = OR_OK, it = 0;
  double rel = 0.0;
  if (!r || !p || !q) {
    st = OR_ERR_OOM;
    goto done;
  }
  double bb = dot(b, b, V);
  for (size_t i = 0; i < V; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
    p[i] = b[i];
  }
  if (bb == 0.0) goto done;
  double rr = bb;
  for (;;) {
    if (rr <= tol * tol * bb) { /* recompute the true residual */
      st = oracle_matvec(n, table, nbar, w, x, q);
      if (st) goto done;
      for (size_t i = 0; i < V; ++i) r[i] = b[i] - q[i];
      rr = dot(r, r, V);
      rel = sqrt(rr / bb);
      if (rel <= tol) break;
      for (size_t i = 0; i < V; ++i) p[i] = r[i];
    }
    if (it >= max_iter) {
      rel = sqrt(rr / bb);
      st = OR_ERR_NOT_CONVERGED;
      break;
    }
    st = oracle_matvec(n, table, nbar, w, p, q);
    if (st) goto done;
    double pq = dot(p, q, V);
    if (!(pq > 0.0) || !isfinite(pq)) {
      st = OR_ERR_BREAKDOWN;
      break;
    }
    double alpha = rr / pq;
    for (size_t i = 0; i < V; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    double rr_new = dot(r, r, V);
    double beta = rr_new / rr;
    rr = rr_new;
    for (size_t i = 0; i < V; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
done:
  if (iters_out) *iters_out = it;
  if (rel_res_out) *rel_res_out = rel;
  free(r);
  free(p);
  free(q);
  return st;
}

/* z = M^-1 r with M^-1 = F^-1 diag(ptable(|k|^2)) F / V_c: a real, even Fourier multiplier,
 * applied with the same FFT as the matvec. */
static int fourier_apply(int n, const double* ptable, const double* r, double* z) {
  size_t N = (size_t)n, V = N * N * N;
  cplx* a = (cplx*)malloc(V * sizeof(cplx));
  if (!a) return OR_ERR_OOM;
  for (size_t i = 0; i < V; ++i) a[i] = r[i];
  int st = oracle_fft3d(a, n, -1);
  if (st == OR_OK) {
    for (size_t ix = 0; ix < N; ++ix)
      for (size_t iy = 0; iy < N; ++iy)
        for (size_t iz = 0; iz < N; ++iz) {
          long kx = sfreq((long)ix, (long)N), ky = sfreq((long)iy, (long)N), kz = sfreq((long)iz, (long)N);
          a[(ix * N + iy) * N + iz] *= ptable[kx * kx + ky * ky + kz * kz];
        }
    st = oracle_fft3d(a, n, +1);
  }
  if (st == OR_OK)
    for (size_t i = 0; i < V; ++i) z[i] = creal(a[i]) / (double)V;
  free(a);
  return st;
}

/* Preconditioned CG (Hestenes-Stiefel with a preconditioner M) on A x = b from x0 = 0, where
 * M^-1 = F^-1 diag(ptable) F is Fourier-diagonal (ptable indexed by n2 = |k|^2 like the prior
 * table, entries > 0).  The paper names only a Krylov-space inversion (Sec. 1, 3.3.1); a
 * Fourier-diagonal preconditioner keeps the same Krylov method on the same canonical system, and
 * with ptable = 1 every step is that of oracle_cg.  Each iteration:
 *   q = A p;  alpha = <r, z> / <p, q>;  x += alpha p;  r -= alpha q;  z = M^-1 r;
 *   beta = <r', z'> / <r, z>;  p = z + beta p      (p0 = z0 = M^-1 b).
 * Stop test as oracle_cg: the true relative residual ||b - A x|| / ||b|| <= tol, recomputed when
 * the recurrence residual ||r|| reaches tol, with r replaced and p restarted if it has not. */
int oracle_pcg(int n, const double* table, const double* ptable, double nbar, const double* w, const double* b,
               double tol, int max_iter, double* x, int* iters_out, double* rel_res_out) {
  size_t V = (size_t)n * n * n;
  double *r = (double*)malloc(V * sizeof(double)), *p = (double*)malloc(V * sizeof(double)),
         *q = (double*)malloc(V * sizeof(double)), *z = (double*)malloc(V * sizeof(double));
  int st = OR_OK, it = 0;
  double rel = 0.0;
  if (!r || !p || !q || !z) {
    st = OR_ERR_OOM;
    goto done;
  }
  double bb = dot(b, b, V);
  for (size_t i = 0; i < V; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
  }
  if (bb == 0.0) goto done;
  st = fourier_apply(n, ptable, r, z);
  if (st) goto done;
  for (size_t i = 0; i < V; ++i) p[i] = z[i];
  double rz = dot(r, z, V), rr = bb;
  for (;;) {
    if (rr <= tol * tol * bb) { /* recompute the true residual */
      st = oracle_matvec(n, table, nbar, w, x, q);
      if (st) goto done;
      for (size_t i = 0; i < V; ++i) r[i] = b[i] - q[i];
      rr = dot(r, r, V);
      rel = sqrt(rr / bb);
      if (rel <= tol) break;
      st = fourier_apply(n, ptable, r, z);
      if (st) goto done;
      for (size_t i = 0; i < V; ++i) p[i] = z[i];
      rz = dot(r, z, V);
    }
    if (it >= max_iter) {
      rel = sqrt(rr / bb);
      st = OR_ERR_NOT_CONVERGED;
      break;
    }
    st = oracle_matvec(n, table, nbar, w, p, q);
    if (st) goto done;
    double pq = dot(p, q, V);
    if (!(pq > 0.0) || !isfinite(pq)) {
      st = OR_ERR_BREAKDOWN;
      break;
    }
    double alpha = rz / pq;
    for (size_t i = 0; i < V; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    st = fourier_apply(n, ptable, r, z);
    if (st) goto done;
    double rz_new = dot(r, z, V);
    double beta = rz_new / rz;
    rz = rz_new;
    rr = dot(r, r, V);
    for (size_t i = 0; i < V; ++i) p[i] = z[i] + beta * p[i];
    ++it;
  }
done:
  if (iters_out) *iters_out = it;
  if (rel_res_out) *rel_res_out = rel;
  free(r);
  free(p);
  free(q);
  free(z);
  return st;
}

/* Sets the number of OpenMP threads for the following calls (no effect without OpenMP). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
