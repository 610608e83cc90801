// wf_fft.cuh -- shared-memory staged mixed-radix (8, 4, 2, 3) FFT engine.
//
// A CTA holds a tile of NL lines of length M in shared memory as tile[i * LD + l] (i = index
// along the transform, l = line).  Lines sit side by side, so a warp's accesses to one row are
// contiguous (conflict-free) and a tile is loaded from / stored to global memory with rows of
// NL consecutive elements.  Each line is served by TPL threads (thread t of line l has
// threadIdx.x = t * NLT + l, NLT >= NL being the line slots of the CTA).
//
// The transform is a self-sorting (Stockham) sequence of radix-R passes: at the pass with
// span NS (product of the earlier radices), butterfly j reads elements j + r M/R, multiplies
// element r by W_{NS R}^{r (j mod NS)}, does an R-point DFT and writes the results to
// (j / NS) NS R + (j mod NS) + r NS.  Each pass reads everything into registers, syncs, and
// writes back in place.  Output is in natural order; no normalisation is applied.
// DIR = -1: forward, exp(-2 pi i jk/M); DIR = +1: inverse, exp(+2 pi i jk/M).
// Twiddles come from a table tw[e] = exp(-2 pi i e / (TWS M)) in shared memory.
#pragma once
#include "wf_common.cuh"

namespace wf {

// ---- radix plan: the largest power-of-two radix up to RMAX first, then 3s ----------------
// RMAX (32, 16 or 8) is the largest radix whose butterfly fits in one thread's elements.
constexpr int pick_radix(int rem, int rmax) {
  return (rmax >= 32 && rem % 32 == 0) ? 32
         : (rmax >= 16 && rem % 16 == 0) ? 16
         : rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : rem % 3 == 0 ? 3 : rem;
}
constexpr int radix_at(int M, int s, int rmax) {
  int rem = M;
  for (int i = 0; i < s; ++i) rem /= pick_radix(rem, rmax);
  return pick_radix(rem, rmax);
}
constexpr int rmax_for(int M, int TPL) {
  return M / TPL >= 32 ? 32 : (M / TPL >= 16 ? 16 : 8);
}

// ---- small DFTs in registers -------------------------------------------------------------
template <int DIR, class R> WF_D void dft2(cx<R>* v) {
  cx<R> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}
template <int DIR, class R> WF_D void dft4(cx<R>* v) {
  cx<R> t0 = v[0] + v[2], t1 = v[0] - v[2];
  cx<R> t2 = v[1] + v[3], t3 = mul_si<DIR>(v[1] - v[3]);
  v[0] = t0 + t2;
  v[2] = t0 - t2;
  v[1] = t1 + t3;
  v[3] = t1 - t3;
}
template <int DIR, class R> WF_D void dft3(cx<R>* v) {
  const R half = RT<R>::c(0.5), s3 = RT<R>::c(0.86602540378443864676);
  cx<R> t = v[1] + v[2], u = v[1] - v[2];
  cx<R> m = v[0] - scale(t, half);
  cx<R> ju = mul_si<DIR>(scale(u, s3));
  v[0] = v[0] + t;
  v[1] = m + ju;
  v[2] = m - ju;
}
template <int DIR, class R> WF_D void dft8(cx<R>* v) {
  cx<R> e[4] = {v[0], v[2], v[4], v[6]};
  cx<R> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<DIR>(e);
  dft4<DIR>(o);
  const R r2 = RT<R>::c(0.70710678118654752440);
  // W8^1 = (1 + DIR i)/sqrt2, W8^2 = DIR i, W8^3 = (-1 + DIR i)/sqrt2
  cx<R> o1 = scale(o[1] + mul_si<DIR>(o[1]), r2);
  cx<R> o2 = mul_si<DIR>(o[2]);
  cx<R> o3 = scale(mul_si<DIR>(o[3]) - o[3], r2);
  v[0] = e[0] + o[0];
  v[4] = e[0] - o[0];
  v[1] = e[1] + o1;
  v[5] = e[1] - o1;
  v[2] = e[2] + o2;
  v[6] = e[2] - o2;
  v[3] = e[3] + o3;
  v[7] = e[3] - o3;
}
template <int RAD, int DIR, class R> WF_D void dft_small(cx<R>* v) {
  if constexpr (RAD == 2) dft2<DIR>(v);
  else if constexpr (RAD == 3) dft3<DIR>(v);
  else if constexpr (RAD == 4) dft4<DIR>(v);
  else dft8<DIR>(v);
}
// cos and sin of 2 pi m / RR at compile time (Taylor series after reduction to the first octant
// by symmetry), used for the internal twiddles of the composite radices.
constexpr double k_pi = 3.14159265358979323846;
constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 12; ++n) {
    term *= -x * x / ((2 * n) * (2 * n + 1));
    sum += term;
  }
  return sum;
}
constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 12; ++n) {
    term *= -x * x / ((2 * n - 1) * (2 * n));
    sum += term;
  }
  return sum;
}
// (cos, sin) of 2 pi m / RR, m in [0, RR)
constexpr double cw_cos(int m, int RR) {
  m = ((m % RR) + RR) % RR;
  if (4 * m == RR || 4 * m == 3 * RR) return 0.0;
  if (2 * m == RR) return -1.0;
  if (m == 0) return 1.0;
  if (4 * m > RR && 4 * m < 3 * RR) return -cw_cos(m + RR / 2, RR);  // cos(x) = -cos(x + pi)
  if (4 * m >= 3 * RR) return cw_cos(RR - m, RR);
  if (8 * m > RR) return taylor_sin(2.0 * k_pi * (double)(RR / 4 - m) / RR);  // cos(x) = sin(pi/2 - x)
  return taylor_cos(2.0 * k_pi * (double)m / RR);
}
constexpr double cw_sin(int m, int RR) { return cw_cos(m - RR / 4 + RR, RR); }  // sin(x) = cos(x - pi/2)

// v * exp(DIR 2 pi i m / RR) with a compile-time m: exact for quarter turns
template <int M_, int RR, int DIR, class R>
WF_D cx<R> twiddle_const(cx<R> v) {
  constexpr int m = M_ % RR;
  if constexpr (m == 0) return v;
  else if constexpr (4 * m == RR) return mul_si<DIR>(v);
  else if constexpr (2 * m == RR) return cx<R>{-v.x, -v.y};
  else if constexpr (4 * m == 3 * RR) return mul_si<-DIR>(v);
  else {
    const R c = RT<R>::c(cw_cos(m, RR)), sn = RT<R>::c(DIR * cw_sin(m, RR));
    return cx<R>{v.x * c - v.y * sn, v.x * sn + v.y * c};
  }
}

template <int N2, int R1, int R2, int DIR, class R>
WF_D void comp_column(cx<R>* v) {
  cx<R> c[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) c[n1] = v[R2 * n1 + N2];
  dft_small<R1, DIR>(c);
  v[N2] = c[0];
  if constexpr (R1 > 1) v[R2 * 1 + N2] = twiddle_const<N2 * 1, R1 * R2, DIR>(c[1]);
  if constexpr (R1 > 2) v[R2 * 2 + N2] = twiddle_const<N2 * 2, R1 * R2, DIR>(c[2]);
  if constexpr (R1 > 3) v[R2 * 3 + N2] = twiddle_const<N2 * 3, R1 * R2, DIR>(c[3]);
  if constexpr (N2 + 1 < R2) comp_column<N2 + 1, R1, R2, DIR>(v);
}

// Radix R1*R2 butterfly (R1 <= 4) as a two-level Cooley-Tukey in registers:
//   X[k1 + R1 k2] = sum_n2 W_R2^(n2 k2) W_R1R2^(n2 k1) sum_n1 x[R2 n1 + n2] W_R1^(n1 k1)
// with the internal twiddles W_R1R2^(n2 k1) as compile-time constants.
template <int R1, int R2, int DIR, class R>
WF_D void dft_comp(cx<R>* v, const cx<R>*, int) {
  constexpr int RR = R1 * R2;
  comp_column<0, R1, R2, DIR>(v);
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) dft_small<R2, DIR>(v + R2 * k1);
  cx<R> o[RR];
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) o[k1 + R1 * k2] = v[R2 * k1 + k2];
#pragma unroll
  for (int r = 0; r < RR; ++r) v[r] = o[r];
}

// tstep: table stride of W_RAD^1 (only the composite radices use the table)
template <int RAD, int DIR, class R> WF_D void dft(cx<R>* v, const cx<R>* tw, int tstep) {
  if constexpr (RAD == 32) dft_comp<4, 8, DIR>(v, tw, tstep);
  else if constexpr (RAD == 16) dft_comp<4, 4, DIR>(v, tw, tstep);
  else dft_small<RAD, DIR>(v);
}

// ---- element addressing ------------------------------------------------------------------
// A line's element i lives at col[map(i)]: Strided<LD> for the side-by-side tiles above, other
// maps for swizzled or blocked tiles.
template <int LD> struct Strided {
  WF_D int operator()(int i) const { return i * LD; }
};

// ---- one Stockham pass -------------------------------------------------------------------
template <class R, int M, int RAD, int NS, int TPL, int DIR, int TWS, class MAP>
WF_D void fft_pass(cx<R>* col, const MAP& map, int t, const cx<R>* tw, bool act) {
  constexpr int NB = M / RAD;
  constexpr int PER = (NB + TPL - 1) / TPL;
  cx<R> v[PER][RAD];
#pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int j = t + m * TPL;
    if (act && ((NB % TPL) == 0 || j < NB)) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[m][r] = col[map(j + r * NB)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int j = t + m * TPL;
    if (act && ((NB % TPL) == 0 || j < NB)) {
      const int k = j % NS;
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          cx<R> w = tw[TWS * (r * k * (M / (NS * RAD)))];
          if constexpr (DIR > 0) w = conj(w);
          v[m][r] = v[m][r] * w;
        }
      }
      dft<RAD, DIR>(v[m], tw, TWS * (M / RAD));
      const int base = (j / NS) * NS * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) col[map(base + r * NS)] = v[m][r];
    }
  }
  __syncthreads();
}

template <class R, int M, int S, int NS, int TPL, int DIR, int TWS, int RMAX, class MAP>
WF_D void fft_passes(cx<R>* col, const MAP& map, int t, const cx<R>* tw, bool act) {
  if constexpr (NS < M) {
    constexpr int RAD = radix_at(M, S, RMAX);
    fft_pass<R, M, RAD, NS, TPL, DIR, TWS>(col, map, t, tw, act);
    fft_passes<R, M, S + 1, NS * RAD, TPL, DIR, TWS, RMAX>(col, map, t, tw, act);
  }
}

// Transform the line whose element i is at col[map(i)], of length M, with TPL threads (thread
// index t in [0, TPL)).  Every thread of the CTA must call this (it synchronises the CTA);
// threads with act = false only take part in the barriers.  The twiddle table holds
// exp(-2 pi i e / (M TWS)), so W_M^e = tw[TWS e].  RMAX caps the radix: 8 keeps every
// butterfly in the small kernels; 16 or 32 allows the composite butterflies (fewer shared
// memory round trips, more registers), which measured faster only for the z passes.
template <class R, int M, int TPL, int DIR, int TWS = 1, int RMAX = 8, class MAP>
WF_D void fft_line_map(cx<R>* col, const MAP& map, int t, const cx<R>* tw, bool act = true) {
  fft_passes<R, M, 0, 1, TPL, DIR, TWS, RMAX>(col, map, t, tw, act);
}
// the same for the line col[i * LD]
template <class R, int M, int TPL, int LD, int DIR, int TWS = 1, int RMAX = 8>
WF_D void fft_line(cx<R>* col, int t, const cx<R>* tw, bool act = true) {
  fft_passes<R, M, 0, 1, TPL, DIR, TWS, RMAX>(col, Strided<LD>{}, t, tw, act);
}

// Threads per line for a line of length M: one radix-8-or-smaller butterfly group per thread
// at elements-per-thread E.
constexpr int tpl_for(int M, int E) { return M / E >= 1 ? M / E : 1; }

}  // namespace wf
