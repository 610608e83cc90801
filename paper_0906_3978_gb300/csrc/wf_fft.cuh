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

// ---- radix plan: 8s first, then 4, 2, then 3s -------------------------------------------
constexpr int pick_radix(int rem) {
  return rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : rem % 2 == 0 ? 2 : rem % 3 == 0 ? 3 : rem;
}
constexpr int radix_at(int M, int s) {
  int rem = M;
  for (int i = 0; i < s; ++i) rem /= pick_radix(rem);
  return pick_radix(rem);
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
template <int RAD, int DIR, class R> WF_D void dft(cx<R>* v) {
  if constexpr (RAD == 2) dft2<DIR>(v);
  else if constexpr (RAD == 3) dft3<DIR>(v);
  else if constexpr (RAD == 4) dft4<DIR>(v);
  else dft8<DIR>(v);
}

// ---- one Stockham pass -------------------------------------------------------------------
template <class R, int M, int RAD, int NS, int TPL, int LD, int DIR, int TWS>
WF_D void fft_pass(cx<R>* col, int t, const cx<R>* tw, bool act) {
  constexpr int NB = M / RAD;
  constexpr int PER = (NB + TPL - 1) / TPL;
  cx<R> v[PER][RAD];
#pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int j = t + m * TPL;
    if (act && ((NB % TPL) == 0 || j < NB)) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[m][r] = col[(j + r * NB) * LD];
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
      dft<RAD, DIR>(v[m]);
      const int base = (j / NS) * NS * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) col[(base + r * NS) * LD] = v[m][r];
    }
  }
  __syncthreads();
}

template <class R, int M, int S, int NS, int TPL, int LD, int DIR, int TWS>
WF_D void fft_passes(cx<R>* col, int t, const cx<R>* tw, bool act) {
  if constexpr (NS < M) {
    constexpr int RAD = radix_at(M, S);
    fft_pass<R, M, RAD, NS, TPL, LD, DIR, TWS>(col, t, tw, act);
    fft_passes<R, M, S + 1, NS * RAD, TPL, LD, DIR, TWS>(col, t, tw, act);
  }
}

// Transform column `col` (stride LD) of length M with TPL threads (thread index t in
// [0, TPL)).  Every thread of the CTA must call this (it synchronises the CTA); threads with
// act = false only take part in the barriers.  The twiddle table holds
// exp(-2 pi i e / (M TWS)), so W_M^e = tw[TWS e].
template <class R, int M, int TPL, int LD, int DIR, int TWS = 1>
WF_D void fft_line(cx<R>* col, int t, const cx<R>* tw, bool act = true) {
  fft_passes<R, M, 0, 1, TPL, LD, DIR, TWS>(col, t, tw, act);
}

// Threads per line for a line of length M: one radix-8-or-smaller butterfly group per thread
// at elements-per-thread E.
constexpr int tpl_for(int M, int E) { return M / E >= 1 ? M / E : 1; }

}  // namespace wf
