// wf_spectral.cuh -- 3D FFT passes over the packed half spectrum, with the Wiener operator's
// diagonal factors fused into them.
//
// Spectrum layout ("packed half spectrum"): complex [N][N][N/2], index (kx, ky, kz) with
// kx, ky in [0, N) (signed frequency = index, or index - N above N/2) and kz in [0, N/2).
// Column kz = 0 carries two real-field planes: after the z transform of real lines, the
// kz = 0 and kz = N/2 coefficients are both real, and they are stored as (re, im) of element
// kz = 0.  The y and x transforms act on that complex plane linearly, so the column holds
// Z = P0 + i PN with P0, PN the 2D transforms of the two planes.  A real, even Fourier
// multiplier m(k) applied to the unpacked planes becomes
//     Z'(k) = (m0 + mN)/2 Z(k) + (m0 - mN)/2 conj(Z(-k)),
// with m0 = m(kx, ky, 0), mN = m(kx, ky, N/2) and -k = (-kx, -ky); this is why the x passes,
// where multipliers are applied, also read the "partner" line at -ky for column 0.
// The inner product of two real fields u, v is (1/V_c) sum over the packed spectrum of
// wgt * Re(conj(u) v) with wgt = 1 on column 0 and 2 elsewhere.
//
// Passes (all one CTA per tile of NL lines):
//   y pass      complex FFT along y, in place
//   x passes    multiplier(s) + complex FFT along x, fused with CG vector updates
//   z turn      packed -> C2R -> multiply by a real diagonal -> R2C -> packed (one z line)
//   z fwd/inv   real rows <-> packed spectrum rows, with epilogues
#pragma once
#include "wf_fft.cuh"

namespace wf {

// Device-resident CG scalars.  Written only by the single-CTA finisher kernels.
struct CgScal {
  double rr;          // <r, r> of the preconditioned residual
  double pq;          // <p, A p>
  double alpha;       // rr / pq of the last iteration
  double alpha_prev;  // alpha still to be applied to x (fused into the next x pass)
  double beta;
  double bb;          // ||b||^2 of the canonical system (real space)
  double rc2;         // upper estimate of the canonical ||b - A s||^2 (real space)
  double tol2;        // stop when rc2 <= tol2 * bb
  double rr_stop;     // inner solves: stop when rc2 <= rr_stop (absolute)
  double aux[4];
  int iter;
  int max_iter;
  int done;           // 1: converged (estimate); 2: iteration cap; 3: breakdown
  int status;
};

template <class R> constexpr int tile_lines() { return 128 / (int)sizeof(cx<R>); }
template <class R> constexpr int elems_per_thread() { return sizeof(cx<R>) == 8 ? 16 : 8; }
template <class R, int M> constexpr int tpl() {
  return M / elems_per_thread<R>() >= 1 ? M / elems_per_thread<R>() : 1;
}
constexpr int cmin(int a, int b) { return a < b ? a : b; }
// largest divisor of n that is <= cap (tile widths must divide the dimension they tile)
constexpr int div_le(int n, int cap) {
  int d = cap < n ? cap : n;
  while (d > 1 && n % d != 0) --d;
  return d;
}
// lines per CTA of the x / y passes: consecutive kz columns, a divisor of N/2
template <class R, int N> constexpr int xy_lines() { return div_le(N / 2, tile_lines<R>()); }

// signed frequency of an index on an axis of length n
WF_D int sfreq(int j, int n) { return j <= (n >> 1) ? j : j - n; }

// Load the length-M twiddles exp(-2 pi i e / M) from a length-TN FP64 table into shared memory.
template <class R, int M, int TN>
WF_D void load_tw(cx<R>* tw, const double2* tab, int tid, int nt) {
  for (int e = tid; e < M; e += nt) tw[e] = ld_c<R>(tab + e * (TN / M));
}

// ------------------------------------------------------------------------------------------
// y pass: complex FFT along y of every (x, kz) line; in place.
// grid (N/2 / NL, N), block NL * TPL.
// ------------------------------------------------------------------------------------------
template <class R, int N, int DIR>
__global__ void __launch_bounds__(xy_lines<R, N>() * tpl<R, N>())
k_ypass(typename Store<R>::T* __restrict__ spec, const double2* __restrict__ twtab,
        const CgScal* __restrict__ sc) {
  using ST = typename Store<R>::T;
  constexpr int M = N, NH = N / 2, NL = xy_lines<R, N>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = NL * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;
  if (sc && sc->done) return;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * NL, x = blockIdx.y;
  load_tw<R, M, 2 * N>(tw, twtab, tid, NT);
  ST* base = spec + (size_t)x * N * NH + kz0;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, l = idx % NL;
    tile[i * LD + l] = ld_c<R>(base + (size_t)i * NH + l);
  }
  __syncthreads();
  fft_line<R, M, TPL, LD, DIR>(tile + tid % NL, tid / NL, tw);
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, l = idx % NL;
    st_c(base + (size_t)i * NH + l, tile[i * LD + l]);
  }
}

// Apply the packed-column multiplier pair to column 0 of a tile (slot 0) using the partner
// line in slot NL.  tab is indexed by n2 = kx^2 + ky^2 + kz^2.  Must be called by all
// threads; synchronises before returning.
template <class R, int N, int LD, int NL, class TAB>
WF_D void combine_col0(cx<R>* tile, int ky_s, const TAB* tab, int tid, int nt) {
  constexpr int NH = N / 2;
  for (int kx = tid; kx < N; kx += nt) {
    const int kxs = sfreq(kx, N);
    const int n2 = kxs * kxs + ky_s * ky_s;
    const R m0 = RT<R>::c((double)tab[n2]);
    const R mN = RT<R>::c((double)tab[n2 + NH * NH]);
    const R h = RT<R>::c(0.5);
    const R a = (m0 + mN) * h, b = (m0 - mN) * h;
    const cx<R> z = tile[kx * LD];
    const cx<R> zp = conj(tile[((N - kx) % N) * LD + NL]);
    tile[kx * LD] = scale(z, a) + scale(zp, b);
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// CG x pass 1 (start of A p):  p_new = r + beta p_old;  x += alpha_prev p_old;
//                              T = IFFT_x( c (.) p_new )
// grid (N/2 / NL, N), block (NL + 1) * TPL; slot NL holds the partner line (ky' = -ky) of
// column 0 when kz0 == 0.
// ------------------------------------------------------------------------------------------
template <class R, int N>
__global__ void __launch_bounds__((xy_lines<R, N>() + 1) * tpl<R, N>())
k_cg_xinv(const typename Store<R>::T* __restrict__ r, const typename Store<R>::T* __restrict__ pold,
          typename Store<R>::T* __restrict__ pnew, typename Store<R>::T* __restrict__ x,
          typename Store<R>::T* __restrict__ T, const typename Store<R>::S* __restrict__ ctab,
          const double2* __restrict__ twtab, const CgScal* __restrict__ sc) {
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  constexpr int M = N, NH = N / 2, NL = xy_lines<R, N>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = (NL + 1) * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;
  if (sc->done) return;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * NL, ky = blockIdx.y;
  const int ky_s = sfreq(ky, N);
  const SS beta = (SS)sc->beta, alpha_prev = (SS)sc->alpha_prev;
  load_tw<R, M, 2 * N>(tw, twtab, tid, NT);
  const size_t rowstride = (size_t)N * NH;
  const size_t base = (size_t)ky * NH + kz0;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, l = idx % NL;
    const size_t e = base + (size_t)i * rowstride + l;
    const ST rv = r[e], po = pold[e];
    ST pn;
    pn.x = rv.x + beta * po.x;
    pn.y = rv.y + beta * po.y;
    pnew[e] = pn;
    ST xv = x[e];
    xv.x += alpha_prev * po.x;
    xv.y += alpha_prev * po.y;
    x[e] = xv;
    tile[i * LD + l] = ld_c<R>(&pn);
  }
  if (kz0 == 0) {  // partner line of column 0: p_new at (kx, -ky, 0), recomputed from inputs
    const size_t pb = (size_t)((N - ky) % N) * NH;
    for (int i = tid; i < M; i += NT) {
      const size_t e = pb + (size_t)i * rowstride;
      const ST rv = r[e], po = pold[e];
      ST pn;
      pn.x = rv.x + beta * po.x;
      pn.y = rv.y + beta * po.y;
      tile[i * LD + NL] = ld_c<R>(&pn);
    }
  }
  __syncthreads();
  // multiplier c(k)
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, l = idx % NL;
    if (kz0 + l == 0) continue;
    const int kxs = sfreq(i, N), kz = kz0 + l;
    tile[i * LD + l] = scale(tile[i * LD + l], RT<R>::c((double)ctab[kxs * kxs + ky_s * ky_s + kz * kz]));
  }
  if (kz0 == 0) combine_col0<R, N, LD, NL>(tile, ky_s, ctab, tid, NT);
  else __syncthreads();
  const int l = tid % (NL + 1), t = tid / (NL + 1);
  fft_line<R, M, TPL, LD, +1>(tile + l, t, tw);
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, ll = idx % NL;
    st_c(T + base + (size_t)i * rowstride + ll, tile[i * LD + ll]);
  }
}

// ------------------------------------------------------------------------------------------
// CG x pass 2 (end of A p):  T^ = FFT_x(T);  q = m (.) p + c (.) T^;  partial <p, q>
// ------------------------------------------------------------------------------------------
template <class R, int N>
__global__ void __launch_bounds__((xy_lines<R, N>() + 1) * tpl<R, N>())
k_cg_xfwd(const typename Store<R>::T* __restrict__ T, const typename Store<R>::T* __restrict__ p,
          typename Store<R>::T* __restrict__ q, const typename Store<R>::S* __restrict__ ctab,
          const typename Store<R>::S* __restrict__ mtab, const double2* __restrict__ twtab,
          double* __restrict__ partials, const CgScal* __restrict__ sc) {
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  constexpr int M = N, NH = N / 2, NL = xy_lines<R, N>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = (NL + 1) * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;
  __shared__ double red[32];
  if (sc->done) return;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * NL, ky = blockIdx.y;
  const int ky_s = sfreq(ky, N);
  const int pky = (N - ky) % N;
  load_tw<R, M, 2 * N>(tw, twtab, tid, NT);
  const size_t rowstride = (size_t)N * NH;
  const size_t base = (size_t)ky * NH + kz0;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, l = idx % NL;
    tile[i * LD + l] = ld_c<R>(T + base + (size_t)i * rowstride + l);
  }
  if (kz0 == 0)
    for (int i = tid; i < M; i += NT) tile[i * LD + NL] = ld_c<R>(T + (size_t)pky * NH + (size_t)i * rowstride);
  __syncthreads();
  {
    const int l = tid % (NL + 1), t = tid / (NL + 1);
    fft_line<R, M, TPL, LD, -1>(tile + l, t, tw);
  }
  if (kz0 == 0) combine_col0<R, N, LD, NL>(tile, ky_s, ctab, tid, NT);
  typename AccFor<SS>::T acc;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, l = idx % NL;
    const int kxs = sfreq(i, N), kz = kz0 + l;
    const size_t e = base + (size_t)i * rowstride + l;
    const ST pv = p[e];
    cx<R> t = tile[i * LD + l];
    ST qv;
    if (kz == 0) {
      // packed column: m-term combined with the partner element p(-kx, -ky, 0)
      const int n2 = kxs * kxs + ky_s * ky_s;
      const double m0 = (double)mtab[n2], mN = (double)mtab[n2 + NH * NH];
      const ST pp = p[(size_t)((N - i) % N) * rowstride + (size_t)pky * NH];
      const double a = 0.5 * (m0 + mN), b = 0.5 * (m0 - mN);
      const double mx = a * (double)pv.x + b * (double)pp.x;
      const double my = a * (double)pv.y - b * (double)pp.y;
      qv.x = (SS)(mx + RT<R>::to_d(t.x));
      qv.y = (SS)(my + RT<R>::to_d(t.y));
    } else {
      const int n2 = kxs * kxs + ky_s * ky_s + kz * kz;
      const cx<R> ct = scale(t, RT<R>::c((double)ctab[n2]));
      const SS m = mtab[n2];
      qv.x = (SS)(m * pv.x + (SS)RT<R>::to_d(ct.x));
      qv.y = (SS)(m * pv.y + (SS)RT<R>::to_d(ct.y));
    }
    q[e] = qv;
    const SS wgt = kz == 0 ? (SS)1 : (SS)2;
    acc.add_prod(wgt * pv.x, qv.x);
    acc.add_prod(wgt * pv.y, qv.y);
  }
  const double s = block_sum(acc.get(), red);
  if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// ------------------------------------------------------------------------------------------
// Generic x pass:  out = [IFFT_x]( tab (.) [FFT_x](in) ),  optional partial of wgt |out|^2.
// in != out (the partner line of column 0 is read from `in`).
// ------------------------------------------------------------------------------------------
template <class R, int N, bool FWD, bool INV, bool DOT>
__global__ void __launch_bounds__((xy_lines<R, N>() + 1) * tpl<R, N>())
k_xmul(const typename Store<R>::T* __restrict__ in, typename Store<R>::T* __restrict__ out,
       const typename Store<R>::S* __restrict__ tab, const double2* __restrict__ twtab,
       double* __restrict__ partials, const CgScal* __restrict__ sc) {
  using SS = typename Store<R>::S;
  constexpr int M = N, NH = N / 2, NL = xy_lines<R, N>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = (NL + 1) * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;
  __shared__ double red[32];
  if (sc && sc->done) return;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * NL, ky = blockIdx.y;
  const int ky_s = sfreq(ky, N);
  const int pky = (N - ky) % N;
  load_tw<R, M, 2 * N>(tw, twtab, tid, NT);
  const size_t rowstride = (size_t)N * NH;
  const size_t base = (size_t)ky * NH + kz0;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, l = idx % NL;
    tile[i * LD + l] = ld_c<R>(in + base + (size_t)i * rowstride + l);
  }
  if (kz0 == 0)
    for (int i = tid; i < M; i += NT) tile[i * LD + NL] = ld_c<R>(in + (size_t)pky * NH + (size_t)i * rowstride);
  __syncthreads();
  const int l = tid % (NL + 1), t = tid / (NL + 1);
  if constexpr (FWD) fft_line<R, M, TPL, LD, -1>(tile + l, t, tw);
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, ll = idx % NL;
    if (kz0 + ll == 0) continue;
    const int kxs = sfreq(i, N), kz = kz0 + ll;
    tile[i * LD + ll] = scale(tile[i * LD + ll], RT<R>::c((double)tab[kxs * kxs + ky_s * ky_s + kz * kz]));
  }
  if (kz0 == 0) combine_col0<R, N, LD, NL>(tile, ky_s, tab, tid, NT);
  else __syncthreads();
  if constexpr (INV) fft_line<R, M, TPL, LD, +1>(tile + l, t, tw);
  typename AccFor<SS>::T acc;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int i = idx / NL, ll = idx % NL;
    const cx<R> v = tile[i * LD + ll];
    st_c(out + base + (size_t)i * rowstride + ll, v);
    if constexpr (DOT) {
      const SS wgt = (kz0 + ll == 0) ? (SS)1 : (SS)2;
      const SS vx = (SS)RT<R>::to_d(v.x), vy = (SS)RT<R>::to_d(v.y);
      acc.add_prod(wgt * vx, vx);
      acc.add_prod(wgt * vy, vy);
    }
  }
  if constexpr (DOT) {
    const double s = block_sum(acc.get(), red);
    if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------------------------------
// z direction helpers: real line of length N <-> packed half spectrum of length h = N/2,
// through a complex FFT of length h on z_m = x_2m + i x_2m+1.  tw holds exp(-2 pi i e/(2N)),
// e < 2N (so W_N^k = tw[2k] and the length-h FFT uses stride 4).
// ------------------------------------------------------------------------------------------
// C2R pre-step on one line (stride LD): X (packed) -> Z with z = IFFT_h(Z) the real samples.
template <class R, int N, int LD>
WF_D void c2r_prep(cx<R>* col, int t, int tpl_, const cx<R>* tw) {
  constexpr int H = N / 2;
  for (int k = t; k <= H / 2; k += tpl_) {
    if (k == 0) {
      const cx<R> v = col[0];
      col[0] = cx<R>{v.x + v.y, v.x - v.y};
    } else {
      const int k2 = H - k;
      const cx<R> a = col[k * LD], b = col[k2 * LD];
      // Z_k = (X_k + conj X_{h-k}) + i W_N^{+k} (X_k - conj X_{h-k})
      const cx<R> s1 = a + conj(b), d1 = a - conj(b);
      const cx<R> s2 = b + conj(a), d2 = b - conj(a);
      const cx<R> w1 = conj(tw[2 * k]), w2 = conj(tw[2 * k2]);
      col[k * LD] = s1 + mul_i(w1 * d1);
      if (k2 != k) col[k2 * LD] = s2 + mul_i(w2 * d2);
    }
  }
}
// R2C post-step on one line: Z = FFT_h(z) -> packed X (X_0, X_h in element 0).
template <class R, int N, int LD>
WF_D void r2c_post(cx<R>* col, int t, int tpl_, const cx<R>* tw) {
  constexpr int H = N / 2;
  const R half = RT<R>::c(0.5);
  for (int k = t; k <= H / 2; k += tpl_) {
    if (k == 0) {
      const cx<R> v = col[0];
      col[0] = cx<R>{v.x + v.y, v.x - v.y};
    } else {
      const int k2 = H - k;
      const cx<R> a = col[k * LD], b = col[k2 * LD];
      // X_k = (Z_k + conj Z_{h-k})/2 - (i/2) W_N^{-k} (Z_k - conj Z_{h-k})
      const cx<R> s1 = a + conj(b), d1 = a - conj(b);
      const cx<R> s2 = b + conj(a), d2 = b - conj(a);
      const cx<R> w1 = tw[2 * k], w2 = tw[2 * k2];
      col[k * LD] = scale(s1 - mul_i(w1 * d1), half);
      if (k2 != k) col[k2 * LD] = scale(s2 - mul_i(w2 * d2), half);
    }
  }
}

// ------------------------------------------------------------------------------------------
// z turn (middle of A p): each (x, y) line: packed -> real (C2R), times D(x, y, z), -> packed.
// D = nbar w / V_c carries the 1/V_c of the inverse transform.  grid (N*N / NL), block NL*TPL.
// ------------------------------------------------------------------------------------------
template <class R, int N>
__global__ void __launch_bounds__(tile_lines<R>() * tpl<R, N / 2>())
k_zturn(typename Store<R>::T* __restrict__ spec, const typename Store<R>::S* __restrict__ D,
        const double2* __restrict__ twtab, const CgScal* __restrict__ sc) {
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  constexpr int H = N / 2, M = H, NL = tile_lines<R>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = NL * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;  // 2N entries
  if (sc && sc->done) return;
  const int tid = threadIdx.x;
  const size_t row0 = (size_t)blockIdx.x * NL;
  for (int e = tid; e < 2 * N; e += NT) tw[e] = ld_c<R>(twtab + e);
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int l = idx / M, i = idx % M;
    tile[i * LD + l] = ld_c<R>(spec + (row0 + l) * H + i);
  }
  __syncthreads();
  const int l = tid % NL, t = tid / NL;
  c2r_prep<R, N, LD>(tile + l, t, TPL, tw);
  __syncthreads();
  fft_line<R, M, TPL, LD, +1, 4>(tile + l, t, tw);
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int ll = idx / M, i = idx % M;
    const ST dv = *reinterpret_cast<const ST*>(D + (row0 + ll) * N + 2 * i);
    cx<R> v = tile[i * LD + ll];
    v.x = v.x * RT<R>::c((double)dv.x);
    v.y = v.y * RT<R>::c((double)dv.y);
    tile[i * LD + ll] = v;
  }
  __syncthreads();
  fft_line<R, M, TPL, LD, -1, 4>(tile + l, t, tw);
  r2c_post<R, N, LD>(tile + l, t, TPL, tw);
  __syncthreads();
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int ll = idx / M, i = idx % M;
    st_c(spec + (row0 + ll) * H + i, tile[i * LD + ll]);
  }
}

// ------------------------------------------------------------------------------------------
// z forward: real rows (FP64) -> packed spectrum rows.  Optional partial of sum(in^2).
// grid (N*N / NL), block NL*TPL, shared (H*LD + 2N) complex.
// ------------------------------------------------------------------------------------------
template <class R, int N, bool SQ>
__global__ void __launch_bounds__(tile_lines<R>() * tpl<R, N / 2>())
k_zfwd(const double* __restrict__ in, typename Store<R>::T* __restrict__ out,
       const double2* __restrict__ twtab, double* __restrict__ partials, const CgScal* __restrict__ sc) {
  constexpr int H = N / 2, M = H, NL = tile_lines<R>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = NL * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;
  __shared__ double red[32];
  if (sc && sc->done) return;
  const int tid = threadIdx.x;
  const size_t row0 = (size_t)blockIdx.x * NL;
  for (int e = tid; e < 2 * N; e += NT) tw[e] = ld_c<R>(twtab + e);
  const double2* in2 = reinterpret_cast<const double2*>(in);
  AccD acc;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int l = idx / M, i = idx % M;
    const double2 v = in2[(row0 + l) * H + i];
    tile[i * LD + l] = ld_c<R>(&v);
    if constexpr (SQ) {
      acc.add_prod(v.x, v.x);
      acc.add_prod(v.y, v.y);
    }
  }
  __syncthreads();
  const int l = tid % NL, t = tid / NL;
  fft_line<R, M, TPL, LD, -1, 4>(tile + l, t, tw);
  r2c_post<R, N, LD>(tile + l, t, TPL, tw);
  __syncthreads();
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int ll = idx / M, i = idx % M;
    st_c(out + (row0 + ll) * H + i, tile[i * LD + ll]);
  }
  if constexpr (SQ) {
    const double s = block_sum(acc.get(), red);
    if (tid == 0) partials[blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------------------------------
// z inverse: packed spectrum rows -> real rows (FP64), value v = scale * C2R(in), then
//   ZI_STORE: out = v
//   ZI_RESID: out = b - (v + nbar w s), partial sum(out^2)
//   ZI_ACCUM: out += v
// ------------------------------------------------------------------------------------------
enum { ZI_STORE = 0, ZI_RESID = 1, ZI_ACCUM = 2 };
template <class R, int N, int MODE>
__global__ void __launch_bounds__(tile_lines<R>() * tpl<R, N / 2>())
k_zinv(const typename Store<R>::T* __restrict__ in, double* __restrict__ out,
       const double* __restrict__ s, const double* __restrict__ w, const double* __restrict__ b,
       double nbar, double scl, const double2* __restrict__ twtab, double* __restrict__ partials,
       const CgScal* __restrict__ sc) {
  constexpr int H = N / 2, M = H, NL = tile_lines<R>(), LD = NL + 1;
  constexpr int TPL = tpl<R, M>(), NT = NL * TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + M * LD;
  __shared__ double red[32];
  if (sc && sc->done) return;
  const int tid = threadIdx.x;
  const size_t row0 = (size_t)blockIdx.x * NL;
  for (int e = tid; e < 2 * N; e += NT) tw[e] = ld_c<R>(twtab + e);
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int l = idx / M, i = idx % M;
    tile[i * LD + l] = ld_c<R>(in + (row0 + l) * H + i);
  }
  __syncthreads();
  const int l = tid % NL, t = tid / NL;
  c2r_prep<R, N, LD>(tile + l, t, TPL, tw);
  __syncthreads();
  fft_line<R, M, TPL, LD, +1, 4>(tile + l, t, tw);
  double2* out2 = reinterpret_cast<double2*>(out);
  AccD acc;
  for (int idx = tid; idx < M * NL; idx += NT) {
    const int ll = idx / M, i = idx % M;
    const size_t e = (row0 + ll) * H + i;
    const cx<R> v = tile[i * LD + ll];
    double2 val = make_double2(RT<R>::to_d(v.x) * scl, RT<R>::to_d(v.y) * scl);
    if constexpr (MODE == ZI_RESID) {
      const double2 sv = reinterpret_cast<const double2*>(s)[e];
      const double2 wv = reinterpret_cast<const double2*>(w)[e];
      const double2 bv = reinterpret_cast<const double2*>(b)[e];
      val.x = bv.x - (val.x + nbar * wv.x * sv.x);
      val.y = bv.y - (val.y + nbar * wv.y * sv.y);
      acc.add_prod(val.x, val.x);
      acc.add_prod(val.y, val.y);
    } else if constexpr (MODE == ZI_ACCUM) {
      const double2 o = out2[e];
      val.x += o.x;
      val.y += o.y;
    }
    out2[e] = val;
  }
  if constexpr (MODE == ZI_RESID) {
    const double sum = block_sum(acc.get(), red);
    if (tid == 0) partials[blockIdx.x] = sum;
  }
}

// ------------------------------------------------------------------------------------------
// CG update: r -= alpha q; partials [2 per block]: <r, r> (packed weights, without 1/V_c) and
// an upper estimate of V_c ||C^-1 r||^2 (the canonical residual): on column 0 the larger of
// the two planes' 1/c^2 is used.  Grid-stride; fixed grid size.
// ------------------------------------------------------------------------------------------
template <class R, int N>
__global__ void __launch_bounds__(256)
k_update(typename Store<R>::T* __restrict__ r, const typename Store<R>::T* __restrict__ q,
         const typename Store<R>::S* __restrict__ ctab, double* __restrict__ partials,
         const CgScal* __restrict__ sc) {
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  constexpr int NH = N / 2;
  __shared__ double red[32];
  if (sc->done) return;
  const SS alpha = (SS)sc->alpha;
  const size_t total = (size_t)N * N * NH;
  typename AccFor<SS>::T a_rr, a_rc;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    ST rv = r[e];
    const ST qv = q[e];
    rv.x -= alpha * qv.x;
    rv.y -= alpha * qv.y;
    r[e] = rv;
    const int kz = (int)(e % NH);
    const int ky = (int)((e / NH) % N);
    const int kx = (int)(e / ((size_t)N * NH));
    const int kxs = sfreq(kx, N), kys = sfreq(ky, N);
    const int n2 = kxs * kxs + kys * kys + kz * kz;
    SS c = ctab[n2];
    SS ic2 = (SS)1 / (c * c);
    if (kz == 0) {
      const SS cN = ctab[n2 + NH * NH];
      const SS i2 = (SS)1 / (cN * cN);
      ic2 = ic2 > i2 ? ic2 : i2;
    }
    const SS wgt = kz == 0 ? (SS)1 : (SS)2;
    const SS m2 = rv.x * rv.x + rv.y * rv.y;
    a_rr.add_prod(wgt, m2);
    a_rc.add_prod(wgt * ic2, m2);
  }
  const double s1 = block_sum(a_rr.get(), red);
  const double s2 = block_sum(a_rc.get(), red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s1;
    partials[2 * blockIdx.x + 1] = s2;
  }
}

// x += alpha_prev p (applies the last alpha after the loop ends); alpha_prev is then cleared
template <class ST>
__global__ void k_axpy_final(ST* __restrict__ x, const ST* __restrict__ p, size_t n, CgScal* sc) {
  const double a = sc->alpha_prev;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    ST xv = x[e];
    const ST pv = p[e];
    xv.x += (decltype(xv.x))a * pv.x;
    xv.y += (decltype(xv.y))a * pv.y;
    x[e] = xv;
  }
}

// ---- single-CTA finishers: fixed-order sums of the per-block partials ------------------
WF_D double sum_partials(const double* p, int n, int stride, int off, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i * stride + off];
  return block_sum(v, red);
}

// After the initial r = C b (k_xmul with DOT): rr = <r, r>; reset the recurrences.
static __global__ void k_fin_init(const double* __restrict__ partials, int n, CgScal* sc) {
  __shared__ double red[32];
  const double rr = sum_partials(partials, n, 1, 0, red);
  if (threadIdx.x == 0) {
    sc->rr = rr;
    sc->beta = 0.0;
    sc->alpha = 0.0;
    sc->alpha_prev = 0.0;
    sc->rc2 = sc->bb;
    sc->done = (rr == 0.0 || sc->bb == 0.0) ? 1 : 0;
    sc->status = 0;
  }
}

static __global__ void k_fin_alpha(const double* __restrict__ partials, int n, CgScal* sc) {
  __shared__ double red[32];
  if (sc->done) return;
  const double pq = sum_partials(partials, n, 1, 0, red);
  if (threadIdx.x == 0) {
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->done = 3;
      sc->alpha = 0.0;
      sc->alpha_prev = 0.0;
    } else {
      sc->alpha = sc->rr / pq;
    }
  }
}

// stop rule: rc2 * inv_vc <= max(tol2 * bb, rr_stop)
static __global__ void k_fin_beta(const double* __restrict__ partials, int n, double inv_vc, CgScal* sc) {
  __shared__ double red[32];
  if (sc->done) return;
  const double rr = sum_partials(partials, n, 2, 0, red);
  const double rc = sum_partials(partials, n, 2, 1, red);
  if (threadIdx.x == 0) {
    const double rc2 = rc * inv_vc;
    sc->beta = rr / sc->rr;
    sc->rr = rr;
    sc->rc2 = rc2;
    sc->alpha_prev = sc->alpha;
    sc->iter += 1;
    const double lim = fmax(sc->tol2 * sc->bb, sc->rr_stop);
    if (!isfinite(rr) || !isfinite(rc2)) sc->done = 3;
    else if (rc2 <= lim) sc->done = 1;
    else if (sc->iter >= sc->max_iter) sc->done = 2;
  }
}

// sum of partials into sc->aux[slot] (slot >= 0, host reads it) or into sc->bb (slot < 0)
static __global__ void k_fin_sum(const double* __restrict__ partials, int n, int slot, CgScal* sc) {
  __shared__ double red[32];
  const double v = sum_partials(partials, n, 1, 0, red);
  if (threadIdx.x == 0) {
    if (slot >= 0) sc->aux[slot] = v;
    else sc->bb = v;
  }
}

}  // namespace wf
