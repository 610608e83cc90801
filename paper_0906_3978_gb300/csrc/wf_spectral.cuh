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
// Passes (one CTA per tile of NL lines, or persistent CTAs walking the tiles):
//   y pass      complex FFT along y, in place (tiles moved by tensor copies)
//   x passes    multiplier(s) + complex FFT along x, fused with CG vector updates
//   z turn      packed -> C2R -> multiply by a real diagonal -> R2C -> packed (one z line)
//   z fwd/inv   real rows <-> packed spectrum rows, with epilogues
#pragma once
#include <type_traits>

#include "wf_fft.cuh"
#include "wf_tma.cuh"

namespace wf {

// Device-resident CG scalars of one system.  Written by the single-CTA finisher kernels (and by
// the host between solves).  A batch keeps one per system, indexed by blockIdx.z.
struct __align__(16) CgScal {
  double rr;          // <r, r> of the preconditioned residual
  double pq;          // <p, A p>
  double alpha;       // rr / pq of the last iteration
  double alpha_prev;  // alpha still to be applied to x (fused into the next x pass)
  double beta;
  double bb;          // ||b||^2 of the canonical system (real space)
  double rc2;         // upper estimate of the canonical ||b - A s||^2 (real space)
  double tol2;        // stop when rc2 <= tol2 * bb
  double rr_stop;     // inner solves: stop when rc2 <= rr_stop (absolute)
  double nbar;        // mean density of this system
  double aux[4];
  double rzo;         // deflated inner solves: <r, z> of the last iteration
  int iter;           // iterations since the solve began
  int max_iter;
  int done;           // 0 running; 1 converged (estimate); 2 iteration cap; 3 breakdown; 4 idle
  int status;
  int lit;            // iterations since the last reset of p: p_old = P[lit & 1]
  int defl;           // deflated inner solves: 2 start step (alpha = 1) pending, 1 first iteration
  int noco;           // deflated groups: 1 = this system runs its inner solves without the coarse space
  int pad;
};

// Distances between consecutive systems of a batch (elements of each array type).
struct Bat {
  size_t spec;  // complex elements of a spectrum
  size_t real;  // elements of a real-space field
  int tab;      // entries of a Fourier table
  int part;     // partial sums per system
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

// a table entry in the arithmetic type (no FP64 round trip when the types agree)
template <class R, class T> WF_D R tab_to(T v) {
  if constexpr (std::is_same<R, T>::value) return v;
  else return RT<R>::c((double)v);
}

// signed frequency of an index on an axis of length n
WF_D int sfreq(int j, int n) { return j <= (n >> 1) ? j : j - n; }

// Load the length-M twiddles exp(-2 pi i e / M) from a length-TN table into shared memory.  The
// table has the kernel's storage type (FP32 kernels read an FP32 copy: converting FP64 entries would
// put the start of every CTA on GB300's 1/64-rate FP64 unit).
template <class R, int M, int TN, class TT>
WF_D void load_tw(cx<R>* tw, const TT* tab, int tid, int nt) {
  for (int e = tid; e < M; e += nt) tw[e] = ld_c<R>(tab + e * (TN / M));
}

// ------------------------------------------------------------------------------------------
// Geometry of the x / y passes: a tile is M = N rows (the transform axis) by NL consecutive
// kz columns; each line is transformed by TPL threads holding E elements each, so the CTA
// has exactly NL * TPL threads.  Tiles move between global and shared memory as 16-byte
// vectors (VW elements), PER vectors per thread, fully unrolled so every load of a thread is
// in flight at once.  The shared tile has a pad column (LD = NL + 1) that also holds the
// partner line of column 0.
// ------------------------------------------------------------------------------------------
// Elements per thread: 32 (FP32) / 16 (16-byte types) on long lines, fewer on short ones so that
// a CTA still has about 128 threads.
template <class R> constexpr int max_elems() { return sizeof(cx<R>) == 8 ? 32 : 16; }
template <class R> constexpr int elems_for(int M, int NL) {
  return div_le(M, M * NL / 128 >= max_elems<R>() ? max_elems<R>() : (M * NL / 128 >= 4 ? M * NL / 128 : 4));
}

template <class R, int N, int EX = elems_for<R>(N, xy_lines<R, N>())>
struct XYG {
  using ST = typename Store<R>::T;
  static constexpr int M = N, NH = N / 2;
  static constexpr int NL = xy_lines<R, N>();
  static constexpr int E = EX;
  static constexpr int TPL = M / E >= 1 ? M / E : 1;
  static constexpr int NT = NL * TPL;
  static constexpr int LD = NL + 1;
  static constexpr int VW = (sizeof(ST) == 8 && NL % 2 == 0) ? 2 : 1;
  static constexpr int NV = NL / VW;
  static constexpr int NVEC = M * NV;
  static constexpr int PER = (NVEC + NT - 1) / NT;
  static constexpr bool EVEN = NVEC % NT == 0;
  using VT = typename std::conditional<VW == 2, float4, ST>::type;
  static constexpr size_t SMEM = (size_t)(M * LD + M) * sizeof(cx<R>);
};

template <class G, class R>
WF_D void vec_to_tile(cx<R>* tile, int i, int c0, const typename G::VT& v) {
  if constexpr (G::VW == 2) {
    const float4 f = *reinterpret_cast<const float4*>(&v);
    tile[i * G::LD + c0] = cx<R>{RT<R>::from_f(f.x), RT<R>::from_f(f.y)};
    tile[i * G::LD + c0 + 1] = cx<R>{RT<R>::from_f(f.z), RT<R>::from_f(f.w)};
  } else {
    tile[i * G::LD + c0] = ld_c<R>(&v);
  }
}
template <class G, class R>
WF_D typename G::VT tile_to_vec(const cx<R>* tile, int i, int c0) {
  typename G::VT v;
  if constexpr (G::VW == 2) {
    const cx<R> a = tile[i * G::LD + c0], b = tile[i * G::LD + c0 + 1];
    *reinterpret_cast<float4*>(&v) = make_float4(RT<R>::to_f(a.x), RT<R>::to_f(a.y), RT<R>::to_f(b.x), RT<R>::to_f(b.y));
  } else {
    st_c(&v, tile[i * G::LD + c0]);
  }
  return v;
}

// Load / store a whole tile whose element (i, l) is at g[i * rowstride + l].
template <class G, class R>
WF_D void tile_load(cx<R>* tile, const typename G::ST* g, size_t rowstride, int tid) {
  using VT = typename G::VT;
  VT buf[G::PER];
#pragma unroll
  for (int k = 0; k < G::PER; ++k) {
    const int idx = tid + k * G::NT;
    if (G::EVEN || idx < G::NVEC) {
      const int i = idx / G::NV, v = idx % G::NV;
      buf[k] = *reinterpret_cast<const VT*>(g + (size_t)i * rowstride + v * G::VW);
    }
  }
#pragma unroll
  for (int k = 0; k < G::PER; ++k) {
    const int idx = tid + k * G::NT;
    if (G::EVEN || idx < G::NVEC) vec_to_tile<G>(tile, idx / G::NV, (idx % G::NV) * G::VW, buf[k]);
  }
}
template <class G, class R>
WF_D void tile_store(const cx<R>* tile, typename G::ST* g, size_t rowstride, int tid) {
  using VT = typename G::VT;
#pragma unroll
  for (int k = 0; k < G::PER; ++k) {
    const int idx = tid + k * G::NT;
    if (G::EVEN || idx < G::NVEC) {
      const int i = idx / G::NV, v = idx % G::NV;
      *reinterpret_cast<VT*>(g + (size_t)i * rowstride + v * G::VW) = tile_to_vec<G>(tile, i, v * G::VW);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Persistent passes with tensor copies.  Geometry: a tile is M = N rows (the transform axis) by
// NL consecutive kz columns, stored densely in shared memory (row i, column l at i NL + l: a row
// is NL x 8 bytes for FP32, so two rows fill the 32 banks and a warp's row accesses need the two
// wavefronts 256 bytes take anyway).  The tensor copy moves the tile as NBOX boxes of BR rows
// (a box side is at most 256).  A CTA keeps STG tiles in flight and walks the tiles t =
// blockIdx.x, blockIdx.x + gridDim.x, ... of all systems, skipping finished ones.
// ------------------------------------------------------------------------------------------
// lines per tile of the tensor-copy passes: the largest divisor of N/2 up to the 128-byte row
// whose row and column offsets keep the copies 16-byte aligned (2 NL reals a multiple of 16 bytes)
template <class R, int N> constexpr int tma_lines() {
  int d = cmin(N / 2, tile_lines<R>());
  while (d > 1 && ((N / 2) % d != 0 || (2 * d * (int)sizeof(typename Store<R>::S)) % 16 != 0)) --d;
  return d;
}

template <class R, int N, int NL_, int STG_, int EX = elems_for<R>(N, NL_)>
struct TG {
  using ST = typename Store<R>::T;
  static constexpr int M = N, NH = N / 2, NL = NL_, STG = STG_;
  static constexpr int E = EX;  // elements per thread (a divisor of N)
  static constexpr int TPL = M / E >= 1 ? M / E : 1;
  static constexpr int NT = NL * TPL;
  static constexpr int BR = N <= 256 ? N : N / 2;  // rows per tensor box
  static constexpr int NBOX = N / BR;
  static constexpr unsigned TILE_BYTES = (unsigned)(M * NL * sizeof(ST));
  // buffers start on 128-byte boundaries (tensor copies into shared memory need that)
  static constexpr int SSTR = (int)(((TILE_BYTES + 127) / 128) * 128 / sizeof(ST));  // elements
  static constexpr int KB = NH / NL;  // kz blocks per plane
  static constexpr int TPS = KB * N;  // tiles per system
  static constexpr size_t SMEM = 128 + (size_t)STG * SSTR * sizeof(cx<R>) + (size_t)M * sizeof(cx<R>) + 16 * STG;
  static_assert(NH % NL == 0 && BR <= 256 && N % BR == 0 && N % E == 0, "tile geometry");
  static_assert((2 * NL * sizeof(typename Store<R>::S)) % 16 == 0, "16-byte aligned tensor copies");
  static_assert(NBOX == 1 || (BR * NL * sizeof(ST)) % 128 == 0, "boxes of a tile on 128-byte boundaries");
  static_assert(sizeof(cx<R>) == sizeof(ST), "tiles hold storage elements");
};

// Tile order of the persistent passes: id -> (system z, plane index a, kz block kb).
template <class G> struct TileSeq {
  const CgScal* sc;
  int total;
  WF_D bool live(int id) const { return !(sc && sc[id / G::TPS].done); }
  // the first live tile at or after id in steps of `step` (total if none)
  WF_D int next(int id, int step) const {
    while (id < total && !live(id)) id += step;
    return id < total ? id : total;
  }
};

// Wait (bounded) for the tile in buffer s; returns false for every thread if any thread timed
// out, after reporting it in *err.  Must be called by all threads.
// (A thread whose own wait completed has consumed that phase: its parity bit flips and the buffer
// leaves its `pending` set.)
template <int STG>
WF_D bool tile_arrived(uint64_t* bar, int s, unsigned& phase, unsigned& pending, int* err) {
  const bool mine = mbar_wait(&bar[s], (phase >> s) & 1u);
  if (mine) {
    phase ^= 1u << s;
    pending &= ~(1u << s);
  }
  const bool bad = __syncthreads_or(!mine);
  if (bad && threadIdx.x == 0 && err) atomicExch(err, 1);
  return !bad;
}

// Before the CTA exits: wait for its stores, and after a timeout also (bounded) for the loads
// still in flight into its buffers.  Thread 0 only.
template <int STG>
WF_D void tiles_drain(uint64_t* bar, unsigned phase, unsigned pending, bool ok) {
  if (!ok)
    for (int j = 0; j < STG; ++j)
      if ((pending >> j) & 1u) (void)mbar_wait(&bar[j], (phase >> j) & 1u);
  bulk_wait<0>();
}

// y pass with tensor copies: complex FFT along y of every (x, kz) line, in place.  The map covers
// the spectra with box {2 NL, BR, 1, 1} (rows = y).  grid: persistent.
// RMAX caps the radix of the transform's stages (8, 16 or 32: larger radices take fewer
// shared-memory round trips and more registers).
template <class R, int N, int DIR, int NL, int STG, int RMAX>
__global__ void __launch_bounds__(TG<R, N, NL, STG>::NT)
k_ypass_tma(const __grid_constant__ CUtensorMap tm, const typename Store<R>::T* __restrict__ twtab,
            const CgScal* __restrict__ sc, int nb, int* __restrict__ err) {
  using G = TG<R, N, NL, STG>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
  cx<R>* tw = buf + STG * G::SSTR;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tw + G::M);
  const int tid = threadIdx.x;
  const TileSeq<G> seq{sc, nb * G::TPS};
  if (tid == 0) {
    prefetch_tensormap(&tm);
    for (int s = 0; s < STG; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  load_tw<R, G::M, 2 * N>(tw, twtab, tid, G::NT);
  auto issue = [&](int id, int s) {
    const int z = id / G::TPS, rem = id % G::TPS, x = rem / G::KB, kz0 = (rem % G::KB) * NL;
    mbar_expect_tx(&bar[s], G::TILE_BYTES);
    for (int q = 0; q < G::NBOX; ++q) tma_load_4d(buf + s * G::SSTR + q * G::BR * NL, &tm, 2 * kz0, q * G::BR, x, z, &bar[s]);
  };
  // the tiles of this CTA, STG - 1 of them loading ahead of the one being transformed
  int ids[STG];
  ids[0] = seq.next(blockIdx.x, gridDim.x);
  for (int j = 1; j < STG; ++j) ids[j] = seq.next(ids[j - 1] < seq.total ? ids[j - 1] + gridDim.x : seq.total, gridDim.x);
  unsigned pending = 0;  // buffers with a load in flight (thread 0's view)
  if (tid == 0)
    for (int j = 0; j < STG - 1; ++j)
      if (ids[j] < seq.total) {
        issue(ids[j], j);
        pending |= 1u << j;
      }
  unsigned phase = 0;
  bool ok = true;
  for (int k = 0; ids[0] < seq.total; ++k) {
    const int s = k % STG;
    // refill the buffer the previous tile used (its store must have finished reading it)
    if (tid == 0 && ids[STG - 1] < seq.total) {
      bulk_wait_read<0>();
      issue(ids[STG - 1], (k + STG - 1) % STG);
      pending |= 1u << ((k + STG - 1) % STG);
    }
    ok = tile_arrived<STG>(bar, s, phase, pending, err);
    if (!ok) break;
    cx<R>* tile = buf + s * G::SSTR;
    fft_line<R, G::M, G::TPL, NL, DIR, 1, cmin(RMAX, rmax_for(G::M, G::TPL))>(tile + tid % NL, tid / NL, tw);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      const int id = ids[0];
      const int z = id / G::TPS, rem = id % G::TPS, x = rem / G::KB, kz0 = (rem % G::KB) * NL;
      for (int q = 0; q < G::NBOX; ++q) tma_store_4d(&tm, 2 * kz0, q * G::BR, x, z, tile + q * G::BR * NL);
      bulk_commit();
    }
    for (int j = 0; j < STG - 1; ++j) ids[j] = ids[j + 1];
    ids[STG - 1] = seq.next(ids[STG - 2] < seq.total ? ids[STG - 2] + gridDim.x : seq.total, gridDim.x);
  }
  if (tid == 0) tiles_drain<STG>(bar, phase, pending, ok);
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
    const R m0 = tab_to<R>(tab[n2]);
    const R mN = tab_to<R>(tab[n2 + NH * NH]);
    const R h = RT<R>::c(0.5);
    const R a = (m0 + mN) * h, b = (m0 - mN) * h;
    const cx<R> z = tile[kx * LD];
    const cx<R> zp = conj(tile[((N - kx) % N) * LD + NL]);
    tile[kx * LD] = scale(z, a) + scale(zp, b);
  }
  __syncthreads();
}

// Multiply every tile element except column 0 of the kz0 = 0 tile by tab[n2].
template <class G, class R, class TAB>
WF_D void tile_mul(cx<R>* tile, int kz0, int ky_s, const TAB* tab, int tid) {
  for (int idx = tid; idx < G::M * G::NL; idx += G::NT) {
    const int i = idx / G::NL, l = idx % G::NL, kz = kz0 + l;
    if (kz == 0) continue;
    const int kxs = sfreq(i, G::M);
    tile[i * G::LD + l] = scale(tile[i * G::LD + l], tab_to<R>(tab[kxs * kxs + ky_s * ky_s + kz * kz]));
  }
}

// ------------------------------------------------------------------------------------------
// CG x pass 1 (start of A p):  p_new = r + beta p_old;  x += alpha_prev p_old;
//                              T = IFFT_x( c (.) p_new );  partial of <p_new, m p_new>
// grid (N/2 / NL, N).  <p, A p> = <p, m p> + <c p, D (c p)>: the first term is summed here,
// where p_new is formed, the second by the z turn, where the real field of c p is at hand.
// For the packed column the m term is m0 |P0|^2 + mN |PN|^2 of the two planes it holds,
// P0 = (Z + conj Z(-k)) / 2 and PN = (Z - conj Z(-k)) / 2i (Z(-k) from the partner line).
// UNIT_M: m = 1 at every k != 0 (the preconditioned system), so m is read only on column 0.
// ------------------------------------------------------------------------------------------
template <class R, int N, bool UNIT_M, int RMAX = 8, int MINB = 0>
__global__ void __launch_bounds__(XYG<R, N>::NT, MINB)
k_cg_xinv(const typename Store<R>::T* __restrict__ r, typename Store<R>::T* P0, typename Store<R>::T* P1,
          typename Store<R>::T* __restrict__ x, typename Store<R>::T* __restrict__ T,
          const typename Store<R>::S* __restrict__ ctab, const typename Store<R>::S* __restrict__ mtab,
          const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials, const CgScal* __restrict__ sc,
          Bat bt) {
  using G = XYG<R, N>;
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  using VT = typename G::VT;
  constexpr int NH = G::NH;
  static_assert(std::is_same<R, SS>::value, "the CG passes compute in their storage type");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::M * G::LD;
  __shared__ double red[32];
  const int z = blockIdx.z;
  sc += z;
  if (sc->done) return;
  // p_old / p_new alternate between P0 and P1 with this system's iteration count
  const ST* __restrict__ pold = ((sc->lit & 1) ? P1 : P0) + z * bt.spec;
  ST* __restrict__ pnew = ((sc->lit & 1) ? P0 : P1) + z * bt.spec;
  r += z * bt.spec;
  x += z * bt.spec;
  T += z * bt.spec;
  ctab += z * bt.tab;
  mtab += z * bt.tab;
  partials += z * bt.part;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * G::NL, ky = blockIdx.y;
  const int ky_s = sfreq(ky, N);
  const SS beta = (SS)sc->beta, alpha_prev = (SS)sc->alpha_prev;
  load_tw<R, G::M, 2 * N>(tw, twtab, tid, G::NT);
  const size_t rowstride = (size_t)N * NH;
  const size_t base = (size_t)ky * NH + kz0;
  typename AccFor<SS>::T acc;  // <p_new, m p_new> over the columns kz != 0 (weight 2)
  constexpr int CH = 4;  // vectors per thread whose three loads are in flight together
  constexpr int SPV = sizeof(VT) / sizeof(SS);
#pragma unroll
  for (int k0 = 0; k0 < G::PER; k0 += CH) {
    VT rv[CH], pv[CH], xv[CH];
    SS cv[CH][G::VW], mv[CH][G::VW];
#pragma unroll
    for (int k = 0; k < CH && k0 + k < G::PER; ++k) {
      const int idx = tid + (k0 + k) * G::NT;
      if (G::EVEN || idx < G::NVEC) {
        const int i = idx / G::NV, c0 = (idx % G::NV) * G::VW;
        const size_t e = base + (size_t)i * rowstride + c0;
        rv[k] = *reinterpret_cast<const VT*>(r + e);
        pv[k] = *reinterpret_cast<const VT*>(pold + e);
        xv[k] = *reinterpret_cast<const VT*>(x + e);
        const int kxs = sfreq(i, N);
#pragma unroll
        for (int u = 0; u < G::VW; ++u) {
          const int kz = kz0 + c0 + u;
          const int n2 = kxs * kxs + ky_s * ky_s + kz * kz;
          cv[k][u] = ctab[n2];
          mv[k][u] = UNIT_M ? (SS)1 : mtab[n2];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CH && k0 + k < G::PER; ++k) {
      const int idx = tid + (k0 + k) * G::NT;
      if (G::EVEN || idx < G::NVEC) {
        const int i = idx / G::NV, c0 = (idx % G::NV) * G::VW;
        const size_t e = base + (size_t)i * rowstride + c0;
        SS* rs = reinterpret_cast<SS*>(&rv[k]);
        SS* ps = reinterpret_cast<SS*>(&pv[k]);
        SS* xs = reinterpret_cast<SS*>(&xv[k]);
        VT nv;
        SS* ns = reinterpret_cast<SS*>(&nv);
#pragma unroll
        for (int q = 0; q < SPV; ++q) {
          ns[q] = rs[q] + beta * ps[q];
          xs[q] = xs[q] + alpha_prev * ps[q];
        }
        *reinterpret_cast<VT*>(pnew + e) = nv;
        *reinterpret_cast<VT*>(x + e) = xv[k];
        // the tile gets c (.) p_new; column kz = 0 stays raw for the packed-column combine.  The
        // terms of <p, m p> are >= 0, so a vector's few terms are summed in the storage type
        // before entering the accumulator.
        SS part = 0;
#pragma unroll
        for (int u = 0; u < G::VW; ++u)
          if (kz0 + c0 + u != 0) {
            part += (SS)2 * mv[k][u] * (ns[2 * u] * ns[2 * u] + ns[2 * u + 1] * ns[2 * u + 1]);
            ns[2 * u] *= cv[k][u];
            ns[2 * u + 1] *= cv[k][u];
          }
        acc.add(part);
        vec_to_tile<G>(tile, i, c0, nv);
      }
    }
  }
  if (kz0 == 0) {  // partner line of column 0: p_new at (kx, -ky, 0), recomputed from inputs
    const size_t pb = (size_t)((N - ky) % N) * NH;
    for (int i = tid; i < G::M; i += G::NT) {
      const size_t e = pb + (size_t)i * rowstride;
      const ST rv = r[e], po = pold[e];
      ST pn;
      pn.x = rv.x + beta * po.x;
      pn.y = rv.y + beta * po.y;
      tile[i * G::LD + G::NL] = ld_c<R>(&pn);
    }
  }
  __syncthreads();
  if (kz0 == 0) {
    // m term of the packed column (weight 1), from the raw column and its partner line
    for (int kx = tid; kx < N; kx += G::NT) {
      const int kxs = sfreq(kx, N);
      const int n2 = kxs * kxs + ky_s * ky_s;
      const cx<R> zc = tile[kx * G::LD];
      const cx<R> zp = tile[((N - kx) % N) * G::LD + G::NL];
      const SS zr = (SS)zc.x, zi = (SS)zc.y, pr = (SS)zp.x, pi = (SS)zp.y;  // R is the storage type
      const SS h = (SS)0.5;
      const SS a0 = h * (zr + pr), b0 = h * (zi - pi);  // P0
      const SS aN = h * (zi + pi), bN = h * (pr - zr);  // PN
      const SS m0 = mtab[n2], mN = mtab[n2 + NH * NH];
      acc.add(m0 * (a0 * a0 + b0 * b0) + mN * (aN * aN + bN * bN));
    }
    combine_col0<R, N, G::LD, G::NL>(tile, ky_s, ctab, tid, G::NT);
  }
  fft_line<R, G::M, G::TPL, G::LD, +1, 1, cmin(RMAX, rmax_for(G::M, G::TPL))>(tile + tid % G::NL, tid / G::NL, tw);
  tile_store<G>(tile, T + base, rowstride, tid);
  const double sum = block_sum(acc.get(), red);
  if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = sum;
}

// ------------------------------------------------------------------------------------------
// CG x pass 2 (end of A p) fused with the CG update:
//   T^ = FFT_x(T);  q = m p + c T^;  r -= alpha q;  partials of <r, r> and ||C^-1 r||^2.
// alpha = rr / <p, A p> is already known: both terms of <p, A p> were summed by the first x pass
// and the z turn, and the finisher ran before this pass.  So q never goes to memory: the pass
// reads T, p and r and writes r (4 spectra), where a separate transform and update sweep moved 6.
// On the packed column c is applied to T^ as a pair (it needs the partner line -ky), and the m term
// combines p with its partner element p(-kx, -ky, 0).  partials [2 per block]: <r, r> (packed
// weights, without 1/V_c) and an upper estimate of V_c ||C^-1 r||^2 (the canonical residual): on
// column 0 the larger of the two planes' 1/c^2 is used.  grid (N/2 / NL, N).
// ------------------------------------------------------------------------------------------
template <class R, int N, bool UNIT_M, int RMAX = 8, int MINB = 0>
__global__ void __launch_bounds__(XYG<R, N>::NT, MINB)
k_cg_xupd(const typename Store<R>::T* __restrict__ T, typename Store<R>::T* __restrict__ r,
          const typename Store<R>::T* P0, const typename Store<R>::T* P1,
          const typename Store<R>::S* __restrict__ ctab, const typename Store<R>::S* __restrict__ mtab,
          const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials,
          const CgScal* __restrict__ sc, Bat bt) {
  using G = XYG<R, N>;
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  using VT = typename G::VT;
  constexpr int NH = G::NH;
  static_assert(std::is_same<R, SS>::value, "the CG passes compute in their storage type");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::M * G::LD;
  __shared__ double red[32];
  const int z = blockIdx.z;
  sc += z;
  if (sc->done) return;
  const ST* __restrict__ p = ((sc->lit & 1) ? P0 : P1) + z * bt.spec;  // this iteration's p_new
  T += z * bt.spec;
  r += z * bt.spec;
  ctab += z * bt.tab;
  mtab += z * bt.tab;
  partials += z * bt.part;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * G::NL, ky = blockIdx.y;
  const int ky_s = sfreq(ky, N);
  const int pky = (N - ky) % N;
  const SS alpha = (SS)sc->alpha;
  load_tw<R, G::M, 2 * N>(tw, twtab, tid, G::NT);
  const size_t rowstride = (size_t)N * NH;
  const size_t base = (size_t)ky * NH + kz0;
  tile_load<G>(tile, T + base, rowstride, tid);
  if (kz0 == 0)
    for (int i = tid; i < G::M; i += G::NT) tile[i * G::LD + G::NL] = ld_c<R>(T + (size_t)pky * NH + (size_t)i * rowstride);
  __syncthreads();
  fft_line<R, G::M, G::TPL, G::LD, -1, 1, cmin(RMAX, rmax_for(G::M, G::TPL))>(tile + tid % G::NL, tid / G::NL, tw);
  if (kz0 == 0) {  // transform the partner line too, then apply c to column 0 as a packed pair
    fft_line<R, G::M, G::TPL, G::LD, -1, 1, cmin(RMAX, rmax_for(G::M, G::TPL))>(tile + G::NL, tid / G::NL, tw,
                                                                                 tid % G::NL == 0);
    combine_col0<R, N, G::LD, G::NL>(tile, ky_s, ctab, tid, G::NT);
  }
  // epilogue: r -= alpha (m p + c T^), vector by vector in the tile's row layout
  typename AccFor<SS>::T a_rr, a_rc;
  constexpr int CH = 4;  // vectors per thread whose two loads are in flight together
  constexpr int SPV = sizeof(VT) / sizeof(SS);
#pragma unroll
  for (int k0 = 0; k0 < G::PER; k0 += CH) {
    VT rv[CH], pv[CH];
#pragma unroll
    for (int k = 0; k < CH && k0 + k < G::PER; ++k) {
      const int idx = tid + (k0 + k) * G::NT;
      if (G::EVEN || idx < G::NVEC) {
        const int i = idx / G::NV, c0 = (idx % G::NV) * G::VW;
        const size_t e = base + (size_t)i * rowstride + c0;
        rv[k] = *reinterpret_cast<const VT*>(r + e);
        pv[k] = *reinterpret_cast<const VT*>(p + e);
      }
    }
#pragma unroll
    for (int k = 0; k < CH && k0 + k < G::PER; ++k) {
      const int idx = tid + (k0 + k) * G::NT;
      if (G::EVEN || idx < G::NVEC) {
        const int i = idx / G::NV, c0 = (idx % G::NV) * G::VW;
        const size_t e = base + (size_t)i * rowstride + c0;
        SS* rs = reinterpret_cast<SS*>(&rv[k]);
        const SS* ps = reinterpret_cast<const SS*>(&pv[k]);
        const int kxs = sfreq(i, N);
        SS s_rr = 0, s_rc = 0;
#pragma unroll
        for (int u = 0; u < G::VW; ++u) {
          const int kz = kz0 + c0 + u;
          const int n2 = kxs * kxs + ky_s * ky_s + kz * kz;
          const cx<R> t = tile[i * G::LD + c0 + u];
          const SS c = ctab[n2];
          SS ic2 = (SS)1 / (c * c);
          SS q0, q1;
          if (kz == 0) {
            // packed column: T^ already carries c; the m term combines p with p(-kx, -ky, 0) (in the
            // storage type: FP64 here would run on GB300's 1/64-rate unit)
            const SS cN = ctab[n2 + NH * NH];
            const SS i2 = (SS)1 / (cN * cN);
            ic2 = ic2 > i2 ? ic2 : i2;
            const SS m0 = mtab[n2], mN = mtab[n2 + NH * NH];
            const SS a = (SS)0.5 * (m0 + mN), b = (SS)0.5 * (m0 - mN);
            ST pp = ST{};
            if (b != (SS)0) pp = p[(size_t)((N - i) % N) * rowstride + (size_t)pky * NH];
            q0 = a * ps[2 * u] + b * pp.x + (SS)t.x;
            q1 = a * ps[2 * u + 1] - b * pp.y + (SS)t.y;
          } else {
            const SS m = UNIT_M ? (SS)1 : mtab[n2];
            q0 = m * ps[2 * u] + c * (SS)t.x;
            q1 = m * ps[2 * u + 1] + c * (SS)t.y;
          }
          rs[2 * u] -= alpha * q0;
          rs[2 * u + 1] -= alpha * q1;
          const SS wgt = kz == 0 ? (SS)1 : (SS)2;
          const SS m2 = wgt * (rs[2 * u] * rs[2 * u] + rs[2 * u + 1] * rs[2 * u + 1]);
          s_rr += m2;
          s_rc += ic2 * m2;
        }
        (void)SPV;
        *reinterpret_cast<VT*>(r + e) = rv[k];
        // the terms are >= 0: a vector's terms are summed in the storage type first
        a_rr.add(s_rr);
        a_rc.add(s_rc);
      }
    }
  }
  const double s1 = block_sum(a_rr.get(), red);
  const double s2 = block_sum(a_rc.get(), red);
  if (tid == 0) {
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    partials[2 * bid] = s1;
    partials[2 * bid + 1] = s2;
  }
}

// ------------------------------------------------------------------------------------------
// CG x pass 2 with its r and p tiles prefetched: the same work as k_cg_xupd, but the tile's r and p
// rows are requested (per-thread asynchronous 16-byte copies into shared memory) before T is loaded
// and transformed, so the epilogue reads them from shared memory instead of waiting on HBM.  One
// tile per CTA, NL lines (8 leaves shared memory for two CTAs per SM).  grid (N/2 / NL, N).
// ------------------------------------------------------------------------------------------
template <class R, int N, int NL_, int EX>
struct XYP {
  using ST = typename Store<R>::T;
  static constexpr int M = N, NH = N / 2, NL = NL_;
  static constexpr int E = EX;
  static constexpr int TPL = M / E >= 1 ? M / E : 1;
  static constexpr int NT = NL * TPL;
  static constexpr int LD = NL + 1;  // padded transform tile
  static constexpr int VW = (sizeof(ST) == 8 && NL % 2 == 0) ? 2 : 1;
  static constexpr int NV = NL / VW;
  static constexpr int NVEC = M * NV;
  static constexpr int PER = (NVEC + NT - 1) / NT;
  static constexpr bool EVEN = NVEC % NT == 0;
  using VT = typename std::conditional<VW == 2, float4, ST>::type;
  // transform tile, twiddles, then the dense r and p tiles (16-byte aligned)
  static constexpr size_t TILE = (size_t)M * LD * sizeof(cx<R>), TWB = (size_t)M * sizeof(cx<R>);
  static constexpr size_t OFF_R = ((TILE + TWB + 127) / 128) * 128;
  static constexpr size_t DENSE = (size_t)M * NL * sizeof(ST);
  static constexpr size_t SMEM = OFF_R + 2 * DENSE;
  static_assert(NH % NL == 0 && (NL * sizeof(ST)) % 16 == 0, "whole 16-byte pieces per row");
};

template <class R, int N, bool UNIT_M, int RMAX, int NL, int EX>
__global__ void __launch_bounds__(XYP<R, N, NL, EX>::NT)
k_cg_xupd_pf(const typename Store<R>::T* __restrict__ T, typename Store<R>::T* __restrict__ r,
             const typename Store<R>::T* P0, const typename Store<R>::T* P1,
             const typename Store<R>::S* __restrict__ ctab, const typename Store<R>::S* __restrict__ mtab,
             const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials,
             const CgScal* __restrict__ sc, Bat bt) {
  using G = XYP<R, N, NL, EX>;
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  constexpr int NH = G::NH;
  static_assert(std::is_same<R, SS>::value, "the CG passes compute in their storage type");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::M * G::LD;
  cx<R>* rt = reinterpret_cast<cx<R>*>(smem_raw + G::OFF_R);  // r rows, dense
  cx<R>* pt = rt + G::M * NL;                                  // p rows, dense
  __shared__ double red[32];
  const int z = blockIdx.z;
  sc += z;
  if (sc->done) return;
  const ST* __restrict__ p = ((sc->lit & 1) ? P0 : P1) + z * bt.spec;  // this iteration's p_new
  T += z * bt.spec;
  r += z * bt.spec;
  ctab += z * bt.tab;
  mtab += z * bt.tab;
  partials += z * bt.part;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * NL, ky = blockIdx.y;
  const int ky_s = sfreq(ky, N);
  const int pky = (N - ky) % N;
  const size_t rowstride = (size_t)N * NH;
  const size_t base = (size_t)ky * NH + kz0;
  // r and p rows first: they arrive while T is loaded and transformed
  {
    constexpr int PV = 16 / (int)sizeof(ST), NVR = NL / PV;
    for (int idx = tid; idx < G::M * NVR; idx += G::NT) {
      const int i = idx / NVR, v = (idx % NVR) * PV;
      cp_async16(rt + i * NL + v, r + base + (size_t)i * rowstride + v);
      cp_async16(pt + i * NL + v, p + base + (size_t)i * rowstride + v);
    }
    cp_async_commit();
  }
  const SS alpha = (SS)sc->alpha;
  load_tw<R, G::M, 2 * N>(tw, twtab, tid, G::NT);
  tile_load<G>(tile, T + base, rowstride, tid);
  if (kz0 == 0)
    for (int i = tid; i < G::M; i += G::NT) tile[i * G::LD + NL] = ld_c<R>(T + (size_t)pky * NH + (size_t)i * rowstride);
  __syncthreads();
  fft_line<R, G::M, G::TPL, G::LD, -1, 1, cmin(RMAX, rmax_for(G::M, G::TPL))>(tile + tid % NL, tid / NL, tw);
  if (kz0 == 0) {  // transform the partner line too, then apply c to column 0 as a packed pair
    fft_line<R, G::M, G::TPL, G::LD, -1, 1, cmin(RMAX, rmax_for(G::M, G::TPL))>(tile + NL, tid / NL, tw,
                                                                                 tid % NL == 0);
    combine_col0<R, N, G::LD, NL>(tile, ky_s, ctab, tid, G::NT);
  }
  cp_async_wait<0>();
  __syncthreads();
  // epilogue: r -= alpha (m p + c T^), two elements of a row per step, stored as one vector
  typename AccFor<SS>::T a_rr, a_rc;
  constexpr int W = G::VW;
#pragma unroll 4
  for (int idx = tid; idx < G::M * (NL / W); idx += G::NT) {
    const int i = idx / (NL / W), c0 = (idx % (NL / W)) * W;
    const int kxs = sfreq(i, N);
    cx<R> out[W];
    SS s_rr = 0, s_rc = 0;
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const int kz = kz0 + c0 + u;
      const int n2 = kxs * kxs + ky_s * ky_s + kz * kz;
      const cx<R> t = tile[i * G::LD + c0 + u], pv = pt[i * NL + c0 + u];
      cx<R> rv = rt[i * NL + c0 + u];
      const SS c = ctab[n2];
      SS ic2 = (SS)1 / (c * c);
      SS q0, q1;
      if (kz == 0) {
        const SS cN = ctab[n2 + NH * NH];
        const SS i2 = (SS)1 / (cN * cN);
        ic2 = ic2 > i2 ? ic2 : i2;
        const SS m0 = mtab[n2], mN = mtab[n2 + NH * NH];
        const SS a = (SS)0.5 * (m0 + mN), b = (SS)0.5 * (m0 - mN);
        ST pp = ST{};
        if (b != (SS)0) pp = p[(size_t)((N - i) % N) * rowstride + (size_t)pky * NH];
        q0 = a * pv.x + b * pp.x + t.x;
        q1 = a * pv.y - b * pp.y + t.y;
      } else {
        const SS m = UNIT_M ? (SS)1 : mtab[n2];
        q0 = m * pv.x + c * t.x;
        q1 = m * pv.y + c * t.y;
      }
      rv.x -= alpha * q0;
      rv.y -= alpha * q1;
      out[u] = rv;
      const SS wgt = kz == 0 ? (SS)1 : (SS)2;
      const SS m2 = wgt * (rv.x * rv.x + rv.y * rv.y);
      s_rr += m2;
      s_rc += ic2 * m2;
    }
    *reinterpret_cast<typename G::VT*>(r + base + (size_t)i * rowstride + c0) = *reinterpret_cast<const typename G::VT*>(out);
    a_rr.add(s_rr);
    a_rc.add(s_rc);
  }
  const double s1 = block_sum(a_rr.get(), red);
  const double s2 = block_sum(a_rc.get(), red);
  if (tid == 0) {
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    partials[2 * bid] = s1;
    partials[2 * bid + 1] = s2;
  }
}

// ------------------------------------------------------------------------------------------
// Persistent CG x passes with tensor copies.  A stage holds NS tiles (one per staged stream), all
// loaded by tensor copies along x (box {2 NL, 1, BR, 1}) and completed on the stage's barrier.
// The packed column's partner line (-ky) is read with plain loads into its own buffer, only by
// the tiles that hold column kz = 0.  Partial sums are written per tile, at index
// ky * (N/2 / NL) + kz0 / NL of the system, so the finishers sum them in a fixed order.
// ------------------------------------------------------------------------------------------
// lines per tile of the staged x passes: the largest divisor of N/2 up to the 128-byte row that
// keeps the copies 16-byte aligned and lets STG stages of NS tiles fit in shared memory
template <class R, int N, int NS, int STG> constexpr int xtma_lines() {
  int d = cmin(N / 2, tile_lines<R>());
  while (d > 1 && ((N / 2) % d != 0 || (2 * d * (int)sizeof(typename Store<R>::S)) % 16 != 0 ||
                   (long)STG * NS * N * d * (long)sizeof(cx<R>) + 2L * N * (long)sizeof(cx<R>) > 200L * 1024))
    --d;
  return d;
}

// shared memory of a staged x pass: STG stages of NS tiles, the twiddles, the partner line, one
// tile of Fourier-table entries and the barriers
template <class R, int N, int NL, int STG, int NS>
struct TXG {
  using G = TG<R, N, NL, STG>;
  static constexpr size_t SMEM = 128 + (size_t)STG * NS * G::SSTR * sizeof(cx<R>) + 2 * (size_t)N * sizeof(cx<R>) +
                                 (size_t)N * NL * sizeof(typename Store<R>::S) + 16 * STG;
};

// Row copies of a dense x-pass tile (M rows of NL elements, row i at g + i rowstride) as 16-byte
// pieces, each thread a fixed share: per-thread asynchronous copies in, plain vector stores out.
template <class G, class R, class ST>
WF_D void tile_rows_async(cx<R>* tile, const ST* g, size_t rowstride, int tid) {
  constexpr int VW = 16 / (int)sizeof(ST), NV = G::NL / VW, NVEC = G::M * NV;
  static_assert(G::NL % VW == 0, "whole 16-byte pieces per row");
#pragma unroll 4
  for (int idx = tid; idx < NVEC; idx += G::NT) {
    const int i = idx / NV, v = (idx % NV) * VW;
    cp_async16(tile + i * G::NL + v, g + (size_t)i * rowstride + v);
  }
}
template <class G, class R, class ST>
WF_D void tile_rows_store(const cx<R>* tile, ST* g, size_t rowstride, int tid) {
  constexpr int VW = 16 / (int)sizeof(ST), NV = G::NL / VW, NVEC = G::M * NV;
#pragma unroll 4
  for (int idx = tid; idx < NVEC; idx += G::NT) {
    const int i = idx / NV, v = (idx % NV) * VW;
    *reinterpret_cast<float4*>(g + (size_t)i * rowstride + v) = *reinterpret_cast<const float4*>(tile + i * G::NL + v);
  }
}

// The multiplier pair of the packed column (slot 0 of each row) with its partner line held in
// `part` (element kx at part[kx]).  Must be called by all threads; synchronises.
template <class R, int N, int LD, class TAB>
WF_D void combine_col0_sep(cx<R>* tile, const cx<R>* part, int ky_s, const TAB* tab, int tid, int nt) {
  constexpr int NH = N / 2;
  for (int kx = tid; kx < N; kx += nt) {
    const int kxs = sfreq(kx, N);
    const int n2 = kxs * kxs + ky_s * ky_s;
    const R m0 = tab_to<R>(tab[n2]);
    const R mN = tab_to<R>(tab[n2 + NH * NH]);
    const R h = RT<R>::c(0.5);
    const R a = (m0 + mN) * h, b = (m0 - mN) * h;
    const cx<R> zc = tile[kx * LD];
    const cx<R> zp = conj(part[(N - kx) % N]);
    tile[kx * LD] = scale(zc, a) + scale(zp, b);
  }
  __syncthreads();
}

// x pass 1, staged (the work of k_cg_xinv):  p_new = r + beta p_old;  x += alpha_prev p_old;
// T = IFFT_x(c (.) p_new);  partial of <p_new, m p_new>.  Stage tiles: r (becomes p_new), p_old
// (becomes c p_new, then T), x.  COPY 0: tensor copies (maps mR, mP0, mP1, mX, mT) completed on
// the stage's barrier, tensor stores; COPY 1: per-thread asynchronous row copies completed by
// copy groups, plain stores (the maps are unused).
template <class R, int N, bool UNIT_M, int NL, int STG, int RMAX, int EX, int COPY>
__global__ void __launch_bounds__(TG<R, N, NL, STG, EX>::NT)
k_cg_xinv_tma(const __grid_constant__ CUtensorMap mR, const __grid_constant__ CUtensorMap mP0,
              const __grid_constant__ CUtensorMap mP1, const __grid_constant__ CUtensorMap mX,
              const __grid_constant__ CUtensorMap mT, const typename Store<R>::T* __restrict__ r,
              typename Store<R>::T* P0, typename Store<R>::T* P1, typename Store<R>::T* __restrict__ xg,
              typename Store<R>::T* __restrict__ Tg,
              const typename Store<R>::S* __restrict__ ctab, const typename Store<R>::S* __restrict__ mtab,
              const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials,
              const CgScal* __restrict__ sc, Bat bt, int nb, int* __restrict__ err) {
  using G = TG<R, N, NL, STG, EX>;
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  constexpr int NS = 3, M = N, NH = N / 2;
  static_assert(std::is_same<R, SS>::value, "the CG passes compute in their storage type");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[32];
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
  cx<R>* tw = buf + STG * NS * G::SSTR;
  cx<R>* pl = tw + M;  // partner line of the packed column
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<typename Store<R>::S*>(pl + M) + M * NL);
  const int tid = threadIdx.x;
  const TileSeq<G> seq{sc, nb * G::TPS};
  if (tid == 0) {
    prefetch_tensormap(&mR);
    prefetch_tensormap(&mX);
    prefetch_tensormap(&mT);
    for (int s = 0; s < STG; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  load_tw<R, M, 2 * N>(tw, twtab, tid, G::NT);
  const size_t rowstride = (size_t)N * NH;
  auto issue = [&](int id, int s) {
    const int z = id / G::TPS, rem = id % G::TPS, ky = rem / G::KB, kz0 = (rem % G::KB) * NL;
    if constexpr (COPY == 0) {
      const CUtensorMap* mpo = (sc[z].lit & 1) ? &mP1 : &mP0;  // p_old
      mbar_expect_tx(&bar[s], NS * G::TILE_BYTES);
      for (int q = 0; q < G::NBOX; ++q) {
        const int off = q * G::BR * NL;
        tma_load_4d(buf + (s * NS + 0) * G::SSTR + off, &mR, 2 * kz0, ky, q * G::BR, z, &bar[s]);
        tma_load_4d(buf + (s * NS + 1) * G::SSTR + off, mpo, 2 * kz0, ky, q * G::BR, z, &bar[s]);
        tma_load_4d(buf + (s * NS + 2) * G::SSTR + off, &mX, 2 * kz0, ky, q * G::BR, z, &bar[s]);
      }
    } else {
      const size_t o = z * bt.spec + (size_t)ky * NH + kz0;
      const ST* po = ((sc[z].lit & 1) ? P1 : P0) + o;
      tile_rows_async<G>(buf + (s * NS + 0) * G::SSTR, r + o, rowstride, tid);
      tile_rows_async<G>(buf + (s * NS + 1) * G::SSTR, po, rowstride, tid);
      tile_rows_async<G>(buf + (s * NS + 2) * G::SSTR, xg + o, rowstride, tid);
    }
  };
  int ids[STG];
  ids[0] = seq.next(blockIdx.x, gridDim.x);
  for (int j = 1; j < STG; ++j) ids[j] = seq.next(ids[j - 1] < seq.total ? ids[j - 1] + gridDim.x : seq.total, gridDim.x);
  unsigned pending = 0, phase = 0;
  for (int j = 0; j < STG - 1; ++j) {
    if (COPY == 0 && tid == 0 && ids[j] < seq.total) {
      issue(ids[j], j);
      pending |= 1u << j;
    }
    if constexpr (COPY == 1) {
      if (ids[j] < seq.total) issue(ids[j], j);
      cp_async_commit();
    }
  }
  // Fourier-table entries of this thread's elements, one tile ahead: the next tile's are gathered
  // while the current one is processed, so their latency overlaps the work
  constexpr int PER = G::E;  // elements per thread: M NL / NT
  SS cv[PER], mv[PER], cn[PER], mn[PER];
  auto gather = [&](int id, SS* c, SS* m) {
    const int z = id / G::TPS, rem = id % G::TPS, ky = rem / G::KB, kz0 = (rem % G::KB) * NL;
    const int ky_s = sfreq(ky, N);
    const SS* ctz = ctab + z * bt.tab;
    const SS* mtz = mtab + z * bt.tab;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = tid + k * G::NT, i = e / NL, kz = kz0 + e % NL;
      const int kxs = sfreq(i, N);
      const int n2 = kxs * kxs + ky_s * ky_s + kz * kz;
      c[k] = ctz[n2];
      m[k] = UNIT_M ? (SS)1 : mtz[n2];
    }
  };
  if (ids[0] < seq.total) gather(ids[0], cv, mv);
  bool ok = true;
  for (int k = 0; ids[0] < seq.total; ++k) {
    const int s = k % STG;
    if constexpr (COPY == 0) {
      if (tid == 0 && ids[STG - 1] < seq.total) {
        bulk_wait_read<0>();
        issue(ids[STG - 1], (k + STG - 1) % STG);
        pending |= 1u << ((k + STG - 1) % STG);
      }
    } else {
      if (ids[STG - 1] < seq.total) issue(ids[STG - 1], (k + STG - 1) % STG);
      cp_async_commit();
    }
    const int id = ids[0];
    const int z = id / G::TPS, rem = id % G::TPS, ky = rem / G::KB, kb = rem % G::KB, kz0 = kb * NL;
    const int ky_s = sfreq(ky, N);
    const CgScal& S = sc[z];
    const SS beta = (SS)S.beta, alpha_prev = (SS)S.alpha_prev;
    const size_t o = z * bt.spec + (size_t)ky * NH + kz0;
    const SS* ct = ctab + z * bt.tab;
    const SS* mt = mtab + z * bt.tab;
    // partner line of column 0: p_new at (kx, -ky, 0), recomputed from the inputs (plain loads,
    // in flight while the tiles arrive)
    if (kz0 == 0) {
      const ST* pold = ((S.lit & 1) ? P1 : P0) + z * bt.spec;
      const ST* rz = r + z * bt.spec;
      const size_t pb = (size_t)((N - ky) % N) * NH;
      for (int i = tid; i < M; i += G::NT) {
        const size_t e = pb + (size_t)i * N * NH;
        const ST rv = rz[e], po = pold[e];
        pl[i] = cx<R>{rv.x + beta * po.x, rv.y + beta * po.y};
      }
    }
    if (STG > 1 && ids[1] < seq.total) gather(ids[1], cn, mn);
    if constexpr (COPY == 0) {
      ok = tile_arrived<STG>(bar, s, phase, pending, err);
      if (!ok) break;
    } else {
      cp_async_wait<STG - 1>();
      __syncthreads();
    }
    cx<R>* tr = buf + (s * NS + 0) * G::SSTR;  // r -> p_new
    cx<R>* tp = buf + (s * NS + 1) * G::SSTR;  // p_old -> c p_new -> T
    cx<R>* tx = buf + (s * NS + 2) * G::SSTR;  // x
    typename AccFor<SS>::T acc;  // <p_new, m p_new> over the columns kz != 0 (weight 2)
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = tid + k * G::NT, kz = kz0 + e % NL;
      const cx<R> rv = tr[e], po = tp[e], xv = tx[e];
      const cx<R> pn = cx<R>{rv.x + beta * po.x, rv.y + beta * po.y};
      tx[e] = cx<R>{xv.x + alpha_prev * po.x, xv.y + alpha_prev * po.y};
      tr[e] = pn;
      if (kz != 0) {
        acc.add((SS)2 * mv[k] * (pn.x * pn.x + pn.y * pn.y));
        tp[e] = cx<R>{pn.x * cv[k], pn.y * cv[k]};
      } else {
        tp[e] = pn;  // the packed column stays raw for the pair combine
      }
    }
    if constexpr (COPY == 0) {
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {  // p_new and x are final: store them while T is transformed
        const CUtensorMap* mpn = (S.lit & 1) ? &mP0 : &mP1;
        for (int q = 0; q < G::NBOX; ++q) {
          tma_store_4d(mpn, 2 * kz0, ky, q * G::BR, z, tr + q * G::BR * NL);
          tma_store_4d(&mX, 2 * kz0, ky, q * G::BR, z, tx + q * G::BR * NL);
        }
      }
    } else {
      __syncthreads();
      tile_rows_store<G>(tr, ((S.lit & 1) ? P0 : P1) + o, rowstride, tid);
      tile_rows_store<G>(tx, xg + o, rowstride, tid);
    }
    if (kz0 == 0) {
      // m term of the packed column (weight 1): m0 |P0|^2 + mN |PN|^2 of its two planes
      for (int kx = tid; kx < N; kx += G::NT) {
        const int kxs = sfreq(kx, N);
        const int n2 = kxs * kxs + ky_s * ky_s;
        const cx<R> zc = tp[kx * NL];
        const cx<R> zp = pl[(N - kx) % N];
        const SS h = (SS)0.5;
        const SS a0 = h * (zc.x + zp.x), b0 = h * (zc.y - zp.y);
        const SS aN = h * (zc.y + zp.y), bN = h * (zp.x - zc.x);
        acc.add(mt[n2] * (a0 * a0 + b0 * b0) + mt[n2 + NH * NH] * (aN * aN + bN * bN));
      }
      combine_col0_sep<R, N, NL>(tp, pl, ky_s, ct, tid, G::NT);
    }
    fft_line<R, M, G::TPL, NL, +1, 1, cmin(RMAX, rmax_for(M, G::TPL))>(tp + tid % NL, tid / NL, tw);
    if constexpr (COPY == 0) {
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        for (int q = 0; q < G::NBOX; ++q) tma_store_4d(&mT, 2 * kz0, ky, q * G::BR, z, tp + q * G::BR * NL);
        bulk_commit();
      }
    } else {
      tile_rows_store<G>(tp, Tg + o, rowstride, tid);
    }
    const double sum = block_sum(acc.get(), red);
    if (tid == 0) partials[z * bt.part + ky * G::KB + kb] = sum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      cv[j] = cn[j];
      mv[j] = mn[j];
    }
    for (int j = 0; j < STG - 1; ++j) ids[j] = ids[j + 1];
    ids[STG - 1] = seq.next(ids[STG - 2] < seq.total ? ids[STG - 2] + gridDim.x : seq.total, gridDim.x);
  }
  if (COPY == 0 && tid == 0) tiles_drain<STG>(bar, phase, pending, ok);
  if constexpr (COPY == 1) cp_async_wait<0>();
}

// x pass 2, staged (the work of k_cg_xupd):  T^ = FFT_x(T);  q = m p + c T^;  r -= alpha q;
// partials of <r, r> and ||C^-1 r||^2 (two per tile).  Stage tiles: T, r, p_new.  COPY as for
// x pass 1.
template <class R, int N, bool UNIT_M, int NL, int STG, int RMAX, int EX, int COPY>
__global__ void __launch_bounds__(TG<R, N, NL, STG, EX>::NT)
k_cg_xupd_tma(const __grid_constant__ CUtensorMap mT, const __grid_constant__ CUtensorMap mR,
              const __grid_constant__ CUtensorMap mP0, const __grid_constant__ CUtensorMap mP1,
              const typename Store<R>::T* __restrict__ T, const typename Store<R>::T* P0,
              const typename Store<R>::T* P1, typename Store<R>::T* __restrict__ rg,
              const typename Store<R>::S* __restrict__ ctab,
              const typename Store<R>::S* __restrict__ mtab, const typename Store<R>::T* __restrict__ twtab,
              double* __restrict__ partials, const CgScal* __restrict__ sc, Bat bt, int nb, int* __restrict__ err) {
  using G = TG<R, N, NL, STG, EX>;
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  constexpr int NS = 3, M = N, NH = N / 2;
  static_assert(std::is_same<R, SS>::value, "the CG passes compute in their storage type");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[32];
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));
  cx<R>* tw = buf + STG * NS * G::SSTR;
  cx<R>* pl = tw + M;  // partner line of the packed column
  typename Store<R>::S* ctile = reinterpret_cast<typename Store<R>::S*>(pl + M);  // c(k) of the tile
  uint64_t* bar = reinterpret_cast<uint64_t*>(ctile + M * NL);
  const int tid = threadIdx.x;
  const TileSeq<G> seq{sc, nb * G::TPS};
  if (tid == 0) {
    prefetch_tensormap(&mT);
    prefetch_tensormap(&mR);
    for (int s = 0; s < STG; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  __syncthreads();
  load_tw<R, M, 2 * N>(tw, twtab, tid, G::NT);
  const size_t rowstride = (size_t)N * NH;
  auto issue = [&](int id, int s) {
    const int z = id / G::TPS, rem = id % G::TPS, ky = rem / G::KB, kz0 = (rem % G::KB) * NL;
    if constexpr (COPY == 0) {
      const CUtensorMap* mp = (sc[z].lit & 1) ? &mP0 : &mP1;  // this iteration's p_new
      mbar_expect_tx(&bar[s], NS * G::TILE_BYTES);
      for (int q = 0; q < G::NBOX; ++q) {
        const int off = q * G::BR * NL;
        tma_load_4d(buf + (s * NS + 0) * G::SSTR + off, &mT, 2 * kz0, ky, q * G::BR, z, &bar[s]);
        tma_load_4d(buf + (s * NS + 1) * G::SSTR + off, &mR, 2 * kz0, ky, q * G::BR, z, &bar[s]);
        tma_load_4d(buf + (s * NS + 2) * G::SSTR + off, mp, 2 * kz0, ky, q * G::BR, z, &bar[s]);
      }
    } else {
      const size_t o = z * bt.spec + (size_t)ky * NH + kz0;
      tile_rows_async<G>(buf + (s * NS + 0) * G::SSTR, T + o, rowstride, tid);
      tile_rows_async<G>(buf + (s * NS + 1) * G::SSTR, rg + o, rowstride, tid);
      tile_rows_async<G>(buf + (s * NS + 2) * G::SSTR, ((sc[z].lit & 1) ? P0 : P1) + o, rowstride, tid);
    }
  };
  int ids[STG];
  ids[0] = seq.next(blockIdx.x, gridDim.x);
  for (int j = 1; j < STG; ++j) ids[j] = seq.next(ids[j - 1] < seq.total ? ids[j - 1] + gridDim.x : seq.total, gridDim.x);
  unsigned pending = 0, phase = 0;
  for (int j = 0; j < STG - 1; ++j) {
    if (COPY == 0 && tid == 0 && ids[j] < seq.total) {
      issue(ids[j], j);
      pending |= 1u << j;
    }
    if constexpr (COPY == 1) {
      if (ids[j] < seq.total) issue(ids[j], j);
      cp_async_commit();
    }
  }
  // c(k) of this thread's elements, one tile ahead (gathered while the current tile is processed)
  constexpr int PER = G::E;  // elements per thread: M NL / NT
  SS cv[PER], cn[PER];
  auto gather = [&](int id, SS* c) {
    const int z = id / G::TPS, rem = id % G::TPS, ky = rem / G::KB, kz0 = (rem % G::KB) * NL;
    const int ky_s = sfreq(ky, N);
    const SS* ctz = ctab + z * bt.tab;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = tid + k * G::NT, i = e / NL, kz = kz0 + e % NL;
      const int kxs = sfreq(i, N);
      c[k] = ctz[kxs * kxs + ky_s * ky_s + kz * kz];
    }
  };
  if (ids[0] < seq.total) gather(ids[0], cv);
  bool ok = true;
  for (int k = 0; ids[0] < seq.total; ++k) {
    const int s = k % STG;
    if constexpr (COPY == 0) {
      if (tid == 0 && ids[STG - 1] < seq.total) {
        bulk_wait_read<0>();
        issue(ids[STG - 1], (k + STG - 1) % STG);
        pending |= 1u << ((k + STG - 1) % STG);
      }
    } else {
      if (ids[STG - 1] < seq.total) issue(ids[STG - 1], (k + STG - 1) % STG);
      cp_async_commit();
    }
    const int id = ids[0];
    const int z = id / G::TPS, rem = id % G::TPS, ky = rem / G::KB, kb = rem % G::KB, kz0 = kb * NL;
    const int ky_s = sfreq(ky, N), pky = (N - ky) % N;
    const CgScal& S = sc[z];
    const SS alpha = (SS)S.alpha;
    const SS* ct = ctab + z * bt.tab;
    const SS* mt = mtab + z * bt.tab;
    const ST* p = ((S.lit & 1) ? P0 : P1) + z * bt.spec;
    if (kz0 == 0) {  // partner line of T at -ky, column 0 (plain loads)
      const ST* Tz = T + z * bt.spec;
      for (int i = tid; i < M; i += G::NT) pl[i] = ld_c<R>(Tz + (size_t)pky * NH + (size_t)i * N * NH);
    }
    if (STG > 1 && ids[1] < seq.total) gather(ids[1], cn);
    if constexpr (COPY == 0) {
      ok = tile_arrived<STG>(bar, s, phase, pending, err);
      if (!ok) break;
    } else {
      cp_async_wait<STG - 1>();
      __syncthreads();
    }
    cx<R>* tt = buf + (s * NS + 0) * G::SSTR;
    cx<R>* tr = buf + (s * NS + 1) * G::SSTR;
    const cx<R>* tp = buf + (s * NS + 2) * G::SSTR;
    fft_line<R, M, G::TPL, NL, -1, 1, cmin(RMAX, rmax_for(M, G::TPL))>(tt + tid % NL, tid / NL, tw);
    if (kz0 == 0) {  // transform the partner line too, then apply c to column 0 as a packed pair
      // (by all threads, a few elements each: a separate, small instance of the transform keeps
      // the main one's register budget)
      fft_line_map<R, M, G::NT, -1, 1, 8>(pl, Strided<1>{}, tid, tw);
      combine_col0_sep<R, N, NL>(tt, pl, ky_s, ct, tid, G::NT);
    }
    typename AccFor<SS>::T a_rr, a_rc;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = tid + k * G::NT, i = e / NL, kz = kz0 + e % NL;
      const cx<R> t = tt[e], pv = tp[e];
      cx<R> rv = tr[e];
      const SS c = cv[k];
      SS ic2 = (SS)1 / (c * c);
      SS q0, q1;
      if (kz == 0) {
        const int kxs = sfreq(i, N);
        const int n2 = kxs * kxs + ky_s * ky_s;
        // packed column: T^ already carries c; the m term combines p with p(-kx, -ky, 0) (in the
        // storage type: FP64 here would run on GB300's 1/64-rate unit)
        const SS cN = ct[n2 + NH * NH];
        const SS i2 = (SS)1 / (cN * cN);
        ic2 = ic2 > i2 ? ic2 : i2;
        const SS m0 = mt[n2], mN = mt[n2 + NH * NH];
        const SS a = (SS)0.5 * (m0 + mN), b = (SS)0.5 * (m0 - mN);
        ST pp = ST{};
        if (b != (SS)0) pp = p[(size_t)((N - i) % N) * N * NH + (size_t)pky * NH];
        q0 = a * pv.x + b * pp.x + t.x;
        q1 = a * pv.y - b * pp.y + t.y;
      } else {
        SS m = (SS)1;
        if constexpr (!UNIT_M) {
          const int kxs = sfreq(i, N);
          m = mt[kxs * kxs + ky_s * ky_s + kz * kz];
        }
        q0 = m * pv.x + c * t.x;
        q1 = m * pv.y + c * t.y;
      }
      rv.x -= alpha * q0;
      rv.y -= alpha * q1;
      tr[e] = rv;
      const SS wgt = kz == 0 ? (SS)1 : (SS)2;
      const SS m2 = wgt * (rv.x * rv.x + rv.y * rv.y);
      a_rr.add(m2);
      a_rc.add(ic2 * m2);
    }
    if constexpr (COPY == 0) {
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        for (int q = 0; q < G::NBOX; ++q) tma_store_4d(&mR, 2 * kz0, ky, q * G::BR, z, tr + q * G::BR * NL);
        bulk_commit();
      }
    } else {
      __syncthreads();
      tile_rows_store<G>(tr, rg + z * bt.spec + (size_t)ky * NH + kz0, rowstride, tid);
    }
    const double s1 = block_sum(a_rr.get(), red);
    const double s2 = block_sum(a_rc.get(), red);
    if (tid == 0) {
      partials[z * bt.part + 2 * (ky * G::KB + kb)] = s1;
      partials[z * bt.part + 2 * (ky * G::KB + kb) + 1] = s2;
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) cv[j] = cn[j];
    for (int j = 0; j < STG - 1; ++j) ids[j] = ids[j + 1];
    ids[STG - 1] = seq.next(ids[STG - 2] < seq.total ? ids[STG - 2] + gridDim.x : seq.total, gridDim.x);
  }
  if (COPY == 0 && tid == 0) tiles_drain<STG>(bar, phase, pending, ok);
  if constexpr (COPY == 1) cp_async_wait<0>();
}

// ------------------------------------------------------------------------------------------
// Generic x pass:  out = [IFFT_x]( tab (.) [FFT_x](in) ),  optional partial of wgt |out|^2.
// in != out (the partner line of column 0 is read from `in`).
// ------------------------------------------------------------------------------------------
template <class R, int N, bool FWD, bool INV, bool DOT>
__global__ void __launch_bounds__(XYG<R, N>::NT)
k_xmul(const typename Store<R>::T* __restrict__ in, typename Store<R>::T* __restrict__ out,
       const typename Store<R>::S* __restrict__ tab, const typename Store<R>::T* __restrict__ twtab,
       double* __restrict__ partials, const CgScal* __restrict__ sc, Bat bt) {
  using G = XYG<R, N>;
  using SS = typename Store<R>::S;
  constexpr int NH = G::NH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::M * G::LD;
  __shared__ double red[32];
  const int z = blockIdx.z;
  if (sc && sc[z].done) return;
  in += z * bt.spec;
  out += z * bt.spec;
  tab += z * bt.tab;
  partials += z * bt.part;
  const int tid = threadIdx.x;
  const int kz0 = blockIdx.x * G::NL, ky = blockIdx.y;
  const int ky_s = sfreq(ky, N);
  const int pky = (N - ky) % N;
  load_tw<R, G::M, 2 * N>(tw, twtab, tid, G::NT);
  const size_t rowstride = (size_t)N * NH;
  const size_t base = (size_t)ky * NH + kz0;
  tile_load<G>(tile, in + base, rowstride, tid);
  if (kz0 == 0)
    for (int i = tid; i < G::M; i += G::NT) tile[i * G::LD + G::NL] = ld_c<R>(in + (size_t)pky * NH + (size_t)i * rowstride);
  __syncthreads();
  const int l = tid % G::NL, t = tid / G::NL;
  if constexpr (FWD) {
    fft_line<R, G::M, G::TPL, G::LD, -1>(tile + l, t, tw);
    if (kz0 == 0) fft_line<R, G::M, G::TPL, G::LD, -1>(tile + G::NL, t, tw, l == 0);
  }
  tile_mul<G>(tile, kz0, ky_s, tab, tid);
  if (kz0 == 0) combine_col0<R, N, G::LD, G::NL>(tile, ky_s, tab, tid, G::NT);
  else __syncthreads();
  if constexpr (INV) fft_line<R, G::M, G::TPL, G::LD, +1>(tile + l, t, tw);
  tile_store<G>(tile, out + base, rowstride, tid);
  if constexpr (DOT) {
    typename AccFor<SS>::T acc;
    for (int idx = tid; idx < G::M * G::NL; idx += G::NT) {
      const int i = idx / G::NL, ll = idx % G::NL;
      const cx<R> v = tile[i * G::LD + ll];
      const SS wgt = (kz0 + ll == 0) ? (SS)1 : (SS)2;
      const SS vx = (SS)RT<R>::to_d(v.x), vy = (SS)RT<R>::to_d(v.y);
      acc.add_prod(wgt * vx, vx);
      acc.add_prod(wgt * vy, vy);
    }
    const double s = block_sum(acc.get(), red);
    if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------------------------------
// z direction helpers: real line of length N <-> packed half spectrum of length h = N/2,
// through a complex FFT of length h on z_m = x_2m + i x_2m+1.  tw holds exp(-2 pi i e/(2N)),
// e < 2N (so W_N^k = tw[2k] and the length-h FFT uses stride 4).
// ------------------------------------------------------------------------------------------
// C2R pre-step on one line (element k at col[map(k)]): X (packed) -> Z with z = IFFT_h(Z) the
// real samples.
template <class R, int N, class MAP>
WF_D void c2r_prep_map(cx<R>* col, const MAP& map, int t, int tpl_, const cx<R>* tw) {
  constexpr int H = N / 2;
  for (int k = t; k <= H / 2; k += tpl_) {
    if (k == 0) {
      const cx<R> v = col[map(0)];
      col[map(0)] = cx<R>{v.x + v.y, v.x - v.y};
    } else {
      const int k2 = H - k;
      const cx<R> a = col[map(k)], b = col[map(k2)];
      // Z_k = (X_k + conj X_{h-k}) + i W_N^{+k} (X_k - conj X_{h-k})
      const cx<R> s1 = a + conj(b), d1 = a - conj(b);
      const cx<R> s2 = b + conj(a), d2 = b - conj(a);
      const cx<R> w1 = conj(tw[2 * k]), w2 = conj(tw[2 * k2]);
      col[map(k)] = s1 + mul_i(w1 * d1);
      if (k2 != k) col[map(k2)] = s2 + mul_i(w2 * d2);
    }
  }
}
// R2C post-step on one line: Z = FFT_h(z) -> packed X (X_0, X_h in element 0).
template <class R, int N, class MAP>
WF_D void r2c_post_map(cx<R>* col, const MAP& map, int t, int tpl_, const cx<R>* tw) {
  constexpr int H = N / 2;
  const R half = RT<R>::c(0.5);
  for (int k = t; k <= H / 2; k += tpl_) {
    if (k == 0) {
      const cx<R> v = col[map(0)];
      col[map(0)] = cx<R>{v.x + v.y, v.x - v.y};
    } else {
      const int k2 = H - k;
      const cx<R> a = col[map(k)], b = col[map(k2)];
      // X_k = (Z_k + conj Z_{h-k})/2 - (i/2) W_N^{-k} (Z_k - conj Z_{h-k})
      const cx<R> s1 = a + conj(b), d1 = a - conj(b);
      const cx<R> s2 = b + conj(a), d2 = b - conj(a);
      const cx<R> w1 = tw[2 * k], w2 = tw[2 * k2];
      col[map(k)] = scale(s1 - mul_i(w1 * d1), half);
      if (k2 != k) col[map(k2)] = scale(s2 - mul_i(w2 * d2), half);
    }
  }
}
template <class R, int N, int LD>
WF_D void c2r_prep(cx<R>* col, int t, int tpl_, const cx<R>* tw) {
  c2r_prep_map<R, N>(col, Strided<LD>{}, t, tpl_, tw);
}
template <class R, int N, int LD>
WF_D void r2c_post(cx<R>* col, int t, int tpl_, const cx<R>* tw) {
  r2c_post_map<R, N>(col, Strided<LD>{}, t, tpl_, tw);
}

// ------------------------------------------------------------------------------------------
// Geometry of the z passes: NL consecutive rows (x, y) per CTA, each a line of H = N/2
// complex values; TPL threads per line with E elements each.  Rows are contiguous in memory,
// so tiles move as 16-byte vectors along the row (VW elements each).
// ------------------------------------------------------------------------------------------
template <class R, int N> constexpr int z_elems() { return elems_for<R>(N / 2, tile_lines<R>()); }
template <class R, int N, int EZ = z_elems<R, N>()>
struct ZG {
  using ST = typename Store<R>::T;
  static constexpr int H = N / 2, M = H;
  static constexpr int NL = tile_lines<R>();
  static constexpr int E = EZ;
  static constexpr int TPL = M / E >= 1 ? M / E : 1;
  static constexpr int NT = NL * TPL;
  static constexpr int LD = NL + 1;
  static constexpr int VW = (sizeof(ST) == 8 && M % 2 == 0) ? 2 : 1;
  static constexpr int NV = M / VW;
  static constexpr int NVEC = NL * NV;
  static constexpr int PER = (NVEC + NT - 1) / NT;
  static constexpr bool EVEN = NVEC % NT == 0;
  using VT = typename std::conditional<VW == 2, float4, ST>::type;
  static constexpr size_t SMEM = (size_t)(M * LD + 2 * N) * sizeof(cx<R>);
};

// rows [row0, row0 + NL) of a packed spectrum (H complex per row) <-> tile
template <class G, class R>
WF_D void zrows_load(cx<R>* tile, const typename G::ST* g, size_t row0, int tid) {
  using VT = typename G::VT;
  VT buf[G::PER];
#pragma unroll
  for (int k = 0; k < G::PER; ++k) {
    const int idx = tid + k * G::NT;
    if (G::EVEN || idx < G::NVEC)
      buf[k] = *reinterpret_cast<const VT*>(g + (row0 + idx / G::NV) * G::H + (idx % G::NV) * G::VW);
  }
#pragma unroll
  for (int k = 0; k < G::PER; ++k) {
    const int idx = tid + k * G::NT;
    if (!(G::EVEN || idx < G::NVEC)) continue;
    const int l = idx / G::NV, i = (idx % G::NV) * G::VW;
    if constexpr (G::VW == 2) {
      const float4 f = *reinterpret_cast<const float4*>(&buf[k]);
      tile[i * G::LD + l] = cx<R>{RT<R>::from_f(f.x), RT<R>::from_f(f.y)};
      tile[(i + 1) * G::LD + l] = cx<R>{RT<R>::from_f(f.z), RT<R>::from_f(f.w)};
    } else {
      tile[i * G::LD + l] = ld_c<R>(&buf[k]);
    }
  }
}
template <class G, class R>
WF_D void zrows_store(const cx<R>* tile, typename G::ST* g, size_t row0, int tid) {
  using VT = typename G::VT;
#pragma unroll
  for (int k = 0; k < G::PER; ++k) {
    const int idx = tid + k * G::NT;
    if (!(G::EVEN || idx < G::NVEC)) continue;
    const int l = idx / G::NV, i = (idx % G::NV) * G::VW;
    VT v;
    if constexpr (G::VW == 2) {
      const cx<R> a = tile[i * G::LD + l], b = tile[(i + 1) * G::LD + l];
      *reinterpret_cast<float4*>(&v) = make_float4(RT<R>::to_f(a.x), RT<R>::to_f(a.y), RT<R>::to_f(b.x), RT<R>::to_f(b.y));
    } else {
      st_c(&v, tile[i * G::LD + l]);
    }
    *reinterpret_cast<VT*>(g + (row0 + l) * G::H + i) = v;
  }
}

// ------------------------------------------------------------------------------------------
// z turn (middle of A p): each (x, y) line: packed -> real (C2R), times D(x, y, z), -> packed.
// D = nbar w / V_c carries the 1/V_c of the inverse transform.  grid (N*N / NL).
// ------------------------------------------------------------------------------------------
template <class R, int N, int EZ = z_elems<R, N>()>
__global__ void __launch_bounds__(ZG<R, N, EZ>::NT)
k_zturn(typename Store<R>::T* __restrict__ spec, const typename Store<R>::S* __restrict__ D,
        const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials, const CgScal* __restrict__ sc,
        Bat bt) {
  using G = ZG<R, N, EZ>;
  using SS = typename Store<R>::S;
  static_assert(std::is_same<R, SS>::value, "the CG passes compute in their storage type");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::M * G::LD;  // 2N entries
  __shared__ double red[32];
  const int z = blockIdx.z;
  if (sc && sc[z].done) return;
  spec += z * bt.spec;
  D += z * bt.real;
  partials += z * bt.part;
  const int tid = threadIdx.x;
  const size_t row0 = (size_t)blockIdx.x * G::NL;
  // the D rows go to L2 while the rows are transformed
  if (tid < G::NL) prefetch_l2(D + (row0 + tid) * N, N * sizeof(SS));
  for (int e = tid; e < 2 * N; e += G::NT) tw[e] = ld_c<R>(twtab + e);
  zrows_load<G>(tile, spec, row0, tid);
  __syncthreads();
  const int l = tid % G::NL, t = tid / G::NL;
  c2r_prep<R, N, G::LD>(tile + l, t, G::TPL, tw);
  __syncthreads();
  fft_line<R, G::M, G::TPL, G::LD, +1, 4, rmax_for(G::M, G::TPL)>(tile + l, t, tw);
  // real samples 2i, 2i+1 of line l sit in element i: multiply by D, VW elements at a time,
  // and sum D T^2 (the <c p, D (c p)> term of <p, A p>)
  using DV = typename std::conditional<G::VW == 2, float4, double2>::type;  // 2 VW reals of D
  typename AccFor<SS>::T acc;
#pragma unroll 4
  for (int k = 0; k < G::PER; ++k) {
    const int idx = tid + k * G::NT;
    if (!(G::EVEN || idx < G::NVEC)) continue;
    const int ll = idx / G::NV, i = (idx % G::NV) * G::VW;
    const SS* dp = D + (row0 + ll) * N + 2 * i;
    if constexpr (G::VW == 2) {
      const float4 d = *reinterpret_cast<const float4*>(dp);
      cx<R> a = tile[i * G::LD + ll], b = tile[(i + 1) * G::LD + ll];
      const cx<R> a0 = a, b0 = b;
      a.x = a.x * RT<R>::from_f(d.x);
      a.y = a.y * RT<R>::from_f(d.y);
      b.x = b.x * RT<R>::from_f(d.z);
      b.y = b.y * RT<R>::from_f(d.w);
      // D T^2 >= 0: the vector's four terms are summed first (in R = the storage type)
      acc.add((SS)(a.x * a0.x + a.y * a0.y + b.x * b0.x + b.y * b0.y));
      tile[i * G::LD + ll] = a;
      tile[(i + 1) * G::LD + ll] = b;
    } else {
      const double2 d = *reinterpret_cast<const double2*>(dp);
      cx<R> a = tile[i * G::LD + ll];
      const cx<R> a0 = a;
      a.x = a.x * RT<R>::c(d.x);
      a.y = a.y * RT<R>::c(d.y);
      acc.add((SS)(a.x * a0.x + a.y * a0.y));
      tile[i * G::LD + ll] = a;
    }
  }
  (void)sizeof(DV);
  __syncthreads();
  fft_line<R, G::M, G::TPL, G::LD, -1, 4, rmax_for(G::M, G::TPL)>(tile + l, t, tw);
  r2c_post<R, N, G::LD>(tile + l, t, G::TPL, tw);
  __syncthreads();
  zrows_store<G>(tile, spec, row0, tid);
  const double sum = block_sum(acc.get(), red);
  if (tid == 0) partials[blockIdx.x] = sum;
}

// ------------------------------------------------------------------------------------------
// z forward: real rows (FP64) -> packed spectrum rows.  Optional partial of sum(in^2).
// ------------------------------------------------------------------------------------------
template <class R, int N, bool SQ>
__global__ void __launch_bounds__(ZG<R, N>::NT)
k_zfwd(const double* __restrict__ in, typename Store<R>::T* __restrict__ out,
       const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials, const CgScal* __restrict__ sc,
       Bat bt) {
  using G = ZG<R, N>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::M * G::LD;
  __shared__ double red[32];
  const int z = blockIdx.z;
  if (sc && sc[z].done) return;
  in += z * bt.real;
  out += z * bt.spec;
  partials += z * bt.part;
  const int tid = threadIdx.x;
  const size_t row0 = (size_t)blockIdx.x * G::NL;
  for (int e = tid; e < 2 * N; e += G::NT) tw[e] = ld_c<R>(twtab + e);
  const double2* in2 = reinterpret_cast<const double2*>(in);
  AccD acc;
  constexpr int NE = G::NL * G::M, PE = (NE + G::NT - 1) / G::NT;
  double2 buf[PE];
#pragma unroll
  for (int k = 0; k < PE; ++k) {
    const int idx = tid + k * G::NT;
    if (NE % G::NT == 0 || idx < NE) buf[k] = in2[(row0 + idx / G::M) * G::H + idx % G::M];
  }
#pragma unroll
  for (int k = 0; k < PE; ++k) {
    const int idx = tid + k * G::NT;
    if (!(NE % G::NT == 0 || idx < NE)) continue;
    tile[(idx % G::M) * G::LD + idx / G::M] = ld_c<R>(&buf[k]);
    if constexpr (SQ) {
      acc.add_prod(buf[k].x, buf[k].x);
      acc.add_prod(buf[k].y, buf[k].y);
    }
  }
  __syncthreads();
  const int l = tid % G::NL, t = tid / G::NL;
  fft_line<R, G::M, G::TPL, G::LD, -1, 4, rmax_for(G::M, G::TPL)>(tile + l, t, tw);
  r2c_post<R, N, G::LD>(tile + l, t, G::TPL, tw);
  __syncthreads();
  zrows_store<G>(tile, out, row0, tid);
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
__global__ void __launch_bounds__(ZG<R, N>::NT)
k_zinv(const typename Store<R>::T* __restrict__ in, double* __restrict__ out,
       const double* __restrict__ s, const double* __restrict__ w, const double* __restrict__ b,
       double scl, const typename Store<R>::T* __restrict__ twtab, double* __restrict__ partials,
       const CgScal* __restrict__ sc, Bat bt) {
  using G = ZG<R, N>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* tw = tile + G::M * G::LD;
  __shared__ double red[32];
  const int z = blockIdx.z;
  // RESID reads nbar from the system's scalars; the other modes skip idle systems (done = 4)
  const double nbar = sc ? sc[z].nbar : 0.0;
  if (MODE != ZI_RESID && sc && sc[z].done == 4) return;
  in += z * bt.spec;
  out += z * bt.real;
  if (s) s += z * bt.real;
  if (w) w += z * bt.real;
  if (b) b += z * bt.real;
  partials += z * bt.part;
  const int tid = threadIdx.x;
  const size_t row0 = (size_t)blockIdx.x * G::NL;
  for (int e = tid; e < 2 * N; e += G::NT) tw[e] = ld_c<R>(twtab + e);
  zrows_load<G>(tile, in, row0, tid);
  __syncthreads();
  const int l = tid % G::NL, t = tid / G::NL;
  c2r_prep<R, N, G::LD>(tile + l, t, G::TPL, tw);
  __syncthreads();
  fft_line<R, G::M, G::TPL, G::LD, +1, 4, rmax_for(G::M, G::TPL)>(tile + l, t, tw);
  double2* out2 = reinterpret_cast<double2*>(out);
  AccD acc;
  constexpr int NE = G::NL * G::M;
#pragma unroll 4
  for (int idx = tid; idx < NE; idx += G::NT) {
    const int ll = idx / G::M, i = idx % G::M;
    const size_t e = (row0 + ll) * G::H + i;
    const cx<R> v = tile[i * G::LD + ll];
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

// x += alpha_prev p_last after the loop ends (p_last = P[lit & 1], the last direction);
// grid (., systems).  Systems whose alpha_prev is 0 (nothing pending) skip the sweep.
template <class ST>
__global__ void k_axpy_final(ST* __restrict__ x, const ST* P0, const ST* P1, size_t n, const CgScal* sc, Bat bt) {
  const int z = blockIdx.y;
  sc += z;
  const double a = sc->alpha_prev;
  if (a == 0.0) return;
  const ST* __restrict__ p = ((sc->lit & 1) ? P1 : P0) + z * bt.spec;
  x += z * bt.spec;
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

// After the initial r = C b (k_xmul with DOT): rr = <r, r>; reset the recurrences.  Systems
// marked idle (done = 4) stay idle.  grid = systems.
static __global__ void k_fin_init(const double* __restrict__ partials, int n, CgScal* sc, Bat bt) {
  __shared__ double red[32];
  sc += blockIdx.x;
  if (sc->done == 4) return;
  const double rr = sum_partials(partials + blockIdx.x * bt.part, n, 1, 0, red);
  if (threadIdx.x == 0) {
    sc->rr = rr;
    sc->beta = 0.0;
    sc->alpha = 0.0;
    sc->alpha_prev = 0.0;
    sc->lit = 0;
    sc->rc2 = sc->bb;
    sc->done = (rr == 0.0 || sc->bb == 0.0) ? 1 : 0;
    sc->status = 0;
  }
}

// <p, A p> = partials [0, n1) (the m term, from the x pass) + [off2, off2 + n2) (the data term,
// from the z turn); alpha = rr / <p, A p>.
// (the first n1 partials of the system, and n2 from offset off2)
static __global__ void k_fin_alpha(const double* __restrict__ partials, int n1, int off2, int n2, CgScal* sc, Bat bt) {
  __shared__ double red[32];
  sc += blockIdx.x;
  if (sc->done) return;
  const double pm = sum_partials(partials + blockIdx.x * bt.part, n1, 1, 0, red);
  const double pd = sum_partials(partials + blockIdx.x * bt.part + off2, n2, 1, 0, red);
  const double pq = pm + pd;
  if (threadIdx.x == 0) {
    sc->pq = pq;
    if (sc->defl == 2) {  // the start step of a deflated solve moves by exactly Z mu
      sc->alpha = 1.0;
    } else if (!(pq > 0.0) || !isfinite(pq)) {
      sc->done = 3;
      sc->alpha = 0.0;
      sc->alpha_prev = 0.0;
    } else {
      sc->alpha = sc->rr / pq;
    }
  }
}

// stop rule: rc2 * inv_vc <= max(tol2 * bb, rr_stop)
static __global__ void k_fin_beta(const double* __restrict__ partials, int n, double inv_vc, CgScal* sc, Bat bt) {
  __shared__ double red[32];
  sc += blockIdx.x;
  if (sc->done) return;
  partials += blockIdx.x * bt.part;
  const double rr = sum_partials(partials, n, 2, 0, red);
  const double rc = sum_partials(partials, n, 2, 1, red);
  if (threadIdx.x == 0) {
    const double rc2 = rc * inv_vc;
    sc->beta = rr / sc->rr;
    sc->rr = rr;
    sc->rc2 = rc2;
    sc->alpha_prev = sc->alpha;
    sc->iter += 1;
    sc->lit += 1;
    if (sc->defl == 2) sc->defl = 1;
    const double lim = fmax(sc->tol2 * sc->bb, sc->rr_stop);
    if (!isfinite(rr) || !isfinite(rc2)) sc->done = 3;
    else if (rc2 <= lim) sc->done = 1;
    else if (sc->iter >= sc->max_iter) sc->done = 2;
  }
}

// sum of partials into sc->aux[slot] (slot >= 0, host reads it) or into sc->bb (slot < 0);
// grid = systems
static __global__ void k_fin_sum(const double* __restrict__ partials, int n, int slot, CgScal* sc, Bat bt) {
  __shared__ double red[32];
  sc += blockIdx.x;
  const double v = sum_partials(partials + blockIdx.x * bt.part, n, 1, 0, red);
  if (threadIdx.x == 0) {
    if (slot >= 0) sc->aux[slot] = v;
    else sc->bb = v;
  }
}

}  // namespace wf
