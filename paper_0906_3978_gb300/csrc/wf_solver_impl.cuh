// wf_solver_impl.cuh -- drivers of the Wiener solve (Kitaura et al. 2009, Sec. 3.3.1, Eq. eq:WF).
//
// System: A s = b with A = S^-1 + diag(nbar w), S^-1 = F^-1 diag(dV/P(k)) F, b = R^T N^-1 d.
//
// The iteration runs in Fourier variables.  With C = F^-1 diag(c) F a real, even Fourier
// multiplier, CG is applied to (C A C) y = C b and s = C y; the CG vectors are stored as
// packed half spectra (the DFT of the real-space vectors).  In those variables
//     (C A C) y^ = m (.) y^ + c (.) F( D (.) F^-1 (c (.) y^) ),   D = nbar w,
// with m = c^2 S^-1.  precond = 1 takes c = S^(1/2) (m = 1 except at k = 0, where
// c_0 = (nbar sum(w)/V_c)^(-1/2) and m_0 = 0); precond = 0 takes c = 1, m = S^-1, which is
// textbook CG on A itself.  Either way the stop test is on the canonical residual b - A s:
// its norm is estimated every iteration from the preconditioned residual (||C^-1 r~||) and,
// once the estimate is below tol, recomputed in FP64 from s.
//
// One CG iteration = 5 FFT passes (17 spectra of traffic):
//   x pass 1: p = r + beta p, x += alpha_prev p_old, T = IFFT_x(c p)
//   y pass  : IFFT_y
//   z turn  : IFFT_z, times D / V_c, FFT_z
//   y pass  : FFT_y
//   finisher: alpha = rr / <p, A p> (<p, m p> from x pass 1, <c p, D c p> from the z turn)
//   x pass 2: FFT_x, q = m p + c T, r -= alpha q, <r, r>, ||C^-1 r||^2 (q is never stored)
// (for FP32 at the sizes plane_cs() lists, the three middle passes run as one thread-block
// cluster kernel per x-plane, k_plane_turn)
//   finisher: beta, stop test
#pragma once
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <vector>

#include "wf_ctx.h"
#include "wf_solver_group.h"
#include "wf_plane.cuh"
#include "wf_spectral.cuh"
#include "wf_deflate.cuh"

namespace wf {

// Arithmetic of the FP64-storage transforms.  The engine also runs in double-float (df32, FP32
// units, ~2^-48 relative accuracy), which measured slower than native FP64 for the y pass at
// the tile shapes used here, so native FP64 is used.
using FP64Arith = double;

template <class K>
static inline cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Launch geometry and launchers of the spectral passes for one arithmetic type and size; every
// launcher covers `nb` systems laid out with the strides `bt` (blockIdx.z = system).
template <class R, int N>
struct Spec {
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  static constexpr int NH = N / 2;
  static constexpr int NLxy = XYG<R, N>::NL;
  static_assert(NH % NLxy == 0 && (N * N) % tile_lines<R>() == 0, "tile widths must divide the grid");
  static constexpr int NTy = XYG<R, N>::NT;
  static constexpr int NTx = XYG<R, N>::NT;
  static constexpr size_t SMxy = XYG<R, N>::SMEM;
  static constexpr int NLz = ZG<R, N>::NL;
  static constexpr int NTz = ZG<R, N>::NT;
  static constexpr size_t SMz = ZG<R, N>::SMEM;
  static constexpr int GXY = (NH / NLxy) * N;   // blocks of an x or y pass (per system)
  static constexpr int GZ = N * N / NLz;        // blocks of a z pass (per system)
  static constexpr size_t SPEC = (size_t)N * N * NH;  // complex elements of a spectrum
  static constexpr size_t V = (size_t)N * N * N;
  static constexpr int TAB = 3 * (N / 2) * (N / 2) + 1;
  // partial sums per system.  An x pass writes one (the first) or two (the second) per tile, at
  // most NX tiles whatever its variant; the middle passes (z turn or plane kernel) write theirs
  // from offset NX.
  static constexpr int NX = N * NH;
  static constexpr int NMID = GZ > N * 8 ? GZ : N * 8;
  static constexpr int NPART = NX + NMID > 2 * NX ? NX + NMID : 2 * NX;
  static dim3 gxy(int nb) { return dim3(NH / NLxy, N, nb); }
  static dim3 gz(int nb) { return dim3(GZ, 1, nb); }
  static Bat bat() { return Bat{SPEC, V, TAB, NPART}; }

  // launch-profile class of a pass: FP64-storage launches (the solves' FP64 residuals, the FP64
  // solve) are kept apart from the FP32 inner passes of the same name
  static const char* cls(const char* f32, const char* f64) { return sizeof(SS) == 8 ? f64 : f32; }
  // algorithmic bytes of one launch per system (DRAM traffic the pass cannot avoid)
  static constexpr double BS = (double)SPEC * sizeof(ST);
  static constexpr double BV = (double)V;
  // cluster size of the fused y / z / y plane kernel (0: not available at this size)
  static constexpr int PCS = plane_cs<R, N>(), PE = plane_e<R, N>();
  // the persistent passes with tensor copies: tile lines and buffers in flight
  static constexpr int NLT = tma_lines<R, N>();

  static cudaError_t attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define WF_A(k, b) if (e == cudaSuccess) e = set_smem(k, b)
    WF_A((k_cg_xinv<R, N, true>), SMxy);
    WF_A((k_cg_xinv<R, N, false>), SMxy);
    WF_A((k_cg_xupd<R, N, true>), SMxy);
    WF_A((k_cg_xupd<R, N, false>), SMxy);
    WF_A((k_xmul<R, N, true, false, true>), SMxy);
    WF_A((k_xmul<R, N, false, true, false>), SMxy);
    WF_A((k_xmul<R, N, true, true, false>), SMxy);
    WF_A((k_zturn<R, N>), SMz);
    if constexpr (std::is_same<R, float>::value) {
      WF_A((k_zcoarse<R, N>), SMz);
      WF_A((k_xcr<R, N, 32>), SMxy);
      WF_A(k_gj_update, kUpdSmem);
      WF_A((k_ycoarse<R, N>), (size_t)N * (kDeflMaxRadius + 2) * sizeof(cx<R>));
    }
    if constexpr (PCS > 0) WF_A((k_plane_turn<R, N, PCS, PE>), (PlaneG<R, N, PCS, PE>::SMEM));
    WF_A((k_zfwd<R, N, true>), SMz);
    WF_A((k_zfwd<R, N, false>), SMz);
    WF_A((k_zinv<R, N, ZI_STORE>), SMz);
    WF_A((k_zinv<R, N, ZI_RESID>), SMz);
    WF_A((k_zinv<R, N, ZI_ACCUM>), SMz);
#undef WF_A
    for (const PassVariant& v : yvariants())
      if (e == cudaSuccess) e = v.setup();
    for (const XVariant& v : xvariants())
      if (e == cudaSuccess) e = v.setup();
    for (const ZVariant& v : zvariants())
      if (e == cudaSuccess) e = v.setup();
    if (e == cudaSuccess) done = true;
    return e;
  }

  // persistent grid: every SM holds its resident CTAs, capped by the number of tiles
  static unsigned persistent_grid(const Ctx& c, int occ, long long tiles) {
    const long long g = (long long)occ * (c.sm_count > 0 ? c.sm_count : 152);
    return (unsigned)(tiles < g ? tiles : g);
  }
  // ---- launch variants of a pass (tile lines, buffers in flight, radix cap); the context's
  // tuning table picks one per (pass, precision, size), variant 0 by default ------------------
  using PassRun = void (*)(Ctx&, int, ST*, const ST*, const CgScal*, int, cudaStream_t);
  struct PassVariant {
    const char* name;
    cudaError_t (*setup)();
    PassRun run;
  };
  // y pass variant <NL, STG, RMAX>: complex FFT along y of every (x, kz) line, in place
  template <int NL, int STG, int RMAX>
  struct YV {
    using G = TG<R, N, NL, STG>;
    static inline int occ = 1;  // resident CTAs per SM
    static cudaError_t setup() {
      cudaError_t e = set_smem(k_ypass_tma<R, N, -1, NL, STG, RMAX>, G::SMEM);
      if (e == cudaSuccess) e = set_smem(k_ypass_tma<R, N, +1, NL, STG, RMAX>, G::SMEM);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ypass_tma<R, N, -1, NL, STG, RMAX>, G::NT, G::SMEM);
      if (occ < 1) occ = 1;
      return e;
    }
    static void run(Ctx& c, int nb, ST* t, const ST* tw, const CgScal* sc, int dir, cudaStream_t st) {
      CUtensorMap m;
      if (!make_spectrum_map(&m, t, N, nb, sizeof(SS) == 8, NL, G::BR, 1)) {
        c.map_failed = true;
        return;
      }
      const unsigned grid = persistent_grid(c, occ, (long long)nb * G::TPS);
      c.launch(cls("ypass", "ypass_f64"), 2 * BS * nb, st, [&] {
        if (dir < 0) k_ypass_tma<R, N, -1, NL, STG, RMAX><<<grid, G::NT, G::SMEM, st>>>(m, tw, sc, nb, c.dev_err);
        else k_ypass_tma<R, N, +1, NL, STG, RMAX><<<grid, G::NT, G::SMEM, st>>>(m, tw, sc, nb, c.dev_err);
      });
    }
  };
  // candidates: FP32 grids of 128 and up (the inner solves) get a few; everything else the default
  static const std::vector<PassVariant>& yvariants() {
    static const std::vector<PassVariant> v = [] {
      std::vector<PassVariant> out{{"nl_s2_r8", YV<NLT, 2, 8>::setup, YV<NLT, 2, 8>::run}};
      if constexpr (std::is_same<R, float>::value && N >= 128) {
        constexpr int H = NLT / 2;
        out.push_back({"nl_s2_r32", YV<NLT, 2, 32>::setup, YV<NLT, 2, 32>::run});
        out.push_back({"nl_s3_r32", YV<NLT, 3, 32>::setup, YV<NLT, 3, 32>::run});
        out.push_back({"nl/2_s2_r32", YV<H, 2, 32>::setup, YV<H, 2, 32>::run});
        out.push_back({"nl/2_s3_r16", YV<H, 3, 16>::setup, YV<H, 3, 16>::run});
      }
      return out;
    }();
    return v;
  }
  // ---- x-pass variants: the two CG x passes, staged by tensor copies (<NL, STG, RMAX>) or the
  // register-staged kernels; each launcher returns the number of partial sums it wrote -------
  using XinvRun = int (*)(Ctx&, int, ST*, ST*, ST*, ST*, ST*, const SS*, const SS*, bool, const ST*, double*,
                          CgScal*, cudaStream_t);
  using XupdRun = int (*)(Ctx&, int, const ST*, ST*, ST*, ST*, const SS*, const SS*, bool, const ST*, double*,
                          CgScal*, cudaStream_t);
  struct XVariant {
    const char* name;
    cudaError_t (*setup)();
    XinvRun xinv;
    XupdRun xupd;
  };
  template <int NL, int STG, int RMAX, int EX = elems_for<R>(N, NL), int COPY = 0>
  struct XV {
    using G = TG<R, N, NL, STG, EX>;
    static constexpr size_t SM = TXG<R, N, NL, STG, 3>::SMEM;
    static inline int occ = 1;
    static cudaError_t setup() {
      cudaError_t e = set_smem(k_cg_xinv_tma<R, N, true, NL, STG, RMAX, EX, COPY>, SM);
      if (e == cudaSuccess) e = set_smem(k_cg_xinv_tma<R, N, false, NL, STG, RMAX, EX, COPY>, SM);
      if (e == cudaSuccess) e = set_smem(k_cg_xupd_tma<R, N, true, NL, STG, RMAX, EX, COPY>, SM);
      if (e == cudaSuccess) e = set_smem(k_cg_xupd_tma<R, N, false, NL, STG, RMAX, EX, COPY>, SM);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_xinv_tma<R, N, true, NL, STG, RMAX, EX, COPY>,
                                                          G::NT, SM);
      if (occ < 1) occ = 1;
      return e;
    }
    // tensor maps for the tensor-copy form; the row-copy form passes zeroed (unused) maps
    static bool map(Ctx& c, CUtensorMap* m, const void* p, int nb) {
      if (COPY == 1) {
        std::memset(m, 0, sizeof(*m));
        return true;
      }
      if (make_spectrum_map(m, const_cast<void*>(p), N, nb, sizeof(SS) == 8, NL, 1, G::BR)) return true;
      c.map_failed = true;
      return false;
    }
    static int xinv(Ctx& c, int nb, ST* r, ST* P0, ST* P1, ST* x, ST* T, const SS* ctab, const SS* mtab, bool unit_m,
                    const ST* tw, double* part, CgScal* sc, cudaStream_t st) {
      CUtensorMap mr, m0, m1, mx, mt;
      if (!map(c, &mr, r, nb) || !map(c, &m0, P0, nb) || !map(c, &m1, P1, nb) || !map(c, &mx, x, nb) ||
          !map(c, &mt, T, nb))
        return G::TPS;
      const unsigned grid = persistent_grid(c, occ, (long long)nb * G::TPS);
      c.launch(cls("cg_xinv", "cg_xinv_f64"), 6 * BS * nb, st, [&] {
        if (unit_m)
          k_cg_xinv_tma<R, N, true, NL, STG, RMAX, EX, COPY><<<grid, G::NT, SM, st>>>(
              mr, m0, m1, mx, mt, r, P0, P1, x, T, ctab, mtab, tw, part, sc, bat(), nb, c.dev_err);
        else
          k_cg_xinv_tma<R, N, false, NL, STG, RMAX, EX, COPY><<<grid, G::NT, SM, st>>>(
              mr, m0, m1, mx, mt, r, P0, P1, x, T, ctab, mtab, tw, part, sc, bat(), nb, c.dev_err);
      });
      return G::TPS;
    }
    static int xupd(Ctx& c, int nb, const ST* T, ST* r, ST* P0, ST* P1, const SS* ctab, const SS* mtab, bool unit_m,
                    const ST* tw, double* part, CgScal* sc, cudaStream_t st) {
      CUtensorMap mt, mr, m0, m1;
      if (!map(c, &mt, T, nb) || !map(c, &mr, r, nb) || !map(c, &m0, P0, nb) || !map(c, &m1, P1, nb)) return G::TPS;
      const unsigned grid = persistent_grid(c, occ, (long long)nb * G::TPS);
      c.launch(cls("cg_xupd", "cg_xupd_f64"), 4 * BS * nb, st, [&] {
        if (unit_m)
          k_cg_xupd_tma<R, N, true, NL, STG, RMAX, EX, COPY><<<grid, G::NT, SM, st>>>(
              mt, mr, m0, m1, T, P0, P1, r, ctab, mtab, tw, part, sc, bat(), nb, c.dev_err);
        else
          k_cg_xupd_tma<R, N, false, NL, STG, RMAX, EX, COPY><<<grid, G::NT, SM, st>>>(
              mt, mr, m0, m1, T, P0, P1, r, ctab, mtab, tw, part, sc, bat(), nb, c.dev_err);
      });
      return G::TPS;
    }
  };
  // the register-staged kernels (one CTA per tile, loads through registers), radix cap RMAX, at
  // least MINB resident CTAs per SM (the register cap that allows them: 128 for 2, 85 for 3)
  template <int RMAX, int MINB = 0>
  struct XReg {
    static cudaError_t setup() {
      cudaError_t e = set_smem(k_cg_xinv<R, N, true, RMAX, MINB>, SMxy);
      if (e == cudaSuccess) e = set_smem(k_cg_xinv<R, N, false, RMAX, MINB>, SMxy);
      if (e == cudaSuccess) e = set_smem(k_cg_xupd<R, N, true, RMAX, MINB>, SMxy);
      if (e == cudaSuccess) e = set_smem(k_cg_xupd<R, N, false, RMAX, MINB>, SMxy);
      return e;
    }
    static int xinv(Ctx& c, int nb, ST* r, ST* P0, ST* P1, ST* x, ST* T, const SS* ctab, const SS* mtab, bool unit_m,
                    const ST* tw, double* part, CgScal* sc, cudaStream_t st) {
      c.launch(cls("cg_xinv", "cg_xinv_f64"), 6 * BS * nb, st, [&] {
        if (unit_m)
          k_cg_xinv<R, N, true, RMAX, MINB><<<gxy(nb), NTx, SMxy, st>>>(r, P0, P1, x, T, ctab, mtab, tw, part, sc, bat());
        else
          k_cg_xinv<R, N, false, RMAX, MINB><<<gxy(nb), NTx, SMxy, st>>>(r, P0, P1, x, T, ctab, mtab, tw, part, sc, bat());
      });
      return GXY;
    }
    static int xupd(Ctx& c, int nb, const ST* T, ST* r, ST* P0, ST* P1, const SS* ctab, const SS* mtab, bool unit_m,
                    const ST* tw, double* part, CgScal* sc, cudaStream_t st) {
      c.launch(cls("cg_xupd", "cg_xupd_f64"), 4 * BS * nb, st, [&] {
        if (unit_m)
          k_cg_xupd<R, N, true, RMAX, MINB><<<gxy(nb), NTx, SMxy, st>>>(T, r, P0, P1, ctab, mtab, tw, part, sc, bat());
        else
          k_cg_xupd<R, N, false, RMAX, MINB><<<gxy(nb), NTx, SMxy, st>>>(T, r, P0, P1, ctab, mtab, tw, part, sc, bat());
      });
      return GXY;
    }
  };
  // x pass 2 with its r and p rows prefetched into shared memory (NL lines, EX elements per thread)
  template <int RMAX, int NL, int EX>
  struct XPf {
    using G = XYP<R, N, NL, EX>;
    static cudaError_t setup() {
      cudaError_t e = set_smem(k_cg_xupd_pf<R, N, true, RMAX, NL, EX>, G::SMEM);
      if (e == cudaSuccess) e = set_smem(k_cg_xupd_pf<R, N, false, RMAX, NL, EX>, G::SMEM);
      return e;
    }
    static int xupd(Ctx& c, int nb, const ST* T, ST* r, ST* P0, ST* P1, const SS* ctab, const SS* mtab, bool unit_m,
                    const ST* tw, double* part, CgScal* sc, cudaStream_t st) {
      const dim3 grid(N / 2 / NL, N, nb);
      c.launch(cls("cg_xupd", "cg_xupd_f64"), 4 * BS * nb, st, [&] {
        if (unit_m)
          k_cg_xupd_pf<R, N, true, RMAX, NL, EX><<<grid, G::NT, G::SMEM, st>>>(T, r, P0, P1, ctab, mtab, tw, part, sc,
                                                                              bat());
        else
          k_cg_xupd_pf<R, N, false, RMAX, NL, EX><<<grid, G::NT, G::SMEM, st>>>(T, r, P0, P1, ctab, mtab, tw, part,
                                                                               sc, bat());
      });
      return (N / 2 / NL) * N;
    }
  };
  static constexpr int NLX = xtma_lines<R, N, 3, 2>();
  static const std::vector<XVariant>& xvariants() {
    static const std::vector<XVariant> v = [] {
      // variant 0: the register-staged kernels, measured fastest at every size (512^3 FP32: 0.72 and
      // 0.58 ms against 1.23-1.83 ms for the staged forms, whose single resident CTA per SM
      // serialises each tile's table gathers, transform and epilogue); the staged forms stay
      // candidates for the tuner on the FP32 grids of 128 and up
      std::vector<XVariant> out{{"registers", XReg<8>::setup, XReg<8>::xinv, XReg<8>::xupd}};
      if constexpr (std::is_same<R, float>::value && N >= 128) {
        out.push_back({"registers_r16", XReg<16>::setup, XReg<16>::xinv, XReg<16>::xupd});
        out.push_back({"registers_r32", XReg<32>::setup, XReg<32>::xinv, XReg<32>::xupd});
        // x pass 2 only (its x pass 1 entry is the radix-32 register kernel again)
        if constexpr ((N / 2) % 8 == 0 && N % 16 == 0) {
          using P1 = XPf<32, 8, 16>;
          using P2 = XPf<16, 8, 16>;
          out.push_back({"prefetch_nl8_e16_r32", P1::setup, XReg<32>::xinv, P1::xupd});
          out.push_back({"prefetch_nl8_e16_r16", P2::setup, XReg<32>::xinv, P2::xupd});
        }
      }
      if constexpr (std::is_same<R, float>::value && N >= 128 && N % 8 == 0 && NLX * (N / 8) <= 512) {
        using E8 = XV<NLX, 2, 8, 8, 1>;  // per-thread row copies, 8 elements per thread
        using T8 = XV<NLX, 2, 8, 8, 0>;  // tensor copies, 8 elements per thread
        out.push_back({"rows_s2_e8", E8::setup, E8::xinv, E8::xupd});
        out.push_back({"tensor_s2_e8", T8::setup, T8::xinv, T8::xupd});
      }
      return out;
    }();
    return v;
  }
  // ---- z-turn variants: elements per thread (threads per CTA) ------------------------------
  using ZRun = void (*)(Ctx&, int, ST*, const SS*, const ST*, double*, const CgScal*, cudaStream_t);
  struct ZVariant {
    const char* name;
    cudaError_t (*setup)();
    ZRun run;
  };
  template <int EZ>
  struct ZV {
    static cudaError_t setup() { return set_smem(k_zturn<R, N, EZ>, ZG<R, N, EZ>::SMEM); }
    static void run(Ctx& c, int nb, ST* T, const SS* D, const ST* tw, double* part, const CgScal* sc,
                    cudaStream_t st) {
      c.launch(cls("zturn", "zturn_f64"), (2 * BS + sizeof(SS) * BV) * nb, st, [&] {
        k_zturn<R, N, EZ><<<gz(nb), ZG<R, N, EZ>::NT, ZG<R, N, EZ>::SMEM, st>>>(T, D, tw, part, sc, bat());
      });
    }
  };
  static const std::vector<ZVariant>& zvariants() {
    static const std::vector<ZVariant> v = [] {
      constexpr int E0 = z_elems<R, N>();
      std::vector<ZVariant> out{{"e_default", ZV<E0>::setup, ZV<E0>::run}};
      if constexpr (std::is_same<R, float>::value && N >= 128) {
        if constexpr (E0 / 2 >= 4 && (N / 2) % (E0 / 2) == 0) out.push_back({"e/2", ZV<E0 / 2>::setup, ZV<E0 / 2>::run});
        if constexpr (E0 / 4 >= 4 && (N / 2) % (E0 / 4) == 0) out.push_back({"e/4", ZV<E0 / 4>::setup, ZV<E0 / 4>::run});
      }
      return out;
    }();
    return v;
  }
  static std::string tune_key(const char* pass) {
    return std::string(pass) + (sizeof(SS) == 8 ? "/f64/" : "/f32/") + std::to_string(N);
  }
  template <class V>
  static const V& pick(const Ctx& c, const char* pass, const std::vector<V>& vs) {
    auto it = c.tuned.find(tune_key(pass));
    const int i = it == c.tuned.end() ? 0 : it->second;
    return vs[i >= 0 && i < (int)vs.size() ? i : 0];
  }
  // complex FFT along y of every (x, kz) line of nb spectra, in place
  static void ypass(Ctx& c, int nb, ST* t, const ST* tw, const CgScal* sc, int dir, cudaStream_t st) {
    pick(c, "ypass", yvariants()).run(c, nb, t, tw, sc, dir, st);
  }
  // out = [IFFT_x] tab (.) [FFT_x] in
  template <bool FWD, bool INV, bool DOT>
  static void xmul(Ctx& c, int nb, const ST* in, ST* out, const SS* tab, const ST* tw, double* part,
                   const CgScal* sc, cudaStream_t st) {
    c.launch(cls("xmul", "xmul_f64"), 2 * BS * nb, st,
             [&] { k_xmul<R, N, FWD, INV, DOT><<<gxy(nb), NTx, SMxy, st>>>(in, out, tab, tw, part, sc, bat()); });
  }
  static void zfwd(Ctx& c, int nb, const double* in, ST* out, const ST* tw, double* part, bool sq,
                   const CgScal* sc, cudaStream_t st) {
    c.launch(cls("zfwd", "zfwd_f64"), (BS + 8 * BV) * nb, st, [&] {
      if (sq) k_zfwd<R, N, true><<<gz(nb), NTz, SMz, st>>>(in, out, tw, part, sc, bat());
      else k_zfwd<R, N, false><<<gz(nb), NTz, SMz, st>>>(in, out, tw, part, sc, bat());
    });
  }
  template <int MODE>
  static void zinv(Ctx& c, int nb, const ST* in, double* out, const double* s, const double* w, const double* b,
                   double scl, const ST* tw, double* part, const CgScal* sc, cudaStream_t st) {
    const double vb = MODE == ZI_RESID ? 4 : (MODE == ZI_ACCUM ? 2 : 1);
    c.launch(cls("zinv", "zinv_f64"), (BS + 8 * vb * BV) * nb, st,
             [&] { k_zinv<R, N, MODE><<<gz(nb), NTz, SMz, st>>>(in, out, s, w, b, scl, tw, part, sc, bat()); });
  }

  struct NoHook {
    void operator()(cudaStream_t) const {}
  };
  // One CG iteration of every unfinished system (no host synchronisation).  The first x pass forms
  // p from rin (default r); after_xinv(st) is enqueued right after it.
  template <class H = NoHook>
  static void iteration(Ctx& c, int nb, ST* r, ST* P0, ST* P1, ST* x, ST* T, const SS* D, const SS* ctab,
                        const SS* mtab, bool unit_m, const ST* tw, double* part, CgScal* sc, double inv_vc,
                        cudaStream_t st, ST* rin = nullptr, H after_xinv = H()) {
    const Bat b = bat();
    const int n1 = pick(c, "xinv", xvariants())
                       .xinv(c, nb, rin ? rin : r, P0, P1, x, T, ctab, mtab, unit_m, tw, part, sc, st);
    after_xinv(st);
    int nmid = GZ;  // blocks that sum the data term of <p, A p> into part[NX ...]
    bool fused = false;
    if constexpr (PCS > 0) {
      if (c.fused_planes) {
        c.launch("plane_turn", (2 * BS + sizeof(SS) * BV) * nb, st,
                 [&] { plane_turn_launch<R, N, PCS, PE>(T, D, tw, part + NX, sc, b, nb, st); });
        nmid = N * PCS;
        fused = true;
      }
    }
    if (!fused) {
      ypass(c, nb, T, tw, sc, +1, st);
      pick(c, "zturn", zvariants()).run(c, nb, T, D, tw, part + NX, sc, st);
      ypass(c, nb, T, tw, sc, -1, st);
    }
    c.launch("fin", 0, st, [&] { k_fin_alpha<<<nb, 1024, 0, st>>>(part, n1, NX, nmid, sc, b); });
    const int n3 = pick(c, "xupd", xvariants()).xupd(c, nb, T, r, P0, P1, ctab, mtab, unit_m, tw, part, sc, st);
    c.launch("fin", 0, st, [&] { k_fin_beta<<<nb, 1024, 0, st>>>(part, n3, inv_vc, sc, b); });
  }
};

// ---- small batched elementwise helpers (blockIdx.y = system) -----------------------------
// D = w * nbar / V_c (nbar from the system's scalars), in the type of the spectral arithmetic
template <class SSo>
__global__ void k_make_D(const double* __restrict__ w, SSo* __restrict__ D, const CgScal* __restrict__ sc,
                         double inv_vc, size_t n) {
  const int z = blockIdx.y;
  const double f = sc[z].nbar * inv_vc;
  w += z * n;
  D += z * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    D[i] = (SSo)(w[i] * f);
}
// partials[z * pstride + block] of sum(in) (SQ = false) or sum(in^2) (SQ = true)
template <bool SQ>
__global__ void k_sum(const double* __restrict__ in, size_t n, double* __restrict__ partials, int pstride) {
  __shared__ double red[32];
  const int z = blockIdx.y;
  in += z * n;
  AccD acc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (SQ) acc.add_prod(in[i], in[i]);
    else acc.add(in[i]);
  }
  const double s = block_sum(acc.get(), red);
  if (threadIdx.x == 0) partials[z * pstride + blockIdx.x] = s;
}

// Tables: ctab[n2] = c(k), mtab[n2] = c^2 S^-1 (k) for one system.
static void make_tables(const std::vector<double>& sinv, bool precond, double c0, double* ct, double* mt) {
  const size_t L = sinv.size();
  for (size_t i = 0; i < L; ++i) {
    if (!precond) {
      ct[i] = 1.0;
      mt[i] = sinv[i];
    } else if (i == 0) {
      ct[i] = c0;
      mt[i] = 0.0;
    } else {
      ct[i] = 1.0 / std::sqrt(sinv[i]);
      mt[i] = 1.0;
    }
  }
}

// Device table `name` from v, converted to T, through a page-locked staging buffer of the same
// name (an asynchronous copy: the staging buffer is rewritten only by a later solve of the same
// workspace, after this one's stream has finished).
template <class T>
static inline wf_status upload_tables(Ctx& c, const std::string& name, const std::vector<double>& v, T** out,
                                      cudaStream_t st) {
  T *h, *d;
  WF_TRY(c.get_pinned(name + "_stage", v.size() * sizeof(T), (void**)&h));
  for (size_t i = 0; i < v.size(); ++i) h[i] = (T)v[i];
  WF_TRY(c.get(name, v.size() * sizeof(T), (void**)&d));
  WF_CUDA(cudaMemcpyAsync(d, h, v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  *out = d;
  return WF_OK;
}

// ==========================================================================================
// A group: `nb` systems of one grid size and precision, solved together.  The host drives it
// as a state machine: enqueue() launches the next block of device work (ending with a copy of
// the scalars to pinned host memory), advance() consumes those scalars after the stream is
// synchronised and picks the next phase.
// ==========================================================================================

// Shared pieces: contiguous copies of w and b, sum(w), ||b||^2, tables, scalars.
template <int N>
struct GroupCommon : Group {
  static constexpr size_t V = (size_t)N * N * N;
  static constexpr int TAB = 3 * (N / 2) * (N / 2) + 1;
  std::string key;
  double *W = nullptr, *B = nullptr, *S = nullptr, *RES = nullptr, *part = nullptr;
  CgScal *sc = nullptr, *hsc = nullptr;
  const double2* tw = nullptr;
  std::vector<CgScal> h;       // host copy of the scalars
  std::vector<double> bb0, sumw, rel;
  std::vector<int> state;      // 0 running, 1 finished
  std::vector<int> bad;        // 1: rejected input (status already set)
  int phase = 0;
  double inv_vc = 1.0 / (double)V;
  // CUDA graph of one block of CG iterations (kernel arguments are fixed for the group)
  cudaGraphExec_t gexec = nullptr;
  long long glaunches = 0;

  ~GroupCommon() override {
    if (gexec) cudaGraphExecDestroy(gexec);
  }
  // Enqueue `body(stream)` on st: directly while the profiler times launches, otherwise as a
  // graph captured on the first call (on the context's capture stream) and replayed.
  template <class F>
  wf_status run_block(Ctx& c, cudaStream_t st, F&& body) {
    if (c.prof.on) {
      body(st);
      return WF_OK;
    }
    if (!gexec) {
      cudaStream_t cs;
      WF_TRY(c.capture_stream(&cs));
      const long long before = c.prof.launches;
      WF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      body(cs);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      glaunches = c.prof.launches - before;
      c.prof.launches = before;
      if (e != cudaSuccess) {
        gexec = nullptr;
        set_last_error("graph capture of the CG block", e);
        return WF_ERR_CUDA;
      }
    }
    WF_CUDA(cudaGraphLaunch(gexec, st));
    c.prof.launches += glaunches;
    return WF_OK;
  }

  wf_status push_scalars(cudaStream_t st) {
    for (int m = 0; m < nb; ++m) hsc[m] = h[m];
    WF_CUDA(cudaMemcpyAsync(sc, hsc, nb * sizeof(CgScal), cudaMemcpyHostToDevice, st));
    return WF_OK;
  }
  wf_status pull_scalars(cudaStream_t st) {
    WF_CUDA(cudaMemcpyAsync(hsc, sc, nb * sizeof(CgScal), cudaMemcpyDeviceToHost, st));
    return WF_OK;
  }
  void read_scalars() { h.assign(hsc, hsc + nb); }
  bool all_done() const {
    for (int m = 0; m < nb; ++m)
      if (h[m].done == 0) return false;
    return true;
  }
};

// Per-system sums of w and b^2: two reductions into the partial slots [0,152) and [152,304),
// enqueued with the copy of the scalars back to the host (no synchronisation) ...
template <int N>
static wf_status group_sums_begin(Ctx& c, GroupCommon<N>& g, int npart, cudaStream_t st) {
  const size_t V = GroupCommon<N>::V;
  g.h.assign(g.nb, CgScal{});
  WF_TRY(g.push_scalars(st));
  const Bat b{0, 0, 0, npart};
  c.launch("reduce", 8.0 * V * g.nb, st, [&] { k_sum<false><<<dim3(152, g.nb), 256, 0, st>>>(g.W, V, g.part, npart); });
  c.launch("fin", 0, st, [&] { k_fin_sum<<<g.nb, 1024, 0, st>>>(g.part, 152, 0, g.sc, b); });
  c.launch("reduce", 8.0 * V * g.nb, st, [&] { k_sum<true><<<dim3(152, g.nb), 256, 0, st>>>(g.B, V, g.part, npart); });
  c.launch("fin", 0, st, [&] { k_fin_sum<<<g.nb, 1024, 0, st>>>(g.part, 152, 1, g.sc, b); });
  WF_CUDA(cudaGetLastError());
  return g.pull_scalars(st);
}
// ... and read once the stream has passed them.
template <int N>
static void group_sums_end(GroupCommon<N>& g) {
  g.read_scalars();
  g.sumw.resize(g.nb);
  g.bb0.resize(g.nb);
  g.bad.assign(g.nb, 0);
  for (int m = 0; m < g.nb; ++m) {
    g.sumw[m] = g.h[m].aux[0];
    g.bb0[m] = g.h[m].aux[1];
    // an empty window or a non-finite w or b is this system's argument error, not the batch's
    if (!(g.sumw[m] > 0.0) || !std::isfinite(g.sumw[m]) || !std::isfinite(g.bb0[m])) {
      g.bad[m] = 1;
      g.sumw[m] = 1.0;
      g.bb0[m] = 0.0;
      if (g.info[m]) *g.info[m] = wf_solve_info{0, 0, 0.0, g.sys[m]->nbar, WF_ERR_ARG};
    }
  }
}

// The last inner solve of a mixed solve aims at kInnerMargin x the remaining reduction (its stop
// test is an upper estimate of the canonical residual; the FP64 residual that follows decides).
// 0.9 saved ~2% of the iterations at 512^3 but moved the result from 5e-7 to 8e-7 of the solution
// converged to 1e-10, too close to the mixed path's 1e-6 bound.
constexpr double kInnerMargin = 0.5;

// Check interval: grids of 256^3 and up check the device flags every 4 iterations.
template <int N> constexpr int check_every() { return N >= 256 ? 4 : (N >= 128 ? 8 : 16); }

// ------------------------------------------------------------------------------------------
// FP64 group: FP64 storage, spectral arithmetic R.
// Phases: 1 CG loop, 2 post (s = C x, explicit residual), 3 restart, 9 done.
// ------------------------------------------------------------------------------------------
template <class R, int N>
struct GroupFP64 : GroupCommon<N> {
  using SP = Spec<R, N>;
  using ST = typename Store<R>::T;
  using Base = GroupCommon<N>;
  using Base::nb; using Base::sys; using Base::info; using Base::key; using Base::W; using Base::B;
  using Base::S; using Base::RES; using Base::part; using Base::sc; using Base::tw; using Base::h;
  using Base::phase; using Base::inv_vc; using Base::bb0; using Base::rel; using Base::state;
  ST *xh, *rh, *P0, *P1, *T, *T2;
  double *D, *ct, *mt, *stab;
  std::vector<int> restarts;
  bool unit_m = true;

  wf_status prepare_begin(Ctx& c, cudaStream_t st) override {
    nb = (int)sys.size();
    key = this->tag + "f64_" + std::to_string(N) + "_";
    int* err;
    WF_TRY(c.err_word(&err));
    WF_CUDA(SP::attrs());
    const size_t SPEC = SP::SPEC, V = SP::V;
    WF_TRY(c.tw(N, &tw));
    const char* nm[6] = {"x", "r", "p0", "p1", "T", "T2"};
    ST** ptr[6] = {&xh, &rh, &P0, &P1, &T, &T2};
    for (int i = 0; i < 6; ++i) WF_TRY(c.get(key + nm[i], nb * SPEC * sizeof(ST), (void**)ptr[i]));
    WF_TRY(c.get(key + "D", nb * V * sizeof(double), (void**)&D));
    WF_TRY(c.get(key + "W", nb * V * sizeof(double), (void**)&W));
    WF_TRY(c.get(key + "B", nb * V * sizeof(double), (void**)&B));
    WF_TRY(c.get(key + "S", nb * V * sizeof(double), (void**)&S));
    WF_TRY(c.get(key + "RES", nb * V * sizeof(double), (void**)&RES));
    WF_TRY(c.get(key + "part", (size_t)nb * SP::NPART * sizeof(double), (void**)&part));
    WF_TRY(c.get(key + "sc", nb * sizeof(CgScal), (void**)&sc));
    WF_TRY(c.get_pinned(key + "hsc", nb * sizeof(CgScal), (void**)&this->hsc));
    for (int m = 0; m < nb; ++m) {
      WF_CUDA(cudaMemcpyAsync(W + m * V, sys[m]->w, V * sizeof(double), cudaMemcpyDefault, st));
      WF_CUDA(cudaMemcpyAsync(B + m * V, sys[m]->b, V * sizeof(double), cudaMemcpyDefault, st));
    }
    return group_sums_begin<N>(c, *this, SP::NPART, st);
  }
  wf_status prepare_end(Ctx& c, cudaStream_t st) override {
    const size_t SPEC = SP::SPEC, V = SP::V;
    group_sums_end<N>(*this);
    // tables
    const int TAB = SP::TAB;
    std::vector<double> vc((size_t)nb * TAB), vm((size_t)nb * TAB), vs((size_t)nb * TAB);
    unit_m = true;
    for (int m = 0; m < nb; ++m) {
      const bool pre = sys[m]->opts.precond != 0;
      unit_m = unit_m && pre;
      const double c0 = 1.0 / std::sqrt(sys[m]->nbar * this->sumw[m] * inv_vc);
      make_tables(sys[m]->sinv, pre, c0, vc.data() + (size_t)m * TAB, vm.data() + (size_t)m * TAB);
      std::copy(sys[m]->sinv.begin(), sys[m]->sinv.end(), vs.begin() + (size_t)m * TAB);
    }
    WF_TRY(upload_tables<double>(c, key + "tc", vc, &ct, st));
    WF_TRY(upload_tables<double>(c, key + "tm", vm, &mt, st));
    WF_TRY(upload_tables<double>(c, key + "ts", vs, &stab, st));
    // scalars
    h.assign(nb, CgScal{});
    for (int m = 0; m < nb; ++m) {
      h[m].nbar = sys[m]->nbar;
      h[m].max_iter = sys[m]->opts.max_iter;
      h[m].tol2 = sys[m]->opts.tol * sys[m]->opts.tol;
      h[m].bb = bb0[m];
      if (this->bad[m]) h[m].done = 4;
    }
    WF_TRY(this->push_scalars(st));
    c.launch("make_D", 16.0 * V * nb, st, [&] { k_make_D<double><<<dim3(152 * 4, nb), 256, 0, st>>>(W, D, sc, inv_vc, V); });
    WF_CUDA(cudaMemsetAsync(xh, 0, nb * SPEC * sizeof(ST), st));
    rel.assign(nb, 1.0);
    state.assign(this->bad.begin(), this->bad.end());
    restarts.assign(nb, 0);
    WF_TRY(start_cg(c, B, st));
    phase = 1;
    return WF_OK;
  }
  // r = C F(rhs) for every system; p = 0; reset the recurrences of the running systems
  wf_status start_cg(Ctx& c, const double* rhs, cudaStream_t st) {
    const size_t SPEC = SP::SPEC;
    SP::zfwd(c, nb, rhs, T, tw, part, false, nullptr, st);
    SP::ypass(c, nb, T, tw, nullptr, -1, st);
    SP::template xmul<true, false, true>(c, nb, T, rh, ct, tw, part, nullptr, st);
    const Bat b = SP::bat();
    c.launch("fin", 0, st, [&] { k_fin_init<<<nb, 1024, 0, st>>>(part, SP::GXY, sc, b); });
    WF_CUDA(cudaMemsetAsync(P0, 0, nb * SPEC * sizeof(ST), st));
    WF_CUDA(cudaMemsetAsync(P1, 0, nb * SPEC * sizeof(ST), st));
    WF_CUDA(cudaGetLastError());
    return WF_OK;
  }
  wf_status block(Ctx& c, cudaStream_t st) {
    return this->run_block(c, st, [&](cudaStream_t s2) {
      for (int i = 0; i < check_every<N>(); ++i)
        SP::iteration(c, nb, rh, P0, P1, xh, T, D, ct, mt, unit_m, tw, part, sc, inv_vc, s2);
    });
  }
  wf_status enqueue(Ctx& c, cudaStream_t st) override {
    if (phase == 1) {
      WF_TRY(block(c, st));
    } else if (phase == 2) {
      const Bat b = SP::bat();
      c.launch("axpy", 3 * SP::BS * nb, st,
               [&] { k_axpy_final<<<dim3(152 * 4, nb), 256, 0, st>>>(xh, P0, P1, SP::SPEC, sc, b); });
      SP::template xmul<false, true, false>(c, nb, xh, T, ct, tw, part, nullptr, st);
      SP::ypass(c, nb, T, tw, nullptr, +1, st);
      SP::template zinv<ZI_STORE>(c, nb, T, S, nullptr, nullptr, nullptr, inv_vc, tw, part, nullptr, st);
      // residual b - A s
      SP::zfwd(c, nb, S, T, tw, part, false, nullptr, st);
      SP::ypass(c, nb, T, tw, nullptr, -1, st);
      SP::template xmul<true, true, false>(c, nb, T, T2, stab, tw, part, nullptr, st);
      SP::ypass(c, nb, T2, tw, nullptr, +1, st);
      SP::template zinv<ZI_RESID>(c, nb, T2, RES, S, W, B, inv_vc, tw, part, sc, st);
      c.launch("fin", 0, st, [&] { k_fin_sum<<<nb, 1024, 0, st>>>(part, SP::GZ, 0, sc, b); });
    } else if (phase == 3) {
      WF_TRY(this->push_scalars(st));
      WF_TRY(start_cg(c, RES, st));
      phase = 1;
      WF_TRY(block(c, st));
    }
    WF_CUDA(cudaGetLastError());
    return this->pull_scalars(st);
  }
  wf_status advance(Ctx&) override {
    this->read_scalars();
    if (phase == 1) {
      if (this->all_done()) phase = 2;
      return WF_OK;
    }
    if (phase == 2) {
      bool any = false;
      for (int m = 0; m < nb; ++m) {
        if (state[m]) {
          h[m].done = 4;
          continue;
        }
        rel[m] = bb0[m] > 0 ? std::sqrt(h[m].aux[0] / bb0[m]) : 0.0;
        wf_status st = WF_OK;
        bool fin = true;
        if (bb0[m] == 0.0 || rel[m] <= sys[m]->opts.tol) st = WF_OK;
        else if (h[m].done == 3) st = WF_ERR_BREAKDOWN;
        else if (h[m].iter >= sys[m]->opts.max_iter || restarts[m] >= 8) st = WF_ERR_NOT_CONVERGED;
        else fin = false;
        if (fin) {
          state[m] = 1;
          h[m].done = 4;
          if (info[m]) *info[m] = wf_solve_info{h[m].iter, restarts[m], rel[m], sys[m]->nbar, st};
        } else {
          restarts[m] += 1;
          h[m].done = 0;
          any = true;
        }
      }
      phase = any ? 3 : 9;
    }
    return WF_OK;
  }
  bool done() const override { return phase == 9; }
  wf_status finish(Ctx&, cudaStream_t st) override {
    for (int m = 0; m < nb; ++m)
      WF_CUDA(cudaMemcpyAsync(sys[m]->s_out, S + m * SP::V, SP::V * sizeof(double), cudaMemcpyDefault, st));
    return WF_OK;
  }
};

// ------------------------------------------------------------------------------------------
// Mixed group: outer FP64 refinement x += e, inner CG on A e = res in FP32 spectra.
// Phases: 0 inner start, 1 CG loop, 2 accumulate + FP64 residual, 9 done.
// ------------------------------------------------------------------------------------------
template <int N>
struct GroupMixed : GroupCommon<N> {
  using SF = Spec<float, N>;
  using SD = Spec<FP64Arith, N>;
  using Base = GroupCommon<N>;
  using Base::nb; using Base::sys; using Base::info; using Base::key; using Base::W; using Base::B;
  using Base::S; using Base::RES; using Base::part; using Base::sc; using Base::tw; using Base::h;
  using Base::phase; using Base::inv_vc; using Base::bb0; using Base::rel; using Base::state;
  float2 *xh, *rh, *P0, *P1, *T;
  float* D;
  double2 *T64, *T64b;
  const float2* tw32 = nullptr;  // FP32 copy of the twiddle table for the FP32 passes
  float *ct, *mt;
  double* stab;
  std::vector<int> outer, iters;
  std::vector<int> noco;  // per system: inner solves without the coarse space after a failed one
  bool unit_m = true;
  static constexpr int NPART = SF::NPART > SD::NPART ? SF::NPART : SD::NPART;
  // coarse space of a deflated group (K > 0; every system of the group has the same K)
  int K = 0, nh = 0, ncp = 0;
  int4* dmodes = nullptr;
  float *Einv = nullptr, *gco = nullptr, *rco = nullptr, *Pb = nullptr, *Rp = nullptr, *Cp = nullptr;
  float2 *Gz = nullptr, *Gy = nullptr, *rsave = nullptr, *DH = nullptr;
  double *dpart = nullptr, *normp = nullptr;  // normp: per-CTA row-sum maxima of E and E^-1
  int* doff = nullptr;  // per system: 1 = the coarse block failed the condition guard (plain CG)
  size_t gzs = 0, gys = 0;

  wf_status prepare_begin(Ctx& c, cudaStream_t st) override {
    nb = (int)sys.size();
    K = sys[0]->opts.deflate;
    // groups of one size with different coarse radii run side by side: their workspaces differ by K
    key = this->tag + "mix_" + std::to_string(N) + "_" + (K > 0 ? "k" + std::to_string(K) + "_" : std::string());
    int* err;
    WF_TRY(c.err_word(&err));
    WF_CUDA(SF::attrs());
    WF_CUDA(SD::attrs());
    const size_t SPEC = SF::SPEC, V = SF::V;
    WF_TRY(c.tw(N, &tw));
    WF_TRY(c.tw32(N, &tw32));
    const char* nm[5] = {"x", "r", "p0", "p1", "T"};
    float2** ptr[5] = {&xh, &rh, &P0, &P1, &T};
    for (int i = 0; i < 5; ++i) WF_TRY(c.get(key + nm[i], nb * SPEC * sizeof(float2), (void**)ptr[i]));
    WF_TRY(c.get(key + "D", nb * V * sizeof(float), (void**)&D));
    WF_TRY(c.get(key + "T64", nb * SPEC * sizeof(double2), (void**)&T64));
    WF_TRY(c.get(key + "T64b", nb * SPEC * sizeof(double2), (void**)&T64b));
    WF_TRY(c.get(key + "W", nb * V * sizeof(double), (void**)&W));
    WF_TRY(c.get(key + "B", nb * V * sizeof(double), (void**)&B));
    WF_TRY(c.get(key + "S", nb * V * sizeof(double), (void**)&S));
    WF_TRY(c.get(key + "RES", nb * V * sizeof(double), (void**)&RES));
    WF_TRY(c.get(key + "part", (size_t)nb * NPART * sizeof(double), (void**)&part));
    WF_TRY(c.get(key + "sc", nb * sizeof(CgScal), (void**)&sc));
    WF_TRY(c.get_pinned(key + "hsc", nb * sizeof(CgScal), (void**)&this->hsc));
    for (int m = 0; m < nb; ++m) {
      WF_CUDA(cudaMemcpyAsync(W + m * V, sys[m]->w, V * sizeof(double), cudaMemcpyDefault, st));
      WF_CUDA(cudaMemcpyAsync(B + m * V, sys[m]->b, V * sizeof(double), cudaMemcpyDefault, st));
    }
    if (K > 0) WF_TRY(defl_alloc(c, st));
    return group_sums_begin<N>(c, *this, NPART, st);
  }
  // the coarse-space buffers and the mode table
  wf_status defl_alloc(Ctx& c, cudaStream_t st) {
    const std::vector<int4> modes = deflation_modes(K);
    nh = (int)modes.size();
    ncp = deflation_ncp(K);
    const size_t C = 4 * K + 1;
    gzs = (size_t)N * N * (K + 1);
    gys = (size_t)(2 * K + 1) * (K + 1) * N;
    const std::string dk = key + "d" + std::to_string(K) + "_";
    WF_TRY(c.get(dk + "E", (size_t)nb * ncp * ncp * sizeof(float), (void**)&Einv));
    WF_TRY(c.get(dk + "gco", (size_t)nb * ncp * sizeof(float), (void**)&gco));
    WF_TRY(c.get(dk + "rco", (size_t)nb * ncp * sizeof(float), (void**)&rco));
    WF_TRY(c.get(dk + "P", (size_t)nb * 2 * kDeflTile * kDeflTile * sizeof(float), (void**)&Pb));
    WF_TRY(c.get(dk + "Rp", (size_t)nb * kDeflTile * ncp * sizeof(float), (void**)&Rp));
    WF_TRY(c.get(dk + "Cp", (size_t)nb * ncp * kDeflTile * sizeof(float), (void**)&Cp));
    WF_TRY(c.get(dk + "Gz", (size_t)nb * gzs * sizeof(float2), (void**)&Gz));
    WF_TRY(c.get(dk + "Gy", (size_t)nb * gys * sizeof(float2), (void**)&Gy));
    WF_TRY(c.get(dk + "rsave", (size_t)nb * (2 * nh + 1) * sizeof(float2), (void**)&rsave));
    WF_TRY(c.get(dk + "DH", (size_t)nb * C * C * C * sizeof(float2), (void**)&DH));
    WF_TRY(c.get(dk + "dpart", (size_t)nb * (nh + 1) * sizeof(double), (void**)&dpart));
    WF_TRY(c.get(dk + "normp", (size_t)nb * 2 * (ncp / 8) * sizeof(double), (void**)&normp));
    WF_TRY(c.get(dk + "doff", (size_t)nb * sizeof(int), (void**)&doff));
    WF_TRY(c.get(dk + "modes", modes.size() * sizeof(int4), (void**)&dmodes));
    int4* hm;
    WF_TRY(c.get_pinned(dk + "hmodes", modes.size() * sizeof(int4), (void**)&hm));
    std::copy(modes.begin(), modes.end(), hm);
    WF_CUDA(cudaMemcpyAsync(dmodes, hm, modes.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    WF_CUDA(cudaMemsetAsync(gco, 0, (size_t)nb * ncp * sizeof(float), st));
    WF_CUDA(cudaMemsetAsync(rco, 0, (size_t)nb * ncp * sizeof(float), st));
    return WF_OK;
  }
  // E^-1 of every system: the transform of w (FP32 passes, P0 as scratch), Dh at the differences
  // of coarse modes, the Galerkin block, and its block Gauss-Jordan exchange
  wf_status defl_setup(Ctx& c, cudaStream_t st) {
    const Bat bf = SF::bat();
    std::vector<double> ones((size_t)nb * SF::TAB, 1.0);
    float* tone;
    WF_TRY(upload_tables<float>(c, key + "t1", ones, &tone, st));
    SF::zfwd(c, nb, W, T, tw32, part, false, nullptr, st);
    SF::ypass(c, nb, T, tw32, nullptr, -1, st);
    SF::template xmul<true, false, true>(c, nb, T, P0, tone, tw32, part, nullptr, st);
    const int C = 4 * K + 1;
    c.launch("defl_dh", 0, st, [&] {
      k_dh_gather<float, N><<<dim3((C * C * C + 255) / 256, nb), 256, 0, st>>>(P0, DH, K, inv_vc, sc, bf);
    });
    c.launch("defl_E", 0, st, [&] {
      k_ebuild<float><<<dim3(ncp / 16, ncp / 16, nb), dim3(16, 16), 0, st>>>(DH, ct, mt, dmodes, nh, ncp, K, Einv,
                                                                            SF::TAB);
    });
    const int nbk = ncp / kDeflTile;
    double* pe = normp;
    double* pi = normp + (size_t)nb * (ncp / 8);
    c.launch("defl_norm", 0, st, [&] { k_defl_rownorm<<<dim3(ncp / 8, nb), 256, 0, st>>>(Einv, ncp, pe); });
    c.launch("gj_pivot", 0, st, [&] { k_gj_pivot<<<dim3(1, 1, nb), 64, 0, st>>>(Einv, Pb, ncp); });
    for (int kb = 0; kb < nbk; ++kb) {
      c.launch("gj_panel", 0, st, [&] { k_gj_panel<<<dim3(nbk, 1, nb), 64, 0, st>>>(Einv, Pb, Rp, Cp, ncp, kb); });
      c.launch("gj_update", 0, st, [&] {
        k_gj_update<<<dim3(nbk / 2, nbk / 2, nb), 256, kUpdSmem, st>>>(Einv, Pb, Rp, Cp, ncp, kb);
      });
    }
    c.launch("defl_norm", 0, st, [&] { k_defl_rownorm<<<dim3(ncp / 8, nb), 256, 0, st>>>(Einv, ncp, pi); });
    c.launch("defl_norm", 0, st, [&] { k_defl_guard<<<nb, 256, 0, st>>>(pe, pi, ncp, doff); });
    WF_CUDA(cudaGetLastError());
    return WF_OK;
  }
  // coordinates of A' r - r and of r, and r -= Z E^-1 g kept aside (MODE 1); or the start vector
  // Z E^-1 Z^T r into `out` (MODE 0)
  template <int MODE>
  void defl_project(Ctx& c, float2* out, cudaStream_t st) {
    const Bat bf = SF::bat();
    const int gw = (nh + 1 + 7) / 8;
    if constexpr (MODE == 1) {
      defl_xr(c, st);
      SF::ypass(c, nb, T, tw32, sc, +1, st);
      c.launch("defl_z", (SF::BS + 4 * SF::BV) * nb, st, [&] {
        k_zcoarse<float, N><<<SF::gz(nb), SF::NTz, SF::SMz, st>>>(T, D, tw32, Gz, K, sc, bf, gzs);
      });
      const size_t ysm = ((size_t)N * (K + 1) + N) * sizeof(float2);
      c.launch("defl_y", 8.0 * gzs * nb, st, [&] {
        k_ycoarse<float, N><<<dim3(N, nb), 256, ysm, st>>>(Gz, tw32, Gy, K, sc, gzs, gys);
      });
    }
    c.launch("defl_x", 8.0 * gys * nb, st, [&] {
      k_xcoarse<float, N, MODE><<<dim3(gw, nb), 256, 0, st>>>(Gy, rh, ct, mt, tw32, dmodes, nh, K, gco, rco, sc, bf,
                                                              gys, ncp);
    });
    c.launch("defl_mu", 4.0 * ncp * ncp * nb, st, [&] {
      k_defl_mu<float, N, MODE><<<dim3(gw, nb), 256, ncp * sizeof(float), st>>>(Einv, gco, rco, dmodes, nh, ncp,
                                                                                 out, rsave, dpart, sc, bf, doff);
    });
  }
  // T = IFFT_x(c r), register-staged (a persistent form on tensor copies along x, the y pass's tile
  // walk with the table multiply and partner column added, took 0.52 ms at 512^3 against 0.42: one
  // CTA per SM cannot hide the table gathers and the strided partner loads)
  void defl_xr(Ctx& c, cudaStream_t st) {
    const Bat bf = SF::bat();
    c.launch("defl_xr", 2 * SF::BS * nb, st, [&] {
      k_xcr<float, N, 32><<<SF::gxy(nb), SF::NTx, SF::SMxy, st>>>(rh, T, ct, tw32, sc, bf);
    });
  }
  // one deflated inner iteration: p = (r - Z mu) + beta p with mu from the coarse projection
  void defl_iteration(Ctx& c, cudaStream_t st) {
    const Bat bf = SF::bat();
    defl_project<1>(c, rh, st);
    c.launch("fin", 0, st, [&] { k_fin_defl<<<nb, 256, 0, st>>>(dpart, nh, sc); });
    SF::iteration(c, nb, rh, P0, P1, xh, T, D, ct, mt, unit_m, tw32, part, sc, inv_vc, st, nullptr,
                  [&](cudaStream_t s) {
                    c.launch("defl_restore", 0, s, [&] {
                      k_defl_restore<float, N><<<dim3((nh + 1 + 255) / 256, nb), 256, 0, s>>>(rh, rsave, dmodes, nh,
                                                                                               sc, bf);
                    });
                  });
  }
  wf_status prepare_end(Ctx& c, cudaStream_t st) override {
    const size_t V = SF::V;
    group_sums_end<N>(*this);
    const int TAB = SF::TAB;
    std::vector<double> vc((size_t)nb * TAB), vm((size_t)nb * TAB), vs((size_t)nb * TAB);
    unit_m = true;
    for (int m = 0; m < nb; ++m) {
      const bool pre = sys[m]->opts.precond != 0;
      unit_m = unit_m && pre;
      const double c0 = 1.0 / std::sqrt(sys[m]->nbar * this->sumw[m] * inv_vc);
      make_tables(sys[m]->sinv, pre, c0, vc.data() + (size_t)m * TAB, vm.data() + (size_t)m * TAB);
      std::copy(sys[m]->sinv.begin(), sys[m]->sinv.end(), vs.begin() + (size_t)m * TAB);
    }
    WF_TRY(upload_tables<float>(c, key + "tc", vc, &ct, st));
    WF_TRY(upload_tables<float>(c, key + "tm", vm, &mt, st));
    WF_TRY(upload_tables<double>(c, key + "ts", vs, &stab, st));
    h.assign(nb, CgScal{});
    for (int m = 0; m < nb; ++m) h[m].nbar = sys[m]->nbar;
    WF_TRY(this->push_scalars(st));
    c.launch("make_D", 12.0 * V * nb, st, [&] { k_make_D<float><<<dim3(152 * 4, nb), 256, 0, st>>>(W, D, sc, inv_vc, V); });
    if (K > 0) WF_TRY(defl_setup(c, st));
    // x = 0 (accumulated in S), res = b
    WF_CUDA(cudaMemsetAsync(S, 0, nb * V * sizeof(double), st));
    WF_CUDA(cudaMemcpyAsync(RES, B, nb * V * sizeof(double), cudaMemcpyDeviceToDevice, st));
    rel.assign(nb, 1.0);
    state.assign(this->bad.begin(), this->bad.end());
    outer.assign(nb, 0);
    iters.assign(nb, 0);
    noco.assign(nb, 0);
    for (int m = 0; m < nb; ++m)
      if (bb0[m] == 0.0 && !state[m]) {
        state[m] = 1;
        rel[m] = 0.0;
        if (info[m]) *info[m] = wf_solve_info{0, 0, 0.0, sys[m]->nbar, WF_OK};
      }
    phase = 0;
    return WF_OK;
  }
  wf_status enqueue(Ctx& c, cudaStream_t st) override {
    const Bat bf = SF::bat();
    if (phase == 0) {
      // Each inner solve aims at the remaining reduction (kInnerMargin of it) but at most
      // inner_tol (1e-4 by default) per step, so at least two FP64 refinement steps run for
      // tol <= 1e-6: the second removes the FP32 rounding error the first leaves in the
      // low-eigenvalue directions (at 512^3 a single step to 1e-6 saves ~6% of the iterations but
      // leaves the solution 3.6e-5 from the converged one, two steps 5e-7).
      const double inner_tol_def = 1e-4;
      for (int m = 0; m < nb; ++m) {
        CgScal z{};
        z.nbar = sys[m]->nbar;
        if (state[m]) {
          z.done = 4;
        } else {
          const double itol = sys[m]->opts.inner_tol > 0.0 ? sys[m]->opts.inner_tol : inner_tol_def;
          const double target = std::max(itol, kInnerMargin * sys[m]->opts.tol / rel[m]);
          z.tol2 = target * target;
          z.bb = rel[m] * rel[m] * bb0[m];
          z.max_iter = std::max(1, sys[m]->opts.max_iter - iters[m]);
          if (K > 0 && !noco[m]) z.max_iter = std::min(z.max_iter, kDeflInnerCap);
          z.noco = noco[m];
          outer[m] += 1;
        }
        h[m] = z;
      }
      WF_TRY(this->push_scalars(st));
      const size_t SPEC = SF::SPEC;
      SF::zfwd(c, nb, RES, T, tw32, part, false, nullptr, st);
      SF::ypass(c, nb, T, tw32, nullptr, -1, st);
      SF::template xmul<true, false, true>(c, nb, T, rh, ct, tw32, part, nullptr, st);
      c.launch("fin", 0, st, [&] { k_fin_init<<<nb, 1024, 0, st>>>(part, SF::GXY, sc, bf); });
      WF_CUDA(cudaMemsetAsync(P0, 0, nb * SPEC * sizeof(float2), st));
      WF_CUDA(cudaMemsetAsync(P1, 0, nb * SPEC * sizeof(float2), st));
      WF_CUDA(cudaMemsetAsync(xh, 0, nb * SPEC * sizeof(float2), st));
      if (K > 0) {
        // the start step of the two-level form: p = Z E^-1 Z^T r (in the FP64 scratch spectrum),
        // taken with alpha = 1 so that x = Z E^-1 Z^T b and Z^T r = 0 afterwards
        float2* Rc = reinterpret_cast<float2*>(T64);
        WF_CUDA(cudaMemsetAsync(Rc, 0, nb * SPEC * sizeof(float2), st));
        c.launch("fin", 0, st, [&] { k_defl_arm<<<nb, 32, 0, st>>>(sc); });
        defl_project<0>(c, Rc, st);
        SF::iteration(c, nb, rh, P0, P1, xh, T, D, ct, mt, unit_m, tw32, part, sc, inv_vc, st, Rc);
      }
      phase = 1;
    }
    if (phase == 1) {
      WF_TRY(this->run_block(c, st, [&](cudaStream_t s2) {
        for (int i = 0; i < check_every<N>(); ++i) {
          if (K > 0) defl_iteration(c, s2);
          else SF::iteration(c, nb, rh, P0, P1, xh, T, D, ct, mt, unit_m, tw32, part, sc, inv_vc, s2);
        }
      }));
    } else if (phase == 2) {
      c.launch("axpy", 3 * SF::BS * nb, st,
               [&] { k_axpy_final<<<dim3(152 * 4, nb), 256, 0, st>>>(xh, P0, P1, SF::SPEC, sc, bf); });
      // x += C e (FP32 transform, FP64 accumulation) for the systems that ran
      SF::template xmul<false, true, false>(c, nb, xh, T, ct, tw32, part, nullptr, st);
      SF::ypass(c, nb, T, tw32, nullptr, +1, st);
      SF::template zinv<ZI_ACCUM>(c, nb, T, S, nullptr, nullptr, nullptr, inv_vc, tw32, part, sc, st);
      // FP64 residual res = b - A x
      SD::zfwd(c, nb, S, T64, tw, part, false, nullptr, st);
      SD::ypass(c, nb, T64, tw, nullptr, -1, st);
      SD::template xmul<true, true, false>(c, nb, T64, T64b, stab, tw, part, nullptr, st);
      SD::ypass(c, nb, T64b, tw, nullptr, +1, st);
      SD::template zinv<ZI_RESID>(c, nb, T64b, RES, S, W, B, inv_vc, tw, part, sc, st);
      const Bat bd = SD::bat();
      c.launch("fin", 0, st, [&] { k_fin_sum<<<nb, 1024, 0, st>>>(part, SD::GZ, 0, sc, bd); });
    }
    WF_CUDA(cudaGetLastError());
    return this->pull_scalars(st);
  }
  wf_status advance(Ctx&) override {
    this->read_scalars();
    if (phase == 1) {
      if (this->all_done()) phase = 2;
      return WF_OK;
    }
    if (phase == 2) {
      bool any = false;
      for (int m = 0; m < nb; ++m) {
        if (state[m]) continue;
        iters[m] += h[m].iter;
        const double rn = std::sqrt(h[m].aux[0] / bb0[m]);
        const bool broke = h[m].done == 3 && !(rn < rel[m]);
        // a deflated inner solve that broke down or reached kDeflInnerCap hands the system to plain
        // CG from the next refinement step on (its FP64 residual restarts the inner solve)
        const bool defl_failed = K > 0 && !noco[m] && std::isfinite(rn) &&
                                 (h[m].done == 3 || (h[m].done == 2 && h[m].iter >= kDeflInnerCap));
        rel[m] = rn;
        wf_status st = WF_OK;
        bool fin = true;
        if (rel[m] <= sys[m]->opts.tol) st = WF_OK;
        else if (defl_failed && outer[m] < 12 && iters[m] < sys[m]->opts.max_iter) {
          noco[m] = 1;
          fin = false;
        } else if (broke) st = WF_ERR_BREAKDOWN;
        else if (outer[m] >= 12 || iters[m] >= sys[m]->opts.max_iter) st = WF_ERR_NOT_CONVERGED;
        else fin = false;
        if (fin) {
          state[m] = 1;
          if (info[m]) *info[m] = wf_solve_info{iters[m], outer[m], rel[m], sys[m]->nbar, st};
        } else {
          any = true;
        }
      }
      phase = any ? 0 : 9;
    }
    return WF_OK;
  }
  bool done() const override { return phase == 9; }
  wf_status finish(Ctx&, cudaStream_t st) override {
    for (int m = 0; m < nb; ++m)
      WF_CUDA(cudaMemcpyAsync(sys[m]->s_out, S + m * SF::V, SF::V * sizeof(double), cudaMemcpyDefault, st));
    return WF_OK;
  }
};

// out = F^-1 [g(|m|^2) F in] for one FP64 field, with the multiplier given as a table over
// n2 = |m|^2 (3 (N/2)^2 + 1 entries): the Gaussian smoothing of Sec. 4.1 and the deconvolution
// B^-1 Z^-1 of Eq. eq:DEC.  The x pass applies the table as it applies the prior; the transforms
// are the solver's FP64 passes.  in may equal out.
template <int N>
wf_status fourier_multiply_n(Ctx& c, const double* in, double* out, const std::vector<double>& table, cudaStream_t st) {
  using SD = Spec<FP64Arith, N>;
  if ((int)table.size() != SD::TAB) return WF_ERR_ARG;
  int* err;
  WF_TRY(c.err_word(&err));
  WF_CUDA(SD::attrs());
  const double2* tw;
  WF_TRY(c.tw(N, &tw));
  double2 *T, *T2;
  double* part;
  WF_TRY(c.get("sm_T", SD::SPEC * sizeof(double2), (void**)&T));
  WF_TRY(c.get("sm_T2", SD::SPEC * sizeof(double2), (void**)&T2));
  WF_TRY(c.get("sm_part", (size_t)SD::NPART * sizeof(double), (void**)&part));
  double* gt;
  WF_TRY(upload_tables<double>(c, "sm_g", table, &gt, st));
  SD::zfwd(c, 1, in, T, tw, part, false, nullptr, st);
  SD::ypass(c, 1, T, tw, nullptr, -1, st);
  SD::template xmul<true, true, false>(c, 1, T, T2, gt, tw, part, nullptr, st);
  SD::ypass(c, 1, T2, tw, nullptr, +1, st);
  SD::template zinv<ZI_STORE>(c, 1, T2, out, nullptr, nullptr, nullptr, 1.0 / (double)SD::V, tw, part, nullptr,
                              st);
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaStreamSynchronize(st));
  return c.check_device_errors();
}

// ---- autotuner: time each launch variant of a pass on a working set larger than L2 ----------
template <class SP, class V>
wf_status tune_pass(Ctx& c, const char* pass, const std::vector<V>& vs, typename SP::ST* buf, int nb,
                    const typename SP::ST* tw, cudaStream_t st, std::string& report) {
  const std::string key = SP::tune_key(pass);
  char head[160];
  std::snprintf(head, sizeof head, "{\"pass\": \"%s\", \"systems\": %d, \"variants\": [", key.c_str(), nb);
  report += head;
  cudaEvent_t a, b;
  WF_CUDA(cudaEventCreate(&a));
  WF_CUDA(cudaEventCreate(&b));
  int best = 0;
  float best_ms = 1e30f;
  const bool prof = c.prof.on;
  c.prof.on = false;  // the tuner's launches are not part of a profile
  wf_status status = WF_OK;
  for (size_t i = 0; i < vs.size() && status == WF_OK; ++i) {
    constexpr int kWarm = 2, kRuns = 6;
    for (int r = 0; r < kWarm; ++r) vs[i].run(c, nb, buf, tw, nullptr, -1, st);
    cudaEventRecord(a, st);
    for (int r = 0; r < kRuns; ++r) vs[i].run(c, nb, buf, tw, nullptr, r & 1 ? +1 : -1, st);
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
      set_last_error("autotune timing", e);
      status = WF_ERR_CUDA;
      break;
    }
    ms /= kRuns;
    char item[128];
    std::snprintf(item, sizeof item, "%s{\"name\": \"%s\", \"ms\": %.5f}", i ? ", " : "", vs[i].name, ms);
    report += item;
    if (ms < best_ms) {
      best_ms = ms;
      best = (int)i;
    }
  }
  c.prof.on = prof;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  WF_TRY(status);
  WF_TRY(c.check_device_errors());
  c.tuned[key] = best;
  char tail[96];
  std::snprintf(tail, sizeof tail, "], \"chosen\": \"%s\"}", vs[best].name);
  report += tail;
  return WF_OK;
}

template <class SP>
wf_status tune_spec(Ctx& c, std::string& report) {
  using ST = typename SP::ST;
  int* err;
  WF_TRY(c.err_word(&err));
  WF_CUDA(SP::attrs());
  const ST* tw;
  if constexpr (sizeof(typename SP::SS) == 8) {
    WF_TRY(c.tw(SP::NH * 2, &tw));
  } else {
    WF_TRY(c.tw32(SP::NH * 2, &tw));
  }
  // enough systems that the working set (read and written once per pass) is at least 256 MB,
  // so that the passes stream from HBM as they do in a large solve or a batch
  const double spec_bytes = (double)SP::SPEC * sizeof(ST);
  int nb = (int)std::ceil((256.0 * (1 << 20)) / spec_bytes);
  nb = std::max(1, std::min(nb, 64));
  ST* buf;
  WF_TRY(c.get("tune_spec", (size_t)nb * SP::SPEC * sizeof(ST), (void**)&buf));
  cudaStream_t st;
  WF_TRY(c.stream(0, &st));
  WF_CUDA(cudaMemsetAsync(buf, 0, (size_t)nb * SP::SPEC * sizeof(ST), st));
  WF_TRY(tune_pass<SP>(c, "ypass", SP::yvariants(), buf, nb, tw, st, report));
  WF_CUDA(cudaStreamSynchronize(st));
  c.release_prefix("tune_spec");
  // the CG x passes: five spectra per system, scalars of running systems, unit tables
  using SS = typename SP::SS;
  const size_t SPEC = SP::SPEC;
  ST* xb;
  SS* tab;
  double* part;
  CgScal* sc;
  WF_TRY(c.get("tune_x", (size_t)5 * nb * SPEC * sizeof(ST), (void**)&xb));
  WF_TRY(c.get("tune_xtab", (size_t)nb * SP::TAB * sizeof(SS), (void**)&tab));
  WF_TRY(c.get("tune_xpart", (size_t)nb * SP::NPART * sizeof(double), (void**)&part));
  WF_TRY(c.get("tune_xsc", (size_t)nb * sizeof(CgScal), (void**)&sc));
  WF_CUDA(cudaMemsetAsync(xb, 0, (size_t)5 * nb * SPEC * sizeof(ST), st));
  WF_CUDA(cudaMemsetAsync(sc, 0, (size_t)nb * sizeof(CgScal), st));
  {
    std::vector<SS> ones((size_t)nb * SP::TAB, (SS)1);
    WF_CUDA(cudaMemcpyAsync(tab, ones.data(), ones.size() * sizeof(SS), cudaMemcpyHostToDevice, st));
    WF_CUDA(cudaStreamSynchronize(st));
  }
  ST *r = xb, *P0 = xb + nb * SPEC, *P1 = xb + 2 * nb * SPEC, *x = xb + 3 * nb * SPEC, *T = xb + 4 * nb * SPEC;
  struct XRun {
    const typename SP::XVariant* v;
    bool inv;
    const char* name;
    void run(Ctx& c, int nb, cudaStream_t st, ST* r, ST* P0, ST* P1, ST* x, ST* T, const SS* tab, const ST* tw,
             double* part, CgScal* sc, int, int) const {
      if (inv) v->xinv(c, nb, r, P0, P1, x, T, tab, tab, true, tw, part, sc, st);
      else v->xupd(c, nb, T, r, P0, P1, tab, tab, true, tw, part, sc, st);
    }
  };
  for (int inv = 1; inv >= 0; --inv) {
    std::vector<XRun> runs;
    for (const auto& v : SP::xvariants()) runs.push_back(XRun{&v, inv == 1, v.name});
    struct Adapter {
      const XRun* x;
      ST *r, *P0, *P1, *xx, *T;
      const SS* tab;
      double* part;
      CgScal* sc;
      const char* name;
      void run(Ctx& c, int nb, ST*, const ST* tw, const CgScal*, int, cudaStream_t st) const {
        x->run(c, nb, st, r, P0, P1, xx, T, tab, tw, part, sc, 0, 0);
      }
    };
    std::vector<Adapter> ad;
    for (const auto& rr : runs) ad.push_back(Adapter{&rr, r, P0, P1, x, T, tab, part, sc, rr.name});
    report += ", ";
    WF_TRY(tune_pass<SP>(c, inv ? "xinv" : "xupd", ad, r, nb, tw, st, report));
  }
  {  // the z turn: T and D (FP32/FP64 real field, one spectrum's bytes or half) from the scratch
    struct ZAdapter {
      const typename SP::ZVariant* v;
      SS* D;
      double* part;
      CgScal* sc;
      const char* name;
      void run(Ctx& c, int nb, ST* buf, const ST* tw, const CgScal*, int, cudaStream_t st) const {
        v->run(c, nb, buf, D, tw, part, sc, st);
      }
    };
    std::vector<ZAdapter> za;
    SS* D = reinterpret_cast<SS*>(x);  // the x buffer holds nb fields of V reals (zeroed)
    for (const auto& v : SP::zvariants()) za.push_back(ZAdapter{&v, D, part, sc, v.name});
    report += ", ";
    WF_TRY(tune_pass<SP>(c, "zturn", za, T, nb, tw, st, report));
  }
  WF_CUDA(cudaStreamSynchronize(st));
  c.release_prefix("tune_x");
  return WF_OK;
}

template <int N>
wf_status autotune_n(Ctx& c, int prec, std::string& report) {
  if (prec == WF_MIXED) return tune_spec<Spec<float, N>>(c, report);
  return tune_spec<Spec<FP64Arith, N>>(c, report);
}

template <int N>
Group* make_group(int prec) {
  if (prec == WF_MIXED) return new GroupMixed<N>();
  return new GroupFP64<FP64Arith, N>();
}

}  // namespace wf
