// wf_solver_impl.cuh -- drivers of the Wiener solve (Kitaura et al. 2009, Sec. 2.5.1, Eq. eq:WF).
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
// One CG iteration = 5 FFT passes + 1 update sweep:
//   x pass 1: p = r + beta p, x += alpha_prev p_old, T = IFFT_x(c p)
//   y pass  : IFFT_y
//   z turn  : IFFT_z, times D / V_c, FFT_z
//   y pass  : FFT_y
//   x pass 2: FFT_x, q = m p + c T, <p, q>
//   finisher: alpha;  update: r -= alpha q, <r, r>, ||C^-1 r||^2;  finisher: beta, stop test
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "wf_ctx.h"
#include "wf_spectral.cuh"

namespace wf {

template <class K>
static inline cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Launch geometry and launchers of the spectral passes for one arithmetic type and size.
template <class R, int N>
struct Spec {
  using ST = typename Store<R>::T;
  using SS = typename Store<R>::S;
  static constexpr int NH = N / 2;
  static constexpr int NLxy = xy_lines<R, N>();
  static_assert(NH % NLxy == 0 && (N * N) % tile_lines<R>() == 0, "tile widths must divide the grid");
  static constexpr int TPLn = tpl<R, N>();
  static constexpr int NTy = NLxy * TPLn;
  static constexpr int NTx = (NLxy + 1) * TPLn;
  static constexpr size_t SMxy = (size_t)(N * (NLxy + 1) + N) * sizeof(cx<R>);
  static constexpr int NLz = tile_lines<R>();
  static constexpr int TPLh = tpl<R, NH>();
  static constexpr int NTz = NLz * TPLh;
  static constexpr size_t SMz = (size_t)(NH * (NLz + 1) + 2 * N) * sizeof(cx<R>);
  static constexpr int GXY = (NH / NLxy) * N;   // blocks of an x or y pass
  static constexpr int GZ = N * N / NLz;        // blocks of a z pass
  static constexpr int GU = 152 * 4;            // blocks of the update sweep
  static constexpr size_t SPEC = (size_t)N * N * NH;  // complex elements of a spectrum
  static dim3 gxy() { return dim3(NH / NLxy, N); }

  static cudaError_t attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define WF_A(k, b) if (e == cudaSuccess) e = set_smem(k, b)
    WF_A((k_ypass<R, N, -1>), SMxy);
    WF_A((k_ypass<R, N, +1>), SMxy);
    WF_A((k_cg_xinv<R, N>), SMxy);
    WF_A((k_cg_xfwd<R, N>), SMxy);
    WF_A((k_xmul<R, N, true, false, true>), SMxy);
    WF_A((k_xmul<R, N, true, false, false>), SMxy);
    WF_A((k_xmul<R, N, false, true, false>), SMxy);
    WF_A((k_xmul<R, N, true, true, false>), SMxy);
    WF_A((k_zturn<R, N>), SMz);
    WF_A((k_zfwd<R, N, true>), SMz);
    WF_A((k_zfwd<R, N, false>), SMz);
    WF_A((k_zinv<R, N, ZI_STORE>), SMz);
    WF_A((k_zinv<R, N, ZI_RESID>), SMz);
    WF_A((k_zinv<R, N, ZI_ACCUM>), SMz);
#undef WF_A
    if (e == cudaSuccess) done = true;
    return e;
  }

  // algorithmic bytes of one launch (DRAM traffic the pass cannot avoid)
  static constexpr double BS = (double)SPEC * sizeof(ST);   // one spectrum
  static constexpr double BV = (double)N * N * N;           // cells

  static void ypass(Ctx& c, ST* t, const double2* tw, const CgScal* sc, int dir, cudaStream_t st) {
    c.launch("ypass", 2 * BS, st, [&] {
      if (dir < 0) k_ypass<R, N, -1><<<gxy(), NTy, SMxy, st>>>(t, tw, sc);
      else k_ypass<R, N, +1><<<gxy(), NTy, SMxy, st>>>(t, tw, sc);
    });
  }
  // out = [IFFT_x] tab (.) [FFT_x] in
  template <bool FWD, bool INV, bool DOT>
  static void xmul(Ctx& c, const ST* in, ST* out, const SS* tab, const double2* tw, double* part,
                   const CgScal* sc, cudaStream_t st) {
    c.launch("xmul", 2 * BS, st, [&] { k_xmul<R, N, FWD, INV, DOT><<<gxy(), NTx, SMxy, st>>>(in, out, tab, tw, part, sc); });
  }
  static void zfwd(Ctx& c, const double* in, ST* out, const double2* tw, double* part, bool sq, const CgScal* sc,
                   cudaStream_t st) {
    c.launch("zfwd", BS + 8 * BV, st, [&] {
      if (sq) k_zfwd<R, N, true><<<GZ, NTz, SMz, st>>>(in, out, tw, part, sc);
      else k_zfwd<R, N, false><<<GZ, NTz, SMz, st>>>(in, out, tw, part, sc);
    });
  }
  template <int MODE>
  static void zinv(Ctx& c, const ST* in, double* out, const double* s, const double* w, const double* b, double nbar,
                   double scl, const double2* tw, double* part, const CgScal* sc, cudaStream_t st) {
    const double vb = MODE == ZI_RESID ? 4 : (MODE == ZI_ACCUM ? 2 : 1);
    c.launch("zinv", BS + 8 * vb * BV, st,
             [&] { k_zinv<R, N, MODE><<<GZ, NTz, SMz, st>>>(in, out, s, w, b, nbar, scl, tw, part, sc); });
  }

  // One CG iteration on the device (no host synchronisation).
  static void iteration(Ctx& c, ST* r, ST* pold, ST* pnew, ST* x, ST* T, ST* q, const SS* D, const SS* ctab,
                        const SS* mtab, const double2* tw, double* part, CgScal* sc, double inv_vc,
                        cudaStream_t st) {
    c.launch("cg_xinv", 6 * BS, st, [&] { k_cg_xinv<R, N><<<gxy(), NTx, SMxy, st>>>(r, pold, pnew, x, T, ctab, tw, sc); });
    c.launch("ypass", 2 * BS, st, [&] { k_ypass<R, N, +1><<<gxy(), NTy, SMxy, st>>>(T, tw, sc); });
    c.launch("zturn", 2 * BS + sizeof(SS) * BV, st, [&] { k_zturn<R, N><<<GZ, NTz, SMz, st>>>(T, D, tw, sc); });
    c.launch("ypass", 2 * BS, st, [&] { k_ypass<R, N, -1><<<gxy(), NTy, SMxy, st>>>(T, tw, sc); });
    c.launch("cg_xfwd", 3 * BS, st, [&] { k_cg_xfwd<R, N><<<gxy(), NTx, SMxy, st>>>(T, pnew, q, ctab, mtab, tw, part, sc); });
    c.launch("fin", 0, st, [&] { k_fin_alpha<<<1, 1024, 0, st>>>(part, GXY, sc); });
    c.launch("cg_update", 3 * BS, st, [&] { k_update<R, N><<<GU, 256, 0, st>>>(r, q, ctab, part, sc); });
    c.launch("fin", 0, st, [&] { k_fin_beta<<<1, 1024, 0, st>>>(part, GU, inv_vc, sc); });
  }
};

// ---- small elementwise helpers -----------------------------------------------------------
template <class SSo>
__global__ void k_scale_copy(const double* __restrict__ in, SSo* __restrict__ out, double f, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (SSo)(in[i] * f);
}
static __global__ void k_sum(const double* __restrict__ in, size_t n, double* __restrict__ partials) {
  __shared__ double red[32];
  AccD acc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc.add(in[i]);
  const double s = block_sum(acc.get(), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}
static __global__ void k_sumsq(const double* __restrict__ in, size_t n, double* __restrict__ partials) {
  __shared__ double red[32];
  AccD acc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc.add_prod(in[i], in[i]);
  const double s = block_sum(acc.get(), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Tables: sinv[n2]; ctab[n2] = c(k), mtab[n2] = c^2 S^-1 (k).
static void make_tables(const std::vector<double>& sinv, bool precond, double c0, std::vector<double>& ct,
                        std::vector<double>& mt) {
  const size_t L = sinv.size();
  ct.resize(L);
  mt.resize(L);
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

static inline wf_status read_scal(Ctx& c, const CgScal* dsc, CgScal* out, cudaStream_t st) {
  CgScal* h = reinterpret_cast<CgScal*>(c.host_pinned);
  WF_CUDA(cudaMemcpyAsync(h, dsc, sizeof(CgScal), cudaMemcpyDeviceToHost, st));
  WF_CUDA(cudaStreamSynchronize(st));
  *out = *h;
  return WF_OK;
}
static inline wf_status write_scal(Ctx& c, CgScal* dsc, const CgScal& v, cudaStream_t st) {
  CgScal* h = reinterpret_cast<CgScal*>(c.host_pinned) + 1;
  *h = v;
  WF_CUDA(cudaMemcpyAsync(dsc, h, sizeof(CgScal), cudaMemcpyHostToDevice, st));
  WF_CUDA(cudaStreamSynchronize(st));
  return WF_OK;
}

template <class T>
static inline wf_status upload(Ctx& c, const char* name, const std::vector<double>& v, const T** out, cudaStream_t st) {
  std::vector<T> tmp(v.begin(), v.end());
  T* d;
  WF_TRY(c.get(name, tmp.size() * sizeof(T), (void**)&d));
  WF_CUDA(cudaMemcpyAsync(d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  WF_CUDA(cudaStreamSynchronize(st));  // tmp goes out of scope
  *out = d;
  return WF_OK;
}

// Explicit canonical residual: res = b - A s (FP64 storage), returns ||res||^2 via *rr.
// Uses spectra T, T2 and the FP64 S^-1 table.
template <class RD, int N>
static wf_status residual(Ctx& c, const double* s, const double* w, const double* b, double nbar,
                          const double* sinv_d, double* res, typename Store<RD>::T* T, typename Store<RD>::T* T2,
                          double* part, CgScal* sc, double* rr, cudaStream_t st) {
  using SP = Spec<RD, N>;
  const double2* tw;
  WF_TRY(c.tw(N, &tw));
  const double inv_vc = 1.0 / ((double)N * N * N);
  SP::zfwd(c, s, T, tw, part, false, nullptr, st);
  SP::ypass(c, T, tw, nullptr, -1, st);
  SP::template xmul<true, true, false>(c, T, T2, sinv_d, tw, part, nullptr, st);
  SP::ypass(c, T2, tw, nullptr, +1, st);
  SP::template zinv<ZI_RESID>(c, T2, res, s, w, b, nbar, inv_vc, tw, part, nullptr, st);
  c.launch("fin", 0, st, [&] { k_fin_sum<<<1, 1024, 0, st>>>(part, SP::GZ, 0, sc); });
  WF_CUDA(cudaGetLastError());
  CgScal h;
  WF_TRY(read_scal(c, sc, &h, st));
  *rr = h.aux[0];
  return WF_OK;
}

// Run CG iterations until the device reports done; returns the final CgScal.
// P[0], P[1]: ping-pong search directions; `j0` = iterations run since they were reset.
template <class R, int N>
static wf_status cg_loop(Ctx& c, typename Store<R>::T* r, typename Store<R>::T** P, typename Store<R>::T* x,
                         typename Store<R>::T* T, typename Store<R>::T* q, const typename Store<R>::S* D,
                         const typename Store<R>::S* ctab, const typename Store<R>::S* mtab, double* part, CgScal* sc,
                         CgScal* out, cudaStream_t st) {
  using SP = Spec<R, N>;
  const double2* tw;
  WF_TRY(c.tw(N, &tw));
  const double inv_vc = 1.0 / ((double)N * N * N);
  CgScal h;
  WF_TRY(read_scal(c, sc, &h, st));
  const int it_start = h.iter;
  int launched = 0;
  // check the device flag every `blk` iterations; small grids check less often
  const int blk = N >= 256 ? 4 : (N >= 128 ? 16 : 32);
  while (!h.done) {
    for (int i = 0; i < blk; ++i) {
      const int j = launched + i;
      SP::iteration(c, r, P[j & 1], P[(j + 1) & 1], x, T, q, D, ctab, mtab, tw, part, sc, inv_vc, st);
    }
    WF_CUDA(cudaGetLastError());
    launched += blk;
    WF_TRY(read_scal(c, sc, &h, st));
  }
  // apply the last alpha: the direction of the last completed iteration
  const int jl = h.iter - it_start - 1;
  if (jl >= 0) {
    c.launch("axpy", 3 * SP::BS, st, [&] { k_axpy_final<<<152 * 4, 256, 0, st>>>(x, P[(jl + 1) & 1], SP::SPEC, sc); });
    WF_CUDA(cudaGetLastError());
  }
  *out = h;
  return WF_OK;
}

// ==========================================================================================
// FP64 solve: FP64 storage; spectral arithmetic in R (double or df32).
// ==========================================================================================
template <class R, int N>
static wf_status solve_fp64(Ctx& c, SolveArgs& a, wf_solve_info* info, cudaStream_t st) {
  using SP = Spec<R, N>;
  using ST = double2;
  static_assert(sizeof(typename Store<R>::T) == sizeof(double2), "FP64 storage");
  WF_CUDA(SP::attrs());
  WF_CUDA(Spec<double, N>::attrs());
  const size_t V = (size_t)N * N * N, SPEC = SP::SPEC;
  const double inv_vc = 1.0 / (double)V;
  const double2* tw;
  WF_TRY(c.tw(N, &tw));
  ST *xh, *rh, *P[2], *qh, *T, *T2;
  double *D, *res, *part;
  CgScal* sc;
  WF_TRY(c.get("s_x", SPEC * sizeof(ST), (void**)&xh));
  WF_TRY(c.get("s_r", SPEC * sizeof(ST), (void**)&rh));
  WF_TRY(c.get("s_p0", SPEC * sizeof(ST), (void**)&P[0]));
  WF_TRY(c.get("s_p1", SPEC * sizeof(ST), (void**)&P[1]));
  WF_TRY(c.get("s_q", SPEC * sizeof(ST), (void**)&qh));
  WF_TRY(c.get("s_T", SPEC * sizeof(ST), (void**)&T));
  WF_TRY(c.get("s_T2", SPEC * sizeof(ST), (void**)&T2));
  WF_TRY(c.get("s_D", V * sizeof(double), (void**)&D));
  WF_TRY(c.get("s_res", V * sizeof(double), (void**)&res));
  const size_t np = (size_t)std::max({SP::GXY, SP::GZ, 2 * SP::GU});
  WF_TRY(c.get("s_part", np * sizeof(double), (void**)&part));
  WF_TRY(c.get("s_sc", sizeof(CgScal), (void**)&sc));

  // sum(w) for c_0 and ||b||^2
  CgScal init{};
  init.max_iter = a.opts.max_iter;
  init.tol2 = a.opts.tol * a.opts.tol;
  WF_TRY(write_scal(c, sc, init, st));
  c.launch("reduce", 8.0 * V, st, [&] { k_sum<<<SP::GU, 256, 0, st>>>(a.w, V, part); });
  c.launch("fin", 0, st, [&] { k_fin_sum<<<1, 1024, 0, st>>>(part, SP::GU, 1, sc); });
  WF_CUDA(cudaGetLastError());
  CgScal h;
  WF_TRY(read_scal(c, sc, &h, st));
  const double sum_w = h.aux[1];
  if (!(sum_w > 0.0)) return WF_ERR_ARG;
  const double c0 = 1.0 / std::sqrt(a.nbar * sum_w * inv_vc);
  std::vector<double> ct, mt;
  make_tables(a.sinv, a.opts.precond != 0, c0, ct, mt);
  const double *ctab, *mtab, *stab;
  WF_TRY(upload<double>(c, "t_c", ct, &ctab, st));
  WF_TRY(upload<double>(c, "t_m", mt, &mtab, st));
  WF_TRY(upload<double>(c, "t_s", a.sinv, &stab, st));
  c.launch("scale_copy", 16.0 * V, st, [&] { k_scale_copy<double><<<SP::GU, 256, 0, st>>>(a.w, D, a.nbar * inv_vc, V); });

  int iters = 0, restarts = 0;
  double rel = 1.0;
  wf_status status = WF_OK;
  // r = C b (with ||b||^2), x = 0
  const double* rhs = a.b;
  for (;;) {
    SP::zfwd(c, rhs, T, tw, part, true, nullptr, st);
    if (rhs == a.b) c.launch("fin", 0, st, [&] { k_fin_sum<<<1, 1024, 0, st>>>(part, SP::GZ, -1, sc); });
    SP::ypass(c, T, tw, nullptr, -1, st);
    SP::template xmul<true, false, true>(c, T, rh, ctab, tw, part, nullptr, st);
    c.launch("fin", 0, st, [&] { k_fin_init<<<1, 1024, 0, st>>>(part, SP::GXY, sc); });
    WF_CUDA(cudaMemsetAsync(P[0], 0, SPEC * sizeof(ST), st));
    WF_CUDA(cudaMemsetAsync(P[1], 0, SPEC * sizeof(ST), st));
    if (rhs == a.b) WF_CUDA(cudaMemsetAsync(xh, 0, SPEC * sizeof(ST), st));
    WF_CUDA(cudaGetLastError());
    CgScal fin;
    WF_TRY(cg_loop<R, N>(c, rh, P, xh, T, qh, D, ctab, mtab, part, sc, &fin, st));
    iters = fin.iter;
    if (fin.bb == 0.0) {  // b = 0: s = 0
      WF_CUDA(cudaMemsetAsync(a.s_out, 0, V * sizeof(double), st));
      rel = 0.0;
      break;
    }
    // s = C x (real space)
    SP::template xmul<false, true, false>(c, xh, T, ctab, tw, part, nullptr, st);
    SP::ypass(c, T, tw, nullptr, +1, st);
    SP::template zinv<ZI_STORE>(c, T, a.s_out, nullptr, nullptr, nullptr, 0.0, inv_vc, tw, part, nullptr, st);
    WF_CUDA(cudaGetLastError());
    double rr;
    WF_TRY((residual<R, N>(c, a.s_out, a.w, a.b, a.nbar, stab, res, T, T2, part, sc, &rr, st)));
    rel = std::sqrt(rr / fin.bb);
    if (rel <= a.opts.tol) break;
    if (fin.done == 3) {
      status = WF_ERR_BREAKDOWN;
      break;
    }
    if (fin.iter >= a.opts.max_iter || restarts >= 8) {
      status = WF_ERR_NOT_CONVERGED;
      break;
    }
    // restart from the recomputed residual; the done flag is cleared by k_fin_init
    ++restarts;
    rhs = res;
  }
  if (info) {
    info->iters = iters;
    info->outer_iters = restarts;
    info->rel_residual = rel;
    info->nbar = a.nbar;
    info->status = status;
  }
  return status;
}

// ==========================================================================================
// Mixed precision: outer FP64 refinement x += e, inner CG on A e = res in FP32 spectra.
// ==========================================================================================
template <int N>
static wf_status solve_mixed(Ctx& c, SolveArgs& a, wf_solve_info* info, cudaStream_t st) {
  using SF = Spec<float, N>;
  using SD = Spec<double, N>;
  WF_CUDA(SF::attrs());
  WF_CUDA(SD::attrs());
  const size_t V = (size_t)N * N * N, SPEC = SF::SPEC;
  const double inv_vc = 1.0 / (double)V;
  const double2* tw;
  WF_TRY(c.tw(N, &tw));
  float2 *xh, *rh, *P[2], *qh, *T;
  float* D;
  double2 *T64, *T64b;
  double *res, *part;
  CgScal* sc;
  WF_TRY(c.get("m_x", SPEC * sizeof(float2), (void**)&xh));
  WF_TRY(c.get("m_r", SPEC * sizeof(float2), (void**)&rh));
  WF_TRY(c.get("m_p0", SPEC * sizeof(float2), (void**)&P[0]));
  WF_TRY(c.get("m_p1", SPEC * sizeof(float2), (void**)&P[1]));
  WF_TRY(c.get("m_q", SPEC * sizeof(float2), (void**)&qh));
  WF_TRY(c.get("m_T", SPEC * sizeof(float2), (void**)&T));
  WF_TRY(c.get("m_D", V * sizeof(float), (void**)&D));
  WF_TRY(c.get("s_T", SPEC * sizeof(double2), (void**)&T64));
  WF_TRY(c.get("s_T2", SPEC * sizeof(double2), (void**)&T64b));
  WF_TRY(c.get("s_res", V * sizeof(double), (void**)&res));
  // partials: the FP32 inner passes and the FP64 residual passes both write here
  const size_t np = (size_t)std::max({SF::GXY, SF::GZ, 2 * SF::GU, SD::GXY, SD::GZ, 2 * SD::GU});
  WF_TRY(c.get("s_part", np * sizeof(double), (void**)&part));
  WF_TRY(c.get("s_sc", sizeof(CgScal), (void**)&sc));

  CgScal init{};
  WF_TRY(write_scal(c, sc, init, st));
  c.launch("reduce", 8.0 * V, st, [&] { k_sum<<<SF::GU, 256, 0, st>>>(a.w, V, part); });
  c.launch("fin", 0, st, [&] { k_fin_sum<<<1, 1024, 0, st>>>(part, SF::GU, 1, sc); });
  WF_CUDA(cudaGetLastError());
  CgScal h;
  WF_TRY(read_scal(c, sc, &h, st));
  const double sum_w = h.aux[1];
  if (!(sum_w > 0.0)) return WF_ERR_ARG;
  const double c0 = 1.0 / std::sqrt(a.nbar * sum_w * inv_vc);
  std::vector<double> ct, mt;
  make_tables(a.sinv, a.opts.precond != 0, c0, ct, mt);
  const float *ctab, *mtab;
  const double* stab;
  WF_TRY(upload<float>(c, "tf_c", ct, &ctab, st));
  WF_TRY(upload<float>(c, "tf_m", mt, &mtab, st));
  WF_TRY(upload<double>(c, "t_s", a.sinv, &stab, st));
  c.launch("scale_copy", 12.0 * V, st, [&] { k_scale_copy<float><<<SF::GU, 256, 0, st>>>(a.w, D, a.nbar * inv_vc, V); });
  // x = s_out = 0; res = b; ||b||^2
  double* x = a.s_out;
  WF_CUDA(cudaMemsetAsync(x, 0, V * sizeof(double), st));
  WF_CUDA(cudaMemcpyAsync(res, a.b, V * sizeof(double), cudaMemcpyDeviceToDevice, st));
  c.launch("reduce", 8.0 * V, st, [&] { k_sumsq<<<SF::GU, 256, 0, st>>>(a.b, V, part); });
  c.launch("fin", 0, st, [&] { k_fin_sum<<<1, 1024, 0, st>>>(part, SF::GU, 0, sc); });
  WF_CUDA(cudaGetLastError());
  WF_TRY(read_scal(c, sc, &h, st));
  const double bb = h.aux[0];
  wf_status status = WF_OK;
  int total_iters = 0, outer = 0;
  double rel = 1.0;
  const double inner_tol = a.opts.inner_tol > 0.0 ? a.opts.inner_tol : 1e-4;
  if (bb == 0.0) rel = 0.0;
  while (rel > a.opts.tol) {
    if (outer >= 12 || total_iters >= a.opts.max_iter) {
      status = WF_ERR_NOT_CONVERGED;
      break;
    }
    ++outer;
    const double target = std::max(inner_tol, 0.3 * a.opts.tol / rel);
    // inner: r~ = C res (FP32), CG to ||res - A e|| <= target ||res||
    CgScal in{};
    in.max_iter = a.opts.max_iter - total_iters;
    in.tol2 = target * target;
    in.bb = rel * rel * bb;
    WF_TRY(write_scal(c, sc, in, st));
    SF::zfwd(c, res, T, tw, part, false, nullptr, st);
    SF::ypass(c, T, tw, nullptr, -1, st);
    SF::template xmul<true, false, true>(c, T, rh, ctab, tw, part, nullptr, st);
    c.launch("fin", 0, st, [&] { k_fin_init<<<1, 1024, 0, st>>>(part, SF::GXY, sc); });
    WF_CUDA(cudaMemsetAsync(P[0], 0, SPEC * sizeof(float2), st));
    WF_CUDA(cudaMemsetAsync(P[1], 0, SPEC * sizeof(float2), st));
    WF_CUDA(cudaMemsetAsync(xh, 0, SPEC * sizeof(float2), st));
    WF_CUDA(cudaGetLastError());
    CgScal fin;
    WF_TRY(cg_loop<float, N>(c, rh, P, xh, T, qh, D, ctab, mtab, part, sc, &fin, st));
    total_iters += fin.iter;
    // x += C e (FP32 transform, FP64 accumulation)
    SF::template xmul<false, true, false>(c, xh, T, ctab, tw, part, nullptr, st);
    SF::ypass(c, T, tw, nullptr, +1, st);
    SF::template zinv<ZI_ACCUM>(c, T, x, nullptr, nullptr, nullptr, 0.0, inv_vc, tw, part, nullptr, st);
    WF_CUDA(cudaGetLastError());
    // FP64 residual
    double rr;
    WF_TRY((residual<double, N>(c, x, a.w, a.b, a.nbar, stab, res, T64, T64b, part, sc, &rr, st)));
    const double rel_new = std::sqrt(rr / bb);
    if (!(rel_new < rel) && fin.done == 3) {
      rel = rel_new;
      status = WF_ERR_BREAKDOWN;
      break;
    }
    rel = rel_new;
  }
  if (info) {
    info->iters = total_iters;
    info->outer_iters = outer;
    info->rel_residual = rel;
    info->nbar = a.nbar;
    info->status = status;
  }
  return status;
}

template <int N>
wf_status solve_sized(Ctx& c, SolveArgs& a, wf_solve_info* info, cudaStream_t st) {
  if (a.opts.prec == WF_MIXED) return solve_mixed<N>(c, a, info, st);
  return solve_fp64<double, N>(c, a, info, st);
}

}  // namespace wf
