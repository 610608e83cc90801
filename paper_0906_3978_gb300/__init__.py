"""Thin Python binding of libwf.so, the GB300 Wiener-reconstruction library (include/wf.h).

Argument marshalling only: every step of the reconstruction runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (passed by data pointer), streams are torch
streams.  There is no fallback: if libwf.so is missing, importing the binding's entry points
raises.

Functions mirror the C ABI:
  Context.grid_assign   wf_grid_assign   supersampled CIC/TSC gridding (paper Sec. 3.1.2)
  Context.build_noise   wf_build_noise   window, nbar, data, noise (Sec. 3.1.3-3.2)
  Context.solve         wf_solve         Wiener filter by CG (Sec. 3.3.1, Eq. eq:WF)
  Context.solve_batch   wf_solve_batch
  Context.solve_response wf_solve_response  the Sec. 3.3.2 variant with Z and B inside R
  Context.jackknife_solve wf_jackknife_solve  mean of the Jackknife-like SD reconstructions
  Context.submit/poll   wf_submit / wf_poll (serving)
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwf.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "wf.h")

OK, PENDING = 0, 1
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_BREAKDOWN = -1, -2, -3, -4, -5
ERR_TIMEOUT, ERR_OVERFLOW, ERR_BUSY, ERR_UNSUPPORTED = -6, -7, -8, -9
CIC, TSC = 1, 2
FP64, MIXED = 0, 1

c_int, c_double, c_int64, c_uint64, c_void_p = (ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                                ctypes.c_uint64, ctypes.c_void_p)
dp = ctypes.POINTER(ctypes.c_double)


class Grid(ctypes.Structure):
    _fields_ = [("n", c_int), ("box", c_double), ("supersample", c_int)]


class SelectionC(ctypes.Structure):
    _fields_ = [("observer", c_double * 3), ("axis", c_double * 3), ("half_angle", c_double),
                ("n_holes", c_int), ("holes", dp), ("radial_kind", c_int),
                ("radial_params", c_double * 4)]


class Power(ctypes.Structure):
    _fields_ = [("k", dp), ("p", dp), ("n", c_int)]


class CompareResult(ctypes.Structure):
    _fields_ = [("r", c_double), ("d_euc", c_double), ("d_kl", c_double), ("kl_excluded", c_int64)]


class DensityMoments(ctypes.Structure):
    _fields_ = [("n_cells", c_double), ("mean", c_double), ("mu2", c_double), ("mu3", c_double),
                ("mu4", c_double), ("skewness", c_double), ("kurtosis", c_double), ("pearson", c_double)]


class Response(ctypes.Structure):
    _fields_ = [("bias", c_double), ("beta", c_double), ("sigma_v", c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int), ("prec", c_int), ("inner_tol", c_double),
                ("precond", c_int), ("deflate", c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", c_int), ("outer_iters", c_int), ("rel_residual", c_double),
                ("nbar", c_double), ("status", c_int), ("latency_s", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def build() -> str:
    from . import _build
    return _build.build()


def lib():
    """The loaded libwf.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libwf.so not built (run __graft_entry__.build()): " + LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.wf_create.argtypes = [P(c_void_p), c_int, ctypes.c_size_t]
        L.wf_destroy.argtypes = [c_void_p]
        L.wf_supported_size.argtypes = [c_int]
        L.wf_deflate_radius.argtypes = [c_int, c_int]
        L.wf_deflate_radius.restype = c_int
        L.wf_status_string.argtypes = [c_int]
        L.wf_status_string.restype = ctypes.c_char_p
        L.wf_last_error.restype = ctypes.c_char_p
        L.wf_grid_assign.argtypes = [c_void_p, P(Grid), c_int, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]
        L.wf_build_noise.argtypes = [c_void_p, P(Grid), P(SelectionC), c_void_p, c_int64, c_void_p, c_void_p,
                                     c_void_p, P(c_double), c_void_p]
        L.wf_solve.argtypes = [c_void_p, P(Grid), P(Power), c_void_p, c_double, c_void_p, P(SolveOpts), c_void_p,
                               P(SolveInfo), c_void_p]
        L.wf_solve_response.argtypes = [c_void_p, P(Grid), P(Power), P(Response), c_void_p, c_double, c_void_p,
                                        P(SolveOpts), c_void_p, P(SolveInfo), c_void_p]
        L.wf_jackknife_solve.argtypes = [c_void_p, P(Grid), c_int, P(Power), c_void_p, c_int64, c_void_p, c_void_p,
                                         c_int, c_double, c_void_p, c_void_p, c_double, P(SolveOpts), c_void_p,
                                         c_void_p, c_void_p]
        L.wf_solve_batch.argtypes = [c_void_p, c_int, P(Grid), P(Power), P(c_void_p), P(c_double), P(c_void_p),
                                     P(SolveOpts), P(c_void_p), P(SolveInfo), c_void_p]
        L.wf_submit.argtypes = [c_void_p, P(Grid), P(Power), c_void_p, c_double, c_void_p, P(SolveOpts), P(c_uint64)]
        L.wf_poll.argtypes = [c_void_p, c_uint64, c_int, c_void_p, P(SolveInfo)]
        L.wf_profile.argtypes = [c_void_p, c_int]
        L.wf_set_fused_planes.argtypes = [c_void_p, c_int]
        L.wf_autotune.argtypes = [c_void_p, c_int, c_int, ctypes.c_char_p, c_int]
        L.wf_tune_get.argtypes = [c_void_p, ctypes.c_char_p, c_int]
        L.wf_tune_set.argtypes = [c_void_p, ctypes.c_char_p]
        L.wf_fp64_rate.argtypes = [c_void_p, P(c_double)]
        L.wf_smooth.argtypes = [c_void_p, P(Grid), c_void_p, c_double, c_void_p, c_void_p]
        L.wf_project_mask.argtypes = [c_void_p, P(Grid), c_void_p, c_int, c_int, c_double, c_double, c_double,
                                      c_double, P(c_double), c_double, c_int, P(c_double), c_void_p, c_void_p,
                                      c_void_p]
        L.wf_sd_noise.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p,
                                  c_void_p]
        L.wf_jackknife_masses.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_double, c_void_p, c_void_p]
        L.wf_rsd_factor.argtypes = [c_int64, P(c_double), c_double, c_double, P(c_double)]
        L.wf_deconvolve.argtypes = [c_void_p, P(Grid), c_void_p, c_double, c_double, c_double, c_void_p, c_void_p]
        L.wf_selection_eval.argtypes = [c_void_p, P(SelectionC), c_void_p, c_int64, c_int, c_void_p, c_void_p]
        L.wf_grid_assign_weighted.argtypes = [c_void_p, P(Grid), c_int, c_void_p, c_void_p, c_int64, c_void_p,
                                              c_void_p, c_void_p]
        L.wf_compare.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, P(CompareResult), c_void_p]
        L.wf_density_stats.argtypes = [c_void_p, P(Grid), c_void_p, c_void_p, P(c_double), c_int, P(c_double),
                                       c_double, c_double, c_int, P(c_int64), P(DensityMoments), c_void_p]
        L.wf_profile_read.argtypes = [c_void_p, P(c_int64), P(c_int)]
        L.wf_profile_class.argtypes = [c_void_p, c_int, ctypes.c_char_p, c_int, P(c_int64), P(c_double),
                                       P(c_double)]
        for name in ("wf_create", "wf_destroy", "wf_grid_assign", "wf_build_noise", "wf_solve", "wf_solve_batch",
                     "wf_submit", "wf_poll", "wf_profile", "wf_profile_read", "wf_profile_class",
                     "wf_set_fused_planes", "wf_smooth", "wf_compare", "wf_density_stats",
                     "wf_selection_eval", "wf_grid_assign_weighted", "wf_rsd_factor", "wf_deconvolve",
                     "wf_sd_noise", "wf_jackknife_masses", "wf_project_mask", "wf_solve_response",
                     "wf_jackknife_solve", "wf_autotune", "wf_tune_get", "wf_tune_set", "wf_fp64_rate"):
            getattr(L, name).restype = c_int
        L.wf_supported_size.restype = c_int
        _lib = L
    return _lib


def rsd_factor(k, beta: float, sigma_v: float) -> np.ndarray:
    """<K D>_mu at wavenumbers k (wf_rsd_factor; host arrays, no GPU)."""
    k = np.ascontiguousarray(np.atleast_1d(np.asarray(k, dtype=np.float64)))
    out = np.empty_like(k)
    st = lib().wf_rsd_factor(k.size, k.ctypes.data_as(ctypes.POINTER(c_double)), float(beta), float(sigma_v),
                             out.ctypes.data_as(ctypes.POINTER(c_double)))
    if st != OK:
        raise WfError(st, "wf_rsd_factor")
    return out


class WfError(RuntimeError):
    def __init__(self, status: int, what: str, info=None):
        msg = "%s: %s" % (what, lib().wf_status_string(status).decode())
        le = lib().wf_last_error().decode()
        if le:
            msg += " (" + le + ")"
        super().__init__(msg)
        self.status = status
        self.info = info


def status_string(s: int) -> str:
    return lib().wf_status_string(s).decode()


def supported_size(n: int) -> bool:
    return bool(lib().wf_supported_size(n))


def deflate_radius(n: int, prec=None) -> int:
    """The coarse radius deflate = -1 takes for a solve of grid size n (wf_deflate_radius)."""
    return int(lib().wf_deflate_radius(int(n), int(MIXED if prec is None else prec)))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dvec(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(dp)


def make_selection(sel):
    """ctypes wf_selection from an object with observer, axis, half_angle, holes, radial_kind,
    radial_params; returns (struct, keepalive)."""
    holes = np.ascontiguousarray(np.asarray(sel.holes, dtype=np.float64).reshape(-1, 4))
    s = SelectionC()
    s.observer[:] = [float(v) for v in sel.observer]
    s.axis[:] = [float(v) for v in sel.axis]
    s.half_angle = float(sel.half_angle)
    s.n_holes = holes.shape[0]
    s.holes = holes.ctypes.data_as(dp) if holes.size else ctypes.cast(None, dp)
    s.radial_kind = int(sel.radial_kind)
    rp = list(sel.radial_params) + [0.0] * 4
    s.radial_params[:] = [float(v) for v in rp[:4]]
    return s, holes


def make_power(pk_k, pk_p):
    k, kp = _dvec(pk_k)
    p, pp = _dvec(pk_p)
    pw = Power(kp, pp, k.size)
    return pw, (k, p)


def make_opts(tol=1e-6, max_iter=5000, prec=FP64, inner_tol=0.0, precond=1, deflate=0):
    return SolveOpts(float(tol), int(max_iter), int(prec), float(inner_tol), int(precond), int(deflate))


class Context:
    """A wf_ctx on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self._h = c_void_p()
        st = lib().wf_create(ctypes.byref(self._h), device, hbm_budget)
        if st != OK:
            raise WfError(st, "wf_create")
        self.device = device

    def close(self):
        if self._h:
            lib().wf_destroy(self._h)
            self._h = c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- Sec. 3.1.2 -----------------------------------------------------------------------
    def grid_assign(self, pos, n: int, box: float, scheme: int = TSC, supersample: int = 2, fine_out=None,
                    n_obs=None, stream=None, check=True):
        """n_obs [n,n,n] float64 (torch, on the device) from positions pos [N_gal,3] float64."""
        import torch
        dev = torch.device("cuda", self.device)
        if n_obs is None:
            n_obs = torch.empty((n, n, n), dtype=torch.float64, device=dev)
        g = Grid(n, float(box), supersample)
        ngal = 0 if pos is None else int(pos.shape[0])
        st = lib().wf_grid_assign(self._h, ctypes.byref(g), scheme, _ptr(pos) if ngal else None, ngal,
                                  _ptr(fine_out), _ptr(n_obs), _stream(stream))
        if check and st != OK:
            raise WfError(st, "wf_grid_assign")
        return n_obs if check else (st, n_obs)

    # ---- Sec. 3.1.3-3.2 -------------------------------------------------------------------
    def build_noise(self, sel, n_obs, n_gal: int, box: float, stream=None, want_d=True, check=True):
        """(w, d, b, nbar): window, data and R^T N^-1 d on the device; nbar on the host."""
        import torch
        n = int(n_obs.shape[0])
        w = torch.empty_like(n_obs)
        d = torch.empty_like(n_obs) if want_d else None
        b = torch.empty_like(n_obs)
        s, keep = make_selection(sel)
        nb = c_double(0.0)
        g = Grid(n, float(box), 1)
        st = lib().wf_build_noise(self._h, ctypes.byref(g), ctypes.byref(s), _ptr(n_obs), int(n_gal), _ptr(w),
                                  _ptr(d), _ptr(b), ctypes.byref(nb), _stream(stream))
        if check and st != OK:
            raise WfError(st, "wf_build_noise")
        return (w, d, b, nb.value) if check else (st, w, d, b, nb.value)

    # ---- Sec. 3.1.3: the 3D mask from a sky map ---------------------------------------------
    def project_mask(self, sky, n: int, box: float, alpha0: float, dalpha: float, delta0: float, ddelta: float,
                     observer, dr: float, wr, want_counts=False, stream=None):
        """The 3D mask [n, n, n] from the sky map sky [n_delta, n_alpha] (device FP64) and the radial
        table wr (host) along rays (wf_project_mask); with want_counts also the samples per cell."""
        import torch
        if sky.dim() != 2 or sky.dtype != torch.float64 or not sky.is_contiguous() or not sky.is_cuda:
            raise ValueError("sky must be a contiguous [n_delta, n_alpha] float64 CUDA tensor")
        w = torch.empty((n, n, n), dtype=torch.float64, device=sky.device)
        cnt = torch.empty((n, n, n), dtype=torch.int64, device=sky.device) if want_counts else None
        wr = np.ascontiguousarray(np.asarray(wr, dtype=np.float64).ravel())
        obs = (c_double * 3)(*[float(v) for v in observer])
        g = Grid(int(n), float(box), 1)
        st = lib().wf_project_mask(self._h, ctypes.byref(g), _ptr(sky), int(sky.shape[1]), int(sky.shape[0]),
                                   float(alpha0), float(dalpha), float(delta0), float(ddelta), obs, float(dr),
                                   wr.size, wr.ctypes.data_as(ctypes.POINTER(c_double)), _ptr(w), _ptr(cnt),
                                   _stream(stream))
        if st != OK:
            raise WfError(st, "wf_project_mask")
        return (w, cnt) if want_counts else w

    # ---- signal-dependent noise -----------------------------------------------------------
    def sd_noise(self, n_obs, w, nbar: float, lam=None, stream=None):
        """(D, b): nbar^2 w / lambda and nbar^2 d / lambda (lambda None: the flat-prior mean
        (n_obs + 1) / w); solve with solve(D, 1.0, b, ...) (wf_sd_noise)."""
        import torch
        D, b = torch.empty_like(n_obs), torch.empty_like(n_obs)
        st = lib().wf_sd_noise(self._h, int(n_obs.numel()), _ptr(n_obs), _ptr(w), _ptr(lam), float(nbar), _ptr(D),
                               _ptr(b), _stream(stream))
        if st != OK:
            raise WfError(st, "wf_sd_noise")
        return D, b

    def jackknife_masses(self, w_gal, u, alpha: float, stream=None):
        """Galaxy masses of a Jackknife-like subsample: 1 / alpha where u < alpha / w, else 0
        (wf_jackknife_masses)."""
        import torch
        out = torch.empty_like(w_gal)
        st = lib().wf_jackknife_masses(self._h, int(w_gal.numel()), _ptr(w_gal), _ptr(u), float(alpha), _ptr(out),
                                       _stream(stream))
        if st != OK:
            raise WfError(st, "wf_jackknife_masses")
        return out

    # ---- Sec. 4: the inverse-weighting estimator -----------------------------------------
    def selection_eval(self, sel, pos, reciprocal=False, stream=None):
        """w (or 1 / w, 0 where w = 0) at positions pos [m, 3] (device FP64) with the window's
        formula (wf_selection_eval)."""
        import torch
        m = int(pos.shape[0])
        w = torch.empty(m, dtype=torch.float64, device=pos.device)
        s, keep = make_selection(sel)
        st = lib().wf_selection_eval(self._h, ctypes.byref(s), _ptr(pos), m, 1 if reciprocal else 0, _ptr(w),
                                     _stream(stream))
        if st != OK:
            raise WfError(st, "wf_selection_eval")
        return w

    def grid_assign_weighted(self, pos, wgt, n: int, box: float, scheme: int = TSC, supersample: int = 2,
                             fine_out=None, n_obs=None, stream=None, check=True):
        """Low-passed counts of galaxies with masses wgt (e.g. 1 / w for inverse weighting),
        [n, n, n] FP64 on the device (wf_grid_assign_weighted)."""
        import torch
        if n_obs is None:
            n_obs = torch.empty((n, n, n), dtype=torch.float64, device=pos.device)
        g = Grid(n, float(box), supersample)
        ngal = int(pos.shape[0])
        st = lib().wf_grid_assign_weighted(self._h, ctypes.byref(g), scheme, _ptr(pos) if ngal else None,
                                           _ptr(wgt) if ngal else None, ngal, _ptr(fine_out), _ptr(n_obs),
                                           _stream(stream))
        if check and st != OK:
            raise WfError(st, "wf_grid_assign_weighted")
        return n_obs if check else (st, n_obs)

    # ---- Sec. 3.3.1 ---------------------------------------------------------------------
    def solve(self, w, nbar: float, b, box: float, pk_k, pk_p, tol=1e-6, max_iter=5000, prec=FP64,
              inner_tol=0.0, precond=1, s_out=None, stream=None, check=True, deflate=0):
        """(s, info): Wiener mean s solving (S^-1 + nbar diag(w)) s = b.  deflate = K > 0 (WF_MIXED):
        inner solves preconditioned on the coarse Fourier modes |k| <= K."""
        import torch
        n = int(b.shape[0])
        if s_out is None:
            s_out = torch.empty_like(b)
        g = Grid(n, float(box), 1)
        pw, keep = make_power(pk_k, pk_p)
        o = make_opts(tol, max_iter, prec, inner_tol, precond, deflate)
        info = SolveInfo()
        st = lib().wf_solve(self._h, ctypes.byref(g), ctypes.byref(pw), _ptr(w), float(nbar), _ptr(b),
                            ctypes.byref(o), _ptr(s_out), ctypes.byref(info), _stream(stream))
        if check and st != OK:
            raise WfError(st, "wf_solve", info)
        return s_out, info

    def solve_response(self, w, nbar: float, b, box: float, pk_k, pk_p, bias: float, beta: float, sigma_v: float,
                       tol=1e-6, max_iter=5000, prec=FP64, inner_tol=0.0, precond=1, s_out=None, stream=None,
                       check=True, deflate=0):
        """(s_m, info): the real-space matter field solving (S^-1 + G nbar diag(w) G) s_m = G b with
        G the Fourier factor bias sqrt(<K D>_mu) (wf_solve_response)."""
        import torch
        n = int(b.shape[0])
        if s_out is None:
            s_out = torch.empty_like(b)
        g = Grid(n, float(box), 1)
        pw, keep = make_power(pk_k, pk_p)
        rs = Response(float(bias), float(beta), float(sigma_v))
        o = make_opts(tol, max_iter, prec, inner_tol, precond, deflate)
        info = SolveInfo()
        st = lib().wf_solve_response(self._h, ctypes.byref(g), ctypes.byref(pw), ctypes.byref(rs), _ptr(w),
                                     float(nbar), _ptr(b), ctypes.byref(o), _ptr(s_out), ctypes.byref(info),
                                     _stream(stream))
        if check and st != OK:
            raise WfError(st, "wf_solve_response", info)
        return s_out, info

    def jackknife_solve(self, pos, w_gal, u, alpha: float, n_obs, w, nbar: float, n: int, box: float, pk_k, pk_p,
                        scheme=TSC, supersample=2, tol=1e-6, max_iter=5000, prec=FP64, inner_tol=0.0, precond=1,
                        stream=None, check=True, deflate=0):
        """(s_mean, [info]): the mean of the signal-dependent-noise reconstructions of the n_sub
        Jackknife-like subsamples drawn with u [n_sub, n_gal] (wf_jackknife_solve)."""
        import torch
        n_sub, n_gal = int(u.shape[0]), int(u.shape[1])
        if not (u.is_contiguous() and pos.is_contiguous() and w_gal.is_contiguous()):
            raise ValueError("pos, w_gal and u must be contiguous")
        s_mean = torch.empty((n, n, n), dtype=torch.float64, device=n_obs.device)
        g = Grid(int(n), float(box), int(supersample))
        pw, keep = make_power(pk_k, pk_p)
        o = make_opts(tol, max_iter, prec, inner_tol, precond, deflate)
        infos = (SolveInfo * n_sub)()
        st = lib().wf_jackknife_solve(self._h, ctypes.byref(g), int(scheme), ctypes.byref(pw), _ptr(pos), n_gal,
                                      _ptr(w_gal), _ptr(u), n_sub, float(alpha), _ptr(n_obs), _ptr(w), float(nbar),
                                      ctypes.byref(o), _ptr(s_mean), ctypes.cast(infos, c_void_p), _stream(stream))
        if check and st != OK:
            raise WfError(st, "wf_jackknife_solve")
        return s_mean, list(infos)

    def solve_batch(self, problems, stream=None):
        """problems: list of dicts with w, nbar, b, box, pk_k, pk_p, tol, max_iter, prec, inner_tol,
        precond, deflate (and optional s_out).  Returns (status, [s], [info])."""
        import torch
        cnt = len(problems)
        grids = (Grid * cnt)()
        pows = (Power * cnt)()
        opts = (SolveOpts * cnt)()
        infos = (SolveInfo * cnt)()
        wp = (c_void_p * cnt)()
        bp = (c_void_p * cnt)()
        sp = (c_void_p * cnt)()
        nb = (c_double * cnt)()
        keep, outs = [], []
        for i, pr in enumerate(problems):
            n = int(pr["b"].shape[0])
            grids[i] = Grid(n, float(pr["box"]), 1)
            pw, kk = make_power(pr["pk_k"], pr["pk_p"])
            keep.append(kk)
            pows[i] = pw
            opts[i] = make_opts(pr.get("tol", 1e-6), pr.get("max_iter", 5000), pr.get("prec", FP64),
                                pr.get("inner_tol", 0.0), pr.get("precond", 1), pr.get("deflate", 0))
            s = pr.get("s_out")
            if s is None:
                s = torch.empty_like(pr["b"])
            outs.append(s)
            wp[i], bp[i], sp[i] = _ptr(pr["w"]), _ptr(pr["b"]), _ptr(s)
            nb[i] = float(pr["nbar"])
        st = lib().wf_solve_batch(self._h, cnt, grids, pows, wp, nb, bp, opts, sp, infos, _stream(stream))
        return st, outs, list(infos)

    # ---- tracing ------------------------------------------------------------------------
    # ---- Sec. 4.1 and 5.5: evaluation of a reconstruction ---------------------------------
    def smooth(self, field, box: float, r_s: float, out=None, stream=None):
        """Field convolved with the normalised Gaussian of radius r_s (box units) on the periodic
        grid (wf_smooth); FP64 [n,n,n] device tensors, out may be field."""
        import torch
        if out is None:
            out = torch.empty_like(field)
        g = Grid(int(field.shape[0]), float(box), 1)
        st = lib().wf_smooth(self._h, ctypes.byref(g), _ptr(field), float(r_s), _ptr(out), _stream(stream))
        if st != OK:
            raise WfError(st, "wf_smooth")
        return out

    def deconvolve(self, field, box: float, beta: float, sigma_v: float, bias: float, out=None, stream=None):
        """Matter field in real space from a galaxy field in redshift space, B^-1 Z^-1 (wf_deconvolve)."""
        import torch
        if out is None:
            out = torch.empty_like(field)
        g = Grid(int(field.shape[0]), float(box), 1)
        st = lib().wf_deconvolve(self._h, ctypes.byref(g), _ptr(field), float(beta), float(sigma_v), float(bias),
                                 _ptr(out), _stream(stream))
        if st != OK:
            raise WfError(st, "wf_deconvolve")
        return out

    def compare(self, rec, truth, stream=None) -> dict:
        """{"r", "d_euc", "d_kl", "kl_excluded"} of rec against truth (wf_compare)."""
        res = CompareResult()
        st = lib().wf_compare(self._h, int(rec.numel()), _ptr(rec), _ptr(truth), ctypes.byref(res), _stream(stream))
        if st != OK:
            raise WfError(st, "wf_compare")
        return {f: getattr(res, f) for f, _ in res._fields_}

    def density_stats(self, delta, w, box: float, observer, shells, lo: float, width: float, n_bins: int,
                      stream=None):
        """(hist [S, 2, n_bins + 2] int64 with the below/above-range counts last, moments [S, 2, 8]
        in DensityMoments order) of 1 + delta per shell and region (wf_density_stats)."""
        shells = np.ascontiguousarray(np.asarray(shells, dtype=np.float64).reshape(-1, 2))
        S = shells.shape[0]
        obs = (c_double * 3)(*[float(v) for v in observer])
        hist = np.zeros((S, 2, n_bins + 2), dtype=np.int64)
        mom = (DensityMoments * (2 * S))()
        g = Grid(int(delta.shape[0]), float(box), 1)
        st = lib().wf_density_stats(self._h, ctypes.byref(g), _ptr(delta), _ptr(w), obs, S,
                                    shells.ctypes.data_as(ctypes.POINTER(c_double)), float(lo), float(width),
                                    int(n_bins), hist.ctypes.data_as(ctypes.POINTER(c_int64)), mom, _stream(stream))
        if st != OK:
            raise WfError(st, "wf_density_stats")
        m = np.array([[getattr(x, f) for f, _ in DensityMoments._fields_] for x in mom]).reshape(S, 2, 8)
        return hist, m

    def set_fused_planes(self, on: bool = True):
        """FP32 y / z / y transforms as one cluster kernel per x-plane (True) or as three
        separate passes (False, the default), for solves started afterwards
        (wf_set_fused_planes)."""
        st = lib().wf_set_fused_planes(self._h, 1 if on else 0)
        if st != OK:
            raise WfError(st, "wf_set_fused_planes")

    def autotune(self, n: int, prec=MIXED, report_len: int = 1 << 16):
        """Time the launch variants of the spectral passes for grid size n and precision prec and
        keep the fastest per pass for later solves (wf_autotune); returns the report (a list of
        per-pass dicts: variants with ms per launch, the one chosen)."""
        import json
        buf = ctypes.create_string_buffer(report_len)
        st = lib().wf_autotune(self._h, int(n), int(prec), buf, report_len)
        if st != OK:
            raise WfError(st, "wf_autotune")
        return json.loads(buf.value.decode())

    def fp64_rate(self) -> float:
        """Measured FP64 FMA throughput of the device in flop/s (wf_fp64_rate)."""
        v = ctypes.c_double(0.0)
        st = lib().wf_fp64_rate(self._h, ctypes.byref(v))
        if st != OK:
            raise WfError(st, "wf_fp64_rate")
        return v.value

    def tune_get(self) -> dict:
        """The context's tuning table {"pass/prec/n": variant} (wf_tune_get)."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        st = lib().wf_tune_get(self._h, buf, 1 << 16)
        if st != OK:
            raise WfError(st, "wf_tune_get")
        return json.loads(buf.value.decode())

    def tune_set(self, table: dict):
        """Merge a saved tuning table into the context's (wf_tune_set)."""
        import json
        st = lib().wf_tune_set(self._h, json.dumps(table).encode())
        if st != OK:
            raise WfError(st, "wf_tune_set")

    def profile(self, enable: bool = True):
        """Reset launch counters; enable/disable per-kernel CUDA-event timing (wf_profile)."""
        st = lib().wf_profile(self._h, 1 if enable else 0)
        if st != OK:
            raise WfError(st, "wf_profile")

    def profile_read(self):
        """{"launches": total kernel launches, "classes": [{name, launches, ms, bytes, gbs}]}."""
        nl, nc = c_int64(), c_int()
        st = lib().wf_profile_read(self._h, ctypes.byref(nl), ctypes.byref(nc))
        if st != OK:
            raise WfError(st, "wf_profile_read")
        out = []
        for i in range(nc.value):
            buf = ctypes.create_string_buffer(64)
            la, ms, by = c_int64(), c_double(), c_double()
            lib().wf_profile_class(self._h, i, buf, 64, ctypes.byref(la), ctypes.byref(ms), ctypes.byref(by))
            out.append({"name": buf.value.decode(), "launches": la.value, "ms": ms.value, "bytes": by.value,
                        "gbs": (by.value / (ms.value / 1e3) / 1e9) if ms.value > 0 else None})
        return {"launches": nl.value, "classes": out}

    # ---- serving ------------------------------------------------------------------------
    def submit(self, w_host, nbar, b_host, box, pk_k, pk_p, tol=1e-6, max_iter=5000, prec=FP64, inner_tol=0.0,
               precond=1, deflate=0) -> int:
        """Queue a solve from HOST float64 arrays; returns the request id."""
        w_host = np.ascontiguousarray(w_host, dtype=np.float64)
        b_host = np.ascontiguousarray(b_host, dtype=np.float64)
        n = int(b_host.shape[0])
        g = Grid(n, float(box), 1)
        pw, keep = make_power(pk_k, pk_p)
        o = make_opts(tol, max_iter, prec, inner_tol, precond, deflate)
        rid = c_uint64(0)
        st = lib().wf_submit(self._h, ctypes.byref(g), ctypes.byref(pw), w_host.ctypes.data, float(nbar),
                             b_host.ctypes.data, ctypes.byref(o), ctypes.byref(rid))
        if st != OK:
            raise WfError(st, "wf_submit")
        return rid.value

    def poll(self, request_id: int, timeout_ms: int = 0, s_out=None):
        """(status, info); s_out: host float64 array of n^3 to receive the solution (or None)."""
        info = SolveInfo()
        ptr = None
        if s_out is not None:
            assert s_out.dtype == np.float64 and s_out.flags["C_CONTIGUOUS"]
            ptr = s_out.ctypes.data
        st = lib().wf_poll(self._h, c_uint64(request_id), int(timeout_ms), ptr, ctypes.byref(info))
        return st, info
