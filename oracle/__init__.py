"""CPU FP64 oracle of the Wiener-reconstruction hot path (ctypes wrapper over oracle.c).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg use it; the library under ``paper_0906_3978_gb300`` never imports it.

Each function follows the paper (Kitaura et al. 2009, arXiv:0906.3978):
  assign      Sec. 3.1.2 "Supersampling step", Eq. def:ngrid (fixed-point CIC/TSC)
  lowpass     Sec. 3.1.2, supersampling step 2 (ideal low-pass, sampling at target grid)
  window      Sec. 3.1.3 (3D mask w <= 1; analytic cone x holes x radial law)
  project_mask
              Sec. 3.1.3, projection of a sky completeness map and a radial completeness table
              along rays (Eq. eq:transf), NGP-assigned and averaged per cell
  window_at, assign_weighted
              Sec. 4, Eq. def:ngrid with galaxy mass 1/w (the inverse-weighting estimator)
  build_noise Sec. 3.2, Eqs. eq:datamodel, eq:nmean, eq:noiseav
  sinv_table  Sec. 3.3.1, Fourier-diagonal prior S
  matvec/cg   Sec. 3.3.1, Eq. eq:WF, by a Krylov (CG) inversion
  pcg         the same Krylov inversion with a Fourier-diagonal preconditioner
  coarse.adef2
              the same Krylov inversion with the two-level (coarse Fourier modes) preconditioner of
              the library's mixed solves, in numpy (oracle/coarse.py)

Parity is pinned by the ``-m "not gpu"`` tests (closed forms, dense direct solve, brute
force, invariants); see tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_ARG, ERR_OOM, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_OVERFLOW = 0, -1, -2, -4, -5, -7


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP64, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        ip = ctypes.POINTER(ctypes.c_int)
        i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        L.oracle_assign.argtypes = [i, d, i, i, dp, i64, u64p]
        L.oracle_lowpass.argtypes = [i, i, u64p, dp]
        L.oracle_lowpass_scaled.argtypes = [i, i, u64p, d, dp]
        L.oracle_assign_weighted.argtypes = [i, d, i, i, dp, dp, i64, u64p]
        L.oracle_window_at.argtypes = [i64, dp, dp, dp, d, i, dp, i, dp, dp]
        L.oracle_project_mask.argtypes = [i, d, dp, i, i, d, d, d, d, dp, d, i, dp, dp,
                                          ctypes.POINTER(ctypes.c_int64), d, ctypes.POINTER(ctypes.c_int64)]
        L.oracle_lowpass_point.argtypes = [i, i, u64p, i, i, i]
        L.oracle_lowpass_point.restype = d
        L.oracle_window.argtypes = [i, d, dp, dp, d, i, dp, i, dp, dp]
        L.oracle_build_noise.argtypes = [i, dp, dp, i64, dp, dp, dp]
        L.oracle_sinv_table.argtypes = [i, d, dp, dp, i, dp]
        L.oracle_fft1d.argtypes = [ctypes.c_void_p, i, i]
        L.oracle_fft3d.argtypes = [ctypes.c_void_p, i, i]
        L.oracle_matvec.argtypes = [i, dp, d, dp, dp, dp]
        L.oracle_cg.argtypes = [i, dp, d, dp, dp, d, i, dp, ip, dp]
        L.oracle_pcg.argtypes = [i, dp, dp, d, dp, dp, d, i, dp, ip, dp]
        L.oracle_threads.restype = i
        L.oracle_set_threads.restype = None
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s failed with status %d" % (what, status))
        self.status = status


def _check(st, what):
    if st != OK:
        raise OracleError(st, what)


def threads() -> int:
    return int(lib().oracle_threads())


def set_threads(n: int) -> None:
    """OpenMP threads for the following oracle calls."""
    lib().oracle_set_threads(int(n))


def assign(pos, n: int, box: float, scheme: int, ss: int = 2) -> np.ndarray:
    """Fine Q48 grid [(ss*n)^3] uint64 (scheme 1 = CIC, 2 = TSC); Sec. 3.1.2."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    nf = ss * n
    fine = np.empty(nf ** 3, dtype=np.uint64)
    _check(lib().oracle_assign(n, box, ss, scheme, _dp(pos), pos.shape[0], _u64p(fine)), "assign")
    return fine.reshape(nf, nf, nf)


def lowpass(fine, n: int, ss: int = 2) -> np.ndarray:
    """n_obs [n^3] FP64 from the fine grid: ideal low-pass then sampling; Sec. 3.1.2 step 2."""
    fine = np.ascontiguousarray(fine, dtype=np.uint64)
    out = np.empty(n ** 3, dtype=np.float64)
    _check(lib().oracle_lowpass(n, ss, _u64p(fine), _dp(out)), "lowpass")
    return out.reshape(n, n, n)


def lowpass_point(fine, n: int, ss: int, j) -> float:
    """One output node of the low-pass by the direct sum over the fine grid."""
    fine = np.ascontiguousarray(fine, dtype=np.uint64)
    return float(lib().oracle_lowpass_point(n, ss, _u64p(fine), int(j[0]), int(j[1]), int(j[2])))


def lowpass_scaled(fine, n: int, ss: int, unit: float) -> np.ndarray:
    """The low-pass of a fine grid holding fine * unit galaxies per cell (2^-32 for
    ``assign_weighted``)."""
    fine = np.ascontiguousarray(fine, dtype=np.uint64)
    out = np.empty(n ** 3, dtype=np.float64)
    _check(lib().oracle_lowpass_scaled(n, ss, _u64p(fine), float(unit), _dp(out)), "lowpass_scaled")
    return out.reshape(n, n, n)


def assign_weighted(pos, wgt, n: int, box: float, scheme: int, ss: int = 2) -> np.ndarray:
    """Fine grid [(ss n)^3] uint64 in Q32 units of weighted galaxies: each node contribution is
    rint(Q48 weight * wgt * 2^-16) (Sec. 4, Eq. def:ngrid with galaxy mass wgt)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    wgt = np.ascontiguousarray(wgt, dtype=np.float64).ravel()
    nf = ss * n
    fine = np.empty(nf ** 3, dtype=np.uint64)
    _check(lib().oracle_assign_weighted(n, box, ss, scheme, _dp(pos), _dp(wgt), pos.shape[0], _u64p(fine)),
           "assign_weighted")
    return fine.reshape(nf, nf, nf)


def window_at(sel, pts) -> np.ndarray:
    """The selection w at arbitrary positions pts [m, 3] (Sec. 3.1.3, the completeness at a galaxy)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    obs = np.ascontiguousarray(sel.observer, dtype=np.float64)
    ax = np.ascontiguousarray(sel.axis, dtype=np.float64)
    holes = np.ascontiguousarray(np.asarray(sel.holes, dtype=np.float64).reshape(-1, 4))
    rp = np.ascontiguousarray(np.resize(np.asarray(sel.radial_params, dtype=np.float64), 4))
    w = np.empty(pts.shape[0], dtype=np.float64)
    _check(lib().oracle_window_at(pts.shape[0], _dp(pts), _dp(obs), _dp(ax), float(sel.half_angle),
                                  holes.shape[0], _dp(holes), int(sel.radial_kind), _dp(rp), _dp(w)),
           "window_at")
    return w


def project_mask(sky, n: int, box: float, alpha0: float, dalpha: float, delta0: float, ddelta: float,
                 observer, dr: float, wr, face_margin: float = 0.0):
    """(w [n, n, n], counts [n, n, n]): the 3D mask from the sky map sky [n_delta, n_alpha] and the
    radial completeness wr [n_r] at r_k = (k + 1/2) dr, projected along rays (Sec. 3.1.3), each
    sample's cell decided in exact FP64 geometry.  With face_margin > 0 a third array is returned:
    per cell, the samples within face_margin cells of a face of this cell or a neighbour's (the
    samples that a position error below face_margin could move, and the cells they could move
    between)."""
    sky = np.ascontiguousarray(sky, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64).ravel()
    obs = np.ascontiguousarray(observer, dtype=np.float64)
    w = np.empty(n ** 3, dtype=np.float64)
    cnt = np.empty(n ** 3, dtype=np.int64)
    near = np.empty(n ** 3, dtype=np.int64) if face_margin > 0 else None
    i64p = ctypes.POINTER(ctypes.c_int64)
    _check(lib().oracle_project_mask(n, box, _dp(sky), sky.shape[1], sky.shape[0], alpha0, dalpha, delta0, ddelta,
                                     _dp(obs), dr, wr.size, _dp(wr), _dp(w), cnt.ctypes.data_as(i64p),
                                     float(face_margin), near.ctypes.data_as(i64p) if near is not None else None),
           "project_mask")
    if near is not None:
        return w.reshape(n, n, n), cnt.reshape(n, n, n), near.reshape(n, n, n)
    return w.reshape(n, n, n), cnt.reshape(n, n, n)


def window(sel, n: int, box: float) -> np.ndarray:
    """w [n^3] at the nodes; Sec. 3.1.3.  ``sel`` has observer, axis, half_angle, holes [h,4],
    radial_kind and radial_params (e.g. ``synth.Selection``)."""
    obs = np.ascontiguousarray(sel.observer, dtype=np.float64)
    ax = np.ascontiguousarray(sel.axis, dtype=np.float64)
    holes = np.ascontiguousarray(np.asarray(sel.holes, dtype=np.float64).reshape(-1, 4))
    rp = np.ascontiguousarray(np.resize(np.asarray(sel.radial_params, dtype=np.float64), 4))
    w = np.empty(n ** 3, dtype=np.float64)
    _check(lib().oracle_window(n, box, _dp(obs), _dp(ax), float(sel.half_angle), holes.shape[0],
                               _dp(holes), int(sel.radial_kind), _dp(rp), _dp(w)), "window")
    return w.reshape(n, n, n)


def build_noise(n_obs, w, n_gal: int):
    """(d, b, nbar): Sec. 3.2, eq:datamodel, eq:nmean, eq:noiseav."""
    n = n_obs.shape[0]
    n_obs = np.ascontiguousarray(n_obs, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    d = np.empty_like(n_obs)
    b = np.empty_like(n_obs)
    nbar = ctypes.c_double(0.0)
    _check(lib().oracle_build_noise(n, _dp(n_obs), _dp(w), int(n_gal), _dp(d), _dp(b),
                                    ctypes.byref(nbar)), "build_noise")
    return d, b, nbar.value


def sinv_table(n: int, box: float, pk_k, pk_p) -> np.ndarray:
    """S^-1 as a function of the integer n2 = |k|^2 (2 pi/L)^-2, length 3(n/2)^2+1."""
    pk_k = np.ascontiguousarray(pk_k, dtype=np.float64)
    pk_p = np.ascontiguousarray(pk_p, dtype=np.float64)
    t = np.empty(3 * (n // 2) ** 2 + 1, dtype=np.float64)
    _check(lib().oracle_sinv_table(n, box, _dp(pk_k), _dp(pk_p), pk_k.size, _dp(t)), "sinv_table")
    return t


def fft1d(a, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128).copy()
    _check(lib().oracle_fft1d(a.ctypes.data, a.size, sign), "fft1d")
    return a


def fft3d(a, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128).copy()
    _check(lib().oracle_fft3d(a.ctypes.data, a.shape[0], sign), "fft3d")
    return a


def matvec(table, nbar: float, w, p) -> np.ndarray:
    n = p.shape[0]
    w = np.ascontiguousarray(w, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = np.empty_like(p)
    _check(lib().oracle_matvec(n, _dp(np.ascontiguousarray(table)), nbar, _dp(w), _dp(p), _dp(q)),
           "matvec")
    return q


def cg(table, nbar: float, w, b, tol: float = 1e-12, max_iter: int = 100000, allow_unconverged=False):
    """(x, iters, rel_residual); raises OracleError unless converged (or, with
    allow_unconverged, unless the failure is the iteration cap)."""
    n = b.shape[0]
    w = np.ascontiguousarray(w, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib().oracle_cg(n, _dp(np.ascontiguousarray(table)), nbar, _dp(w), _dp(b), tol, max_iter,
                         _dp(x), ctypes.byref(it), ctypes.byref(rel))
    if not (allow_unconverged and st == ERR_NOT_CONVERGED):
        _check(st, "cg")
    return x, it.value, rel.value


def pcg(table, ptable, nbar: float, w, b, tol: float = 1e-12, max_iter: int = 100000, allow_unconverged=False):
    """(x, iters, rel_residual) of preconditioned CG with M^-1 = F^-1 diag(ptable[|k|^2]) F;
    ptable = 1 everywhere is textbook CG.  Raises like ``cg``."""
    n = b.shape[0]
    w = np.ascontiguousarray(w, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    ptable = np.ascontiguousarray(ptable, dtype=np.float64)
    x = np.empty_like(b)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib().oracle_pcg(n, _dp(np.ascontiguousarray(table)), _dp(ptable), nbar, _dp(w), _dp(b), tol, max_iter,
                          _dp(x), ctypes.byref(it), ctypes.byref(rel))
    if not (allow_unconverged and st == ERR_NOT_CONVERGED):
        _check(st, "pcg")
    return x, it.value, rel.value
