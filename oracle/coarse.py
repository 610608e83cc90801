"""CPU FP64 oracle of the coarse-space (two-level) preconditioned inner CG.

Test infrastructure only: the tests use it; the library under ``paper_0906_3978_gb300`` never
imports it.

The Wiener system of Sec. 3.3.1 (Eq. eq:WF), A s = b with A = S^-1 + diag(nbar w), is solved in
Fourier variables: with C = F^-1 diag(c) F, CG runs on (C A C) y = C b and s = C y, where c = S^(1/2)
away from k = 0 and c_0 = (nbar sum(w) / V_c)^(-1/2), so that in the spectrum of y

    A' y = m (.) y + c (.) F( nbar w (.) F^-1 (c (.) y) ),   m = c^2 S^-1 (1 away from k = 0, 0 at it).

The paper names a Krylov inversion only.  Its iterations are here preconditioned by the two-level
"A-DEF2" operator of Tang, Nabben, Vuik and Erlangga (2009, "Comparison of two-level
preconditioners derived from deflation, domain decomposition and multigrid methods", J. Sci.
Comput. 39, Sec. 2.3.3).  Z holds the unit vectors of the Fourier modes with |k|^2 <= K^2 (k in grid
units), E = Z^H A' Z their Galerkin block and Q = Z E^-1 Z^H:

    start   x_0 = Q b',  r_0 = b' - A' x_0              (b' = c (.) F b; counted as one iteration)
    precond z = r - Q (A' r - r)
    CG      alpha = <r, z> / <p, A' p>,  x += alpha p,  r -= alpha A' p,
            beta = <r_new, z_new> / <r, z>,  p = z_new + beta p   (p_0 = z_0)

This module writes those steps out in FP64 on full complex spectra (numpy's FFT) with E formed
entry by entry from the transform of nbar w at the differences of the coarse modes and solved by a
dense LU factorisation.  It shares nothing with the GPU path.  Pins: tests/test_oracle_pins.py
(test_adef2_*).
"""
from __future__ import annotations

import numpy as np


def _grid(table, nbar: float, w):
    n = w.shape[0]
    f = np.fft.fftfreq(n, 1.0 / n).astype(np.int64)
    n2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2
    sinv = np.asarray(table, dtype=np.float64)[n2]
    c = np.empty(n2.shape)
    m = np.ones(n2.shape)
    nz = n2 > 0
    c[nz] = 1.0 / np.sqrt(sinv[nz])
    c[~nz] = 1.0 / np.sqrt(nbar * w.sum() / w.size)
    m[~nz] = 0.0
    return f, n2, c, m


class Problem:
    """The split-preconditioned system of one (table, nbar, w, b) with the coarse space of radius K
    (K = None: no coarse space, so Q = 0 and the iteration is plain CG on A')."""

    def __init__(self, table, nbar: float, w, b, K):
        w = np.asarray(w, dtype=np.float64)
        self.n = w.shape[0]
        self.V = w.size
        self.f, self.n2, self.c, self.m = _grid(table, nbar, w)
        self.D = nbar * w
        self.rhs = self.c * np.fft.fftn(np.asarray(b, dtype=np.float64))
        if K is None:
            self.idx = None
            return
        sel = np.argwhere(self.n2 <= K * K)                 # coarse modes (index triples)
        self.idx = tuple(sel.T)
        dh = np.fft.fftn(self.D)                           # transform of nbar w
        d = (sel[:, None, :] - sel[None, :, :]) % self.n   # k_p - k_q, per axis
        cc = self.c[self.idx]
        # E(p, q) = m(p) delta_pq + c(p) c(q) Dh(k_p - k_q) / V: the coarse block of A'
        E = (cc[:, None] * cc[None, :]) * dh[d[..., 0], d[..., 1], d[..., 2]] / self.V
        E[np.diag_indices_from(E)] += self.m[self.idx]
        self.E = E

    def apply(self, y):
        """A' y."""
        return self.m * y + self.c * np.fft.fftn(self.D * np.fft.ifftn(self.c * y))

    def coarse(self, v):
        """Q v = Z E^-1 Z^H v."""
        out = np.zeros_like(v)
        if self.idx is not None:
            out[self.idx] = np.linalg.solve(self.E, v[self.idx])
        return out

    def precond(self, r):
        """z = r - Q (A' r - r)."""
        return r - self.coarse(self.apply(r) - r)

    def solution(self, y):
        """s = C y (real space)."""
        return np.real(np.fft.ifftn(self.c * y))


def _dot(u, v) -> float:
    return float(np.real(np.vdot(u, v)))


def adef2(table, nbar: float, w, b, K, tol: float = 1e-12, max_iter: int = 100000, return_state: bool = False):
    """(s, iters, rel) of the A-DEF2-preconditioned CG above, from y = 0, stopping when
    ||r|| <= tol ||b'|| (r the residual of the y system) or after max_iter iterations (the start step
    is the first).  return_state adds (problem, y, r)."""
    pb = Problem(table, nbar, w, b, K)
    r0n = np.sqrt(_dot(pb.rhs, pb.rhs))
    y = pb.coarse(pb.rhs)            # start step, alpha = 1
    r = pb.rhs - pb.apply(y)
    it = 1
    rel = np.sqrt(_dot(r, r)) / r0n if r0n > 0 else 0.0
    if rel > tol and it < max_iter:
        z = pb.precond(r)
        p = z.copy()
        rz = _dot(r, z)
        while it < max_iter:
            q = pb.apply(p)
            alpha = rz / _dot(p, q)
            y = y + alpha * p
            r = r - alpha * q
            it += 1
            rel = np.sqrt(_dot(r, r)) / r0n
            if rel <= tol:
                break
            z = pb.precond(r)
            rz_new = _dot(r, z)
            p = z + (rz_new / rz) * p
            rz = rz_new
    s = pb.solution(y)
    if return_state:
        return s, it, rel, (pb, y, r)
    return s, it, rel
