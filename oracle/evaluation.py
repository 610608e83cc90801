"""CPU FP64 oracle of the steps around the solve (Kitaura et al. 2009, arXiv:0906.3978): the
redshift-distortion factor, the deconvolution B^-1 Z^-1 (Eq. eq:DEC) and the Wiener filter with
Z and B inside the response operator, all of Sec. 3.3, the mean of the Jackknife-like signal-dependent-noise
reconstructions (Sec. 3.4), and the evaluation of a reconstruction of Sec. 4.1 "Statistical correlation
measures" and Sec. 5.5 "Statistics of the density field": Gaussian smoothing, the correlation coefficient
r, the Euclidean distance D_Euc, the normalised Kullback-Leibler distance D_KL, and binned density statistics (counts in 1+delta bins
per radial shell and observed / unobserved region; mean, central moments, skewness, kurtosis,
Pearson's skewness).

Test infrastructure only (tests, ``__graft_entry__.smoke()``, the benchmark's CPU leg); the
library never imports it.  Each function is the plain definition, in FP64, with the oracle's own
FFT (``oracle.fft3d``) as the only library step.  Readings where the paper is silent or garbled:

  * eq:GAUSS prints exp(+|r|^2 / 2 r_S^2); the kernel is read as the normalised Gaussian
    exp(-|r|^2 / 2 r_S^2) / ((2 pi)^(3/2) r_S^3), applied on the periodic grid as the multiplier
    exp(-|k|^2 r_S^2 / 2) of the DFT (k = 2 pi m / L, m the signed index in (-N/2, N/2]).
  * D_KL takes log(x) only where both 1 + delta are > 0; other cells are left out of the sum
    (the 1 / N_cells normalisation keeps all cells) and counted.
  * The density bins are [lo + i width, lo + (i + 1) width) in 1 + delta, bin index
    floor(((1 + delta) - lo) / width) in FP64; values below bin 0 or above the last bin are
    counted apart and do not enter the moments.  Moments use the bin centres (the paper's
    "density at the center of the bins"); Pearson's mode is the first bin of largest count.
  * A node lies in shell [r_lo, r_hi) when r_lo <= r < r_hi, r = |i H - o| (nodes at i H, no
    periodic wrap, as for the window); observed means w > 0.
"""
from __future__ import annotations

import numpy as np

from . import assign_weighted, cg, fft3d, lowpass_scaled


def gaussian_multiplier(n: int, box: float, r_s: float) -> np.ndarray:
    """exp(-|k|^2 r_S^2 / 2) on the full [n, n, n] DFT grid (Sec. 4.1, eq:GAUSS as read above)."""
    m = np.fft.fftfreq(n, 1.0 / n)
    m[n // 2] = n // 2  # the Nyquist index as +N/2 (its square is the same)
    k2 = (2.0 * np.pi / box) ** 2 * (m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    return np.exp(-0.5 * k2 * r_s * r_s)


def smooth(field, box: float, r_s: float) -> np.ndarray:
    """Field convolved with the normalised Gaussian of radius r_s on the periodic grid."""
    f = np.asarray(field, dtype=np.float64)
    n = f.shape[0]
    spec = fft3d(f.astype(np.complex128), -1)
    out = fft3d(spec * gaussian_multiplier(n, box, r_s), +1)
    return np.real(out) / float(n) ** 3


def compare(rec, true) -> dict:
    """Sec. 4.1: r = sum(t r) / sqrt(sum t^2 sum r^2); D_Euc = sqrt(mean (r - t)^2);
    D_KL = (1 / N_cells) sum (1 + r) log((1 + r) / (1 + t)) over the cells where both 1 + delta > 0."""
    r = np.asarray(rec, dtype=np.float64).ravel()
    t = np.asarray(true, dtype=np.float64).ravel()
    nc = r.size
    corr = np.sum(t * r) / (np.sqrt(np.sum(t * t)) * np.sqrt(np.sum(r * r)))
    d_euc = np.sqrt(np.sum((r - t) ** 2) / nc)
    a, b = 1.0 + r, 1.0 + t
    ok = (a > 0.0) & (b > 0.0)
    d_kl = np.sum(a[ok] * np.log(a[ok] / b[ok])) / nc
    return {"r": float(corr), "d_euc": float(d_euc), "d_kl": float(d_kl), "kl_excluded": int(nc - np.count_nonzero(ok))}


def node_radius(n: int, box: float, observer) -> np.ndarray:
    """|i H - o| at every node, in the same operation order as the window: ((dx dx + dy dy) + dz dz)."""
    h = box / n
    i = np.arange(n, dtype=np.float64) * h
    dx = (i - float(observer[0]))[:, None, None]
    dy = (i - float(observer[1]))[None, :, None]
    dz = (i - float(observer[2]))[None, None, :]
    return np.sqrt((dx * dx + dy * dy) + dz * dz)


def density_hist(delta, w, box: float, observer, shells, lo: float, width: float, n_bins: int):
    """Counts of 1 + delta in n_bins bins of `width` from `lo`, per shell (rows of `shells`:
    r_lo, r_hi) and region (0: w > 0, 1: w = 0).  Returns (hist [S, 2, n_bins], under [S, 2],
    over [S, 2]) as int64."""
    d = np.asarray(delta, dtype=np.float64)
    n = d.shape[0]
    r = node_radius(n, box, observer).ravel()
    obs = (np.asarray(w, dtype=np.float64).ravel() > 0.0)
    b = np.floor(((1.0 + d.ravel()) - lo) / width)
    shells = np.asarray(shells, dtype=np.float64).reshape(-1, 2)
    S = shells.shape[0]
    hist = np.zeros((S, 2, n_bins), dtype=np.int64)
    under = np.zeros((S, 2), dtype=np.int64)
    over = np.zeros((S, 2), dtype=np.int64)
    for s, (r_lo, r_hi) in enumerate(shells):
        ins = (r >= r_lo) & (r < r_hi)
        for g, sel in enumerate((obs, ~obs)):
            bb = b[ins & sel]
            under[s, g] = np.count_nonzero(bb < 0)
            over[s, g] = np.count_nonzero(bb >= n_bins)
            inr = bb[(bb >= 0) & (bb < n_bins)].astype(np.int64)
            hist[s, g] = np.bincount(inr, minlength=n_bins)
    return hist, under, over


MOMENT_FIELDS = ("n_cells", "mean", "mu2", "mu3", "mu4", "skewness", "kurtosis", "pearson")


def density_moments(hist, lo: float, width: float) -> np.ndarray:
    """Sec. 5.5 from the bin counts f_i at the bin centres delta_i = lo + (i + 1/2) width - 1:
    N = sum f, mean, mu_n = sum f (delta - mean)^n / N, s = mu3 / sigma^3, k = mu4 / sigma^4 - 3,
    s_P = (mean - delta_mode) / sigma.  Returns [..., 8] in MOMENT_FIELDS order (NaN if N = 0)."""
    h = np.asarray(hist, dtype=np.int64)
    nb = h.shape[-1]
    c = lo + (np.arange(nb) + 0.5) * width - 1.0
    flat = h.reshape(-1, nb)
    out = np.full((flat.shape[0], 8), np.nan)
    for j, f in enumerate(flat):
        N = int(f.sum())
        out[j, 0] = N
        if N == 0:
            continue
        ff = f.astype(np.float64)
        mean = float(np.sum(ff * c)) / N
        dev = c - mean
        mu2, mu3, mu4 = (float(np.sum(ff * dev ** p)) / N for p in (2, 3, 4))
        sig = np.sqrt(mu2)
        mode = c[int(np.argmax(f))]
        out[j, 1:] = (mean, mu2, mu3, mu4, mu3 / sig ** 3, mu4 / sig ** 4 - 3.0, (mean - mode) / sig)
    return out.reshape(h.shape[:-1] + (8,))


# ---------------------------------------------------------------- redshift distortions (Sec. 3.3.2-3.3.3)
def rsd_factor(k, beta: float, sigma_v: float) -> np.ndarray:
    """<K D>_mu: the mean over mu in [0, 1] of the Kaiser factor (1 + beta mu^2)^2 times the
    Lorentzian damping 1 / (1 + k^2 sigma_v^2 mu^2 / 2) (Sec. 3.3.3, "Redshift distortion operator"),
    by adaptive quadrature of the definition.  The real-space power spectrum times this factor is
    the redshift-space one; its square root is the operator Z."""
    from scipy.integrate import quad
    out = []
    for kk in np.atleast_1d(np.asarray(k, dtype=np.float64)):
        a = 0.5 * (kk * sigma_v) ** 2
        val, _ = quad(lambda m: (1.0 + beta * m * m) ** 2 / (1.0 + a * m * m), 0.0, 1.0,
                      epsabs=1e-16, epsrel=2e-14, limit=400)
        out.append(val)
    return np.array(out)


def deconvolve(field, box: float, beta: float, sigma_v: float, bias: float) -> np.ndarray:
    """Eq. eq:DEC with a constant bias b: the galaxy field in redshift space mapped to the matter
    field in real space, B^-1 Z^-1, i.e. the DFT multiplied by 1 / (b sqrt(<K D>_mu(|k|)))."""
    f = np.asarray(field, dtype=np.float64)
    n = f.shape[0]
    m = np.fft.fftfreq(n, 1.0 / n)
    m[n // 2] = n // 2
    n2 = (m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2).astype(np.int64)
    u, inv = np.unique(n2, return_inverse=True)
    mult = 1.0 / (bias * np.sqrt(rsd_factor(2.0 * np.pi * np.sqrt(u) / box, beta, sigma_v)))
    spec = fft3d(f.astype(np.complex128), -1) * mult[inv].reshape(n2.shape)
    return np.real(fft3d(spec, +1)) / float(n) ** 3


def n2_grid(n: int) -> np.ndarray:
    """|m|^2 of the signed DFT index m in (-N/2, N/2] at every node of the [n, n, n] grid."""
    m = np.fft.fftfreq(n, 1.0 / n).astype(np.int64)
    m[n // 2] = n // 2
    return m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2


def response_table(n: int, box: float, bias: float, beta: float, sigma_v: float) -> np.ndarray:
    """g[n2] = b sqrt(<K D>_mu(|k|)), |k| = 2 pi sqrt(n2) / L: the Fourier factor of the response
    Z B of Sec. 3.2.1 and 3.3.3 (bias and mu-averaged redshift operator), by n2 up to 3 (n/2)^2."""
    n2 = np.arange(3 * (n // 2) ** 2 + 1)
    return bias * np.sqrt(rsd_factor(2.0 * np.pi * np.sqrt(n2) / box, beta, sigma_v))


def _fourier_apply(x, mult) -> np.ndarray:
    """F^-1 diag(mult) F x for a real field x (unnormalised forward DFT, 1/V on the inverse)."""
    return np.real(fft3d(fft3d(np.asarray(x, dtype=np.complex128), -1) * mult, +1)) / float(x.size)


def response_matvec(sinv_tab, g_tab, nbar: float, w, s) -> np.ndarray:
    """(S^-1 + G nbar diag(w) G) s with G = F^-1 diag(g) F: the Wiener operator of Sec. 3.3.1 with
    the response R = W Z B of Sec. 3.3.2 (Z and B inside R)."""
    n2 = n2_grid(s.shape[0])
    gs = _fourier_apply(s, g_tab[n2])
    return _fourier_apply(s, sinv_tab[n2]) + _fourier_apply(nbar * np.asarray(w) * gs, g_tab[n2])


def solve_response(sinv_tab, g_tab, nbar: float, w, b, tol: float = 1e-12, max_iter: int = 20000):
    """The matter field s_m of the literal system (S^-1 + G nbar diag(w) G) s_m = G b by textbook
    (Hestenes-Stiefel) CG from 0, stopped on the relative residual recomputed from s_m (the same
    rule as the oracle's plain CG).  Returns (s_m, iterations, relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    rhs = _fourier_apply(b, np.asarray(g_tab)[n2_grid(b.shape[0])])
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    bb = float(np.sum(rhs * rhs))
    if bb == 0.0:
        return x, 0, 0.0
    rr, it = bb, 0
    while True:
        if rr <= tol * tol * bb:
            r = rhs - response_matvec(sinv_tab, g_tab, nbar, w, x)
            rr = float(np.sum(r * r))
            if np.sqrt(rr / bb) <= tol:
                return x, it, float(np.sqrt(rr / bb))
            p = r.copy()
        if it >= max_iter:
            raise RuntimeError("solve_response: not converged")
        q = response_matvec(sinv_tab, g_tab, nbar, w, p)
        alpha = rr / float(np.sum(p * q))
        x += alpha * p
        r -= alpha * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1


# ---------------------------------------------------------------- signal-dependent noise (Sec. 3.4)
def lambda_mean(n_obs, w) -> np.ndarray:
    """Flat-prior mean estimator of the underlying counts, lambda_mean = (N^o + 1) / w, on w > 0
    (0 elsewhere) (Sec. "flat prior": the posterior mean of a Poisson intensity)."""
    n = np.asarray(n_obs, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros_like(n)
    ok = w > 0.0
    out[ok] = (n[ok] + 1.0) / w[ok]
    return out


def jackknife_masses(w_gal, u, alpha: float) -> np.ndarray:
    """Eq. eq:selfunc: a galaxy is kept with probability alpha / w(x_g) (u_g < alpha / w_g with
    u_g uniform in [0, 1), drawn by the caller) and then carries mass 1 / alpha, so that the
    gridded subsample is N'' = N' / alpha, an unbiased estimate of lambda."""
    w = np.asarray(w_gal, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    keep = (w > 0.0) & (u < alpha / np.where(w > 0.0, w, 1.0))
    return np.where(keep, 1.0 / alpha, 0.0)


def sd_noise(n_obs, w, lam, nbar: float):
    """Eq. eq:noisecov, N^SD = w lambda / nbar^2 (per cell): the solve's diagonal
    R^T N^-1 R = nbar^2 w / lambda and right-hand side R^T N^-1 d = nbar^2 d / lambda with
    d = n_obs / nbar - w.  Cells with w = 0 or lambda <= 0 carry no data term (0, 0).  The LSQ
    noise is the case lambda = nbar.  Returns (D, b)."""
    n = np.asarray(n_obs, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    d = n / nbar - w
    ok = (w > 0.0) & (lam > 0.0)
    nb2 = nbar * nbar
    D = np.where(ok, nb2 * w / np.where(ok, lam, 1.0), 0.0)
    b = np.where(ok, nb2 * d / np.where(ok, lam, 1.0), 0.0)
    return D, b


def jackknife_solve(pos, w_gal, u, alpha: float, n_obs, w, nbar: float, n: int, box: float, scheme: int,
                    ss: int, sinv_tab, tol: float = 1e-12):
    """The mean over the subsamples j of the signal-dependent-noise reconstructions with
    lambda = N''_j (Sec. "Statistically unbiased Jackknife-like scheme"; Sec. 4.2 shows the mean of 200
    such reconstructions): masses of Eq. eq:selfunc from u[j], their supersampled gridding and ideal
    low-pass N''_j, the noise of Eq. eq:noisecov, and textbook CG on (S^-1 + diag(D_j)) s_j = b_j.
    Returns (mean, [s_j])."""
    sols = []
    for uj in np.asarray(u, dtype=np.float64):
        fine = assign_weighted(pos, jackknife_masses(w_gal, uj, alpha), n, box, scheme, ss)
        lam = lowpass_scaled(fine, n, ss, 2.0 ** -32)
        D, b = sd_noise(n_obs, w, lam, nbar)
        sols.append(cg(sinv_tab, 1.0, D, b, tol=tol)[0])
    return np.mean(sols, axis=0), sols
