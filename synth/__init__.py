"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle's tests.

This module makes inputs only: galaxy catalogues, power-spectrum tables and selection
descriptions.  It holds none of the reconstruction's arithmetic (no gridding, no
low-pass, no window at the nodes, no noise model, no solve); the thinning of the mock
galaxies by the survey selection is the simulated survey itself, done here at each
galaxy's continuous position with its own code.

Recipe (stand-in for the paper's SDSS DR6 and Millennium-mock workloads, Sec. 2 and 4,
which are not available):
  * Gaussian field G on the N^3 grid: unit white noise filtered in Fourier space by
    sqrt(P(k)/dV) (so <|G_k|^2> = V_c P(k)/dV), mean mode removed, optional spherical cut
    at k_Nyq;
  * log-normal density delta = exp(G - sigma_G^2/2) - 1;
  * Poisson counts per cell with mean nbar_true dV (1 + delta) (Eq. eq:pois), positions
    uniform inside the cell;
  * binomial thinning: each galaxy kept with probability w(x) (Eq. eq:bin), nbar_true set
    so that the expected observed number equals the target.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------------------
# Selection description (input to both sides; evaluated at nodes by each side separately)
# ---------------------------------------------------------------------------------------
@dataclass
class Selection:
    observer: tuple = (0.0, 0.0, 0.0)
    axis: tuple = (1.0, 0.0, 0.0)          # unit vector
    half_angle: float = math.pi            # cone half-opening (rad); pi = whole sky
    holes: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))  # [h,4]: unit dir, radius
    radial_kind: int = 0                   # 0 flat, 1 exp(-(r/p0)^2), 2 gamma law peak p0, slope p1
    radial_params: tuple = (0.0, 0.0, 0.0, 0.0)


def uniform_selection(n: int, box: float) -> Selection:
    """w = 1 at every node: observer half a cell outside the box corner, whole sky."""
    h = box / n
    return Selection(observer=(-0.5 * h, -0.5 * h, -0.5 * h), axis=(1.0, 0.0, 0.0),
                     half_angle=math.pi, radial_kind=0)


def _rot_frame(axis):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    t = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(a, t)
    u /= np.linalg.norm(u)
    v = np.cross(a, u)
    return a, u, v


def random_holes(axis, half_angle: float, radius: float, cover: float, rng) -> np.ndarray:
    """Caps of angular radius `radius` with centres uniform on the cone's cap, as many as cover
    the fraction `cover` of the cone solid angle (overlaps ignored)."""
    a, u, v = _rot_frame(axis)
    cone = TWO_PI * (1.0 - math.cos(half_angle))
    cap = TWO_PI * (1.0 - math.cos(radius))
    nh = int(round(cover * cone / cap))
    mu = 1.0 - rng.random(nh) * (1.0 - math.cos(half_angle))
    phi = TWO_PI * rng.random(nh)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    d = mu[:, None] * a + (s * np.cos(phi))[:, None] * u + (s * np.sin(phi))[:, None] * v
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([d, np.full((nh, 1), radius)], axis=1)


def survey_completeness(sel: Selection, pos: np.ndarray) -> np.ndarray:
    """Selection probability of galaxies at continuous positions (the simulated survey)."""
    d = pos - np.asarray(sel.observer)[None, :]
    r = np.sqrt(np.einsum("ij,ij->i", d, d))
    rs = np.where(r > 0, r, 1.0)
    cosang = (d @ np.asarray(sel.axis)) / rs
    ok = (cosang >= math.cos(sel.half_angle)) & (r > 0)
    for h in np.asarray(sel.holes).reshape(-1, 4):
        ok &= ~((d @ h[:3]) / rs > math.cos(h[3]))
    p = sel.radial_params
    if sel.radial_kind == 0:
        f = np.ones_like(r)
    elif sel.radial_kind == 1:
        f = np.exp(-(r / p[0]) ** 2)
    else:
        t = r / p[0]
        f = t ** p[1] * np.exp(p[1] * (1.0 - t))
    return np.where(ok, f, 0.0)


# ---------------------------------------------------------------------------------------
# Power spectra (tables handed to the solver as its prior)
# ---------------------------------------------------------------------------------------
def power_law_table(amp: float, slope: float, kmin: float, kmax: float, npts: int = 64):
    k = np.geomspace(kmin, kmax, npts)
    return k, amp * k ** slope


def eh_nowiggle_transfer(k, omega_m=0.24, omega_b=0.04, h=0.73, t_cmb=2.728):
    """Eisenstein & Hu (1998, ApJ 496, 605) zero-baryon-oscillation fit, Eqs. 26, 28-31;
    k in h/Mpc."""
    theta = t_cmb / 2.7
    om_h2 = omega_m * h * h
    ob_h2 = omega_b * h * h
    fb = omega_b / omega_m
    s = 44.5 * np.log(9.83 / om_h2) / np.sqrt(1.0 + 10.0 * ob_h2 ** 0.75)      # Mpc
    a_gam = 1.0 - 0.328 * np.log(431.0 * om_h2) * fb + 0.38 * np.log(22.3 * om_h2) * fb * fb
    k_mpc = k * h
    gam = omega_m * h * (a_gam + (1.0 - a_gam) / (1.0 + (0.43 * k_mpc * s) ** 4))
    q = k * theta * theta / gam
    L0 = np.log(2.0 * math.e + 1.8 * q)
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q * q)


def sigma_r(k, pk, R):
    """rms of the top-hat smoothed field, by the trapezoid rule in ln k."""
    x = k * R
    W = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    integrand = k ** 3 * pk * W * W / (2.0 * math.pi ** 2)
    lk = np.log(k)
    return math.sqrt(float(np.sum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(lk))))


def lcdm_table(sigma8=0.8, ns=1.0, kmin=1e-4, kmax=1e2, npts=256, **cosmo):
    """Smooth LCDM-shaped linear P(k) [ (Mpc/h)^3 ] normalised to sigma8 (R = 8 Mpc/h)."""
    kk = np.geomspace(1e-5, 1e3, 20000)
    raw = kk ** ns * eh_nowiggle_transfer(kk, **cosmo) ** 2
    amp = (sigma8 / sigma_r(kk, raw, 8.0)) ** 2
    k = np.geomspace(kmin, kmax, npts)
    return k, amp * k ** ns * eh_nowiggle_transfer(k, **cosmo) ** 2


# ---------------------------------------------------------------------------------------
# Fields and catalogues
# ---------------------------------------------------------------------------------------
def _kgrid2(n: int):
    f = np.fft.fftfreq(n, 1.0 / n)
    fz = np.fft.rfftfreq(n, 1.0 / n)
    return (f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2)


def gaussian_field(n: int, box: float, pk_k, pk_p, rng, cut_nyquist=False, amp=1.0):
    """Real Gaussian field with <|G_k|^2> = V_c amp P(k)/dV; returns float64 [n,n,n]."""
    try:
        import scipy.fft as sfft
        rfftn = lambda a: sfft.rfftn(a, workers=-1)
        irfftn = lambda a, s: sfft.irfftn(a, s=s, workers=-1)
    except ImportError:  # pragma: no cover
        rfftn = np.fft.rfftn
        irfftn = lambda a, s: np.fft.irfftn(a, s=s)
    dv = (box / n) ** 3
    noise = rng.standard_normal((n, n, n))
    spec = rfftn(noise)
    del noise
    n2 = _kgrid2(n)
    k = (TWO_PI / box) * np.sqrt(n2)
    ks = np.where(n2 > 0, k, 1.0)
    p = np.exp(np.interp(np.log(ks), np.log(pk_k), np.log(pk_p)))
    filt = np.sqrt(amp * p / dv)
    filt[0, 0, 0] = 0.0
    if cut_nyquist:
        filt[k > math.pi * n / box] = 0.0
    spec *= filt
    return irfftn(spec, (n, n, n))


def field_sigma2(n: int, box: float, pk_k, pk_p, cut_nyquist=False) -> float:
    """Expected per-cell variance of gaussian_field: (1/V_c) sum_k P(k)/dV (k != 0)."""
    dv = (box / n) ** 3
    f = np.fft.fftfreq(n, 1.0 / n)
    n2 = (f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    k = (TWO_PI / box) * np.sqrt(n2)
    m = n2 > 0
    if cut_nyquist:
        m &= k <= math.pi * n / box
    p = np.exp(np.interp(np.log(k[m]), np.log(pk_k), np.log(pk_p)))
    return float(np.sum(p / dv) / n ** 3)


def lognormal_catalogue(n: int, box: float, pk_k, pk_p, sel: Selection, n_target: float, seed: int,
                        cut_nyquist=False, amp=1.0):
    """Observed galaxy positions [N_gal, 3] float64 in [0, box)."""
    rng = np.random.default_rng(seed)
    g = gaussian_field(n, box, pk_k, pk_p, rng, cut_nyquist=cut_nyquist, amp=amp)
    var = float(np.var(g))
    dens = np.exp(g - 0.5 * var)           # 1 + delta
    del g
    h = box / n
    centres = (np.arange(n) + 0.5) * h
    # expected observed count with w at the cell centres fixes nbar_true
    wsum = 0.0
    for ix in range(n):
        cx = np.stack(np.meshgrid([centres[ix]], centres, centres, indexing="ij"), -1).reshape(-1, 3)
        wsum += float(np.sum(survey_completeness(sel, cx) * dens[ix].reshape(-1)))
    if wsum <= 0:
        return np.zeros((0, 3))
    lam_scale = n_target / wsum
    counts = rng.poisson(dens.reshape(-1) * lam_scale)
    del dens
    idx = np.repeat(np.arange(n ** 3, dtype=np.int64), counts)
    ix, rem = np.divmod(idx, n * n)
    iy, iz = np.divmod(rem, n)
    pos = (np.stack([ix, iy, iz], axis=1) + rng.random((idx.size, 3))) * h
    keep = rng.random(idx.size) < survey_completeness(sel, pos)
    return np.ascontiguousarray(pos[keep])


def uniform_catalogue(n_gal: int, box: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.random((n_gal, 3)) * box


# ---------------------------------------------------------------------------------------
# Workload configurations (grid sizes, boxes, galaxy numbers of the paper's setups)
# ---------------------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    n: int
    box: float
    scheme: int            # 1 CIC, 2 TSC
    ss: int
    tol: float
    pk_k: np.ndarray
    pk_p: np.ndarray
    sel: Selection
    pos: np.ndarray

    @property
    def n_gal(self) -> int:
        return int(self.pos.shape[0])


def selection_c1(box=200.0) -> Selection:
    a = np.ones(3) / math.sqrt(3.0)
    return Selection(observer=(0.0, 0.0, 0.0), axis=tuple(a), half_angle=math.radians(30.0),
                     radial_kind=1, radial_params=(120.0, 0.0, 0.0, 0.0))


def selection_sdss_like(box: float, seed: int, half_angle_deg=30.0, r_peak=None, gamma=2.0,
                        observer=None) -> Selection:
    """Cone along +x from (0, L/2, 0.04 L) (the mock observer (0, 250, 20) of a 500 Mpc/h box),
    radial gamma law peaking at 0.3 L (150 Mpc/h for L = 500), 2-degree holes covering 5%."""
    rng = np.random.default_rng(seed)
    if r_peak is None:
        r_peak = 0.3 * box
    axis = (1.0, 0.0, 0.0)
    holes = random_holes(axis, math.radians(half_angle_deg), math.radians(2.0), 0.05, rng)
    obs = observer if observer is not None else (0.0, 0.5 * box, 0.04 * box)
    return Selection(observer=tuple(obs), axis=axis, half_angle=math.radians(half_angle_deg),
                     holes=holes, radial_kind=2, radial_params=(r_peak, gamma, 0.0, 0.0))


def c1_power(n=64, box=200.0):
    """P = A k^-1.5 with A such that the k_Nyq-cut Gaussian field has sigma_G = 1 per cell."""
    k, p = power_law_table(1.0, -1.5, 1e-3, 1e2)
    s2 = field_sigma2(n, box, k, p, cut_nyquist=True)
    return k, p / s2


_CACHE = os.environ.get("WF_SYNTH_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                        "_cache"))


def _cached_catalogue(key: str, make):
    os.makedirs(_CACHE, exist_ok=True)
    path = os.path.join(_CACHE, key + ".npy")
    if os.path.exists(path):
        return np.load(path)
    pos = make()
    tmp = path + ".tmp%d.npy" % os.getpid()
    np.save(tmp, pos)
    os.replace(tmp, path)
    return pos


def problem(name: str, n_override: int | None = None, n_gal_override: float | None = None,
            cache: bool = True) -> Problem:
    """The named workload: 'c1' (64^3, 200 Mpc/h, CIC), 'c2' (256^3, 500 Mpc/h, TSC) or 'c3'
    (512^3, 500 Mpc/h, TSC).  n_override/n_gal_override give a reduced-size copy with the
    same recipe (box scaled to keep the cell size for c2/c3)."""
    if name == "c1":
        n, box, ng, scheme, tol, seed = 64, 200.0, 2e4, 1, 1e-8, 1001
        if n_override:
            n = n_override
        pk_k, pk_p = c1_power(n, box)
        sel = selection_c1(box)
        cut = True
        amp = 1.0
    elif name in ("c2", "c3"):
        n, box, ng, tol = (256, 500.0, 1.5e5, 1e-6) if name == "c2" else (512, 500.0, 5e5, 1e-6)
        seed = 1002 if name == "c2" else 1003
        scheme = 2
        if n_override:
            box = box * n_override / n
            ng = ng * (n_override / n) ** 3
            n = n_override
        pk_k, pk_p = lcdm_table()
        sel = selection_sdss_like(box, seed)
        cut = False
        amp = 1.0
    else:
        raise ValueError(name)
    if n_gal_override is not None:
        ng = n_gal_override
    key = "%s_n%d_g%d_s%d" % (name, n, int(ng), seed)
    make = lambda: lognormal_catalogue(n, box, pk_k, pk_p, sel, ng, seed, cut_nyquist=cut, amp=amp)
    pos = _cached_catalogue(key, make) if cache else make()
    return Problem(name, n, box, scheme, 2, tol, pk_k, pk_p, sel, pos)
