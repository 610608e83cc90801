"""Pins of the evaluation oracle (Sec. 4.1 and Sec. 5.5: Gaussian smoothing, correlation and
distance measures, binned density statistics) against closed forms and hand-worked cases."""
import math

import numpy as np
import pytest

from oracle import evaluation as ev


def test_smoothing_plane_wave_closed_form():
    """A plane wave is an eigenfunction: it is scaled by exp(-|k|^2 r_S^2 / 2)."""
    n, box, rs = 16, 40.0, 3.0
    x = np.arange(n) * box / n
    m = (1, 2, 3)
    f = np.cos(2 * np.pi * (m[0] * x[:, None, None] + m[1] * x[None, :, None] + m[2] * x[None, None, :]) / box)
    k2 = (2 * np.pi / box) ** 2 * sum(v * v for v in m)
    got = ev.smooth(f + 2.0, box, rs)
    assert np.max(np.abs(got - (2.0 + math.exp(-0.5 * k2 * rs * rs) * f))) <= 1e-13


def test_smoothing_impulse_is_the_normalised_gaussian():
    """The response to a unit impulse at the origin is the normalised Gaussian sampled at the
    nodes (r_S = 2.5 cells: the multiplier is negligible at the Nyquist frequency and the
    periodic images are negligible at the centre region)."""
    n, box = 32, 32.0
    rs = 2.5
    f = np.zeros((n, n, n))
    f[0, 0, 0] = 1.0
    got = ev.smooth(f, box, rs)
    i = np.fft.fftfreq(n, 1.0 / n)  # signed offsets (H = 1)
    r2 = i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2
    want = np.exp(-0.5 * r2 / rs ** 2) / ((2 * np.pi) ** 1.5 * rs ** 3)
    near = r2 <= 36
    assert np.max(np.abs(got[near] - want[near])) <= 1e-12 * want.max()
    assert abs(got.sum() - 1.0) <= 1e-12


def test_smoothing_keeps_the_mean_and_zero_radius_is_identity():
    rng = np.random.default_rng(3)
    f = rng.standard_normal((12, 12, 12))
    assert abs(ev.smooth(f, 50.0, 7.0).mean() - f.mean()) <= 1e-14
    assert np.max(np.abs(ev.smooth(f, 50.0, 0.0) - f)) <= 1e-13


def test_compare_identities():
    rng = np.random.default_rng(4)
    x = rng.uniform(-0.5, 2.0, (8, 8, 8))
    same = ev.compare(x, x)
    assert abs(same["r"] - 1.0) <= 1e-15 and same["d_euc"] == 0.0 and same["d_kl"] == 0.0
    assert abs(ev.compare(2.5 * x, x)["r"] - 1.0) <= 1e-15
    assert abs(ev.compare(-x, x)["r"] + 1.0) <= 1e-15
    assert abs(ev.compare(x + 0.25, x)["d_euc"] - 0.25) <= 1e-15


def test_compare_hand_worked():
    rec = np.array([0.0, 1.0, -2.0, 3.0])  # 1 + delta = 1, 2, -1, 4
    true = np.array([0.0, 0.0, 0.0, -1.0])  # 1 + delta = 1, 1, 1, 0
    got = ev.compare(rec, true)
    assert got["kl_excluded"] == 2
    assert abs(got["d_kl"] - (2.0 * math.log(2.0)) / 4.0) <= 1e-16
    assert abs(got["r"] - (-3.0) / (1.0 * math.sqrt(14.0))) <= 1e-15
    assert abs(got["d_euc"] - math.sqrt((0 + 1 + 4 + 16) / 4.0)) <= 1e-15


def test_histogram_bins_edges_and_overflow():
    """Exact edges (width 0.25) go to the upper bin; values outside are counted apart."""
    d = np.array([-0.75, -0.5, -0.26, 0.0, 0.24999, 1.9, 5.0, -3.0]).reshape(2, 2, 2)
    w = np.array([1, 1, 1, 1, 0, 0, 0, 0], float).reshape(2, 2, 2)
    # 1 + delta = 0.25, 0.5, 0.74, 1.0 | 1.24999, 2.9, 6.0, -2.0 ; bins of 0.25 from lo = 0
    hist, under, over = ev.density_hist(d, w, 2.0, (0.0, 0.0, 0.0), [[0.0, 1e9]], 0.0, 0.25, 8)
    assert hist[0, 0].tolist() == [0, 1, 2, 0, 1, 0, 0, 0]  # 0.25 | 0.5, 0.74 | 1.0
    assert hist[0, 1].tolist() == [0, 0, 0, 0, 1, 0, 0, 0]
    assert under[0].tolist() == [0, 1] and over[0].tolist() == [0, 2]


def test_histogram_shells():
    """Node (1, 0, 0) at distance H = 1 from the origin is in [1, 2), not in [0, 1)."""
    n, box = 4, 4.0
    d = np.zeros((n, n, n))
    w = np.ones((n, n, n))
    hist, _, _ = ev.density_hist(d, w, box, (0.0, 0.0, 0.0), [[0.0, 1.0], [1.0, 2.0]], 0.0, 0.5, 4)
    r = ev.node_radius(n, box, (0.0, 0.0, 0.0))
    assert hist[0, 0].sum() == np.count_nonzero(r < 1.0) == 1
    assert hist[1, 0].sum() == np.count_nonzero((r >= 1.0) & (r < 2.0))


def test_moments_discrete_uniform_closed_form():
    """Equal counts in m bins: s = 0, k = -6 (m^2 + 1) / (5 (m^2 - 1)), s_P from the first bin."""
    m, width, lo = 7, 0.03, 0.4
    mom = ev.density_moments(np.full((1, 1, m), 5, dtype=np.int64), lo, width)[0, 0]
    sigma = width * math.sqrt((m * m - 1) / 12.0)
    assert mom[0] == 5 * m
    assert abs(mom[1] - (lo + (m / 2.0) * width - 1.0)) <= 1e-14
    assert abs(mom[2] - sigma ** 2) <= 1e-15
    assert abs(mom[5]) <= 1e-10
    assert abs(mom[6] + 6.0 * (m * m + 1) / (5.0 * (m * m - 1))) <= 1e-12
    assert abs(mom[7] - ((m - 1) / 2.0) * width / sigma) <= 1e-12


def test_moments_two_point_skewness():
    """Counts p q in two bins one width apart: skewness (q - p) / sqrt(pq) with weights p, q."""
    p, q = 3, 1
    h = np.zeros((1, 1, 5), dtype=np.int64)
    h[0, 0, 1], h[0, 0, 2] = p, q
    mom = ev.density_moments(h, 0.0, 1.0)[0, 0]
    P, Q = p / (p + q), q / (p + q)
    assert abs(mom[5] - (P - Q) / math.sqrt(P * Q)) <= 1e-12
    assert abs(mom[6] - (1 - 6 * P * Q) / (P * Q)) <= 1e-12  # excess kurtosis of a two-point law


def test_moments_empty_region_is_nan():
    mom = ev.density_moments(np.zeros((1, 1, 4), dtype=np.int64), 0.0, 0.1)[0, 0]
    assert mom[0] == 0 and np.all(np.isnan(mom[1:]))


# ---------------------------------------------------------------- inverse weighting (Sec. 4)
import oracle  # noqa: E402
import synth  # noqa: E402


def test_weighted_assignment_power_of_two_weight_is_exact():
    """Weight 2^16 turns a Q48 contribution into the same integer in Q32 units: no rounding."""
    pr = synth.problem("c1", n_override=16, cache=False)
    for scheme in (1, 2):
        f = oracle.assign(pr.pos, 16, pr.box, scheme, 2)
        fw = oracle.assign_weighted(pr.pos, np.full(len(pr.pos), 65536.0), 16, pr.box, scheme, 2)
        assert np.array_equal(f, fw)
        assert np.array_equal(oracle.lowpass_scaled(fw, 16, 2, 2.0 ** -32), oracle.lowpass(f, 16, 2) * 65536.0)


def test_weighted_assignment_rounding_bound_and_mass():
    """Unit weights: each contribution is the Q48 weight rounded to Q32, so a cell is within
    half a unit per contribution of the unweighted cell / 2^16, and the mass within half a unit
    per node of N_gal 2^32."""
    rng = np.random.default_rng(6)
    pos = rng.uniform(0.0, 30.0, (500, 3))
    f = oracle.assign(pos, 8, 30.0, 2, 2).astype(np.float64) / 65536.0
    fw = oracle.assign_weighted(pos, np.ones(500), 8, 30.0, 2, 2).astype(np.float64)
    assert np.max(np.abs(fw - f)) <= 0.5 * 27 * 500
    assert abs(fw.sum() - 500 * 2.0 ** 32) <= 0.5 * 27 * 500


def test_weighted_assignment_hand_worked():
    """One CIC galaxy at fine coordinate (1.25, 0.5, 0) cells of weight 3: node weights
    (3/4, 1/4) x (1/2, 1/2) x (1, 0) of 2^48, times 3, in Q32 units."""
    box, n = 8.0, 4  # fine cell = 1
    fw = oracle.assign_weighted(np.array([[1.25, 0.5, 0.0]]), np.array([3.0]), n, box, 1, 2)
    want = {(1, 0, 0): 0.75 * 0.5, (2, 0, 0): 0.25 * 0.5, (1, 1, 0): 0.75 * 0.5, (2, 1, 0): 0.25 * 0.5}
    for idx, frac in want.items():
        assert fw[idx] == round(frac * 3.0 * 2.0 ** 32)
    assert np.count_nonzero(fw) == 4


def test_window_at_nodes_equals_window():
    """The selection at node positions i H is the window itself, value for value."""
    pr = synth.problem("c2", n_override=16, cache=False)
    n, h = 16, pr.box / 16
    i = np.arange(n) * h
    pts = np.stack(np.meshgrid(i, i, i, indexing="ij"), axis=-1).reshape(-1, 3)
    assert np.array_equal(oracle.window_at(pr.sel, pts), oracle.window(pr.sel, n, pr.box).ravel())


def test_inverse_weighting_uniform_selection():
    """With a uniform completeness c the inverse-weighted grid is the plain grid / c (up to the
    Q32 rounding of each contribution)."""
    rng = np.random.default_rng(9)
    pos = rng.uniform(0.0, 20.0, (300, 3))
    c = 0.37
    f = oracle.lowpass(oracle.assign(pos, 8, 20.0, 2, 2), 8, 2)
    fw = oracle.lowpass_scaled(oracle.assign_weighted(pos, np.full(300, 1.0 / c), 8, 20.0, 2, 2), 8, 2, 2.0 ** -32)
    assert np.max(np.abs(fw - f / c)) <= 1e-8


# ---------------------------------------------------------------- redshift distortions (Sec. 3.3.2-3.3.3)
@pytest.mark.parametrize("beta", [0.0, 0.42, 1.0])
def test_rsd_factor_limits(beta):
    """k = 0 or sigma_v = 0: the angle-averaged Kaiser factor 1 + 2 beta / 3 + beta^2 / 5;
    beta = 0: the averaged Lorentzian arctan(sqrt(a)) / sqrt(a), a = k^2 sigma_v^2 / 2."""
    kaiser = 1.0 + 2.0 * beta / 3.0 + beta * beta / 5.0
    assert abs(ev.rsd_factor(0.0, beta, 5.0)[0] - kaiser) <= 1e-14
    assert abs(ev.rsd_factor(0.3, beta, 0.0)[0] - kaiser) <= 1e-14
    k = np.array([0.05, 0.3, 2.0])
    a = 0.5 * (k * 5.0) ** 2
    lor = np.arctan(np.sqrt(a)) / np.sqrt(a)
    assert np.max(np.abs(ev.rsd_factor(k, 0.0, 5.0) - lor) / lor) <= 1e-13


def test_rsd_factor_decreases_with_k():
    f = ev.rsd_factor(np.linspace(0.0, 5.0, 40), 0.42, 5.0)
    assert np.all(np.diff(f) < 0.0)


def test_deconvolution_plane_wave_and_bias():
    n, box, beta, sv, b = 16, 64.0, 0.42, 5.0, 1.7
    x = np.arange(n) * box / n
    f = np.cos(2 * np.pi * (1 * x[:, None, None] + 2 * x[None, :, None] + 2 * x[None, None, :]) / box)
    k = 2 * np.pi * 3.0 / box  # |m| = 3
    want = f / (b * math.sqrt(ev.rsd_factor(k, beta, sv)[0]))
    assert np.max(np.abs(ev.deconvolve(f, box, beta, sv, b) - want)) <= 1e-13
    g = np.random.default_rng(2).standard_normal((8, 8, 8))
    assert np.max(np.abs(ev.deconvolve(g, 30.0, 0.0, 0.0, 2.0) - g / 2.0)) <= 1e-14


# ---------------------------------------------------------------- signal-dependent noise
def test_sd_noise_reduces_to_the_lsq_noise():
    """lambda = nbar everywhere: the diagonal is nbar w and the right-hand side nbar d, the LSQ
    Wiener filter's (Sec. 3.2, eq:noiseav)."""
    pr = synth.problem("c1", n_override=16, cache=False)
    nobs = oracle.lowpass(oracle.assign(pr.pos, 16, pr.box, pr.scheme, 2), 16, 2)
    w = oracle.window(pr.sel, 16, pr.box)
    d, b, nbar = oracle.build_noise(nobs, w, pr.n_gal)
    D, bsd = ev.sd_noise(nobs, w, np.full_like(w, nbar), nbar)
    assert np.max(np.abs(D - nbar * w)) <= 1e-14 * nbar
    assert np.max(np.abs(bsd - b)) <= 1e-12 * np.max(np.abs(b))


def test_sd_noise_hand_worked_and_unobserved_cells():
    n_obs = np.array([2.0, 0.0, 5.0, 1.0])
    w = np.array([0.5, 0.25, 0.0, 1.0])
    lam = ev.lambda_mean(n_obs, w)
    assert lam.tolist() == [6.0, 4.0, 0.0, 2.0]
    D, b = ev.sd_noise(n_obs, w, lam, 2.0)
    assert D.tolist() == [4 * 0.5 / 6.0, 4 * 0.25 / 4.0, 0.0, 4 * 1.0 / 2.0]
    assert b.tolist() == [4 * (1.0 - 0.5) / 6.0, 4 * (0.0 - 0.25) / 4.0, 0.0, 4 * (0.5 - 1.0) / 2.0]


def test_jackknife_masses_rule_and_unbiasedness():
    """Kept when u < alpha / w, mass 1 / alpha; over many draws the total mass averages
    sum_g 1 / w_g, the number of galaxies of the complete sample the observed one was selected
    from (Sec. "Jackknife-like scheme": <N''> = lambda, not the observed counts)."""
    w = np.array([0.5, 0.01, 0.0, 1.0])
    m = ev.jackknife_masses(w, np.array([0.0199, 0.5, 0.0, 0.0101]), 0.01)
    assert m.tolist() == [100.0, 100.0, 0.0, 0.0]
    rng = np.random.default_rng(12)
    wg = rng.uniform(0.2, 1.0, 2000)
    alpha = 0.1
    tot = np.array([ev.jackknife_masses(wg, rng.uniform(size=2000), alpha).sum() for _ in range(400)])
    p = alpha / wg
    sigma = math.sqrt(np.sum(p * (1 - p)) / alpha ** 2 / 400)
    assert abs(tot.mean() - np.sum(1.0 / wg)) <= 4 * sigma


# ---------------------------------------------------------------- sky-mask projection (Sec. 3.1.3)
def test_mask_single_ray():
    """One pixel on the +x axis, samples every 0.25 cells: 4 samples per crossed cell (2 in the
    first, which the ray enters half way), the mask is sky value x radial value."""
    w, c = oracle.project_mask(np.array([[0.75]]), 8, 8.0, -0.01, 0.02, -0.01, 0.02, (0.5, 2.5, 2.5), 0.25,
                               np.full(40, 0.5))
    assert c[:, 2, 2].tolist() == [2, 4, 4, 4, 4, 4, 4, 4] and c.sum() == 30
    assert np.all(w[:, 2, 2] == 0.375) and np.count_nonzero(w) == 8  # values exact in Q32


def test_mask_radial_average_and_linearity():
    """A radial ramp is averaged over each cell's samples; sky values scale the mask linearly."""
    n_r = 32
    wr = (np.arange(n_r) + 0.5) / n_r
    w, c = oracle.project_mask(np.array([[1.0]]), 8, 8.0, -0.01, 0.02, -0.01, 0.02, (0.0, 4.5, 4.5), 0.25, wr)
    r = (np.arange(n_r) + 0.5) * 0.25
    for cell in range(8):
        sel = (r >= cell) & (r < cell + 1)
        assert abs(w[cell, 4, 4] - wr[sel].mean()) <= 1e-9
    w2, _ = oracle.project_mask(np.array([[0.5]]), 8, 8.0, -0.01, 0.02, -0.01, 0.02, (0.0, 4.5, 4.5), 0.25, wr)
    assert np.max(np.abs(w2 - 0.5 * w)) <= 1e-12


def test_mask_uniform_sky_is_the_hit_indicator():
    """Sky and radial completeness 1 everywhere: w = 1 exactly in every reached cell, 0 elsewhere."""
    sky = np.ones((18, 36))
    w, c = oracle.project_mask(sky, 12, 24.0, 0.0, 2 * np.pi / 36, -np.pi / 2, np.pi / 18, (12.0, 12.0, 12.0), 0.5,
                               np.ones(30))
    assert np.array_equal(w > 0, c > 0) and np.all(w[c > 0] == 1.0)


# ------------------------------------------------------------------ Z and B inside R (Sec. 3.3.2)
def _response_case(n, seed, box=60.0):
    rng = np.random.default_rng(seed)
    k, p = synth.lcdm_table()
    sinv = oracle.sinv_table(n, box, k, p)
    w = np.clip(rng.uniform(-0.3, 1.0, (n, n, n)), 0.0, 1.0)   # about a quarter of the cells unobserved
    b = rng.standard_normal((n, n, n)) * w
    return box, sinv, w, b


def test_response_unit_factor_is_the_plain_filter():
    """g = 1 (bias 1, beta 0, no damping) leaves the plain system, solved by the C textbook CG."""
    n = 8
    box, sinv, w, b = _response_case(n, 5)
    g = ev.response_table(n, box, 1.0, 0.0, 0.0)
    assert np.allclose(g, 1.0, rtol=0, atol=1e-14)
    s, _, rel = ev.solve_response(sinv, g, 0.7, w, b, tol=1e-13)
    ref = oracle.cg(sinv, 0.7, w, b, tol=1e-13)[0]
    assert rel <= 1e-13
    assert np.linalg.norm(s - ref) <= 1e-11 * np.linalg.norm(ref)


def test_response_uniform_selection_closed_form():
    """w = 1: every Fourier mode decouples, s_m(k) = g(k) b(k) / (S^-1(k) + nbar g(k)^2)."""
    n, nbar = 8, 0.4
    box, sinv, _, _ = _response_case(n, 6)
    b = np.random.default_rng(7).standard_normal((n, n, n))
    g = ev.response_table(n, box, 1.3, 0.45, 5.0)
    n2 = ev.n2_grid(n)
    s, _, _ = ev.solve_response(sinv, g, nbar, np.ones((n, n, n)), b, tol=1e-14)
    ref = np.real(np.fft.ifftn(np.fft.fftn(b) * g[n2] / (sinv[n2] + nbar * g[n2] ** 2)))
    assert np.linalg.norm(s - ref) <= 1e-12 * np.linalg.norm(ref)


def test_response_matches_a_dense_cosine_sum_operator():
    """4^3 cells: S^-1 and G written as dense cosine sums over the modes (no FFT),
    A = S^-1 + G diag(nbar w) G and right-hand side G b solved directly."""
    n, nbar = 4, 0.9
    box, sinv, w, b = _response_case(n, 8, box=20.0)
    g = ev.response_table(n, box, 1.1, 0.6, 3.0)
    f = np.fft.fftfreq(n, 1.0 / n).astype(int)
    K = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1).reshape(-1, 3)
    x = np.arange(n)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    ph = 2 * np.pi * (X @ K.T) / n
    C, S = np.cos(ph), np.sin(ph)
    n2 = np.sum(K * K, axis=1)

    def dense(m):
        return ((C * m) @ C.T + (S * m) @ S.T) / n ** 3

    G = dense(g[n2])
    A = dense(sinv[n2]) + G @ np.diag(nbar * w.ravel()) @ G
    ref = np.linalg.solve(A, G @ b.ravel()).reshape(n, n, n)
    s, _, _ = ev.solve_response(sinv, g, nbar, w, b, tol=1e-14)
    assert np.linalg.norm(s - ref) <= 1e-11 * np.linalg.norm(ref)


def test_response_equals_redshift_prior_then_deconvolution():
    """s_g = G s_m turns the system into the plain one with prior g^2 P (S^-1 / g^2); deconvolving
    its solution by 1 / g (Eq. eq:DEC) gives the same s_m."""
    n, nbar, bias, beta, sv = 8, 0.6, 1.2, 0.5, 5.0
    box, sinv, w, b = _response_case(n, 9)
    g = ev.response_table(n, box, bias, beta, sv)
    s_m, _, _ = ev.solve_response(sinv, g, nbar, w, b, tol=1e-14)
    s_g = oracle.cg(sinv / g ** 2, nbar, w, b, tol=1e-14)[0]
    via = ev.deconvolve(s_g, box, beta, sv, bias)
    assert np.linalg.norm(via - s_m) <= 1e-11 * np.linalg.norm(s_m)


def _ray_positions(n, box, na, nd, nr, dr, obs, geo):
    """Sample positions x / H [pixels, samples, 3] written out with numpy."""
    H = box / n
    al = geo[0] + (np.arange(na) + 0.5) * geo[1]
    de = geo[2] + (np.arange(nd) + 0.5) * geo[3]
    u = np.stack([np.cos(de)[:, None] * np.cos(al)[None, :], np.cos(de)[:, None] * np.sin(al)[None, :],
                  np.broadcast_to(np.sin(de)[:, None], (nd, na))], -1).reshape(-1, 3)
    r = (np.arange(nr) + 0.5) * dr
    return (np.asarray(obs)[None, None, :] + r[None, :, None] * u[:, None, :]) / H


def test_mask_counts_are_the_exact_geometry():
    """Per-cell sample counts equal a numpy count of floor((o + r u) / H), except for samples within
    1e-9 cells of a face (numpy's cos/sin and libm's may differ in the last bit), which the oracle's
    own near-face report covers."""
    n, box, na, nd, nr = 12, 30.0, 40, 20, 90
    dr = 0.31 * box / n
    obs = (0.37 * box, 0.52 * box, 0.44 * box)
    geo = (0.0, 2 * np.pi / na, -np.pi / 2, np.pi / nd)
    _, c, near = oracle.project_mask(np.full((nd, na), 0.5), n, box, *geo, obs, dr, np.ones(nr), face_margin=1e-9)
    X = _ray_positions(n, box, na, nd, nr, dr, obs, geo)
    F = np.floor(X)
    inside = np.all((F >= 0) & (F < n), axis=-1)
    cells = (F[..., 0] * n + F[..., 1]) * n + F[..., 2]
    exact = np.bincount(cells[inside].astype(np.int64), minlength=n ** 3).reshape(n, n, n)
    assert exact.sum() > 10000  # most rays cross the box
    assert np.array_equal(c[near == 0], exact[near == 0])
    assert np.all(np.abs(c - exact) <= near)


def test_mask_near_face_report_by_brute_force():
    """The near-face report for a wide margin (0.05 cells): each sample within the margin of a
    face adds one to its own cell and to every cell across such faces (inside the box); numpy
    enumerates the same cells sample by sample."""
    n, box, na, nd, nr = 8, 20.0, 12, 6, 40
    dr = 0.37 * box / n
    obs = (0.41 * box, 0.47 * box, 0.53 * box)
    geo = (0.1, 2 * np.pi / na, -np.pi / 2, np.pi / nd)
    m = 0.05
    _, _, near = oracle.project_mask(np.full((nd, na), 1.0), n, box, *geo, obs, dr, np.ones(nr), face_margin=m)
    X = _ray_positions(n, box, na, nd, nr, dr, obs, geo).reshape(-1, 3)
    ref = np.zeros((n, n, n), dtype=np.int64)
    for x in X:
        f = np.floor(x)
        lo = f - ((x - f) < m)
        hi = f + ((f + 1 - x) < m)
        if np.array_equal(lo, f) and np.array_equal(hi, f):
            continue
        for a in range(int(lo[0]), int(hi[0]) + 1):
            for b in range(int(lo[1]), int(hi[1]) + 1):
                for c in range(int(lo[2]), int(hi[2]) + 1):
                    if 0 <= a < n and 0 <= b < n and 0 <= c < n:
                        ref[a, b, c] += 1
    assert ref.sum() > 100
    assert np.array_equal(near, ref)


# ------------------------------------------------------------------ Jackknife ensemble (Sec. 3.4)
def _jk_case(n=16):
    pr = synth.problem("c1", n_override=n, cache=False)
    nobs = oracle.lowpass(oracle.assign(pr.pos, n, pr.box, pr.scheme, 2), n, 2)
    w = oracle.window(pr.sel, n, pr.box)
    _, _, nbar = oracle.build_noise(nobs, w, pr.n_gal)
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    return pr, nobs, w, nbar, tab


def test_jackknife_ensemble_keeping_every_galaxy_is_the_sd_filter_on_the_counts():
    """alpha = 1 and u = 0 keep every galaxy with mass 1, so N'' is the unit-mass low-passed grid
    (up to the Q32 rounding of the masses' weights) and every reconstruction is the SD filter with
    lambda = n_obs."""
    pr, nobs, w, nbar, tab = _jk_case()
    n = pr.n
    mean, sols = ev.jackknife_solve(pr.pos, np.ones(pr.n_gal), np.zeros((2, pr.n_gal)), 1.0, nobs, w, nbar, n,
                                    pr.box, pr.scheme, 2, tab)
    D, b = ev.sd_noise(nobs, w, nobs, nbar)
    ref = oracle.cg(tab, 1.0, D, b, tol=1e-12)[0]
    # Q32 mass weights move N'' by ~1e-10 relative; the solves' residual is 1e-12
    assert np.linalg.norm(mean - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.array_equal(sols[0], sols[1])


def test_jackknife_ensemble_is_the_mean_of_the_subsample_solves():
    """Three subsamples: the ensemble is their plain average, and repeating one subsample's numbers
    three times gives that subsample's reconstruction."""
    pr, nobs, w, nbar, tab = _jk_case()
    n = pr.n
    wg = oracle.window_at(pr.sel, pr.pos)
    alpha = 0.9 * wg[wg > 0].min()
    u = np.random.default_rng(8).uniform(size=(3, pr.n_gal))
    mean, sols = ev.jackknife_solve(pr.pos, wg, u, alpha, nobs, w, nbar, n, pr.box, pr.scheme, 2, tab)
    assert np.allclose(mean, (sols[0] + sols[1] + sols[2]) / 3.0, rtol=0, atol=1e-14 * np.abs(mean).max())
    assert not np.array_equal(sols[0], sols[1])
    rep, _ = ev.jackknife_solve(pr.pos, wg, np.repeat(u[:1], 3, axis=0), alpha, nobs, w, nbar, n, pr.box,
                                pr.scheme, 2, tab)
    assert np.linalg.norm(rep - sols[0]) <= 1e-14 * np.linalg.norm(sols[0])
