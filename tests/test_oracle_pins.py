"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle by a route that does not reuse its code: hand-worked values,
textbook kernels, numpy's FFT, brute-force sums and dense linear algebra, closed forms.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q48 = 2.0 ** 48


# ----------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 18, 24, 27, 32, 36, 48, 54, 64, 72, 96])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_matches_naive_dft(n, sign):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    M = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    ref = M @ a
    got = oracle.fft1d(a, sign)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [128, 192, 256, 384, 512, 1024])
def test_fft1d_matches_numpy(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(oracle.fft1d(a, -1), np.fft.fft(a), rtol=0, atol=1e-11 * np.sqrt(n))
    assert np.allclose(oracle.fft1d(a, +1), np.fft.ifft(a) * n, rtol=0, atol=1e-11 * np.sqrt(n))


@pytest.mark.parametrize("n", [4, 6, 8, 12, 16])
def test_fft3d_matches_numpy(n):
    rng = np.random.default_rng(100 + n)
    a = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    assert np.allclose(oracle.fft3d(a, -1), np.fft.fftn(a), atol=1e-10)
    assert np.allclose(oracle.fft3d(a, +1), np.fft.ifftn(a) * n ** 3, atol=1e-10)


# ----------------------------------------------------------------------------- assignment
def _golden_axis_cases():
    rows = []
    with open(os.path.join(GOLDEN, "assign_axis_cases.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                rows.append((line[0], float(line[1]), [int(v) for v in line[2:]]))
    return rows


@pytest.mark.parametrize("case", _golden_axis_cases())
def test_assign_axis_weights_golden(case):
    scheme_name, x, nw = case
    scheme = 1 if scheme_name == "CIC" else 2
    # NF = 8 fine cells over L = 8; put the galaxy at (x, 1.5, 2.5) and marginalise y, z
    fine = oracle.assign(np.array([[x, 1.5, 2.5]]), 4, 8.0, scheme, 2).astype(object)
    marg = [sum(int(v) for v in fine[i].ravel()) for i in range(8)]
    expect = [0] * 8
    for node, wgt in zip(nw[0::2], nw[1::2]):
        expect[node] += wgt * 2 ** 32
    assert marg == expect


@pytest.mark.parametrize("scheme", [1, 2])
def test_assign_mass_conservation_exact(scheme):
    rng = np.random.default_rng(7)
    pos = rng.uniform(-30.0, 230.0, size=(3000, 3))      # includes wrapped positions
    fine = oracle.assign(pos, 16, 200.0, scheme, 2)
    assert int(fine.astype(object).sum()) == 3000 * 2 ** 48


@pytest.mark.parametrize("scheme", [1, 2])
def test_assign_matches_continuous_kernel(scheme):
    """Fixed-point weights equal the textbook CIC/TSC kernels to the Q16 quantisation."""
    rng = np.random.default_rng(11)
    nf, L = 16, 16.0
    for _ in range(40):
        p = rng.uniform(0, L, 3)
        fine = oracle.assign(p[None, :], nf // 2, L, scheme, 2).astype(np.float64) / Q48
        ref = np.zeros((nf, nf, nf))
        ws = []
        for a in range(3):
            u = p[a]
            if scheme == 1:
                i = int(math.floor(u))
                f = u - i
                ws.append([(i % nf, 1 - f), ((i + 1) % nf, f)])
            else:
                j = int(math.floor(u + 0.5))
                d = u - j
                ws.append([((j - 1) % nf, 0.5 * (0.5 - d) ** 2), (j % nf, 0.75 - d * d),
                           ((j + 1) % nf, 0.5 * (0.5 + d) ** 2)])
        for ix, wx in ws[0]:
            for iy, wy in ws[1]:
                for iz, wz in ws[2]:
                    ref[ix, iy, iz] += wx * wy * wz
        assert np.max(np.abs(fine - ref)) < 4 * 2.0 ** -16


def test_assign_overflow_detected():
    pos = np.tile([[1.0, 1.0, 1.0]], (65536, 1))        # exactly on a fine node, CIC
    with pytest.raises(oracle.OracleError) as e:
        oracle.assign(pos, 4, 8.0, 1, 2)
    assert e.value.status == oracle.ERR_OVERFLOW
    fine = oracle.assign(pos[:65535], 4, 8.0, 1, 2)
    assert int(fine[1, 1, 1]) == 65535 * 2 ** 48


def test_assign_rejects_non_finite():
    with pytest.raises(oracle.OracleError) as e:
        oracle.assign(np.array([[1.0, np.nan, 2.0]]), 4, 8.0, 2, 2)
    assert e.value.status == oracle.ERR_ARG


# ----------------------------------------------------------------------------- low-pass


def test_lowpass_matches_numpy_definition():
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 100.0, size=(500, 3))
    fine = oracle.assign(pos, 12, 100.0, 2, 2)
    got = oracle.lowpass(fine, 12, 2)
    # numpy's ifftn divides by n^3, which is the 1/V_c of the definition
    F = np.fft.fftn(fine.astype(np.float64) / Q48)
    k = np.fft.fftfreq(12, 1.0 / 12).astype(int)
    keep = np.abs(k) < 6
    sel = np.mod(k, 24)
    C = F[np.ix_(sel, sel, sel)] * (keep[:, None, None] & keep[None, :, None] & keep[None, None, :])
    ref = np.real(np.fft.ifftn(C))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(got.sum() - 500.0) <= 1e-10


def test_lowpass_direct_sum_points():
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, 50.0, size=(200, 3))
    fine = oracle.assign(pos, 8, 50.0, 1, 2)
    full = oracle.lowpass(fine, 8, 2)
    for j in [(0, 0, 0), (3, 5, 7), (7, 1, 4), (4, 4, 4)]:
        assert abs(oracle.lowpass_point(fine, 8, 2, j) - full[j]) <= 1e-12 * np.max(np.abs(full))


@pytest.mark.parametrize("k,passes", [(1, True), (3, True), (5, True), (6, False), (7, False), (11, False)])
def test_lowpass_plane_wave(k, passes):
    """A wave below the coarse Nyquist survives at the coarse nodes; at or above it, only the
    mean is left (the filter is ideal and the Nyquist plane is dropped).  A coarse cell holds
    the mass of 2^3 fine cells, hence the factor 8."""
    n, nf = 12, 24
    i = np.arange(nf)
    wave = 2.0 + np.cos(2 * np.pi * k * i / nf)[:, None, None] * np.ones((nf, nf, nf))
    fine = np.round(wave * 2.0 ** 40).astype(np.uint64)
    got = oracle.lowpass(fine, n, 2) * 2.0 ** 8 / 8.0
    j = np.arange(n)
    if passes:
        ref = 2.0 + np.cos(2 * np.pi * k * (2 * j) / nf)[:, None, None] * np.ones((n, n, n))
    else:
        ref = np.full((n, n, n), 2.0)
    assert np.max(np.abs(got - ref)) <= 1e-9


def test_lowpass_ss1_is_plain_gridding():
    rng = np.random.default_rng(5)
    fine = oracle.assign(rng.uniform(0, 10, (50, 3)), 8, 10.0, 2, 1)
    assert np.array_equal(oracle.lowpass(fine, 8, 1), fine.astype(np.float64) / Q48)


# ----------------------------------------------------------------------------- window
def test_window_uniform_is_one():
    sel = synth.uniform_selection(16, 100.0)
    assert np.all(oracle.window(sel, 16, 100.0) == 1.0)


def test_window_matches_angles():
    """Cone/hole membership by explicit angles (arccos), away from the boundaries."""
    box, n = 300.0, 24
    sel = synth.selection_sdss_like(box, seed=5, half_angle_deg=40.0)
    sel.holes = np.array([[0.0, 0.0, 0.0, 0.0]])[:0]
    h = synth.random_holes(sel.axis, sel.half_angle, math.radians(6.0), 0.3, np.random.default_rng(2))
    sel.holes = h
    w = oracle.window(sel, n, box)
    H = box / n
    g = np.arange(n) * H
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    d = np.stack([X, Y, Z], -1) - np.asarray(sel.observer)
    r = np.linalg.norm(d, axis=-1)
    rs = np.where(r > 0, r, 1)
    ang = np.arccos(np.clip(d @ np.asarray(sel.axis) / rs, -1, 1))
    inside = (ang <= sel.half_angle) & (r > 0)
    margin = np.abs(ang - sel.half_angle) > 1e-9
    for hole in h:
        ah = np.arccos(np.clip(d @ hole[:3] / rs, -1, 1))
        inside &= ~(ah < hole[3])
        margin &= np.abs(ah - hole[3]) > 1e-9
    t = r / sel.radial_params[0]
    g2 = sel.radial_params[1]
    f = t ** g2 * np.exp(g2 * (1 - t))
    ref = np.where(inside, f, 0.0)
    assert np.allclose(w[margin], ref[margin], rtol=1e-14, atol=0)
    assert inside.sum() > 100 and (~inside).sum() > 100


def test_window_radial_laws():
    n, box = 8, 80.0
    H = box / n
    for kind, params, r_at, val in [(1, (120.0,), 120.0, math.exp(-1.0)), (2, (30.0, 2.0), 30.0, 1.0)]:
        sel = synth.Selection(observer=(-r_at, 0.0, 0.0), axis=(1.0, 0.0, 0.0), half_angle=math.pi,
                              radial_kind=kind, radial_params=params + (0.0,) * (4 - len(params)))
        w = oracle.window(sel, n, box)
        assert abs(w[0, 0, 0] - val) <= 1e-15
    sel = synth.Selection(observer=(H, 2 * H, 3 * H), half_angle=math.pi)
    assert oracle.window(sel, n, box)[1, 2, 3] == 0.0


# ----------------------------------------------------------------------------- noise
def test_build_noise_fair_sample_identities():
    pr = synth.problem("c1", n_override=16, n_gal_override=3000, cache=False)
    fine = oracle.assign(pr.pos, 16, pr.box, pr.scheme, 2)
    nobs = oracle.lowpass(fine, 16, 2)
    w = oracle.window(pr.sel, 16, pr.box)
    d, b, nbar = oracle.build_noise(nobs, w, pr.n_gal)
    assert abs(nbar - pr.n_gal / np.sum(w)) <= 1e-14 * nbar   # eq:nmean, cells as volume
    assert abs(np.sum(d)) <= 1e-10 * np.sum(np.abs(d))  # sum n_obs = N_gal => sum d = 0
    assert np.all(b[w == 0] == 0.0)
    assert np.allclose(b[w > 0], (nobs - nbar * w)[w > 0], rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- prior
def test_sinv_table_power_law_closed_form():
    n, box = 16, 100.0
    k, p = synth.power_law_table(3.0, -1.5, 1e-3, 1e2)
    t = oracle.sinv_table(n, box, k, p)
    n2 = np.arange(1, t.size)
    kk = 2 * np.pi / box * np.sqrt(n2)
    assert t[0] == 0.0
    assert np.allclose(t[1:], (box / n) ** 3 / (3.0 * kk ** -1.5), rtol=1e-12)


def test_sinv_table_broken_power_law_by_hand():
    """A three-segment broken power law with slopes +1, -2, -3 and breakpoints at k = 0.1, 0.4,
    1.6, 3.2 h/Mpc: log-log interpolation is exact inside each segment, so every entry equals the
    piecewise law written out by hand, including n2 exactly at each breakpoint (the grid's k is
    built with the same operations as the table's), below the first point (extrapolated with the
    first segment) and above the last (extrapolated with the last).  An off-by-one in the segment
    search or a clamped end would put the wrong slope on some n2 and fail."""
    n = 128
    box = 40.0 * np.pi                            # 2 pi / L = 0.05 h/Mpc; kmax = 0.05 sqrt(3 * 64^2) = 5.5
    kf = 2.0 * np.pi / box
    n2_break = np.array([4, 64, 1024, 4096])      # k = 0.1, 0.4, 1.6, 3.2 (up to one rounding of kf)
    pk_k = kf * np.sqrt(n2_break.astype(np.float64))
    pk_p = np.array([100.0, 400.0, 25.0, 3.125])  # slopes +1, -2, -3 between the points
    t = oracle.sinv_table(n, box, pk_k, pk_p)
    n2 = np.arange(t.size)
    k = kf * np.sqrt(n2.astype(np.float64))
    seg = np.searchsorted(n2_break, n2, side="left") - 1   # n2 == break: the segment ending there
    seg = np.clip(seg, 0, 2)
    slope = np.array([1.0, -2.0, -3.0])[seg]
    P = pk_p[seg] * (k / pk_k[seg]) ** slope
    dV = (box / n) ** 3
    assert t[0] == 0.0
    assert np.allclose(t[1:], dV / P[1:], rtol=1e-12, atol=0)
    # the cases the docstring names are all present
    assert n2[1] < 4 and t.size - 1 > 4096
    for j, p in zip(n2_break, pk_p):
        assert abs(t[j] - dV / p) <= 1e-13 * (dV / p)
    # hand values: k = 0.05 (below the table), 0.2, 0.8, 2.4 (inside segments 1-3), 4.0 (above it)
    for j, p in [(1, 50.0), (16, 200.0), (256, 100.0), (2304, 25.0 / 3.375), (6400, 1.6)]:
        assert abs(t[j] - dV / p) <= 1e-12 * (dV / p), (j, dV / t[j], p)


# ----------------------------------------------------------------------------- operator/CG
def _small_problem(n=8, seed=0, uniform=False, nbar=0.7):
    rng = np.random.default_rng(seed)
    box = 40.0
    k, p = synth.lcdm_table()
    t = oracle.sinv_table(n, box, k, p)
    if uniform:
        w = np.ones((n, n, n))
    else:
        w = rng.uniform(0, 1, (n, n, n)) * (rng.uniform(0, 1, (n, n, n)) > 0.3)
    b = rng.standard_normal((n, n, n)) * (w > 0)
    return t, nbar, w, b, box


def _dense_operator(n, table, nbar, w):
    """A_ij = (1/V_c) sum_k S^-1(k) cos(k.(x_i - x_j)) + nbar w_i delta_ij, no FFT."""
    f = np.fft.fftfreq(n, 1.0 / n).astype(int)
    K = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1).reshape(-1, 3)
    sk = table[np.sum(K * K, axis=1)]
    g = np.arange(n)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    phase = 2 * np.pi * (X @ K.T) / n           # [cells, modes]
    C, S = np.cos(phase), np.sin(phase)
    A = (C * sk) @ C.T + (S * sk) @ S.T        # sum_k s_k cos(k.(xi-xj))
    A /= n ** 3
    A += np.diag(nbar * w.ravel())
    return A


def test_matvec_matches_dense_operator():
    t, nbar, w, b, _ = _small_problem()
    A = _dense_operator(8, t, nbar, w)
    rng = np.random.default_rng(9)
    p = rng.standard_normal((8, 8, 8))
    assert np.allclose(oracle.matvec(t, nbar, w, p).ravel(), A @ p.ravel(), rtol=0, atol=1e-12 * np.abs(A @ p.ravel()).max())


def test_operator_symmetric_positive():
    t, nbar, w, b, _ = _small_problem(n=12, seed=3)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((12, 12, 12))
    v = rng.standard_normal((12, 12, 12))
    au, av = oracle.matvec(t, nbar, w, u), oracle.matvec(t, nbar, w, v)
    assert abs(np.vdot(u, av) - np.vdot(au, v)) <= 1e-13 * abs(np.vdot(u, av))
    assert np.vdot(u, au) > 0


def test_cg_matches_dense_cholesky():
    t, nbar, w, b, _ = _small_problem()
    A = _dense_operator(8, t, nbar, w)
    L = np.linalg.cholesky(A)
    ref = np.linalg.solve(L.T, np.linalg.solve(L, b.ravel()))
    x, it, rel = oracle.cg(t, nbar, w, b, tol=1e-13)
    assert rel <= 1e-13
    assert np.linalg.norm(x.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_cg_uniform_selection_closed_form():
    """w = 1: A is Fourier-diagonal and s_k = P/(P + dV/nbar) d_k (d = b/nbar)."""
    n = 16
    t, nbar, w, b, box = _small_problem(n=n, seed=4, uniform=True, nbar=0.3)
    x, it, rel = oracle.cg(t, nbar, w, b, tol=1e-13)
    f = np.fft.fftfreq(n, 1.0 / n).astype(int)
    n2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2
    sinv = t[n2]                                   # dV / P
    d_k = np.fft.fftn(b / nbar)
    s_k = d_k / (1.0 + sinv / nbar)                # = P/(P + dV/nbar) d_k; k = 0 keeps d_0
    ref = np.real(np.fft.ifftn(s_k))
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_cg_noiseless_limit():
    """nbar -> infinity with w = 1: s -> d, error bounded by max_k dV/(nbar P(k))."""
    n = 8
    t, _, w, b, box = _small_problem(n=n, seed=6, uniform=True)
    d = b.copy()
    for nbar in (1e3, 1e6):
        x, it, rel = oracle.cg(t, nbar, w, nbar * d, tol=1e-14)
        bound = np.max(t) / nbar
        assert np.linalg.norm(x - d) <= 1.01 * bound * np.linalg.norm(d)


def test_unobserved_cells_carry_no_data():
    """Sec. 5.4 'Cluster prediction': data in w = 0 cells never reaches the solution."""
    pr = synth.problem("c1", n_override=16, n_gal_override=3000, cache=False)
    fine = oracle.assign(pr.pos, 16, pr.box, pr.scheme, 2)
    nobs = oracle.lowpass(fine, 16, 2)
    w = oracle.window(pr.sel, 16, pr.box)
    t = oracle.sinv_table(16, pr.box, pr.pk_k, pr.pk_p)
    d, b, nbar = oracle.build_noise(nobs, w, pr.n_gal)
    nobs2 = nobs.copy()
    nobs2[w == 0] += 5.0
    d2, b2, nbar2 = oracle.build_noise(nobs2, w, pr.n_gal)
    assert np.array_equal(b, b2) and nbar == nbar2
    x1 = oracle.cg(t, nbar, w, b, tol=1e-12)[0]
    x2 = oracle.cg(t, nbar2, w, b2, tol=1e-12)[0]
    assert np.array_equal(x1, x2)
    assert np.abs(x1[w == 0]).max() > 0            # the prior extrapolates into the gaps


def _dense_fourier_multiplier(n, table):
    """M_ij = (1/V_c) sum_k table(|k|^2) cos(k.(x_i - x_j)): the dense form of a Fourier-diagonal
    operator, built by cosine sums (no FFT)."""
    return _dense_operator(n, table, 0.0, np.zeros((n, n, n)))


def _prior_preconditioner(table, nbar, w):
    """The Fourier-diagonal preconditioner of the GPU's split-preconditioned CG, c^2 with
    c = S^(1/2) off k = 0 and c_0^2 = V_c / (nbar sum w) at k = 0."""
    p = np.empty_like(table)
    p[1:] = 1.0 / table[1:]
    p[0] = w.size / (nbar * w.sum())
    return p


def test_pcg_unit_preconditioner_is_textbook_cg():
    """ptable = 1 makes z = r (up to one FFT round trip), so every iterate is textbook CG's."""
    t, nbar, w, b, _ = _small_problem(n=12, seed=11)
    for k in (1, 4, 15):
        x1 = oracle.cg(t, nbar, w, b, tol=1e-15, max_iter=k, allow_unconverged=True)[0]
        x2 = oracle.pcg(t, np.ones_like(t), nbar, w, b, tol=1e-15, max_iter=k, allow_unconverged=True)[0]
        assert np.linalg.norm(x2 - x1) <= 1e-12 * np.linalg.norm(x1)


def test_pcg_exact_preconditioner_solves_in_one_step():
    """w = 1 makes A Fourier-diagonal, A = F^-1 diag(S^-1 + nbar) F; with M^-1 = A^-1 the first PCG
    step lands on the solution, the closed form s_k = b_k / (S^-1(k) + nbar)."""
    n = 16
    t, nbar, w, b, _ = _small_problem(n=n, seed=12, uniform=True, nbar=0.35)
    x, it, rel = oracle.pcg(t, 1.0 / (t + nbar), nbar, w, b, tol=1e-12)
    assert it == 1 and rel <= 1e-12
    f = np.fft.fftfreq(n, 1.0 / n).astype(int)
    n2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2
    ref = np.real(np.fft.ifftn(np.fft.fftn(b) / (t[n2] + nbar)))
    assert np.linalg.norm(x - ref) <= 1e-13 * np.linalg.norm(ref)


def test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space():
    """Brute force at 4^3: the k-th PCG iterate is the A-norm-closest point to the solution in
    K_k(M^-1 A, M^-1 b), i.e. x_k = Q (Q^T A Q)^-1 Q^T b with Q an orthonormal basis of that space
    (dense A and M^-1 from cosine sums).  A transposed operand, a wrong beta (e.g. <r,r> in place
    of <r,z>) or an unpreconditioned residual changes x_k."""
    n = 4
    t, nbar, w, b, _ = _small_problem(n=n, seed=13)
    pt = _prior_preconditioner(t, nbar, w)
    A = _dense_operator(n, t, nbar, w)
    Mi = _dense_fourier_multiplier(n, pt)
    bv = b.ravel()
    v = Mi @ bv
    K = []
    for k in range(1, 6):
        K.append(v)
        v = Mi @ (A @ v)
        Q, _ = np.linalg.qr(np.stack(K, 1))
        ref = Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ bv)
        x = oracle.pcg(t, pt, nbar, w, b, tol=1e-15, max_iter=k, allow_unconverged=True)[0]
        assert np.linalg.norm(x.ravel() - ref) <= 1e-10 * np.linalg.norm(ref), k


def test_pcg_matches_dense_cholesky():
    """The prior preconditioner leaves the solution unchanged: 8^3 against the dense solve."""
    t, nbar, w, b, _ = _small_problem()
    A = _dense_operator(8, t, nbar, w)
    L = np.linalg.cholesky(A)
    ref = np.linalg.solve(L.T, np.linalg.solve(L, b.ravel()))
    x, it, rel = oracle.pcg(t, _prior_preconditioner(t, nbar, w), nbar, w, b, tol=1e-13)
    assert rel <= 1e-13
    assert np.linalg.norm(x.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)
    true = np.linalg.norm(b - oracle.matvec(t, nbar, w, x)) / np.linalg.norm(b)
    assert true <= 1e-13


def test_cg_zero_rhs_and_residual_contract():
    t, nbar, w, b, _ = _small_problem(seed=8)
    x, it, rel = oracle.cg(t, nbar, w, np.zeros_like(b), tol=1e-8)
    assert it == 0 and np.all(x == 0)
    x, it, rel = oracle.cg(t, nbar, w, b, tol=1e-6)
    true = np.linalg.norm(b - oracle.matvec(t, nbar, w, x)) / np.linalg.norm(b)
    assert true <= 1e-6 and abs(true - rel) <= 1e-12


# ----------------------------------------------------------------------------- coarse-space CG
# oracle.coarse.adef2: the mixed solves' inner CG with the two-level A-DEF2 preconditioner on the
# Fourier modes |k|^2 <= K^2 (test infrastructure for the GPU's coarse-space solves).
def _dense_solve(t, nbar, w, b):
    A = _dense_operator(w.shape[0], t, nbar, w)
    L = np.linalg.cholesky(A)
    return np.linalg.solve(L.T, np.linalg.solve(L, b.ravel())).reshape(b.shape)


def test_adef2_full_coarse_space_solves_in_the_start_step():
    """With every mode of the 8^3 grid coarse (|k|^2 <= 48 < 7^2), E is the whole operator and the
    start step x_0 = Z E^-1 Z^H b' is the solution: the dense solve in real space, to 1e-10."""
    from oracle.coarse import adef2
    t, nbar, w, b, _ = _small_problem()
    s, it, rel = adef2(t, nbar, w, b, 7, tol=1e-12, max_iter=20)
    assert it == 1 and rel <= 1e-12
    ref = _dense_solve(t, nbar, w, b)
    assert np.linalg.norm(s - ref) <= 1e-10 * np.linalg.norm(ref)


def test_adef2_without_coarse_space_is_the_prior_preconditioned_cg():
    """No coarse modes: Q = 0, the start step is empty, z = r, and k more iterations are the
    oracle's preconditioned CG with M^-1 = C^2 (oracle.pcg, C code) after k iterations."""
    from oracle.coarse import adef2
    t, nbar, w, b, _ = _small_problem(n=12, seed=21)
    pt = _prior_preconditioner(t, nbar, w)
    for k in (1, 4, 11):
        ref = oracle.pcg(t, pt, nbar, w, b, tol=1e-15, max_iter=k, allow_unconverged=True)[0]
        s = adef2(t, nbar, w, b, None, tol=1e-15, max_iter=k + 1)[0]
        assert np.linalg.norm(s - ref) <= 1e-11 * np.linalg.norm(ref), k


@pytest.mark.parametrize("K", [1, 2, 3])
def test_adef2_converges_to_the_dense_solution(K):
    from oracle.coarse import adef2
    t, nbar, w, b, _ = _small_problem(seed=22)
    s, it, rel = adef2(t, nbar, w, b, K, tol=1e-13, max_iter=400)
    assert rel <= 1e-13
    ref = _dense_solve(t, nbar, w, b)
    assert np.linalg.norm(s - ref) <= 1e-10 * np.linalg.norm(ref)
    # the canonical residual of the returned s, by the oracle's own operator
    assert np.linalg.norm(b - oracle.matvec(t, nbar, w, s)) <= 1e-11 * np.linalg.norm(b)


def test_adef2_start_step_leaves_no_coarse_residual():
    """After the start step the residual has no component on the coarse modes (Z^H r_0 = 0), and
    CG keeps it so (Z^H A' p = 0 for every search direction)."""
    from oracle.coarse import adef2
    t, nbar, w, b, _ = _small_problem(n=12, seed=23)
    for k in (1, 2, 6):
        _, _, _, (pb, y, r) = adef2(t, nbar, w, b, 2, tol=1e-15, max_iter=k, return_state=True)
        assert np.linalg.norm(r[pb.idx]) <= 1e-11 * np.linalg.norm(pb.rhs[pb.idx]), k


def test_adef2_iterates_equal_deflated_cg_on_dense_matrices():
    """Brute force at 4^3: with the start x_0 = Q b', A-DEF2's iterates are those of deflated CG
    (Saad, Yeung, Erhel and Guyomarc'h 2000: p = r + beta p - Z E^-1 Z^H A' r, alpha and beta from
    <r, r>), here run on the dense operator A' = diag(m) + diag(c) F diag(nbar w) F^-1 diag(c) built
    from explicit exponential sums, not an FFT.  A wrong sign of the coarse term, a dropped r in
    z = r - Q (A' r - r), or a transposed E changes them."""
    from oracle.coarse import adef2
    n, K = 4, 1
    t, nbar, w, b, _ = _small_problem(n=n, seed=24)
    f = np.fft.fftfreq(n, 1.0 / n).astype(int)
    modes = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1).reshape(-1, 3)
    g = np.arange(n)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    F = np.exp(-2j * np.pi * (modes @ X.T) / n)                 # forward DFT [modes, cells]
    n2 = np.sum(modes * modes, axis=1)
    c = np.where(n2 > 0, 1.0 / np.sqrt(np.where(n2 > 0, t[n2], 1.0)), 1.0 / np.sqrt(nbar * w.sum() / w.size))
    m = np.where(n2 > 0, 1.0, 0.0)
    Ap = np.diag(m) + (c[:, None] * F) @ np.diag(nbar * w.ravel()) @ (F.conj().T * c[None, :]) / n ** 3
    rhs = c * (F @ b.ravel())
    Z = np.eye(n ** 3)[:, n2 <= K * K]
    E = Z.T @ Ap @ Z
    Q = lambda v: Z @ np.linalg.solve(E, Z.T @ v)
    dot = lambda u, v: float(np.real(np.vdot(u, v)))
    x = Q(rhs)
    r = rhs - Ap @ x
    p = r - Q(Ap @ r)
    xs = [x.copy()]
    for _ in range(5):
        q = Ap @ p
        rr = dot(r, r)
        a = rr / dot(p, q)
        x = x + a * p
        r = r - a * q
        xs.append(x.copy())
        p = r + (dot(r, r) / rr) * p - Q(Ap @ r)
    for k, xk in enumerate(xs):
        sk = np.real((F.conj().T @ (c * xk)) / n ** 3).reshape(b.shape)
        s = adef2(t, nbar, w, b, K, tol=1e-15, max_iter=k + 1)[0]
        assert np.linalg.norm(s - sk) <= 1e-10 * np.linalg.norm(sk), k
