"""GPU path vs the CPU oracle, through the C ABI, on seeded synthetic inputs.

Tolerances: the fine mass grid is compared bit for bit; n_obs, w, d, b to relative L2 1e-13
(FP64 arithmetic on both sides, different summation orders); the FP64 Wiener solution to
relative L2 1e-10 with both solvers at residual 1e-12; the mixed-precision solution to 1e-6
after refinement.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0906_3978_gb300 as wf  # noqa: E402


def rl2(a, r):
    a, r = np.asarray(a), np.asarray(r)
    den = np.linalg.norm(r)
    return float(np.linalg.norm(a - r) / (den if den > 0 else 1.0))


@pytest.fixture(scope="module")
def ctx():
    wf.build()
    c = wf.Context(0)
    yield c
    c.close()


DEV = "cuda:0"


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def fine_host(t, shape):
    return host(t).view(np.uint64).reshape(shape)


# ------------------------------------------------------------------------ assignment
def _positions(kind, n, box, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.uniform(-0.3 * box, 1.3 * box, size=(4000, 3))       # wrap both ways
    if kind == "clustered":
        c = rng.uniform(0, box, size=(20, 3))
        return (c[rng.integers(0, 20, 6000)] + rng.normal(0, box / (4 * n), size=(6000, 3))) % box
    # nodes and half-nodes of the fine grid, exactly representable
    h = box / (2 * n)
    i = rng.integers(0, 2 * n, size=(3000, 3)).astype(np.float64)
    return (i + rng.integers(0, 2, size=(3000, 3)) * 0.5) * h


@pytest.mark.parametrize("n", [16, 24, 64, 108])
@pytest.mark.parametrize("scheme", [wf.CIC, wf.TSC])
@pytest.mark.parametrize("ss", [1, 2])
@pytest.mark.parametrize("kind", ["uniform", "clustered", "nodes"])
def test_assign_fine_grid_bit_exact(ctx, n, scheme, ss, kind):
    box = 64.0 if kind == "nodes" else 100.0 + n
    pos = _positions(kind, n, box, seed=n * 7 + scheme + ss)
    nf = ss * n
    fine = torch.empty(nf ** 3, dtype=torch.int64, device=DEV)
    nobs = ctx.grid_assign(gpu(pos), n, box, scheme, ss, fine_out=fine)
    ref = oracle.assign(pos, n, box, scheme, ss)
    assert np.array_equal(fine_host(fine, ref.shape), ref)
    ref_obs = oracle.lowpass(ref, n, ss)
    got = host(nobs)
    assert rl2(got, ref_obs) <= 1e-13
    assert abs(got.sum() - pos.shape[0]) <= 1e-9 * pos.shape[0]


def test_assign_deterministic(ctx):
    pos = _positions("clustered", 32, 120.0, 3)
    outs = []
    for _ in range(2):
        fine = torch.empty(64 ** 3, dtype=torch.int64, device=DEV)
        ctx.grid_assign(gpu(pos[::-1].copy() if outs else pos), 32, 120.0, wf.TSC, 2, fine_out=fine)
        outs.append(host(fine))
    assert np.array_equal(outs[0], outs[1])      # order of galaxies does not matter


def test_assign_edge_cases(ctx):
    # no galaxies
    nobs = ctx.grid_assign(None, 16, 50.0, wf.TSC, 2)
    assert np.all(host(nobs) == 0.0)
    # non-finite position
    bad = gpu(np.array([[1.0, np.nan, 2.0], [3.0, 4.0, 5.0]]))
    st, _ = ctx.grid_assign(bad, 16, 50.0, wf.TSC, 2, check=False)
    assert st == wf.ERR_ARG
    # 65536 galaxies exactly on one fine node overflow a uint64 cell (65536 * 2^48 = 2^64)
    pos = np.tile([[2.0, 2.0, 2.0]], (65536, 1))
    st, _ = ctx.grid_assign(gpu(pos), 16, 16.0, wf.CIC, 2, check=False)
    assert st == wf.ERR_OVERFLOW
    fine = torch.empty(32 ** 3, dtype=torch.int64, device=DEV)
    ctx.grid_assign(gpu(pos[:65535]), 16, 16.0, wf.CIC, 2, fine_out=fine)
    assert int(fine_host(fine, (32, 32, 32))[4, 4, 4]) == 65535 * 2 ** 48
    # unsupported size, bad box
    st, _ = ctx.grid_assign(gpu(pos[:10]), 20, 16.0, wf.CIC, 2, n_obs=torch.empty(8000, dtype=torch.float64,
                                                                                  device=DEV), check=False)
    assert st == wf.ERR_UNSUPPORTED
    st, _ = ctx.grid_assign(gpu(pos[:10]), 16, -1.0, wf.CIC, 2, check=False)
    assert st == wf.ERR_ARG


# ------------------------------------------------------------------------ window / noise
def _pipeline_oracle(pr):
    fine = oracle.assign(pr.pos, pr.n, pr.box, pr.scheme, 2)
    nobs = oracle.lowpass(fine, pr.n, 2)
    w = oracle.window(pr.sel, pr.n, pr.box)
    d, b, nbar = oracle.build_noise(nobs, w, pr.n_gal)
    return fine, nobs, w, d, b, nbar


@pytest.mark.parametrize("name,n", [("c1", 32), ("c1", 48), ("c2", 32), ("c2", 64)])
def test_noise_parity(ctx, name, n):
    pr = synth.problem(name, n_override=n, cache=False)
    fine, nobs_o, w_o, d_o, b_o, nbar_o = _pipeline_oracle(pr)
    nobs = gpu(nobs_o)
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
    # the oracle sums w in sequence: relative rounding error up to (V - 1) u, u = 2^-53
    assert abs(nbar - nbar_o) <= n ** 3 * 1.2e-16 * nbar_o
    assert rl2(host(w), w_o) <= 1e-14
    assert np.array_equal(host(w) > 0, w_o > 0)      # identical membership decisions
    assert rl2(host(d), d_o) <= 1e-13
    assert rl2(host(b), b_o) <= 1e-13


def test_noise_rejects_empty_window(ctx):
    sel = synth.Selection(observer=(-1e3, 0, 0), axis=(-1.0, 0.0, 0.0), half_angle=0.1)
    nobs = torch.zeros((16, 16, 16), dtype=torch.float64, device=DEV)
    st = ctx.build_noise(sel, nobs, 10, 50.0, check=False)[0]
    assert st == wf.ERR_ARG


# ------------------------------------------------------------------------ solve
def _solve_inputs(name, n):
    pr = synth.problem(name, n_override=n, cache=False)
    _, nobs, w, d, b, nbar = _pipeline_oracle(pr)
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    return pr, w, b, nbar, tab


@pytest.mark.parametrize("name,n", [("c1", 16), ("c1", 24), ("c1", 32), ("c2", 32), ("c2", 48), ("c1", 64),
                                    ("c2", 72), ("c2", 108)])
@pytest.mark.parametrize("precond", [1, 0])
def test_solve_fp64_parity(ctx, name, n, precond):
    pr, w, b, nbar, tab = _solve_inputs(name, n)
    ref, it_o, rel_o = oracle.cg(tab, nbar, w, b, tol=1e-12)
    s, info = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-12, max_iter=20000,
                        prec=wf.FP64, precond=precond)
    assert info.status == wf.OK and info.rel_residual <= 1e-12
    assert rl2(host(s), ref) <= 1e-10
    # the oracle's operator agrees that the GPU solution solves the system
    res = b - oracle.matvec(tab, nbar, w, host(s))
    assert np.linalg.norm(res) <= 2e-12 * np.linalg.norm(b)
    if precond == 0:
        assert abs(info.iters - it_o) <= max(3, 0.05 * it_o)     # same algorithm


@pytest.mark.parametrize("name,n", [("c1", 24), ("c1", 32), ("c2", 48), ("c2", 64), ("c2", 72), ("c2", 108)])
def test_solve_mixed_parity(ctx, name, n):
    pr, w, b, nbar, tab = _solve_inputs(name, n)
    ref = oracle.cg(tab, nbar, w, b, tol=1e-12)[0]
    s, info = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-9, prec=wf.MIXED)
    assert info.status == wf.OK and info.rel_residual <= 1e-9 and info.outer_iters >= 2
    assert rl2(host(s), ref) <= 1e-6
    # at the production tolerance the residual contract still holds in FP64
    s6, info6 = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-6, prec=wf.MIXED)
    res = b - oracle.matvec(tab, nbar, w, host(s6))
    assert np.linalg.norm(res) <= 1.0001e-6 * np.linalg.norm(b)


def test_solve_uniform_selection_closed_form(ctx):
    n, box, nbar = 32, 80.0, 0.4
    k, p = synth.lcdm_table()
    rng = np.random.default_rng(2)
    b = rng.standard_normal((n, n, n))
    w = np.ones((n, n, n))
    s, info = ctx.solve(gpu(w), nbar, gpu(b), box, k, p, tol=1e-13, max_iter=20000)
    tab = oracle.sinv_table(n, box, k, p)
    f = np.fft.fftfreq(n, 1.0 / n).astype(int)
    n2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2
    ref = np.real(np.fft.ifftn(np.fft.fftn(b / nbar) / (1.0 + tab[n2] / nbar)))
    assert rl2(host(s), ref) <= 1e-11


def test_solve_zero_rhs_and_errors(ctx):
    pr, w, b, nbar, tab = _solve_inputs("c1", 16)
    z = np.zeros_like(b)
    s, info = ctx.solve(gpu(w), nbar, gpu(z), pr.box, pr.pk_k, pr.pk_p, tol=1e-8)
    assert info.status == wf.OK and info.iters == 0 and np.all(host(s) == 0.0)
    for prec in (wf.FP64, wf.MIXED):
        s, info = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-12, max_iter=3, prec=prec,
                            check=False)
        assert info.status == wf.ERR_NOT_CONVERGED and info.iters >= 3 and info.rel_residual > 1e-12
    for bad in [dict(nbar=0.0), dict(tol=0.0), dict(max_iter=0)]:
        kw = dict(nbar=nbar, tol=1e-6, max_iter=100)
        kw.update(bad)
        with pytest.raises(wf.WfError) as e:
            ctx.solve(gpu(w), kw["nbar"], gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=kw["tol"], max_iter=kw["max_iter"])
        assert e.value.status == wf.ERR_ARG
    with pytest.raises(wf.WfError) as e:
        ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k[::-1].copy(), pr.pk_p, tol=1e-6)
    assert e.value.status == wf.ERR_ARG


def test_solve_fixed_iterations_match_textbook_cg(ctx):
    """precond = 0 is textbook CG: after k iterations from 0 both sides hold the same x_k."""
    pr, w, b, nbar, tab = _solve_inputs("c2", 48)
    for k in (1, 2, 7):
        ref = oracle.cg(tab, nbar, w, b, tol=1e-14, max_iter=k, allow_unconverged=True)[0]
        s, info = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=k, precond=0,
                            check=False)
        assert info.status == wf.ERR_NOT_CONVERGED and info.iters == k
        assert rl2(host(s), ref) <= 1e-11


def test_solve_deterministic(ctx):
    pr, w, b, nbar, tab = _solve_inputs("c2", 32)
    s1, _ = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-8)
    a = host(s1).copy()
    s2, _ = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-8)
    assert np.array_equal(a, host(s2))


def test_end_to_end_pipeline(ctx):
    pr = synth.problem("c1", n_override=32, cache=False)
    fine_o, nobs_o, w_o, d_o, b_o, nbar_o = _pipeline_oracle(pr)
    tab = oracle.sinv_table(pr.n, pr.box, pr.pk_k, pr.pk_p)
    ref = oracle.cg(tab, nbar_o, w_o, b_o, tol=1e-12)[0]
    nobs = ctx.grid_assign(gpu(pr.pos), pr.n, pr.box, pr.scheme, 2)
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
    s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-12)
    assert rl2(host(s), ref) <= 1e-10


@pytest.mark.parametrize("n", [128, 256])
def test_fresh_context_mixed_first(n):
    """A new context whose first solve is mixed precision sizes every workspace itself."""
    pr = synth.problem("c2", n_override=n, cache=False)
    with wf.Context(0) as c2:
        nobs = c2.grid_assign(gpu(pr.pos), pr.n, pr.box, pr.scheme, 2)
        w, d, b, nbar = c2.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
        sm, im = c2.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=wf.MIXED)
        sd, idd = c2.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=wf.FP64)
        assert im.status == wf.OK and idd.status == wf.OK
        assert im.rel_residual <= 1e-8 and idd.rel_residual <= 1e-8
        assert rl2(host(sm), host(sd)) <= 1e-6


@pytest.mark.parametrize("n", [128, 256])
def test_fixed_iterations_large_grid(ctx, n):
    """Several tiles per pass and many CTAs: k textbook-CG iterations match the oracle's."""
    pr = synth.problem("c2", n_override=n, cache=False)
    nobs = ctx.grid_assign(gpu(pr.pos), pr.n, pr.box, pr.scheme, 2)
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
    wh, bh = host(w), host(b)
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    ref = oracle.cg(tab, nbar, wh, bh, tol=1e-14, max_iter=3, allow_unconverged=True)[0]
    s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=3, precond=0, check=False)
    assert info.iters == 3
    assert rl2(host(s), ref) <= 1e-11


def _prior_preconditioner(tab, nbar, w):
    """m = c^2 of the GPU's split preconditioning (precond = 1): c = S^(1/2) off k = 0 (m = P/dV =
    1/S^-1) and c_0^2 = V_c / (nbar sum w).  CG on (C A C) y = C b with s = C y takes the same
    iterates as preconditioned CG on A s = b with M^-1 = C^2, which the oracle runs."""
    m = np.empty_like(tab)
    m[1:] = 1.0 / tab[1:]
    m[0] = w.size / (nbar * w.sum())
    return m


def fp32_iterate_tol(n):
    """Bound for a few FP32 CG iterates against the FP64 ones.  One FP32 operator application
    (a forward and an inverse 3D transform of log2(V) radix stages each, storage in FP32) has a
    relative error of about 2 log2(V) u, u = 2^-24; the tolerance allows twice that,
    4 log2(V) u (5e-6 at 128^3, 6.4e-6 at 512^3).  For the iterates checked here (k <= 3 with
    the prior preconditioner, k <= 20 textbook) the Krylov recurrences do not amplify that error:
    a CPU emulation of the FP32 arithmetic (FP32 vectors and transforms, FP64 dots) stays at
    2e-7 to 4e-7 of the FP64 iterates at 128^3 and 256^3.  (With the prior preconditioner at
    k = 20 the FP32 and FP64 iterates part by a few percent: the recurrences have lost
    orthogonality at different rates, so that case is not an iterate comparison.)"""
    return 4.0 * 3 * math.log2(n) * 2.0 ** -24


@pytest.mark.parametrize("n", [48, 128, 256])
def test_fixed_iterations_preconditioned_match_oracle_pcg(ctx, n):
    """precond = 1 (the production solver): after k iterations from 0, the FP64 path holds the
    oracle's preconditioned-CG iterate to 1e-11, and the FP32 inner solve of the mixed path (one
    refinement step, k inner iterations, s = C e_k) holds it within the FP32 bound."""
    pr = synth.problem("c2", n_override=n, cache=False)
    nobs = ctx.grid_assign(gpu(pr.pos), pr.n, pr.box, pr.scheme, 2)
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
    wh, bh = host(w), host(b)
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    pt = _prior_preconditioner(tab, nbar, wh)
    for k in ((1, 3, 7) if n <= 48 else (3,)):
        ref = oracle.pcg(tab, pt, nbar, wh, bh, tol=1e-14, max_iter=k, allow_unconverged=True)[0]
        s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=k, precond=1, prec=wf.FP64,
                            check=False)
        assert info.status == wf.ERR_NOT_CONVERGED and info.iters == k
        assert rl2(host(s), ref) <= 1e-11, k
        if k > 3:
            continue
        s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=k, precond=1, prec=wf.MIXED,
                            check=False)
        assert info.status == wf.ERR_NOT_CONVERGED and info.iters == k and info.outer_iters == 1
        assert rl2(host(s), ref) <= fp32_iterate_tol(n), k


def test_autotune_every_variant_matches_oracle(ctx):
    """wf_autotune times each launch variant of the FP32 passes at 128^3 and keeps the fastest;
    every variant (forced through the tuning table) gives the oracle's preconditioned-CG iterate
    within the FP32 bound, and the table round-trips through its JSON form."""
    n = 128
    pr = synth.problem("c2", n_override=n, cache=False)
    nobs = ctx.grid_assign(gpu(pr.pos), pr.n, pr.box, pr.scheme, 2)
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
    wh, bh = host(w), host(b)
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    ref = oracle.pcg(tab, _prior_preconditioner(tab, nbar, wh), nbar, wh, bh, tol=1e-14, max_iter=3,
                     allow_unconverged=True)[0]
    before = ctx.tune_get()
    report = ctx.autotune(n, wf.MIXED)
    passes = {p["pass"]: p for p in report}
    table = ctx.tune_get()
    assert set(passes) <= set(table)
    for key, p in passes.items():
        names = [v["name"] for v in p["variants"]]
        assert len(names) >= 2 and all(v["ms"] > 0 for v in p["variants"])
        assert names[table[key]] == p["chosen"]
        assert p["variants"][table[key]]["ms"] == min(v["ms"] for v in p["variants"])
        for i in range(len(names)):
            ctx.tune_set({key: i})
            s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=3, precond=1,
                                prec=wf.MIXED, check=False)
            assert info.iters == 3
            assert rl2(host(s), ref) <= fp32_iterate_tol(n), (key, names[i])
    ctx.tune_set(table)
    assert ctx.tune_get() == table
    ctx.tune_set({k: 0 for k in table if k not in before})   # leave the shared context as it was
    ctx.tune_set(before)


def test_fp64_rate_is_plausible(ctx):
    """wf_fp64_rate, the FP64 peak the bench reports the FP64 passes against: positive, repeatable
    to 10%, and within the range GB300-class parts span (0.3-100 TFLOP/s FP64 FMA)."""
    a, b = ctx.fp64_rate(), ctx.fp64_rate()
    assert 0.3e12 < a < 100e12 and abs(a - b) <= 0.1 * max(a, b)


def test_fixed_iterations_full_size_workload(ctx):
    """The 512^3 workload the benchmark times, where a converged oracle solve does not fit in test
    time: both sides run k = 20 textbook-CG iterations from 0 (precond = 0).  The FP64 path holds
    the oracle's x_20 to 1e-10; the FP32 inner solve of the mixed path (its 512^3 geometry: 32
    elements per thread, radix-16/32 z passes, 16-line tiles) within the FP32 bound."""
    pr = synth.problem("c3")
    n, k = pr.n, 20
    nobs = ctx.grid_assign(gpu(pr.pos), n, pr.box, pr.scheme, 2)
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box, want_d=False)
    del nobs, d
    wh, bh = host(w), host(b)
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=k, precond=0, prec=wf.FP64,
                        check=False)
    assert info.status == wf.ERR_NOT_CONVERGED and info.iters == k
    s64 = host(s).copy()
    s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=k, precond=0, prec=wf.MIXED,
                        check=False)
    assert info.status == wf.ERR_NOT_CONVERGED and info.iters == k and info.outer_iters == 1
    s32 = host(s).copy()
    del s, w, b
    ref = oracle.cg(tab, nbar, wh, bh, tol=1e-14, max_iter=k, allow_unconverged=True)[0]
    assert rl2(s64, ref) <= 1e-10
    assert rl2(s32, ref) <= fp32_iterate_tol(n)


@pytest.mark.parametrize("n", [128, 192, 256, 384])
def test_fused_planes_match_separate_passes(n):
    """The cluster kernel for the y / z / y transforms (clusters of 2, 3, 4, 6 CTAs at these
    sizes) and the three separate passes apply the same FP32 operator: a few inner iterations
    give the same iterate, and a solve with the cluster kernel meets the FP64 residual."""
    pr = synth.problem("c2", n_override=n, cache=False)
    with wf.Context(0) as c:
        nobs = c.grid_assign(gpu(pr.pos), pr.n, pr.box, pr.scheme, 2)
        w, d, b, nbar = c.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
        out, its = [], []
        for fused in (False, True):
            c.set_fused_planes(fused)
            s, info = c.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=6, prec=wf.MIXED,
                              check=False)
            out.append(host(s).copy())
            its.append(info.iters)
        assert its[0] == its[1] and 0 < its[0] <= 6
        assert rl2(out[1], out[0]) <= 1e-5
        s, info = c.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=wf.MIXED)
        assert info.status == wf.OK and info.rel_residual <= 1e-8
        c.set_fused_planes(False)
        s0, info0 = c.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=wf.MIXED)
        assert rl2(host(s), host(s0)) <= 1e-6


def test_full_size_workload(ctx):
    """The 512^3 workload the benchmark times (1024^3 fine grid, TSC, the same launches): the
    fine grid bit for bit against the oracle's, the window's membership decisions exactly and
    its values to 1e-14, n_obs at sampled nodes against the oracle's direct low-pass sum, and
    the mixed solve's residual recomputed by the oracle's own operator."""
    pr = synth.problem("c3")
    n, nf = pr.n, 2 * pr.n
    fine_d = torch.empty(nf ** 3, dtype=torch.int64, device=DEV)
    nobs = ctx.grid_assign(gpu(pr.pos), n, pr.box, pr.scheme, 2, fine_out=fine_d)
    fine = fine_host(fine_d, (nf, nf, nf))
    del fine_d
    ref = oracle.assign(pr.pos, n, pr.box, pr.scheme, 2)
    assert np.array_equal(fine, ref)
    del fine
    nobs_h = host(nobs)
    pts = [tuple(int(v) for v in np.unravel_index(i, (n, n, n)))
           for i in np.argsort(nobs_h, axis=None)[-3:]]
    rng = np.random.default_rng(5)
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(3)] + [(0, 0, 0)]
    vals = [oracle.lowpass_point(ref, n, 2, j) for j in pts]
    scale = max(1.0, max(abs(v) for v in vals))
    for j, v in zip(pts, vals):
        assert abs(nobs_h[j] - v) <= 1e-11 * scale, (j, nobs_h[j], v)
    del ref
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box, want_d=False)
    wh, w_ref = host(w), oracle.window(pr.sel, n, pr.box)
    assert np.array_equal(wh > 0, w_ref > 0)
    assert rl2(wh, w_ref) <= 1e-14
    assert abs(nbar - pr.n_gal / w_ref.sum()) <= 1e-12 * nbar
    s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=pr.tol, prec=wf.MIXED)
    assert info.status == wf.OK and info.rel_residual <= pr.tol
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    bh = host(b)
    res = bh - oracle.matvec(tab, nbar, wh, host(s))
    assert np.linalg.norm(res) <= 1.0001 * pr.tol * np.linalg.norm(bh)


# ------------------------------------------------------------------------ batched solves
def _mock(n, seed, box_per_cell=1.953):
    """A small mock of the batched workload: LCDM prior, SDSS-like selection, its own seed."""
    pr = synth.problem("c2", n_override=n, cache=False)
    rng = np.random.default_rng(seed)
    box = n * box_per_cell
    sel = synth.selection_sdss_like(box, seed)
    pos = synth.lognormal_catalogue(n, box, pr.pk_k, pr.pk_p, sel, float(rng.uniform(2e3, 2e4)), seed)
    return box, sel, pos, pr.pk_k, pr.pk_p


@pytest.mark.parametrize("prec", [wf.FP64, wf.MIXED])
def test_batch_equals_individual_solves(ctx, prec):
    """Systems of uneven sizes solved in one batch give the same result as solved alone."""
    probs, singles = [], []
    for i, n in enumerate([32, 48, 32, 64, 48, 24]):
        box, sel, pos, k, p = _mock(n, 2000 + i)
        nobs = ctx.grid_assign(gpu(pos), n, box, wf.TSC, 2)
        w, d, b, nbar = ctx.build_noise(sel, nobs, pos.shape[0], box)
        probs.append(dict(w=w, nbar=nbar, b=b, box=box, pk_k=k, pk_p=p, tol=1e-8, prec=prec))
        s, info = ctx.solve(w, nbar, b, box, k, p, tol=1e-8, prec=prec)
        singles.append((host(s).copy(), info.iters))
    st, outs, infos = ctx.solve_batch(probs)
    assert st == wf.OK
    for (ref, it), s, info in zip(singles, outs, infos):
        assert info.status == wf.OK and info.rel_residual <= 1e-8
        tol = 1e-12 if prec == wf.FP64 else 1e-6
        assert rl2(host(s), ref) <= tol
        if prec == wf.FP64:
            assert info.iters == it                        # same iterates, same count


def test_batch_matches_oracle(ctx):
    probs, refs = [], []
    for i, n in enumerate([24, 32]):
        box, sel, pos, k, p = _mock(n, 2100 + i)
        fine = oracle.assign(pos, n, box, 2, 2)
        nobs = oracle.lowpass(fine, n, 2)
        w = oracle.window(sel, n, box)
        d, b, nbar = oracle.build_noise(nobs, w, pos.shape[0])
        tab = oracle.sinv_table(n, box, k, p)
        refs.append(oracle.cg(tab, nbar, w, b, tol=1e-12)[0])
        probs.append(dict(w=gpu(w), nbar=nbar, b=gpu(b), box=box, pk_k=k, pk_p=p, tol=1e-12, max_iter=20000))
    st, outs, infos = ctx.solve_batch(probs)
    assert st == wf.OK
    for ref, s in zip(refs, outs):
        assert rl2(host(s), ref) <= 1e-10


# ------------------------------------------------------------------------ serving
def _serve_inputs(n, seed):
    box, sel, pos, k, p = _mock(n, seed)
    c = wf.Context(0)
    nobs = c.grid_assign(gpu(pos), n, box, wf.TSC, 2)
    w, d, b, nbar = c.build_noise(sel, nobs, pos.shape[0], box)
    out = (host(w).copy(), host(b).copy(), nbar, box, k, p)
    c.close()
    return out


def test_serving_results_same_alone_and_in_mix():
    """Requests of mixed sizes and precisions, some submitted while others run, give the same
    solution as the same request solved alone."""
    wf.build()
    reqs = [(32, 3000, wf.FP64), (48, 3001, wf.MIXED), (64, 3002, wf.FP64), (32, 3003, wf.MIXED),
            (64, 3004, wf.MIXED), (24, 3005, wf.FP64)]
    inputs = [_serve_inputs(n, seed) for n, seed, _ in reqs]
    with wf.Context(0) as ctx:
        ids = []
        for i, ((n, seed, prec), (w, b, nbar, box, k, p)) in enumerate(zip(reqs, inputs)):
            ids.append(ctx.submit(w, nbar, b, box, k, p, tol=1e-8, prec=prec))
            if i == 2:  # the first requests are resident while the rest arrive
                st, _ = ctx.poll(ids[0], timeout_ms=0)
                assert st in (wf.PENDING, wf.OK)
        results = []
        for rid, (n, _, _) in zip(ids, reqs):
            s = np.empty(n ** 3)
            st, info = ctx.poll(rid, timeout_ms=-1, s_out=s)
            assert st == wf.OK and info.rel_residual <= 1e-8 and info.latency_s > 0
            results.append(s.reshape(n, n, n))
        for (n, seed, prec), (w, b, nbar, box, k, p), s in zip(reqs, inputs, results):
            alone, info = ctx.solve(gpu(w), nbar, gpu(b), box, k, p, tol=1e-8, prec=prec)
            assert rl2(s, host(alone)) <= (1e-12 if prec == wf.FP64 else 1e-6)


def test_serving_errors():
    wf.build()
    w, b, nbar, box, k, p = _serve_inputs(16, 3010)
    with wf.Context(0) as ctx:
        with pytest.raises(wf.WfError) as e:
            ctx.submit(w, -1.0, b, box, k, p)
        assert e.value.status == wf.ERR_ARG
        st, _ = ctx.poll(12345, timeout_ms=0)
        assert st == wf.ERR_ARG
        rid = ctx.submit(w, nbar, b, box, k, p, tol=1e-6)
        st, info = ctx.poll(rid, timeout_ms=-1)
        assert st == wf.OK
        st, _ = ctx.poll(rid, timeout_ms=0)          # released after the final poll
        assert st == wf.ERR_ARG


# ------------------------------------------------------------------------ failure handling
def test_budget_exceeded_is_reported():
    """A context whose HBM budget cannot hold the workspaces returns WF_ERR_OOM, and a
    following call on a context with room succeeds."""
    wf.build()
    pr, w, b, nbar, tab = _solve_inputs("c1", 32)
    with wf.Context(0, hbm_budget=1 << 20) as small:
        s, info = small.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-8, check=False)
        assert info.status == wf.ERR_OOM
    with wf.Context(0) as c:
        s, info = c.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-8)
        assert info.status == wf.OK


def test_serving_admission_under_tight_budget():
    """With room for about two systems at a time, requests queue and are admitted a few at a time,
    and all complete."""
    wf.build()
    w, b, nbar, box, k, p = _serve_inputs(32, 3020)
    one = 32 ** 3 * 8 * 20
    with wf.Context(0, hbm_budget=one) as ctx:
        ids = [ctx.submit(w, nbar, b, box, k, p, tol=1e-8, prec=wf.MIXED) for _ in range(4)]
        outs = []
        for rid in ids:
            s = np.empty(32 ** 3)
            st, info = ctx.poll(rid, timeout_ms=-1, s_out=s)
            assert st == wf.OK
            outs.append(s)
        for s in outs[1:]:
            assert np.array_equal(s, outs[0])


@pytest.mark.parametrize("prec", [wf.FP64, wf.MIXED])
def test_non_finite_input_is_rejected(prec):
    """A NaN in b or w is that system's argument error; batch-mates still solve."""
    pr, w, b, nbar, tab = _solve_inputs("c1", 16)
    bn = b.copy()
    bn[3, 4, 5] = np.nan
    wn = w.copy()
    wn[1, 2, 3] = np.inf
    with wf.Context(0) as c:
        s, info = c.solve(gpu(w), nbar, gpu(bn), pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=prec, check=False)
        assert info.status == wf.ERR_ARG
        probs = [dict(w=gpu(w), nbar=nbar, b=gpu(bn), box=pr.box, pk_k=pr.pk_k, pk_p=pr.pk_p, prec=prec),
                 dict(w=gpu(wn), nbar=nbar, b=gpu(b), box=pr.box, pk_k=pr.pk_k, pk_p=pr.pk_p, prec=prec),
                 dict(w=gpu(w), nbar=nbar, b=gpu(b), box=pr.box, pk_k=pr.pk_k, pk_p=pr.pk_p, prec=prec, tol=1e-8)]
        st, outs, infos = c.solve_batch(probs)
        assert st == wf.ERR_ARG
        assert [i.status for i in infos] == [wf.ERR_ARG, wf.ERR_ARG, wf.OK]
        assert infos[2].rel_residual <= 1e-8
