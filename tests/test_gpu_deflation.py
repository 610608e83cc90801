"""Deflated inner solves (wf_solve_opts.deflate = K): the mixed-precision solve with each inner CG
preconditioned on the coarse space of the Fourier modes |k| <= K.  Same system, same residual
contract, same solution as the oracle's converged CG (Sec. 3.3.1, Eq. eq:WF) within the mixed
path's 1e-6; fewer iterations; batching and serving keep the result of the solve alone.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0906_3978_gb300 as wf  # noqa: E402

DEV = "cuda:0"


def rl2(a, r):
    a, r = np.asarray(a), np.asarray(r)
    return float(np.linalg.norm(a - r) / np.linalg.norm(r))


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def ctx():
    wf.build()
    c = wf.Context(0)
    yield c
    c.close()


def _inputs(name, n):
    pr = synth.problem(name, n_override=n, cache=False)
    fine = oracle.assign(pr.pos, pr.n, pr.box, pr.scheme, 2)
    nobs = oracle.lowpass(fine, pr.n, 2)
    w = oracle.window(pr.sel, pr.n, pr.box)
    d, b, nbar = oracle.build_noise(nobs, w, pr.n_gal)
    tab = oracle.sinv_table(n, pr.box, pr.pk_k, pr.pk_p)
    return pr, w, b, nbar, tab


@pytest.mark.parametrize("name,n,K", [("c2", 64, 4), ("c2", 64, 12), ("c1", 64, 6), ("c2", 108, 6)])
def test_deflated_mixed_matches_oracle(ctx, name, n, K):
    pr, w, b, nbar, tab = _inputs(name, n)
    ref = oracle.cg(tab, nbar, w, b, tol=1e-12)[0]
    s, info = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-9, prec=wf.MIXED, deflate=K)
    assert info.status == wf.OK and info.rel_residual <= 1e-9
    assert rl2(host(s), ref) <= 1e-6
    s6, info6 = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-6, prec=wf.MIXED, deflate=K)
    assert info6.status == wf.OK
    res = b - oracle.matvec(tab, nbar, w, host(s6))
    assert np.linalg.norm(res) <= 1.0001e-6 * np.linalg.norm(b)


@pytest.mark.parametrize("n,K", [(48, 4), (64, 6), (128, 6)])
def test_fixed_iterations_match_oracle_adef2(ctx, n, K):
    """After k iterations (the start step x_0 = Q b' is the first), the FP32 inner solve of the mixed
    path (one refinement step, s = C y_k) holds the iterate of the oracle's FP64 A-DEF2 CG
    (oracle/coarse.py, numpy FFTs and a dense LU solve of E).  Bound: the FP32 operator's
    4 log2(V) u plus 0.1 kappa(E) u for the FP32 inverse of E (an inverse's forward error grows with
    the condition); kappa(E) is 1.5e3, 3.6e3 and 1.3e4 for these cases, and the measured deviations
    are 0.015-0.034 kappa u (an FP32 emulation on the CPU at 48^3 and 64^3: 0.9e-6 to 3.3e-6).  A
    wrong sign or a transposed coarse block moves the iterates by 1e-2 or more."""
    from oracle.coarse import Problem, adef2
    pr, w, b, nbar, tab = _inputs("c2", n)
    ev = np.linalg.eigvalsh(Problem(tab, nbar, w, b, K).E)
    u = 2.0 ** -24
    bound = 4.0 * 3 * np.log2(n) * u + 0.1 * (ev[-1] / ev[0]) * u
    for k in (1, 2, 3):
        ref = adef2(tab, nbar, w, b, K, tol=1e-15, max_iter=k)[0]
        s, info = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-14, max_iter=k, prec=wf.MIXED,
                            deflate=K, check=False)
        assert info.status == wf.ERR_NOT_CONVERGED and info.iters == k and info.outer_iters == 1
        assert rl2(host(s), ref) <= bound, (k, rl2(host(s), ref), bound)


@pytest.mark.parametrize("n,K", [(128, 8), (192, 10)])
def test_deflation_cuts_iterations(ctx, n, K):
    """At the 512^3 workload's cell size the coarse space removes the slow long-wavelength modes:
    fewer than 0.6 x the iterations of the undeflated mixed solve at the same residual, and a
    solution at least as close to the converged one.  (A relative residual of 1e-6 leaves errors
    of up to ~1e-4 in the weakly constrained directions, so the two 1e-6 solutions are compared
    with the solve converged to 1e-10, not with each other.)"""
    pr = synth.problem("c3", n_override=n, cache=False)
    nobs = ctx.grid_assign(gpu(pr.pos), n, pr.box, pr.scheme, 2)
    w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box, want_d=False)
    s0, i0 = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-6, prec=wf.MIXED)
    s1, i1 = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-6, prec=wf.MIXED, deflate=K)
    assert i0.status == wf.OK and i1.status == wf.OK and i1.rel_residual <= 1e-6
    assert i1.iters < 0.6 * i0.iters, (i1.iters, i0.iters)
    s0, s1 = host(s0).copy(), host(s1).copy()
    ex, ie = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-10, prec=wf.MIXED)
    assert ie.status == wf.OK
    ex = host(ex)
    e0, e1 = rl2(s0, ex), rl2(s1, ex)
    assert e1 <= max(2.0 * e0, 1e-6), (e1, e0)


def test_deflated_batch_equals_individual_solves(ctx):
    """A batch mixing deflated systems (two sizes, several systems per coarse block set-up) with
    undeflated ones gives every system the result and the iteration count it gets alone: a system's
    arithmetic does not depend on its batch-mates."""
    probs, singles = [], []
    for i, (name, n, K) in enumerate([("c2", 64, 4), ("c2", 48, 4), ("c1", 64, 4), ("c2", 64, 0), ("c1", 48, 6),
                                      ("c2", 72, 4)]):
        pr, w, b, nbar, tab = _inputs(name, n)
        probs.append(dict(w=gpu(w), nbar=nbar, b=gpu(b), box=pr.box, pk_k=pr.pk_k, pk_p=pr.pk_p, tol=1e-8,
                          prec=wf.MIXED, deflate=K))
        s, info = ctx.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=wf.MIXED, deflate=K)
        singles.append((host(s).copy(), info.iters))
    st, outs, infos = ctx.solve_batch(probs)
    assert st == wf.OK, [i.status for i in infos]
    for (ref, it), s, info in zip(singles, outs, infos):
        assert info.status == wf.OK and info.rel_residual <= 1e-8
        assert info.iters == it
        assert rl2(host(s), ref) <= 1e-12


def test_deflated_serving_same_as_alone():
    wf.build()
    pr, w, b, nbar, tab = _inputs("c2", 64)
    with wf.Context(0) as c:
        s_alone, info = c.solve(gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=wf.MIXED, deflate=5)
        ref = host(s_alone).copy()
        ids = [c.submit(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-8, prec=wf.MIXED, deflate=d) for d in (5, 0, 5)]
        for rid in ids:
            s = np.empty(pr.n ** 3)
            st, inf = c.poll(rid, timeout_ms=-1, s_out=s)
            assert st == wf.OK and inf.rel_residual <= 1e-8
            assert rl2(s.reshape(ref.shape), ref) <= 1e-6


def test_deflate_argument_errors(ctx):
    pr, w, b, nbar, tab = _inputs("c1", 32)
    args = (gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p)
    for prec, K in [(wf.FP64, 4), (wf.MIXED, 8), (wf.MIXED, 13), (wf.MIXED, -2)]:   # 4 K < n; K <= 12
        s, info = ctx.solve(*args, tol=1e-6, prec=prec, deflate=K, check=False)
        assert info.status == wf.ERR_ARG
    assert "deflate" in wf.lib().wf_last_error().decode()
    s, info = ctx.solve(*args, tol=1e-6, prec=wf.MIXED, deflate=7)
    assert info.status == wf.OK
    # -1 picks the radius by size: none at 32^3 (the plain mixed solve, same iterations), and for
    # FP64 it is no coarse space at all
    s0, i0 = ctx.solve(*args, tol=1e-8, prec=wf.MIXED)
    s1, i1 = ctx.solve(*args, tol=1e-8, prec=wf.MIXED, deflate=-1)
    assert i1.status == wf.OK and i1.iters == i0.iters
    s2, i2 = ctx.solve(*args, tol=1e-8, prec=wf.FP64, deflate=-1)
    assert i2.status == wf.OK


def test_automatic_radius_at_64(ctx):
    """deflate = -1 at 64^3 is the radius-3 coarse space: the same iterations and solution."""
    pr, w, b, nbar, tab = _inputs("c2", 64)
    args = (gpu(w), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p)
    s3, i3 = ctx.solve(*args, tol=1e-8, prec=wf.MIXED, deflate=3)
    sa, ia = ctx.solve(*args, tol=1e-8, prec=wf.MIXED, deflate=-1)
    assert ia.status == wf.OK and ia.iters == i3.iters
    assert rl2(host(sa), host(s3)) <= 1e-12


def _ball_window(n, radius, amp):
    """A window concentrated in a ball: amp inside radius cells of the centre, 1e-9 amp outside."""
    x = np.indices((n, n, n)) - n // 2
    return np.where(np.sqrt((x ** 2).sum(0)) <= radius, amp, 1e-9 * amp)


def test_condition_guard_turns_an_ill_conditioned_coarse_space_off(ctx):
    """Noise weights concentrated in a ball of radius 6 cells at 48^3, coarse radius 4.  At amplitude 1
    the coarse block E has kappa_inf ~ 1e4 and the coarse space halves the iterations (26 for 52).  At
    amplitude 1e3 (kappa_inf 1.5e9 in FP64, far past what a block built and inverted in FP32 holds)
    the guard on ||E||_inf ||E^-1||_inf turns it off for that system: the solve runs as plain CG
    (the undeflated iteration count, plus the start step) and converges to the oracle's solution.
    In a batch each system keeps the decision and the result it gets alone."""
    from oracle.coarse import Problem
    n, K = 48, 4
    pr, w, b, nbar, tab = _inputs("c2", n)
    batch, alone = [], []
    for amp, well in ((1.0, True), (1e3, False)):
        wb = _ball_window(n, 6, amp)
        E = Problem(tab, nbar, wb, b, K).E
        kinf = np.abs(E).sum(1).max() * np.abs(np.linalg.inv(E)).sum(1).max()
        assert (kinf < 1e5) if well else (kinf > 1e9), kinf
        ref = oracle.cg(tab, nbar, wb, b, tol=1e-11)[0]
        args = (gpu(wb), nbar, gpu(b), pr.box, pr.pk_k, pr.pk_p)
        s0, i0 = ctx.solve(*args, tol=1e-9, prec=wf.MIXED)
        s1, i1 = ctx.solve(*args, tol=1e-9, prec=wf.MIXED, deflate=K)
        assert i0.status == wf.OK and i1.status == wf.OK and i1.rel_residual <= 1e-9
        assert rl2(host(s1), ref) <= 1e-6
        if well:
            assert i1.iters < 0.6 * i0.iters, (i1.iters, i0.iters)
        else:
            assert abs(i1.iters - (i0.iters + 1)) <= 0.02 * i0.iters + 2, (i1.iters, i0.iters)
        alone.append((host(s1).copy(), i1.iters))
        batch.append(dict(w=args[0], nbar=nbar, b=args[2], box=pr.box, pk_k=pr.pk_k, pk_p=pr.pk_p, tol=1e-9,
                          prec=wf.MIXED, deflate=K))
    st, outs, infos = ctx.solve_batch(batch[::-1])
    assert st == wf.OK
    for (ref, it), s, info in zip(alone[::-1], outs, infos):
        assert info.status == wf.OK and info.iters == it
        assert rl2(host(s), ref) <= 1e-12
