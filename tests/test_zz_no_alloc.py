"""wf_build_noise_noalloc -- window, nbar and data without any device allocation.

Callers that cannot let a library call cudaMalloc (a host code owning the GPU through its own
pool at its memory limit, a latency-critical pipeline that must not see cudaMalloc's implicit
synchronisation) use this entry point.  It must give the results of the oracle's window and
noise step (Sec. 3.1.3, 3.2) and of wf_build_noise, leave the device's free memory unchanged,
and hold the largest hole table its fixed scratch allows.  Collected last so that a failure here
leaves every other test already run.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0906_3978_gb300 as wf  # noqa: E402

MAX_HOLES = 256


def _noalloc_fn():
    L = wf.lib()
    f = L.wf_build_noise_noalloc
    f.argtypes = [ctypes.POINTER(wf.Grid), ctypes.POINTER(wf.SelectionC), ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _call_noalloc(f, sel, nobs, n_gal, box, out=None):
    n = int(nobs.shape[0])
    w, d, b = out if out is not None else (torch.empty_like(nobs), torch.empty_like(nobs), torch.empty_like(nobs))
    s, keep = wf.make_selection(sel)
    nb = ctypes.c_double(0.0)
    g = wf.Grid(n, float(box), 1)
    st = f(ctypes.byref(g), ctypes.byref(s), nobs.data_ptr(), int(n_gal), w.data_ptr(), d.data_ptr(), b.data_ptr(),
           ctypes.byref(nb), torch.cuda.current_stream().cuda_stream)
    return st, w, d, b, nb.value


def rl2(a, r):
    a, r = np.asarray(a), np.asarray(r)
    return float(np.linalg.norm(a - r) / np.linalg.norm(r))


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _many_holes(box, seed):
    """An SDSS-like selection with exactly MAX_HOLES caps of 1 degree inside its 30-degree cone."""
    sel = synth.selection_sdss_like(box, seed)
    rng = np.random.default_rng(seed)
    holes = synth.random_holes(sel.axis, sel.half_angle, math.radians(1.0), 0.35, rng)
    assert holes.shape[0] >= MAX_HOLES
    sel.holes = np.ascontiguousarray(holes[:MAX_HOLES])
    return sel


def _check_against_oracle(pr, sel, nobs_h, w, d, b, nbar):
    """The window and noise step against the oracle (Sec. 3.1.3, 3.2): identical membership, w to
    1e-14, d and b to 1e-13, nbar to the oracle's sequential-sum rounding (V - 1) 2^-53."""
    n = pr.n
    w_o = oracle.window(sel, n, pr.box)
    d_o, b_o, nbar_o = oracle.build_noise(nobs_h, w_o, pr.n_gal)
    assert abs(nbar - nbar_o) <= n ** 3 * 1.2e-16 * nbar_o
    assert np.array_equal(w > 0, w_o > 0)
    assert rl2(w, w_o) <= 1e-14
    assert rl2(d, d_o) <= 1e-13
    assert rl2(b, b_o) <= 1e-13


def test_noalloc_matches_oracle_and_build_noise_twice():
    wf.build()
    f = _noalloc_fn()
    dev = torch.device("cuda", 0)
    with wf.Context(0) as ctx:
        # two calls in a row on different problems (the second with the largest hole table): the
        # second must not see the first's scratch
        for name, n, many in [("c2", 64, False), ("c1", 32, True)]:
            pr = synth.problem(name, n_override=n, cache=False)
            sel = _many_holes(pr.box, 11) if many else pr.sel
            nobs = ctx.grid_assign(torch.from_numpy(pr.pos).to(dev), pr.n, pr.box, pr.scheme, 2)
            w0, d0, b0, nb0 = ctx.build_noise(sel, nobs, pr.n_gal, pr.box)
            st, w1, d1, b1, nb1 = _call_noalloc(f, sel, nobs, pr.n_gal, pr.box)
            assert st == wf.OK
            w1h, d1h, b1h = _host(w1), _host(d1), _host(b1)
            _check_against_oracle(pr, sel, _host(nobs), w1h, d1h, b1h, nb1)
            # and the same as the allocating entry point
            assert abs(nb1 - nb0) <= n ** 3 * 1.2e-16 * nb0
            assert rl2(w1h, _host(w0)) <= 1e-14
            assert rl2(d1h, _host(d0)) <= 1e-13
            assert rl2(b1h, _host(b0)) <= 1e-13


def test_noalloc_leaves_free_device_memory_unchanged():
    """After a first call (which looks up the scratch address), a second call with every buffer
    already allocated leaves cudaMemGetInfo's free bytes exactly as they were."""
    wf.build()
    f = _noalloc_fn()
    pr = synth.problem("c2", n_override=48, cache=False)
    sel = _many_holes(pr.box, 12)
    n = pr.n
    fine = oracle.assign(pr.pos, n, pr.box, pr.scheme, 2)
    nobs_h = oracle.lowpass(fine, n, 2)
    nobs = torch.from_numpy(nobs_h).to("cuda:0")
    out = tuple(torch.empty_like(nobs) for _ in range(3))
    st = _call_noalloc(f, sel, nobs, pr.n_gal, pr.box, out=out)[0]
    assert st == wf.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    st, w, d, b, nbar = _call_noalloc(f, sel, nobs, pr.n_gal, pr.box, out=out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(0)[0]
    assert st == wf.OK
    assert free1 == free0
    _check_against_oracle(pr, sel, nobs_h, _host(w), _host(d), _host(b), nbar)


def test_noalloc_rejects_oversized_hole_table():
    wf.build()
    f = _noalloc_fn()
    sel = synth.selection_sdss_like(100.0, 3)
    sel.holes = np.tile(sel.holes[:1], (MAX_HOLES + 1, 1))
    nobs = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda:0")
    st = _call_noalloc(f, sel, nobs, 10, 100.0)[0]
    assert st == wf.ERR_ARG
    assert "256" in wf.lib().wf_last_error().decode()
