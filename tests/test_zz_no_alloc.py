"""wf_build_noise_noalloc -- window, nbar and data without any device allocation.

Callers that cannot let a library call cudaMalloc (a host code owning the GPU through its own
pool at its memory limit, a latency-critical pipeline that must not see cudaMalloc's implicit
synchronisation) use this entry point; it must give the same results as wf_build_noise.
Collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0906_3978_gb300 as wf  # noqa: E402


def _noalloc_fn():
    L = wf.lib()
    f = L.wf_build_noise_noalloc
    f.argtypes = [ctypes.POINTER(wf.Grid), ctypes.POINTER(wf.SelectionC), ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _call_noalloc(f, sel, nobs, n_gal, box):
    n = int(nobs.shape[0])
    w, d, b = torch.empty_like(nobs), torch.empty_like(nobs), torch.empty_like(nobs)
    s, keep = wf.make_selection(sel)
    nb = ctypes.c_double(0.0)
    g = wf.Grid(n, float(box), 1)
    st = f(ctypes.byref(g), ctypes.byref(s), nobs.data_ptr(), int(n_gal), w.data_ptr(), d.data_ptr(), b.data_ptr(),
           ctypes.byref(nb), torch.cuda.current_stream().cuda_stream)
    return st, w, d, b, nb.value


def rl2(a, r):
    return float(torch.linalg.norm(a - r) / torch.linalg.norm(r))


def test_noalloc_matches_build_noise_twice():
    wf.build()
    f = _noalloc_fn()
    dev = torch.device("cuda", 0)
    with wf.Context(0) as ctx:
        # two calls in a row on different problems: the second must not see the first's scratch
        for name, n in [("c2", 64), ("c1", 32)]:
            pr = synth.problem(name, n_override=n, cache=False)
            nobs = ctx.grid_assign(torch.from_numpy(pr.pos).to(dev), pr.n, pr.box, pr.scheme, 2)
            w0, d0, b0, nb0 = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
            st, w1, d1, b1, nb1 = _call_noalloc(f, pr.sel, nobs, pr.n_gal, pr.box)
            torch.cuda.synchronize()
            assert st == wf.OK
            assert abs(nb1 - nb0) <= n ** 3 * 1.2e-16 * nb0
            assert rl2(w1, w0) <= 1e-14
            assert rl2(d1, d0) <= 1e-13
            assert rl2(b1, b0) <= 1e-13


def test_noalloc_rejects_oversized_hole_table():
    wf.build()
    f = _noalloc_fn()
    sel = synth.selection_sdss_like(100.0, 3)
    sel.holes = np.tile(sel.holes[:1], (257, 1))
    nobs = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda:0")
    st = _call_noalloc(f, sel, nobs, 10, 100.0)[0]
    assert st == wf.ERR_ARG
    assert "256" in wf.lib().wf_last_error().decode()
