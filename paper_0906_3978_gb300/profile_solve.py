"""Run one reconstruction (gridding, window/noise, a fixed number of CG iterations), or one
projection of a sky map into the 3D mask, and print the per-kernel-class profile.  Small and
bounded, for use under a kernel profiler:

    python -m paper_0906_3978_gb300.profile_solve --n 256 --prec mixed --iters 4
    python -m paper_0906_3978_gb300.profile_solve --n 256 --what mask

--tune times the launch variants first (wf_autotune) and prints the report; --variant
xinv/f32/256=1 forces a variant of a pass (the context's tuning table).  A whole solve of the
512^3 workload with the coarse-space inner solves:

    python -m paper_0906_3978_gb300.profile_solve --problem c3 --n 512 --tol 1e-6 --iters 5000 --deflate 10
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch
    import paper_0906_3978_gb300 as wf
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--precond", type=int, default=1)
    ap.add_argument("--what", choices=["solve", "mask"], default="solve")
    ap.add_argument("--tune", action="store_true")
    ap.add_argument("--variant", action="append", default=[])
    ap.add_argument("--problem", choices=["c2", "c3"], default="c2")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--deflate", type=int, default=0)
    a = ap.parse_args()
    wf.build()
    full = 256 if a.problem == "c2" else 512
    pr = synth.problem(a.problem, n_override=None if a.n == full else a.n, cache=False)
    if a.what == "mask":
        return mask(wf, pr)
    with wf.Context(0) as ctx:
        prec = wf.MIXED if a.prec == "mixed" else wf.FP64
        if a.tune:
            for p in ctx.autotune(pr.n, prec):
                print("tune %-14s chosen %-16s %s" % (p["pass"], p["chosen"],
                                                       " ".join("%s=%.4f" % (v["name"], v["ms"]) for v in p["variants"])))
        for v in a.variant:
            key, idx = v.split("=")
            ctx.tune_set({key: int(idx)})
        ctx.profile(True)
        nobs = ctx.grid_assign(torch.from_numpy(pr.pos).cuda(), pr.n, pr.box, pr.scheme, 2)
        w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
        s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=a.tol, max_iter=a.iters,
                            prec=wf.MIXED if a.prec == "mixed" else wf.FP64, precond=a.precond, check=False,
                            deflate=a.deflate)
        torch.cuda.synchronize()
        p = ctx.profile_read()
    print("n=%d prec=%s iters=%d status=%d launches=%d" % (pr.n, a.prec, info.iters, info.status, p["launches"]))
    for c in sorted(p["classes"], key=lambda c: -c["ms"]):
        print("  %-12s launches %5d  ms %9.3f  GB/s %s" % (c["name"], c["launches"], c["ms"],
                                                           "%.0f" % c["gbs"] if c["gbs"] else "-"))
    return 0


def mask(wf, pr):
    """The sky map of 2N x N pixels (completeness 0.9 in the survey cone, 0 elsewhere) and the radial
    law every 0.25 H out to N H, projected once: 8 N^3 ray samples."""
    import math
    import numpy as np
    import torch
    n, box = pr.n, pr.box
    na, nd, nr = 2 * n, n, 4 * n
    dr = 0.25 * box / n
    al = (np.arange(na) + 0.5) * 2 * math.pi / na
    de = -math.pi / 2 + (np.arange(nd) + 0.5) * math.pi / nd
    ax = np.asarray(pr.sel.axis, dtype=np.float64)
    dot = (np.cos(de)[:, None] * np.cos(al)[None, :] * ax[0] + np.cos(de)[:, None] * np.sin(al)[None, :] * ax[1]
           + np.sin(de)[:, None] * ax[2])
    sky = torch.from_numpy(np.where(dot >= math.cos(pr.sel.half_angle), 0.9, 0.0)).cuda()
    wr = np.ones(nr)
    with wf.Context(0) as ctx:
        ctx.profile(True)
        ctx.project_mask(sky, n, box, 0.0, 2 * math.pi / na, -math.pi / 2, math.pi / nd, pr.sel.observer, dr, wr)
        torch.cuda.synchronize()
        p = ctx.profile_read()
    print("n=%d mask samples=%d launches=%d" % (n, na * nd * nr, p["launches"]))
    for c in sorted(p["classes"], key=lambda c: -c["ms"]):
        print("  %-12s launches %5d  ms %9.3f" % (c["name"], c["launches"], c["ms"]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
