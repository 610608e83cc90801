"""Run one reconstruction (gridding, window/noise, a fixed number of CG iterations) and print
the per-kernel-class profile.  Small and bounded, for use under a kernel profiler:

    python -m paper_0906_3978_gb300.profile_solve --n 256 --prec mixed --iters 4
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
    a = ap.parse_args()
    wf.build()
    pr = synth.problem("c2", n_override=None if a.n == 256 else a.n, cache=False)
    with wf.Context(0) as ctx:
        ctx.profile(True)
        nobs = ctx.grid_assign(torch.from_numpy(pr.pos).cuda(), pr.n, pr.box, pr.scheme, 2)
        w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, pr.box)
        s, info = ctx.solve(w, nbar, b, pr.box, pr.pk_k, pr.pk_p, tol=1e-12, max_iter=a.iters,
                            prec=wf.MIXED if a.prec == "mixed" else wf.FP64, precond=a.precond, check=False)
        torch.cuda.synchronize()
        p = ctx.profile_read()
    print("n=%d prec=%s iters=%d status=%d launches=%d" % (pr.n, a.prec, info.iters, info.status, p["launches"]))
    for c in sorted(p["classes"], key=lambda c: -c["ms"]):
        print("  %-12s launches %5d  ms %9.3f  GB/s %s" % (c["name"], c["launches"], c["ms"],
                                                           "%.0f" % c["gbs"] if c["gbs"] else "-"))
    return 0


if __name__ == "__main__":
    sys.exit(main())
