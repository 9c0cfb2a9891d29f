"""Writes tests/golden/helmholtz2d_n1024_p4.json from the CPU oracle only.

The paper prints no worked example (its Tables 2-3 need matrices that are not
available), so the stored values here are the oracle's own recursive residual
histories on the seeded 32x32 2D Helmholtz problem (Sec. 3 setting: X0 = 0,
tol 1e-10, stopping rule ||xi_m||_F/||B||_F of Algorithms 2-3).  They serve as a
regression fixture for the oracle and as stored expected values for the GPU tests.

With --full3d it also runs the oracle's full bl_cocr_rq solve of the 64^3 Helmholtz
problem (n = 262,144, p = 16, tol 1e-10; several minutes on a CPU) and writes
tests/golden/helmholtz3d_n262144_p16.json (status, iteration count, true relative
residual and the whole recursive history).

With --quad3d it runs the first 20 iterations of bl_cocr_rq on the same 64^3 problem twice
with oracle/blcoc_oracle_xp.py, in complex128 and in numpy.clongdouble (80-bit extended on
x86, binary128 on aarch64; tens of minutes), and writes
tests/golden/helmholtz3d_n262144_p16_extended.json: both histories and the FP64 run's
relative deviation from the extended one at every m (the FP64 rounding floor of a
residual-history comparison on this problem).

Run:  python tests/golden/make_golden.py [--full3d] [--quad3d]
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.blcoc_oracle as O                      # noqa: E402
from paper_1601_05362_gb300 import problems as P      # noqa: E402


def main():
    out = {"source": "oracle/blcoc_oracle.py (Algorithms 2-3, Sec. 2.2)", "problem": None, "runs": {}}
    for method, f in (("cocg_rq", O.bl_cocg_rq), ("cocr_rq", O.bl_cocr_rq)):
        pr = P.helmholtz2d_n1024_p4(method)
        A = pr.A.to_scipy()
        r = f(A, pr.B, tol=pr.tol, maxit=pr.maxit)
        out["problem"] = pr.name
        out["runs"][method] = {"status": r.status, "iters": r.iters, "hist": r.hist,
                               "trr": O.true_relres(A, pr.B, r.X)}
    with open(os.path.join(HERE, "helmholtz2d_n1024_p4.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def full3d():
    pr = P.helmholtz3d_n262144_p16("cocr_rq")
    A = pr.A.to_scipy()
    r = O.bl_cocr_rq(A, pr.B, tol=pr.tol, maxit=2000)
    out = {"source": "oracle/blcoc_oracle.py bl_cocr_rq (Algorithm 3, Sec. 2.2)", "problem": pr.name,
           "status": r.status, "iters": r.iters, "trr": O.true_relres(A, pr.B, r.X), "hist": r.hist}
    with open(os.path.join(HERE, "helmholtz3d_n262144_p16.json"), "w") as fh:
        json.dump(out, fh, indent=0)


def quad3d(iters=20):
    import platform

    import numpy as np
    import oracle.blcoc_oracle_xp as XP
    pr = P.helmholtz3d_n262144_p16("cocr_rq")
    h64, _, _ = XP.bl_cocr_rq_xp(pr.A, pr.B, iters, np.complex128)
    hx, _, _ = XP.bl_cocr_rq_xp(pr.A, pr.B, iters, XP.EXTENDED)
    hx = [float(v) for v in hx]
    dev = [abs(a - b) / b for a, b in zip(h64, hx)]
    out = {"source": "oracle/blcoc_oracle_xp.py bl_cocr_rq_xp (Algorithm 3, Sec. 2.2)", "problem": pr.name,
           "iters": iters, "extended": f"numpy.clongdouble on {platform.machine()}, eps "
                                       f"{float(np.finfo(np.longdouble).eps):.3g}",
           "hist_fp64": [float(v) for v in h64], "hist_extended": hx, "fp64_rel_dev": dev}
    with open(os.path.join(HERE, "helmholtz3d_n262144_p16_extended.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    if "--quad3d" not in sys.argv or "--full3d" in sys.argv:
        main()
    if "--full3d" in sys.argv:
        full3d()
    if "--quad3d" in sys.argv:
        quad3d()
