"""Writes riemann_mix_oracle.txt: for every 1D two-state Riemann request of
the seeded serving mix (seed 0, 1000 requests), whether
the FP64 oracle's state after the requested steps is non-physical (rho <= 0
or not finite) -- the requests on which the scheme itself, at the mix's
Riemann parameters (tau 0.55, T unit 0.15, fixed-state reservoirs), leaves
the physical range whatever the precision.  Calls only oracle/ and the
seeded input generators; several minutes on 8 cores."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2501_00620_gb300 import workloads as W  # noqa: E402


def main():
    reqs = [r for r in W.serving_requests() if r["dim"] == 1 and r["kind"] == "riemann"]
    lines = ["# id nx steps fatal  (1D Riemann requests of the seeded serving mix; FP64 oracle)"]
    for r in sorted(reqs, key=lambda r: r["id"]):
        rho, u, T = W.request_fields(r)
        tau, T0, thermal, bc = W.request_params(r)
        o = oracle.Sim(1, r["nx"], tau=tau, T0=T0, thermal=thermal, bc=bc)
        o.init(rho, u, T)
        o.step(r["steps"])
        orho, _, oT = o.moments()
        fatal = not (np.isfinite(orho).all() and np.isfinite(oT).all() and (orho > 0).all())
        lines.append("%d %d %d %d" % (r["id"], r["nx"], r["steps"], int(fatal)))
    with open(os.path.join(HERE, "riemann_mix_oracle.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
