"""Writes mrf512_lb_star.txt: the FP64 oracle's bound trajectory on the
512x512x4 MRF grid (seed 1, Potts U(0,2)) over 2,000 iterations of Alg. 1
(omega = 0.5), the LB* against which bench.py reports the GPU's iterations and
time to come within 1e-4 (relative) of it.  Calls only the oracle and the
seeded generator; single-threaded, about 20 minutes.

    python tests/golden/make_mrf512_lb_star.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ilpgen  # noqa: E402
import oracle  # noqa: E402

ITERS = 2000


def main():
    g = ilpgen.mrf_grid(512, 512, 4, 1, potts_max=2.0)
    orc = oracle.Problem.from_ilp(g)
    t0 = time.perf_counter()
    tr = orc.iterate(ITERS, 0.5)
    dt = time.perf_counter() - t0
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mrf512_lb_star.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle, Alg. 1 with omega = 0.5, on ilpgen.mrf_grid(512, 512, 4, 1, potts_max=2.0)\n")
        f.write(f"# written by tests/golden/make_mrf512_lb_star.py ({dt:.0f} s single-threaded)\n")
        f.write(f"iterations: {ITERS}\n")
        f.write(f"lb_star: {float(tr[-1])!r}\n")
        for k in (100, 200, 500, 1000, 1500, 2000):
            f.write(f"lb_after_{k}: {float(tr[k - 1])!r}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
