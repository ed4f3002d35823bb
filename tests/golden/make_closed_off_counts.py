"""Write closed_off_oracle_counts.txt: the oracle's #Matvec for the closed-off problem (Sec. 2.1,
k = 40) at the grid sizes of Table 2, in the paper's configuration (17-node coarsening rule,
left-preconditioned full GMRES with the preconditioned stopping rule, IDR(4) on the true
residual with the seeded shadow space).  It calls only the oracle and the input generators; at
129^3 and 193^3 nodes the oracle needs tens of minutes and about 20 GB, so the counts are stored
here rather than recomputed by the tests.

    python tests/golden/make_closed_off_counts.py [n ...]     (default: 128 192; other sizes kept)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2308_06085_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_off_oracle_counts.txt")


def counts(n, k=40.0):
    shape = I.unknown_shape(n, oracle.DIRICHLET)
    o = oracle.Solver(n, 1.0 / n, oracle.DIRICHLET, np.full(shape, k * k), coarsest_n=I.coarsest_by_node_rule(n))
    b = oracle.rhs_closed_off(n, k)
    # full GMRES: the paper's counts are 137-146, so 150 vectors are never restarted (at 257^3
    # nodes the basis alone takes 40 GB)
    g = o.gmres(b, restart=150, tol=1e-6, max_iter=150, left=True)
    r = o.idrs(b, I.shadow_space(shape, 4), tol=1e-6, max_iter=2000)
    assert g["status"] == 0 and r["status"] == 0
    return g["iters"], r["iters"]


def main(sizes):
    rows = {}
    if os.path.exists(OUT):  # keep the sizes not recomputed
        with open(OUT) as f:
            for ln in f:
                if ln.strip() and not ln.startswith("#"):
                    rows[int(ln.split()[0])] = ln.strip()
    for n in sizes:
        t = time.time()
        g, r = counts(n)
        rows[n + 1] = f"{n + 1} {g} {r}"
        print(f"n = {n}: GMRES (left) {g}, IDR(4) {r}, {time.time() - t:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("# Oracle #Matvec for the closed-off problem, k = 40, in the paper's configuration (written by\n"
                "# make_closed_off_counts.py, which calls only the oracle).  Columns: nodes per side,\n"
                "# left-preconditioned GMRES, IDR(4) with inputs.shadow_space(shape, 4).\n")
        f.write("\n".join(rows[k] for k in sorted(rows)) + "\n")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [128, 192])
