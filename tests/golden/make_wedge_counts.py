"""Write wedge_oracle_counts.txt: the oracle's #Matvec for the wedge workloads solved by
right-preconditioned GMRES(30) with one CSLP V-cycle (beta2 = -0.5) to a true relative
residual of 1e-6 from x0 = 0, point source at the top-face centre.  It calls only the oracle
and the input generators.  At n = 256 (257^3 unknowns) one oracle solve takes minutes and
about 9 GB, so the count is stored here: the CPU reference arm of bench.py scales its bounded
per-step sample by it, and a CPU test checks the file's form.

    python tests/golden/make_wedge_counts.py [workload:n ...]   (default: wedge:128 mixed:256)
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2308_06085_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wedge_oracle_counts.txt")


def count(name, n):
    w = I.workload(name, n)
    o = oracle.Solver(w["n"], w["h"], oracle.SOMMERFELD, w["k2"])
    b = oracle.rhs_point(o.shape, oracle.SOMMERFELD, w["h"], w["sources"])
    r = o.gmres(b, restart=30, tol=1e-6, max_iter=3000)
    assert r["status"] == 0
    return r["iters"], r["relres"]


def main(items):
    rows = {}
    if os.path.exists(OUT):  # keep the rows not recomputed
        with open(OUT) as f:
            for ln in f:
                if ln.strip() and not ln.startswith("#"):
                    rows[tuple(ln.split()[:2])] = ln.strip()
    for it in items:
        name, n = it.split(":")
        t = time.time()
        iters, relres = count(name, int(n))
        rows[(name, n)] = f"{name} {n} {iters}"
        print(f"{name} n = {n}: GMRES(30) {iters} (relres {relres:.3e}), {time.time() - t:.0f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("# Oracle #Matvec of right-preconditioned GMRES(30) + one CSLP V-cycle (beta2 = -0.5) to a true\n"
                "# relative residual of 1e-6 on the wedge workloads (inputs.workload), written by\n"
                "# make_wedge_counts.py, which calls only the oracle.  Columns: workload, n, #Matvec.\n")
        f.write("\n".join(rows[k] for k in sorted(rows)) + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["wedge:128", "mixed:256"])
