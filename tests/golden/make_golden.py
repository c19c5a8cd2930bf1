"""Write tests/golden/config_counts.txt: exact triangle counts of the seeded
parity workloads, computed by the CPU oracle alone (graphgen inputs + oracle).

Run from the repository root:  python tests/golden/make_golden.py [names...]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = {
    "rmat_s14_ef16_seed1": graphgen.rmat_s14,
    "rmat_s23_ef16_seed2": graphgen.rmat_s23,
}
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config_counts.txt")


def main(names):
    rows = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                k, *vals = line.split()
                rows[k] = vals
    for name in names:
        t0 = time.time()
        n, rp, ci = WORKLOADS[name]()
        pr = oracle.prepare(n, rp, ci)
        T = oracle.tc_hmap(n, pr["rowptr"], pr["colidx"])
        wf = oracle.work_figures(n, pr["rowptr"], pr["colidx"])
        rows[name] = [str(n), str(pr["m"]), str(T), str(wf["wedges"]), str(wf["wmin"])]
        print(name, rows[name], f"{time.time() - t0:.1f}s", flush=True)
    with open(OUT, "w") as f:
        f.write("# Exact counts of the seeded workloads, written by tests/golden/make_golden.py\n")
        f.write("# from graphgen inputs and the CPU oracle only (Alg. 3 over the oriented CSR).\n")
        f.write("# name n m triangles wedges(sum d+(v) over edges) wmin_bytes\n")
        for k in sorted(rows):
            f.write(" ".join([k] + rows[k]) + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or sorted(WORKLOADS))
