"""Write tests/golden/rho_trace_L64_counts.txt: the cooperator count after each of the 1000 MCS of
the L = 64, r = 4, K = 0.5, p = 0.5, seed 1 workload, computed by the CPU oracle only.

A regression fixture: the oracle's trajectory for this workload is fixed by the paper's rules
(Section III) and the documented random-stream layout, so a later change that moves it, in the
oracle and the library together, shows up against this file. Run from the repository root:
    python tests/golden/make_rho_trace_L64.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1704_08098_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rho_trace_L64_counts.txt")


def main():
    w = inputs.WORKLOADS["rho_trace_L64"]
    o = oracle.Oracle()
    lat = o.init(w["L"], w["seed"], w["p"])
    counts = o.run(lat, w["r"], w["K"], w["seed"], 0, w["n_mcs"])
    with open(OUT, "w") as f:
        f.write(f"# cooperator count after each MCS: L={w['L']} r={w['r']} K={w['K']} p={w['p']} "
                f"seed={w['seed']}, {w['n_mcs']} MCS; written by tests/golden/make_rho_trace_L64.py "
                "from the CPU oracle\n")
        f.write(f"# initial count {int(o.init(w['L'], w['seed'], w['p']).sum())}\n")
        for c in counts:
            f.write(f"{int(c)}\n")


if __name__ == "__main__":
    main()
