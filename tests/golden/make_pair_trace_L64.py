"""Write tests/golden/pair_trace_L64_counts.txt: the cooperator count after each of 600 MCS of the
pairwise game (Section VI) on L = 64 with the weak prisoner's dilemma (R, S, T, P) = (1, 0, 1.04, 0),
K = 0.1, p = 0.5, seed 1, computed by the CPU oracle only (a regression fixture like
rho_trace_L64_counts.txt). Run from the repository root:
    python tests/golden/make_pair_trace_L64.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pair_trace_L64_counts.txt")
L, PAY, K, P, SEED, N_MCS = 64, (1.0, 0.0, 1.04, 0.0), 0.1, 0.5, 1, 600


def main():
    o = oracle.Oracle()
    lat = o.init(L, SEED, P)
    counts = o.pair_run(lat, PAY, K, SEED, 0, N_MCS)
    with open(OUT, "w") as f:
        f.write(f"# cooperator count after each MCS: pairwise game L={L} (R,S,T,P)={PAY} K={K} p={P} "
                f"seed={SEED}, {N_MCS} MCS; written by tests/golden/make_pair_trace_L64.py from the CPU "
                "oracle\n")
        for c in counts:
            f.write(f"{int(c)}\n")


if __name__ == "__main__":
    main()
