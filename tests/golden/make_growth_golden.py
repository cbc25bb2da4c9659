"""Write the oracle's growth series for the L = 2^14 growth workload.

Workload: L = 16384 periodic lattice, striped start h = (x+y) mod 2, p = 1,
q = 0, selection factor 1/2, Philox seed 7, 10^4 sweeps, W^2 at 40
log-spaced times plus t = 0. Each record holds t, H0 = h(0,0), the exact sums
S1 = sum h and S2 = sum h^2, and W^2; the last line holds the SHA-256 of the
final bond planes in the packed layout (X plane then Y plane, row-major,
little-endian 32-bit words, bit b of word w of row y = bond at x = 32w + b).

Calls only the CPU oracle. Run from the repository root:
    OMP_NUM_THREADS=8 python tests/golden/make_growth_golden.py
(about two hours on eight x86 cores).
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

L, P, Q, SEED, T, NSAMP = 16384, 1.0, 0.0, 7, 10000, 40
OUT = os.path.join(HERE, "growth_L16384_p1_q0_seed7.txt")


def main():
    sim = oracle.Sim(L, P, Q, SEED, s_sel=0.5)
    times = oracle.sample_times(T, NSAMP)
    lines = [
        "# oracle growth series: L=%d p=%g q=%g s_sel=0.5 seed=%d T=%d samples=%d"
        % (L, P, Q, SEED, T, NSAMP),
        "# written by tests/golden/make_growth_golden.py (CPU oracle only)",
        "# columns: t H0 S1 S2 W2",
    ]
    t_start = time.time()
    for t in times:
        if t > sim.t:
            sim.sweep(t - sim.t)
        S1, S2 = sim.sums()
        w2 = sim.width2()
        lines.append("%d %d %d %d %.17g" % (sim.t, sim.H0, S1, S2, w2))
        print(lines[-1], "(%.0fs)" % (time.time() - t_start), flush=True)
    Xw, Yw = sim.packed()
    digest = hashlib.sha256(Xw.tobytes() + Yw.tobytes()).hexdigest()
    lines.append("# final_planes_sha256 %s" % digest)
    with open(OUT + ".tmp", "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()
