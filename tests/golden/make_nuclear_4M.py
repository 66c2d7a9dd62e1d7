"""Write tests/golden/nuclear_4M_trace.txt from the oracle alone.

The two-compartment workload at its full size (12 um spherical cell, 5 um
nucleus, 4,000,000 agents, seed 42) stepped by the serial oracle for 50
steps: the digest after every step and the counts vector every 10 steps.
The oracle needs about 20 s per step of this model, so the GPU test reads
this record instead of running it.  It calls nothing but oracle/ and the
workload description; run it again after any change to the oracle or to
the workload (about 20 minutes on one core).
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

STEPS = 50


def main():
    t0 = time.time()
    sim = oracle.OracleSim(W.nuclear(4_000_000), W.NUCLEAR_SEED)
    lines = ["# step digest [counts every 10 steps]  (oracle, two-compartment workload, 4M agents, seed 42)",
             "0 %016x %s" % (sim.digest(), " ".join(str(int(v)) for v in sim.counts()))]
    for s in range(1, STEPS + 1):
        sim.step(1)
        extra = " " + " ".join(str(int(v)) for v in sim.counts()) if s % 10 == 0 else ""
        lines.append("%d %016x%s" % (s, sim.digest(), extra))
        print(f"step {s} ({time.time() - t0:.0f} s)", flush=True)
    sim.close()
    with open(os.path.join(HERE, "nuclear_4M_trace.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
