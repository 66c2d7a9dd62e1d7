"""Write tests/golden/toy_trace.txt from the oracle alone.

The fixture is a regression record of the oracle on the toy workload
(A + B -> C, 1 um cube, 2,500 + 2,500 agents, seed 1): the digest and the
counts vector at a few steps.  It calls nothing but oracle/.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

STEPS = [0, 1, 2, 5, 10, 25, 50, 100, 200]


def main():
    sim = oracle.OracleSim(W.toy(), W.TOY_SEED)
    lines = ["# step digest counts[A,B,C,bound(A+B),next_id]  (oracle, toy workload, seed 1)"]
    t = 0
    for s in STEPS:
        sim.step(s - t)
        t = s
        lines.append("%d %016x %s" % (s, sim.digest(), " ".join(str(int(v)) for v in sim.counts())))
    with open(os.path.join(HERE, "toy_trace.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
