"""Writes adjoint_cfg5_16cube_200steps.txt: J and the exact dJ/dI_k of the
16^3 adjoint workload (4 x 4 heater patches, walls, 200 steps: the 16^3
instance of the adjoint workload) from the FP64 oracle by complex-step
differentiation (one complex run per patch; about 7 minutes).  Calls only
oracle/ and the seeded workload definitions.

    python tests/golden/make_adjoint_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import complex_step as cs  # noqa: E402

STEPS = 200


def main():
    w = W.config5(n=16)
    J, g = cs.capture_gradient(w, STEPS)
    assert w.steps == STEPS
    path = os.path.join(HERE, "adjoint_cfg5_16cube_200steps.txt")
    with open(path, "w") as fh:
        fh.write("# 16^3 adjoint workload (workloads.config5(n=16)), 200 steps, FP64 oracle,\n")
        fh.write("# complex-step derivatives (oracle/complex_step.py; h = 1e-30).\n")
        fh.write("# line 1: J; lines 2-17: dJ/dI_k, k = 0..15\n")
        fh.write(f"{J:.17e}\n")
        for v in g:
            fh.write(f"{v:.17e}\n")
    print(path)


if __name__ == "__main__":
    main()
