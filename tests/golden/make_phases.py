"""Write tests/golden/phases_*.txt: QSP phases fitted by the oracle (oracle/qsvt.fit_phases)
for the odd 1/x target polynomial of oracle/qsvt.inverse_target.  Only oracle/ is used."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import qsvt as Q  # noqa: E402

CASES = [(10.0, 31), (4.0, 9), (1000.0, 13)]

if __name__ == "__main__":
    for kappa, d in CASES:
        target, scale = Q.inverse_target(kappa, d)
        ph = Q.fit_phases(target, d)
        path = os.path.join(HERE, f"phases_k{int(kappa)}_d{d}.txt")
        with open(path, "w") as fh:
            fh.write(f"# QSP phases (reflection convention) for the 1/x target, kappa={kappa}, d={d},\n")
            fh.write(f"# scale={scale!r}; written by tests/golden/make_phases.py from oracle/ only\n")
            for v in ph:
                fh.write(repr(float(v)) + "\n")
        print(path)
