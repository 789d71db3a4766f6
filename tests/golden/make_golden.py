"""Write tests/golden/small_minimiser.txt: the exact minimiser of Eq. 6 (FP64 oracle:
coordinate descent + Newton polish, KKT-certified) for the first 8 pixels of the small
stack (N=25, L=200 on [-100, 100] m, 10 dB, seed 1), as support and complex values.

The paper prints no numeric example, so these values come from the oracle alone; the
file lets GPU tests compare against stored answers and lets the CPU tests notice any
change in what the oracle computes.  Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1805_01759_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_minimiser.txt")


def main() -> None:
    st = synth.workload_small(P=8, seed=1)
    A = oracle.operator(st.geom)
    r = oracle.minimise_batch(A, st.g, st.lam)
    assert np.all(r["flags"] == 0), r["flags"]
    lines = ["# exact minimiser of Eq. 6 for pixels 0..7 of the small stack (N=25, L=200, seed 1)",
             "# written by tests/golden/make_golden.py from the FP64 oracle (no numbers are printed in the paper)",
             f"# lambda {st.lam!r}",
             "# pixel l re im   (one line per nonzero; a pixel with x* = 0 has the line 'pixel zero')"]
    for p in range(st.g.shape[0]):
        nz = np.nonzero(r["x"][p])[0]
        if nz.size == 0:
            lines.append(f"{p} zero")
        for l in nz:
            v = r["x"][p, l]
            lines.append(f"{p} {l} {float(v.real)!r} {float(v.imag)!r}")
    open(OUT, "w").write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
