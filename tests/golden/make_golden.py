"""Writes the stored expected values of tests/golden/ from the oracle alone.

The paper prints no numerical example (its Si walk-through shows commands, not numbers), so the
fixtures here are the oracle's own results on small seeded inputs, kept as text so that a change
of the oracle's arithmetic shows up as a diff, and so that the GPU can be checked against a file.

  sigma_gw_small.txt   Sigma~ (Eqs. sigma_gw, tilde_W_DF2) of the seeded system below, FP64
  ir_nodes_l100.txt    tau nodes of the IR grid with Lambda = 100, eps = 1e-10, beta = 10

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import gw as O  # noqa: E402
from oracle import ir  # noqa: E402
from paper_2406_18479_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SMALL = dict(name="golden", nk3=(2, 1, 1), nao=2, naux=3, ntau=4, nomega=4, beta=5.0, mu=0.0, decay=4.0, seed=11,
             solid=True)


def small_case():
    w = I.Workload(**SMALL)
    return w, I.make_inputs(w)


def main():
    w, (h, v, g) = small_case()
    sig = O.sigma_eval(v, g, w.nk3, w.beta, 2.0)["Sig"]
    with open(os.path.join(HERE, "sigma_gw_small.txt"), "w") as f:
        f.write("# Sigma~[k][t][i][j] (re im) of the seeded 2x1x1, nao 2, naux 3, ntau 4, beta 5 system; "
                "oracle/gw.py sigma_eval; written by tests/golden/make_golden.py\n")
        for x in sig.ravel():
            f.write(f"{x.real:.17e} {x.imag:.17e}\n")
    tau, _, _, _ = ir.ir_grid(10.0, 100.0, 1e-10, 1)
    with open(os.path.join(HERE, "ir_nodes_l100.txt"), "w") as f:
        f.write("# tau nodes of the IR grid, Lambda = 100, eps = 1e-10, beta = 10; oracle/ir.py; "
                "written by tests/golden/make_golden.py\n")
        for t in tau:
            f.write(f"{t:.17e}\n")


if __name__ == "__main__":
    main()
