"""Writes tests/golden/sqrt_pieces.json: the oracle's fit of the six-piece
rational approximant of sqrt(x) on [0, 1] (Sec. 3.4; the paper's own
coefficients are in its supplement, which is not available).  Calls only
oracle/."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from oracle import tt  # noqa: E402

if __name__ == "__main__":
    table = tt.fit_sqrt_pieces()
    out = {"source": "oracle.tt.fit_sqrt_pieces (Nelder-Mead minimax of the absolute error per piece)",
           "form": "(c0 + c1 x) / (1 + d1 x) on [breaks[k], breaks[k+1])",
           "breaks": list(tt.SQRT_BREAKS), "coeffs": table.tolist()}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "sqrt_pieces.json"), "w") as f:
        json.dump(out, f, indent=1)
