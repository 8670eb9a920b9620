"""Writes minimax_sign.json: composite minimax sign stages computed by the
oracle's Remez routine (oracle/sign.py), for the sensitivities of the paper's
Table 2 (alpha 8 with three degree-15 stages; alpha 16 with six, one more than
Table 2's five because the paper's jointly optimised LLNK20 composition is not
printed).  The GPU tests and bench.py read the file; only this script calls
the oracle.  Run: python tests/golden/make_minimax_sign.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import sign  # noqa: E402


def main():
    out = {}
    for name, alpha, degs in [("alpha8_15x3", 8, [15, 15, 15]), ("alpha16_15x6", 16, [15] * 6)]:
        stages, err = sign.composite_minimax(alpha, degs)
        out[name] = {"alpha": alpha, "degrees": degs, "stages": stages, "error": err, "beta": sign.beta(err)}
        print(name, "error", err, "beta", sign.beta(err))
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "minimax_sign.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
