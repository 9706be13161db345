"""Writes oracle_energies.json: oracle regression values for fixed seeds.

The paper prints no value that can pin this method on synthetic inputs (its
Table 1 needs LSDalton HF/CCSD data and its figures carry no numbers), so the
stored values come from the oracle alone; the oracle itself is pinned by
tests/test_oracle_pins.py.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1609_08094_gb300 import synth  # noqa: E402

CASES = [(4, 20, 72, 1), (3, 7, None, 5), (5, 13, None, 9), (2, 33, None, 3)]


def main():
    out = []
    for o, v, naux, seed in CASES:
        inst = synth.make_instance(o, v, naux, seed)
        e4, e5, e = oracle.energy(inst)
        out.append({"o": o, "v": v, "naux": inst.naux, "seed": seed,
                    "E4": e4, "E5": e5, "E": e})
    doc = {"source": "oracle (tests/golden/make_golden.py); the paper prints no "
                     "usable worked example for synthetic inputs",
           "cases": out}
    with open(os.path.join(HERE, "oracle_energies.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
