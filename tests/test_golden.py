"""The oracle reproduces its stored regression values (no GPU)."""
import json
import os

import oracle
from paper_1609_08094_gb300 import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_regression_values(oracle_lib):
    doc = json.load(open(os.path.join(HERE, "oracle_energies.json")))
    for c in doc["cases"]:
        inst = synth.make_instance(c["o"], c["v"], c["naux"], c["seed"])
        e4, e5, e = oracle.energy(inst)
        assert abs(e - c["E"]) <= 1e-11 * abs(c["E"])
        assert abs(e4 - c["E4"]) <= 1e-11 * abs(c["E4"])
        assert abs(e5 - c["E5"]) <= 1e-9 * abs(c["E5"])
