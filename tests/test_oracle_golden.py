"""The oracle reproduces its stored cfg0 record (tests/golden/cfg0_stout.json,
written by tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np

import fieldgen
from oracle import gauge, stout

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cfg0_record():
    rec = json.load(open(os.path.join(HERE, "golden", "cfg0_stout.json")))
    U = fieldgen.haar_su3((4, 4, 4, 4), 0)
    out = stout.stout_smear(U, 0.1, 1, (0, 1, 2, 3))
    assert np.allclose(gauge.plaquette(U), rec["plaquette_before"], rtol=0, atol=1e-14)
    assert np.allclose(gauge.plaquette(out), rec["plaquette_after"], rtol=0, atol=1e-14)
    for s in rec["links_after"]:
        v = out[s["t"], s["z"], s["y"], s["x"], s["mu"], s["i"], s["j"]]
        assert abs(v - (s["re"] + 1j * s["im"])) < 1e-14
    # Haar links: the plaquette before smearing is consistent with zero
    assert abs(rec["plaquette_before"][0]) < 0.05
