"""Writes the stored expected values under tests/golden/ by calling only the oracle.

Run from the repository root:  python tests/golden/make_golden.py

cfg0_stout.json: the plain-method workload -- 4^4 periodic lattice, Haar SU(3)
links from seed 0, one stout step rho = 0.1 in all four directions (stout
smearing as defined by Morningstar & Peardon 2004, Sec. II); average,
spatial and temporal plaquette before and after, and a few smeared link
elements.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import fieldgen  # noqa: E402
from oracle import gauge, stout  # noqa: E402


def main():
    U = fieldgen.haar_su3((4, 4, 4, 4), 0)
    out = stout.stout_smear(U, 0.1, 1, (0, 1, 2, 3))
    samples = []
    for (t, z, y, x, mu, i, j) in [(0, 0, 0, 0, 0, 0, 0), (1, 2, 3, 0, 1, 2, 1),
                                   (3, 3, 3, 3, 3, 1, 2), (2, 0, 1, 3, 2, 0, 2)]:
        v = out[t, z, y, x, mu, i, j]
        samples.append({"t": t, "z": z, "y": y, "x": x, "mu": mu, "i": i, "j": j,
                        "re": float(v.real), "im": float(v.imag)})
    rec = {
        "workload": "4^4 periodic, Haar SU(3) seed 0, 1 stout step rho=0.1, dirs xyzt",
        "source": "oracle (stout smearing, Morningstar & Peardon 2004 Sec. II-III)",
        "plaquette_before": list(gauge.plaquette(U)),
        "plaquette_after": list(gauge.plaquette(out)),
        "links_after": samples,
    }
    with open(os.path.join(HERE, "cfg0_stout.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
