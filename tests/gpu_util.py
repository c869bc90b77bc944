"""Helpers shared by the GPU tests: move oracle-layout arrays through the C ABI."""
import numpy as np

import paper_1105_2279_gb300 as lq


def upload_links(U, prec):
    """U: oracle link array (Lt,Lz,Ly,Lx,4,3,3) complex128 -> device LINKS field."""
    lt, lz, ly, lx = U.shape[:4]
    g = lq.Geometry((lx, ly, lz, lt))
    return lq.Field.from_host(g, lq.LQ_LINKS, prec, U)


def links_err(a, b):
    """max |a - b| over link elements, and the max relative error over elements with |b| >= 1e-3."""
    d = np.abs(a.astype(np.complex128) - b)
    big = np.abs(b) >= 1e-3
    return float(d.max()), float((d[big] / np.abs(b[big])).max())
