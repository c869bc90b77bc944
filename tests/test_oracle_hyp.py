"""Pins of the HYP oracle (oracle/hyp.py): unit fields and zero weights are
fixed points, with a2 = a3 = 0 it is one APE step of weight a1 (APE is pinned
on its own), it is gauge covariant and translation invariant, and a smeared
link depends exactly on the links of the hypercubes that contain it."""
import numpy as np
import pytest

import fieldgen
from oracle import ape, gauge, hyp, lattice
from oracle.su3 import unitarity_violation

ALL = (0, 1, 2, 3)
W = (0.75, 0.6, 0.3)


def test_unit_field_and_zero_weights():
    dims = (3, 3, 2, 3)
    one = fieldgen.unit_links(dims)
    assert np.max(np.abs(hyp.hyp_smear(one, *W, 2) - one)) < 1e-15
    U = fieldgen.haar_su3(dims, 60)
    assert np.max(np.abs(hyp.hyp_step(U, 0.0, 0.0, 0.0) - U)) < 1e-14


def test_outer_level_alone_is_ape():
    """Equal up to rounding: the staples are associated differently, and the
    projection amplifies rounding by the condition number of V (large on
    Haar-random fields, where V = 0.3 U + 0.7/6 C can come near singular)."""
    U = fieldgen.near_identity_su3((3, 4, 3, 3), 61)
    assert np.max(np.abs(hyp.hyp_step(U, 0.7, 0.0, 0.0) - ape.ape_step(U, 0.7, ALL))) < 1e-14
    H = fieldgen.haar_su3((3, 4, 3, 3), 61)
    assert np.max(np.abs(hyp.hyp_step(H, 0.7, 0.0, 0.0) - ape.ape_step(H, 0.7, ALL))) < 1e-11


def test_gauge_covariance_and_su3():
    dims = (3, 3, 4, 3)
    U = fieldgen.near_identity_su3(dims, 62)
    g = fieldgen.gauge_field_g(dims, 63)
    a = hyp.hyp_step(gauge.gauge_transform(U, g), *W)
    b = gauge.gauge_transform(hyp.hyp_step(U, *W), g)
    assert np.max(np.abs(a - b)) < 1e-13
    du, dd = unitarity_violation(b)
    assert du < 1e-13 and dd < 1e-13


def test_translation_invariance():
    dims = (4, 3, 3, 5)
    U = fieldgen.haar_su3(dims, 64)
    off = (2, 1, 0, 3)
    a = hyp.hyp_step(lattice.translate(U, off), *W)
    b = lattice.translate(hyp.hyp_step(U, *W), off)
    assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("link,inside", [
    ((1, 0, 0, 0, 2), True),     # U_z(x + e_x): in a hypercube attached to the link
    ((0, 1, 1, 0, 0), True),     # U_x(x + e_y + e_z): far corner of an attached hypercube
    ((0, -1, 0, -1, 1), True),   # U_y(x - e_y - e_t): backward corner
    ((1, 1, 1, 0, 2), False),    # U_z(x + e_x + e_y + e_z) reaches z + 2: outside
    ((0, 2, 0, 0, 0), False),    # U_x(x + 2 e_y): two steps across
    ((3, 0, 0, 0, 1), False),
])
def test_hypercube_locality(link, inside):
    """V_x(0) (mu = 0 at the origin) against one perturbed link (dx, dy, dz, dt, dir)."""
    dims = (6, 6, 6, 6)
    U = fieldgen.haar_su3(dims, 65)
    base = hyp.hyp_step(U, *W)[0, 0, 0, 0, 0]
    P = U.copy()
    dx, dy, dz, dt, d = link
    idx = (dt % 6, dz % 6, dy % 6, dx % 6, d)
    P[idx] = fieldgen.haar_su3((1, 1, 1, 1), 66)[0, 0, 0, 0, 0] @ P[idx]
    changed = np.max(np.abs(hyp.hyp_step(P, *W)[0, 0, 0, 0, 0] - base))
    assert (changed > 1e-6) if inside else (changed == 0.0)
