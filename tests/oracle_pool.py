"""Runs the FP64 oracle on many small periodic boxes in parallel processes
(the sampled full-size parity checks).  This module imports numpy and the
oracle only, so that spawned workers start without torch or a GPU context."""
import multiprocessing as mp
import os

from oracle import stout


def _box_center(args):
    box, rho, n, dirs = args
    return stout.stout_smear(box, rho, n, dirs)[n, n, n, n]


def stout_box_centers(boxes, rho, n, dirs):
    """The smeared links at the centre site of each box (side 2n+1: exact for
    the full lattice, n steps reach n sites), computed in a spawned pool."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=min(len(boxes), os.cpu_count() or 1)) as pool:
        return pool.map(_box_center, [(b, rho, n, dirs) for b in boxes])
