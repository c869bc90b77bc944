"""The (step, slab) schedule of the host-streamed smearing (lq_stout_smear_host),
restated on the CPU: the first two and the last two steps run as items in
the order of the key 2k + d(i) (d the cyclic distance of slab i from slab
0, stable within a key), the steps between as whole-lattice launches, all
on one stream.  Step k of slab i reads the step k-1 field of slabs i-1, i,
i+1 and overwrites the field that step k-1 of those slabs read, so it must
follow step k-1 of its neighbours; the same key runs as one launch, so two
items of one key must not depend on each other.  Checked for 1-24 slabs and
0-9 steps."""
import pytest


def cyclic_distance(i, nc):
    return min(i, nc - i)


def schedule(nc, n_steps):
    """[(key_group, k, i)], i = -1 for a whole-lattice step."""
    def wave(k_lo, k_hi):
        w = [(2 * k + cyclic_distance(i, nc), k, i) for k in range(k_lo, k_hi + 1) for i in range(nc)]
        return sorted(w, key=lambda t: t[0])     # stable
    items = []
    if n_steps <= 4:
        items += wave(1, n_steps)
    else:
        items += wave(1, 2)
        items += [(None, k, -1) for k in range(3, n_steps - 1)]
        items += wave(n_steps - 1, n_steps)
    return items


@pytest.mark.parametrize("nc", range(1, 25))
@pytest.mark.parametrize("n_steps", range(0, 10))
def test_every_item_follows_the_items_it_reads(nc, n_steps):
    items = schedule(nc, n_steps)
    done = {}          # (k, slab) -> position of the launch that produced it
    launch = -1
    prev_key = object()
    for key, k, i in items:
        if i < 0 or key != prev_key:
            launch += 1
        prev_key = key if i >= 0 else object()
        slabs = range(nc) if i < 0 else [i]
        for s in slabs:
            if k > 1:
                for j in ((s - 1) % nc, s, (s + 1) % nc):
                    # produced by an earlier launch, never by this one
                    assert done[(k - 1, j)] < launch, (nc, n_steps, k, s, j)
            done[(k, s)] = launch
    # every (step, slab) ran exactly once
    assert sorted(done) == sorted((k, s) for k in range(1, n_steps + 1) for s in range(nc))
