"""Host logic of bench.py's roofline model, checked without a GPU.

The launch schedule that bench.py rebuilds from the host loop must transform each
band pair exactly once under the pair symmetry (every logical (k, a, q, j) pair is
either transformed or the mirror of a transformed pair), and without the symmetry
the per-pass byte model must reduce to the 48 bytes per grid point and logical pair
of the plain three-pass pipeline plus its per-target terms.
"""
import itertools

import pytest

import bench


def transformed_set(nk, n_occ, n_tgt, T):
    """Pairs (k, a, q, j) the symmetric host loop transforms, by its rules."""
    out = set()
    for k, q, a, j in itertools.product(range(nk), range(nk), range(n_tgt), range(n_occ)):
        if a >= n_occ:
            out.add((k, a, q, j))                       # targets past the occupied set
        elif q > k:
            out.add((k, a, q, j))                       # blocks q > k, whole square
        elif q == k and a // T <= j // T:
            out.add((k, a, q, j))                       # k = q tiles I <= J
    return out


@pytest.mark.parametrize("nk,n_occ,n_tgt,TA,TJ,G", [(1, 8, 8, 3, 3, 1), (3, 5, 7, 2, 4, 1),
                                                     (4, 6, 6, 4, 4, 1), (2, 9, 12, 5, 3, 1),
                                                     (8, 4, 6, 3, 3, 1), (8, 4, 6, 6, 4, 8),
                                                     (5, 3, 5, 5, 3, 2), (7, 2, 2, 2, 2, 3)])
def test_schedule_transforms_every_pair_once(nk, n_occ, n_tgt, TA, TJ, G):
    """G > 1: several k-points' occupied sets share a batch (the same pairs, fewer
    and wider launches)."""
    T = min(TA, TJ)
    tset = transformed_set(nk, n_occ, n_tgt, T)
    sched = bench.batch_schedule(nk, n_occ, n_tgt, TA, TJ, G)
    assert all(tj <= max(TJ, G * n_occ) for _, _, tj in sched)
    assert sum(ta * tj for _, ta, tj in sched) == len(tset)
    # mirrored launches carry exactly the transformed pairs whose mirror is not
    # transformed itself (tiles I < J and blocks q > k)
    mirrored = sum(ta * tj for kind, ta, tj in sched if kind == "mirrored")
    assert mirrored == sum(1 for (k, a, q, j) in tset
                           if a < n_occ and (q, j, k, a) not in tset)
    # every logical pair is covered exactly once
    covered = set()
    for (k, a, q, j) in tset:
        assert (k, a, q, j) not in covered
        covered.add((k, a, q, j))
        if a < n_occ and (q, j, k, a) not in tset:
            covered.add((q, j, k, a))
    assert len(covered) == nk * n_tgt * nk * n_occ


def test_byte_model_without_symmetry_is_48_bytes_per_point():
    class W:                                    # the fields pass_bytes_per_step reads
        grid = (24, 24, 24)
    nk, n_occ, n_tgt, TA, TJ = 3, 10, 12, 5, 4
    sched = bench.batch_schedule(nk, n_occ, n_tgt, TA, TJ, sym=False)
    n3 = 24 ** 3
    pairs = nk * n_tgt * nk * n_occ
    assert sum(ta * tj for _, ta, tj in sched) == pairs
    b = bench.pass_bytes_per_step(W, sched)
    launches_per_target = nk * nk * -(-n_occ // TJ)       # (k, q, occupied batch) per target
    per_target = n_tgt * launches_per_target
    assert b["pass_a"] == 16 * n3 * pairs + 8 * n3 * per_target
    assert b["pass_b"] == 16 * n3 * pairs
    assert b["pass_c"] == 16 * n3 * pairs + 32 * n3 * per_target
    assert sum(b.values()) == 48 * n3 * pairs + 40 * n3 * per_target


@pytest.mark.parametrize("nk,n_occ,n_tgt,TA,TJ,G", [(8, 160, 192, 64, 80, 1), (8, 4, 6, 6, 4, 8),
                                                     (5, 3, 5, 5, 3, 2), (3, 5, 7, 2, 4, 1)])
@pytest.mark.parametrize("world", [2, 3, 8])
def test_sharded_schedules_add_up_to_the_whole(nk, n_occ, n_tgt, TA, TJ, G, world):
    """Each block {k, q} belongs to one shard (the library's assignment, host code):
    the shards' schedules transform, between them, exactly the unsharded pairs."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import xx
    owner = xx.xx_shard_blocks(nk, n_occ, n_tgt, world)

    def owned_by(r):
        def f(k, q):
            k, q = min(k, q), max(k, q)
            return owner[k * nk - k * (k - 1) // 2 + (q - k)] == r
        return f
    whole = sum(ta * tj for _, ta, tj in bench.batch_schedule(nk, n_occ, n_tgt, TA, TJ, G))
    parts = [sum(ta * tj for _, ta, tj in bench.batch_schedule(nk, n_occ, n_tgt, TA, TJ, G,
                                                               owned=owned_by(r)))
             for r in range(world)]
    assert sum(parts) == whole
    if nk == 8 and n_occ == 160:
        # the beta-boron workload: every shard within 5 % of the mean
        assert max(parts) <= 1.05 * whole / world
