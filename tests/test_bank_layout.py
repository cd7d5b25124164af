"""The plane layouts (Lay<N> in xx_kernels.cuh) against the shared-memory bank model.

csrc/bank_layout.py counts the wavefronts that the plane transforms' 8-byte shared
accesses take (half-warp phases, 16 bank pairs).  Every committed (S, LD) must be
a minimum of that count over the search space, and the replay ratios stated in
the kernel header must hold.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_1111_0716_gb300", "csrc"))

import bank_layout as bl  # noqa: E402

LAY = bl.lay_from_header()


def test_every_supported_length_has_a_layout():
    assert sorted(LAY) == [24, 32, 36, 40, 48, 54, 60, 64, 72, 80, 96, 108]
    for N, (A, B, S, LD) in LAY.items():
        assert A * B == N and S >= B and LD >= max(N, (A - 1) * S + B)


def test_phase_cost_counts_distinct_elements_per_bank_pair():
    assert bl.phase_cost(list(range(32))) == (2, 2)            # consecutive: conflict-free
    assert bl.phase_cost([0] * 32) == (2, 2)                   # one element: broadcast
    assert bl.phase_cost([16 * l for l in range(32)]) == (32, 2)
    assert bl.phase_cost([2 * l for l in range(32)]) == (4, 2)  # stride 2: two-way
    assert bl.phase_cost([None] * 16 + list(range(16))) == (1, 1)


@pytest.mark.parametrize("N", sorted(LAY))
def test_committed_layout_minimises_the_x_step_count(N):
    A, B, S, LD = LAY[N]
    best = bl.search(N, A, B)[0][0]
    assert bl.x_cost(N, A, B, S, LD)[0] == best


def test_x_step_replay_ratios():
    ratio = {N: (lambda c: c[0] / c[1])(bl.x_cost(N, *LAY[N])) for N in LAY}
    for N in (32, 36, 96):
        assert ratio[N] == 1.0
    for N in (24, 60, 72):
        assert ratio[N] <= 1.2
    assert ratio[108] <= 1.34
    for N in (40, 48, 54, 64, 80):
        assert ratio[N] <= 1.5


@pytest.mark.parametrize("N", sorted(LAY))
def test_y_steps_conflict_only_at_the_column_wrap(N):
    """Any kept half-width h: conflict-free when 16 divides N, at most 2x otherwise."""
    for h in range(1, (N - 1) // 2 + 1):
        c, i = bl.y_cost(N, h)
        if N % 16 == 0:
            assert c == i, h
        else:
            assert c <= 2 * i, h


@pytest.mark.parametrize("N", sorted(LAY))
def test_staged_reads_conflict_free_at_a_pitch_of_b_mod_16(N):
    """The staged plane's reads replay at pitch N; a pitch equal to B modulo 16 removes
    every conflict (the layout a padded staging would use)."""
    A, B, S, LD = LAY[N]
    c, i = bl.staged_read_cost(N, A, B)
    assert c >= i
    c, i = bl.staged_read_cost(N, A, B, bl.conflict_free_pitch(N, B))
    assert c == i
