"""The copy schedule of the d >= 8 DP's shared-memory windows, checked on the
CPU (no GPU).

The DP kernel (paper_1811_11076_gb300/csrc/dp.cuh, the WIN variant) keeps, per
lane group of G lanes, the last W query rows (and, symmetrically, series
columns) in a shared-memory window.  In step s lane lam reads row
s - h0 - P*lam; the group's loader lanes copy the row of step s + AHEAD
asynchronously into its slot, and a copy may land at any time after it is
issued.  The window is correct if (a) every row a lane reads in a step is the
one its slot holds by then, and (b) no copy lands on a slot whose previous row
a lane may still read, in the same step or in the one before (lanes of a warp
meet only at each step's __syncwarp).  This emulates the schedule with the
kernel's own constants and slot map, read from the source, for every compiled
group shape and a range of band offsets, including the fill of a new pair's
window (the (G-1)P rows before the first step and the first AHEAD pieces).
"""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1811_11076_gb300", "csrc", "dp.cuh")


def _ahead():
    with open(SRC) as f:
        m = re.search(r"constexpr int DP_WIN_AHEAD = (\d+);", f.read())
    assert m, "DP_WIN_AHEAD not found"
    return int(m.group(1))


def _rows(G, P, ahead):
    # dp_win_rows: the power of two >= (G-1)P + 2 + DP_WIN_AHEAD
    w = 1
    while w < (G - 1) * P + 2 + ahead:
        w <<= 1
    return w


def _slot(r, P, W):
    # dp_win_slot: rows P apart take adjacent slots
    lp = P.bit_length() - 1
    wp_mask = W // P - 1
    return (r & (P - 1)) * (wp_mask + 1) + ((r >> lp) & wp_mask)


@pytest.mark.parametrize("G", [8, 16, 32])
@pytest.mark.parametrize("P", [2, 4])
def test_async_window_copies_never_overwrite_a_live_row(G, P):
    A = _ahead()
    W = _rows(G, P, A)
    # the slot map is a bijection on residues mod W
    assert sorted(_slot(r, P, W) for r in range(W)) == list(range(W))
    for h0 in range(-(G * P + 8), 1):
        s0 = -3
        held = {}  # slot -> (row, step from which a lane may read it)
        # a new pair: the (G-1)P rows before the first step's newest, then the
        # pieces of the first A steps, all issued before step s0
        for k in range((G - 1) * P):
            r = s0 - h0 - (G - 1) * P + k
            held[_slot(r, P, W)] = r
        for t in range(A):
            r = s0 + t - h0
            held[_slot(r, P, W)] = r
        assert len(held) == (G - 1) * P + A, "fill rows share a slot"
        for s in range(s0, s0 + 4 * W):
            # the copy for step s + A, issued in step s
            r_new = s + A - h0
            sl = _slot(r_new, P, W)
            old = held.get(sl)
            if old is not None:
                # the old row is read last in step old + h0 + (G-1)P, which
                # must come before step s - 1 (a lagging lane may still be in
                # step s - 1 when the copy lands)
                assert old + h0 + (G - 1) * P <= s - 2, (G, P, h0, s, old)
            held[sl] = r_new
            # every row read in step s is in its slot
            for lam in range(G):
                r = s - h0 - P * lam
                assert held.get(_slot(r, P, W)) == r, (G, P, h0, s, lam)
