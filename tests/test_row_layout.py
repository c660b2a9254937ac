"""Bank-aware shared-memory placement of a down-spin row (host only, no device).

The continued-fraction apply holds each row in an order sorted by hop count (so that a
warp's elements have equal trip counts); the FP32 kernel stages each row of V_k in shared
memory and gathers the down-spin hop targets of 64 elements per warp (two per lane) one
hop slot at a time.  The
library chooses a slot per element so that the gathers of a half-warp hit fewer bank
conflicts.  These tests recompute the access sets and their worst-bank counts in plain
Python from the sector's hop structure, and check the library's numbers against them."""
import itertools

import numpy as np
import pytest

THREADS = 256


def _down_hops(L, n, periodic=True):
    states = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(L), n))
    rank = {s: i for i, s in enumerate(states)}
    nb = L if periodic else L - 1
    hops = []
    for s in states:
        h = []
        for i in range(nb):
            j = (i + 1) % L
            if ((s >> i) & 1) != ((s >> j) & 1):
                h.append(rank[s ^ (1 << i) ^ (1 << j)])
        hops.append(h)
    return hops


def _in_row_order(hops):
    """Hop lists by position: the states sorted by hop count (descending, stable),
    targets renamed to their positions."""
    order = sorted(range(len(hops)), key=lambda d: -len(hops[d]))
    pos = {d: p for p, d in enumerate(order)}
    return order, [[pos[t] for t in hops[d]] for d in order]


def _mean_worst_bank(hops, slot):
    D = len(hops)
    half = D // 2
    zero = D                                   # slot of the zero word past the row
    pos = list(slot) + [zero]
    costs = []
    for it in range((half + THREADS - 1) // THREADS):
        for w in range(THREADS // 32):
            q0 = it * THREADS + 32 * w
            if q0 >= half:
                continue
            qs = [q for q in range(q0, q0 + 32) if q < half]
            ndw = max(max(len(hops[2 * q]), len(hops[2 * q + 1])) for q in qs)
            for hw in range(2):
                hq = [q for q in range(q0 + 16 * hw, q0 + 16 * hw + 16) if q < half]
                if not hq:
                    continue
                for k in range(ndw):
                    for par in range(2):
                        words = {pos[hops[2 * q + par][k]] if k < len(hops[2 * q + par]) else zero for q in hq}
                        costs.append(np.bincount([p % 16 for p in words], minlength=16).max())
    return float(np.mean(costs))


@pytest.mark.parametrize("L,n,periodic", [(8, 4, True), (12, 6, True), (10, 5, False), (7, 3, True)])
def test_row_order_sorts_by_hop_count(L, n, periodic):
    from paper_2506_09551_gb300 import api
    order = api.row_order(L, n, periodic)
    hops = _down_hops(L, n, periodic)
    assert sorted(order.tolist()) == list(range(len(hops)))
    ref, _ = _in_row_order(hops)
    assert order.tolist() == ref


@pytest.mark.parametrize("L,n", [(8, 4), (10, 5), (12, 6)])
def test_layout_is_a_permutation_with_fewer_conflicts(L, n):
    from paper_2506_09551_gb300 import api
    slot, c_plain, c_layout = api.row_layout(L, n)
    D = len(slot)
    assert sorted(slot.tolist()) == list(range(D))
    _, hops = _in_row_order(_down_hops(L, n))
    assert c_plain == pytest.approx(_mean_worst_bank(hops, range(D)), rel=1e-12)
    assert c_layout == pytest.approx(_mean_worst_bank(hops, slot), rel=1e-12)
    assert 1.0 <= c_layout < c_plain
    slot2, _, c2 = api.row_layout(L, n)
    assert (slot2 == slot).all() and c2 == c_layout


def test_open_chain_layout():
    from paper_2506_09551_gb300 import api
    slot, c_plain, c_layout = api.row_layout(10, 5, periodic=False)
    assert c_layout == pytest.approx(_mean_worst_bank(_in_row_order(_down_hops(10, 5, periodic=False))[1], slot),
                                     rel=1e-12)
    assert c_layout <= c_plain


def test_odd_sector_is_rejected():
    from paper_2506_09551_gb300 import api, native
    with pytest.raises(native.MsbError):
        api.row_layout(7, 3)                       # C(7, 3) = 35 states
