"""Bank-aware shared-memory placement and hop schedule of a down-spin row (host only, no
device).

The continued-fraction apply holds each row in an order sorted by hop count (so that a
warp's elements have equal trip counts); the FP32 kernel stages each row of V_k in shared
memory (lane i stores positions 2i and 2i + 1 at their slots, 16 zero words follow the
row) and gathers the down-spin hop targets of 64 positions per warp (two per lane), one
hop per position per round, for the warp's largest hop count.  The library chooses a slot
per position and the round of each hop so that the gathers of a half-warp hit fewer bank
conflicts.  These tests recompute, in plain Python from the sector's hop structure, the
kernel's access sets and their worst-bank counts, check the library's numbers against
them, and check that the schedule reads every hop of every position exactly once."""
import itertools

import numpy as np
import pytest

THREADS = 256
ZERO_WORDS = 16


def _down_hops(L, n, periodic=True):
    """Hop targets (rank) and sign bits of every state: the wrap bond of a ring passes
    the other n - 1 electrons of the species (sign bit set when n - 1 is odd)."""
    states = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(L), n))
    rank = {s: i for i, s in enumerate(states)}
    nb = L if periodic else L - 1
    hops = []
    for s in states:
        h = []
        for i in range(nb):
            j = (i + 1) % L
            if ((s >> i) & 1) != ((s >> j) & 1):
                neg = (j == 0 and (n - 1) % 2 == 1)
                h.append((rank[s ^ (1 << i) ^ (1 << j)], int(neg)))
        hops.append(h)
    return hops


def _in_row_order(hops):
    """Hop lists by position: the states sorted by hop count (descending, stable),
    targets renamed to their positions."""
    order = sorted(range(len(hops)), key=lambda d: -len(hops[d]))
    pos = {d: p for p, d in enumerate(order)}
    return order, [[(pos[t], sg) for t, sg in hops[d]] for d in order]


def _warps(D):
    half = D // 2
    for it in range((half + THREADS - 1) // THREADS):
        for w in range(THREADS // 32):
            q0 = it * THREADS + 32 * w
            if q0 < half:
                yield q0, [q for q in range(q0, q0 + 32) if q < half]


def _mean_worst_bank(D, entry, slot_of, counts):
    """Mean over the access sets (warp, half-warp, round k < R_w, parity) of the largest
    number of distinct words on one bank pair; entry(k, p) -> the word's position."""
    half = D // 2
    costs = []
    for q0, qs in _warps(D):
        R = max(max(counts[2 * q], counts[2 * q + 1]) for q in qs)
        for hw in range(2):
            hq = [q for q in range(q0 + 16 * hw, q0 + 16 * hw + 16) if q < half]
            if not hq:
                continue
            for k in range(R):
                for par in range(2):
                    words = {slot_of(entry(k, 2 * q + par)) for q in hq}
                    costs.append(np.bincount([p % 16 for p in words], minlength=16).max())
    return float(np.mean(costs))


def _plain_cost(hops):
    D = len(hops)
    counts = [len(h) for h in hops]
    return _mean_worst_bank(D, lambda k, p: hops[p][k][0] if k < len(hops[p]) else D, lambda t: t, counts)


@pytest.mark.parametrize("L,n,periodic", [(8, 4, True), (12, 6, True), (10, 5, False), (7, 3, True)])
def test_row_order_sorts_by_hop_count(L, n, periodic):
    from paper_2506_09551_gb300 import api
    order = api.row_order(L, n, periodic)
    hops = _down_hops(L, n, periodic)
    assert sorted(order.tolist()) == list(range(len(hops)))
    ref, _ = _in_row_order(hops)
    assert order.tolist() == ref


def _check_layout(L, n, periodic):
    from paper_2506_09551_gb300 import api
    slot, c_plain, c_layout, tab = api.row_layout(L, n, periodic, hops=True)
    D = len(slot)
    assert sorted(slot.tolist()) == list(range(D))
    _, hops = _in_row_order(_down_hops(L, n, periodic))
    counts = [len(h) for h in hops]
    assert tab.shape == (L if periodic else L - 1, D)
    # every hop of every position read exactly once, idle rounds on zero words,
    # nothing past the warp's round count is read
    for q0, qs in _warps(D):
        R = max(max(counts[2 * q], counts[2 * q + 1]) for q in qs)
        for q in qs:
            for p in (2 * q, 2 * q + 1):
                col = [int(v) for v in tab[:R, p]]
                real = sorted((v >> 1, v & 1) for v in col if (v >> 1) < D)
                assert real == sorted(hops[p]), (p, col, hops[p])
                assert all(D <= (v >> 1) < D + ZERO_WORDS and (v & 1) == 0 for v in col if (v >> 1) >= D)
    slot_of = lambda t: int(slot[t]) if t < D else t          # zero words sit past the row
    assert c_plain == pytest.approx(_plain_cost(hops), rel=1e-12)
    assert c_layout == pytest.approx(_mean_worst_bank(D, lambda k, p: int(tab[k, p]) >> 1, slot_of, counts),
                                     rel=1e-12)
    # staging stores: 16 consecutive lanes store positions 2i + par; full blocks hit 16 bank pairs
    half = D // 2
    for i0 in range(0, half - half % 16, 16):
        for par in range(2):
            assert len({int(slot[2 * i + par]) % 16 for i in range(i0, i0 + 16)}) == 16
    return slot, c_plain, c_layout


@pytest.mark.parametrize("L,n", [(8, 4), (10, 5), (12, 6), (14, 7)])
def test_layout_and_schedule(L, n):
    from paper_2506_09551_gb300 import api
    slot, c_plain, c_layout = _check_layout(L, n, True)
    assert 1.0 <= c_layout < c_plain
    assert c_layout <= 1.2                 # near one wavefront per half-warp gather
    slot2, _, c2 = api.row_layout(L, n)
    assert (slot2 == slot).all() and c2 == c_layout


def test_open_chain_layout():
    _, c_plain, c_layout = _check_layout(10, 5, False)
    assert c_layout <= c_plain


def test_odd_sector_is_rejected():
    from paper_2506_09551_gb300 import api, native
    with pytest.raises(native.MsbError):
        api.row_layout(7, 3)                       # C(7, 3) = 35 states
