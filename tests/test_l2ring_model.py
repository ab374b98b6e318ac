"""A discrete-event model of the single-launch four-step's work schedule
(fourstep_l2.cuh with the ring geometry of api.cu's l2_geometry), no GPU.

The protocol restated: rows are cut into chunks of R rows; a round of work is
the 2 TT items (TT = R L / C column tiles per phase) of phase 1 of chunk r and
phase 2 of chunk r - lag; items are claimed in order from one counter, each
CTA holding the claim of its next item while it works on the current one.  A
phase-2 item of chunk c waits until all TT phase-1 items of c are done; a
phase-1 item of chunk c >= S waits until all phase-2 items of chunk c - S (the
previous user of ring slot c mod S) are done.  Geometry as planned: lag =
ceil(2 G / (2 TT)) + 1 for a grid of G CTAs, S = min(2 lag, chunks).

Checked for every (L, R, G, batch) tried, with random item durations: every
ring slot, row and column index stays in bounds; a slot is never written by a
chunk while its previous chunk's phase 2 is unfinished; every item finishes
(no deadlock, no lost item); a minimal-margin stress (S = lag + 1) as well.
"""
import heapq
import random

import pytest


def l2_geometry(R, L, C, G):
    round_items = 2 * R * (L // C)
    lag = (2 * G + round_items - 1) // round_items + 1
    return lag, 2 * lag


def simulate(batch, R, L, C, G, slots_planned, lag, seed):
    rnd = random.Random(seed)
    TT = R * (L // C)
    nch = (batch + R - 1) // R
    slots = min(slots_planned, nch)
    total = (nch + lag) * 2 * TT
    done1, done2 = [0] * nch, [0] * nch
    owner = {}
    counter = 0
    held = {}
    events = []
    for cta in range(min(G, total)):
        held[cta] = counter
        counter += 1
        events.append((0.0, cta, "claim", None))
    heapq.heapify(events)
    retired = 0
    steps = 0
    while events:
        steps += 1
        assert steps < 10 ** 7, "schedule did not finish"
        tm, cta, state, item = heapq.heappop(events)
        if state == "claim":
            w = held[cta]
            held[cta] = counter  # the next claim is in flight while w runs
            counter += 1
            if w >= total:
                retired += 1
                continue
            r, off = divmod(w, 2 * TT)
            p1 = off < TT
            chunk = r if p1 else r - lag
            tile = off if p1 else off - TT
            if not 0 <= chunk < nch:  # an empty item of the first or last rounds
                heapq.heappush(events, (tm + 0.01, cta, "claim", None))
                continue
            row, group = divmod(tile, L // C)
            assert 0 <= row < R and 0 <= group * C < L
            slot = chunk % slots
            assert 0 <= slot < min(slots_planned, nch)
            heapq.heappush(events, (tm, cta, "wait", (p1, chunk, slot, tm)))
        elif state == "wait":
            p1, chunk, slot, t0 = item
            if p1:
                ready = chunk < slots or done2[chunk - slots] >= TT
            else:
                ready = done1[chunk] >= TT
            if not ready:
                assert tm - t0 < 1e4, f"deadlock waiting on {item}"
                heapq.heappush(events, (tm + 0.05, cta, "wait", item))
                continue
            if p1:
                prev = owner.get(slot)
                assert prev is None or prev == chunk or done2[prev] == TT, "slot reused too early"
                owner[slot] = chunk
            else:
                assert owner[slot] == chunk
            heapq.heappush(events, (tm + rnd.uniform(0.5, 2.0), cta, "done", item))
        else:
            p1, chunk = item[0], item[1]
            (done1 if p1 else done2)[chunk] += 1
            heapq.heappush(events, (tm, cta, "claim", None))
    assert all(d == TT for d in done1) and all(d == TT for d in done2), "lost item"
    assert retired == min(G, total)


@pytest.mark.parametrize("L", [64, 128, 256])
def test_planned_geometry_finishes_and_stays_in_bounds(L):
    for R in (8, 16, 32, 64):
        for G in (1, 7, 152 * 8, 152 * 12):
            lag, slots = l2_geometry(R, L, 16, G)
            assert slots > lag
            for batch in (1, R - 1, R, R + 1, 3 * R + 5, 20 * R):
                for seed in range(2):
                    simulate(batch, R, L, 16, G, slots, lag, seed)


def test_minimal_margin_still_finishes():
    for lag in range(0, 4):
        for slots in range(lag + 1, lag + 3):
            for G in (1, 3, 50, 500):
                simulate(37, 4, 64, 16, G, slots, lag, 3)
