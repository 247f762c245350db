"""Reference of fused-group plans for kernel DAGs beyond contiguous partitions: a node may
be recomputed by the groups that consume it instead of being stored (Sec. VI-A's fusable
sets with the ordering restriction of Sec. VII (a) relaxed; Sec. VI-D's traffic).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain definitions and brute force.

A plan is (cuts, X): the contiguous ranges of the stage order that `cuts` gives (bit i
cuts between stages i+1 and i+2, as for contiguous partitions) and a set X of inlined
nodes (never the output). A group computes its range plus every inlined node that it
needs and does not hold -- an inlined node read by a stage of the group, recursively
through inlined inputs. A range node that is inlined and not needed by its own range is
not computed there. A node is stored by the group that holds it in its range when it is
the output, or when a path from it through inlined nodes reaches a stage outside the
range (that stage's group reads it or recomputes from it). Traffic of a group over
tiles of TX x TY pixels (B = W H T / (TX TY) tiles): per external input e (a node no
group member computes, read by a member) its tile grown by its halo h_e on every side,
(TX + 2 h_e)(TY + 2 h_e) pixels of 1 byte (the frame) or 4 bytes (a map), plus TX TY x
4 bytes per stored node. Halos: a stored node needs 0; a member or external input needs
the largest (halo of a consumer member + that consumer's radius) over its consumers in
the group; a member no stored node depends on is not computed.

On-chip bytes of a group (the executor's shared memory per block, the feasibility test
of Sec. VII (c)): the group's tiles are held in equal slots of (TX + 2 h_max)(TY + 2
h_max) floats, h_max the largest halo in the group; the external inputs are loaded
first (in node order), then the computed members run in node order, each taking a free
slot (or a new one) for its tile, and an input's slot is freed after its last consumer
in the group has taken its own; the group needs as many slots as were ever taken.
"""
from __future__ import annotations

import itertools

TX, TY = 32, 16


def radius(row) -> int:
    kind, _, _, r, _, _ = row
    return r if kind == 4 else (1 if kind == 5 else 0)


def inputs(rows, j: int) -> list[int]:
    kind, i1, i2, _, _, _ = rows[j - 1]
    return [i1, i2] if kind == 3 and i2 != i1 else [i1]


def consumers(rows) -> list[list[int]]:
    n = len(rows)
    cons = [[] for _ in range(n + 1)]
    for j in range(1, n + 1):
        for i in inputs(rows, j):
            cons[i].append(j)
    return cons


def ranges(n: int, cuts: int) -> list[tuple[int, int]]:
    out, a = [], 1
    for b in range(1, n + 1):
        if b == n or (cuts >> (b - 1)) & 1:
            out.append((a, b))
            a = b + 1
    return out


def group_members(rows, a: int, b: int, X: set[int]) -> set[int]:
    """The range's needed nodes plus the inlined nodes it must recompute."""
    n = len(rows)
    cons = consumers(rows)
    rng = set(range(a, b + 1))
    # a range node is needed unless it is inlined and no range node needs it
    needed = set()
    for j in sorted(rng, reverse=True):
        if j not in X or any(c in needed for c in cons[j]):
            needed.add(j)
    members = set(needed)
    stack = list(needed)
    while stack:
        j = stack.pop()
        for i in inputs(rows, j):
            if i != 0 and i in X and i not in members:
                members.add(i)
                stack.append(i)
    return members


def stored(rows, a: int, b: int, X: set[int], j: int) -> bool:
    """Whether the group of range [a, b] stores its range node j."""
    n = len(rows)
    if j == n:
        return True
    if j in X:
        return False
    cons = consumers(rows)
    seen, stack = set(), [j]
    while stack:
        u = stack.pop()
        for c in cons[u]:
            if c > b:
                return True
            if c in X and c not in seen:
                seen.add(c)
                stack.append(c)
    return False


def group_traffic(rows, a: int, b: int, X: set[int]) -> tuple[float, set[int], dict[int, int]]:
    """(bytes per tile, stored nodes, halo per node) of the group of range [a, b]."""
    members = group_members(rows, a, b, X)
    cons = consumers(rows)
    outs = {j for j in members if a <= j <= b and stored(rows, a, b, X, j)}
    halo = {}
    for j in sorted(members, reverse=True):  # a member no stored node depends on stays at -1 (not computed)
        h = 0 if j in outs else -1
        for c in cons[j]:
            if c in members and halo[c] >= 0:
                h = max(h, halo[c] + radius(rows[c - 1]))
        halo[j] = h
    ext = {}
    for j in members:
        if halo[j] < 0:
            continue
        for i in inputs(rows, j):
            if i not in members:
                ext[i] = max(ext.get(i, -1), halo[j] + radius(rows[j - 1]))
    t = sum((TX + 2 * h) * (TY + 2 * h) * (1 if e == 0 else 4) for e, h in ext.items())
    t += TX * TY * 4 * len(outs)
    return float(t), outs, {**halo, **{e: h for e, h in ext.items()}}


def onchip_bytes(rows, a: int, b: int, X: set[int]) -> int:
    """Shared-memory bytes per block of the group of range [a, b]."""
    _, _, halo = group_traffic(rows, a, b, X)
    members = group_members(rows, a, b, X)
    live = {j for j in members if halo[j] >= 0}
    ext = sorted(e for e in halo if e not in members)
    cons = consumers(rows)
    last = {}
    for j in list(ext) + sorted(live):
        cs = [c for c in cons[j] if c in live]
        if cs:
            last[j] = max(cs)
    hmax = max([0] + [halo[j] for j in list(ext) + sorted(live)])
    free, slots, taken = [], {}, 0
    for e in ext:
        slots[e] = free.pop() if free else taken
        taken = max(taken, slots[e] + 1)
    for j in sorted(live):
        slots[j] = free.pop() if free else taken
        taken = max(taken, slots[j] + 1)
        for i in inputs(rows, j):
            if last.get(i) == j and i in slots:
                free.append(slots.pop(i))
    return taken * (TX + 2 * hmax) * (TY + 2 * hmax) * 4


def valid(rows, cuts: int, X: set[int]) -> bool:
    """Every external input of a group is the frame or stored by an earlier group."""
    n = len(rows)
    if n in X:
        return False
    stored_by = {}
    for k, (a, b) in enumerate(ranges(n, cuts)):
        members = group_members(rows, a, b, X)
        for j in members:
            for i in inputs(rows, j):
                if i != 0 and i not in members and stored_by.get(i, k) >= k:
                    return False
        for j in range(a, b + 1):
            if stored(rows, a, b, X, j):
                stored_by[j] = k
    return True


def plan_traffic(rows, cuts: int, X: set[int], W: int, H: int, T: int) -> float:
    tiles = W * H * T / (TX * TY)
    return tiles * sum(group_traffic(rows, a, b, X)[0] for a, b in ranges(len(rows), cuts))


def brute_force(rows, W: int, H: int, T: int, feasible=lambda rows, a, b, X: True):
    """(cost, cuts, X) of the cheapest valid plan over every cut mask and inline set."""
    n = len(rows)
    best = None
    for cuts in range(1 << (n - 1)):
        for xs in itertools.product([0, 1], repeat=n - 1):
            X = {j + 1 for j in range(n - 1) if xs[j]}
            if not valid(rows, cuts, X):
                continue
            if not all(feasible(rows, a, b, X) for a, b in ranges(n, cuts)):
                continue
            c = plan_traffic(rows, cuts, X, W, H, T)
            if best is None or c < best[0] - 1e-9:
                best = (c, cuts, X)
    return best
