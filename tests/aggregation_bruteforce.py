"""A second, independent statement of the aggregation rule in plain Python
(dictionaries and sets, no arrays shared with the oracle), used on small
graphs to pin the oracle's aggregation bit for bit.

The rule (a reading of Sec. 3.1.1; the paper defers details to the cited
aggregation papers):
* an edge is a matching candidate when its weight is at least a quarter of
  the largest weight at either end;
* rounds: every unmatched node chooses its best unmatched candidate edge
  (weight, then hash, then smaller endpoints), mutual choices pair up;
  stop when a round pairs nobody or after `rounds` rounds;
* pass 1 keeps leftovers as singletons; pass 2 (on the contracted graph)
  lets each leftover join the pair of its best neighbour when that
  neighbour is paired;
* groups are numbered in the order of their smallest member.
"""
from __future__ import annotations


def fmix32(h: int) -> int:
    h &= 0xFFFFFFFF
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def edge_hash(a: int, b: int, seed: int) -> int:
    return fmix32(((a * 2654435761) & 0xFFFFFFFF) ^ b ^ seed)


def vertex_hash(v: int, seed: int) -> int:
    return fmix32(((v * 2654435761) & 0xFFFFFFFF) ^ seed ^ 0x5BD1E995)


def edge_key(i, j, w, seed):
    a, b = min(i, j), max(i, j)
    return (w, edge_hash(a, b, seed), -a, -b)


def to_adj(rowptr, col, w):
    adj = []
    for i in range(len(rowptr) - 1):
        adj.append({int(col[p]): int(w[p]) for p in range(rowptr[i], rowptr[i + 1])})
    return adj


def matching_pass(adj, rounds=32, seed=0, attach=False):
    n = len(adj)
    maxw = [max(a.values()) if a else 0 for a in adj]
    mate = [None] * n
    for _ in range(rounds):
        choice = {}
        for i in range(n):
            if mate[i] is not None:
                continue
            cands = [(edge_key(i, j, wij, seed), j) for j, wij in adj[i].items()
                     if mate[j] is None and (4 * wij >= maxw[i] or 4 * wij >= maxw[j])]
            if cands:
                choice[i] = max(cands)[1]
        pairs = [(i, j) for i, j in choice.items() if choice.get(j) == i]
        if not pairs:
            break
        for i, j in pairs:
            mate[i] = j
    owner = {}
    for i in range(n):
        owner[i] = i if mate[i] is None else min(i, mate[i])
    if attach:
        for i in range(n):
            if mate[i] is not None or not adj[i]:
                continue
            _, j = max((edge_key(i, j, wij, seed), j) for j, wij in adj[i].items())
            if mate[j] is not None:
                owner[i] = min(j, mate[j])
    members = {}
    for i in range(n):
        members.setdefault(owner[i], []).append(i)
    order = sorted(members.values(), key=min)
    group = [0] * n
    for g, mem in enumerate(order):
        for i in mem:
            group[i] = g
    return group, len(order)


def contract(adj, group, ng):
    out = [dict() for _ in range(ng)]
    for i, a in enumerate(adj):
        for j, wij in a.items():
            gi, gj = group[i], group[j]
            if gi != gj:
                out[gi][gj] = out[gi].get(gj, 0) + wij
    return out


def aggregate(adj, rounds=32, seed=0):
    g1, n1 = matching_pass(adj, rounds, seed, attach=False)
    g2, n2 = matching_pass(contract(adj, g1, n1), rounds, seed, attach=True)
    comp = [g2[g1[i]] for i in range(len(adj))]
    first = {}
    for i, a in enumerate(comp):
        first.setdefault(a, i)
    order = sorted(first, key=lambda a: first[a])
    rank = {a: r for r, a in enumerate(order)}
    return [rank[a] for a in comp], len(order)


def colour(adj, seed=0, passes=4):
    """Jones-Plassmann rounds with priority (degree, vertex hash, index), then
    `passes` passes of iterated greedy recolouring, classes visited from the
    highest colour down."""
    n = len(adj)
    col = [-1] * n
    prio = [(len(adj[i]), vertex_hash(i, seed), i) for i in range(n)]

    def smallest_free(i, c):
        used = {c[j] for j in adj[i] if c[j] >= 0}
        k = 0
        while k in used:
            k += 1
        return k

    while any(c < 0 for c in col):
        snap = list(col)
        for i in range(n):
            if snap[i] >= 0:
                continue
            if all(snap[j] >= 0 or prio[j] < prio[i] for j in adj[i]):
                col[i] = smallest_free(i, snap)
    for _ in range(passes):
        new = [-1] * n
        for c in range(max(col), -1, -1):
            for i in range(n):
                if col[i] == c:
                    new[i] = smallest_free(i, new)
        col = new
    return col
