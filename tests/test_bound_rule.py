"""The rule by which the insertion-matrix tiles skip customers never changes a pick.

The device scores the insertion-delta matrix tile by tile and skips, in a
tile, every customer whose lower bound over the tile shows that none of its
entries there can matter to the repair operator (Section 4.2.3: greedy,
regret-2, regret-3, regret-m).  The bounds are the bests scored so far: per
vehicle group (v mod 4) the least (dz, dt) key, and per drop vehicle the
least key.  A customer is kept in a tile when
  - its bound is at most the least group best (it may hold the best entry), or,
    for regret-2 and regret-3,
  - its bound's makespan is at most the second (third) least group makespan
    and below the largest best makespan among the tile's drop vehicles (it
    may lower a vehicle's best makespan that counts);
  - regret-m keeps every customer with an admissible entry.
This test restates that rule and the selection on random matrices, with
many ties, bounds that are looser than the tile's true least key, adjacent
entries scored up front and tiles taken in random order, and checks that the
pick (customer, drop gap, pickup gap) is always the one made from the full
matrix.  It checks the rule, not the kernel: the GPU tests compare the
kernel's searches with the oracle's, which scores every entry.
"""
import numpy as np

INF = 1 << 40
GROUPS = 4


def key_of(dz, dt):
    return (int(dz), int(dt))


def pick_from(ent, nrem, m, G, kind):
    """ent[ti]: list of (row, col, dz, dt, v).  Returns the pick (customer slot,
    row, col) as the selection makes it from the per-vehicle bests and per-row
    keys, with what it rests on: every customer's best entry and, under
    regret-k, its k least vehicle makespans."""
    best, regret, least = [], [], []
    for ti in range(nrem):
        # per drop vehicle: least (dz, dt, row); per row: least (dz, dt, col)
        vb = {}
        rowkey = {}
        for (r, c, dz, dt, v) in ent[ti]:
            k = (dz, dt, r)
            if v not in vb or k < vb[v]:
                vb[v] = k
            k2 = (dz, dt, c)
            if r not in rowkey or k2 < rowkey[r]:
                rowkey[r] = k2
        if not vb:
            return None                        # a customer with no feasible insertion: the repair fails
        b = min(vb.values())
        col = rowkey[b[2]][2]
        best.append((b[0], b[1], b[2], col))
        opts = sorted(vb[v][0] if v in vb else INF for v in range(m))
        kk = {1: 2, 2: 3, 3: m}.get(kind, 0)
        least.append(tuple(opts[:kk]))
        reg = 0
        if kind:
            for i in range(1, kk):
                reg += (opts[i] if i < m else INF) - opts[0]
        regret.append(reg)
    if kind == 0:
        order = sorted(range(nrem), key=lambda ti: (best[ti][0], best[ti][1], best[ti][2] * G + best[ti][3], ti))
        p = order[0]
    else:
        p = 0
        for ti in range(1, nrem):
            if regret[ti] > regret[p]:
                p = ti
    return (p, best[p][2], best[p][3]), best, least


def kept_entries(rng, ent, tiles, seeds, m, kind):
    """Score the seeds, then the tiles in random order, skipping a customer in
    a tile by the rule; returns the entries scored per customer."""
    nrem = len(ent)
    scored = [[] for _ in range(nrem)]
    gbest = [[(INF, INF)] * GROUPS for _ in range(nrem)]
    vbest = [[(INF, INF)] * m for _ in range(nrem)]

    def score(ti, e):
        r, c, dz, dt, v = e
        scored[ti].append(e)
        k = key_of(dz, dt)
        g = v % GROUPS
        if k < gbest[ti][g]:
            gbest[ti][g] = k
        if k < vbest[ti][v]:
            vbest[ti][v] = k

    for ti, e in seeds:
        score(ti, e)
    for tile in rng.permutation(len(tiles)):
        for ti in range(nrem):
            es = tiles[tile][ti]
            if not es:
                continue
            least = min(key_of(e[2], e[3]) for e in es)
            # a lower bound at or below the least key, sometimes strictly below
            slack = int(rng.integers(0, 3))
            lb = (least[0], max(0, least[1] - slack)) if rng.random() < 0.5 else \
                (max(0, least[0] - slack), least[1])
            vehicles = {e[4] for e in es}
            keep = True
            if kind <= 2:
                u = min(gbest[ti])
                keep = lb <= u
                if not keep and kind > 0:
                    d = sorted(gk[0] for gk in gbest[ti])
                    vb = max(vbest[ti][v][0] for v in vehicles)
                    keep = lb[0] <= d[kind] and lb[0] < vb
            if keep:
                for e in es:
                    score(ti, e)
    return scored


def one_case(rng, kind):
    m = int(rng.integers(1, 9))
    nrem = int(rng.integers(1, 9))
    G = int(rng.integers(m + 2, 40))
    route = np.sort(rng.integers(0, m, size=G))        # drop vehicle of each row (gap)
    vals_z = int(rng.integers(1, 4))                  # few distinct values: many ties
    vals_t = int(rng.integers(1, 6))
    ent = []
    for _ in range(nrem):
        es = []
        for r in range(G):
            for c in range(G):
                if rng.random() < 0.35:
                    es.append((r, c, int(rng.integers(0, vals_z)), int(rng.integers(0, vals_t)), int(route[r])))
        ent.append(es)
    # tiles: rectangles of rows x columns
    tr, tc = int(rng.integers(1, 8)), int(rng.integers(1, 12))
    tiles_map = {}
    seeds = []
    for ti, es in enumerate(ent):
        for e in es:
            if e[0] == e[1] and rng.random() < 0.7:   # an adjacent entry, scored up front
                seeds.append((ti, e))
                continue
            t = (e[0] // tr, e[1] // tc)
            tiles_map.setdefault(t, [[] for _ in range(nrem)])[ti].append(e)
    tiles = list(tiles_map.values())
    full = pick_from(ent, nrem, m, G, kind)
    kept = kept_entries(rng, ent, tiles, seeds, m, kind)
    got = pick_from(kept, nrem, m, G, kind)
    return full, got


def test_bound_rule_keeps_every_pick():
    rng = np.random.default_rng(20261204)
    for trial in range(2400):
        kind = trial % 4
        full, got = one_case(rng, kind)
        assert got == full, (trial, kind, full, got)


def test_bound_rule_skips_something():
    """The rule is not vacuous: on these matrices it skips customers in tiles."""
    rng = np.random.default_rng(7)
    skipped = 0
    for trial in range(200):
        kind = trial % 3
        m, nrem, G = 4, 4, 24
        route = np.sort(rng.integers(0, m, size=G))
        ent = [[(r, c, int(rng.integers(0, 3)), int(rng.integers(0, 6)), int(route[r]))
                for r in range(G) for c in range(G) if rng.random() < 0.5] for _ in range(nrem)]
        tiles_map = {}
        for ti, es in enumerate(ent):
            for e in es:
                tiles_map.setdefault((e[0] // 4, e[1] // 8), [[] for _ in range(nrem)])[ti].append(e)
        tiles = list(tiles_map.values())
        kept = kept_entries(rng, ent, tiles, [], m, kind)
        skipped += sum(len(a) - len(b) for a, b in zip(ent, kept))
        assert pick_from(kept, nrem, m, G, kind) == pick_from(ent, nrem, m, G, kind)
    assert skipped > 0
