"""Interleaving models of the lock-free steps of the interleaved-label fitness kernels (Section
III-C, Eq. 13), run on the CPU.

The kernels share one label array per member among many threads with no locks:
* a flatten pass, in which each node's owner points it at the top of its piece while other
  owners walk through it.  In the last pass the roots also turn into counters (-1) as those walks
  go on;
* unions by compare-and-swap with path halving;
* the neighbour-sampling step, which skips a union when a neighbour's label, read before any
  union, equals the node's current label.

Each model thread below is a generator that yields before every access to the shared labels.  A
seeded scheduler runs the threads in random interleavings, each access being one atomic step (a
compare-and-swap is one step).  The final labels are then checked against the sequential answer:
the pieces of the forest, or the components of the forest plus the sampled edges.  The models
mirror the kernels' order of accesses: kFlatInFlight = 4 items per thread, grid-stride
assignment, and the single-item tail loop.  They check the argument that makes the concurrent
passes exact.
"""
import random

import pytest

DEAD = -(2 ** 31)


def run_interleaved(threads, rng):
    live = list(threads)
    while live:
        i = rng.randrange(len(live))
        try:
            next(live[i])
        except StopIteration:
            live.pop(i)


def random_forest(n, rng, p_dead=0.2, p_root=0.1):
    """Labels as after the cut: deleted nodes DEAD; every live node points at itself or at a live
    node with a smaller number (tree parents and fallback parents both have smaller numbers)."""
    L = [0] * n
    live = []
    for v in range(n):
        if rng.random() < p_dead:
            L[v] = DEAD
            continue
        L[v] = v if (not live or rng.random() < p_root) else rng.choice(live)
        live.append(v)
    return L


def roots_of(L):
    r = list(L)
    for v in range(len(L)):
        if L[v] == DEAD:
            continue
        x = v
        while L[x] != x:
            x = L[x]
        r[v] = x
    return r


def flatten_thread(L, items, counters):
    """One thread of the flatten kernel over its items, kFlatInFlight at a time: first all the
    items' labels, then their parents' labels, then the walks and the owner writes."""
    def top(x):  # ig_top: stop at a self-pointing or a negative (counter) label
        yield
        p = L[x]
        while p != x and p >= 0:
            x = p
            yield
            p = L[x]
        return x

    batches = [items[i:i + 4] for i in range(0, len(items) - len(items) % 4, 4)]
    tail = items[len(items) - len(items) % 4:]
    for batch in batches:
        p = []
        for v in batch:
            yield
            p.append(L[v])
        q = []
        for v, pv in zip(batch, p):
            if pv != DEAD and pv != v:
                yield
                q.append(L[pv])
            else:
                q.append(pv)
        for v, pv, qv in zip(batch, p, q):
            if pv == DEAD:
                continue
            if pv == v:
                if counters:
                    yield
                    L[v] = -1
                continue
            r = pv if (qv == pv or qv < 0) else (yield from top(qv))
            if r != pv:
                yield
                L[v] = r
    for v in tail:
        yield
        pv = L[v]
        if pv == DEAD:
            continue
        if pv == v:
            if counters:
                yield
                L[v] = -1
            continue
        r = yield from top(pv)
        if r != pv:
            yield
            L[v] = r


def grid_stride(n, threads):
    return [list(range(t, n, threads)) for t in range(threads)]


@pytest.mark.parametrize("counters", [False, True])
@pytest.mark.parametrize("seed", range(12))
def test_flatten_under_interleavings(seed, counters):
    rng = random.Random(seed * 2 + counters)
    n = rng.choice([37, 64, 150])
    L = random_forest(n, rng)
    want = roots_of(L)
    run_interleaved([flatten_thread(L, items, counters) for items in grid_stride(n, rng.choice([3, 8, 32]))], rng)
    for v in range(n):
        if want[v] == DEAD:
            assert L[v] == DEAD
        elif want[v] == v:
            assert L[v] == (-1 if counters else v), v
        else:
            assert L[v] == want[v], v  # flat: every other live node points straight at its root


def find(L, x):
    """ig_find: path halving (a halving store only ever moves a label to an ancestor)."""
    while True:
        yield
        p = L[x]
        if p == x:
            return x
        yield
        gp = L[p]
        if gp == p:
            return p
        yield
        L[x] = gp
        x = gp


def unite(L, a, b):
    """ig_unite: hook the larger root under the smaller by compare-and-swap, retry on failure."""
    a = yield from find(L, a)
    b = yield from find(L, b)
    while a != b:
        if a < b:
            a, b = b, a
        yield
        old = L[a]  # the compare-and-swap, one atomic step
        if old == a:
            L[a] = b
            return
        a = yield from find(L, old)
        b = yield from find(L, b)


def components(n, L0, edges):
    """Sequential reference: pieces of the forest L0 joined along edges (both ends live)."""
    parent = list(range(n))

    def f(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for v in range(n):
        if L0[v] != DEAD and L0[v] != v:
            parent[f(v)] = f(L0[v])
    for a, b in edges:
        if L0[a] != DEAD and L0[b] != DEAD:
            parent[f(a)] = f(b)
    return [f(v) if L0[v] != DEAD else DEAD for v in range(n)]


def same_partition(L, want):
    lab = roots_of(L)
    pairs = {}
    for x, y in zip(lab, want):
        if (x == DEAD) != (y == DEAD):
            return False
        if x != DEAD and pairs.setdefault(y, x) != x:
            return False
    return len(set(pairs.values())) == len(pairs)


def random_edges(n, m, rng):
    return [(rng.randrange(n), rng.randrange(n)) for _ in range(m)]


@pytest.mark.parametrize("seed", range(12))
def test_cas_unions_under_interleavings(seed):
    """Concurrent unions along random edges (the join and the outside-node scan) give the
    components of the forest plus those edges, whatever the interleaving, even when the quick
    check sees stale labels (a stale label is still an ancestor, so equal ones prove one set)."""
    rng = random.Random(100 + seed)
    n = rng.choice([30, 80, 160])
    L = random_forest(n, rng)
    edges = random_edges(n // 2, 2 * n, rng)  # repeated ends, so cached labels are reused
    want = components(n, L, edges)
    work = [(a, b) for a, b in edges if L[a] != DEAD and L[b] != DEAD]
    chunks = [work[i::8] for i in range(8)]

    def thread(es):
        # the join's quick check reads the two labels through L1, which may return a value this
        # thread saw earlier: modelled by a per-thread cache that answers half of the repeat reads
        cache = {}
        for a, b in es:
            lab = []
            for x in (a, b):
                if x in cache and rng.random() < 0.5:
                    lab.append(cache[x])
                else:
                    yield
                    cache[x] = L[x]
                    lab.append(cache[x])
            la, lb = lab
            if la == lb:
                continue
            yield from unite(L, la, lb)

    run_interleaved([thread(c) for c in chunks], rng)
    assert same_partition(L, want)
    assert all(L[v] == DEAD or L[v] <= v for v in range(n))  # labels still point downwards


def adjacency(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        if a != b and b not in adj[a]:
            adj[a].append(b)
            adj[b].append(a)
    return adj


@pytest.mark.parametrize("seed", range(12))
def test_neighbour_sampling_under_interleavings(seed):
    """The sampling step: every live node looks at its first four adjacency entries, reads their
    labels before any union, and unites with up to two live neighbours unless a label read early
    equals its own current one.  The result is exactly the forest plus the edges to those (up to
    two) live neighbours: a skipped union was already implied."""
    rng = random.Random(200 + seed)
    n = rng.choice([40, 90, 170])
    L = random_forest(n, rng, p_dead=0.3, p_root=0.4)
    adj = adjacency(n, random_edges(n, 3 * n, rng))
    sampled = []
    for v in range(n):
        if L[v] == DEAD:
            continue
        live_nb = [w for w in adj[v][:4] if L[w] != DEAD][:2]
        sampled += [(v, w) for w in live_nb]
    want = components(n, L, sampled)

    def thread(nodes):
        for v in nodes:
            yield
            if L[v] == DEAD:
                continue
            nb = adj[v][:4]
            lw = []
            for w in nb:  # labels of the first entries, loaded together
                yield
                lw.append(L[w])
            linked = 0
            for w, x in zip(nb, lw):
                if linked >= 2 or x == DEAD:
                    continue
                yield
                if x != L[v]:
                    yield from unite(L, v, w)
                linked += 1

    run_interleaved([thread(items) for items in grid_stride(n, rng.choice([4, 16]))], rng)
    assert same_partition(L, want)


def test_models_detect_a_wrong_walk():
    """The flatten model is sharp: a walk that stopped only at self-pointing labels (ignoring
    counters) would run through a root turned into -1 and index with it.  Some interleaving
    exposes that, as an index out of range or as a wrong label."""
    failures = 0
    for seed in range(40):
        rng = random.Random(seed)
        n = 64
        L = random_forest(n, rng, p_dead=0.1, p_root=0.05)
        want = roots_of(L)

        def bad_thread(items):
            for v in items:
                yield
                pv = L[v]
                if pv == DEAD:
                    continue
                if pv == v:
                    yield
                    L[v] = -1
                    continue
                x = pv
                yield
                p = L[x]
                while p != x:  # no stop at a counter
                    x = p
                    if not 0 <= x < n:
                        raise IndexError("the walk left the label array")
                    yield
                    p = L[x]
                yield
                L[v] = x

        try:
            run_interleaved([bad_thread(items) for items in grid_stride(n, 16)], rng)
            ok = all(want[v] == DEAD or L[v] == (-1 if want[v] == v else want[v]) for v in range(n))
        except IndexError:
            ok = False
        failures += not ok
    assert failures > 0


def test_models_detect_a_non_atomic_hook():
    """The union model is sharp too: hooking a root by a plain read and a later store, instead of
    one compare-and-swap, loses unions in some interleaving."""
    def bad_unite(L, a, b):
        a = yield from find(L, a)
        b = yield from find(L, b)
        while a != b:
            if a < b:
                a, b = b, a
            yield
            old = L[a]
            if old == a:
                yield  # another thread may hook a in between
                L[a] = b
                return
            a = yield from find(L, old)
            b = yield from find(L, b)

    failures = 0
    for seed in range(40):
        rng = random.Random(300 + seed)
        n = 60
        L = random_forest(n, rng, p_dead=0.0, p_root=0.6)
        edges = random_edges(n, n, rng)
        want = components(n, L, edges)

        def thread(es):
            for a, b in es:
                yield from bad_unite(L, a, b)

        run_interleaved([thread(edges[i::8]) for i in range(8)], rng)
        failures += not same_partition(L, want)
    assert failures > 0


# ---------------------------------------------------------------------------
# The sparse kernel's class union-find: values are terminal + 1 with 0 = R (the reference class,
# never hooked); the larger root hooks under the smaller by compare-and-swap, and a find points
# the links on its path that still lie below the root it found straight at that root, stopping at
# the first link at or above it.

def sp_find(C, a, bound=True):
    r = a
    while r != 0:
        p = C[r - 1]
        yield
        if p == r:
            break
        r = p
    while (a > r) if bound else (a != r):
        if a == 0:
            raise IndexError("link of R read")
        p = C[a - 1]
        yield
        if bound and p <= r:  # the kernel's stop: never write r above itself
            break
        if not bound and (p == a or p == r):  # a stop that lets the walk pass r
            break
        C[a - 1] = r
        yield
        a = p
    return r


def sp_unite(C, a, b, bound=True):
    a = yield from sp_find(C, a, bound)
    b = yield from sp_find(C, b, bound)
    while a != b:
        if a < b:
            a, b = b, a
        old = C[a - 1]
        if old == a:
            C[a - 1] = b  # compare-and-swap: one step
            yield
            return
        yield
        a = yield from sp_find(C, old, bound)
        b = yield from sp_find(C, b, bound)


def sp_classes(m, pairs):
    """Sequential classes of m terminals (values 1..m) and R (0) under the pairs."""
    parent = list(range(m + 1))

    def f(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for a, b in pairs:
        ra, rb = f(a), f(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    return [f(x) for x in range(m + 1)]


def sp_check(C, want):
    m = len(C)
    got = [0] * (m + 1)
    for v in range(1, m + 1):
        x, steps = v, 0
        while x != 0 and C[x - 1] != x:
            assert C[x - 1] < x, "a link points up"
            x = C[x - 1]
            steps += 1
            assert steps <= m, "a cycle"
        got[v] = x
    for a in range(m + 1):
        for b in range(m + 1):
            assert (got[a] == got[b]) == (want[a] == want[b])


@pytest.mark.parametrize("seed", range(40))
def test_sparse_class_unions_under_interleavings(seed):
    """Unions of terminal classes, some with R, by many threads at once (linking, then the join's
    unions with R): the classes equal the sequential ones, links only point down, no cycles."""
    rng = random.Random(seed)
    m = rng.randrange(4, 40)
    pairs = []
    for _ in range(rng.randrange(m, 3 * m)):
        a = rng.randrange(1, m + 1)
        b = 0 if rng.random() < 0.15 else rng.randrange(1, m + 1)
        pairs.append((a, b))
    C = list(range(1, m + 1))
    threads = [sp_unite(C, a, b) for a, b in pairs]
    # interleave in a few threads per "warp": every pair is a thread here
    run_interleaved([t for t in threads], rng)
    sp_check(C, sp_classes(m, pairs))


def test_sparse_class_models_detect_compression_past_the_root():
    """The earlier stop rule (break only at a root or at the root found) lets a find walk above the
    root it found once another thread has compressed past it, writing that root into an ancestor
    (a cycle) or reading the link of R; the interleavings find it."""
    failures = 0
    for seed in range(300):
        rng = random.Random(seed)
        m = rng.randrange(4, 12)
        pairs = [(rng.randrange(1, m + 1), 0 if rng.random() < 0.3 else rng.randrange(1, m + 1))
                 for _ in range(4 * m)]
        C = list(range(1, m + 1))
        threads = [sp_unite(C, a, b, bound=False) for a, b in pairs]
        try:
            run_interleaved(threads, rng)
            sp_check(C, sp_classes(m, pairs))
        except (AssertionError, IndexError, RecursionError):
            failures += 1
    assert failures > 0
