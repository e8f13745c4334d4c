"""Pins of the fp64 surrogate reference: central finite differences for every
gradient, the closed form of the first AdamW step, and Spearman on known cases."""
import numpy as np

import synth
from oracle import surrogate_ref as sr


def _setup(seed=0, n=60, k=6, B=9):
    g = synth.ba_graph(n, 2, 3)
    rng = np.random.default_rng(seed)
    params = {
        "W1": rng.normal(0, 0.3, (sr.IN, sr.HID)), "b1": rng.normal(0, 0.1, sr.HID),
        "W2": rng.normal(0, 0.1, (sr.HID, sr.HID)), "b2": rng.normal(0, 0.1, sr.HID),
        "w3": rng.normal(0, 0.1, sr.HID), "b3": rng.normal(0, 0.1, 1),
        "E": rng.normal(0, 0.5, (n, sr.EMB)),
    }
    pop = np.stack([rng.choice(n, k, replace=False) for _ in range(B)]).astype(np.int32)
    t = rng.normal(0, 1, B)
    return g, params, pop, t


def test_gradients_match_central_differences():
    g, params, pop, t = _setup()
    loss, grads, _ = sr.loss_and_grads(params, pop, t, g.row_ptr, g.col)
    rng = np.random.default_rng(1)
    h = 1e-6
    for name, p in params.items():
        idx = [tuple(rng.integers(0, s) for s in p.shape) for _ in range(6)]
        if name == "E":  # rows that occur in the batch, and one that does not
            idx = [(int(pop[0, 0]), 3), (int(pop[2, 1]), 40), (int(pop[5, 4]), 63)]
            absent = next(v for v in range(g.n) if v not in set(pop.ravel().tolist()))
            idx.append((absent, 7))
        for ix in idx:
            old = p[ix]
            p[ix] = old + h
            lp, _, _ = sr.loss_and_grads(params, pop, t, g.row_ptr, g.col)
            p[ix] = old - h
            lm, _, _ = sr.loss_and_grads(params, pop, t, g.row_ptr, g.col)
            p[ix] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[name][ix]) <= 1e-6 + 1e-5 * abs(fd), (name, ix, fd, grads[name][ix])


def test_features_closed_forms():
    g = synth.named_graph("star", 9)  # centre 0 (degree 8), leaves 1..8
    E = np.zeros((9, sr.EMB))
    E[0, 0] = 3.0
    E[4, 1] = 2.0
    x = sr.features(np.array([[0, 4]]), E, g.row_ptr, g.col)[0]
    assert np.isclose(x[0], 3 / np.sqrt(2)) and np.isclose(x[1], 2 / np.sqrt(2))
    q = np.log1p([8.0, 1.0])
    assert np.isclose(x[64], q.mean()) and np.isclose(x[65], q.max())
    assert np.isclose(x[66], np.std(q)) and np.isclose(x[67], 9 / 16)
    # deleting the centre isolates the 7 live leaves; none keeps exactly one live neighbour
    assert np.isclose(x[68], np.log1p(7)) and x[69] == 0 and x[70] == 0
    assert np.all(x[71:] == 0)


def test_standardised_counts_closed_forms():
    z = sr.standardised_counts([[0, 3, 7], [2, 3, 7]])  # r0: mean 1, sd 1; r1, r2 constant
    assert z[:, 0].tolist() == [-1.0, 1.0] and np.all(z[:, 1:] == 0)
    z = sr.standardised_counts([[0, 0, 0], [0, 0, 0], [0, 0, 0], [1, 0, 0]])  # sd 0.433 < 1: divided by 1
    assert z[:, 0].tolist() == [-0.25, -0.25, -0.25, 0.75]
    z = sr.standardised_counts([[0, 0, 0], [10, 0, 0]])  # mean 5, sd 5
    assert z[:, 0].tolist() == [-1.0, 1.0]
    # features standardise over the rows passed together: star with centre 0 and 5 leaves
    g = synth.named_graph("star", 6)
    x = sr.features(np.array([[0], [1], [2], [3]]), np.zeros((6, sr.EMB)), g.row_ptr, g.col)
    # r0 = 5, 0, 0, 0: mean 1.25, sd sqrt(25/4 - 1.5625) = 2.165
    sd = np.sqrt(25 / 4 - 1.25 ** 2)
    assert np.allclose(x[:, 71], (np.array([5, 0, 0, 0]) - 1.25) / sd, atol=1e-6)
    assert np.all(x[:, 72:] == 0)


def test_residual_degree_counts_closed_forms():
    path = synth.named_graph("path", 5)  # 0-1-2-3-4
    assert sr.residual_degree_counts(path.row_ptr, path.col, []) == (0, 0, 0)  # the ends were pendant already
    assert sr.residual_degree_counts(path.row_ptr, path.col, [2]) == (0, 2, 2)  # 1 and 3; the pairs {0,1} and {3,4}
    assert sr.residual_degree_counts(path.row_ptr, path.col, [1, 3]) == (3, 0, 0)
    assert sr.residual_degree_counts(path.row_ptr, path.col, [0]) == (0, 1, 0)
    # a node of degree 0 is never counted: it has no deleted neighbour
    lone = synth.graphs.disjoint_union(synth.named_graph("path", 2), synth.named_graph("path", 1))
    assert sr.residual_degree_counts(lone.row_ptr, lone.col, []) == (0, 0, 0)
    assert sr.residual_degree_counts(lone.row_ptr, lone.col, [0]) == (1, 0, 0)
    star = synth.named_graph("star", 6)  # centre 0
    assert sr.residual_degree_counts(star.row_ptr, star.col, [1]) == (0, 0, 0)  # the centre keeps 4 leaves
    assert sr.residual_degree_counts(star.row_ptr, star.col, [1, 2, 3, 4]) == (0, 1, 1)  # {0, 5} is left
    assert sr.residual_degree_counts(star.row_ptr, star.col, [0]) == (5, 0, 0)


def test_residual_degree_counts_brute_force():
    """Adjacency-list loops over every node on small random graphs and deletion sets."""
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(2, 40))
        g = synth.er_graph(n, int(rng.integers(0, min(2 * n, n * (n - 1) // 2) + 1)), seed=trial)
        k = int(rng.integers(0, n))
        genes = rng.choice(n, k, replace=False)
        dead = set(genes.tolist())
        r0 = r1 = 0
        for u in range(n):
            if u in dead:
                continue
            nb = g.col[g.row_ptr[u]:g.row_ptr[u + 1]].tolist()
            live = sum(1 for w in nb if w not in dead)
            if live < len(nb):  # u has a deleted neighbour
                r0 += int(live == 0)
                r1 += int(live == 1)
        # two-node components by a BFS over the live graph
        seen, r2 = set(), 0
        for u in range(n):
            if u in dead or u in seen:
                continue
            comp, stack = [], [u]
            seen.add(u)
            while stack:
                x = stack.pop()
                comp.append(x)
                for w in g.col[g.row_ptr[x]:g.row_ptr[x + 1]].tolist():
                    if w not in dead and w not in seen:
                        seen.add(w)
                        stack.append(w)
            if len(comp) == 2:
                touches = any(w in dead for x in comp for w in g.col[g.row_ptr[x]:g.row_ptr[x + 1]].tolist())
                r2 += int(touches)
        assert sr.residual_degree_counts(g.row_ptr, g.col, genes) == (r0, r1, r2)


def test_first_adamw_step_closed_form():
    # tau = 1: m_hat = g, v_hat = g^2, so p <- p - lr * (g / (|g| + eps) + wd * p)
    p = {"a": np.array([1.0, -2.0, 0.5, 3.0])}
    g = {"a": np.array([0.3, -4.0, 0.0, 1e-3])}
    want = p["a"] - 1e-3 * (g["a"] / (np.abs(g["a"]) + 1e-8) + 0.01 * p["a"])
    sr.adamw_step(p, g, {}, 1)
    assert np.allclose(p["a"], want, rtol=0, atol=1e-15)


def test_spearman_known_values():
    assert sr.spearman([1, 2, 3, 4], [10, 20, 30, 40]) == 1.0
    assert sr.spearman([1, 2, 3, 4], [4, 3, 2, 1]) == -1.0
    # textbook case with no ties: 1 - 6 sum d^2 / (n (n^2 - 1)) = 1 - 6*2/(5*24) = 0.9
    assert np.isclose(sr.spearman([1, 2, 3, 4, 5], [2, 1, 3, 4, 5]), 0.9)


# --- the BF16-stored variant (the GPU's storage roundings) -------------------------------------

def test_round_bf16_hand_worked_and_against_torch():
    # hand-worked: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 and goes to the even one (1.0);
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6 and goes to 1 + 2^-6 (even);
    # 1 + 2^-8 + 2^-20 is above halfway and rounds up; representable values stay
    cases = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6, 1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7,
             -3.0: -3.0, 0.0: 0.0, 2 ** -130: 2 ** -130}
    got = sr.round_bf16(np.array(list(cases), dtype=np.float32))
    assert got.tolist() == list(cases.values())
    torch = __import__("pytest").importorskip("torch")
    x = np.random.default_rng(3).normal(0, 10, 4096).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(sr.round_bf16(x), want)


def test_stored_variant_without_rounding_is_the_reference():
    g, params, pop, t = _setup(seed=5)
    loss, grads, y = sr.loss_and_grads(params, pop, t, g.row_ptr, g.col)
    loss2, grads2, y2 = sr.loss_and_grads_stored(params, pop, t, g.row_ptr, g.col, rnd=lambda a: np.asarray(a))
    assert loss2 == loss and np.array_equal(y2, y)
    for name in grads:
        assert np.array_equal(grads2[name], grads[name]), name


def test_stored_variant_rounds_only_by_bf16_amounts():
    """The BF16 roundings move the scores by about the BF16 unit roundoff (2^-9 relative per
    stored value) and the gradients by a few per cent, never more than 10 % in relative L2 norm
    with cosine >= 0.99 (a bug in a rounding point - a wrong mask, a dropped layer - moves them
    by order one)."""
    g, params, pop, t = _setup(seed=6, n=120, k=10, B=24)
    _, grads, y = sr.loss_and_grads(params, pop, t, g.row_ptr, g.col)
    _, grads2, y2 = sr.loss_and_grads_stored(params, pop, t, g.row_ptr, g.col)
    assert np.linalg.norm(y2 - y) / np.linalg.norm(y) < 2e-2
    for name in grads:
        a, b = np.ravel(grads2[name]), np.ravel(grads[name])
        if np.linalg.norm(b) == 0:
            assert np.linalg.norm(a) == 0, name
            continue
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 0.1, name
        assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b)) >= 0.99, name
