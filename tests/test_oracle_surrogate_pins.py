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
    deg = sr.degrees_from_csr(g.row_ptr)
    loss, grads, _ = sr.loss_and_grads(params, pop, t, deg, g.num_edges)
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
            lp, _, _ = sr.loss_and_grads(params, pop, t, deg, g.num_edges)
            p[ix] = old - h
            lm, _, _ = sr.loss_and_grads(params, pop, t, deg, g.num_edges)
            p[ix] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[name][ix]) <= 1e-6 + 1e-5 * abs(fd), (name, ix, fd, grads[name][ix])


def test_features_closed_forms():
    g = synth.named_graph("star", 9)
    deg = sr.degrees_from_csr(g.row_ptr)  # centre 8, leaves 1
    E = np.zeros((9, sr.EMB))
    E[0, 0] = 3.0
    E[4, 1] = 2.0
    x = sr.features(np.array([[0, 4]]), E, deg, g.num_edges)[0]
    assert np.isclose(x[0], 3 / np.sqrt(2)) and np.isclose(x[1], 2 / np.sqrt(2))
    q = np.log1p([8.0, 1.0])
    assert np.isclose(x[64], q.mean()) and np.isclose(x[65], q.max())
    assert np.isclose(x[66], np.std(q)) and np.isclose(x[67], 9 / 16)
    assert np.all(x[68:] == 0)


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
