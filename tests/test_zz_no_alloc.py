"""The allocation-free fitness entry point (gapa_fitness_noalloc).

It serves callers that cannot allocate device memory: a library embedded in a
host program whose device memory belongs to that program's allocator under a
fixed budget, and latency-critical loops that cannot take the device-wide
synchronisation of cudaMalloc.  Its label scratch is a static array in the
library, shared by every call.  These tests call it through the C ABI on two
calls in a row - so that the labels left behind by one call cannot leak into
the next - and compare each result with the CPU oracle and with the
context-based gapa_fitness on the same inputs.  Fitness is an integer, so the
comparisons are exact.

The file name sorts last so that, in a run that stops at the first failure,
every other test has already run; the tests need no state from other files
and pass in a fresh process as well as after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _edges_on_device(g):
    import torch

    u, v = g.edge_list()
    return torch.from_numpy(np.stack([u, v], axis=1).astype(np.int32)).cuda()


def _context_fitness(g, pop):
    from paper_2412_20980_gb300 import Context

    with Context(0) as ctx:
        ctx.graph_upload(g.row_ptr, g.col)
        f = ctx.fitness(pop)
        ctx.sync()
        return f.cpu().numpy()


@pytest.mark.parametrize("make,k,s", [
    (lambda: synth.ba_graph(20000, 4, 1), 1000, 300),   # one wave
    (lambda: synth.ba_graph(100000, 3, 1), 2000, 200),  # 83 members per wave: three waves
])
def test_noalloc_matches_oracle_and_context_entry_point_twice(make, k, s):
    import torch

    from paper_2412_20980_gb300 import build as b
    from paper_2412_20980_gb300.gapa import fitness_noalloc

    b.build()
    g = make()
    edges = _edges_on_device(g)
    for call, seed in enumerate((11, 12)):
        pop_np = synth.random_deletion_sets(g.n, k, s, seed)
        pop = torch.from_numpy(pop_np).cuda()
        out = torch.full((s,), -1, dtype=torch.int64, device="cuda")
        fitness_noalloc(edges, pop, g.n, out)
        got = out.cpu().numpy()
        assert np.array_equal(got, oracle.fitness(g.row_ptr, g.col, pop_np)), f"call {call}: oracle"
        assert np.array_equal(got, _context_fitness(g, pop)), f"call {call}: gapa_fitness"


def test_noalloc_rejects_oversize_and_bad_input():
    import torch

    from paper_2412_20980_gb300 import GapaError
    from paper_2412_20980_gb300 import build as b
    from paper_2412_20980_gb300.gapa import fitness_noalloc

    b.build()
    edges = torch.tensor([[0, 1], [1, 2]], dtype=torch.int32, device="cuda")
    pop = torch.tensor([[0]], dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(GapaError) as ei:
        fitness_noalloc(edges, pop, 8 * 1024 * 1024 + 1, out)
    assert ei.value.code == -1
    bad = torch.tensor([[0, 1], [1, 7]], dtype=torch.int32, device="cuda")
    with pytest.raises(GapaError) as ei:
        fitness_noalloc(bad, pop, 3, out)
    assert ei.value.code == -7
    # the status word is cleared by the next call: path 0-1-2 with node 0 deleted leaves {1,2}
    fitness_noalloc(edges, pop, 3, out)
    assert out.item() == 1
    # a gene equal to n is rejected on the device, and again the next call starts clean
    with pytest.raises(GapaError) as ei:
        fitness_noalloc(edges, torch.tensor([[3]], dtype=torch.int32, device="cuda"), 3, out)
    assert ei.value.code == -7
    fitness_noalloc(edges, torch.tensor([[2]], dtype=torch.int32, device="cuda"), 3, out)
    assert out.item() == 1
    # an output shorter than the population is refused before any launch
    with pytest.raises(ValueError):
        fitness_noalloc(edges, torch.zeros((2, 1), dtype=torch.int32, device="cuda"), 3, out)


def test_noalloc_k0_and_empty_population():
    import torch

    from paper_2412_20980_gb300 import build as b
    from paper_2412_20980_gb300.gapa import fitness_noalloc

    b.build()
    g = synth.ba_graph(5000, 3, 4)  # connected: k = 0 gives C(n, 2) for every member
    edges = _edges_on_device(g)
    s = 7
    out = torch.full((s,), -1, dtype=torch.int64, device="cuda")
    fitness_noalloc(edges, torch.zeros((s, 0), dtype=torch.int32, device="cuda"), g.n, out)
    assert out.cpu().tolist() == [g.n * (g.n - 1) // 2] * s
    # s = 0: returns without touching the output
    sentinel = torch.full((3,), -5, dtype=torch.int64, device="cuda")
    fitness_noalloc(edges, torch.zeros((0, 4), dtype=torch.int32, device="cuda"), g.n, sentinel)
    assert sentinel.cpu().tolist() == [-5, -5, -5]
