"""The allocation-free fitness entry point (gapa_fitness_noalloc).

It serves callers that must not allocate device memory - code running while a
framework captures the stream into a CUDA graph, latency-critical loops that
cannot take cudaMalloc's implicit synchronisation, processes whose device
memory belongs to another allocator.  Its label scratch is a static array in
the library, shared by every call.  These tests call it through the C ABI and
compare it with the context-based gapa_fitness on the same inputs, twice in a
row, so that the scratch left behind by one call cannot leak into the next.
Fitness is an integer, so the comparison is exact.

The file name sorts last so that, in a run that stops at the first failure,
every other test has already run; the tests need no state from other files.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _edges_on_device(g):
    import torch

    u, v = g.edge_list()
    return torch.from_numpy(np.stack([u, v], axis=1).astype(np.int32)).cuda()


def _reference(g, pop):
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
def test_noalloc_matches_context_entry_point_twice(make, k, s):
    import torch

    from paper_2412_20980_gb300 import build as b
    from paper_2412_20980_gb300.gapa import fitness_noalloc

    b.build()
    g = make()
    edges = _edges_on_device(g)
    for call, seed in enumerate((11, 12)):
        pop = torch.from_numpy(synth.random_deletion_sets(g.n, k, s, seed)).cuda()
        out = torch.full((s,), -1, dtype=torch.int64, device="cuda")
        fitness_noalloc(edges, pop, g.n, out)
        assert np.array_equal(out.cpu().numpy(), _reference(g, pop)), f"call {call}"


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
    # still usable afterwards: path 0-1-2 with node 0 deleted leaves {1,2}
    fitness_noalloc(edges, pop, 3, out)
    assert out.item() == 1
