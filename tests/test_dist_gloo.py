"""The multi-process host logic on CPU: two and three gloo ranks.

Independent populations (the benchmark's N > 1 mode) need only the rank seeds
and the max-over-ranks timing; a population split by members needs the shard
bounds and the all-gather of fitness slices.  The split generation runs here
with the oracle standing in for the device (offspring = the oracle's
generation with the children's fitness erased, fitness = the oracle's), and
must equal the oracle's unsplit generation on both ranks.
"""
import os
import socket

import numpy as np
import pytest

from paper_2412_20980_gb300 import dist as gd


def test_shard_bounds_cover_exactly():
    for total in (0, 1, 7, 1023, 1024):
        for world in (1, 2, 3, 8):
            spans = [gd.shard_bounds(total, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        gd.shard_bounds(5, 2, 2)


class _OracleCtx:
    """offspring()/fitness() with the oracle on host tensors; records which rows it evaluated."""

    def __init__(self, g):
        self.g = g
        self.rows = 0

    def offspring(self, cfg, gen, pop_in, fit_in, pop_out, fit_out):
        import torch

        import oracle

        pop, fit = oracle.generation(self.g.row_ptr, self.g.col, pop_in.numpy(), fit_in.numpy(), gen,
                                     tourn=cfg.tourn, pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr, seed=cfg.seed)
        pop_out.copy_(torch.from_numpy(pop))
        fit_out.fill_(-1)
        fit_out[0] = int(fit[0])

    def fitness(self, pop, out):
        import torch

        import oracle

        self.rows += pop.shape[0]
        out.copy_(torch.from_numpy(oracle.fitness(self.g.row_ptr, self.g.col, pop.numpy())))

    def sync(self):
        pass


def _rank_main(rank, world, port, result_dir):
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2412_20980_gb300 import make_config

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # independent populations: seeds differ, the slowest rank's time is the job's
        assert gd.rank_seed(5, rank) == 5 + rank
        assert gd.max_over_ranks(10.0 * (rank + 1)) == 10.0 * world
        # a population split by members
        g = synth.ba_graph(600, 3, 2)
        cfg = make_config(k=30, pop=41, tourn=2, pc=0.8, pm=0.05, seed=9)
        pop = oracle.pop_init(g.n, cfg.k, cfg.pop, cfg.seed)
        fit = oracle.fitness(g.row_ptr, g.col, pop)
        want_pop, want_fit = pop, fit
        ctx = _OracleCtx(g)
        cur_p, cur_f = torch.from_numpy(pop.copy()), torch.from_numpy(fit.copy())
        for gen in range(1, 4):
            nxt_p, nxt_f = torch.empty_like(cur_p), torch.empty_like(cur_f)
            gd.sharded_generation(ctx, cfg, gen, cur_p, cur_f, nxt_p, nxt_f)
            want_pop, want_fit = oracle.generation(g.row_ptr, g.col, want_pop, want_fit, gen, tourn=cfg.tourn,
                                                   pc_thr=cfg.pc_thr, pm_thr=cfg.pm_thr, seed=cfg.seed)
            assert np.array_equal(nxt_p.numpy(), want_pop) and np.array_equal(nxt_f.numpy(), want_fit), gen
            cur_p, cur_f = nxt_p, nxt_f
        lo, hi = gd.shard_bounds(cfg.pop - 1, world, rank)
        assert ctx.rows == 3 * (hi - lo)  # each rank evaluated only its slice
        open(os.path.join(result_dir, f"ok{rank}"), "w").write("ok")
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks(tmp_path, world):
    """Two ranks split the 40 children 20/20; three ranks split them 14/13/13 (uneven slices)."""
    import torch.multiprocessing as mp

    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    assert sorted(os.listdir(tmp_path)) == [f"ok{r}" for r in range(world)]
