"""The member split of Section III-D (SM mode) on NCCL with device tensors, under torchrun.

One rank (this machine has one GPU per job): the generation runs as operators + fitness of the
rank's slice + an NCCL all-gather of the int64 fitness, ordered on the context's stream with no
host synchronisation, and must equal both the plain gapa_generation and the oracle bit-exactly.
Ranks whose collectives wait on one another are never run on one GPU; the two- and three-rank
split is covered on CPU by tests/test_dist_gloo.py.
"""
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import os, sys
sys.path.insert(0, os.environ["GAPA_ROOT"])
import numpy as np
import torch
import torch.distributed as dist

import oracle
import synth
from paper_2412_20980_gb300 import Context, make_config
from paper_2412_20980_gb300 import dist as gd

local = int(os.environ["LOCAL_RANK"])
torch.cuda.set_device(local)
dist.init_process_group("nccl", device_id=torch.device("cuda", local))
assert dist.get_world_size() == 1
g = synth.ba_graph(20000, 4, 1)
cfg = make_config(k=1000, pop=256, tourn=2, pc=0.8, pm=0.02, seed=4)
with Context(local) as ctx:
    ctx.graph_upload(g.row_ptr, g.col)
    pop = ctx.pop_init(cfg)
    fit = ctx.fitness(pop)
    ref_p, ref_f = pop.clone(), fit.clone()
    want_p, want_f = pop.cpu().numpy(), fit.cpu().numpy()
    for gen in range(1, 4):
        nxt_p, nxt_f = torch.empty_like(pop), torch.full_like(fit, -1)
        gd.sharded_generation(ctx, cfg, gen, pop, fit, nxt_p, nxt_f)
        r_p, r_f = ctx.generation(cfg, gen, ref_p, ref_f)
        want_p, want_f = oracle.generation(g.row_ptr, g.col, want_p, want_f, gen, tourn=2, pc_thr=cfg.pc_thr,
                                           pm_thr=cfg.pm_thr, seed=cfg.seed, nthreads=oracle.max_threads())
        ctx.sync()
        assert torch.equal(nxt_p, r_p) and torch.equal(nxt_f, r_f), f"split != gapa_generation at {gen}"
        assert np.array_equal(nxt_p.cpu().numpy(), want_p), f"population != oracle at {gen}"
        assert np.array_equal(nxt_f.cpu().numpy(), want_f), f"fitness != oracle at {gen}"
        pop, fit, ref_p, ref_f = nxt_p, nxt_f, r_p, r_f
dist.destroy_process_group()
print("SPLIT_NCCL_OK")
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_split_generation_under_torchrun_nccl(tmp_path):
    from paper_2412_20980_gb300 import build as b

    b.build()
    script = tmp_path / "split_rank.py"
    script.write_text(RANK_SCRIPT)
    env = dict(os.environ, GAPA_ROOT=ROOT, NCCL_NVLS_ENABLE="0")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=1",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", str(script)]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "SPLIT_NCCL_OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
