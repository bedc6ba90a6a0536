"""Multi-rank host logic on CPU (gloo, world size 2): the job's time is the slowest rank's, the
value counts every rank's units, the reference arm runs on rank 0 only, and the batched
crystals are sharded across ranks (each rank computes the same longest-processing-time-first
assignment; together the ranks cover every system exactly once).  No GPU is touched."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [1000.0, 1250.0][rank]
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    q.put((rank, t, bench.job_throughput(world, 3, 27648.0 ** 2, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1250.0, 1250.0]          # slowest rank, seen by both
    expect = 2 * 3 * 27648.0 ** 2 / 1.25                      # both ranks' units / max time
    assert all(abs(o[2] - expect) <= 1e-9 * expect for o in out)


def test_reference_arm_is_silent_on_nonzero_rank():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def _shard_rank(rank: int, world: int, port: int, q):
    from paper_2607_05853_b300.shard import assembly_work, assign_systems
    from synth import batched_specs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    works = [assembly_work(sp.n_k, sp.n_aux, sp.nv, sp.nc) for sp in batched_specs(16)]
    mine = assign_systems(works, world)[rank]
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)     # what each rank will assemble
    q.put((rank, mine, everyone, works))
    dist.barrier()
    dist.destroy_process_group()


def test_batched_systems_sharded_across_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (_, m0, e0, works), (_, m1, e1, _) = out
    assert e0 == e1 == [m0, m1]                               # both ranks agree without negotiating
    assert sorted(m0 + m1) == list(range(16))                 # every system exactly once
    assert all(works[a] <= works[b] for m in (m0, m1) for a, b in zip(m, m[1:]))   # SJF inside a rank
    loads = [sum(works[i] for i in m) for m in (m0, m1)]
    bound = max(sum(works) / 2, max(works))                   # no assignment beats this
    assert max(loads) <= 4.0 / 3.0 * bound                    # the LPT guarantee
