"""Multi-rank path on the CPU (gloo, world size 2): each rank evaluates its
share of the task list with the CPU oracle, and one all-reduce of the three
energies equals the whole job.  Also checks the weak-scaling batches."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1609_08094_gb300 import partition


def test_rank_ranges_cover_the_list():
    for ntask in (0, 1, 7, 20, 22100):
        for world in (1, 2, 3, 8):
            spans = [partition.rank_range(ntask, r, world) for r in range(world)]
            assert spans[0][0] == 0
            for (f0, c0), (f1, _) in zip(spans, spans[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in spans) == ntask
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def test_step_batches_disjoint_across_ranks():
    ntask, count = 22100, 4
    for world in (2, 4, 8):
        for step in range(10):
            firsts = [partition.step_batch(ntask, r, world, step, count) for r in range(world)]
            sets = [set(range(f, f + count)) for f in firsts]
            assert all(f + count <= ntask for f in firsts)
            assert sum(len(s) for s in sets) == len(set().union(*sets))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch

    import oracle
    from paper_1609_08094_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = synth.make_instance(5, 9, None, 77)
    tasks = oracle.sorted_triples(5)
    first, count = partition.rank_range(len(tasks), rank, world)
    e = oracle.triple_energies(inst, tasks[first:first + count], nthreads=1)
    t = torch.tensor([e[:, 0].sum(), e[:, 1].sum()], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        out.put(t.numpy().tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_sum_to_the_whole_job(oracle_lib):
    import oracle
    from paper_1609_08094_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = oracle.energy(synth.make_instance(5, 9, None, 77))
    assert np.allclose(got, ref[:2], rtol=1e-13, atol=0)
