"""Parity at the full workload size (o=50, v=450, naux=1500, seed 2; one vvvo
slice is 729 MB in FP64) on sampled tasks, through the C ABI (GPU).

The batches are the ones the benchmark times first: 4 tasks per step for
FP64 and 64 for the tensor-core paths, 3 warm-up steps, at the step offsets
of the task partition.  Every precision returns per-task (E[4], E[5]) shares
for its whole batch; the oracle recomputes two non-diagonal tasks of each
batch from the vvvo slices they touch (the per-task energy e_ijk of the
restricted loop, Sec. 3), so the whole sample costs the oracle about 4 x
5.5e11 flop.  Tolerances: 1e-10 relative per task for FP64 and the FP64
emulation, 1e-6 for TF32x3 and BF16x3."""
import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import partition, synth, tcorr

pytestmark = pytest.mark.gpu

O, V, NAUX, SEED = 50, 450, 1500, 2
WARMUP = 3
TOL = {"fp64": 1e-10, "fp64_oz": 1e-10, "tf32x3": 1e-6, "bf16x3": 1e-6}


@pytest.fixture(scope="module")
def full():
    from paper_1609_08094_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    inst = synth.make_instance(O, V, NAUX, SEED, device=torch.device("cuda"))
    torch.cuda.synchronize()
    yield inst
    del inst
    torch.cuda.empty_cache()


def oracle_tasks(inst, tasks):
    """Oracle (E[4], E[5]) of the given sorted triples, from host copies of
    the small arrays and of the vvvo slices the tasks read."""
    need = sorted({int(q) for t in tasks for q in t})
    host = synth.Instance(O, V, NAUX, SEED, inst.eps_occ.cpu().numpy(), inst.eps_vir.cpu().numpy(),
                          inst.t1.cpu().numpy(), inst.t2.cpu().numpy(), None,
                          inst.ooov.cpu().numpy(), inst.ovov.cpu().numpy())
    slices = {q: inst.vvvo[:, :, :, q].contiguous().cpu().numpy() for q in need}
    return oracle.triple_energies(host, np.asarray(tasks, dtype=np.int32), oracle.max_threads(), slices=slices)


def sample_batch(t, count, nsample=2):
    """First task of the first timed batch of ``count`` tasks and the batch
    positions of ``nsample`` tasks in it that are not i = j = k, spread
    across the batch."""
    ntask = t.num_tasks
    first = partition.step_batch(ntask, 0, 1, WARMUP, count)
    pos = [n for n in range(count) if len(set(t.task(first + n))) > 1]
    pick = [pos[0], pos[-1]] if nsample == 2 and len(pos) > 1 else pos[:nsample]
    return first, pick


def check(prec, inst, count):
    with tcorr.Tcorr.from_instance(inst, prec=prec) as t:
        first, pick = sample_batch(t, count)
        tasks = [t.task(first + n) for n in pick]
        tot, per = t.energy_range(first, count, per_task=True)
    assert np.isclose(per.sum(), tot[2], rtol=1e-12, atol=0.0)
    return tasks, per[pick]


def test_full_size_fp64_sampled_tasks(full):
    tasks, got = check("fp64", full, 4)
    ref = oracle_tasks(full, tasks)
    for tk, g, r in zip(tasks, got, ref):
        err = abs(g.sum() - r.sum()) / abs(r.sum())
        print(f"fp64 task {tk}: e = {g.sum():.15e}, oracle {r.sum():.15e}, rel {err:.2e}")
        assert err <= TOL["fp64"]
        assert abs(g[0] - r[0]) <= TOL["fp64"] * abs(r.sum())


@pytest.mark.parametrize("prec", ["fp64_oz", "tf32x3", "bf16x3"])
def test_full_size_tensor_core_sampled_tasks(full, prec):
    try:
        tasks, got = check(prec, full, 64)
    except tcorr.TcorrError as e:
        if e.status == 5:
            pytest.skip(f"{prec} unsupported on this device: {e}")
        raise
    key = "full_size_ref_" + "_".join("%d-%d-%d" % tuple(t) for t in tasks)
    ref = _REF.get(key)
    if ref is None:
        ref = _REF[key] = oracle_tasks(full, tasks)
    for tk, g, r in zip(tasks, got, ref):
        err = abs(g.sum() - r.sum()) / abs(r.sum())
        print(f"{prec} task {tk}: e = {g.sum():.15e}, oracle {r.sum():.15e}, rel {err:.2e}")
        assert err <= TOL[prec]


_REF = {}  # oracle shares of the tensor-core sample, computed once per session
