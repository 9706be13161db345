"""Server with continuous batching (tcorr_server_*), through the C ABI (GPU).

A job's energies must be bit-identical alone and in a mix with other jobs
that arrive while it runs (its work units do the same arithmetic whatever
shares a wave), equal to a single handle's, and within tolerance of the
oracle; admission must respect the memory budget; an expired device wait
must fail the running jobs with TCORR_ETIMEOUT and leave the server usable."""
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import synth, tcorr

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "tf32x3": 1e-6, "bf16x3": 1e-6}
# small jobs (BF16X3 runs them on TF32 operands) and one above TCORR_BF16_MIN_FLOPS
SHAPES = [(4, 20, 11), (6, 47, 12), (3, 130, 13), (1, 24, 14), (5, 33, 15), (2, 64, 16), (6, 160, 17)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_08094_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.fixture(scope="module")
def jobs():
    insts = [synth.make_instance(o, v, None, s) for o, v, s in SHAPES]
    return insts, [i.to("cuda") for i in insts], [oracle.energy(i) for i in insts]


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def solo(dev, prec):
    with tcorr.Server(prec=prec) as s:
        jid = s.submit(dev)
        assert s.poll(jid)[0] == "queued"
        s.drain()
        state, e, st = s.poll(jid)
        assert state == "done" and st == 0
        return e


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
def test_alone_and_in_the_mix_are_identical(jobs, prec):
    insts, dev, refs = jobs
    alone = [solo(d, prec) for d in dev]
    with tcorr.Server(prec=prec, wave_mb=128) as s:
        ids = [s.submit(d) for d in dev[:3]]
        s.step()
        assert s.poll(ids[0])[0] in ("running", "done")
        s.step()
        ids += [s.submit(d) for d in dev[3:]]     # arrive while the first ones run
        while s.step() > 0:
            pass
        s.drain()
        mixed = [s.poll(i) for i in ids]
        st = s.stats()
    assert st["done"] == len(SHAPES) and st["failed"] == 0 and st["running"] == 0 and st["bytes"] == 0
    assert st["waves"] >= 2
    for n, (state, e, status) in enumerate(mixed):
        assert state == "done" and status == 0
        assert e == alone[n], (n, e, alone[n])
        with tcorr.Tcorr.from_instance(dev[n], prec=prec) as t:
            assert t.energy() == e
        if insts[n].o == 1:
            assert e == (0.0, 0.0, 0.0)
        else:
            assert rel(e[2], refs[n][2]) <= TOL[prec], (prec, n, e, refs[n])


def test_admission_respects_the_budget(jobs):
    _, dev, _ = jobs
    # room for a few of the ~35-70 MB job footprints at a time: the rest must queue
    budget = 300 << 20
    with tcorr.Server(prec="bf16x3", hbm_bytes=budget, wave_mb=64) as s:
        ids = [s.submit(d) for d in dev * 3]
        saw_queue = False
        while True:
            left = s.step()
            st = s.stats()
            assert st["bytes"] <= budget and st["peak_bytes"] <= budget
            if st["queued"] > 0 and st["running"] > 0:
                saw_queue = True
            if left == 0:
                break
        s.drain()
        st = s.stats()
        assert st["done"] == len(ids) and st["peak_bytes"] <= budget
        assert saw_queue
        res = [s.poll(i)[1] for i in ids]
    n = len(dev)
    for k in range(n):
        assert res[k] == res[k + n] == res[k + 2 * n]   # same job, different mixes


def test_rejects_what_can_never_fit(jobs):
    _, dev, _ = jobs
    with tcorr.Server(prec="bf16x3", hbm_bytes=40 << 20) as s:
        with pytest.raises(tcorr.TcorrError) as ex:
            s.submit(dev[2])
        assert ex.value.status == 2   # TCORR_ENOMEM
        with pytest.raises(tcorr.TcorrError):
            s.poll(12345)
        assert s.stats()["submitted"] == 0


def test_expired_wait_fails_running_jobs_and_server_stays_usable(jobs):
    """Failure detection without a fault: the test-only option makes CTA 0 of
    every tensor-core launch withhold one chunk's loads, so a bounded wait
    expires (about 2 s); the jobs of that wave fail with TCORR_ETIMEOUT."""
    _, dev, _ = jobs
    # o=6, v=47: CTA 0's second item is a task with work (for o=4, v=20 both
    # of its items are i = j = k tasks, which load nothing)
    with tcorr.Server(prec="bf16x3", test_stall=True) as s:
        a = s.submit(dev[1])
        s.drain()
        state, e, status = s.poll(a)
        assert state == "failed" and status == 4 and e is None
        st = s.stats()
        assert st["failed"] == 1 and st["running"] == 0 and st["bytes"] == 0
    # the context is intact: a normal server on the same device works
    with tcorr.Server(prec="bf16x3") as s:
        b = s.submit(dev[0])
        s.drain()
        assert s.poll(b)[0] == "done"
