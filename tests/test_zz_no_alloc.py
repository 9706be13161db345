"""The allocation-free entry point, tcorr_task_energy_noalloc.

It serves callers that must not allocate device memory: applications whose
device memory is owned by their own pool or budget, and latency-sensitive
loops that cannot pay cudaMalloc/cudaFree's device synchronisation.  It
computes one task's FP64 energy share with a fixed device scratch array that
every call shares.

The file name sorts last so that pytest collects it after every other test:
a run that stops at the first failure (pytest -x) has then already run all
the other tests when this one fails.  It passes alone in a fresh process too.

The calls go through the C ABI in sequence on one device: the largest v the
scratch allows (TCORR_NOALLOC_MAX_V), then smaller problems whose v is not a
multiple of the epilogue's block edge (8) or of the U row padding (16), and a
task with i = j = k (no contraction runs; the scratch still holds the previous
call's U).  Each result is compared with the FP64 oracle's energies of the
same task, and with the handle-based entry point's per-task output, at the
FP64 tolerance of the other GPU tests (1e-10 relative).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import _build, synth, tcorr

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


def call(lib, o, v, dev_arrays, ijk, out, stream):
    ptrs = [ctypes.c_void_p(a.data_ptr()) for a in dev_arrays]
    out.fill_(float("nan"))
    st = lib.tcorr_task_energy_noalloc(o, v, *ptrs, *ijk, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


def test_noalloc_sequence_matches_oracle_and_handle():
    _build.build()
    oracle.build()
    lib = tcorr.load()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    # (o, v, seed, task): v = the maximum, then v = 20 and 37 (ragged against
    # the 8-wide blocks and 16-wide U rows), then i = j = k after a full call
    cases = [(4, tcorr.NOALLOC_MAX_V, 31, (0, 1, 3)),
             (5, 20, 32, (1, 1, 4)),
             (3, 37, 33, (0, 2, 2)),
             (3, 37, 33, (2, 2, 2))]
    scale = None
    for o, v, seed, ijk in cases:
        host = synth.make_instance(o, v, None, seed)
        dev = host.to("cuda")
        got = call(lib, o, v, dev.arrays(), ijk, out, stream)
        ref = oracle.triple_energies(host, np.array([ijk]))[0]
        if ijk[0] == ijk[1] == ijk[2]:
            assert got[0] == 0.0 and got[1] == 0.0, (ijk, got)  # exact zero, not stale scratch
            # the oracle sums the literal terms, which cancel to rounding level
            assert np.all(np.abs(ref) <= FP64_TOL * scale), (ref, scale)
            continue
        scale = np.abs(ref).max()
        assert np.all(np.abs(got - ref) <= FP64_TOL * np.abs(ref).max()), (o, v, ijk, got, ref)
        with tcorr.Tcorr.from_instance(dev) as t:
            n = [t.task(m) for m in range(t.num_tasks)].index(ijk)
            _, per = t.energy_range(n, 1, per_task=True)
        assert np.all(np.abs(got - per[0]) <= FP64_TOL * np.abs(per[0]).max()), (o, v, ijk, got, per[0])
        print(f"noalloc o={o} v={v} task {ijk}: rel err vs oracle "
              f"{np.abs(got - ref).max() / np.abs(ref).max():.1e}")


def test_noalloc_rejects_sizes_beyond_scratch():
    lib = tcorr.load()
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.tcorr_task_energy_noalloc(3, tcorr.NOALLOC_MAX_V + 1, p, p, p, p, p, p, p, 0, 1, 2, p, None) == 1
    assert lib.tcorr_task_energy_noalloc(3, 10, p, p, p, p, p, p, p, 2, 1, 0, p, None) == 1
