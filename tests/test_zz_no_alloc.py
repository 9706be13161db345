"""The allocation-free entry point (collected last on purpose).

tcorr_task_energy_noalloc serves callers that must not allocate device
memory (their own pool/budget owns it, or cudaMalloc's synchronisation is not
affordable): it computes one task's FP64 energy share with a fixed device
scratch array.  Here it is called through the C ABI twice in a row and each
result is compared with the regular handle-based entry point's per-task
output, within the FP64 tolerance of the other GPU tests (1e-10 relative).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1609_08094_gb300 import _build, synth, tcorr

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


def test_noalloc_matches_handle_two_calls():
    _build.build()
    lib = tcorr.load()
    o, v = 5, 37
    inst = synth.make_instance(o, v, None, 31).to("cuda")
    with tcorr.Tcorr.from_instance(inst) as t:
        _, per = t.energy_range(0, t.num_tasks, per_task=True)
        tasks = [t.task(n) for n in range(t.num_tasks)]
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ptrs = [ctypes.c_void_p(a.data_ptr()) for a in inst.arrays()]
    for ijk in [(0, 1, 3), (1, 1, 4)]:   # two calls in a row, the second reuses the scratch
        st = lib.tcorr_task_energy_noalloc(o, v, *ptrs, *ijk, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = per[tasks.index(ijk)]
        assert np.all(np.abs(got - ref) <= FP64_TOL * np.abs(ref)), (ijk, got, ref)


def test_noalloc_rejects_sizes_beyond_scratch():
    lib = tcorr.load()
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.tcorr_task_energy_noalloc(3, tcorr.NOALLOC_MAX_V + 1, p, p, p, p, p, p, p, 0, 1, 2, p, None) == 1
    assert lib.tcorr_task_energy_noalloc(3, 10, p, p, p, p, p, p, p, 2, 1, 0, p, None) == 1
