"""ctypes binding of libtcorr (include/tcorr.h).

Argument marshalling only: every step of the (T) energy runs in the CUDA
library.  There is no fallback: if libtcorr.so is missing or cannot be
loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

PREC = {"fp64": 0, "tf32x3": 1, "bf16x3": 2, "fp64_oz": 3}
STATUS = ["TCORR_OK", "TCORR_EINVAL", "TCORR_ENOMEM", "TCORR_ECUDA", "TCORR_ETIMEOUT",
          "TCORR_EUNSUPPORTED"]
KERNEL_CLASSES = ("prep", "gemm", "epilogue", "reduce")

_lock = threading.Lock()
_lib = None


class TcorrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else f"status {status}"
        super().__init__(f"{name}: {msg}")


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("host_inputs", ctypes.c_int),
                ("batch_tasks", ctypes.c_int), ("profile", ctypes.c_int),
                ("test_stall", ctypes.c_int), ("tune", ctypes.c_int),
                ("eager", ctypes.c_int), ("wave_mb", ctypes.c_int), ("single_sm", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("o", ctypes.c_int), ("v", ctypes.c_int),
                ("eps_occ", ctypes.c_void_p), ("eps_vir", ctypes.c_void_p),
                ("t1", ctypes.c_void_p), ("t2", ctypes.c_void_p),
                ("vvvo", ctypes.c_void_p), ("ooov", ctypes.c_void_p),
                ("ovov", ctypes.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libtcorr.so (built by __graft_entry__.build() or _build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libtcorr.so not found at {path}: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        lib = ctypes.CDLL(path)
        vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
        lib.tcorr_create.restype = ctypes.c_int
        lib.tcorr_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int,
                                     vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Opts), vp]
        lib.tcorr_energy.restype = ctypes.c_int
        lib.tcorr_energy.argtypes = [vp, dp]
        lib.tcorr_energy_range.restype = ctypes.c_int
        lib.tcorr_energy_range.argtypes = [vp, i64, i64, dp, dp]
        lib.tcorr_num_tasks.restype = i64
        lib.tcorr_num_tasks.argtypes = [vp]
        lib.tcorr_task.restype = ctypes.c_int
        lib.tcorr_task.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int)]
        lib.tcorr_kernel_times.restype = ctypes.c_int
        lib.tcorr_kernel_times.argtypes = [vp, dp, ctypes.POINTER(i64), ctypes.c_int]
        lib.tcorr_device_bytes.restype = i64
        lib.tcorr_device_bytes.argtypes = [vp]
        lib.tcorr_destroy.restype = ctypes.c_int
        lib.tcorr_destroy.argtypes = [vp]
        lib.tcorr_last_error.restype = ctypes.c_char_p
        lib.tcorr_last_error.argtypes = [vp]
        lib.tcorr_status_string.restype = ctypes.c_char_p
        lib.tcorr_status_string.argtypes = [ctypes.c_int]
        lib.tcorr_version.restype = ctypes.c_int
        lib.tcorr_version.argtypes = []
        bp = ctypes.c_void_p
        lib.tcorr_batch_create.restype = ctypes.c_int
        lib.tcorr_batch_create.argtypes = [ctypes.POINTER(bp), ctypes.c_int, ctypes.POINTER(Problem),
                                           ctypes.POINTER(Opts), vp]
        lib.tcorr_batch_size.restype = ctypes.c_int
        lib.tcorr_batch_size.argtypes = [bp]
        lib.tcorr_batch_energy.restype = ctypes.c_int
        lib.tcorr_batch_energy.argtypes = [bp, dp]
        lib.tcorr_batch_tile.restype = ctypes.c_int
        lib.tcorr_batch_tile.argtypes = [bp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.tcorr_batch_plan.restype = ctypes.c_int
        lib.tcorr_batch_plan.argtypes = [bp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.tcorr_batch_kernel_times.restype = ctypes.c_int
        lib.tcorr_batch_kernel_times.argtypes = [bp, dp, ctypes.POINTER(i64), ctypes.c_int]
        lib.tcorr_batch_device_bytes.restype = i64
        lib.tcorr_batch_device_bytes.argtypes = [bp]
        lib.tcorr_batch_last_error.restype = ctypes.c_char_p
        lib.tcorr_batch_last_error.argtypes = [bp]
        lib.tcorr_batch_destroy.restype = ctypes.c_int
        lib.tcorr_batch_destroy.argtypes = [bp]
        sp = ctypes.c_void_p
        lib.tcorr_server_create.restype = ctypes.c_int
        lib.tcorr_server_create.argtypes = [ctypes.POINTER(sp), ctypes.POINTER(Opts), i64, vp]
        lib.tcorr_server_submit.restype = ctypes.c_int
        lib.tcorr_server_submit.argtypes = [sp, ctypes.POINTER(Problem), ctypes.POINTER(i64)]
        lib.tcorr_server_step.restype = ctypes.c_int
        lib.tcorr_server_step.argtypes = [sp, ctypes.POINTER(ctypes.c_int)]
        lib.tcorr_server_poll.restype = ctypes.c_int
        lib.tcorr_server_poll.argtypes = [sp, i64, ctypes.POINTER(ctypes.c_int), dp,
                                          ctypes.POINTER(ctypes.c_int)]
        lib.tcorr_server_drain.restype = ctypes.c_int
        lib.tcorr_server_drain.argtypes = [sp]
        lib.tcorr_server_stats.restype = ctypes.c_int
        lib.tcorr_server_stats.argtypes = [sp, ctypes.POINTER(i64)]
        lib.tcorr_server_last_error.restype = ctypes.c_char_p
        lib.tcorr_server_last_error.argtypes = [sp]
        lib.tcorr_server_destroy.restype = ctypes.c_int
        lib.tcorr_server_destroy.argtypes = [sp]
        mp = ctypes.c_void_p
        lib.tcorr_mp2_create.restype = ctypes.c_int
        lib.tcorr_mp2_create.argtypes = [ctypes.POINTER(mp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         vp, vp, vp, ctypes.POINTER(Opts), vp]
        lib.tcorr_mp2_energy.restype = ctypes.c_int
        lib.tcorr_mp2_energy.argtypes = [mp, dp]
        lib.tcorr_mp2_kernel_times.restype = ctypes.c_int
        lib.tcorr_mp2_kernel_times.argtypes = [mp, dp, ctypes.POINTER(i64), ctypes.c_int]
        lib.tcorr_mp2_device_bytes.restype = i64
        lib.tcorr_mp2_device_bytes.argtypes = [mp]
        lib.tcorr_mp2_last_error.restype = ctypes.c_char_p
        lib.tcorr_mp2_last_error.argtypes = [mp]
        lib.tcorr_mp2_destroy.restype = ctypes.c_int
        lib.tcorr_mp2_destroy.argtypes = [mp]
        lib.tcorr_task_energy_noalloc.restype = ctypes.c_int
        lib.tcorr_task_energy_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
        _lib = lib
        return lib


EXPORTS = ("tcorr_create", "tcorr_energy", "tcorr_energy_range", "tcorr_num_tasks",
           "tcorr_task", "tcorr_kernel_times", "tcorr_device_bytes", "tcorr_destroy",
           "tcorr_last_error", "tcorr_status_string", "tcorr_version",
           "tcorr_batch_create", "tcorr_batch_size", "tcorr_batch_energy", "tcorr_batch_tile",
           "tcorr_batch_plan", "tcorr_batch_kernel_times", "tcorr_batch_device_bytes",
           "tcorr_batch_last_error", "tcorr_batch_destroy",
           "tcorr_server_create", "tcorr_server_submit", "tcorr_server_step", "tcorr_server_poll",
           "tcorr_server_drain", "tcorr_server_stats", "tcorr_server_last_error",
           "tcorr_server_destroy",
           "tcorr_mp2_create", "tcorr_mp2_energy", "tcorr_mp2_kernel_times", "tcorr_mp2_device_bytes",
           "tcorr_mp2_last_error", "tcorr_mp2_destroy",
           "tcorr_task_energy_noalloc")
JOB_STATES = ("queued", "running", "done", "failed")
SERVER_STATS = ("submitted", "done", "failed", "running", "queued", "bytes", "peak_bytes", "waves")
NOALLOC_MAX_V = 64
# TCORR_BF16X3 problems below these sizes run on TF32 hi + lo operands (include/tcorr.h)
BF16_MIN_FLOPS = 1e11
MP2_BF16_MIN_TERMS = 16777216


def _prec(prec) -> int:
    """tcorr_precision of a name ('fp64', 'tf32x3', 'bf16x3', 'fp64_oz') or an int."""
    if isinstance(prec, str):
        key = prec.lower()
        if key not in PREC:
            raise ValueError(f"unknown precision {prec!r}; one of {sorted(PREC)}")
        return PREC[key]
    return int(prec)


def _shape_check(name, a, shape):
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(a.shape)}")


def _pointer(name, a, on_device: bool):
    """Raw pointer of a float64 C-contiguous torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError(f"{name}: needs a contiguous float64 tensor")
        if a.is_cuda != on_device:
            raise ValueError(f"{name}: device/host placement differs from the other inputs")
        return a.data_ptr()
    if on_device:
        raise ValueError(f"{name}: numpy array given together with device tensors")
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise ValueError(f"{name}: needs a C-contiguous float64 array")
    return a.ctypes.data


class Tcorr:
    """One (T) problem resident on the GPU.

    Inputs are the seven arrays of tcorr_create (torch CUDA tensors, or all
    numpy / CPU arrays, which are copied in).  ``prec`` is 'fp64', 'fp64_oz',
    'tf32x3' or 'bf16x3'.  ``stream``: a torch.cuda.Stream, an integer cudaStream_t, or
    None for torch's current stream (device inputs) / the default stream."""

    def __init__(self, o, v, eps_occ, eps_vir, t1, t2, vvvo, ooov, ovov, prec="fp64",
                 batch_tasks=0, profile=False, stream=None, test_stall=False, tune=False,
                 single_sm=False):
        lib = load()
        arrays = dict(eps_occ=eps_occ, eps_vir=eps_vir, t1=t1, t2=t2, vvvo=vvvo, ooov=ooov,
                      ovov=ovov)
        shapes = dict(eps_occ=(o,), eps_vir=(v,), t1=(o, v), t2=(o, o, v, v),
                      vvvo=(v, v, v, o), ooov=(o, o, o, v), ovov=(o, v, o, v))
        on_device = bool(getattr(t2, "is_cuda", False))
        ptrs = []
        for k, a in arrays.items():
            _shape_check(k, a, shapes[k])
            ptrs.append(_pointer(k, a, on_device))
        prec = _prec(prec)
        opts = Opts(prec=int(prec), host_inputs=0 if on_device else 1,
                    batch_tasks=int(batch_tasks), profile=1 if profile else 0,
                    test_stall=1 if test_stall else 0, tune=1 if tune else 0,
                    single_sm=1 if single_sm else 0)
        if stream is None and on_device:
            import torch
            stream = torch.cuda.current_stream(t2.device)
        sptr = getattr(stream, "cuda_stream", stream) or 0
        self._stream = stream
        self.o, self.v, self.prec = o, v, int(prec)
        h = ctypes.c_void_p()
        st = lib.tcorr_create(ctypes.byref(h), int(o), int(v), *ptrs, ctypes.byref(opts),
                              ctypes.c_void_p(sptr))
        if st != 0:
            raise TcorrError(st, lib.tcorr_last_error(None).decode())
        self._h = h

    @classmethod
    def from_instance(cls, inst, **kw):
        return cls(inst.o, inst.v, *inst.arrays(), **kw)

    def _check(self, st):
        if st != 0:
            raise TcorrError(st, load().tcorr_last_error(self._h).decode())

    @property
    def num_tasks(self) -> int:
        return int(load().tcorr_num_tasks(self._h))

    def task(self, idx: int):
        ijk = (ctypes.c_int * 3)()
        self._check(load().tcorr_task(self._h, int(idx), ijk))
        return tuple(ijk)

    def energy(self):
        """(E[4], E[5], E(T))."""
        e = (ctypes.c_double * 3)()
        self._check(load().tcorr_energy(self._h, e))
        return tuple(e)

    def energy_range(self, first: int, count: int, per_task: bool = False):
        """(E[4], E[5], E(T)) of tasks first..first+count-1; with per_task the
        [count][2] array of (E[4], E[5]) shares is returned as well."""
        e = (ctypes.c_double * 3)()
        et = np.zeros((max(count, 0), 2), dtype=np.float64) if per_task else None
        ptr = et.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if per_task else None
        self._check(load().tcorr_energy_range(self._h, int(first), int(count), e, ptr))
        return (tuple(e), et) if per_task else tuple(e)

    def kernel_times(self, reset: bool = False):
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        self._check(load().tcorr_kernel_times(self._h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}

    @property
    def device_bytes(self) -> int:
        return int(load().tcorr_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().tcorr_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ARRAY_NAMES = ("eps_occ", "eps_vir", "t1", "t2", "vvvo", "ooov", "ovov")


class Batch:
    """Many independent (T) problems of uneven (o, v) evaluated together
    (tcorr_batch_*): their tasks share waves of the same kernels, and the
    launch sequence is replayed from a CUDA graph after the first call.

    ``problems``: a sequence of (o, v, eps_occ, eps_vir, t1, t2, vvvo, ooov,
    ovov) tuples (or objects with ``o``, ``v`` and ``arrays()``), all on the
    device or all on the host.  ``energy()`` returns an [n][3] array of
    (E[4], E[5], E(T))."""

    def __init__(self, problems, prec="fp64", batch_tasks=0, profile=False, stream=None,
                 tune=False, eager=False, wave_mb=0, single_sm=False):
        lib = load()
        items = []
        for p in problems:
            if hasattr(p, "arrays"):
                items.append((p.o, p.v, *p.arrays()))
            else:
                items.append(tuple(p))
        if not items:
            raise ValueError("a batch needs at least one problem")
        on_device = bool(getattr(items[0][5], "is_cuda", False))
        arr = (Problem * len(items))()
        keep = []
        for n, it in enumerate(items):
            o, v = int(it[0]), int(it[1])
            shapes = dict(eps_occ=(o,), eps_vir=(v,), t1=(o, v), t2=(o, o, v, v),
                          vvvo=(v, v, v, o), ooov=(o, o, o, v), ovov=(o, v, o, v))
            ptrs = []
            for name, a in zip(_ARRAY_NAMES, it[2:]):
                _shape_check(f"problem {n} {name}", a, shapes[name])
                ptrs.append(_pointer(f"problem {n} {name}", a, on_device))
                keep.append(a)
            arr[n] = Problem(o, v, *ptrs)
        prec = _prec(prec)
        opts = Opts(prec=int(prec), host_inputs=0 if on_device else 1,
                    batch_tasks=int(batch_tasks), profile=1 if profile else 0,
                    tune=1 if tune else 0, eager=1 if eager else 0, wave_mb=int(wave_mb),
                    single_sm=1 if single_sm else 0)
        if stream is None and on_device:
            import torch
            stream = torch.cuda.current_stream(items[0][5].device)
        sptr = getattr(stream, "cuda_stream", stream) or 0
        self._stream = stream
        self.n, self.prec = len(items), int(prec)
        self.shapes = [(int(it[0]), int(it[1])) for it in items]
        h = ctypes.c_void_p()
        st = lib.tcorr_batch_create(ctypes.byref(h), len(items), arr, ctypes.byref(opts),
                                    ctypes.c_void_p(sptr))
        if st != 0:
            raise TcorrError(st, lib.tcorr_batch_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != 0:
            raise TcorrError(st, load().tcorr_batch_last_error(self._h).decode())

    def energy(self) -> np.ndarray:
        """[n][3] array: (E[4], E[5], E(T)) of every problem."""
        e = np.zeros((self.n, 3), dtype=np.float64)
        self._check(load().tcorr_batch_energy(self._h, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return e

    def tile(self, idx: int):
        """(pb, kb) of problem idx's tensor-core tile; (0, 0) for FP64."""
        t = (ctypes.c_int * 2)()
        self._check(load().tcorr_batch_tile(self._h, int(idx), t))
        return tuple(t)

    def plan(self):
        """(waves, kernel launches) of one energy call."""
        w, n = ctypes.c_int64(), ctypes.c_int64()
        self._check(load().tcorr_batch_plan(self._h, ctypes.byref(w), ctypes.byref(n)))
        return int(w.value), int(n.value)

    def kernel_times(self, reset: bool = False):
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        self._check(load().tcorr_batch_kernel_times(self._h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}

    @property
    def device_bytes(self) -> int:
        return int(load().tcorr_batch_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().tcorr_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of (T) jobs (tcorr_server_*).  ``submit`` queues a
    job (device arrays that must stay alive until it is done; this object
    keeps references until then), ``step`` admits what fits the memory budget
    and enqueues one wave of tasks from every running job, ``poll`` reports a
    job's state and energies.  ``hbm_bytes``: memory budget for admitted
    jobs (0 = 80% of free memory)."""

    def __init__(self, prec="bf16x3", hbm_bytes=0, wave_mb=0, batch_tasks=0, profile=False,
                 stream=None, test_stall=False, single_sm=False):
        lib = load()
        prec = _prec(prec)
        opts = Opts(prec=int(prec), host_inputs=0, batch_tasks=int(batch_tasks),
                    profile=1 if profile else 0, test_stall=1 if test_stall else 0,
                    wave_mb=int(wave_mb), single_sm=1 if single_sm else 0)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        sptr = getattr(stream, "cuda_stream", stream) or 0
        self._stream = stream
        self.prec = int(prec)
        self._keep = {}
        h = ctypes.c_void_p()
        st = lib.tcorr_server_create(ctypes.byref(h), ctypes.byref(opts), int(hbm_bytes),
                                     ctypes.c_void_p(sptr))
        if st != 0:
            raise TcorrError(st, lib.tcorr_server_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != 0:
            raise TcorrError(st, load().tcorr_server_last_error(self._h).decode())

    def submit(self, problem) -> int:
        """Queue a job: an Instance (device arrays) or an (o, v, eps_occ, ...,
        ovov) tuple.  Returns the job id."""
        it = (problem.o, problem.v, *problem.arrays()) if hasattr(problem, "arrays") else tuple(problem)
        o, v = int(it[0]), int(it[1])
        shapes = dict(eps_occ=(o,), eps_vir=(v,), t1=(o, v), t2=(o, o, v, v),
                      vvvo=(v, v, v, o), ooov=(o, o, o, v), ovov=(o, v, o, v))
        ptrs = []
        for name, a in zip(_ARRAY_NAMES, it[2:]):
            _shape_check(name, a, shapes[name])
            ptrs.append(_pointer(name, a, True))
        pr = Problem(o, v, *ptrs)
        jid = ctypes.c_int64()
        self._check(load().tcorr_server_submit(self._h, ctypes.byref(pr), ctypes.byref(jid)))
        self._keep[jid.value] = it
        return int(jid.value)

    def step(self) -> int:
        """One scheduling step; returns the number of jobs not yet finished."""
        n = ctypes.c_int()
        self._check(load().tcorr_server_step(self._h, ctypes.byref(n)))
        return int(n.value)

    def poll(self, jid: int):
        """(state, energies or None, status): state in JOB_STATES."""
        st = ctypes.c_int()
        js = ctypes.c_int()
        e = (ctypes.c_double * 3)()
        self._check(load().tcorr_server_poll(self._h, int(jid), ctypes.byref(st), e, ctypes.byref(js)))
        state = JOB_STATES[st.value]
        if state in ("done", "failed"):
            self._keep.pop(int(jid), None)
        return state, (tuple(e) if state == "done" else None), int(js.value)

    def drain(self):
        self._check(load().tcorr_server_drain(self._h))

    def stats(self):
        a = (ctypes.c_int64 * 8)()
        self._check(load().tcorr_server_stats(self._h, a))
        return dict(zip(SERVER_STATS, (int(x) for x in a)))

    def close(self):
        if getattr(self, "_h", None):
            load().tcorr_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mp2:
    """RI-MP2 correlation energy of one problem (tcorr_mp2_*): eps_occ [o],
    eps_vir [v], C [naux][v][o] (all CUDA tensors, or all numpy arrays which
    are copied in).  ``energy()`` returns (E_J, E_K, E_MP2); prec "fp64",
    "tf32x3" or "bf16x3" (the split precisions on the tensor cores)."""

    def __init__(self, o, v, naux, eps_occ, eps_vir, C, profile=False, stream=None, prec="fp64"):
        lib = load()
        on_device = bool(getattr(C, "is_cuda", False))
        shapes = dict(eps_occ=(o,), eps_vir=(v,), C=(naux, v, o))
        ptrs = []
        for name, a in (("eps_occ", eps_occ), ("eps_vir", eps_vir), ("C", C)):
            _shape_check(name, a, shapes[name])
            ptrs.append(_pointer(name, a, on_device))
        prec = _prec(prec)
        opts = Opts(prec=int(prec), host_inputs=0 if on_device else 1, profile=1 if profile else 0)
        if stream is None and on_device:
            import torch
            stream = torch.cuda.current_stream(C.device)
        sptr = getattr(stream, "cuda_stream", stream) or 0
        self._stream = stream
        h = ctypes.c_void_p()
        st = lib.tcorr_mp2_create(ctypes.byref(h), int(o), int(v), int(naux), *ptrs, ctypes.byref(opts),
                                  ctypes.c_void_p(sptr))
        if st != 0:
            raise TcorrError(st, lib.tcorr_mp2_last_error(None).decode())
        self._h = h
        self.o, self.v, self.naux = o, v, naux

    @classmethod
    def from_instance(cls, inst, **kw):
        return cls(inst.o, inst.v, inst.naux, *inst.arrays(), **kw)

    def _check(self, st):
        if st != 0:
            raise TcorrError(st, load().tcorr_mp2_last_error(self._h).decode())

    def energy(self):
        e = (ctypes.c_double * 3)()
        self._check(load().tcorr_mp2_energy(self._h, e))
        return tuple(e)

    def kernel_times(self, reset: bool = False):
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        self._check(load().tcorr_mp2_kernel_times(self._h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "_h", None):
            load().tcorr_mp2_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp2_flops(o: int, v: int, naux: int) -> float:
    """Algorithmic flops of the ERI assembly over the pairs i <= j: 2 v^2 naux
    per pair (Sec. 2.1, Eq. tasks_rimp2)."""
    return 2.0 * v * v * naux * (o * (o + 1) // 2)


def task_energy_noalloc(o, v, eps_occ, eps_vir, t1, t2, vvvo, ooov, ovov, ijk, out, stream=None):
    """FP64 (E[4], E[5]) share of one task into ``out`` (a float64 CUDA tensor
    of 2 elements) without any device allocation by the library: for callers
    whose device memory is owned by their own pool or budget, or that cannot
    pay cudaMalloc's device synchronisation.  Uses a fixed device scratch
    array (v <= NOALLOC_MAX_V); asynchronous on ``stream``.  Calls that overlap
    on the GPU race on the shared scratch; the first call on a device must
    precede any stream capture."""
    import torch
    arrays = dict(eps_occ=eps_occ, eps_vir=eps_vir, t1=t1, t2=t2, vvvo=vvvo, ooov=ooov, ovov=ovov)
    ptrs = [_pointer(k, a, True) for k, a in arrays.items()]
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 2:
        raise ValueError("out: needs a float64 CUDA tensor with 2 elements")
    if stream is None:
        stream = torch.cuda.current_stream(out.device)
    sptr = getattr(stream, "cuda_stream", stream) or 0
    i, j, k = (int(x) for x in ijk)
    st = load().tcorr_task_energy_noalloc(int(o), int(v), *ptrs, i, j, k, out.data_ptr(),
                                          ctypes.c_void_p(sptr))
    if st != 0:
        raise TcorrError(st, "tcorr_task_energy_noalloc rejected the call")


def num_tasks(o: int) -> int:
    return o * (o + 1) * (o + 2) // 6


def algorithmic_flops(o: int, v: int, ntasks: int | None = None) -> float:
    """12 v^3 (v + o) per task with i, j, k not all equal (the six GEMM pairs
    of the W contraction, Sec. 3); i = j = k tasks carry no work."""
    if ntasks is None:
        ntasks = num_tasks(o) - o
    return 12.0 * v ** 3 * (v + o) * ntasks
