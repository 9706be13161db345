"""CPU oracle for the closed-shell (T) triples-correction energy.

TEST INFRASTRUCTURE ONLY: imported by the test suite, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline leg, never by
the product package.  It shares no code with the CUDA path; both sides only
share the seeded input generator.

Two independent implementations:

* ``triple_energies`` / ``energy``: the C oracle (``tcorr_oracle.c``), the
  restricted i <= j <= k loop of Sec. 3 of the paper with Eqs. (2.2.1)-(2.2.5)
  evaluated literally per task (sign reading: D = e_occ - e_vir).
* ``bruteforce``: numpy, every ordered (i, j, k) and every (a, b, c), the
  same equations written with einsum and no permutational symmetry; tiny
  sizes only.

RI-MP2 (the paper's second workload, Sec. 2.1):

* ``mp2_energy``: numpy, Eqs. (mp2_energy), (eri_sym_decomp), (e_orb_diff)
  over every ordered occupied pair (i, j): g = C_i^T C_j with C_i[gamma][a] =
  C^gamma_ai, then -sum_ab g_ab (2 g_ab - g_ba) / (e_a + e_b - e_i - e_j),
  split into the Coulomb part -2 sum g^2 / eps and the exchange part
  +sum g g^T / eps.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcorr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no machine-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_triple_energies.restype = ctypes.c_int
            lib.oracle_triple_energies.argtypes = [
                ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
                ctypes.POINTER(dp), dp, dp, ctypes.c_longlong,
                ctypes.POINTER(ctypes.c_int), dp, ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def sorted_triples(o: int) -> np.ndarray:
    """All i <= j <= k, lexicographic in (i, j, k): C(o+2, 3) tasks
    (Eq. tasks_ccsdpt)."""
    out = [(i, j, k) for i in range(o) for j in range(i, o) for k in range(j, o)]
    return np.asarray(out, dtype=np.int32).reshape(-1, 3)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def vvvo_slices(vvvo: np.ndarray, occ=None):
    """Per-occupied slices [v][v][v] with element [x][y][z] = (xy|zq)."""
    o = vvvo.shape[3]
    occ = range(o) if occ is None else occ
    return {int(q): np.ascontiguousarray(vvvo[:, :, :, q]) for q in occ}


def triple_energies(inst, tasks, nthreads: int = 0, slices=None) -> np.ndarray:
    """(E[4], E[5]) share of each sorted triple in ``tasks`` ([n][3], i<=j<=k).

    ``slices``: optional dict q -> (xy|zq) array, for callers that hold only
    the vvvo slices the tasks touch (large instances)."""
    lib = _load()
    o, v = inst.o, inst.v
    tasks = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 3))
    if slices is None:
        need = sorted({int(x) for x in tasks.reshape(-1)})
        slices = vvvo_slices(inst.vvvo, need)
    arrs = [_c(inst.eps_occ), _c(inst.eps_vir), _c(inst.t1), _c(inst.t2),
            _c(inst.ooov), _c(inst.ovov)]
    sl = [(_c(slices[q]) if q in slices else None) for q in range(o)]
    slice_ptrs = (ctypes.POINTER(ctypes.c_double) * o)(
        *[(_ptr(s) if s is not None else ctypes.POINTER(ctypes.c_double)()) for s in sl])
    out = np.zeros((tasks.shape[0], 2), dtype=np.float64)
    rc = lib.oracle_triple_energies(
        o, v, _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), _ptr(arrs[3]),
        slice_ptrs, _ptr(arrs[4]), _ptr(arrs[5]), tasks.shape[0],
        tasks.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_triple_energies failed with code {rc}")
    return out


def energy(inst, nthreads: int = 0):
    """(E[4], E[5], E(T)) summed over all sorted triples."""
    e = triple_energies(inst, sorted_triples(inst.o), nthreads)
    e4 = float(np.sum(e[:, 0]))
    e5 = float(np.sum(e[:, 1]))
    return e4, e5, e4 + e5


def bruteforce(inst, with_scale: bool = False, per_triple: bool = False):
    """(E[4], E[5], E(T)) by the literal definitions over all ordered (i,j,k)
    and all (a,b,c), no permutational symmetry.  Memory o^3 v^3.

    with_scale=True appends the sum of the absolute values of the individual
    terms of W~ W / D and Y~ W / D (each tilde expanded into its three terms),
    the magnitude against which an exact zero is judged.  per_triple=True returns instead the
    (E[4], E[5]) summands of every ordered (i,j,k) as two [o][o][o] arrays."""
    eo, ev = _c(inst.eps_occ), _c(inst.eps_vir)
    t1, t2, vvvo, ooov, ovov = (_c(inst.t1), _c(inst.t2), _c(inst.vvvo),
                                _c(inst.ooov), _c(inst.ovov))
    # X^{abc}_{ijk} = sum_d t^{ad}_{ij} (ck|bd) - sum_l t^{ab}_{il} (ck|lj)
    # (ck|bd) = (bd|ck) = vvvo[b,d,c,k];  (ck|lj) = (lj|kc) = ooov[l,j,k,c]
    X = (np.einsum("ijad,bdck->ijkabc", t2, vvvo, optimize=True)
         - np.einsum("ilab,ljkc->ijkabc", t2, ooov, optimize=True))
    # P: x^{abc}_{ijk} + x^{acb}_{ikj} + x^{bac}_{jik} + x^{bca}_{jki}
    #    + x^{cab}_{kij} + x^{cba}_{kji}
    W = (np.einsum("ijkabc->ijkabc", X) + np.einsum("ikjacb->ijkabc", X)
         + np.einsum("jikbac->ijkabc", X) + np.einsum("jkibca->ijkabc", X)
         + np.einsum("kijcab->ijkabc", X) + np.einsum("kjicba->ijkabc", X))
    # Y^{abc}_{ijk} = t^a_i g_{jbkc} + t^b_j g_{iakc} + t^c_k g_{iajb}
    Y = (np.einsum("ia,jbkc->ijkabc", t1, ovov)
         + np.einsum("jb,iakc->ijkabc", t1, ovov)
         + np.einsum("kc,iajb->ijkabc", t1, ovov))
    D = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
         + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
         - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])

    def tilde(x):  # 4/3 x^{abc} - 2 x^{acb} + 2/3 x^{bca}, ijk fixed
        return (4.0 / 3.0 * x - 2.0 * np.einsum("ijkacb->ijkabc", x)
                + 2.0 / 3.0 * np.einsum("ijkbca->ijkabc", x))

    f4 = tilde(W) * W / D
    f5 = tilde(Y) * W / D
    if per_triple:
        return f4.sum(axis=(3, 4, 5)), f5.sum(axis=(3, 4, 5))
    e4 = float(np.sum(f4))
    e5 = float(np.sum(f5))
    if with_scale:
        def abs_tilde(x):
            return (4.0 / 3.0 * np.abs(x) + 2.0 * np.abs(np.einsum("ijkacb->ijkabc", x))
                    + 2.0 / 3.0 * np.abs(np.einsum("ijkbca->ijkabc", x)))
        scale = np.sum((abs_tilde(W) + abs_tilde(Y)) * np.abs(W) / np.abs(D))
        return e4, e5, e4 + e5, float(scale)
    return e4, e5, e4 + e5


def mp2_energy(inst):
    """(E_J, E_K, E_MP2) of an RI-MP2 instance (Sec. 2.1): for every ordered
    occupied pair (i, j) the ERIs g_aibj = sum_gamma C^gamma_ai C^gamma_bj
    (Eq. eri_sym_decomp, a library matmul) and the energy terms of Eq.
    (mp2_energy) with eps^{ab}_{ij} = e_a + e_b - e_i - e_j (Eq. e_orb_diff);
    the exchange integral g_ajbi is g_{b a} of the same pair.  FP64."""
    eo = np.asarray(inst.eps_occ, dtype=np.float64)
    ev = np.asarray(inst.eps_vir, dtype=np.float64)
    C = np.asarray(inst.C, dtype=np.float64)
    ej = ek = 0.0
    for i in range(inst.o):
        Ci = C[:, :, i]
        for j in range(inst.o):
            g = Ci.T @ C[:, :, j]
            eps = ev[:, None] + ev[None, :] - eo[i] - eo[j]
            ej -= 2.0 * float(np.sum(g * g / eps))
            ek += float(np.sum(g * g.T / eps))
    return ej, ek, ej + ek
