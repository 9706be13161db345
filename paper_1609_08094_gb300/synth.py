"""Seeded synthetic inputs for the closed-shell (T) triples-correction energy.

This module only draws random numbers and assembles the *input* tensors of
the method (orbital energies, T1/T2 amplitudes and the vvvo, ooov, ovov
integral blocks).  It contains none of the (T) arithmetic: both the CUDA path
and the CPU oracle consume what it returns.

Recipe (the paper initialises its tensors with "unique, yet arbitrary" numbers,
Sec. 4; the distributions below fix that choice):

* Three-index factors B^Q_pq ~ N(0, sigma=0.1), drawn for p <= q (diagonal
  included) and mirrored, so B^Q_pq = B^Q_qp.  Orbitals are ordered occupied
  first (p < o), then virtual.
* Every integral block is (pq|rs) = sum_Q B^Q_pq B^Q_rs (real, 8-fold
  symmetric), in Mulliken notation as in Sec. 2.1.
* eps_occ ~ U[-2.0, -0.3] and eps_vir ~ U[0.1, 5.0] (hartree), each sorted
  ascending.
* T2 are first-order (MP1) amplitudes t_ij^ab = (ia|jb)/(e_i+e_j-e_a-e_b).
* T1 ~ N(0, sigma=1e-3).

Random numbers: a counter-based SplitMix64 stream (Steele, Lea & Flood,
OOPSLA 2014) per array, so each array is independent of the sizes of the
others.  Value n of stream s under seed S is mix64(key(S, s) + (n+1)*GAMMA),
mapped to a double in [0, 1) by its top 53 bits; normals use the Box-Muller
transform on consecutive pairs.

Layouts (row-major, float64), as taken by the C ABI:
  eps_occ[o], eps_vir[v], t1[o][v] = t_i^a, t2[o][o][v][v] = t_ij^ab,
  vvvo[v][v][v][o] = (ab|ci), ooov[o][o][o][v] = (ij|ka),
  ovov[o][v][o][v] = (ia|jb).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (fixed draw order B, eps_occ, eps_vir, T1)
STREAM_B, STREAM_EOCC, STREAM_EVIR, STREAM_T1 = 1, 2, 3, 4


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([(int(seed) * 0x100000001B3 + int(stream)) & 0xFFFFFFFFFFFFFFFF],
                        dtype=np.uint64)
        return _mix64(base)[0]


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from positions offset..offset+n-1 of one stream."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        x = _mix64(_key(seed, stream) + ctr * _GAMMA)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int, chunk: int = 1 << 24) -> np.ndarray:
    """n standard normals (Box-Muller on consecutive uniform pairs)."""
    out = np.empty(n, dtype=np.float64)
    npair = (n + 1) // 2
    for p0 in range(0, npair, chunk):
        p1 = min(npair, p0 + chunk)
        u = uniform(seed, stream, 2 * (p1 - p0), offset=2 * p0)
        u1 = 1.0 - u[0::2]          # (0, 1]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * (p1 - p0))
        z[0::2] = r * np.cos(2.0 * np.pi * u2)
        z[1::2] = r * np.sin(2.0 * np.pi * u2)
        lo, hi = 2 * p0, min(n, 2 * p1)
        out[lo:hi] = z[: hi - lo]
    return out


@dataclass
class Instance:
    """One synthetic (T) problem.  Arrays are numpy (host) or torch tensors."""
    o: int
    v: int
    naux: int
    seed: int
    eps_occ: object
    eps_vir: object
    t1: object
    t2: object
    vvvo: object
    ooov: object
    ovov: object

    def arrays(self):
        return (self.eps_occ, self.eps_vir, self.t1, self.t2,
                self.vvvo, self.ooov, self.ovov)

    def to(self, device):
        """Copy every array to a torch device (torch imported lazily)."""
        import torch
        conv = []
        for a in self.arrays():
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
            conv.append(t.to(device=device, dtype=torch.float64).contiguous())
        return Instance(self.o, self.v, self.naux, self.seed, *conv)

    def numpy(self):
        conv = []
        for a in self.arrays():
            if hasattr(a, "detach"):
                a = a.detach().cpu().numpy()
            conv.append(np.ascontiguousarray(a, dtype=np.float64))
        return Instance(self.o, self.v, self.naux, self.seed, *conv)

    def nbytes(self) -> int:
        o, v = self.o, self.v
        return 8 * (o + v + o * v + o * o * v * v + v ** 3 * o + o ** 3 * v + o * o * v * v)


def factors(o: int, v: int, naux: int, seed: int, sigma: float = 0.1) -> np.ndarray:
    """B[Q][p][q], symmetric in (p, q); p < o occupied, p >= o virtual."""
    n = o + v
    iu, ju = np.triu_indices(n)
    npair = iu.size
    B = np.empty((naux, n, n), dtype=np.float64)
    z = normal(seed, STREAM_B, naux * npair).reshape(naux, npair) * sigma
    B[:, iu, ju] = z
    B[:, ju, iu] = z
    return B


def orbital_energies(o: int, v: int, seed: int):
    eo = np.sort(-2.0 + 1.7 * uniform(seed, STREAM_EOCC, o))
    ev = np.sort(0.1 + 4.9 * uniform(seed, STREAM_EVIR, v))
    return eo, ev


def singles(o: int, v: int, seed: int, sigma: float = 1e-3) -> np.ndarray:
    return (normal(seed, STREAM_T1, o * v) * sigma).reshape(o, v)


def make_instance(o: int, v: int, naux: int | None = None, seed: int = 1,
                  device=None) -> Instance:
    """Build one instance.  device=None: numpy on the host.  Otherwise the
    random draws happen on the host and the integral products are formed with
    torch float64 matmuls on that device (large configurations)."""
    if o < 1 or v < 1:
        raise ValueError("o and v must be >= 1")
    if naux is None:
        naux = 3 * (o + v)
    B = factors(o, v, naux, seed)
    eo, ev = orbital_energies(o, v, seed)
    t1 = singles(o, v, seed)
    Bov = np.ascontiguousarray(B[:, :o, o:])          # [Q][i][a]
    Boo = np.ascontiguousarray(B[:, :o, :o])          # [Q][i][j]
    Bvv = np.ascontiguousarray(B[:, o:, o:])          # [Q][a][b]
    del B
    if device is None:
        Xov = Bov.reshape(naux, o * v)
        ovov = (Xov.T @ Xov).reshape(o, v, o, v)
        Bvo = np.ascontiguousarray(Bov.transpose(0, 2, 1)).reshape(naux, v * o)
        vvvo = (Bvv.reshape(naux, v * v).T @ Bvo).reshape(v, v, v, o)
        ooov = (Boo.reshape(naux, o * o).T @ Xov).reshape(o, o, o, v)
        dd = (eo[:, None, None, None] + eo[None, None, :, None]
              - ev[None, :, None, None] - ev[None, None, None, :])   # [i][a][j][b]
        t2 = np.ascontiguousarray((ovov / dd).transpose(0, 2, 1, 3))  # [i][j][a][b]
        return Instance(o, v, naux, seed, eo, ev, t1, t2, vvvo, ooov, ovov)

    import torch
    f64 = torch.float64
    dev = torch.device(device)
    Xov = torch.from_numpy(Bov).to(dev).reshape(naux, o * v)
    ovov = (Xov.T @ Xov).reshape(o, v, o, v)
    Bvo = torch.from_numpy(Bov).to(dev).permute(0, 2, 1).contiguous().reshape(naux, v * o)
    Bvv_d = torch.from_numpy(Bvv).to(dev).reshape(naux, v * v)
    del Bvv
    vvvo = (Bvv_d.T @ Bvo).reshape(v, v, v, o)
    del Bvv_d, Bvo
    ooov = (torch.from_numpy(Boo).to(dev).reshape(naux, o * o).T @ Xov).reshape(o, o, o, v)
    eo_d = torch.from_numpy(eo).to(dev)
    ev_d = torch.from_numpy(ev).to(dev)
    dd = (eo_d[:, None, None, None] + eo_d[None, None, :, None]
          - ev_d[None, :, None, None] - ev_d[None, None, None, :])
    t2 = (ovov / dd).permute(0, 2, 1, 3).contiguous()
    t1_d = torch.from_numpy(t1).to(dev)
    return Instance(o, v, naux, seed, eo_d, ev_d, t1_d, t2.to(f64),
                    vvvo.contiguous(), ooov.contiguous(), ovov.contiguous())


def make_instance_slices(o: int, v: int, naux: int | None, seed: int, occ):
    """The instance of make_instance(o, v, naux, seed) on the host without the
    full vvvo block (vvvo=None), plus {q: (xy|zq) as [v][v][v]} for the
    occupied indices in ``occ`` -- what a sample of tasks reads."""
    if naux is None:
        naux = 3 * (o + v)
    B = factors(o, v, naux, seed)
    eo, ev = orbital_energies(o, v, seed)
    t1 = singles(o, v, seed)
    Bov = np.ascontiguousarray(B[:, :o, o:])
    Boo = np.ascontiguousarray(B[:, :o, :o])
    Bvv = np.ascontiguousarray(B[:, o:, o:]).reshape(naux, v * v)
    del B
    Xov = Bov.reshape(naux, o * v)
    ovov = (Xov.T @ Xov).reshape(o, v, o, v)
    ooov = (Boo.reshape(naux, o * o).T @ Xov).reshape(o, o, o, v)
    dd = (eo[:, None, None, None] + eo[None, None, :, None]
          - ev[None, :, None, None] - ev[None, None, None, :])
    t2 = np.ascontiguousarray((ovov / dd).transpose(0, 2, 1, 3))
    slices = {}
    for q in sorted(set(int(x) for x in occ)):
        Bvq = np.ascontiguousarray(Bov[:, q, :])                      # [Q][z] = B^Q_{zq}
        slices[q] = (Bvv.T @ Bvq).reshape(v, v, v)
    return Instance(o, v, naux, seed, eo, ev, t1, t2, None, ooov, ovov), slices


def batch_shapes(n: int, seed: int, o_range=(4, 16), v_range=(20, 120)):
    """(o, v, naux, seed) for n independent molecules of uneven size:
    o ~ U{o_range}, v ~ U{v_range} (inclusive), naux = 3(o+v), per-instance
    seed = seed + index."""
    uo = uniform(seed, 11, n)
    uv = uniform(seed, 12, n)
    out = []
    for idx in range(n):
        o = o_range[0] + int(uo[idx] * (o_range[1] - o_range[0] + 1))
        v = v_range[0] + int(uv[idx] * (v_range[1] - v_range[0] + 1))
        out.append((o, v, 3 * (o + v), seed + idx))
    return out


@dataclass
class Mp2Instance:
    """One synthetic RI-MP2 problem: orbital energies and the fitting
    coefficients C[gamma][a][i] (numpy on the host or torch tensors)."""
    o: int
    v: int
    naux: int
    seed: int
    eps_occ: object
    eps_vir: object
    C: object

    def arrays(self):
        return (self.eps_occ, self.eps_vir, self.C)

    def to(self, device):
        import torch
        conv = []
        for a in self.arrays():
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
            conv.append(t.to(device=device, dtype=torch.float64).contiguous())
        return Mp2Instance(self.o, self.v, self.naux, self.seed, *conv)


def make_mp2_instance(o: int, v: int, naux: int | None = None, seed: int = 1) -> Mp2Instance:
    """The RI-MP2 inputs of the synthetic system of make_instance(o, v, naux,
    seed): the same orbital energies and, as fitting coefficients, the
    occupied-virtual block of the same factors, C[gamma][a][i] = B^gamma_{i,o+a}
    (so that sum_gamma C^gamma_ai C^gamma_bj is that system's (ia|jb))."""
    if o < 1 or v < 1:
        raise ValueError("o and v must be >= 1")
    if naux is None:
        naux = 3 * (o + v)
    B = factors(o, v, naux, seed)
    eo, ev = orbital_energies(o, v, seed)
    C = np.ascontiguousarray(B[:, :o, o:].transpose(0, 2, 1))
    return Mp2Instance(o, v, naux, seed, eo, ev, C)
