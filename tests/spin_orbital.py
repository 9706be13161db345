"""Textbook spin-orbital (T) energy, used only as an independent pin.

The closed-shell spatial quantities are expanded to spin orbitals
(P = 2p + spin) and the spin-orbital (T) expression of Crawford & Schaefer
(Rev. Comput. Chem. 14, 33 (2000), Sec. "(T)") is evaluated:

  D t_c = P(i/jk) P(a/bc) [ sum_e t^{ae}_{jk} <ei||bc> - sum_m t^{bc}_{im} <ma||jk> ]
  D t_d = P(i/jk) P(a/bc) t^a_i <jk||bc>
  E(T)  = (1/36) sum t_c D (t_c + t_d),  D = f_ii+f_jj+f_kk-f_aa-f_bb-f_cc,

with P(i/jk) f(ijk) = f(ijk) - f(jik) - f(kji).  Spin adaptation of the
closed-shell amplitudes: t^{AB}_{IJ} = t^{ab}_{ij} d(A,I) d(B,J)
- t^{ba}_{ij} d(A,J) d(B,I) and t^A_I = t^a_i d(A,I), where d compares spins.
Memory (2o)^3 (2v)^3: tiny sizes only.
"""
import numpy as np


def _same(x, y):
    return (x[:, None] == y[None, :]).astype(np.float64)


def energy(inst):
    """(E(T), E[4]) from the spin-orbital formula; E[4] uses t_c alone."""
    o, v = inst.o, inst.v
    O, V = 2 * o, 2 * v
    so, sv = np.arange(O) % 2, np.arange(V) % 2
    io, iv = np.arange(O) // 2, np.arange(V) // 2
    dov = _same(so, sv)
    t1 = np.asarray(inst.t1)[io][:, iv] * dov
    t2s = np.asarray(inst.t2)[io][:, io][:, :, iv][:, :, :, iv]
    t2 = (t2s * dov[:, None, :, None] * dov[None, :, None, :]
          - t2s.transpose(0, 1, 3, 2) * dov[:, None, None, :] * dov[None, :, :, None])
    ovov = np.asarray(inst.ovov)[io][:, iv][:, :, io][:, :, :, iv]        # [J][B][K][C]
    jkbc = ovov.transpose(0, 2, 1, 3) * dov[:, None, :, None] * dov[None, :, None, :]
    oovv = jkbc - jkbc.transpose(0, 1, 3, 2)                              # <JK||BC>
    vvvo = np.asarray(inst.vvvo)[iv][:, iv][:, :, iv][:, :, :, io]        # (eb|ci): [E][B][C][I]
    eibc = vvvo.transpose(0, 3, 1, 2) * _same(sv, sv)[:, None, :, None] * dov[None, :, None, :]
    vovv = eibc - eibc.transpose(0, 1, 3, 2)                              # <EI||BC>
    ooov = np.asarray(inst.ooov)[io][:, io][:, :, io][:, :, :, iv]        # (mj|ka): [M][J][K][A]
    majk = ooov.transpose(0, 3, 1, 2) * _same(so, so)[:, None, :, None] * _same(sv, so)[None, :, None, :]
    ovoo = majk - majk.transpose(0, 1, 3, 2)                              # <MA||JK>
    fo = np.asarray(inst.eps_occ)[io]
    fv = np.asarray(inst.eps_vir)[iv]
    D = (fo[:, None, None, None, None, None] + fo[None, :, None, None, None, None]
         + fo[None, None, :, None, None, None] - fv[None, None, None, :, None, None]
         - fv[None, None, None, None, :, None] - fv[None, None, None, None, None, :])

    def P(x):
        x = x - np.einsum("jikabc->ijkabc", x) - np.einsum("kjiabc->ijkabc", x)
        return x - np.einsum("ijkbac->ijkabc", x) - np.einsum("ijkcba->ijkabc", x)

    tc = P(np.einsum("jkae,eibc->ijkabc", t2, vovv)
           - np.einsum("imbc,majk->ijkabc", t2, ovoo)) / D
    td = P(np.einsum("ia,jkbc->ijkabc", t1, oovv)) / D
    return float(np.sum(tc * D * (tc + td)) / 36.0), float(np.sum(tc * D * tc) / 36.0)
