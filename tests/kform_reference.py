"""Test-only CPU re-derivation of X2C in the paper's orthonormal K-form (Sec. II.A).

It is the second formulation the oracle is pinned against: the paper's appendix
(Eqs. A1-A19) proves that the K-form U^L = K R' K^-1, U^S = 2c K p^-1 X' R' K^-1
(Eq. 22) equals the non-orthogonal form of Eq. 23 that the oracle uses.  Every matrix
operation is counted by kind, so the counts can be compared with Tables II and III.

Steps (Sec. II.A):
  T K = S K t (Eq. 11),  p = sqrt(2 t),  K^-1 by inversion (Sec. III)
  V~ = K+ V K (Eq. 15),  W~^q = p^-1 K+ W^q K p^-1 (Eq. 17)
  H^p = [[V~, c p], [c p, W~ - 2c^2]] (Eq. 14), diagonalised (Eq. 18)
  X' = C_S' (C_L')^-1 (Eq. 19),  R' = (1 + X'+ X')^-1/2 by diagonalisation (Eqs. 20, 38-39)
  H = (R' K^-1)+ (V~ + c p X' + c X'+ p + X'+ (W~ - 2c^2) X') (R' K^-1) (Eq. 21)
  U^L = K R' K^-1,  U^S = 2c K p^-1 X' R' K^-1 (Eq. 22)
"""
from __future__ import annotations

from collections import Counter

import numpy as np
import scipy.linalg as sla

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


class Ops:
    """Counts matrix operations by (kind, dimension label)."""

    def __init__(self, N, two_c):
        self.N, self.two_c, self.c = N, two_c, Counter()

    def _lab(self, A, B=None):
        d = A.shape[0] // self.N
        cplx = np.iscomplexobj(A) or (B is not None and np.iscomplexobj(B))
        return f"{d if d > 1 else ''}N_{'complex' if cplx else 'real'}"

    def mult(self, A, B):
        self.c["mult_" + self._lab(A, B)] += 1
        return A @ B

    def inv(self, A):
        self.c["inv_" + self._lab(A)] += 1
        return np.linalg.inv(A)

    def diag(self, A, B=None):
        self.c["diag_" + self._lab(A)] += 1
        return sla.eigh(A, B)


def x2c_kform(m: dict, c: float):
    """h, U^L, U^S and the operation counts of the K-form X2C."""
    two_c = "Wx" in m
    S, T, V, W0 = m["S"], m["T"], m["V"], m["W0"]
    N = S.shape[0]
    ops = Ops(N, two_c)
    t, K = ops.diag(T, S)
    p = np.sqrt(2.0 * t)
    Kinv = ops.inv(K)
    Vt = ops.mult(ops.mult(K.T, V), K)
    Wq = [W0] + ([m["Wx"], m["Wy"], m["Wz"]] if two_c else [])
    Wt = [ops.mult(ops.mult(K.T, w), K) / np.outer(p, p) for w in Wq]
    if two_c:
        I2 = np.eye(2)
        Vt2 = np.kron(I2, Vt).astype(np.complex128)
        Wt2 = np.kron(I2, Wt[0]) + 1j * sum(np.kron(s, w) for s, w in zip(SIGMA, Wt[1:]))
        p2 = np.concatenate([p, p])
        K2 = np.kron(I2, K)
        Kinv2 = np.kron(I2, Kinv)
    else:
        Vt2, Wt2, p2, K2, Kinv2 = Vt, Wt[0], p, K, Kinv
    n = Vt2.shape[0]
    cp = np.diag(c * p2)
    Hp = np.block([[Vt2, cp], [cp, Wt2 - 2 * c * c * np.eye(n)]])
    eps, C = ops.diag(Hp)
    CL, CS = C[:n, n:], C[n:, n:]
    Xp = ops.mult(CS, ops.inv(CL))
    a, Ca = ops.diag(np.eye(n) + ops.mult(Xp.conj().T, Xp))
    Rp = ops.mult(Ca * a**-0.5, Ca.conj().T)
    XWX = ops.mult(ops.mult(Xp.conj().T, Wt2 - 2 * c * c * np.eye(n)), Xp)
    cpX = (c * p2)[:, None] * Xp
    inner = Vt2 + cpX + cpX.conj().T + XWX
    RK = ops.mult(Rp, Kinv2)
    h = ops.mult(ops.mult(RK.conj().T, inner), RK)
    UL = ops.mult(K2, RK)
    US = 2 * c * ops.mult(K2 / p2[None, :], ops.mult(Xp, RK))
    return dict(h=h, UL=UL, US=US, eps_pos=eps[n:], ops=dict(ops.c))
