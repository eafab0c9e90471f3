"""Plain FP64 CPU oracle of the two decouplings built on the free-particle Foldy-Wouthuysen
transformation: BSS (Sec. II.B) and DKHn with the exponential parametrisation (Sec. II.C,
Table I), each for the whole system and as atomic transforms for the local DLU scheme
(Sec. III.A, Eqs. 42-43).

TEST INFRASTRUCTURE (see the package docstring): only tests/, smoke() and bench.py's
CPU-baseline leg may use it.

Both methods start from the orthonormal kinetic basis of Sec. II.A:
  T K = S K t (Eq. 11),  K+ S K = 1,  p = sqrt(2 t),
  V~ = K+ V K,  W~ = p^-1 K+ W K p^-1  (Eqs. 15-17),
  H^p = [[V~, c p], [c p, W~ - 2 c^2]]  (Eq. 14),
and the free-particle transformation U0 built from E0 = sqrt(c^2 p^2 + c^4),
A = sqrt((E0 + c^2) / 2 E0), B = sqrt((E0 - c^2) / 2 E0)  (Sec. II.B).

Reading of U0's signs: U0 is the orthogonal matrix that brings the free-particle part of H^p
(V = W = 0) to diag(E0 - c^2, -E0 - c^2) with the electronic solutions in the first block
column.  With the coupling +c p of Eq. 14 that first column is [A; B] (second: [-B; A]), so
H^0 = U0^T H^p U0 has the blocks printed in Sec. II.B on its diagonal,
  E = A V~ A + B W~ B + E0 - c^2,   E' = B V~ B + A W~ A - E0 - c^2,
and the off-diagonal block O1 = B W~ A - A V~ B (the printed sign and the printed U0
correspond to the opposite sign of the small-component basis).  The decoupling transforms
follow from this U0 by U0 [1; X''] (BSS) and U0 [U^LL; U^SL] (DKH); the pins (exact
decoupling, the free particle, the renormalisation condition, c -> infinity) hold only with
consistent signs.

Parity status: pinned by tests/test_oracle_fw.py (Table I multiplication counts for n = 2..14,
the free particle, exact decoupling of BSS, DKHn eigenvalue errors of order n + 1 in the
potential strength, Taylor coefficients of the exactly transformed Hamiltonian computed with
matrix exponentials, the renormalisation condition, c -> infinity).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .x2c import C_LIGHT, _blockdiag_spinor, _hermitian_power, _utrans, spinor_inputs


# ------------------------------------------------------------------ orthonormal kinetic basis
def kinetic_basis(m: dict, c: float = C_LIGHT):
    """Sec. II.A: K, p of T K = S K t (Eq. 11) and the orthonormal blocks V~, W~ (Eqs. 15-17).

    Two-component inputs give spinor (complex 2N x 2N, spin-blocked) V~, W~ and the spinor
    K = 1_2 (x) K; spin-free inputs stay real N x N.  Returns dict(K, Kinv, p, Vt, Wt, S, T, V, W)
    with Kinv = K+ S (the inverse of K, Sec. III)."""
    t, Ks = sla.eigh(m["T"], m["S"])
    if np.min(t) <= 0:
        raise np.linalg.LinAlgError("T is not positive definite")
    S, T, V, W = spinor_inputs(m)
    two_c = "Wx" in m
    K = np.kron(np.eye(2), Ks) if two_c else Ks
    p = np.sqrt(2.0 * t)
    if two_c:
        p = np.concatenate([p, p])
    Kinv = K.conj().T @ S
    Vt = K.conj().T @ V @ K
    Wt = (K.conj().T @ W @ K) / np.outer(p, p)
    return dict(K=K, Kinv=Kinv, p=p, Vt=Vt, Wt=Wt, S=S, T=T, V=V, W=W)


def free_particle_fw(p, c: float = C_LIGHT):
    """E0, A, B of the free-particle transformation (Sec. II.B), as vectors over the kinetic
    eigenfunctions."""
    E0 = np.sqrt(c * c * p * p + c**4)
    A = np.sqrt((E0 + c * c) / (2 * E0))
    B = np.sqrt((E0 - c * c) / (2 * E0))
    return E0, A, B


def _hp(kb, c):
    """H^p of Eq. 14 as a dense 4c matrix."""
    Vt, Wt, p = kb["Vt"], kb["Wt"], kb["p"]
    cp = np.diag(c * p).astype(Vt.dtype)
    return np.block([[Vt, cp], [cp, Wt - 2 * c * c * np.eye(len(p))]])


def _u0(A, B):
    """The free-particle transformation, first block column [A; B] (see the module header)."""
    dA, dB = np.diag(A), np.diag(B)
    return np.block([[dA, -dB], [dB, dA]])


def _back(kb, Y, R, c):
    """U^L = K Y_L R K^-1, U^S = 2c K p^-1 Y_S R K^-1 from a 4c column block Y (H^p frame)."""
    M = len(kb["p"])
    K, Kinv, p = kb["K"], kb["Kinv"], kb["p"]
    UL = K @ Y[:M] @ R @ Kinv
    US = 2 * c * (K / p) @ Y[M:] @ R @ Kinv
    return UL, US


# ------------------------------------------------------------------ BSS (Sec. II.B)
def bss_full(m: dict, c: float = C_LIGHT):
    """BSS Hamiltonian of the whole system.

    Steps of Sec. II.B: K and H^p; H^0 = U0^T H^p U0; its positive-energy solutions (eps > -c^2,
    exactly half); X'' = C_S'' (C_L'')^-1; R'' = (1 + X''+ X'')^-1/2; the transforms
    U^L = K (A - B X'') R'' K^-1, U^S = 2c K p^-1 (B + A X'') R'' K^-1 (U0 [1; X''] R'', signs as
    in the module header); h by Eq. 8.  Returns dict(h, UL, US, eps_pos)."""
    kb = kinetic_basis(m, c)
    M = len(kb["p"])
    E0, A, B = free_particle_fw(kb["p"], c)
    U0 = _u0(A, B)
    H0 = U0.T @ _hp(kb, c) @ U0
    eps, C = np.linalg.eigh(H0)
    c2 = c * c
    if not (eps[:M].max() + c2 < 0 < eps[M:].min() + c2):
        raise ArithmeticError("positive/negative energy spectrum does not split at -c^2")
    CL, CS = C[:M, M:], C[M:, M:]
    X = sla.solve(CL.T, CS.T).T  # X CL = CS
    R = _hermitian_power(np.eye(M) + X.conj().T @ X, -0.5)
    Y = U0 @ np.vstack([np.eye(M), X])
    UL, US = _back(kb, Y, R, c)
    h = _utrans(UL, US, kb["V"], kb["T"], kb["W"], c)
    return dict(h=h, UL=UL, US=US, eps_pos=eps[M:])


# ------------------------------------------------------------------ DKHn (Sec. II.C)
class _Term:
    """A term of the transformed Hamiltonian in the H^0 frame, of a given order in the
    potential: even (blocks U upper, L lower) or odd (block O, upper right; the lower left is
    its adjoint).  Blocks are evaluated only when asked for, and every matrix product counts
    as one multiplication (the bookkeeping of Sec. II.C: a commutator with an odd term costs
    one product per diagonal block, one with an even term two products for the odd block;
    lower blocks are computed only when a later commutator needs them)."""

    def __init__(self, dkh, order, parity, kind, **kw):
        self.dkh, self.order, self.parity, self.kind = dkh, order, parity, kind
        self.kw = kw
        self.val = {}

    def block(self, part):
        if part not in self.val:
            self.val[part] = self._eval(part)
        return self.val[part]

    def _eval(self, part):
        d = self.dkh
        if self.kind == "given":
            return self.kw[part]
        if self.kind == "sum":
            return sum(cf * t.block(part) for cf, t in self.kw["terms"])
        if self.kind == "comm":  # [W_k, X]
            Wk, X = self.kw["W"].block("O"), self.kw["X"]
            if X.parity == "even":  # odd result: W X' - X W
                assert part == "O"
                return d.mul(Wk, X.block("L")) - d.mul(X.block("U"), Wk)
            Xo = X.block("O")
            if part == "U":  # W X+ + (W X+)+
                P = d.mul(Wk, Xo.conj().T)
                return P + P.conj().T
            P = d.mul(Wk.conj().T, Xo)  # lower: -(W+ X + (W+ X)+)
            return -(P + P.conj().T)
        if self.kind == "W":  # [W_k, E0] = -O_k: W_ij = O_ij / (E_i + E_j), no product
            return self.kw["src"].block("O") / d.Esum
        raise ValueError(self.kind)


class _DKH:
    """Sequential unitary transformations U_k = exp(W_k), k = 1, 2, ..., of the free-particle
    transformed Hamiltonian H^0 = E0 + E1 + O1 (Sec. II.C), each W_k chosen so that
    [W_k, E0] = -O_k removes the odd term of order k, every exp(ad W_k) expanded and cut at
    order n in the potential."""

    def __init__(self, kb, n, c):
        self.n, self.c = n, c
        M = len(kb["p"])
        E0, A, B = free_particle_fw(kb["p"], c)
        self.E0, self.A, self.B, self.M = E0, A, B, M
        self.Esum = E0[:, None] + E0[None, :]
        self.mults = 0
        Vt, Wt = kb["Vt"], kb["Wt"]
        # blocks of H^0 = U0^T H^p U0 beyond its free part (Sec. II.B; module header)
        E1 = A[:, None] * Vt * A[None, :] + B[:, None] * Wt * B[None, :]
        E1p = B[:, None] * Vt * B[None, :] + A[:, None] * Wt * A[None, :]
        O1 = B[:, None] * Wt * A[None, :] - A[:, None] * Vt * B[None, :]
        self.H = {(1, "even"): _Term(self, 1, "even", "given", U=E1, L=E1p),
                  (1, "odd"): _Term(self, 1, "odd", "given", O=O1)}
        self.W = []

    def mul(self, X, Y):
        self.mults += 1
        return X @ Y

    def transform(self, k):
        """H <- exp(ad W_k) H, cut at order n; ad W_k (E0) = -O_k."""
        Ok = self.H.get((k, "odd"))
        if Ok is None:
            return False
        Wk = _Term(self, k, "odd", "W", src=Ok)
        self.W.append(Wk)
        parts = {}
        for (l, par), Mt in self.H.items():
            parts.setdefault((l, par), []).append((1.0, Mt))
            prev, j = Mt, 1
            while l + j * k <= self.n:
                t = _Term(self, l + j * k, "odd" if prev.parity == "even" else "even", "comm", W=Wk, X=prev)
                parts.setdefault((t.order, t.parity), []).append((1.0 / math.factorial(j), t))
                if Mt is Ok:  # ad^(j+1) E0 = -ad^j O_k
                    parts[(t.order, t.parity)].append((-1.0 / math.factorial(j + 1), t))
                prev, j = t, j + 1
        parts[(k, "odd")] = []  # O_k + [W_k, E0] = 0
        self.H = {}
        for key, terms in parts.items():
            if not terms:
                continue
            if len(terms) == 1 and terms[0][0] == 1.0:
                self.H[key] = terms[0][1]
            else:
                self.H[key] = _Term(self, key[0], key[1], "sum", terms=terms)
        return True


def dkh_hamiltonian(m: dict, order: int, c: float = C_LIGHT, kb=None):
    """DKHn Hamiltonian of the whole system (Sec. II.C): the transformations k = 1 .. n/2
    (later ones change only terms beyond order n), then H_DKHn = E0 - c^2 + sum_{l=1..n} E_l
    (upper blocks only), back-transformed to the primitive basis by K^-1.

    Returns dict(h, H (orthonormal frame), mults): mults counts the matrix products of the
    transformation and Hamiltonian (Table I's P(n))."""
    if order < 1:
        raise ValueError("order >= 1")
    kb = kb or kinetic_basis(m, c)
    d = _DKH(kb, order, c)
    for k in range(1, order // 2 + 1):
        d.transform(k)
    H = np.diag(d.E0 - c * c).astype(kb["Vt"].dtype)
    for l in range(1, order + 1):
        t = d.H.get((l, "even"))
        if t is not None:
            H = H + t.block("U")
    Kinv = kb["Kinv"]
    h = Kinv.conj().T @ H @ Kinv
    return dict(h=h, H=H, mults=d.mults)


def dkh_transforms(m: dict, order: int, c: float = C_LIGHT):
    """DKHn decoupling transforms U^L, U^S (Sec. II.C, for DLU and picture change).

    The transformed frame is H^(n) = V H^0 V^-1 with V = exp(W_n) ... exp(W_1); its electronic
    (upper) block belongs to the H^0-frame columns V^-1 [1; 0] = exp(-W_1) ... exp(-W_n) [1; 0],
    every exponential cut after the powers of order <= n ([U^LL; U^SL], W_1 .. W_n).  That
    column block is renormalised, R'' = (U^LL+ U^LL + U^SL+ U^SL)^-1/2 (the reading of R'' for
    DKH: the cut exponentials are not exactly unitary), and taken to the primitive basis like
    BSS: U0 [U^LL; U^SL] R''.  Returns dict(UL, US)."""
    kb = kinetic_basis(m, c)
    d = _DKH(kb, order, c)
    for k in range(1, order + 1):
        if not d.transform(k):
            break
    M = d.M
    Y = np.vstack([np.eye(M), np.zeros((M, M))]).astype(kb["Vt"].dtype)
    for Wt in reversed(d.W):
        k = Wt.order
        w = Wt.block("O")
        Wfull = np.block([[np.zeros((M, M)), w], [-w.conj().T, np.zeros((M, M))]])
        acc, term = Y.copy(), Y
        for i in range(1, order // k + 1):
            term = -(Wfull @ term) / i
            acc = acc + term
        Y = acc
    R = _hermitian_power(Y.conj().T @ Y, -0.5)
    UL, US = _back(kb, _u0(d.A, d.B) @ Y, R, c)
    return dict(UL=UL, US=US)


# ------------------------------------------------------------------ DLU with BSS / DKHn
def atomic_transforms(m_mol: dict, offsets, atomic_per_atom, method, c: float = C_LIGHT):
    """U^L_AA, U^S_AA of every atom (Eqs. 42-43) by `method`: "bss" or ("dkh", n); the
    atomic inputs are the free-atom dicts of atomic_per_atom (or the molecular diagonal blocks
    where an entry is None)."""
    out, cache = [], {}
    for a in range(len(offsets) - 1):
        atomic = atomic_per_atom[a] if atomic_per_atom is not None else None
        key = id(atomic) if atomic is not None else None
        if key is not None and key in cache:
            out.append(cache[key])
            continue
        if atomic is None:
            o0, o1 = int(offsets[a]), int(offsets[a + 1])
            atomic = {k: v[o0:o1, o0:o1].copy() for k, v in m_mol.items()}
        if method == "bss":
            r = bss_full(atomic, c)
        else:
            r = dkh_transforms(atomic, method[1], c)
        out.append((r["UL"], r["US"]))
        if key is not None:
            cache[key] = out[-1]
    return out


def dlu(m_mol: dict, offsets, atomic_per_atom, method, c: float = C_LIGHT):
    """DLU Hamiltonian (Sec. III.A) with BSS or DKHn atomic transforms: Eq. 8 with the
    block-diagonal U^L, U^S of Eq. 42.  Returns dict(h, UL, US)."""
    tr = atomic_transforms(m_mol, offsets, atomic_per_atom, method, c)
    two_c = "Wx" in m_mol
    UL = _blockdiag_spinor([u[0] for u in tr], offsets, two_c)
    US = _blockdiag_spinor([u[1] for u in tr], offsets, two_c)
    S, T, V, W = spinor_inputs(m_mol)
    return dict(h=_utrans(UL, US, V, T, W, c), UL=UL, US=US)
