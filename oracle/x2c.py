"""Plain, slow, FP64 CPU oracle of the X2C one-electron Hamiltonian and its DLU variant.

TEST INFRASTRUCTURE (see the package docstring): only tests/, smoke() and bench.py's
CPU-baseline leg may use it.

Every function states the passage of the paper it writes out.  Equation numbers are
those of the paper (Peng, Middendorf, Weigend, Reiher, J. Chem. Phys. 138, 184105):

* Eq. 1    modified Dirac equation  D C = M C E,  D = [[V, T], [T, W/4c^2 - T]],
           M = diag(S, T/2c^2)                                       (Sec. II)
* Eq. 4    spin-diagonal S, T, V;  Eq. 5  W from W0, Wx, Wy, Wz      (Sec. II)
* Eq. 8    decoupling transformation  H = U^L+ V U^L + U^L+ T U^S + U^S+ T U^L
                                          + U^S+ (W/4c^2 - T) U^S    (Sec. II)
* Eq. 9    renormalisation condition                                  (Sec. II)
* Eq. A1   X = C_S^+ (C_L^+)^{-1}                                     (Appendix)
* Eq. 23   U^L = S^-1/2 (S^-1/2 (S + X+ T X / 2c^2) S^-1/2)^-1/2 S^1/2,
           U^S = X U^L  (non-orthogonal form)                         (Sec. II.A)
* Eqs. 42-43  DLU: U^{L,S} = direct sum of atomic blocks U^{L,S}_AA computed by the
           same matrix function from atomic inputs, then Eq. 8      (Sec. III.A)
* DLH      relativistic same-atom blocks only, T + V elsewhere        (Sec. III.A)
* picture change of a property:  U^L+ P^LL U^L + U^S+ P^SS U^S        (Sec. II, Eq. 8)

No blocking, fusion or reordering beyond these definitions; LAPACK (via scipy) does the
generalised Hermitian eigenproblem and the linear solves.

Parity status: every function here is pinned by tests/test_oracle_*.py against closed
forms, invariants and an independent K-form re-derivation (see those files).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

C_LIGHT = 137.035999

_SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def spinor_inputs(m: dict):
    """2c spinor-basis matrices of Eqs. 4-5, spin-blocked order (alpha block first).

    Input dict: S, T, V, W0 real N x N and optionally Wx, Wy, Wz (real antisymmetric).
    Returns (S, T, V, W) as complex 2N x 2N when Wx is present, else the real N x N
    scalar matrices (the spin-free case: the SO parts are dropped, Sec. II)."""
    if "Wx" not in m:
        return m["S"], m["T"], m["V"], m["W0"]
    I2 = np.eye(2)
    S = np.kron(I2, m["S"]).astype(np.complex128)
    T = np.kron(I2, m["T"]).astype(np.complex128)
    V = np.kron(I2, m["V"]).astype(np.complex128)
    # Eq. 5: W = [[W0 + i Wz, Wy + i Wx], [-Wy + i Wx, W0 - i Wz]]
    W = np.kron(I2, m["W0"]) + 1j * sum(np.kron(s, m[k]) for s, k in zip(_SIGMA, ("Wx", "Wy", "Wz")))
    return S, T, V, W


def _hermitian_power(A, k):
    """Principal power A^k of a Hermitian positive-definite matrix via its eigenvectors
    (the procedure given for the inverse square root in Sec. III, Eqs. 38-39)."""
    w, C = np.linalg.eigh(A)
    if np.min(w) <= 0:
        raise np.linalg.LinAlgError("matrix is not positive definite")
    return (C * w**k) @ C.conj().T


def x2c_full(m: dict, c: float = C_LIGHT):
    """Exact-decoupling (X2C) one-electron Hamiltonian of the whole system.

    Steps, in the paper's notation:
      1. D and M of Eq. 1 from S, T, V, W (Eqs. 4-5).
      2. Solve D C = M C E (generalised Hermitian; M is positive definite).
      3. Positive-energy solutions: eps + c^2 > 0 (Sec. II, after Eq. 3); exactly half
         of the spectrum must qualify.
      4. X = C_S^+ (C_L^+)^{-1}  (Eq. A1), by a linear solve.
      5. U^L, U^S from the non-orthogonal form, Eq. 23.
      6. h from Eq. 8.
    Returns dict(h, UL, US, X, eps_pos, eps_neg)."""
    S, T, V, W = spinor_inputs(m)
    n = S.shape[0]
    c2 = c * c
    Z = np.zeros_like(S)
    D = np.block([[V, T], [T, W / (4 * c2) - T]])
    M = np.block([[S, Z], [Z, T / (2 * c2)]])
    eps, C = sla.eigh(D, M)
    neg, pos = eps[:n], eps[n:]
    if not (neg.max() + c2 < 0 < pos.min() + c2):
        raise ArithmeticError("positive/negative energy spectrum does not split at -c^2")
    CL, CS = C[:n, n:], C[n:, n:]
    X = sla.solve(CL.T, CS.T).T  # X CL = CS
    St = S + X.conj().T @ T @ X / (2 * c2)
    Sm = _hermitian_power(S, -0.5)
    Sp = _hermitian_power(S, 0.5)
    UL = Sm @ _hermitian_power(Sm @ St @ Sm, -0.5) @ Sp
    US = X @ UL
    h = _utrans(UL, US, V, T, W, c)
    return dict(h=h, UL=UL, US=US, X=X, eps_pos=pos, eps_neg=neg)


def _utrans(UL, US, V, T, W, c):
    """Eq. 8: h = [U^L+ U^S+] [[V, T], [T, W/4c^2 - T]] [U^L; U^S]."""
    Wp = W / (4 * c * c) - T
    ULh, USh = UL.conj().T, US.conj().T
    h = ULh @ V @ UL + ULh @ T @ US + USh @ T @ UL + USh @ Wp @ US
    return h


def electronic_eigenvalues(h, S):
    """Eigenvalues of the two-component electrons-only equation h C = S C eps (Eq. 3)."""
    return sla.eigh(h, S, eigvals_only=True)


def dlu_atomic_inputs(m_mol: dict, offsets, a: int, atomic: dict | None):
    """Atomic input matrices for atom a (Eq. 43).

    atomic is None  -> diagonal blocks of the molecular matrices (literal reading of
                       Eq. 43: the atomic blocks of the input matrices);
    atomic is dict  -> free-atom matrices (potential of atom a's own nucleus only)."""
    o0, o1 = int(offsets[a]), int(offsets[a + 1])
    if atomic is not None:
        return atomic
    return {k: v[o0:o1, o0:o1].copy() for k, v in m_mol.items()}


def dlu_atomic_transforms(m_mol: dict, offsets, atomic_per_atom=None, c: float = C_LIGHT):
    """U^L_AA, U^S_AA of every atom by the full X2C matrix function of atomic inputs
    (Eqs. 42-43).  atomic_per_atom: list (len L) of free-atom input dicts or None."""
    L = len(offsets) - 1
    out = []
    cache = {}
    for a in range(L):
        atomic = None if atomic_per_atom is None else atomic_per_atom[a]
        key = id(atomic) if atomic is not None else None
        if key is not None and key in cache:
            out.append(cache[key])
            continue
        r = x2c_full(dlu_atomic_inputs(m_mol, offsets, a, atomic), c)
        out.append((r["UL"], r["US"]))
        if key is not None:
            cache[key] = out[-1]
    return out


def _blockdiag_spinor(blocks, offsets, two_c: bool):
    """Direct sum over atoms (Eq. 42) in the spin-blocked 2c ordering."""
    N = int(offsets[-1])
    if not two_c:
        U = np.zeros((N, N))
        for a, B in enumerate(blocks):
            o0, o1 = int(offsets[a]), int(offsets[a + 1])
            U[o0:o1, o0:o1] = B
        return U
    U = np.zeros((2 * N, 2 * N), dtype=np.complex128)
    for a, B in enumerate(blocks):
        o0, o1 = int(offsets[a]), int(offsets[a + 1])
        n = o1 - o0
        for s in range(2):
            for t in range(2):
                U[s * N + o0:s * N + o1, t * N + o0:t * N + o1] = B[s * n:(s + 1) * n, t * n:(t + 1) * n]
    return U


def dlu_from_transforms(m_mol: dict, offsets, transforms, c: float = C_LIGHT):
    """Eq. 8 with the block-diagonal U^{L,S} of Eq. 42 built from given atomic transforms
    (one (U^L_AA, U^S_AA) pair per atom, real n x n or spin-blocked complex 2n x 2n), e.g.
    identity matrices for light atoms (the non-relativistic treatment of Sec. III.A).
    Returns dict(h, UL, US)."""
    two_c = "Wx" in m_mol
    UL = _blockdiag_spinor([u[0] for u in transforms], offsets, two_c)
    US = _blockdiag_spinor([u[1] for u in transforms], offsets, two_c)
    S, T, V, W = spinor_inputs(m_mol)
    return dict(h=_utrans(UL, US, V, T, W, c), UL=UL, US=US)


def x2c_dlu(m_mol: dict, offsets, atomic_per_atom=None, c: float = C_LIGHT):
    """DLU Hamiltonian: U^{L,S} = (+)_A U^{L,S}_AA (Eq. 42), then Eq. 8 with the
    molecular V, T, W (Sec. III.A).  Returns dict(h, UL, US)."""
    return dlu_from_transforms(m_mol, offsets, dlu_atomic_transforms(m_mol, offsets, atomic_per_atom, c), c)


def x2c_dlh(m_mol: dict, offsets, atomic_per_atom=None, c: float = C_LIGHT):
    """Diagonal local approximation to the Hamiltonian, DLH (Sec. III.A): only the
    same-atom blocks h_AA are relativistically transformed (Eq. 8 with the atomic U_AA of
    Eq. 43, as in DLU); every atom-other-atom block is the non-relativistic T_AB + V_AB, with
    no spin-dependent part.  Written as: the DLU h, with the atom-other-atom blocks replaced
    by those of T + V (spinor form for two-component)."""
    two_c = "Wx" in m_mol
    h = x2c_dlu(m_mol, offsets, atomic_per_atom, c)["h"]
    S, T, V, W = spinor_inputs(m_mol)
    N = int(offsets[-1])
    atom = np.repeat(np.arange(len(offsets) - 1), np.diff(np.asarray(offsets)))
    same = atom[:, None] == atom[None, :]
    if two_c:
        same = np.kron(np.ones((2, 2), dtype=bool), same)
    assert same.shape == h.shape == (N * (2 if two_c else 1),) * 2
    return np.where(same, h, T + V)


def x2c_nab(m_mol: dict, offsets, neighbours, atomic_per_atom=None, c: float = C_LIGHT):
    """Neighbouring-atomic-blocks approximation (named at the end of Sec. III.A for linear
    scaling; read here as): the DLU Hamiltonian on the pair blocks of neighbouring atoms
    (neighbours[A][B] true; every same-atom block counts) and the non-relativistic T_AB + V_AB,
    with no spin-dependent part, on every other block.  neighbours = all true gives DLU, the
    identity gives DLH."""
    two_c = "Wx" in m_mol
    h = x2c_dlu(m_mol, offsets, atomic_per_atom, c)["h"]
    S, T, V, W = spinor_inputs(m_mol)
    L = len(offsets) - 1
    atom = np.repeat(np.arange(L), np.diff(np.asarray(offsets)))
    nb = np.asarray(neighbours, dtype=bool) | np.eye(L, dtype=bool)
    keep = nb[atom[:, None], atom[None, :]]
    if two_c:
        keep = np.kron(np.ones((2, 2), dtype=bool), keep)
    return np.where(keep, h, T + V)


def picture_change(UL, US, PLL, PSS):
    """Picture-change transformation of a one-electron property operator without
    large-small coupling (Sec. II: the reason the decoupling transforms are kept):
    P2c = U^L+ P^LL U^L + U^S+ P^SS U^S, i.e. Eq. 8 with [[P^LL, 0], [0, P^SS]] in place of
    the Dirac matrix.  All matrices in one representation (real N x N, or the spin-blocked
    complex 2N x 2N of spinor_inputs)."""
    return UL.conj().T @ PLL @ UL + US.conj().T @ PSS @ US


def dlu_pair_block(blocks: dict, ULa, USa, ULb, USb, c: float = C_LIGHT):
    """One pair block h_AB of the DLU Hamiltonian: Eq. 8 restricted to rows of atom A
    and columns of atom B, which is exact because U^{L,S} are block diagonal (Eq. 42).

    blocks: V, T, W0 (and Wx, Wy, Wz for 2c) restricted to [A rows, B cols] (real).
    U*: atomic transforms (real n x n, or complex 2n x 2n spin-blocked)."""
    two_c = "Wx" in blocks
    if two_c:
        I2 = np.eye(2)
        V = np.kron(I2, blocks["V"]).astype(np.complex128)
        T = np.kron(I2, blocks["T"]).astype(np.complex128)
        W = np.kron(I2, blocks["W0"]) + 1j * sum(
            np.kron(s, blocks[k]) for s, k in zip(_SIGMA, ("Wx", "Wy", "Wz")))
    else:
        V, T, W = blocks["V"], blocks["T"], blocks["W0"]
    Wp = W / (4 * c * c) - T
    ha = ULa.conj().T, USa.conj().T
    return ha[0] @ V @ ULb + ha[0] @ T @ USb + ha[1] @ T @ ULb + ha[1] @ Wp @ USb


def quaternion_parts(h2):
    """(h0, h1, h2, h3) of a 2N x 2N spin-blocked matrix h = I2 (x) h0 + i sum_k s_k (x) h_k
    (the structure of Eq. 5); the four parts are read from the alpha-alpha and
    alpha-beta blocks."""
    n = h2.shape[0] // 2
    aa, ab = h2[:n, :n], h2[:n, n:]
    return aa.real.copy(), ab.imag.copy(), ab.real.copy(), aa.imag.copy()


def from_quaternion(h0, h1, h2, h3):
    """Inverse of quaternion_parts."""
    I2 = np.eye(2)
    return np.kron(I2, h0) + 1j * sum(np.kron(s, x) for s, x in zip(_SIGMA, (h1, h2, h3)))


def dirac_ground_state(Z: float, c: float = C_LIGHT, n: int = 1):
    """Point-nucleus Dirac energy (minus rest energy) of the ns_1/2 level (kappa = -1):
    E = c^2 [ (1 + (Z/c)^2 / (n - 1 + sqrt(1 - (Z/c)^2))^2)^{-1/2} - 1 ]."""
    g = np.sqrt(1.0 - (Z / c) ** 2)
    return c * c * (1.0 / np.sqrt(1.0 + (Z / c) ** 2 / (n - 1 + g) ** 2) - 1.0)
