"""Pins of the BSS and DKHn oracle (oracle/fw.py), each independent of its code path:

* Table I: the number of matrix products of the DKHn Hamiltonian equals P(n) of the paper's
  "this work" column for n = 2..14 (tests/golden/dkh_mult_counts.json);
* the terms E_1 .. E_n of DKHn are the Taylor coefficients, in the strength of the potential,
  of the upper block of the free-particle-transformed H^0 after the unitary transformations
  exp(W_k) applied EXACTLY (scipy matrix exponentials, no truncated expansions), extracted by
  a discrete Cauchy integral on the unit circle (built here from the definitions: T K = S K t,
  H^p, U0, [W_k, E0] = -O_k);
* the explicit DKH2 formula of Sec. II.C, E2 = (W1 O1+ + c.t.) / 2, from a dense H^0;
* the free particle (V = W = 0): BSS and every DKHn give h = S K diag(sqrt(c^4 + 2 c^2 t) - c^2) K+ S;
* BSS decouples exactly: the eigenvalues of h over S are the positive-energy eigenvalues of
  Eq. 1 (solved here directly); its h differs from X2C's (another unitary frame);
* DKHn eigenvalues approach the exact ones monotonically as n grows (Z = 47);
* the renormalisation condition (Eq. 9) for the BSS and DKHn transforms;
* c -> infinity: h -> T + V with an error falling as c^-2."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from oracle import fw
from paper_1303_4446_gb300 import workload as w

C = O.C_LIGHT
HERE = os.path.dirname(os.path.abspath(__file__))


def exact_positive(m, c=C):
    S, T, V, W = O.spinor_inputs(m)
    c2 = c * c
    Z = np.zeros_like(S)
    D = np.block([[V, T], [T, W / (4 * c2) - T]])
    M = np.block([[S, Z], [Z, T / (2 * c2)]])
    return sla.eigh(D, M, eigvals_only=True)[S.shape[0]:]


def small_atom(two_c):
    """Every third s30 function of the silver atom (10 functions, exponents 0.04 .. 5.4e6)."""
    m = w.atomic_inputs(47.0, "s30", two_c)
    keep = np.arange(2, 30, 3)
    return {k: v[np.ix_(keep, keep)].copy() for k, v in m.items()}


def test_dkh_multiplication_counts_match_table_I():
    P = json.load(open(os.path.join(HERE, "golden", "dkh_mult_counts.json")))["P"]
    m = small_atom(False)
    for n, ref in P.items():
        assert fw.dkh_hamiltonian(m, int(n))["mults"] == ref, n
    m2 = small_atom(True)
    for n in ("2", "3", "5"):
        assert fw.dkh_hamiltonian(m2, int(n))["mults"] == P[n], n


def _free_frame(m, c=C):
    """H^0(lam) pieces from the definitions (Sec. II.A-B), independent of oracle/fw.py."""
    t, Ks = sla.eigh(m["T"], m["S"])
    S, T, V, W = O.spinor_inputs(m)
    two = "Wx" in m
    K = np.kron(np.eye(2), Ks) if two else Ks
    p = np.sqrt(2 * t)
    p = np.concatenate([p, p]) if two else p
    Vt = K.conj().T @ V @ K
    Wt = (K.conj().T @ W @ K) / np.outer(p, p)
    E0 = np.sqrt(c * c * p * p + c**4)
    A, B = np.sqrt((E0 + c * c) / (2 * E0)), np.sqrt((E0 - c * c) / (2 * E0))
    U0 = np.block([[np.diag(A), -np.diag(B)], [np.diag(B), np.diag(A)]])
    cp = np.diag(c * p)
    M = len(p)
    H0 = lambda lam: U0.T @ np.block([[lam * Vt, cp], [cp, lam * Wt - 2 * c * c * np.eye(M)]]) @ U0
    return H0, E0, M


@pytest.mark.parametrize("two_c", [False, True])
def test_dkh_terms_are_taylor_coefficients_of_the_exact_transformation(two_c):
    m = small_atom(two_c)
    n, Npts = 6, 64
    H0, E0, M = _free_frame(m)
    lam = np.exp(2j * np.pi * np.arange(Npts) / Npts)
    Hs = [H0(l) for l in lam]
    Es = E0[:, None] + E0[None, :]
    for k in range(1, n // 2 + 1):
        Ok = sum(H[:M, M:] * l ** (-k) for H, l in zip(Hs, lam)) / Npts
        wk = Ok / Es
        wf = np.block([[np.zeros((M, M)), wk], [-wk.conj().T, np.zeros((M, M))]])
        Hs = [sla.expm(l**k * wf) @ H @ sla.expm(-(l**k) * wf) for H, l in zip(Hs, lam)]
    kb = fw.kinetic_basis(m)
    d = fw._DKH(kb, n, C)
    for k in range(1, n // 2 + 1):
        d.transform(k)
    for l in range(1, n + 1):
        El = sum(H[:M, :M] * x ** (-l) for H, x in zip(Hs, lam)) / Npts
        ref = d.H[(l, "even")].block("U")
        assert np.abs(El - ref).max() <= 1e-8 * np.abs(ref).max(), l
    # and the whole DKH6 Hamiltonian of the orthonormal frame
    E = sum(sum(H[:M, :M] * x ** (-l) for H, x in zip(Hs, lam)) / Npts for l in range(n + 1))
    H = fw.dkh_hamiltonian(m, n)["H"]
    assert np.abs(E - H).max() <= 1e-12 * np.abs(H).max()


def test_dkh2_explicit_formula():
    m = small_atom(True)
    H0, E0, M = _free_frame(m)
    H = H0(1.0)
    E1 = H[:M, :M] - np.diag(E0 - C * C)
    O1 = H[:M, M:]
    W1 = O1 / (E0[:, None] + E0[None, :])
    E2 = 0.5 * (W1 @ O1.conj().T + (W1 @ O1.conj().T).conj().T)
    ref = np.diag(E0 - C * C) + E1 + E2
    got = fw.dkh_hamiltonian(m, 2)["H"]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("two_c", [False, True])
def test_free_particle(two_c):
    m = w.atomic_inputs(47.0, "s30", two_c)
    for k in ("V", "W0", "Wx", "Wy", "Wz"):
        if k in m:
            m[k] = np.zeros_like(m[k])
    t, Ks = sla.eigh(m["T"], m["S"])
    href = m["S"] @ Ks @ np.diag(np.sqrt(C**4 + 2 * C * C * t) - C * C) @ Ks.T @ m["S"]
    if two_c:
        href = np.kron(np.eye(2), href)
    scale = np.abs(href).max()
    assert np.abs(fw.bss_full(m)["h"] - href).max() <= 1e-12 * scale
    for n in (2, 3, 5):
        assert np.abs(fw.dkh_hamiltonian(m, n)["h"] - href).max() <= 1e-12 * scale, n
        t_ = fw.dkh_transforms(m, n)
        S, T, V, W = O.spinor_inputs(m)
        hu = O.x2c._utrans(t_["UL"], t_["US"], V, T, W, C)
        assert np.abs(hu - href).max() <= 1e-11 * scale, n


@pytest.mark.parametrize("basis,two_c", [("s30", False), ("s30", True), ("s48", True)])
def test_bss_exact_decoupling(basis, two_c):
    m = w.atomic_inputs(47.0, basis, two_c)
    ex = exact_positive(m)
    S = O.spinor_inputs(m)[0]
    h = fw.bss_full(m)["h"]
    assert np.abs(h - h.conj().T).max() <= 1e-13 * np.abs(h).max()
    e = sla.eigh(h, S, eigvals_only=True)
    b = ex < 0
    tol = max(1e-8, 10 * 2.0**-53 * np.abs(ex).max())
    assert np.abs(e - ex)[b].max() < tol
    hx = O.x2c_full(m)["h"]
    assert np.abs(h - hx).max() > 1e-6 * np.abs(hx).max()  # a different unitary frame


def test_dkh_eigenvalues_approach_exact_with_order():
    m = w.atomic_inputs(47.0, "s30", True)
    ex = exact_positive(m)
    S = O.spinor_inputs(m)[0]
    errs = []
    for n in (2, 3, 4, 5, 6, 8, 10):
        e = sla.eigh(fw.dkh_hamiltonian(m, n)["h"], S, eigvals_only=True)
        errs.append(np.abs(e - ex)[ex < 0].max())
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 0.1 and errs[-1] < 1e-5  # DKH2 ~ 0.46 Eh off for Z = 47, DKH10 < 1e-5


@pytest.mark.parametrize("method", ["bss", ("dkh", 2), ("dkh", 4)])
def test_renormalisation_condition(method):
    m = w.atomic_inputs(47.0, "s48", True)
    r = fw.bss_full(m) if method == "bss" else fw.dkh_transforms(m, method[1])
    S, T, V, W = O.spinor_inputs(m)
    lhs = r["UL"].conj().T @ S @ r["UL"] + r["US"].conj().T @ (T / (2 * C * C)) @ r["US"]
    assert np.abs(lhs - S).max() <= 1e-10 * np.abs(S).max()  # the K-form floor (s48: cond(S) 2e6)


@pytest.mark.parametrize("method", ["bss", "dkh2"])
def test_nonrelativistic_limit(method):
    m = w.atomic_inputs(47.0, "s30", False)
    ref = m["T"] + m["V"]
    errs = []
    for c in (1e5, 1e6, 1e7):  # the s30 atom's tightest function has p^2 ~ 1.6e7: c >> 4e3
        h = fw.bss_full(m, c)["h"] if method == "bss" else fw.dkh_hamiltonian(m, 2, c)["h"]
        errs.append(np.abs(h - ref).max() / np.abs(ref).max())
    for a, b in zip(errs, errs[1:]):
        assert 70 < a / b < 130, errs  # c^-2


@pytest.mark.parametrize("method", ["bss", ("dkh", 3)])
def test_dlu_one_atom_uses_the_atomic_transforms(method):
    """DLU of a single atom is Eq. 8 with that atom's own transforms (Eqs. 42-43)."""
    m = w.atomic_inputs(47.0, "s30", True)
    r = fw.dlu(m, [0, 30], [m], method)
    t = fw.bss_full(m) if method == "bss" else fw.dkh_transforms(m, 3)
    S, T, V, W = O.spinor_inputs(m)
    assert np.abs(r["h"] - O.x2c._utrans(t["UL"], t["US"], V, T, W, C)).max() <= 1e-13 * np.abs(r["h"]).max()
    if method == "bss":
        assert np.abs(r["h"] - t["h"]).max() <= 1e-13 * np.abs(r["h"]).max()
