"""Pins of the seeded input generator (integrals S, T, V, W0, geometry, SO blocks).

Each check is independent of the closed forms in ints.c: library special functions,
one-centre closed forms, finite differences of other integrals, and a 1D quadrature of
the Gaussian transform of 1/r.
"""
import numpy as np
import pytest
from scipy import integrate, special

from paper_1303_4446_gb300 import workload as w


@pytest.mark.parametrize("T", [0.0, 1e-10, 1e-3, 0.3, 1.0, 4.0, 11.0, 24.99, 25.01, 39.0, 41.0, 120.0, 1e4])
def test_boys_against_incomplete_gamma(T):
    F = w.boys012(T)
    for m in range(3):
        if T == 0.0:
            ref = 1.0 / (2 * m + 1)
        else:
            a = m + 0.5
            ref = special.gamma(a) * special.gammainc(a, T) / (2.0 * T**a)
        assert abs(F[m] - ref) <= 1e-14 * abs(ref), (m, F[m], ref)


def _one_centre(alpha, Z):
    n = len(alpha)
    return w.integrals_points(np.zeros((n, 3)), alpha, np.zeros((1, 3)), [Z])


def test_one_centre_closed_forms():
    al = w.basis_exponents("s30")[::3]
    Z = 47.0
    I = _one_centre(al, Z)
    a, b = np.meshgrid(al, al, indexing="ij")
    p = a + b
    Na, Nb = (2 * a / np.pi) ** 0.75, (2 * b / np.pi) ** 0.75
    S = (2 * np.sqrt(a * b) / p) ** 1.5
    T = 3 * a * b / p * S
    V = -Z * Na * Nb * 2 * np.pi / p
    # W0 = 4ab <g_a| r^2 (-Z/r) |g_b> = -4abZ Na Nb * 4 pi / (2 p^2)
    W0 = -8 * np.pi * a * b * Z * Na * Nb / p**2
    for k, ref in (("S", S), ("T", T), ("V", V), ("W0", W0)):
        assert np.allclose(I[k], ref, rtol=1e-13, atol=0), k
    assert np.allclose(np.diag(I["W0"]), -2 * np.pi * Z * (2 * al / np.pi) ** 1.5, rtol=1e-13)


def _two_fn(A, B, a, b, nuc, Zs):
    return w.integrals_points(np.array([A, B]), np.array([a, b]), nuc, Zs)


def _mixed_second_derivative(f, A, B, h):
    """sum_k d^2 f / dA_k dB_k by central differences."""
    tot = 0.0
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        tot += (f(A + e, B + e) - f(A + e, B - e) - f(A - e, B + e) + f(A - e, B - e)) / (4 * h * h)
    return tot


@pytest.mark.parametrize("a,b", [(0.7, 1.3), (0.2, 3.0), (2.5, 2.5)])
def test_kinetic_and_w0_from_finite_differences(a, b):
    """T_ab = 1/2 <grad g_a|grad g_b> and W0_ab = <grad g_a|V|grad g_b> are mixed
    derivatives of S_ab and V_ab with respect to the two centres."""
    A = np.array([0.1, -0.2, 0.3])
    B = np.array([0.6, 0.4, -0.5])
    nuc = np.array([[0.0, 0.0, 0.0], [1.1, -0.7, 0.2]])
    Zs = np.array([3.0, 2.0])
    S = lambda A_, B_: _two_fn(A_, B_, a, b, nuc, Zs)["S"][0, 1]
    V = lambda A_, B_: _two_fn(A_, B_, a, b, nuc, Zs)["V"][0, 1]
    # Richardson extrapolation removes the O(h^2) truncation error
    fd = lambda f: (4 * _mixed_second_derivative(f, A, B, 1e-3)
                    - _mixed_second_derivative(f, A, B, 2e-3)) / 3
    I = _two_fn(A, B, a, b, nuc, Zs)
    assert abs(I["T"][0, 1] - 0.5 * fd(S)) < 1e-7 * abs(I["T"][0, 1])
    assert abs(I["W0"][0, 1] - fd(V)) < 1e-7 * abs(I["W0"][0, 1])


def test_nuclear_attraction_by_quadrature():
    """V_ab = -Z (2/sqrt(pi)) int_0^inf <g_a| exp(-u^2 |r-C|^2) |g_b> du; the integrand is a
    three-centre Gaussian overlap, so this checks the Boys-function route independently."""
    a, b = 0.8, 0.35
    A, B, C = np.array([0.0, 0.0, 0.0]), np.array([0.9, 0.3, -0.4]), np.array([-0.5, 0.7, 0.6])
    Z = 5.0
    Na, Nb = (2 * a / np.pi) ** 0.75, (2 * b / np.pi) ** 0.75

    def overlap3(u):
        c = u * u
        q = a + b + c
        P = (a * A + b * B + c * C) / q
        ex = a * A @ A + b * B @ B + c * C @ C - q * P @ P
        return Na * Nb * (np.pi / q) ** 1.5 * np.exp(-ex)

    val, err = integrate.quad(overlap3, 0, np.inf, epsabs=1e-14, epsrel=1e-13, limit=200)
    ref = -Z * 2 / np.sqrt(np.pi) * val
    I = w.integrals_points(np.array([A, B]), np.array([a, b]), C[None, :], [Z])
    assert abs(I["V"][0, 1] - ref) < 1e-11 * abs(ref)


def test_symmetry_and_sign_of_molecular_integrals():
    mol = w.silver_cluster(4, "s30")
    I = w.integrals(mol)
    for k in ("S", "T", "V", "W0"):
        assert np.array_equal(I[k], I[k].T)
    assert np.all(np.linalg.eigvalsh(I["S"]) > 0)
    assert np.all(np.linalg.eigvalsh(I["T"]) > 0)
    # an attractive potential: V and W0 = sum_k p_k V p_k are negative definite
    assert np.linalg.eigvalsh(I["V"]).max() < 0
    assert np.linalg.eigvalsh(I["W0"]).max() < 0


def test_fcc_sites_order_and_shells():
    s = w.fcc_sites(4) / (w.FCC_A / 2)
    assert np.array_equal(s, [[0, 0, 0], [-1, -1, 0], [-1, 0, -1], [-1, 0, 1]])
    d2 = np.rint((w.fcc_sites(309) / (w.FCC_A / 2)) ** 2).sum(1).astype(int)
    shells = np.bincount(d2)
    assert list(shells[[0, 2, 4, 6, 8]]) == [1, 12, 6, 24, 12]
    assert d2[54] == 8 and d2[55] == 10  # Ag55 ends on a complete shell
    assert len(np.unique(w.fcc_sites(309), axis=0)) == 309


def test_so_blocks_antisymmetric_and_keep_w_negative():
    for basis in ("s30", "s48"):
        Wx, Wy, Wz = w.so_blocks(47.0, basis)
        for x in (Wx, Wy, Wz):
            assert np.array_equal(x, -x.T)
            assert np.abs(x).max() > 0
        if basis == "s30":  # s48's W0 is indefinite at the rounding level of its largest entry
            W0 = w.free_atom_integrals(47.0, basis)["W0"]
            sig = (np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]]))
            W = np.kron(np.eye(2), W0) + 1j * sum(np.kron(s, x) for s, x in zip(sig, (Wx, Wy, Wz)))
            assert np.linalg.eigvalsh(W).max() < 0
    # deterministic in the seed
    a = w.so_blocks(47.0, "s30", seed=5)[0]
    b = w.so_blocks(47.0, "s30", seed=5)[0]
    c = w.so_blocks(47.0, "s30", seed=6)[0]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_block_integrals_match_full():
    mol = w.silver_cluster(3, "s30")
    full = w.integrals(mol)
    blk = w.integrals_block(mol, slice(30, 60), slice(0, 90))
    for k in full:
        assert np.array_equal(blk[k], full[k][30:60, 0:90])
