"""Why the synthetic spin-orbit blocks are whitened (and where that stops being enough).

The configured recipe, Wk_ij = 0.02 g_ij sqrt(|W0_ii W0_jj|), makes the atomic W of Eq. 5 far
from negative semi-definite: negative-energy solutions of Eq. 1 then rise above -c^2, so the
positive-energy selection of Sec. II (eps + c^2 > 0, exactly half the spectrum) fails and X2C
is undefined for one silver atom already.  The whitened recipe (same seeded g and strength,
Wk = 0.02 R (g_k / rho) R with R = (-W0_free)^1/2) keeps every atomic W negative semi-definite,
so every atomic problem splits, which is all that DLU needs.  The molecular W of a whole
cluster adds the other nuclei's potential and the atom-other-atom blocks, and from Ag18 (s48)
on the whole-cluster 4c spectrum no longer splits either: the small analogue of the refusal of
the Ag55 two-component full X2C.

Counting: by Sylvester's law of inertia the number of eigenvalues of D C = M C E above -c^2
equals the number of positive eigenvalues of D + c^2 M (M is positive definite)."""
import numpy as np
import pytest

import oracle as O
from paper_1303_4446_gb300 import workload as w


def above_minus_c2(m, c=O.C_LIGHT):
    """(number of eigenvalues of Eq. 1 above -c^2, half the 4c dimension)."""
    S, T, V, W = O.spinor_inputs(m)
    c2 = c * c
    A = np.block([[V + c2 * S, T], [T, W / (4 * c2) - T / 2]])
    return int((np.linalg.eigvalsh(A) > 0).sum()), S.shape[0]


@pytest.mark.parametrize("basis", ["s30", "s48"])
def test_configured_recipe_breaks_the_atomic_split(basis):
    m = w.free_atom_integrals(47.0, basis)
    m["Wx"], m["Wy"], m["Wz"] = w.so_blocks_configured(47.0, basis)
    for x in (m["Wx"], m["Wy"], m["Wz"]):
        assert np.array_equal(x, -x.T)
    pos, half = above_minus_c2(m)
    assert pos > half, (pos, half)
    with pytest.raises(ArithmeticError):
        O.x2c_full(m)


@pytest.mark.parametrize("basis", ["s30", "s48"])
def test_whitened_recipe_keeps_the_atomic_split(basis):
    m = w.atomic_inputs(47.0, basis, True)
    pos, half = above_minus_c2(m)
    assert pos == half
    r = O.x2c_full(m)
    assert len(r["eps_pos"]) == half


def test_smallest_cluster_whose_whole_spectrum_does_not_split():
    """Ag17 s48 two-component splits half/half at -c^2; Ag18 has two states too many above
    -c^2, and the oracle refuses its full X2C."""
    m17 = w.molecule_inputs(w.silver_cluster(17, "s48"), True)
    pos, half = above_minus_c2(m17)
    assert pos == half
    m18 = w.molecule_inputs(w.silver_cluster(18, "s48"), True)
    pos, half = above_minus_c2(m18)
    assert pos == half + 2, (pos, half)
    with pytest.raises(ArithmeticError):
        O.x2c_full(m18)
