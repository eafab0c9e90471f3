"""GPU parity of the BSS (Sec. II.B) and DKHn (Sec. II.C) decouplings against the CPU oracle
(oracle/fw.py), through the C ABI: full builds (h, U^L, U^S), atomic transforms, and DLU
with BSS / DKHn atomic transforms (FP64 and split-precision assembly).

Tolerances: h within 1e-10 max|h| (split assembly: 1e-9), as for X2C.  U within
max(1e-9, 10 x floor) max|U|, where the floor is how far the oracle's own U moves when the
inputs are perturbed by one unit in the last place: both methods reach U^S through the
kinetic basis, U^S = 2c K p^-1 Y_S K^-1, and the factor 2c/p of the most diffuse kinetic
eigenfunctions magnifies rounding in their small components (s48, two-component: the floor
is 6e-6 of max|U^S| while h moves by 1e-13 and U^L by 3e-10)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import fw
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = x.Context(0)
    yield c
    c.close()


def dev(m):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.items()}


def parts(h2c, two_c):
    return list(O.quaternion_parts(h2c)) if two_c else [h2c]


def err(got, ref_full, two_c):
    scale = np.abs(ref_full).max()
    return max(np.abs(g.cpu().numpy() - r).max() for g, r in zip(got, parts(ref_full, two_c))) / scale


def perturbed(m, seed=1):
    """The inputs moved by about one unit in the last place (symmetry kept)."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, a in m.items():
        e = rng.standard_normal(a.shape) * 2.0**-52 * np.abs(a)
        out[k] = a + 0.5 * (e + (e.T if k in ("S", "T", "V", "W0") else -e.T))
    return out


def u_tol(f, m, r, key, two_c):
    """max(1e-9, 10 x the oracle's own change of r[key] under perturbed inputs)."""
    rp = f(perturbed(m))
    floor = max(np.abs(a - b).max() for a, b in zip(parts(rp[key], two_c), parts(r[key], two_c)))
    return max(1e-9, 10 * floor / np.abs(r[key]).max())


CASES = [("atom", "s30", False), ("atom", "s48", True), ("ag4", "s30", False), ("ag4", "s30", True)]


def inputs(kind, basis, two_c):
    if kind == "atom":
        return w.atomic_inputs(47.0, basis, two_c)
    return w.molecule_inputs(w.silver_cluster(4, basis), two_c)


@pytest.mark.parametrize("kind,basis,two_c", CASES)
def test_bss_full(ctx, kind, basis, two_c):
    m = inputs(kind, basis, two_c)
    r = fw.bss_full(m)
    out = x.x2c_build_full(ctx, dev(m), two_component=two_c, want_U=True, decoupling=x.DEC_BSS)
    ctx.status()
    assert err(out["h"], r["h"], two_c) <= 1e-10
    assert err(out["UL"], r["UL"], two_c) <= u_tol(fw.bss_full, m, r, "UL", two_c)
    assert err(out["US"], r["US"], two_c) <= u_tol(fw.bss_full, m, r, "US", two_c)


@pytest.mark.parametrize("order", [2, 3, 4, 8])
@pytest.mark.parametrize("kind,basis,two_c", CASES)
def test_dkh_full_hamiltonian(ctx, kind, basis, two_c, order):
    m = inputs(kind, basis, two_c)
    r = fw.dkh_hamiltonian(m, order)
    out = x.x2c_build_full(ctx, dev(m), two_component=two_c, decoupling=order)
    ctx.status()
    assert err(out["h"], r["h"], two_c) <= 1e-10, order


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("basis,two_c", [("s30", False), ("s48", True)])
def test_dkh_transforms(ctx, basis, two_c, order):
    m = w.atomic_inputs(47.0, basis, two_c)
    r = fw.dkh_transforms(m, order)
    (UL, US), = x.x2c_atomic_transforms(ctx, [dev(m)], two_component=two_c, decoupling=order)
    ctx.status()
    f = lambda mm: fw.dkh_transforms(mm, order)
    assert err(UL, r["UL"], two_c) <= u_tol(f, m, r, "UL", two_c)
    assert err(US, r["US"], two_c) <= u_tol(f, m, r, "US", two_c)


@pytest.mark.parametrize("prec", [x.PREC_FP64, x.PREC_SPLIT_BF16])
@pytest.mark.parametrize("method", [x.DEC_BSS, 2, 4])
@pytest.mark.parametrize("basis,two_c", [("s30", False), ("s30", True), ("s48", True)])
def test_dlu_with_bss_and_dkh(ctx, basis, two_c, method, prec):
    mol = w.silver_cluster(4, basis)
    m = w.molecule_inputs(mol, two_c)
    kind = w.atomic_inputs(47.0, basis, two_c)
    ref = fw.dlu(m, mol.offsets, [kind] * 4, "bss" if method == x.DEC_BSS else ("dkh", method))["h"]
    h = x.x2c_build_dlu(ctx, dev(m), mol.offsets, [0] * 4, [dev(kind)], two_component=two_c, precision=prec,
                        decoupling=method)
    ctx.status()
    assert err(h, ref, two_c) <= (1e-10 if prec == x.PREC_FP64 else 1e-9)


def test_fw_size_limit_and_option_checks(ctx):
    """BSS / DKHn diagonalise T in one CTA: systems above 160 functions are refused, as is an
    order beyond the 14 of Table I."""
    m = dev(w.molecule_inputs(w.silver_cluster(4, "s48"), False))  # n = 192
    with pytest.raises(x.X2CError) as e:
        x.x2c_build_full(ctx, m, decoupling=x.DEC_BSS)
    assert e.value.code == 1
    a = dev(w.atomic_inputs(47.0, "s30", False))
    with pytest.raises(x.X2CError) as e:
        x.x2c_build_full(ctx, a, decoupling=15)
    assert e.value.code == 1
