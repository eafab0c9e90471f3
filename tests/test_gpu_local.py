"""GPU parity of the DLH approximation and of the picture-change transformation.

DLH (Sec. III.A): the same-atom blocks come from the DLU pair assembly, the rest is T + V;
the oracle's x2c_dlh decides every element.  Picture change (Sec. II): P2c = U^L+ P^LL U^L +
U^S+ P^SS U^S through the DLU assembly with the operator in place of the Dirac matrix; the
oracle decides, and with P^LL = S, P^SS = T/2c^2 the result must reproduce S (the
renormalisation condition Eq. 9): exactly for full-X2C transforms, on the same-atom blocks
for atomic ones."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu
C = O.C_LIGHT


@pytest.fixture(scope="module")
def ctx():
    c = x.Context(0)
    yield c
    c.close()


def dev(m):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.items()}


def parts_of(ref, two_c):
    return list(O.quaternion_parts(ref)) if two_c else [ref]


def rel(got, ref_full, two_c):
    scale = np.abs(ref_full).max()
    return max(np.abs(g.cpu().numpy() - r).max() for g, r in zip(got, parts_of(ref_full, two_c))) / scale


@pytest.mark.parametrize("two_c", [False, True])
@pytest.mark.parametrize("mode", ["free_atom", "molecular_block"])
@pytest.mark.parametrize("prec", [x.PREC_FP64, x.PREC_SPLIT_BF16])
def test_dlh_matches_oracle(ctx, two_c, mode, prec):
    # molecular-block mode with split precision: every atom has its own transforms, so each
    # (U_A, U_B) pair class is assembled by its own launches (up to 64 classes per build)
    mol = w.silver_cluster(4, "s30")
    m = w.molecule_inputs(mol, two_c)
    at = w.atomic_inputs(47.0, "s30", two_c)
    g, gk = dev(m), dev(at)
    mb = mode == "molecular_block"
    h = x.x2c_build_dlu(ctx, g, mol.offsets, [0] * 4, [gk], two_component=two_c, precision=prec,
                        dlu_potential=x.DLU_MOLECULAR_BLOCK if mb else x.DLU_FREE_ATOM, local_approx=x.LOCAL_DLH)
    ctx.status()
    ref = O.x2c_dlh(m, mol.offsets, None if mb else [at] * 4)
    tol = 1e-9 if prec == x.PREC_SPLIT_BF16 else 1e-10
    assert rel(h, ref, two_c) <= tol
    # atom-other-atom blocks: T + V exactly, spin parts zero
    off = mol.offsets
    a, b = slice(off[0], off[1]), slice(off[2], off[3])
    assert torch.equal(h[0][a, b], g["T"][a, b] + g["V"][a, b])
    for q in range(1, len(h)):
        assert not h[q][a, b].any()


@pytest.mark.parametrize("two_c", [False, True])
def test_dlu_molecular_block_split(ctx, two_c):
    # the paper-literal atomic blocks (Eq. 43 read literally): ten pair classes for Ag4
    mol = w.silver_cluster(4, "s30")
    m = w.molecule_inputs(mol, two_c)
    at = w.atomic_inputs(47.0, "s30", two_c)
    h = x.x2c_build_dlu(ctx, dev(m), mol.offsets, [0] * 4, [dev(at)], two_component=two_c,
                        precision=x.PREC_SPLIT_BF16, dlu_potential=x.DLU_MOLECULAR_BLOCK)
    ctx.status()
    assert rel(h, O.x2c_dlu(m, mol.offsets, None)["h"], two_c) <= 1e-9


def test_dlh_ag13_two_component_split(ctx):
    mol = w.silver_cluster(13, "s30")
    m = w.molecule_inputs(mol, True)
    at = w.atomic_inputs(47.0, "s30", True)
    h = x.x2c_build_dlu(ctx, dev(m), mol.offsets, [0] * 13, [dev(at)], two_component=True,
                        precision=x.PREC_SPLIT_BF16, local_approx=x.LOCAL_DLH)
    ctx.status()
    assert rel(h, O.x2c_dlh(m, mol.offsets, [at] * 13), True) <= 1e-9


@pytest.mark.parametrize("two_c", [False, True])
@pytest.mark.parametrize("prec", [x.PREC_FP64, x.PREC_SPLIT_BF16])
def test_picture_change_dlu_transforms(ctx, two_c, prec):
    mol = w.silver_cluster(4, "s30")
    m = w.molecule_inputs(mol, two_c)
    at = w.atomic_inputs(47.0, "s30", two_c)
    (UL, US), = x.x2c_atomic_transforms(ctx, [dev(at)], two_component=two_c)
    g = dev(m)
    PSS = g["T"] / (2 * C * C)
    P = x.x2c_picture_change(ctx, g["S"], PSS, mol.offsets, [0] * 4, [(UL, US)], [30], two_component=two_c,
                             precision=prec)
    ctx.status()
    # oracle: the same property with the oracle's own atomic transforms (Eq. 42)
    S, T, V, W = O.spinor_inputs(m)
    d = O.x2c_dlu(m, mol.offsets, [at] * 4)
    ref = O.picture_change(d["UL"], d["US"], S, T / (2 * C * C))
    tol = 1e-9 if prec == x.PREC_SPLIT_BF16 else 1e-10
    assert rel(P, ref, two_c) <= tol
    # renormalisation (Eq. 9) on the same-atom blocks: the atomic U carry the atoms' own S, T
    off = mol.offsets
    for A in range(4):
        a = slice(off[A], off[A + 1])
        err = (P[0][a, a] - g["S"][a, a]).abs().max().item()
        assert err <= (1e-9 if prec == x.PREC_SPLIT_BF16 else 1e-10)
        for q in range(1, len(P)):
            assert P[q][a, a].abs().max().item() <= 1e-9


@pytest.mark.parametrize("two_c", [False, True])
def test_picture_change_full_x2c_renormalisation(ctx, two_c):
    mol = w.silver_cluster(2, "s30")
    m = w.molecule_inputs(mol, two_c)
    g = dev(m)
    full = x.x2c_build_full(ctx, g, two_component=two_c, want_U=True)
    ctx.status()
    n = mol.nbf
    PSS = [g["T"] / (2 * C * C)] + ([None] * 3)
    P = x.x2c_picture_change(ctx, g["S"], PSS, [0, n], [0], [(full["UL"], full["US"])], [n], two_component=two_c)
    ctx.status()
    assert (P[0] - g["S"]).abs().max().item() <= 1e-10 * g["S"].abs().max().item()
    for q in range(1, len(P)):
        assert P[q].abs().max().item() <= 1e-10
    if two_c:
        # a spin-dependent small-component operator: the full spinor W / 4c^2
        SS = [g["W0"] / (4 * C * C)] + [g[k] / (4 * C * C) for k in ("Wx", "Wy", "Wz")]
        P2 = x.x2c_picture_change(ctx, g["V"], SS, [0, n], [0], [(full["UL"], full["US"])], [n], two_component=True,
                                  so_same_atom_only=False)
        ctx.status()
        S_, T_, V_, W_ = O.spinor_inputs(m)
        r = O.x2c_full(m)
        ref = O.picture_change(r["UL"], r["US"], V_, W_ / (4 * C * C))
        assert rel(P2, ref, True) <= 1e-10


@pytest.mark.parametrize("prec", [x.PREC_FP64, x.PREC_SPLIT_BF16])
def test_light_atom_identity_transforms(ctx, prec):
    """The non-relativistic treatment of light atoms (Sec. III.A): identity transforms for the
    light kind, the heavy kind's own, through x2c_build_dlu_with_transforms."""
    mol = w.Molecule(w.fcc_sites(3), np.array([47.0, 1.0, 47.0]), ["s30"] * 3)
    m = w.molecule_inputs(mol, True)
    ag = w.atomic_inputs(47.0, "s30", True)
    (UL, US), = x.x2c_atomic_transforms(ctx, [dev(ag)], two_component=True)
    eye = torch.eye(30, dtype=torch.float64, device="cuda")
    zero = torch.zeros_like(eye)
    ident = ([eye, zero, zero, zero], [eye, zero, zero, zero])
    h = x.x2c_build_dlu_with_transforms(ctx, dev(m), mol.offsets, [0, 1, 0], [(UL, US), ident], [30, 30],
                                        two_component=True, precision=prec)
    ctx.status()
    r = O.x2c_full(ag)
    e2 = (np.eye(60), np.eye(60))
    ref = O.dlu_from_transforms(m, mol.offsets, [(r["UL"], r["US"]), e2, (r["UL"], r["US"])])["h"]
    tol = 1e-9 if prec == x.PREC_SPLIT_BF16 else 1e-10
    assert rel(h, ref, True) <= tol
