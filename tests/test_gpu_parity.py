"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances (from the method's FP64 floor, see the oracle pins):
  h:        max|dh| <= 1e-10 * max|h|   (every quaternion part, relative to max|h|)
  U^L:      max|dU| <= 1e-10 * max|U|
  U^S:      max|dU| <= 1e-9  * max|U|   (U^S is the worse-conditioned factor; the 40-digit
                                         brute force puts the oracle at 2e-12)
  orbitals: |d eps| <= max(1e-8 Eh, 10 u max|eps|) for the bound (eps < 0) eigenvalues of
            h over S (u = 2^-53; for the 48-function basis the FP64 floor 10 u ||H|| is
            1.6e-8 Eh, above the 1e-8 target).
"""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")

import kform_reference as K
import oracle as O
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu
H_TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = x.Context(0)
    yield c
    c.close()


def dev(m):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.items()}


def parts(h2c, two_c):
    return list(O.quaternion_parts(h2c)) if two_c else [h2c]


def assert_parts(got, ref_full, two_c, tol=H_TOL, what="h"):
    ref = parts(ref_full, two_c)
    scale = np.abs(ref_full).max()
    for q, (g, r) in enumerate(zip(got, ref)):
        err = np.abs(g.cpu().numpy() - r).max() / scale
        assert err <= tol, f"{what} part {q}: {err:.3e}"


def orbital_check(h_parts, m, two_c, ref_h, floor_h=None):
    """Bound orbital energies of h over S against the oracle's, within max(1e-8 Eh, 10 u
    max|eps|) or, with floor_h, within twice the spread between the oracle and a second exact
    CPU formulation (floor_h = that formulation's h): in an ill-conditioned S metric the
    eigenvalues of two FP64 formulations already differ by more than 1e-8 Eh."""
    S = m["S"] if not two_c else np.kron(np.eye(2), m["S"])
    hg = O.from_quaternion(*[p.cpu().numpy() for p in h_parts]) if two_c else h_parts[0].cpu().numpy()
    e = sla.eigh(hg, S, eigvals_only=True)
    e0 = sla.eigh(ref_h, S, eigvals_only=True)
    b = e0 < 0
    tol = max(1e-8, 10 * 2.0**-53 * np.abs(e0).max())
    if floor_h is not None:
        e1 = sla.eigh(floor_h, S, eigvals_only=True)
        tol = max(tol, 2 * np.abs(e1 - e0)[b].max())
    assert np.abs(e - e0)[b].max() < tol


@pytest.mark.parametrize("two_c", [False, True])
@pytest.mark.parametrize("basis", ["s30", "s48"])
def test_full_x2c_single_atom(ctx, basis, two_c):
    m = w.atomic_inputs(47.0, basis, two_c)
    r = O.x2c_full(m)
    out = x.x2c_build_full(ctx, dev(m), two_component=two_c, want_U=True)
    ctx.status()
    assert_parts(out["h"], r["h"], two_c)
    assert_parts(out["UL"], r["UL"], two_c, 1e-10, "UL")
    assert_parts(out["US"], r["US"], two_c, 1e-9, "US")
    orbital_check(out["h"], m, two_c, r["h"])


@pytest.mark.parametrize("two_c", [False, True])
def test_full_x2c_ag4(ctx, two_c):
    mol = w.silver_cluster(4, "s30")
    m = w.molecule_inputs(mol, two_c)
    r = O.x2c_full(m)
    out = x.x2c_build_full(ctx, dev(m), two_component=two_c)
    ctx.status()
    assert_parts(out["h"], r["h"], two_c)
    orbital_check(out["h"], m, two_c, r["h"])


@pytest.mark.parametrize("two_c", [False, True])
@pytest.mark.parametrize("L,basis", [(5, "s48"), (13, "s30")])
def test_full_x2c_blocked_factorisation(ctx, L, basis, two_c):
    """Systems above the one-CTA factorisation size (n = 240, 390): blocked Cholesky and
    triangular inverse by GEMMs, multi-CTA Gershgorin scaling and checks."""
    mol = w.silver_cluster(L, basis)
    m = w.molecule_inputs(mol, two_c)
    r = O.x2c_full(m)
    out = x.x2c_build_full(ctx, dev(m), two_component=two_c, want_U=True)
    ctx.status()
    assert_parts(out["h"], r["h"], two_c)
    assert_parts(out["UL"], r["UL"], two_c, 1e-9, "UL")
    # cond(S) = 5e6 (Ag5 s48), 2e6 (Ag13 s30): orbital floor from the K-form re-derivation
    orbital_check(out["h"], m, two_c, r["h"], floor_h=K.x2c_kform(m, x.C_LIGHT)["h"])


def test_not_positive_definite_blocked(ctx):
    """The blocked factorisation reports a non-positive pivot in a late leaf block too."""
    mol = w.silver_cluster(5, "s48")
    m = w.molecule_inputs(mol, False)
    m["S"] = m["S"].copy()
    m["S"][200, 200] = -1.0
    x.x2c_build_full(ctx, dev(m))
    with pytest.raises(x.X2CError) as e:
        ctx.status()
    assert e.value.code == 4


@pytest.mark.parametrize("two_c", [False, True])
@pytest.mark.parametrize("mode", [x.DLU_FREE_ATOM, x.DLU_MOLECULAR_BLOCK])
def test_dlu_ag4(ctx, two_c, mode):
    mol = w.silver_cluster(4, "s30")
    m = w.molecule_inputs(mol, two_c)
    kind = w.atomic_inputs(47.0, "s30", two_c)
    at = [kind] * 4 if mode == x.DLU_FREE_ATOM else None
    r = O.x2c_dlu(m, mol.offsets, at)
    h = x.x2c_build_dlu(ctx, dev(m), mol.offsets, [0] * 4, [dev(kind)], two_component=two_c,
                        dlu_potential=mode)
    ctx.status()
    assert_parts(h, r["h"], two_c)
    orbital_check(h, m, two_c, r["h"])


@pytest.mark.parametrize("two_c", [False, True])
def test_dlu_mixed_basis_ragged(ctx, two_c):
    """Atoms of 30 and 48 functions in one molecule (ragged pair blocks and tiles)."""
    coords = w.fcc_sites(5)
    mol = w.Molecule(coords, np.full(5, 47.0), ["s30", "s48", "s30", "s48", "s48"])
    m = w.molecule_inputs(mol, two_c)
    k30, k48 = w.atomic_inputs(47.0, "s30", two_c), w.atomic_inputs(47.0, "s48", two_c)
    kinds_idx = [0, 1, 0, 1, 1]
    at = [k30 if k == 0 else k48 for k in kinds_idx]
    r = O.x2c_dlu(m, mol.offsets, at)
    h = x.x2c_build_dlu(ctx, dev(m), mol.offsets, kinds_idx, [dev(k30), dev(k48)], two_component=two_c)
    ctx.status()
    assert_parts(h, r["h"], two_c)


def test_dlu_general_so_all_pairs(ctx):
    """so_same_atom_only = 0: Wx, Wy, Wz on every pair block enter the middle matrix."""
    mol = w.silver_cluster(3, "s30")
    m = w.molecule_inputs(mol, True)
    rng = np.random.default_rng(3)
    N = mol.nbf
    for k in ("Wx", "Wy", "Wz"):  # add antisymmetric inter-atomic SO couplings
        a = 1e-3 * rng.standard_normal((N, N)) * np.sqrt(np.abs(np.outer(np.diag(m["W0"]), np.diag(m["W0"]))))
        for A in range(3):
            o = slice(mol.offsets[A], mol.offsets[A + 1])
            a[o, o] = 0
        m[k] = m[k] + (a - a.T)
    kind = w.atomic_inputs(47.0, "s30", True)
    r = O.x2c_dlu(m, mol.offsets, [kind] * 3)
    h = x.x2c_build_dlu(ctx, dev(m), mol.offsets, [0] * 3, [dev(kind)], two_component=True,
                        so_same_atom_only=False)
    ctx.status()
    assert_parts(h, r["h"], True)


def test_dlu_single_atom_equals_full(ctx):
    m = w.atomic_inputs(47.0, "s48", True)
    g = dev(m)
    h = x.x2c_build_dlu(ctx, g, [0, 48], [0], [g], two_component=True)
    f = x.x2c_build_full(ctx, g, two_component=True)
    ctx.status()
    for a, b in zip(h, f["h"]):
        assert torch.equal(a, b) or (a - b).abs().max().item() <= 1e-14 * b.abs().max().item()


def test_single_function_atoms(ctx):
    """Degenerate sizes: atoms with one primitive each."""
    coords = np.array([[0, 0, 0], [0, 0, 3.0], [0, 2.5, 0]])
    mol = w.Molecule(coords, np.array([47.0, 47.0, 47.0]), ["s30"] * 3)
    keep = np.array([14, 44, 74])  # one mid-range exponent per atom
    m = {k: v[np.ix_(keep, keep)] for k, v in w.molecule_inputs(mol, False).items()}
    offs = np.array([0, 1, 2, 3])
    r = O.x2c_dlu(m, offs)
    h = x.x2c_build_dlu(ctx, dev(m), offs, dlu_potential=x.DLU_MOLECULAR_BLOCK)
    ctx.status()
    assert_parts(h, r["h"], False)


def test_batched_equals_single(ctx):
    mols = [w.silver_cluster(n, b) for n, b in ((2, "s30"), (3, "s48"), (1, "s30"), (4, "s30"))]
    kinds = {b: w.atomic_inputs(47.0, b, True) for b in ("s30", "s48")}
    dk = {b: dev(v) for b, v in kinds.items()}
    ms = [dev(w.molecule_inputs(mm, True)) for mm in mols]
    lays = [(mm.offsets, [0] * mm.natoms, [dk[mm.basis[0]]]) for mm in mols]
    outs = x.x2c_build_dlu_batched(ctx, ms, lays, two_component=True)
    ctx.status()
    for mm, g, lay, hb in zip(mols, ms, lays, outs):
        hs = x.x2c_build_dlu(ctx, g, *lay, two_component=True)
        ctx.status()
        for a, b in zip(hb, hs):
            assert (a - b).abs().max().item() <= 1e-13 * b.abs().max().item()


@pytest.mark.parametrize("L,approx,upper", [(3, x.LOCAL_DLU, False), (3, x.LOCAL_DLH, False),
                                             (3, x.LOCAL_DLU, True), (13, x.LOCAL_DLU, False),
                                             (13, x.LOCAL_DLU, True)])
@pytest.mark.parametrize("prec", [x.PREC_FP64, x.PREC_SPLIT_BF16])
def test_host_buffers_equal_device(ctx, L, approx, upper, prec):
    """The host-buffer call copies only the blocks the build reads: NaN in every other block
    of the host inputs must not reach h.  Free-atom DLU runs as a pipeline over row-atom
    chunks (Ag13: eight chunks), and must give the device build's h bit for bit; with
    h_upper_only it writes the upper block triangle, and any block below the diagonal it
    writes holds its exact value (the rest keeps the caller's fill)."""
    mol = w.silver_cluster(L, "s30")
    m = w.molecule_inputs(mol, True)
    kind = w.atomic_inputs(47.0, "s30", True)
    kw = dict(two_component=True, precision=prec, local_approx=approx)
    hd = x.x2c_build_dlu(ctx, dev(m), mol.offsets, [0] * L, [dev(kind)], **kw)
    ctx.status()
    atom = np.repeat(np.arange(L), np.diff(mol.offsets))
    lower = atom[:, None] > atom[None, :]
    other = atom[:, None] != atom[None, :]
    hm = {k: v.copy() for k, v in m.items()}
    hm["S"][other] = np.nan
    for k in ("Wx", "Wy", "Wz"):
        hm[k][other] = np.nan
    if approx == x.LOCAL_DLU:
        for k in ("T", "V", "W0"):
            hm[k][lower] = np.nan
    else:
        hm["W0"][other] = np.nan
    n = mol.nbf
    out = [np.full((n, n), 7.0) for _ in range(4)]
    if L == 13 and upper:  # pinned host buffers: the same-atom spin-orbit blocks are gathered by a kernel
        hm = {k: torch.from_numpy(v).pin_memory() for k, v in hm.items()}
        kind = {k: torch.from_numpy(v).pin_memory() for k, v in kind.items()}
        out = [torch.from_numpy(o).pin_memory() for o in out]
    hh = x.x2c_build_dlu_host(ctx, hm, mol.offsets, [0] * L, [kind], h_upper_only=upper, out=out, **kw)
    hh = [o.numpy() if isinstance(o, torch.Tensor) else o for o in hh]
    for a, b in zip(hd, hh):
        a = a.cpu().numpy()
        if upper:
            assert np.array_equal(a[~lower], b[~lower])
            assert np.all((b[lower] == 7.0) | (b[lower] == a[lower]))
            assert np.any(b[lower] == 7.0)  # most of the lower triangle stays unwritten
        else:
            assert np.array_equal(a, b)
    if upper:  # the lower blocks follow from the symmetry of h0 and antisymmetry of h1..h3
        full = [np.where(lower, (1.0 if q == 0 else -1.0) * b.T, b) for q, b in enumerate(hh)]
        for a, b in zip(hd, full):
            assert np.array_equal(a.cpu().numpy(), b)


def test_quaternion_to_dense(ctx):
    mol = w.silver_cluster(2, "s30")
    m = w.molecule_inputs(mol, True)
    r = O.x2c_full(m)
    out = x.x2c_build_full(ctx, dev(m), two_component=True)
    dense = x.x2c_quaternion_to_dense(out["h"])
    ctx.status()
    assert np.abs(dense.cpu().numpy() - r["h"]).max() <= H_TOL * np.abs(r["h"]).max()


def test_not_positive_definite_is_reported(ctx):
    """A failure made on the host: an overlap with a negative diagonal makes the device
    Cholesky flag X2C_ERR_NOT_POSDEF (no fault, the context stays usable)."""
    m = w.atomic_inputs(47.0, "s30", False)
    m["S"] = m["S"].copy()
    m["S"][5, 5] = -1.0
    x.x2c_build_full(ctx, dev(m), two_component=False)
    with pytest.raises(x.X2CError) as e:
        ctx.status()
    assert e.value.code == 4
    m2 = w.atomic_inputs(47.0, "s30", False)
    x.x2c_build_full(ctx, dev(m2))
    ctx.status()


def test_invalid_arguments(ctx):
    m = dev(w.atomic_inputs(47.0, "s30", False))
    with pytest.raises(x.X2CError) as e:
        x.x2c_build_dlu(ctx, m, [0, 10, 29], [0, 0], [m])  # offsets do not end at n
    assert e.value.code == 1
    with pytest.raises(x.X2CError):
        x.x2c_build_dlu(ctx, m, [0, 30], [3], [m])  # kind index out of range


def test_query_workspace(ctx):
    """x2c_query_workspace sizes a build without running it; larger systems need more."""
    small = w.silver_cluster(4, "s30")
    big = w.silver_cluster(13, "s30")
    ws = []
    for mol in (small, big):
        g = dev(w.molecule_inputs(mol, True))
        gk = dev(w.atomic_inputs(47.0, "s30", True))
        ws.append(x.x2c_query_workspace(ctx, g, mol.offsets, [0] * mol.natoms, [gk], two_component=True))
        full = x.x2c_query_workspace(ctx, g, two_component=True, full=True)
        assert full > 0
    assert 0 < ws[0] < ws[1]
