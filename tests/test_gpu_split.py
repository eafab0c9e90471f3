"""GPU parity of the split-precision (BF16 Ozaki, tcgen05) DLU pair assembly.

The FP64 oracle decides.  The split path is exact up to the dropped digit products (S
slices of 8 bits: relative 2^-8S of the row x column scales, per stage); the tolerance
stated for it is max|dh| <= 1e-9 max|h| at the default S = 5, and the error must fall as
S grows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_1303_4446_gb300 as x
from paper_1303_4446_gb300 import workload as w

pytestmark = pytest.mark.gpu
SPLIT_TOL = 1e-9


@pytest.fixture(scope="module")
def ctx():
    c = x.Context(0)
    yield c
    c.close()


def dev(m):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in m.items()}


def rel_err(h, ref_full, two_c):
    ref = list(O.quaternion_parts(ref_full)) if two_c else [ref_full]
    scale = np.abs(ref_full).max()
    return max(np.abs(g.cpu().numpy() - r).max() for g, r in zip(h, ref)) / scale


@pytest.mark.parametrize("two_c", [False, True])
def test_split_dlu_ag4(ctx, two_c):
    mol = w.silver_cluster(4, "s30")
    m = w.molecule_inputs(mol, two_c)
    kind = w.atomic_inputs(47.0, "s30", two_c)
    ref = O.x2c_dlu(m, mol.offsets, [kind] * 4)["h"]
    g, gk = dev(m), dev(kind)
    errs = {}
    for S in (3, 4, 5, 6):
        h = x.x2c_build_dlu(ctx, g, mol.offsets, [0] * 4, [gk], two_component=two_c,
                            precision=x.PREC_SPLIT_BF16, n_slices=S)
        ctx.status()
        errs[S] = rel_err(h, ref, two_c)
    assert errs[5] <= SPLIT_TOL, errs
    assert errs[3] > errs[4] > errs[5], errs


@pytest.mark.parametrize("two_c", [False, True])
def test_split_dlu_mixed_basis(ctx, two_c):
    """Kinds of 30 and 48 functions: four classes of (A, B) sizes, padded K."""
    mol = w.Molecule(w.fcc_sites(5), np.full(5, 47.0), ["s30", "s48", "s30", "s48", "s48"])
    m = w.molecule_inputs(mol, two_c)
    k30, k48 = w.atomic_inputs(47.0, "s30", two_c), w.atomic_inputs(47.0, "s48", two_c)
    idx = [0, 1, 0, 1, 1]
    ref = O.x2c_dlu(m, mol.offsets, [k30 if i == 0 else k48 for i in idx])["h"]
    h = x.x2c_build_dlu(ctx, dev(m), mol.offsets, idx, [dev(k30), dev(k48)], two_component=two_c,
                        precision=x.PREC_SPLIT_BF16)
    ctx.status()
    assert rel_err(h, ref, two_c) <= SPLIT_TOL


def test_split_matches_fp64_path_ag55_2c(ctx):
    """Ag55 two-component (1540 pair blocks, several chunks of tiles): split vs the
    parity-tested FP64 path on every element, and vs the oracle on sampled pair blocks."""
    mol = w.silver_cluster(55, "s48")
    m = w.molecule_inputs(mol, True)
    kind = w.atomic_inputs(47.0, "s48", True)
    g, gk = dev(m), dev(kind)
    kinds = [0] * mol.natoms
    h64 = x.x2c_build_dlu(ctx, g, mol.offsets, kinds, [gk], two_component=True)
    hs = x.x2c_build_dlu(ctx, g, mol.offsets, kinds, [gk], two_component=True, precision=x.PREC_SPLIT_BF16)
    ctx.status()
    scale = max(a.abs().max().item() for a in h64)
    err = max((a - b).abs().max().item() for a, b in zip(hs, h64)) / scale
    assert err <= SPLIT_TOL, err
    # oracle on a seeded sample of pair blocks
    r = O.x2c_full(kind)
    rng = np.random.default_rng(5)
    N = mol.nbf
    for _ in range(12):
        A, B = sorted(rng.integers(0, mol.natoms, 2))
        ra = slice(mol.offsets[A], mol.offsets[A + 1])
        rb = slice(mol.offsets[B], mol.offsets[B + 1])
        blocks = {k: v[ra, rb] for k, v in m.items() if k != "S"}
        ref = O.dlu_pair_block(blocks, r["UL"], r["US"], r["UL"], r["US"])
        got = O.from_quaternion(*[p[ra, rb].cpu().numpy() for p in hs])
        assert np.abs(got - ref).max() <= SPLIT_TOL * scale


def test_batched_uneven_molecules_split_and_fp64(ctx):
    """Batched DLU over uneven clusters with both bases (the 64-molecule workload's recipe,
    8 molecules here): every molecule's h from the batched launch equals its own build, and
    matches the oracle."""
    mols = w.batched_molecules(count=8, lo=2, hi=9, seed=11)
    kinds = {b: w.atomic_inputs(47.0, b, False) for b in ("s30", "s48")}
    dk = {b: dev(v) for b, v in kinds.items()}
    ms = [w.molecule_inputs(m, False) for m in mols]
    gs = [dev(m) for m in ms]
    order = ["s30", "s48"]
    lays = [(m.offsets, [order.index(b) for b in m.basis], [dk["s30"], dk["s48"]]) for m in mols]
    for prec, tol in ((x.PREC_FP64, 1e-10), (x.PREC_SPLIT_BF16, SPLIT_TOL)):
        outs = x.x2c_build_dlu_batched(ctx, gs, lays, precision=prec)
        ctx.status()
        for mol, m, g, lay, hb in zip(mols, ms, gs, lays, outs):
            hs = x.x2c_build_dlu(ctx, g, *lay, precision=prec)
            ctx.status()
            assert (hb[0] - hs[0]).abs().max().item() <= 1e-13 * hs[0].abs().max().item()
            ref = O.x2c_dlu(m, mol.offsets, [kinds[b] for b in mol.basis])["h"]
            assert np.abs(hb[0].cpu().numpy() - ref).max() <= tol * np.abs(ref).max()


def test_split_variants_give_identical_h(ctx):
    """Every split-kernel variant (N tiles, transposed stage 1) gives bit-identical h, for
    both spins and for mixed atom sizes."""
    mol = w.Molecule(w.fcc_sites(5), np.full(5, 47.0), ["s30", "s48", "s30", "s48", "s48"])
    idx = [0, 1, 0, 1, 1]
    for two_c in (False, True):
        g = dev(w.molecule_inputs(mol, two_c))
        gk = [dev(w.atomic_inputs(47.0, b, two_c)) for b in ("s30", "s48")]
        hs = []
        for v in (0, 1, 2):
            ctx.set_split_variant(v)
            hs.append(x.x2c_build_dlu(ctx, g, mol.offsets, idx, gk, two_component=two_c,
                                      precision=x.PREC_SPLIT_BF16))
            ctx.status()
        ctx.set_split_variant(-1)
        for h in hs[1:]:
            for a, b in zip(hs[0], h):
                assert torch.equal(a, b)


def test_autotuner_choices_give_identical_h():
    """The tile autotuner times every candidate on the first build of a shape; all candidates
    must give bit-identical h (exact digit products), equal to a context without tuning."""
    mol = w.silver_cluster(6, "s48")
    for two_c in (False, True):
        g = dev(w.molecule_inputs(mol, two_c))
        gk = dev(w.atomic_inputs(47.0, "s48", two_c))
        tuned, plain = x.Context(0), x.Context(0)
        plain.set_autotune(False)
        h1 = x.x2c_build_dlu(tuned, g, mol.offsets, [0] * 6, [gk], two_component=two_c, precision=x.PREC_SPLIT_BF16)
        h2 = x.x2c_build_dlu(tuned, g, mol.offsets, [0] * 6, [gk], two_component=two_c, precision=x.PREC_SPLIT_BF16)
        h3 = x.x2c_build_dlu(plain, g, mol.offsets, [0] * 6, [gk], two_component=two_c, precision=x.PREC_SPLIT_BF16)
        tuned.status()
        plain.status()
        log = tuned.tuning_log()
        assert "split S=5" in log and "->" in log, log
        assert plain.tuning_log() == ""
        for a, b, c in zip(h1, h2, h3):
            assert torch.equal(a, b) and torch.equal(a, c)
        tuned.close()
        plain.close()
