"""Seeded synthetic workloads: cluster geometries, primitive s bases, integrals, SO blocks.

This module produces the *inputs* of the relativistic transformation (S, T, V, W of
Sec. II, Eqs. 4-6); it contains none of the decoupling arithmetic.  Both the CUDA
path (tests, bench) and the CPU oracle (tests) take their inputs from here.

Workload recipe (stands in for the paper's Ag_L clusters and rSV(P) bases, which are
not available; Sec. IV and Table VIII describe the originals):

* Sites: fcc lattice points (i, j, k) * a/2 with i + j + k even, a = 7.72 bohr, sorted
  by (i^2 + j^2 + k^2, i, j, k) ascending; the first L points form Ag_L.
* Nuclei: point charges Z = 47 (the paper uses point nuclei, Sec. IV).
* Basis: per atom an even-tempered set of uncontracted s Gaussians,
  "s30": alpha_k = 0.01 * 2^k (k = 0..29), "s48": alpha_k = 0.005 * 1.75^k (k = 0..47),
  ordered atom-major with ascending exponents.
* Spin-orbit parts Wx, Wy, Wz: real antisymmetric, non-zero on same-atom blocks only.
  g_k ~ N(0, 1) is drawn by numpy PCG64 from a seed (k = x, y, z in order, upper
  triangle i < j row-major, g_ji = -g_ij), and
      Wk = 0.02 * R (g_k / rho) R,   R = (-W0_free)^{1/2},
  where W0_free is the free-atom W0 (own nucleus only; eigenvalues of -W0_free below
  zero, which appear only at the rounding level, are clipped) and rho is the spectral
  norm of the 2c operator i sum_k sigma_k (x) g_k.  Then the atomic 2c W of Eq. 5 is
  -(I (x) R)(I - 0.02 i sum_k sigma_k (x) g_k / rho)(I (x) R), negative semi-definite
  like the physical sigma.p V sigma.p with an attractive V, so the positive/negative
  energy spectrum keeps its gap at -c^2.  (Scaling g by sqrt(|W0_ii W0_jj|) instead
  closes that gap: negative-energy states cross -c^2 and X2C is undefined.)  The blocks
  are drawn once per (element, basis, seed) and reused on every atom.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 137.035999  # default speed of light (a.u.)
C_LIGHT_PAPER = 137.0359895  # value used in the paper's calculations (Sec. IV)
FCC_A = 7.72  # bohr
SO_SCALE = 0.02
DEFAULT_SEED = 13034446

BASES = {
    "s30": (0.01, 2.0, 30),
    "s48": (0.005, 1.75, 48),
    # larger even-tempered set, used only to check convergence toward the Dirac limit
    "s64": (0.005, 1.6, 64),
}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO_PATH = os.path.join(_HERE, "_x2c_ints.so")
_lib = None


def build_ints_library(force: bool = False) -> str:
    """Compile the integral generator (plain C + OpenMP) in-tree and return its path."""
    src = os.path.join(_HERE, "ints.c")
    if force or not os.path.exists(_SO_PATH) or os.path.getmtime(_SO_PATH) < os.path.getmtime(src):
        tmp = _SO_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO_PATH)
    return _SO_PATH


def _ints():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_ints_library())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.x2c_ints_block.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        dp, dp, dp, dp, ctypes.c_int64]
        _lib.x2c_ints_full.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp,
                                       dp, dp, dp, dp]
        _lib.x2c_boys012.argtypes = [ctypes.c_double, dp]
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def boys012(T: float) -> np.ndarray:
    out = np.zeros(3)
    _ints().x2c_boys012(float(T), _ptr(out))
    return out


def basis_exponents(kind: str) -> np.ndarray:
    a0, beta, n = BASES[kind]
    return a0 * beta ** np.arange(n, dtype=np.float64)


def fcc_sites(L: int, a: float = FCC_A) -> np.ndarray:
    """First L fcc lattice points by distance from the origin, ties broken by (i, j, k)."""
    r = 1
    while True:
        rng = np.arange(-r, r + 1)
        i, j, k = np.meshgrid(rng, rng, rng, indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        keep = (i + j + k) % 2 == 0
        i, j, k = i[keep], j[keep], k[keep]
        d2 = i * i + j * j + k * k
        order = np.lexsort((k, j, i, d2))
        if L <= len(order) and d2[order[L - 1]] < r * r:  # all points with d2 < r^2 present
            sel = order[:L]
            return np.stack([i[sel], j[sel], k[sel]], axis=1).astype(np.float64) * (a / 2.0)
        r += 1


@dataclass
class Molecule:
    """Point-nucleus cluster with a primitive s basis per atom (atom-major ordering)."""
    coords: np.ndarray                # (L, 3) bohr
    Z: np.ndarray                     # (L,)
    basis: list                       # basis kind name per atom
    offsets: np.ndarray = field(init=False)   # (L + 1,) int32 first function of each atom
    bf_xyz: np.ndarray = field(init=False)
    bf_alpha: np.ndarray = field(init=False)

    def __post_init__(self):
        self.coords = np.ascontiguousarray(self.coords, dtype=np.float64)
        self.Z = np.ascontiguousarray(self.Z, dtype=np.float64)
        sizes = [BASES[b][2] for b in self.basis]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
        self.bf_alpha = np.concatenate([basis_exponents(b) for b in self.basis])
        self.bf_xyz = np.ascontiguousarray(
            np.repeat(self.coords, sizes, axis=0), dtype=np.float64)

    @property
    def natoms(self) -> int:
        return len(self.Z)

    @property
    def nbf(self) -> int:
        return int(self.offsets[-1])

    def kinds(self):
        """Distinct (Z, basis) kinds and the kind index of every atom."""
        keys = [(float(z), b) for z, b in zip(self.Z, self.basis)]
        uniq = sorted(set(keys), key=lambda t: (t[0], BASES[t[1]][2], t[1]))
        idx = np.array([uniq.index(k) for k in keys], dtype=np.int32)
        return uniq, idx


def silver_cluster(L: int, basis: str = "s48", Z: float = 47.0) -> Molecule:
    return Molecule(fcc_sites(L), np.full(L, Z), [basis] * L)


def integrals(mol: Molecule, nuclei: Molecule | None = None, want=("S", "T", "V", "W0")):
    """Full symmetric S, T, V, W0 (N x N, float64) of mol; nuclei default to mol's own."""
    nuc = mol if nuclei is None else nuclei
    n = mol.nbf
    out = {k: (np.empty((n, n)) if k in want else None) for k in ("S", "T", "V", "W0")}
    _ints().x2c_ints_full(nuc.natoms, _ptr(nuc.coords), _ptr(nuc.Z), n, _ptr(mol.bf_xyz),
                          _ptr(mol.bf_alpha), _ptr(out["S"]), _ptr(out["T"]), _ptr(out["V"]),
                          _ptr(out["W0"]))
    return {k: v for k, v in out.items() if v is not None}


def integrals_block(mol: Molecule, rows: slice, cols: slice, want=("S", "T", "V", "W0")):
    """Rectangular block [rows, cols] of S, T, V, W0 of mol (all nuclei of mol)."""
    i0, i1 = rows.start, rows.stop
    j0, j1 = cols.start, cols.stop
    shape = (i1 - i0, j1 - j0)
    out = {k: (np.empty(shape) if k in want else None) for k in ("S", "T", "V", "W0")}
    _ints().x2c_ints_block(mol.natoms, _ptr(mol.coords), _ptr(mol.Z), mol.nbf, _ptr(mol.bf_xyz),
                           _ptr(mol.bf_alpha), i0, i1, j0, j1, _ptr(out["S"]), _ptr(out["T"]),
                           _ptr(out["V"]), _ptr(out["W0"]), shape[1])
    return {k: v for k, v in out.items() if v is not None}


def integrals_points(bf_xyz, bf_alpha, nuc_xyz, nuc_Z, want=("S", "T", "V", "W0")):
    """S, T, V, W0 for primitives at arbitrary centres (bf_xyz: (n, 3)) and nuclei."""
    bf_xyz = np.ascontiguousarray(bf_xyz, dtype=np.float64)
    bf_alpha = np.ascontiguousarray(bf_alpha, dtype=np.float64)
    nuc_xyz = np.ascontiguousarray(nuc_xyz, dtype=np.float64)
    nuc_Z = np.ascontiguousarray(nuc_Z, dtype=np.float64)
    n = len(bf_alpha)
    out = {k: (np.empty((n, n)) if k in want else None) for k in ("S", "T", "V", "W0")}
    _ints().x2c_ints_block(len(nuc_Z), _ptr(nuc_xyz), _ptr(nuc_Z), n, _ptr(bf_xyz),
                           _ptr(bf_alpha), 0, n, 0, n, _ptr(out["S"]), _ptr(out["T"]),
                           _ptr(out["V"]), _ptr(out["W0"]), n)
    return {k: v for k, v in out.items() if v is not None}


def free_atom(Z: float, basis: str) -> Molecule:
    return Molecule(np.zeros((1, 3)), np.array([Z]), [basis])


def free_atom_integrals(Z: float, basis: str):
    return integrals(free_atom(Z, basis))


def so_blocks(Z: float, basis: str, seed: int = DEFAULT_SEED, strength: float = SO_SCALE):
    """Synthetic same-atom spin-orbit blocks (Wx, Wy, Wz), real antisymmetric n x n
    (construction in the module docstring)."""
    w0 = free_atom_integrals(Z, basis)["W0"]
    ev, C = np.linalg.eigh(-w0)
    R = (C * np.sqrt(np.clip(ev, 0.0, None))) @ C.T
    R = 0.5 * (R + R.T)
    n = len(w0)
    rng = np.random.Generator(np.random.PCG64(seed))
    iu = np.triu_indices(n, 1)
    g = []
    for _ in range(3):
        x = np.zeros((n, n))
        x[iu] = rng.standard_normal(len(iu[0]))
        g.append(x - x.T)
    pauli = (np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
             np.array([[1, 0], [0, -1]], dtype=complex))
    G = 1j * sum(np.kron(p, x) for p, x in zip(pauli, g))
    rho = np.abs(np.linalg.eigvalsh(G)).max()
    out = []
    for x in g:
        wk = strength * (R @ (x / rho) @ R)
        out.append(0.5 * (wk - wk.T))
    return tuple(out)


def so_blocks_configured(Z: float, basis: str, seed: int = DEFAULT_SEED, strength: float = SO_SCALE):
    """The configured spin-orbit recipe taken literally, Wk_ij = strength g_ij sqrt(|W0_ii W0_jj|)
    with the same seeded g as so_blocks (free-atom W0).  Not used by any workload: it is
    kept so that a test can show why it was replaced (with it the atomic 4c spectrum no longer
    splits at -c^2, so X2C is undefined for it)."""
    w0 = free_atom_integrals(Z, basis)["W0"]
    n = len(w0)
    rng = np.random.Generator(np.random.PCG64(seed))
    iu = np.triu_indices(n, 1)
    d = np.sqrt(np.abs(np.diag(w0)))
    out = []
    for _ in range(3):
        x = np.zeros((n, n))
        x[iu] = rng.standard_normal(len(iu[0]))
        out.append(strength * (x - x.T) * np.outer(d, d))
    return tuple(out)


def molecular_so(mol: Molecule, seed: int = DEFAULT_SEED):
    """Molecular Wx, Wy, Wz (N x N) holding the synthetic blocks on same-atom blocks."""
    n = mol.nbf
    W = [np.zeros((n, n)) for _ in range(3)]
    cache = {}
    for a in range(mol.natoms):
        key = (float(mol.Z[a]), mol.basis[a])
        if key not in cache:
            cache[key] = so_blocks(key[0], key[1], seed)
        o0, o1 = mol.offsets[a], mol.offsets[a + 1]
        for k in range(3):
            W[k][o0:o1, o0:o1] = cache[key][k]
    return tuple(W)


def molecule_inputs(mol: Molecule, two_component: bool, seed: int = DEFAULT_SEED):
    """dict with S, T, V, W0 (and Wx, Wy, Wz when two_component) for the whole molecule."""
    m = integrals(mol)
    if two_component:
        m["Wx"], m["Wy"], m["Wz"] = molecular_so(mol, seed)
    return m


def atomic_inputs(Z: float, basis: str, two_component: bool, seed: int = DEFAULT_SEED):
    """Free-atom S, T, V, W0 (own nucleus only) plus the synthetic SO blocks."""
    m = free_atom_integrals(Z, basis)
    if two_component:
        m["Wx"], m["Wy"], m["Wz"] = so_blocks(Z, basis, seed)
    return m


def random_cluster_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Cluster sizes drawn uniformly from [lo, hi] (inclusive) by a seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=count)


def batched_molecules(count: int = 64, lo: int = 2, hi: int = 43, seed: int = DEFAULT_SEED):
    """Uneven Ag_n clusters, n uniform in [lo, hi], basis s30 or s48 with equal odds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = rng.integers(lo, hi + 1, size=count)
    kinds = rng.integers(0, 2, size=count)
    return [silver_cluster(int(n), "s30" if k == 0 else "s48") for n, k in zip(sizes, kinds)]


def serving_requests(count: int = 2000, rate: float = 50.0, lo: int = 2, hi: int = 147,
                     frac_2c: float = 0.3, seed: int = DEFAULT_SEED):
    """Open-loop request stream: Poisson arrivals, n log-uniform in [lo, hi], s30/s48 with
    equal odds, two-component with probability frac_2c.  Returns a list of dicts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    n = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=count))).astype(int)
    n = np.clip(n, lo, hi)
    basis = rng.integers(0, 2, size=count)
    twoc = rng.uniform(size=count) < frac_2c
    return [dict(t_arrive=float(t[i]), natoms=int(n[i]), basis="s30" if basis[i] == 0 else "s48",
                 two_component=bool(twoc[i])) for i in range(count)]
