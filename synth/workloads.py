"""Seeded synthetic workloads for the 4-centre ERI batches.

The paper benchmarks on random Gaussians that mimic typical basis-set values
(Section 4, methodology paragraph); there is no public dataset.  Every
generator here draws from ``numpy.random.default_rng(seed)`` so that the
oracle side and the CUDA side see bit-identical inputs.

A *basis* is a dict of numpy arrays in the layout of the C ABI:
  centres (natom,3) f64 bohr, shell_atom/shell_l/shell_K/shell_off (nshell,) i32,
  exps/coefs (nprim,) f64.
A *batch* of one class is (bra_pairs (nbra,2) i32, ket_pairs (nket,2) i32,
quartets (nq,2) i64 of (bra index, ket index)).

Contraction coefficients are seeded weights times the usual normalisation
factor of an x^l-type primitive, N(z,l) = (2z/pi)^(3/4) (4z)^(l/2) / sqrt((2l-1)!!),
so that integral magnitudes are O(1-10); the library uses them verbatim.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "norm_coef", "Basis", "basis_from_shells", "quartet_shells", "class_of",
    "config1_pp_primitive", "class_sweep_pools", "class_sweep_batch", "all_classes",
    "molecule_geometry", "molecule_basis", "adjoint_workload", "split_batch",
    "small_random_batch", "unique_pairs", "class_batches", "all_unique_quartets", "density_weights",
    "three_centre_pools", "three_centre_batch",
]


def _dfact(n: int) -> int:
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def norm_coef(zeta, l: int):
    """Normalisation of the primitive x^l exp(-zeta r^2) (axis independent form)."""
    zeta = np.asarray(zeta, dtype=np.float64)
    return (2.0 * zeta / math.pi) ** 0.75 * (4.0 * zeta) ** (0.5 * l) / math.sqrt(_dfact(2 * l - 1))


@dataclass
class Basis:
    centres: np.ndarray
    shell_atom: np.ndarray
    shell_l: np.ndarray
    shell_K: np.ndarray
    shell_off: np.ndarray
    exps: np.ndarray
    coefs: np.ndarray

    def __getitem__(self, k):
        return getattr(self, k)

    @property
    def natom(self):
        return self.centres.shape[0]

    @property
    def nshell(self):
        return self.shell_l.shape[0]

    @property
    def nprim(self):
        return self.exps.shape[0]

    def copy(self):
        return Basis(*(np.array(getattr(self, f)) for f in
                       ("centres", "shell_atom", "shell_l", "shell_K", "shell_off", "exps", "coefs")))


def basis_from_shells(centres, shells):
    """``shells``: list of (atom, l, exps(list), coefs(list))."""
    atom, ls, Ks, offs, ex, co = [], [], [], [], [], []
    off = 0
    for a, l, e, c in shells:
        atom.append(a); ls.append(l); Ks.append(len(e)); offs.append(off)
        ex.extend(e); co.extend(c); off += len(e)
    return Basis(np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1, 3)),
                 np.asarray(atom, np.int32), np.asarray(ls, np.int32), np.asarray(Ks, np.int32),
                 np.asarray(offs, np.int32), np.asarray(ex, np.float64), np.asarray(co, np.float64))


def quartet_shells(bra_pairs, ket_pairs, quartets):
    """(nq,4) shell indices of a list-form batch (input plumbing for the oracle)."""
    q = np.asarray(quartets, dtype=np.int64).reshape(-1, 2)
    return np.ascontiguousarray(np.concatenate([np.asarray(bra_pairs)[q[:, 0]],
                                                np.asarray(ket_pairs)[q[:, 1]]], axis=1).astype(np.int32))


def class_of(basis, bra_pair, ket_pair):
    l = basis.shell_l
    return (int(l[bra_pair[0]]), int(l[bra_pair[1]]), int(l[ket_pair[0]]), int(l[ket_pair[1]]))


def all_classes(lmax: int = 2):
    return [(a, b, c, d) for a in range(lmax + 1) for b in range(lmax + 1)
            for c in range(lmax + 1) for d in range(lmax + 1)]


# --------------------------------------------------------------------------
# Plain FP64 primitive (pp|pp): 1000 quartets of 4 fresh p shells, K = 1,
# exponents log-uniform in [0.1, 10], centres uniform in a 10-bohr cube.
# --------------------------------------------------------------------------
def config1_pp_primitive(seed: int = 0, nq: int = 1000):
    rng = np.random.default_rng(seed)
    ns = 4 * nq
    centres = rng.uniform(0.0, 10.0, size=(ns, 3))
    exps = 10.0 ** rng.uniform(-1.0, 1.0, size=ns)
    coefs = norm_coef(exps, 1)
    basis = Basis(centres, np.arange(ns, dtype=np.int32), np.ones(ns, np.int32), np.ones(ns, np.int32),
                  np.arange(ns, dtype=np.int32), exps, coefs)
    idx = np.arange(nq, dtype=np.int32)
    bra = np.stack([4 * idx, 4 * idx + 1], axis=1).astype(np.int32)
    ket = np.stack([4 * idx + 2, 4 * idx + 3], axis=1).astype(np.int32)
    quartets = np.stack([idx, idx], axis=1).astype(np.int64)
    return basis, bra, ket, quartets


# --------------------------------------------------------------------------
# Class sweep: pools of shells per l, K per shell, even-tempered exponents
# 0.2*3^k, weights U[0.5,1] x N, centres uniform in a 12-bohr cube; each
# class draws its quartets from random bra/ket pair lists.
# --------------------------------------------------------------------------
def class_sweep_pools(seed: int = 0, lmax: int = 2, pool: int = 512, K: int = 3, cube: float = 12.0,
                      exps_fn=None):
    """One basis holding ``pool`` shells of each l in 0..lmax, each on its own centre.
    ``exps_fn(rng, K)`` draws the exponents of one shell (default even-tempered 0.2*3^k)."""
    rng = np.random.default_rng(seed)
    nl = lmax + 1
    ns = nl * pool
    centres = rng.uniform(0.0, cube, size=(ns, 3))
    shells = []
    for l in range(nl):
        for i in range(pool):
            e = (np.array([0.2 * 3.0 ** k for k in range(K)]) if exps_fn is None else np.asarray(exps_fn(rng, K)))
            w = rng.uniform(0.5, 1.0, size=K)
            shells.append((l * pool + i, l, list(e), list(w * norm_coef(e, l))))
    basis = basis_from_shells(centres, shells)
    pools = {l: np.arange(l * pool, (l + 1) * pool, dtype=np.int32) for l in range(nl)}
    return basis, pools


def class_sweep_batch(pools, cls, seed: int = 0, npairs: int = 2048, nq: int = 100_000):
    """List-form batch of class ``cls`` = (la,lb,lc,ld) drawn from the pools."""
    la, lb, lc, ld = cls
    rng = np.random.default_rng([seed, la, lb, lc, ld])
    bra = np.stack([rng.choice(pools[la], npairs), rng.choice(pools[lb], npairs)], axis=1).astype(np.int32)
    ket = np.stack([rng.choice(pools[lc], npairs), rng.choice(pools[ld], npairs)], axis=1).astype(np.int32)
    quartets = np.stack([rng.integers(0, npairs, nq), rng.integers(0, npairs, nq)], axis=1).astype(np.int64)
    return bra, ket, quartets


def three_centre_pools(seed: int = 0, lxmax: int = 3, lmax: int = 2, pool: int = 512, K: int = 3,
                       cube: float = 12.0):
    """The 3-centre workload: the class-sweep pools of orbital shells (l <= lmax,
    K even-tempered primitives) plus, per l <= lxmax, ``pool`` uncontracted
    auxiliary shells (K = 1, exponent log-uniform in [0.1, 10], as in
    density-fitting bases), all on their own centres in a ``cube``-bohr box.
    Returns (basis, orbital pools {l: shells}, auxiliary pools {l: shells})."""
    rng = np.random.default_rng([seed, 3])
    nob = (lmax + 1) * pool
    nax = (lxmax + 1) * pool
    centres = rng.uniform(0.0, cube, size=(nob + nax, 3))
    shells = []
    for l in range(lmax + 1):
        for i in range(pool):
            e = np.array([0.2 * 3.0 ** k for k in range(K)])
            w = rng.uniform(0.5, 1.0, size=K)
            shells.append((l * pool + i, l, list(e), list(w * norm_coef(e, l))))
    for l in range(lxmax + 1):
        for i in range(pool):
            e = 10.0 ** rng.uniform(-1.0, 1.0, size=1)
            shells.append((nob + l * pool + i, l, list(e), list(norm_coef(e, l))))
    basis = basis_from_shells(centres, shells)
    orb = {l: np.arange(l * pool, (l + 1) * pool, dtype=np.int32) for l in range(lmax + 1)}
    aux = {l: np.arange(nob + l * pool, nob + (l + 1) * pool, dtype=np.int32) for l in range(lxmax + 1)}
    return basis, orb, aux


def three_centre_batch(orb, aux, cls3, seed: int = 0, nx: int = 2048, npairs: int = 2048, nt: int = 100_000):
    """List-form 3-centre batch of class ``cls3`` = (lx, lc, ld): x shells,
    ket pairs and (x index, ket index) triples drawn from the pools."""
    lx, lc, ld = cls3
    rng = np.random.default_rng([seed, 7, lx, lc, ld])
    x = rng.choice(aux[lx], nx).astype(np.int32)
    ket = np.stack([rng.choice(orb[lc], npairs), rng.choice(orb[ld], npairs)], axis=1).astype(np.int32)
    t = np.stack([rng.integers(0, nx, nt), rng.integers(0, npairs, nt)], axis=1).astype(np.int64)
    return x, ket, t


def split_batch(cls, K: int, seed: int = 0, nq: int = 100_000, pool: int = 512, npairs: int = 2048):
    """High angular momentum workload: exponents log-uniform in [0.05, 50], centres in a
    12-bohr cube, K primitives per shell; returns (basis, bra, ket, quartets)."""
    lmax = max(cls)

    def exps_fn(rng, K):
        return 10.0 ** rng.uniform(math.log10(0.05), math.log10(50.0), size=K)

    basis, pools = class_sweep_pools(seed=seed, lmax=lmax, pool=pool, K=K, exps_fn=exps_fn)
    bra, ket, q = class_sweep_batch(pools, cls, seed=seed, npairs=npairs, nq=nq)
    return basis, bra, ket, q


def small_random_batch(cls, K=(1, 1, 1, 1), nq: int = 8, seed: int = 0, cube: float = 3.0, zrange=(0.1, 10.0)):
    """Tiny list-form batch of one class with fresh shells per quartet (tests)."""
    rng = np.random.default_rng([seed, *cls, *K])
    shells, centres = [], []
    for q in range(nq):
        for s in range(4):
            centres.append(rng.uniform(0.0, cube, size=3))
            e = 10.0 ** rng.uniform(math.log10(zrange[0]), math.log10(zrange[1]), size=K[s])
            w = rng.uniform(0.5, 1.0, size=K[s])
            shells.append((len(centres) - 1, cls[s], list(e), list(w * norm_coef(e, cls[s]))))
    basis = basis_from_shells(np.array(centres), shells)
    idx = np.arange(nq, dtype=np.int32)
    bra = np.stack([4 * idx, 4 * idx + 1], axis=1).astype(np.int32)
    ket = np.stack([4 * idx + 2, 4 * idx + 3], axis=1).astype(np.int32)
    return basis, bra, ket, np.stack([idx, idx], axis=1).astype(np.int64)


# --------------------------------------------------------------------------
# Molecule-shaped workloads
# --------------------------------------------------------------------------
def molecule_geometry(natom: int, radius: float, min_sep: float = 1.8, seed: int = 0):
    """Rejection-sample ``natom`` points in a sphere with a minimum separation."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < natom:
        p = rng.uniform(-radius, radius, size=3)
        if p @ p > radius * radius:
            continue
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts)


# per atom: (l, K) -- s x3 (K=6,3,1), p x2 (K=3,1), d x1 (K=1)
MOLECULE_SHELLS = [(0, 6), (0, 3), (0, 1), (1, 3), (1, 1), (2, 1)]


def molecule_basis(natom: int = 64, radius: float = 7.0, seed: int = 0):
    geom = molecule_geometry(natom, radius, seed=seed)
    rng = np.random.default_rng([seed, 1])
    shells = []
    for a in range(natom):
        for l, K in MOLECULE_SHELLS:
            e = np.array([0.2 * 3.0 ** k for k in range(K)])
            w = rng.uniform(0.5, 1.0, size=K)
            shells.append((a, l, list(e), list(w * norm_coef(e, l))))
    return basis_from_shells(geom, shells)


def adjoint_workload(natom: int = 16, radius: float = 4.4, seed: int = 0):
    """Basis of the molecule rule on ``natom`` atoms plus a symmetric density-like
    matrix D (nbf x nbf, upper triangle U[-1,1], mirrored) over Cartesian functions.
    Returns (basis, D, bf_offset per shell)."""
    basis = molecule_basis(natom, radius, seed=seed)
    nc = (basis.shell_l + 1) * (basis.shell_l + 2) // 2
    bf_off = np.concatenate([[0], np.cumsum(nc)[:-1]]).astype(np.int64)
    nbf = int(nc.sum())
    rng = np.random.default_rng([seed, 2])
    U = rng.uniform(-1.0, 1.0, size=(nbf, nbf))
    D = np.triu(U) + np.triu(U, 1).T
    return basis, D, bf_off


# --------------------------------------------------------------------------
# Unique shell quartets of a basis, grouped by class (index plumbing only)
# --------------------------------------------------------------------------
def unique_pairs(basis):
    """All shell pairs (i, j), i >= j, each ordered so that l_first >= l_second."""
    ns = basis.nshell
    i, j = np.tril_indices(ns)
    li, lj = basis.shell_l[i], basis.shell_l[j]
    swap = li < lj
    a = np.where(swap, j, i)
    b = np.where(swap, i, j)
    return np.stack([a, b], axis=1).astype(np.int32)


def class_batches(basis, pairs, quartet_pairs):
    """Group quartets of pair indices (P, Q) by class (l of the four shells).
    Returns {cls: (bra_pairs, ket_pairs, quartets)} with per-class compact
    pair lists and (bra index, ket index) quartets."""
    l = basis.shell_l
    P, Q = quartet_pairs[:, 0], quartet_pairs[:, 1]
    cls_arr = np.stack([l[pairs[P, 0]], l[pairs[P, 1]], l[pairs[Q, 0]], l[pairs[Q, 1]]], axis=1)
    key = ((cls_arr[:, 0] * 8 + cls_arr[:, 1]) * 8 + cls_arr[:, 2]) * 8 + cls_arr[:, 3]
    out = {}
    for k in np.unique(key):
        sel = np.where(key == k)[0]
        cls = tuple(int(x) for x in cls_arr[sel[0]])
        bra_u, bra_inv = np.unique(P[sel], return_inverse=True)
        ket_u, ket_inv = np.unique(Q[sel], return_inverse=True)
        out[cls] = (np.ascontiguousarray(pairs[bra_u]), np.ascontiguousarray(pairs[ket_u]),
                    np.stack([bra_inv, ket_inv], axis=1).astype(np.int64))
    return out


def all_unique_quartets(basis):
    """Every unique quartet (pair P >= pair Q) of the basis, by class."""
    pairs = unique_pairs(basis)
    n = pairs.shape[0]
    P, Q = np.tril_indices(n)
    return pairs, class_batches(basis, pairs, np.stack([P, Q], axis=1))


def density_weights(cls, bra, ket, quartets, D, bf_off):
    """W_abcd = D_ab D_cd over the Cartesian functions of each quartet, in the
    list-form output layout W[q + nq*(ab*ncd + cd)]."""
    la, lb, lc, ld = cls
    nca, ncb, ncc, ncd_ = ((l + 1) * (l + 2) // 2 for l in cls)
    q = np.asarray(quartets)
    A = bf_off[bra[q[:, 0], 0]][:, None] + np.arange(nca)[None, :]
    B = bf_off[bra[q[:, 0], 1]][:, None] + np.arange(ncb)[None, :]
    C = bf_off[ket[q[:, 1], 0]][:, None] + np.arange(ncc)[None, :]
    Dd = bf_off[ket[q[:, 1], 1]][:, None] + np.arange(ncd_)[None, :]
    Dab = D[A[:, :, None], B[:, None, :]].reshape(len(q), -1)   # [q][ab]
    Dcd = D[C[:, :, None], Dd[:, None, :]].reshape(len(q), -1)  # [q][cd]
    W = Dab[:, :, None] * Dcd[:, None, :]                       # [q][ab][cd]
    return np.ascontiguousarray(W.reshape(len(q), -1).T).reshape(-1)
