"""The Coulomb-digestion rule of the plans, checked on the CPU with the
oracle's integrals: summing 2s (ab|cd) D_cd into J'_ab and 2s (ab|cd) D_ab
into J'_cd over the unique quartets only (s = 1/2 for each of a == b,
c == d and (ab) == (cd)), then J = J' + J'^T, gives J_uv = sum over all
ordered (ls) of (uv|ls) D_ls, the plain definition (the reading the GPU
digestion implements)."""
import numpy as np

import oracle
import synth


def test_unique_quartet_expansion_rule():
    basis = synth.molecule_basis(natom=2, radius=1.6, seed=21)
    n = (basis.shell_l + 1) * (basis.shell_l + 2) // 2
    off = np.concatenate([[0], np.cumsum(n)[:-1]])
    nbf = int(n.sum())
    rng = np.random.default_rng(22)
    U = rng.uniform(-1, 1, (nbf, nbf))
    D = np.triu(U) + np.triu(U, 1).T
    ns = basis.nshell
    threads = 8

    def blocks(quartets):
        vals = oracle.eri_quartets(basis, quartets, prec="d", threads=threads)
        pos = np.concatenate([[0], np.cumsum(oracle.shellset_size(basis, quartets))])
        for i, (a, b, c, d) in enumerate(quartets):
            yield a, b, c, d, vals[pos[i]:pos[i + 1]].reshape(n[a], n[b], n[c], n[d])

    def sl(s):
        return slice(off[s], off[s] + n[s])

    allq = np.stack(np.meshgrid(*(np.arange(ns),) * 4, indexing="ij"), -1).reshape(-1, 4).astype(np.int32)
    ref = np.zeros((nbf, nbf))
    for a, b, c, d, blk in blocks(allq):
        ref[sl(a), sl(b)] += np.einsum("abcd,cd->ab", blk, D[sl(c), sl(d)])

    pairs = synth.unique_pairs(basis)
    P, Q = np.tril_indices(len(pairs))
    uq = np.concatenate([pairs[P], pairs[Q]], axis=1).astype(np.int32)
    Jp = np.zeros((nbf, nbf))
    for a, b, c, d, blk in blocks(uq):
        w = 2.0 * (0.5 if a == b else 1.0) * (0.5 if c == d else 1.0) * (0.5 if {a, b} == {c, d} else 1.0)
        Jp[sl(a), sl(b)] += w * np.einsum("abcd,cd->ab", blk, D[sl(c), sl(d)])
        Jp[sl(c), sl(d)] += w * np.einsum("abcd,ab->cd", blk, D[sl(a), sl(b)])
    J = Jp + Jp.T
    assert np.abs(ref - ref.T).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(J - ref).max() <= 1e-12 * np.abs(ref).max()
    # a dropped degeneracy factor breaks it
    bad = Jp.copy()
    a, b = pairs[0]
    bad[sl(a), sl(b)] *= 2.0
    assert np.abs(bad + bad.T - ref).max() > 1e-6 * np.abs(ref).max()
