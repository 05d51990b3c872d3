"""The Coulomb- and exchange-digestion rules of the plans, checked on the
CPU with the oracle's integrals.  Over the unique quartets only, with
s = 1/2 for each of a == b, c == d and (ab) == (cd):
  J'_ab += 2s (ab|cd) D_cd,  J'_cd += 2s (ab|cd) D_ab,
  K'_ac += s (ab|cd) D_bd,  K'_bc += s (ab|cd) D_ad,
  K'_ad += s (ab|cd) D_bc,  K'_bd += s (ab|cd) D_ac,
then J = J' + J'^T and K = K' + K'^T give J_uv = sum_ls (uv|ls) D_ls and
K_ul = sum_vs (uv|ls) D_vs over all ordered quartets, the plain
definitions (the readings the GPU digestion implements)."""
import numpy as np

import oracle
import synth


def test_unique_quartet_expansion_rules():
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
    kref = np.zeros((nbf, nbf))
    for a, b, c, d, blk in blocks(allq):
        ref[sl(a), sl(b)] += np.einsum("abcd,cd->ab", blk, D[sl(c), sl(d)])
        kref[sl(a), sl(c)] += np.einsum("abcd,bd->ac", blk, D[sl(b), sl(d)])

    pairs = synth.unique_pairs(basis)
    P, Q = np.tril_indices(len(pairs))
    uq = np.concatenate([pairs[P], pairs[Q]], axis=1).astype(np.int32)
    Jp = np.zeros((nbf, nbf))
    Kp = np.zeros((nbf, nbf))
    for a, b, c, d, blk in blocks(uq):
        s_ = (0.5 if a == b else 1.0) * (0.5 if c == d else 1.0) * (0.5 if {a, b} == {c, d} else 1.0)
        Jp[sl(a), sl(b)] += 2 * s_ * np.einsum("abcd,cd->ab", blk, D[sl(c), sl(d)])
        Jp[sl(c), sl(d)] += 2 * s_ * np.einsum("abcd,ab->cd", blk, D[sl(a), sl(b)])
        Kp[sl(a), sl(c)] += s_ * np.einsum("abcd,bd->ac", blk, D[sl(b), sl(d)])
        Kp[sl(b), sl(c)] += s_ * np.einsum("abcd,ad->bc", blk, D[sl(a), sl(d)])
        Kp[sl(a), sl(d)] += s_ * np.einsum("abcd,bc->ad", blk, D[sl(b), sl(c)])
        Kp[sl(b), sl(d)] += s_ * np.einsum("abcd,ac->bd", blk, D[sl(a), sl(c)])
    J = Jp + Jp.T
    K = Kp + Kp.T
    assert np.abs(ref - ref.T).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(J - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(kref - kref.T).max() <= 1e-12 * np.abs(kref).max()
    assert np.abs(K - kref).max() <= 1e-12 * np.abs(kref).max()
    # K differs from J (the contraction pattern matters)
    assert np.abs(K - J).max() > 1e-3 * np.abs(J).max()
    # a dropped degeneracy factor breaks it
    bad = Jp.copy()
    a, b = pairs[0]
    bad[sl(a), sl(b)] *= 2.0
    assert np.abs(bad + bad.T - ref).max() > 1e-6 * np.abs(ref).max()
