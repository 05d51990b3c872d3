"""The batched form (eri_plan_*): Schwarz-screened unique quartets of a
molecule-shaped basis, all classes in one persistent graph-replayed kernel,
digested into sum D_ab D_cd (ab|cd) or stored; checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import THREADS, assert_close

pytestmark = pytest.mark.gpu


def nc(l):
    return (l + 1) * (l + 2) // 2


def bf_offsets(basis):
    ncs = (basis.shell_l + 1) * (basis.shell_l + 2) // 2
    return np.concatenate([[0], np.cumsum(ncs)[:-1]]).astype(np.int64), int(ncs.sum())


def weights(basis, shells, D):
    """W[q][ab][cd] = D_ab D_cd for quartets of shell indices (a, b, c, d)."""
    off, _ = bf_offsets(basis)
    l = basis.shell_l
    out = []
    for a, b, c, d in shells:
        ia = off[a] + np.arange(nc(l[a]))
        ib = off[b] + np.arange(nc(l[b]))
        ic = off[c] + np.arange(nc(l[c]))
        id_ = off[d] + np.arange(nc(l[d]))
        out.append(np.einsum("ab,cd->abcd", D[np.ix_(ia, ib)], D[np.ix_(ic, id_)]).ravel())
    return np.concatenate(out)


@pytest.fixture(scope="module")
def tiny():
    basis = synth.molecule_basis(natom=3, radius=2.2, seed=5)
    _, nbf = bf_offsets(basis)
    rng = np.random.default_rng(6)
    U = rng.uniform(-1, 1, (nbf, nbf))
    D = np.triu(U) + np.triu(U, 1).T
    return basis, D


def test_plan_store_matches_oracle(cuda, tiny):
    basis, D = tiny
    db = eri.DeviceBasis(basis)
    plan = eri.Plan(db, threshold=0.0, flags=eri.ERI_PLAN_STORE)
    info = plan.info()
    ns = basis.nshell
    npairs = ns * (ns + 1) // 2
    assert info["nquartets"] == npairs * (npairs + 1) // 2   # every unique quartet, once
    out = torch.full((info["out_len"],), float("nan"), dtype=torch.float64, device=cuda)
    plan.execute(out=out)
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    seen = set()
    for j in range(info["njobs"]):
        cls, nq, off, shells = plan.job(j, with_quartets=True)
        kb, kk = plan.job_degrees(j)
        a0, b0, c0, d0 = shells[0]
        assert (kb, kk) == (basis.shell_K[a0] * basis.shell_K[b0], basis.shell_K[c0] * basis.shell_K[d0])
        nab, ncd = nc(cls[0]) * nc(cls[1]), nc(cls[2]) * nc(cls[3])
        got = host[off:off + nq * nab * ncd].reshape(nab * ncd, nq).T
        ref = oracle.eri_quartets(basis, shells, prec="d", threads=THREADS).reshape(nq, nab * ncd)
        assert_close(got, ref, what=f"plan job {j} {cls}")
        for a, b, c, d in shells:
            key = (min(a, b), max(a, b), min(c, d), max(c, d))
            key = min(key, key[2:] + key[:2])
            assert key not in seen
            seen.add(key)
    assert len(seen) == info["nquartets"]


def test_plan_energy_digest_against_oracle(cuda, tiny):
    basis, D = tiny
    db = eri.DeviceBasis(basis)
    plan = eri.Plan(db, threshold=0.0)
    Dd = torch.as_tensor(D, device=cuda)
    e = torch.zeros(1, dtype=torch.float64, device=cuda)
    plan.execute(D=Dd, energy=e)
    assert plan.status() == eri.ERI_OK
    got = float(e.item())
    store = eri.Plan(db, threshold=0.0, flags=eri.ERI_PLAN_STORE)
    ref = 0.0
    for j in range(store.info()["njobs"]):
        cls, nq, off, shells = store.job(j, with_quartets=True)
        vals = oracle.eri_quartets(basis, shells, prec="d", threads=THREADS)
        ref += float(np.dot(vals, weights(basis, shells, D)))
    assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (got, ref)
    # graph replay gives the same number; the parameters (D) are re-read
    plan.execute(D=Dd, energy=e)
    assert float(e.item()) == pytest.approx(got, rel=1e-13, abs=0)
    plan.execute(D=2.0 * Dd, energy=e)
    assert float(e.item()) == pytest.approx(4.0 * got, rel=1e-12)


def test_plan_schwarz_screening(cuda):
    """The screened plan keeps exactly the quartets with Q_P Q_Q >= threshold,
    Q from the oracle's diagonal integrals, and its energy differs from the
    unscreened one by no more than the bound the dropped quartets allow."""
    basis = synth.molecule_basis(natom=6, radius=9.0, seed=11)
    db = eri.DeviceBasis(basis)
    thr = 1e-8
    plan = eri.Plan(db, threshold=thr)
    full = eri.Plan(db, threshold=0.0)
    pairs = synth.unique_pairs(basis)
    diag = oracle.eri_quartets(basis, np.concatenate([pairs, pairs], axis=1), prec="d", threads=THREADS)
    sizes = oracle.shellset_size(basis, np.concatenate([pairs, pairs], axis=1))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    Q = np.empty(len(pairs))
    for i, (a, b) in enumerate(pairs):
        nab = nc(basis.shell_l[a]) * nc(basis.shell_l[b])
        blk = diag[offs[i]:offs[i + 1]].reshape(nab, nab)
        Q[i] = np.sqrt(np.max(np.abs(np.diag(blk))))
    prod = np.multiply.outer(Q, Q)[np.tril_indices(len(Q))]
    border = np.abs(prod - thr) <= 1e-9 * thr
    kept = int(np.sum(prod >= thr))
    assert abs(plan.info()["nquartets"] - kept) <= int(border.sum())
    assert plan.info()["nquartets"] < full.info()["nquartets"]
    _, nbf = bf_offsets(basis)
    D = torch.as_tensor(np.random.default_rng(3).uniform(-1, 1, (nbf, nbf)), device=cuda)
    D = 0.5 * (D + D.T)
    e1 = torch.zeros(1, dtype=torch.float64, device=cuda)
    e2 = torch.zeros(1, dtype=torch.float64, device=cuda)
    plan.execute(D=D, energy=e1)
    full.execute(D=D, energy=e2)
    dropped = full.info()["nquartets"] - plan.info()["nquartets"]
    # |(ab|cd)| <= Q_P Q_Q < thr for every dropped element; |W| <= 1; at most 6^4 elements each
    assert abs(float(e1.item()) - float(e2.item())) <= dropped * thr * 6 ** 4


def test_plan_split_precision(cuda, tiny):
    basis, D = tiny
    db = eri.DeviceBasis(basis)
    Dd = torch.as_tensor(D, device=cuda)
    e64 = torch.zeros(1, dtype=torch.float64, device=cuda)
    esp = torch.zeros(1, dtype=torch.float64, device=cuda)
    eri.Plan(db, threshold=1e-12).execute(D=Dd, energy=e64)
    eri.Plan(db, threshold=1e-12, flags=eri.ERI_PLAN_SPLIT).execute(D=Dd, energy=esp)
    assert abs(float(esp.item()) - float(e64.item())) <= 1e-10 * max(1.0, abs(float(e64.item())))


def test_plan_budget_timeout_and_recovery(cuda, tiny):
    """A cycle budget bounds the persistent kernel: an exhausted budget is
    reported as ERI_ETIMEOUT (no fault, no hang) and the plan stays usable."""
    basis, D = tiny
    db = eri.DeviceBasis(basis)
    Dd = torch.as_tensor(D, device=cuda)
    plan = eri.Plan(db, threshold=0.0)
    e = torch.zeros(1, dtype=torch.float64, device=cuda)
    plan.execute(D=Dd, energy=e)
    ref = float(e.item())
    plan.set_budget(1)
    plan.execute(D=Dd, energy=e)
    assert plan.status() == eri.ERI_ETIMEOUT
    plan.set_budget(0)
    plan.execute(D=Dd, energy=e)
    assert plan.status() == eri.ERI_OK
    assert float(e.item()) == pytest.approx(ref, rel=1e-13)


def test_plan_misuse(cuda, tiny):
    basis, D = tiny
    db = eri.DeviceBasis(basis)
    plan = eri.Plan(db, threshold=0.0)
    e = torch.zeros(1, dtype=torch.float64, device=cuda)
    with pytest.raises(eri.EriError) as ex:
        plan.execute(D=torch.zeros((3, 3), dtype=torch.float64, device=cuda), energy=e)
    assert ex.value.code == eri.ERI_EPLAN
    store = eri.Plan(db, threshold=0.0, flags=eri.ERI_PLAN_STORE)
    with pytest.raises(eri.EriError) as ex:
        store.execute(out=torch.zeros(10, dtype=torch.float64, device=cuda))
    assert ex.value.code == eri.ERI_EPLAN


def coulomb_reference(basis, D):
    """J_uv = sum_ls (uv|ls) D_ls by its plain definition: the oracle's
    integrals over every ordered shell quartet (no symmetry used)."""
    return jk_reference(basis, D)[0]


def jk_reference(basis, D):
    """(J, K) by their plain definitions, J_uv = sum_ls (uv|ls) D_ls and
    K_ul = sum_vs (uv|ls) D_vs, from the oracle's integrals over every
    ordered shell quartet (no symmetry used)."""
    off, nbf = bf_offsets(basis)
    ns = basis.nshell
    quartets = np.stack(np.meshgrid(*(np.arange(ns),) * 4, indexing="ij"), -1).reshape(-1, 4).astype(np.int32)
    vals = oracle.eri_quartets(basis, quartets, prec="d", threads=THREADS)
    sizes = oracle.shellset_size(basis, quartets)
    pos = np.concatenate([[0], np.cumsum(sizes)])
    n = (basis.shell_l + 1) * (basis.shell_l + 2) // 2
    J = np.zeros((nbf, nbf))
    K = np.zeros((nbf, nbf))

    def sl(x):
        return slice(off[x], off[x] + n[x])

    for i, (a, b, c, d) in enumerate(quartets):
        blk = vals[pos[i]:pos[i + 1]].reshape(n[a], n[b], n[c], n[d])
        J[sl(a), sl(b)] += np.einsum("abcd,cd->ab", blk, D[sl(c), sl(d)])
        K[sl(a), sl(c)] += np.einsum("abcd,bd->ac", blk, D[sl(b), sl(d)])
    return J, K


def test_plan_coulomb_against_oracle(cuda):
    """The Coulomb digestion (eri_plan_coulomb) over the plan's unique
    quartets, expanded by the permutational symmetry, against the plain
    definition over all ordered quartets (2 atoms, s/p/d shells with K = 6,
    3, 1: covers a == b, c == d and bra == ket quartets)."""
    basis = synth.molecule_basis(natom=2, radius=1.6, seed=21)
    _, nbf = bf_offsets(basis)
    rng = np.random.default_rng(22)
    U = rng.uniform(-1, 1, (nbf, nbf))
    D = np.triu(U) + np.triu(U, 1).T
    ref = coulomb_reference(basis, D)
    db = eri.DeviceBasis(basis)
    Dd = torch.as_tensor(D, device=cuda)
    plan = eri.Plan(db, threshold=0.0)
    J = plan.coulomb(Dd)
    torch.cuda.synchronize()
    assert plan.status() == eri.ERI_OK
    got = J.cpu().numpy()
    assert np.array_equal(got, got.T)
    scale = float(np.abs(ref).max())
    assert_close(got, ref, atol=1e-11 * scale, rtol=1e-10, what="J")
    # the replay re-reads its parameters: J of 2D is 2J, and the energy mode still works
    J2 = plan.coulomb(2.0 * Dd)
    # (the atomic additions take another order: entries near zero differ by round-off)
    assert torch.allclose(J2, 2.0 * J, rtol=1e-12, atol=1e-13 * scale)
    e = torch.zeros(1, dtype=torch.float64, device=cuda)
    plan.execute(D=Dd, energy=e)
    assert plan.status() == eri.ERI_OK and np.isfinite(float(e.item()))
    # split-precision transforms
    Js = eri.Plan(db, threshold=0.0, flags=eri.ERI_PLAN_SPLIT).coulomb(Dd).cpu().numpy()
    assert_close(Js, ref, atol=1e-11 * scale, rtol=1e-10, what="J split")


def test_plan_coulomb_screened_and_misuse(cuda):
    """A screened J differs from the unscreened one by no more than the
    dropped quartets allow; a store-mode plan or a wrong nbf is refused."""
    basis = synth.molecule_basis(natom=6, radius=9.0, seed=11)
    _, nbf = bf_offsets(basis)
    db = eri.DeviceBasis(basis)
    D = torch.as_tensor(np.random.default_rng(3).uniform(-1, 1, (nbf, nbf)), device=cuda)
    D = 0.5 * (D + D.T)
    thr = 1e-8
    p1 = eri.Plan(db, threshold=thr)
    p0 = eri.Plan(db, threshold=0.0)
    J1 = p1.coulomb(D).cpu().numpy()
    J0 = p0.coulomb(D).cpu().numpy()
    dropped = p0.info()["nquartets"] - p1.info()["nquartets"]
    assert dropped > 0
    # each dropped element |(ab|cd)| < thr enters at most 8 images with |D| <= 1
    assert np.abs(J1 - J0).max() <= 8 * dropped * thr * 6 ** 2
    store = eri.Plan(db, threshold=thr, flags=eri.ERI_PLAN_STORE)
    with pytest.raises(eri.EriError) as ex:
        store.coulomb(D)
    assert ex.value.code == eri.ERI_EPLAN
    with pytest.raises(eri.EriError) as ex:
        p1.coulomb(D[:3, :3].contiguous())
    assert ex.value.code == eri.ERI_EPLAN


def test_plan_exchange_against_oracle(cuda):
    """The exchange digestion (eri_plan_jk) against the plain definition
    K_ul = sum_vs (uv|ls) D_vs over all ordered quartets, alone and together
    with J in one replay; split-precision transforms too."""
    basis = synth.molecule_basis(natom=2, radius=1.6, seed=21)
    _, nbf = bf_offsets(basis)
    rng = np.random.default_rng(23)
    U = rng.uniform(-1, 1, (nbf, nbf))
    D = np.triu(U) + np.triu(U, 1).T
    Jref, Kref = jk_reference(basis, D)
    db = eri.DeviceBasis(basis)
    Dd = torch.as_tensor(D, device=cuda)
    plan = eri.Plan(db, threshold=0.0)
    sj, sk = float(np.abs(Jref).max()), float(np.abs(Kref).max())
    J, K = plan.jk(Dd)
    torch.cuda.synchronize()
    assert plan.status() == eri.ERI_OK
    assert_close(J.cpu().numpy(), Jref, atol=1e-11 * sj, rtol=1e-10, what="J (jk)")
    Kh = K.cpu().numpy()
    assert np.array_equal(Kh, Kh.T)
    assert_close(Kh, Kref, atol=1e-11 * sk, rtol=1e-10, what="K (jk)")
    _, K1 = plan.jk(Dd, want_j=False)
    assert_close(K1.cpu().numpy(), Kref, atol=1e-11 * sk, rtol=1e-10, what="K alone")
    J1, _ = plan.jk(Dd, want_k=False)
    assert_close(J1.cpu().numpy(), Jref, atol=1e-11 * sj, rtol=1e-10, what="J alone")
    _, Ks = eri.Plan(db, threshold=0.0, flags=eri.ERI_PLAN_SPLIT).jk(Dd, want_j=False)
    assert_close(Ks.cpu().numpy(), Kref, atol=1e-11 * sk, rtol=1e-10, what="K split")
    with pytest.raises(eri.EriError) as ex:
        plan.jk(Dd, want_j=False, want_k=False)
    assert ex.value.code == eri.ERI_EPLAN


def test_plan_full_size_sampled(cuda):
    """The benchmark's batched workload (16 atoms, Schwarz 1e-12, 1.08e7
    unique quartets) in store mode: a sample of 200 quartets spread over the
    jobs against the oracle, and the energy digestion against the stored
    integrals weighted by D_ab D_cd (summed on the GPU)."""
    basis = synth.molecule_basis(natom=16, radius=7.0 * (16 / 64) ** (1 / 3), seed=0)
    _, nbf = bf_offsets(basis)
    db = eri.DeviceBasis(basis)
    store = eri.Plan(db, threshold=1e-12, flags=eri.ERI_PLAN_STORE)
    info = store.info()
    out = torch.empty(info["out_len"], dtype=torch.float64, device=cuda)
    store.execute(out=out)
    torch.cuda.synchronize()
    assert store.status() == eri.ERI_OK
    rng = np.random.default_rng(8)
    U = rng.uniform(-1, 1, (nbf, nbf))
    D = np.triu(U) + np.triu(U, 1).T
    Dd = torch.as_tensor(D, device=cuda)
    off_bf, _ = bf_offsets(basis)
    offd = torch.as_tensor(off_bf, device=cuda)
    e_store = 0.0
    sampled, refs = [], []
    njobs = info["njobs"]
    for j in range(njobs):
        cls, nq, off, shells = store.job(j, with_quartets=True)
        n = [nc(l) for l in cls]
        blk = out[off:off + nq * int(np.prod(n))].view(int(np.prod(n)), nq)  # [abcd][q]
        sh = torch.as_tensor(shells, device=cuda, dtype=torch.int64)
        idx = [offd[sh[:, i]][:, None] + torch.arange(n[i], device=cuda)[None, :] for i in range(4)]
        Dab = Dd[idx[0][:, :, None], idx[1][:, None, :]].reshape(nq, -1)
        Dcd = Dd[idx[2][:, :, None], idx[3][:, None, :]].reshape(nq, -1)
        W = (Dab[:, :, None] * Dcd[:, None, :]).reshape(nq, -1).T
        e_store += float((blk * W).sum())
        pick = rng.choice(nq, min(nq, max(1, 200 // njobs + 1)), replace=False)
        sampled.append(blk[:, torch.as_tensor(pick, device=cuda)].T.cpu().numpy())
        refs.append(oracle.eri_quartets(basis, shells[pick], prec="d", threads=THREADS).reshape(len(pick), -1))
    for got, ref in zip(sampled, refs):
        assert_close(got, ref, what="plan store, 16 atoms")
    e = torch.zeros(1, dtype=torch.float64, device=cuda)
    plan = eri.Plan(db, threshold=1e-12)
    assert plan.info()["nquartets"] == info["nquartets"]
    plan.execute(D=Dd, energy=e)
    assert plan.status() == eri.ERI_OK
    # the two sums take different orders over 1e7 quartets (atomics): relative round-off only
    assert abs(float(e.item()) - e_store) <= 1e-10 * max(1.0, abs(e_store)), (float(e.item()), e_store)


def test_plan_slices_sum_to_whole_plan(cuda):
    """Several ranks on one plan: the slices eri_plan_set_slice keeps for
    ranks 0..n-1 partition the work items (their quartets add up to the
    plan's), and their energies, J and K add up to the whole plan's, which
    itself matches the oracle on the store form.  The slices run one after
    another on one GPU (no rank waits on another)."""
    basis = synth.molecule_basis(natom=4, radius=2.6, seed=8)
    _, nbf = bf_offsets(basis)
    U = np.random.default_rng(9).uniform(-1, 1, (nbf, nbf))
    Dm = torch.as_tensor(np.triu(U) + np.triu(U, 1).T, device=cuda)
    db = eri.DeviceBasis(basis)
    plan = eri.Plan(db, threshold=1e-12)
    info = plan.info()
    e = torch.zeros(1, dtype=torch.float64, device=cuda)
    plan.execute(D=Dm, energy=e)
    J, K = plan.jk(Dm)
    whole = (float(e.item()), J.clone(), K.clone())
    for n in (2, 3):
        tot_e, tot_q, tot_items = 0.0, 0, 0
        tot_J = torch.zeros_like(Dm)
        tot_K = torch.zeros_like(Dm)
        for r in range(n):
            plan.set_slice(r, n)
            si = plan.slice_info()
            assert si["nquartets"] > 0
            tot_q += si["nquartets"]
            tot_items += si["nitems"]
            plan.execute(D=Dm, energy=e)
            tot_e += float(e.item())
            Jr, Kr = plan.jk(Dm)
            tot_J += Jr
            tot_K += Kr
        assert tot_q == info["nquartets"] and tot_items == info["nitems"]
        assert abs(tot_e - whole[0]) <= 1e-12 * max(1.0, abs(whole[0]))
        assert float((tot_J - whole[1]).abs().max()) <= 1e-12 * float(whole[1].abs().max())
        assert float((tot_K - whole[2]).abs().max()) <= 1e-12 * float(whole[2].abs().max())
    plan.set_slice(0, 1)  # the whole plan again
    assert plan.slice_info()["nquartets"] == info["nquartets"]
    plan.execute(D=Dm, energy=e)
    assert abs(float(e.item()) - whole[0]) <= 1e-13 * max(1.0, abs(whole[0]))
    with pytest.raises(eri.EriError):
        plan.set_slice(2, 2)
    plan.destroy()
