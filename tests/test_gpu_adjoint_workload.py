"""The adjoint workload: 16 atoms with the molecule-shaped basis (s x3 with
K = 6, 3, 1, p x2 with K = 3, 1, d with K = 1), W_abcd = D_ab D_cd with a
seeded symmetric D; the gradient of E = sum over every unique quartet of
W (ab|cd) with respect to the 48 coordinates and the 240 exponents.

Checked against central finite differences (h = 1e-5) of E computed by the
plan (a different kernel: the persistent digestion path), and against the
oracle's analytic derivative on a 2000-quartet subset (the gradient is
additive over quartets)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import THREADS

pytestmark = pytest.mark.gpu


def nc(l):
    return (l + 1) * (l + 2) // 2


def device_weights(cls, bra, ket, q, D, bf_off):
    """W in the list-form layout, W[q + nq*(ab*ncd + cd)] = D_ab D_cd (input generation)."""
    dev = D.device
    bra = torch.as_tensor(bra, device=dev, dtype=torch.int64)
    ket = torch.as_tensor(ket, device=dev, dtype=torch.int64)
    q = torch.as_tensor(q, device=dev, dtype=torch.int64)
    off = torch.as_tensor(bf_off, device=dev, dtype=torch.int64)
    idx = []
    for sh, l in ((bra[q[:, 0], 0], cls[0]), (bra[q[:, 0], 1], cls[1]), (ket[q[:, 1], 0], cls[2]),
                  (ket[q[:, 1], 1], cls[3])):
        idx.append(off[sh][:, None] + torch.arange(nc(l), device=dev)[None, :])
    Dab = D[idx[0][:, :, None], idx[1][:, None, :]].reshape(len(q), -1)
    Dcd = D[idx[2][:, :, None], idx[3][:, None, :]].reshape(len(q), -1)
    return (Dab[:, :, None] * Dcd[:, None, :]).reshape(len(q), -1).T.contiguous().reshape(-1)


@pytest.fixture(scope="module")
def workload():
    basis, D, bf_off = synth.adjoint_workload(natom=16, radius=4.4, seed=0)
    pairs, batches = synth.all_unique_quartets(basis)
    return basis, D, bf_off, batches


def gpu_gradient(basis, D, bf_off, batches):
    db = eri.DeviceBasis(basis)
    Dd = torch.as_tensor(D, device="cuda")
    gc = torch.zeros_like(db.centres)
    ge = torch.zeros_like(db.exps)
    for cls, (bra, ket, q) in batches.items():
        W = device_weights(cls, bra, ket, q, Dd, bf_off)
        b = torch.as_tensor(bra, device="cuda")
        k = torch.as_tensor(ket, device="cuda")
        qq = torch.as_tensor(q, device="cuda")
        eri.eri_batch_grad(cls, db, b, k, qq, W, gc, ge)
        del W
    torch.cuda.synchronize()
    return gc.cpu().numpy(), ge.cpu().numpy()


def plan_energy(basis, D):
    db = eri.DeviceBasis(basis)
    plan = eri.Plan(db, threshold=0.0, flags=eri.ERI_PLAN_NO_TUNE)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.execute(D=torch.as_tensor(D, device="cuda"), energy=e)
    assert plan.status() == eri.ERI_OK
    v = float(e.item())
    plan.destroy()
    return v


def test_adjoint_workload_against_finite_differences(cuda, workload):
    basis, D, bf_off, batches = workload
    assert sum(len(v[2]) for v in batches.values()) == 4656 * 4657 // 2
    gc, ge = gpu_gradient(basis, D, bf_off, batches)
    assert np.abs(gc.sum(axis=0)).max() < 1e-9 * np.abs(gc).max()   # translation invariance
    h = 1e-5
    for atom, ax in ((0, 0), (5, 1), (11, 2)):
        bp, bm = basis.copy(), basis.copy()
        bp.centres[atom, ax] += h
        bm.centres[atom, ax] -= h
        fd = (plan_energy(bp, D) - plan_energy(bm, D)) / (2 * h)
        assert abs(fd - gc[atom, ax]) <= 1e-6 * max(1.0, abs(gc[atom, ax])), (atom, ax, fd, gc[atom, ax])
    for prim in (0, 7, 200):
        bp, bm = basis.copy(), basis.copy()
        bp.exps[prim] += h
        bm.exps[prim] -= h
        fd = (plan_energy(bp, D) - plan_energy(bm, D)) / (2 * h)
        assert abs(fd - ge[prim]) <= 1e-6 * max(1.0, abs(ge[prim])), (prim, fd, ge[prim])


def test_adjoint_workload_subset_against_oracle(cuda, workload):
    basis, D, bf_off, batches = workload
    rng = np.random.default_rng(17)
    sub = {}
    total = sum(len(v[2]) for v in batches.values())
    for cls, (bra, ket, q) in batches.items():
        n = max(4, int(round(2000 * len(q) / total)))
        sel = np.sort(rng.choice(len(q), min(n, len(q)), replace=False))
        sub[cls] = (bra, ket, q[sel])
    gc, ge = gpu_gradient(basis, D, bf_off, sub)
    rc = np.zeros_like(gc)
    re = np.zeros_like(ge)
    for cls, (bra, ket, q) in sub.items():
        W = synth.density_weights(cls, bra, ket, q, D, bf_off)
        Wq = W.reshape(-1, len(q)).T.reshape(-1)
        c, e = oracle.eri_grad_quartets(basis, synth.quartet_shells(bra, ket, q), Wq, prec="d", threads=THREADS)
        rc += c.astype(np.float64)
        re += e.astype(np.float64)
    scale = max(1.0, float(np.abs(rc).max()), float(np.abs(re).max()))
    assert np.abs(gc - rc).max() <= 1e-11 * scale + 1e-10 * np.abs(rc).max()
    assert np.abs(ge - re).max() <= 1e-11 * scale + 1e-10 * np.abs(re).max()
