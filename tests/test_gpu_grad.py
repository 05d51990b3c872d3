"""Parity of the CUDA adjoint (eri_batch_grad, ERIFunction) against the
oracle's analytic derivative and against central finite differences of the
CUDA forward path."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import THREADS, to_device

pytestmark = pytest.mark.gpu


def grad_close(got, ref, what, rtol=1e-10):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(1.0, float(np.max(np.abs(ref))))
    err = np.abs(got - ref)
    assert np.all(err <= 1e-11 * scale + rtol * np.abs(ref)), (what, float(err.max()), scale)


def gpu_grad(cls, basis, bra, ket, q, W):
    db = eri.DeviceBasis(basis)
    b, k, qq = to_device(bra, ket, q)
    gc = torch.zeros_like(db.centres)
    ge = torch.zeros_like(db.exps)
    eri.eri_batch_grad(cls, db, b, k, qq, torch.as_tensor(W, device="cuda"), gc, ge)
    torch.cuda.synchronize()
    return gc.cpu().numpy(), ge.cpu().numpy()


@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 0, 1, 0), (1, 1, 1, 1), (2, 0, 1, 0),
                                 (2, 1, 2, 0), (0, 0, 2, 2), (2, 2, 1, 1), (2, 2, 2, 2), (3, 0, 1, 0),
                                 (3, 3, 1, 0), (1, 0, 3, 3), (3, 2, 0, 0)])
@pytest.mark.parametrize("K", [2, 3])
def test_grad_against_oracle(cuda, cls, K):
    """Centre and exponent derivatives of sum W (ab|cd) for random W, K = 2 or
    3 per shell (an odd K leaves a partial chunk of bra primitives), against
    the oracle's shifted-monomial derivative, in each of the two forms
    (X: ket transform over the raised bra range, then W; V: W met with the
    ket E products first) forced in turn, each in two launches (one per
    side's channels) and in one launch for every channel."""
    if K == 3 and sum(cls) > 6:
        pytest.skip("oracle time")
    basis, pools = synth.class_sweep_pools(seed=3, lmax=max(2, max(cls)), pool=24, K=K, cube=5.0)
    nq = 60 if sum(cls) <= 4 else 12
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=4, npairs=20, nq=nq)
    n = eri.out_len(cls, bra.shape[0], ket.shape[0], nq)
    W = np.random.default_rng(8).uniform(-1, 1, n)
    # oracle W layout: per quartet [ab][cd] blocks
    Wq = W.reshape(-1, nq).T.reshape(-1)
    rc, re = oracle.eri_grad_quartets(basis, synth.quartet_shells(bra, ket, q), Wq, prec="d", threads=THREADS)
    try:
        for form in (eri.ERI_GRAD_X, eri.ERI_GRAD_V):
            for one in (False, True):
                # two launches (one per side's channels) or one launch for every channel
                eri.eri_set_grad_forms((1 << form) | (1 << (eri.ERI_GRAD_ONE if one else eri.ERI_GRAD_TWO)))
                gc, ge = gpu_grad(cls, basis, bra, ket, q, W)
                ran = eri.eri_last_grad_forms()
                assert ran in ([(form, eri.ERI_GRAD_ONE), (form, eri.ERI_GRAD_ONE_SWAPPED)] if one else [(form, form)])
                grad_close(gc, rc, f"centres {cls} forms {ran}")
                grad_close(ge, re, f"exponents {cls} forms {ran}")
                assert abs(gc.sum(axis=0)).max() < 1e-10 * max(1.0, abs(gc).max())  # translation invariance
    finally:
        eri.eri_set_grad_forms(0)


@pytest.mark.parametrize("one", [False, True])
@pytest.mark.parametrize("form", [0, 1])
def test_grad_mixed_K_and_product_form(cuda, form, one):
    basis = synth.molecule_basis(natom=5, radius=3.0, seed=2)
    pairs = synth.unique_pairs(basis)
    sel = pairs[(basis.shell_l[pairs[:, 0]] == 1) & (basis.shell_l[pairs[:, 1]] == 0)][:9]
    ket = pairs[(basis.shell_l[pairs[:, 0]] == 0) & (basis.shell_l[pairs[:, 1]] == 0)][:7]
    cls = (1, 0, 0, 0)
    n = eri.out_len(cls, sel.shape[0], ket.shape[0], None)
    W = np.random.default_rng(1).uniform(-1, 1, n)
    db = eri.DeviceBasis(basis)
    b, k, _ = to_device(sel, ket)
    gc = torch.zeros_like(db.centres)
    ge = torch.zeros_like(db.exps)
    try:
        eri.eri_set_grad_forms((1 << form) | (1 << (eri.ERI_GRAD_ONE if one else eri.ERI_GRAD_TWO)))
        eri.eri_batch_grad(cls, db, b, k, None, torch.as_tensor(W, device="cuda"), gc, ge)
        assert eri.eri_last_grad_forms() in ([(form, eri.ERI_GRAD_ONE), (form, eri.ERI_GRAD_ONE_SWAPPED)] if one
                                             else [(form, form)])
    finally:
        eri.eri_set_grad_forms(0)
    q = np.array([(i, j) for j in range(ket.shape[0]) for i in range(sel.shape[0])], dtype=np.int64)
    # product layout [kl][cd][ab][ij] -> per quartet [ab][cd]
    Wq = W.reshape(ket.shape[0], 1, 3, sel.shape[0]).transpose(0, 3, 2, 1).reshape(-1)
    rc, re = oracle.eri_grad_quartets(basis, synth.quartet_shells(sel, ket, q), Wq, prec="d")
    grad_close(gc.cpu().numpy(), rc, "centres product")
    grad_close(ge.cpu().numpy(), re, "exponents product")


def test_autograd_function_and_finite_differences(cuda):
    """ERIFunction: backward(W) equals eri_batch_grad, and both match central
    finite differences (h = 1e-5) of the GPU forward energy."""
    cls = (2, 1, 1, 0)
    basis, pools = synth.class_sweep_pools(seed=6, pool=16, K=2, cube=4.0)
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=7, npairs=12, nq=40)
    db = eri.DeviceBasis(basis)
    b, k, qq = to_device(bra, ket, q)
    W = torch.as_tensor(np.random.default_rng(2).uniform(-1, 1, eri.out_len(cls, 12, 12, 40)), device="cuda")
    centres = db.centres.clone().requires_grad_(True)
    exps = db.exps.clone().requires_grad_(True)
    E = (eri.eri(centres, exps, cls, db, b, k, qq) * W).sum()
    E.backward()
    gc, ge = centres.grad.cpu().numpy(), exps.grad.cpu().numpy()

    def energy(c, e):
        return float((eri.eri_batch(cls, db, b, k, qq, centres=c, exps=e) * W).sum())

    h = 1e-5
    atoms = np.unique(np.concatenate([bra.ravel(), ket.ravel()]))[:4]
    for at in atoms:
        for x in range(3):
            cp = db.centres.clone()
            cm = db.centres.clone()
            cp[basis.shell_atom[at], x] += h
            cm[basis.shell_atom[at], x] -= h
            fd = (energy(cp, db.exps) - energy(cm, db.exps)) / (2 * h)
            g = gc[basis.shell_atom[at], x]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (at, x, fd, g)
    for prim in (int(basis.shell_off[bra[0, 0]]), int(basis.shell_off[ket[0, 1]]) + 1):
        ep = db.exps.clone()
        em = db.exps.clone()
        ep[prim] += h
        em[prim] -= h
        fd = (energy(db.centres, ep) - energy(db.centres, em)) / (2 * h)
        assert abs(fd - ge[prim]) <= 1e-6 * max(1.0, abs(ge[prim])), (prim, fd, ge[prim])


def test_grad_errors(cuda):
    basis, pools = synth.class_sweep_pools(seed=0, pool=8, K=1)
    db = eri.DeviceBasis(basis)
    bra, ket, q = synth.class_sweep_batch(pools, (1, 0, 1, 0), seed=0, npairs=4, nq=6)
    b, k, qq = to_device(bra, ket, q)
    gc = torch.zeros_like(db.centres)
    with pytest.raises(eri.EriError):  # W too short
        eri.eri_batch_grad((1, 0, 1, 0), db, b, k, qq, torch.zeros(3, dtype=torch.float64, device="cuda"), gc, None)
    W = torch.zeros(eri.out_len((1, 0, 1, 0), 4, 4, 6), dtype=torch.float64, device="cuda")
    eri.eri_batch_grad((1, 0, 1, 0), db, b, k, qq, W, gc, None)   # zero weights -> zero gradient
    assert torch.all(gc == 0)


@pytest.mark.parametrize("cls,K", [((1, 1, 1, 1), 8), ((0, 0, 2, 3), 5), ((0, 0, 3, 3), 3), ((1, 3, 3, 3), 2),
                                   ((3, 3, 3, 3), 1)])
def test_grad_contraction_degree_limits(cuda, cls, K):
    """The contraction degrees eri_batch_grad guarantees with the same K on
    all four shells (K = 8 up to L = 4, 5 at L = 5, 3 at L = 6..9, 2 at
    L = 10, 1 at L = 11, 12), on classes that reach exactly that bound (a d-f
    or f-f pair), match the oracle's derivative; one more primitive per shell
    is refused with ERI_EINVAL."""
    basis, bra, ket, q = synth.small_random_batch(cls, K=(K,) * 4, nq=2, seed=6)
    n = eri.out_len(cls, bra.shape[0], ket.shape[0], q.shape[0])
    W = np.random.default_rng(9).uniform(-1, 1, n)
    Wq = W.reshape(-1, q.shape[0]).T.reshape(-1)
    rc, re = oracle.eri_grad_quartets(basis, synth.quartet_shells(bra, ket, q), Wq, prec="d", threads=THREADS)
    gc, ge = gpu_grad(cls, basis, bra, ket, q, W)
    grad_close(gc, rc, f"centres {cls} K={K}")
    grad_close(ge, re, f"exponents {cls} K={K}")
    basis, bra, ket, q = synth.small_random_batch(cls, K=(K + 1,) * 4, nq=2, seed=6)
    with pytest.raises(eri.EriError) as e:
        gpu_grad(cls, basis, bra, ket, q, W)
    assert e.value.code == eri.ERI_EINVAL
