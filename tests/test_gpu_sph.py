"""Solid-harmonic 4-centre output (eri_batch_sph): every centre mapped to real
solid harmonics, against the oracle's Cartesian integrals transformed with
the oracle's own closed-form harmonics (oracle/solid.py)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import assert_close, oracle_blocks, to_device

pytestmark = pytest.mark.gpu


def sph_reference(cls, basis, bra, ket, q):
    la, lb, lc, ld = cls
    nc = [oracle.ncart(l) for l in cls]
    cart = oracle_blocks(cls, basis, bra, ket, q).reshape(len(q), *nc)
    C = [oracle.solid.c2s(l) for l in cls]
    out = np.einsum("qabcd,ia,jb,kc,ld->qijkl", cart, *C)
    return out.reshape(len(q), -1)


def gpu_sph(cls, basis, bra, ket, q, db=None, precision=eri.ERI_PREC_FP64):
    db = db or eri.DeviceBasis(basis)
    b, k, qq = to_device(bra, ket, q)
    out = eri.eri_batch_sph(cls, db, b, k, qq, precision=precision)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(-1, len(q)).T


@pytest.fixture(scope="module")
def pools():
    return synth.class_sweep_pools(seed=0, pool=64, K=2)


@pytest.mark.parametrize("cls", synth.all_classes(2))
def test_sph_against_oracle(cuda, pools, cls):
    basis, pl = pools
    L = sum(cls)
    bra, ket, q = synth.class_sweep_batch(pl, cls, seed=4, npairs=40, nq=97 if L <= 4 else 31)
    assert_close(gpu_sph(cls, basis, bra, ket, q), sph_reference(cls, basis, bra, ket, q), what=f"sph {cls}")


@pytest.mark.parametrize("cls", [(2, 2, 2, 2), (2, 1, 2, 0), (1, 2, 2, 1), (3, 2, 1, 0), (3, 3, 2, 2)])
def test_sph_every_form_and_split(cuda, cls):
    """Each form forced (plain or swapped; full pairs or recursions), and the
    split-precision transforms, with solid-harmonic output."""
    basis, bra, ket, q = synth.split_batch(cls, K=1, seed=50 + sum(cls), nq=23, pool=16, npairs=8)
    ref = sph_reference(cls, basis, bra, ket, q)
    db = eri.DeviceBasis(basis)
    try:
        for form in range(4):
            eri.eri_set_forms(1 << form)
            assert_close(gpu_sph(cls, basis, bra, ket, q, db=db), ref, what=f"sph {cls} form {form}")
    finally:
        eri.eri_set_forms(0)
    assert_close(gpu_sph(cls, basis, bra, ket, q, db=db, precision=eri.ERI_PREC_SPLIT), ref, atol=1e-10,
                 what=f"sph {cls} split")


def test_sph_product_form_and_full_size(cuda):
    basis, pl = synth.class_sweep_pools(seed=0, pool=512, K=3)
    cls = (2, 2, 2, 1)
    bra, ket, q = synth.class_sweep_batch(pl, cls, seed=0, npairs=2048, nq=100_000)
    db = eri.DeviceBasis(basis)
    b, k, qq = to_device(bra, ket, q)
    out = eri.eri_batch_sph(cls, db, b, k, qq)
    torch.cuda.synchronize()
    nq = len(q)
    sample = np.random.default_rng(9).choice(nq, 32, replace=False)
    sample[:2] = [0, nq - 1]
    got = out.view(-1, nq)[:, torch.as_tensor(sample, device=cuda)].T.cpu().numpy()
    assert_close(got, sph_reference(cls, basis, bra, ket, q[sample]), what="sph full size")
    # product form, small
    b2, k2, _ = to_device(bra[:3], ket[:2])
    outp = eri.eri_batch_sph(cls, db, b2, k2, None).cpu().numpy()
    qp = np.array([(i, j) for j in range(2) for i in range(3)], dtype=np.int64)
    ref = sph_reference(cls, basis, bra[:3], ket[:2], qp).reshape(2, 3, 25, 15)  # [k][i][ab][cd]
    assert_close(outp.reshape(2, 15, 25, 3), ref.transpose(0, 3, 2, 1), what="sph product form")
