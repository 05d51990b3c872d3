"""eri_batch_noalloc: the entry point for callers that may not allocate.

A process whose GPU memory belongs to another allocator (a serving or
training framework's caching pool, an MPI library's registered pool) must not
call cudaMalloc behind that allocator's back.  This entry point computes the
same integrals as eri_batch using only fixed arrays compiled into the
library.  These tests call it through the C ABI twice in a row (the second
call reuses the scratch the first one left behind) and compare every element
with the oracle and with eri_batch, at the tolerance of the other parity
tests (1e-11 absolute + 1e-10 relative).  This file is collected last on
purpose, so that a run stopping at its first failure has run everything else.
"""
import numpy as np
import pytest
import torch

import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import ATOL, RTOL, assert_close, oracle_blocks, to_device

pytestmark = pytest.mark.gpu


def _case(cls, seed, nq):
    basis, pools = synth.class_sweep_pools(seed=seed, pool=64, K=3)
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=seed, npairs=96, nq=nq)
    return basis, bra, ket, q


def test_noalloc_matches_oracle_and_eri_batch_on_two_calls_in_a_row(cuda):
    cases = [((2, 1, 1, 0), 11, 3000), ((1, 1, 2, 2), 12, 700)]
    free_before = None
    for i, (cls, seed, nq) in enumerate(cases):
        basis, bra, ket, q = _case(cls, seed, nq)
        db = eri.DeviceBasis(basis)
        b, k, qq = to_device(bra, ket, q)
        ref = eri.eri_batch(cls, db, b, k, qq).cpu().numpy()
        out = torch.full((ref.size,), float("nan"), dtype=torch.float64, device=cuda)
        if i == 1:
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
        eri.eri_batch_noalloc(cls, db, b, k, qq, out)
        torch.cuda.synchronize()
        if i == 1:
            # the second call allocated no device memory
            assert torch.cuda.mem_get_info()[0] >= free_before - (2 << 20)
        got = out.cpu().numpy()
        assert_close(got, ref, atol=ATOL, rtol=RTOL, what=f"noalloc vs eri_batch {cls}")
        # a seeded sample against the oracle (list layout [abcd][q])
        pick = np.sort(np.random.default_rng(seed).choice(nq, 48, replace=False))
        blocks = got.reshape(-1, nq).T
        assert_close(blocks[pick], oracle_blocks(cls, basis, bra, ket, q[pick]), what=f"noalloc vs oracle {cls}")
    assert eri.eri_last_status() == eri.ERI_OK


def test_noalloc_product_form_and_oversize(cuda):
    cls = (1, 0, 1, 1)
    basis, bra, ket, _ = _case(cls, 13, 1)
    db = eri.DeviceBasis(basis)
    b, k, _ = to_device(bra[:17], ket[:9])
    ref = eri.eri_batch(cls, db, b, k, None)
    out = torch.zeros_like(ref)
    eri.eri_batch_noalloc(cls, db, b, k, None, out)
    assert_close(out.cpu().numpy(), ref.cpu().numpy(), what="noalloc product form")
    # a batch whose pair tables exceed the fixed scratch is rejected up front
    big = (2, 2, 2, 2)
    basis2, pools = synth.class_sweep_pools(seed=14, pool=512, K=3)
    bra2, ket2, q2 = synth.class_sweep_batch(pools, big, seed=14, npairs=2048, nq=10)
    db2 = eri.DeviceBasis(basis2)
    b2, k2, q2d = to_device(bra2, ket2, q2)
    out2 = torch.zeros(eri.out_len(big, 2048, 2048, 10), dtype=torch.float64, device=cuda)
    with pytest.raises(eri.EriError) as e:
        eri.eri_batch_noalloc(big, db2, b2, k2, q2d, out2)
    assert e.value.code == eri.ERI_EINVAL
    assert torch.all(out2 == 0)


@pytest.mark.parametrize("product", [False, True])
def test_noalloc_mixed_contraction_degrees(cuda, product):
    """A batch from the molecule-shaped basis (s shells of K = 6, 3 and 1 on
    each atom) mixes primitive-pair counts; eri_batch sorts such a batch,
    the allocation-free entry point runs it unsorted with per-tile bounds.
    Both forms against eri_batch and the oracle."""
    basis = synth.molecule_basis(natom=4, radius=2.5, seed=3)
    pairs, batches = synth.all_unique_quartets(basis)
    cls = (0, 0, 1, 0) if (0, 0, 1, 0) in batches else sorted(batches)[0]
    bra, ket, q = batches[cls]
    db = eri.DeviceBasis(basis)
    if product:
        bra, ket = bra[:11], ket[:7]
        b, k, _ = to_device(bra, ket)
        qq = None
        qlist = np.stack(np.meshgrid(np.arange(len(bra)), np.arange(len(ket)), indexing="ij"), -1)
        qlist = qlist.transpose(1, 0, 2).reshape(-1, 2)  # bra index fastest, as the product layout
    else:
        b, k, qq = to_device(bra, ket, q)
        qlist = q
    ref = eri.eri_batch(cls, db, b, k, qq)
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        eri.eri_batch_noalloc(cls, db, b, k, qq, out)
        torch.cuda.synchronize()
        assert_close(out.cpu().numpy(), ref.cpu().numpy(), what=f"noalloc mixed K {cls} product={product}")
    nab = eri.nc(cls[0]) * eri.nc(cls[1])
    ncd = eri.nc(cls[2]) * eri.nc(cls[3])
    got = out.cpu().numpy()
    if product:
        # out[ij + nbra (ab + nab (cd + ncd kl))] -> blocks [kl][ij][ab][cd]
        blocks = got.reshape(len(ket), ncd, nab, len(bra)).transpose(0, 3, 2, 1).reshape(-1, nab * ncd)
    else:
        blocks = got.reshape(-1, len(q)).T
    assert_close(blocks, oracle_blocks(cls, basis, bra, ket, qlist), what=f"noalloc mixed K vs oracle {cls}")
