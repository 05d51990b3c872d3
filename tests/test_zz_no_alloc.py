"""eri_batch_noalloc: the entry point for callers that may not allocate.

A process whose GPU memory belongs to another allocator (a framework's
memory pool) must not call cudaMalloc itself, and code that runs while a
stream is being captured into a CUDA graph must not allocate at all.  This
entry point computes the same integrals as eri_batch using only a fixed
scratch array compiled into the library.  These tests call it through the C
ABI twice in a row (the second call reuses the scratch the first one left
behind) and compare every element with eri_batch, with the tolerance of the
other parity tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import ATOL, RTOL, assert_close, to_device

pytestmark = pytest.mark.gpu


def _case(cls, seed, nq):
    basis, pools = synth.class_sweep_pools(seed=seed, pool=64, K=3)
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=seed, npairs=96, nq=nq)
    return basis, bra, ket, q


def test_noalloc_matches_eri_batch_on_two_calls_in_a_row(cuda):
    cases = [((2, 1, 1, 0), 11, 3000), ((1, 1, 2, 2), 12, 700)]
    results = []
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
        results.append(assert_close(out.cpu().numpy(), ref, atol=ATOL, rtol=RTOL, what=f"noalloc {cls}"))
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
