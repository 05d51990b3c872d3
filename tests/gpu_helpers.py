"""Shared helpers of the GPU parity tests: run the library, run the oracle,
compare element by element."""
from __future__ import annotations

import os

import numpy as np
import torch

import oracle
import synth
import paper_2506_12501_gb300 as eri

# |got - ref| <= ATOL + RTOL |ref| per element (FP64 path against the oracle)
ATOL, RTOL = 1e-11, 1e-10
THREADS = max(1, min(16, os.cpu_count() or 1))


def nc(l):
    return (l + 1) * (l + 2) // 2


def to_device(bra, ket, q=None, dev="cuda"):
    b = torch.as_tensor(np.ascontiguousarray(bra), dtype=torch.int32, device=dev)
    k = torch.as_tensor(np.ascontiguousarray(ket), dtype=torch.int32, device=dev)
    qq = None if q is None else torch.as_tensor(np.ascontiguousarray(q), dtype=torch.int64, device=dev)
    return b, k, qq


def gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_FP64, dbasis=None):
    """List-form batch on the GPU, returned as blocks [q][ab*ncd+cd]."""
    db = dbasis or eri.DeviceBasis(basis)
    b, k, qq = to_device(bra, ket, q)
    out = eri.eri_batch(cls, db, b, k, qq, precision=precision)
    torch.cuda.synchronize()
    nq = q.shape[0]
    return out.cpu().numpy().reshape(-1, nq).T.copy()


def oracle_blocks(cls, basis, bra, ket, q, prec="d"):
    qs = synth.quartet_shells(bra, ket, q)
    ref = oracle.eri_quartets(basis, qs, prec=prec, threads=THREADS)
    nab, ncd = nc(cls[0]) * nc(cls[1]), nc(cls[2]) * nc(cls[3])
    return ref.astype(np.float64).reshape(len(qs), nab * ncd)


def assert_close(got, ref, atol=ATOL, rtol=RTOL, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    err = np.abs(got - ref)
    bad = err > atol + rtol * np.abs(ref)
    if np.any(bad):
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {int(bad.sum())} of {bad.size} elements out of tolerance; first at {tuple(i)}: "
                             f"got {got[tuple(i)]!r} ref {ref[tuple(i)]!r}; max err {err.max():.3e}")
    return float(err.max())
