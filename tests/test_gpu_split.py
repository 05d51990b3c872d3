"""f-shell classes in FP64 and the split-precision (FP32 hi+lo transforms,
FP64 Boys/R/accumulation) form, against the oracle and against the FP64
path at the 1e-10 absolute bar of the measurement plan."""
import numpy as np
import pytest
import torch

import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import assert_close, gpu_list, oracle_blocks

pytestmark = pytest.mark.gpu

F_CLASSES = [(3, 0, 0, 0), (3, 1, 2, 0), (2, 3, 1, 3), (3, 3, 1, 1), (3, 2, 3, 2), (3, 3, 2, 2), (3, 3, 3, 3)]


@pytest.mark.parametrize("cls", F_CLASSES)
def test_f_classes_fp64_against_oracle(cuda, cls):
    """Exponents log-uniform in [0.05, 50] (the high-l workload), K = 1 and 2."""
    L = sum(cls)
    K = 1 if L >= 10 else 2
    nq = 12 if L >= 10 else 40
    basis, bra, ket, q = synth.split_batch(cls, K=K, seed=L, nq=nq, pool=16, npairs=8)
    got = gpu_list(cls, basis, bra, ket, q)
    ref = oracle_blocks(cls, basis, bra, ket, q, prec="d")
    assert_close(got, ref, what=f"fp64 {cls}")


@pytest.mark.parametrize("cls", F_CLASSES)
def test_f_classes_every_form(cuda, cls):
    """Each of the four forms forced on the f-shell classes (FP64 and split
    transforms), against the oracle.  Where the recursion form is infeasible
    (its (f0|e0) block exceeds the register accumulators or its buffers
    shared memory) the library falls back to a feasible form."""
    L = sum(cls)
    nq = 10 if L >= 10 else 24
    basis, bra, ket, q = synth.split_batch(cls, K=1, seed=200 + L, nq=nq, pool=16, npairs=8)
    ref = oracle_blocks(cls, basis, bra, ket, q, prec="d")
    db = eri.DeviceBasis(basis)
    try:
        for form in range(4):
            eri.eri_set_forms(1 << form)
            for prec in (eri.ERI_PREC_FP64, eri.ERI_PREC_SPLIT):
                got = gpu_list(cls, basis, bra, ket, q, precision=prec, dbasis=db)
                ran = eri.eri_last_form()
                if not (form & 2):
                    assert ran == (bool(form & 1), False)
                assert_close(got, ref, atol=1e-10 if prec == eri.ERI_PREC_SPLIT else 1e-11,
                             what=f"{cls} form {form} ran {ran} prec {prec}")
    finally:
        eri.eri_set_forms(0)


@pytest.mark.parametrize("cls,K,nq", [((2, 2, 2, 2), 1, 4000), ((3, 3, 3, 3), 1, 1000), ((3, 3, 2, 2), 1, 3000),
                                      ((2, 2, 2, 2), 5, 600), ((3, 3, 3, 3), 5, 40), ((3, 3, 2, 2), 5, 300)])
def test_split_against_fp64_path(cuda, cls, K, nq):
    """The split-precision form stays within 1e-10 absolute of the FP64 form on
    the high-l workload (K = 1 and K = 5 per shell), with the benchmark's
    spread of centres (512-shell pools in a 12-bohr cube, 2048 pairs)."""
    basis, bra, ket, q = synth.split_batch(cls, K=K, seed=100 + K, nq=nq, pool=512, npairs=2048)
    f64 = gpu_list(cls, basis, bra, ket, q)
    spl = gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_SPLIT)
    err = np.abs(spl - f64)
    print(f"split {cls} K={K}: max |split - fp64| = {err.max():.3e}, max |fp64| = {np.abs(f64).max():.3e}")
    assert_close(spl, f64, atol=1e-10, rtol=0.0, what=f"split {cls} K={K}")


@pytest.mark.parametrize("cls,K,nq", [((2, 2, 2, 2), 1, 16), ((3, 3, 2, 2), 1, 16), ((3, 3, 3, 3), 1, 8),
                                      ((2, 2, 2, 2), 5, 32), ((3, 3, 3, 3), 5, 16), ((3, 3, 2, 2), 5, 24)])
def test_fp64_and_split_against_oracle(cuda, cls, K, nq):
    """Both forms against the oracle, element by element, on the high-l
    workload (exponents log-uniform in [0.05, 50], centres in a 12-bohr cube),
    the (dd|dd), (ff|ff) and (ff|dd) classes primitive and with K = 5 on every
    shell (25 primitive pairs per side).  FP64 takes the parity bar
    1e-11 + 1e-10 |ref|; split takes the 1e-10 absolute bar (plus the same
    relative term, which only matters for elements above 1)."""
    basis, bra, ket, q = synth.split_batch(cls, K=K, seed=7, nq=nq, pool=16, npairs=8)
    ref = oracle_blocks(cls, basis, bra, ket, q, prec="d")
    f64 = gpu_list(cls, basis, bra, ket, q)
    e64 = assert_close(f64, ref, what=f"fp64 vs oracle {cls} K={K}")
    spl = gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_SPLIT)
    esp = assert_close(spl, ref, atol=1e-10, rtol=1e-10, what=f"split vs oracle {cls} K={K}")
    print(f"{cls} K={K}: max |fp64 - oracle| = {e64:.2e}, max |split - oracle| = {esp:.2e}, "
          f"max |oracle| = {np.abs(ref).max():.2e}")


@pytest.mark.parametrize("cls", [(2, 2, 2, 2), (3, 3, 3, 3), (3, 3, 2, 2)])
def test_k5_full_size_sample_against_oracle(cuda, cls):
    """K = 5 on every shell at the benchmark's pool sizes (512 shells per l,
    2048 pairs per side): FP64 and split over a batch of several thousand
    quartets, compared with the oracle on a seeded sample of them."""
    nq = {(2, 2, 2, 2): 4000, (3, 3, 3, 3): 600, (3, 3, 2, 2): 2000}[cls]
    basis, bra, ket, q = synth.split_batch(cls, K=5, seed=11, nq=nq)
    db = eri.DeviceBasis(basis)
    f64 = gpu_list(cls, basis, bra, ket, q, dbasis=db)
    spl = gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_SPLIT, dbasis=db)
    pick = np.sort(np.random.default_rng(3).choice(nq, 8, replace=False))
    ref = oracle_blocks(cls, basis, bra, ket, q[pick], prec="d")
    assert_close(f64[pick], ref, what=f"fp64 vs oracle {cls} K=5 sample")
    assert_close(spl[pick], ref, atol=1e-10, rtol=1e-10, what=f"split vs oracle {cls} K=5 sample")


@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 1, 0, 2), (2, 2, 1, 1)])
def test_split_low_l_contracted(cuda, cls):
    """The class-sweep inputs (K = 3) in split precision."""
    basis, pools = synth.class_sweep_pools(seed=4, pool=64, K=3)
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=4, npairs=100, nq=500)
    f64 = gpu_list(cls, basis, bra, ket, q)
    spl = gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_SPLIT)
    assert_close(spl, f64, atol=1e-10, rtol=0.0, what=f"split sweep {cls}")


def test_recursion_form_accuracy_guard(cuda):
    """The horizontal-recursion forms magnify rounding by about
    (2|A-B|)^l_b (2|C-D|)^l_d for pairs whose prefactor is not negligible.  On
    the high-l workload (exponents down to 0.05, centres up to 20 bohr apart)
    the library must refuse them, even when forced, and the FP64 result must
    stay at the parity bar against the oracle on a sample; on the class-sweep
    geometry a forced recursion form still runs."""
    cls = (3, 3, 2, 2)
    basis, bra, ket, q = synth.split_batch(cls, K=5, seed=0, nq=2000)
    db = eri.DeviceBasis(basis)
    try:
        eri.eri_set_forms(eri.ERI_FORM_HRR)
        got = gpu_list(cls, basis, bra, ket, q, dbasis=db)
        assert eri.eri_last_form()[1] is False
    finally:
        eri.eri_set_forms(0)
    sample = np.random.default_rng(1).choice(len(q), 24, replace=False)
    assert_close(got[sample], oracle_blocks(cls, basis, bra, ket, q[sample]), what="guarded (ff|dd) K=5")
    sbasis, pools = synth.class_sweep_pools(seed=0, pool=64, K=3)
    sbra, sket, sq = synth.class_sweep_batch(pools, (2, 2, 2, 2), seed=3, npairs=40, nq=50)
    try:
        eri.eri_set_forms(eri.ERI_FORM_HRR)
        gpu_list((2, 2, 2, 2), sbasis, sbra, sket, sq)
        assert eri.eri_last_form()[1] is True
    finally:
        eri.eri_set_forms(0)


@pytest.mark.parametrize("cls", [(3, 3, 3, 3), (3, 3, 3, 2)])
def test_split_packed_chains_mixed_contraction(cuda, cls):
    """The split ket stage on packed FP32 pairs (tiles that accumulate in
    memory: (ff|ff) and (ff|fd)) with contraction degrees 1 to 3 per shell,
    so that one batch holds pairs of 1 to 9 primitives: sorted tiles whose
    own ket count is below the batch's, odd and even counts (the zero partner
    of an odd last primitive), against the oracle at the split bar.  The
    tile shape reported afterwards is one of the two CTA widths."""
    rng = np.random.default_rng(31)
    shells, centres = [], []
    for i in range(12):
        l = cls[i % 4]
        K = 1 + (i // 4) % 3
        e = 10.0 ** rng.uniform(np.log10(0.05), np.log10(50.0), size=K)
        w = rng.uniform(0.5, 1.0, size=K)
        centres.append(rng.uniform(0.0, 4.0, size=3))
        shells.append((i, l, list(e), list(w * synth.norm_coef(e, l))))
    basis = synth.basis_from_shells(np.array(centres), shells)
    by_l = {l: [i for i, s in enumerate(shells) if s[1] == l] for l in set(cls)}
    pb = [(a, b) for a in by_l[cls[0]] for b in by_l[cls[1]]]
    pk = [(c, d) for c in by_l[cls[2]] for d in by_l[cls[3]]]
    bra = np.array([pb[i] for i in rng.choice(len(pb), 6, replace=False)], dtype=np.int32)
    ket = np.array([pk[i] for i in rng.choice(len(pk), 6, replace=False)], dtype=np.int32)
    q = np.array([(i, j) for i in range(len(bra)) for j in range(len(ket))][::3], dtype=np.int64)
    ref = oracle_blocks(cls, basis, bra, ket, q, prec="d")
    got = gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_SPLIT)
    assert_close(got, ref, atol=1e-10, what=f"split packed {cls}")
    assert eri.eri_last_tile()["threads"] in (256, 512)
    got64 = gpu_list(cls, basis, bra, ket, q)
    assert_close(got64, ref, what=f"fp64 {cls}")
