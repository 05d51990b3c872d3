"""Parity of the CUDA forward path (eri_boys, eri_batch) against the CPU
oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import assert_close, gpu_list, oracle_blocks, nc, to_device

pytestmark = pytest.mark.gpu


def test_boys_kernel_against_oracle(cuda):
    """Boys function over the tabulated range, across the grid end (T = 320)
    and far beyond, every order up to ERI_BOYS_MMAX; relative error below
    (2 + 0.3 m) 1e-15 (the recursions add about one rounding per order).
    The arguments include grid points, the midpoints between them (where the
    grid index is decided by a truncated float image of T), tiny and
    subnormal T."""
    rng = np.random.default_rng(0)
    grid = np.arange(0, 320 * 32 + 1) / 32.0
    mids = grid[:-1] + 1.0 / 64
    T = np.concatenate([np.linspace(0.0, 320.5, 4001), rng.uniform(0, 320, 4000), [319.999, 320.0, 320.0001],
                        grid[::7], mids[::5], np.nextafter(mids[::11], 0), np.nextafter(mids[::13], 1e9),
                        np.geomspace(1e-12, 1e5, 500), [0.0, 5e-324, 1e-310, 1e-300]])
    for mmax in (0, 1, 4, 8, 12, 16, 20):
        got = eri.eri_boys(mmax, torch.as_tensor(T, device=cuda)).cpu().numpy()
        ref = oracle.boys(mmax, T, prec="ld").astype(np.float64)
        rel = np.abs(got - ref) / ref
        assert rel.max() < 2e-15 + 3e-16 * mmax, (mmax, rel.max(), T[np.argmax(rel.max(axis=1))])


def test_boys_edge_cases(cuda):
    assert eri.eri_boys(3, torch.zeros(0, dtype=torch.float64, device=cuda)).numel() == 0
    with pytest.raises(eri.EriError):
        eri.eri_boys(eri.ERI_BOYS_MMAX + 1, torch.ones(4, dtype=torch.float64, device=cuda))
    F = eri.eri_boys(5, torch.zeros(1, dtype=torch.float64, device=cuda)).cpu().numpy()[0]
    assert np.allclose(F * (2 * np.arange(6) + 1), 1.0, rtol=1e-15, atol=0)


def test_pp_pp_primitive_full(cuda):
    """All 1000 quartets of the primitive (pp|pp) workload (K = 1, exponents
    log-uniform in [0.1, 10], centres in a 10-bohr cube) against the
    long-double oracle."""
    basis, bra, ket, q = synth.config1_pp_primitive(seed=0, nq=1000)
    got = gpu_list((1, 1, 1, 1), basis, bra, ket, q)
    ref = oracle_blocks((1, 1, 1, 1), basis, bra, ket, q, prec="ld")
    assert_close(got, ref, what="(pp|pp) K=1")


@pytest.fixture(scope="module")
def sweep_pools():
    return synth.class_sweep_pools(seed=0, pool=96, K=3)


@pytest.mark.parametrize("cls", synth.all_classes(2))
def test_class_sweep_contracted(cuda, sweep_pools, cls):
    """Every (la lb|lc ld) class with l <= 2, K = 3 per shell (9 x 9 primitive
    quartets), even-tempered exponents: several tiles plus a ragged tail."""
    basis, pools = sweep_pools
    L = sum(cls)
    nq = 389 if L <= 3 else (131 if L <= 5 else 37)
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=1, npairs=160, nq=nq)
    got = gpu_list(cls, basis, bra, ket, q)
    ref = oracle_blocks(cls, basis, bra, ket, q, prec="d")
    assert_close(got, ref, what=str(cls))


@pytest.mark.parametrize("cls", synth.all_classes(2))
def test_every_form_against_oracle(cuda, sweep_pools, cls):
    """Each of the four forms (plain or side-swapped; full Cartesian pairs or
    (e0|f0) plus horizontal recursions), forced with eri_set_forms, against
    the oracle on the same contracted batch."""
    basis, pools = synth.class_sweep_pools(seed=7, pool=48, K=2)
    L = sum(cls)
    nq = 97 if L <= 4 else 29
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=8, npairs=40, nq=nq)
    ref = oracle_blocks(cls, basis, bra, ket, q, prec="d")
    db = eri.DeviceBasis(basis)
    try:
        for form in range(4):
            eri.eri_set_forms(1 << form)
            got = gpu_list(cls, basis, bra, ket, q, dbasis=db)
            assert eri.eri_last_form() == (bool(form & 1), bool(form & 2))
            assert_close(got, ref, what=f"{cls} form {form}")
    finally:
        eri.eri_set_forms(0)


@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 0, 1, 0), (2, 1, 1, 0), (2, 2, 2, 2)])
def test_product_form_layout(cuda, cls):
    """quartets == NULL: every (bra, ket) combination, written in the
    [ij, ab, cd, kl] column-major layout."""
    basis, pools = synth.class_sweep_pools(seed=2, pool=32, K=2)
    bra, ket, _ = synth.class_sweep_batch(pools, cls, seed=3, npairs=1, nq=1)
    rng = np.random.default_rng(4)
    nbra, nket = (7, 5) if sum(cls) < 8 else (3, 2)
    bra = np.stack([rng.choice(pools[cls[0]], nbra), rng.choice(pools[cls[1]], nbra)], 1).astype(np.int32)
    ket = np.stack([rng.choice(pools[cls[2]], nket), rng.choice(pools[cls[3]], nket)], 1).astype(np.int32)
    db = eri.DeviceBasis(basis)
    b, k, _ = to_device(bra, ket)
    out = eri.eri_batch(cls, db, b, k, None).cpu().numpy()
    nab, ncd = nc(cls[0]) * nc(cls[1]), nc(cls[2]) * nc(cls[3])
    got = out.reshape(nket, ncd, nab, nbra)  # [kl][cd][ab][ij] (C order of the column-major layout)
    q = np.array([(i, j) for j in range(nket) for i in range(nbra)], dtype=np.int64)
    ref = oracle_blocks(cls, basis, bra, ket, q).reshape(nket, nbra, nab, ncd)
    assert_close(got, ref.transpose(0, 3, 2, 1), what=f"product {cls}")


def test_mixed_contraction_degrees(cuda):
    """Shells with K = 6, 3 and 1 in one batch (molecule-shaped basis)."""
    basis = synth.molecule_basis(natom=6, radius=3.0, seed=1)
    s_shells = np.where(basis.shell_l == 0)[0].astype(np.int32)
    p_shells = np.where(basis.shell_l == 1)[0].astype(np.int32)
    rng = np.random.default_rng(9)
    for cls, A, B in [((0, 0, 0, 0), s_shells, s_shells), ((1, 0, 1, 0), p_shells, s_shells),
                      ((1, 1, 0, 0), p_shells, p_shells)]:
        bra = np.stack([rng.choice(A, 40), rng.choice(B, 40)], 1).astype(np.int32)
        ket = np.stack([rng.choice(p_shells if cls[2] else s_shells, 40),
                        rng.choice(p_shells if cls[3] else s_shells, 40)], 1).astype(np.int32)
        q = np.stack([rng.integers(0, 40, 150), rng.integers(0, 40, 150)], 1).astype(np.int64)
        got = gpu_list(cls, basis, bra, ket, q)
        ref = oracle_blocks(cls, basis, bra, ket, q)
        assert_close(got, ref, what=f"mixed K {cls}")


@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 0, 1, 0), (1, 1, 1, 0), (2, 0, 1, 1), (2, 1, 0, 0)])
def test_mixed_degrees_sorted_batches(cuda, cls):
    """Batches mixing K = 6, 3 and 1 run their quartets sorted by the
    primitive-pair counts, each tile looping to its own largest: the list form
    (every form forced in turn, and the split precision), the product form,
    and a batch large enough for the tile tuner, checked on a sample."""
    basis = synth.molecule_basis(natom=6, radius=3.0, seed=2)
    by_l = {l: np.where(basis.shell_l == l)[0].astype(np.int32) for l in range(3)}
    rng = np.random.default_rng([11, *cls])
    bra = np.stack([rng.choice(by_l[cls[0]], 30), rng.choice(by_l[cls[1]], 30)], 1).astype(np.int32)
    ket = np.stack([rng.choice(by_l[cls[2]], 25), rng.choice(by_l[cls[3]], 25)], 1).astype(np.int32)
    q = np.stack([rng.integers(0, 30, 300), rng.integers(0, 25, 300)], 1).astype(np.int64)
    ref = oracle_blocks(cls, basis, bra, ket, q)
    db = eri.DeviceBasis(basis)
    try:
        for form in range(4):
            eri.eri_set_forms(1 << form)
            assert_close(gpu_list(cls, basis, bra, ket, q, dbasis=db), ref, what=f"mixed K {cls} form {form}")
    finally:
        eri.eri_set_forms(0)
    assert_close(gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_SPLIT, dbasis=db), ref,
                 what=f"mixed K split {cls}")
    # product form: [kl][cd][ab][ij]
    nb, nk = 12, 9
    b, k, _ = to_device(bra[:nb], ket[:nk])
    out = eri.eri_batch(cls, db, b, k, None).cpu().numpy()
    nab, ncd = nc(cls[0]) * nc(cls[1]), nc(cls[2]) * nc(cls[3])
    qp = np.array([(i, j) for j in range(nk) for i in range(nb)], dtype=np.int64)
    refp = oracle_blocks(cls, basis, bra[:nb], ket[:nk], qp).reshape(nk, nb, nab, ncd)
    assert_close(out.reshape(nk, ncd, nab, nb), refp.transpose(0, 3, 2, 1), what=f"mixed K product {cls}")
    # a tuned batch: 2e4 quartets, a sample of 200 against the oracle
    qb = np.stack([rng.integers(0, 30, 20000), rng.integers(0, 25, 20000)], 1).astype(np.int64)
    big = gpu_list(cls, basis, bra, ket, qb, dbasis=db)
    pick = rng.choice(20000, 200, replace=False)
    assert_close(big[pick], oracle_blocks(cls, basis, bra, ket, qb[pick]), what=f"mixed K tuned {cls}")


def test_bra_ket_swap_symmetry(cuda):
    """(ab|cd) = (cd|ab): the GPU result of class (2,1|1,0) equals the
    transposed result of class (1,0|2,1) on swapped lists."""
    basis, pools = synth.class_sweep_pools(seed=5, pool=32, K=2)
    bra, ket, q = synth.class_sweep_batch(pools, (2, 1, 1, 0), seed=6, npairs=50, nq=200)
    g1 = gpu_list((2, 1, 1, 0), basis, bra, ket, q)
    g2 = gpu_list((1, 0, 2, 1), basis, ket, bra, q[:, ::-1].copy())
    g2 = g2.reshape(-1, 3, 18).transpose(0, 2, 1).reshape(-1, 54)
    assert_close(g1, g2, atol=1e-13, rtol=1e-12, what="swap")


def test_errors_and_degenerate_sizes(cuda):
    basis, pools = synth.class_sweep_pools(seed=0, pool=8, K=2)
    db = eri.DeviceBasis(basis)
    bra, ket, q = synth.class_sweep_batch(pools, (1, 0, 1, 0), seed=0, npairs=4, nq=6)
    b, k, qq = to_device(bra, ket, q)
    # class mismatch
    with pytest.raises(eri.EriError) as e:
        eri.eri_batch((1, 1, 1, 0), db, b, k, qq)
    assert e.value.code == eri.ERI_ECLASS
    # index out of range
    bad = qq.clone()
    bad[2, 1] = 99
    with pytest.raises(eri.EriError) as e:
        eri.eri_batch((1, 0, 1, 0), db, b, k, bad)
    assert e.value.code == eri.ERI_EINVAL
    # l beyond ERI_LMAX
    with pytest.raises(eri.EriError):
        eri.eri_batch((4, 0, 0, 0), db, b, k, qq)
    # output too short
    with pytest.raises(eri.EriError):
        eri.eri_batch((1, 0, 1, 0), db, b, k, qq, out=torch.empty(5, dtype=torch.float64, device=cuda))
    # empty batch: no-op
    out = torch.full((3,), 7.0, dtype=torch.float64, device=cuda)
    eri.eri_batch((1, 0, 1, 0), db, b, k, qq[:0], out=out)
    assert torch.all(out == 7.0)
    # a single quartet
    got = gpu_list((1, 0, 1, 0), basis, bra, ket, q[:1])
    assert_close(got, oracle_blocks((1, 0, 1, 0), basis, bra, ket, q[:1]), what="nq=1")
    # contraction degree beyond ERI_KMAX
    b2 = basis.copy()
    b2.shell_K = b2.shell_K.copy()
    b2.shell_K[bra[0, 0]] = eri.ERI_KMAX + 1
    with pytest.raises(eri.EriError) as e:
        eri.eri_batch((1, 0, 1, 0), eri.DeviceBasis(b2), b, k, qq)
    assert e.value.code == eri.ERI_EINVAL
    assert eri.eri_last_status() == eri.ERI_OK


@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 1, 2, 0), (2, 0, 1, 2), (1, 1, 1, 2), (2, 2, 2, 2)])
def test_full_size_sampled(cuda, cls):
    """The class-sweep workload at full size (1e5 quartets per class, pools of
    512 shells, 2048 pairs per side, K = 3), in the launch configuration the
    benchmark times (the first call times the cheapest plain and recursion
    forms and remembers the faster); 48 sampled quartets against the oracle,
    and a second call runs the remembered form and tile with identical results."""
    basis, pools = synth.class_sweep_pools(seed=0, pool=512, K=3)
    bra, ket, q = synth.class_sweep_batch(pools, cls, seed=0, npairs=2048, nq=100_000)
    db = eri.DeviceBasis(basis)
    b, k, qq = to_device(bra, ket, q)
    out = eri.eri_batch(cls, db, b, k, qq)
    torch.cuda.synchronize()
    nq = q.shape[0]
    sample = np.random.default_rng(11).choice(nq, 48, replace=False)
    sample[:2] = [0, nq - 1]
    got = out.view(-1, nq)[:, torch.as_tensor(sample, device=cuda)].T.cpu().numpy()
    ref = oracle_blocks(cls, basis, bra, ket, q[sample])
    assert_close(got, ref, what=f"full {cls}")
    assert torch.isfinite(out).all()
    form = eri.eri_last_form()
    out2 = eri.eri_batch(cls, db, b, k, qq)
    assert eri.eri_last_form() == form
    assert torch.equal(out, out2)


@pytest.mark.parametrize("cls,K", [((3, 3, 3, 1), 8), ((3, 3, 3, 2), 7), ((3, 3, 3, 3), 6)])
def test_contraction_degree_limits(cuda, cls, K):
    """The largest contraction degrees eri_batch accepts with the same K on all
    four shells (K = 8 up to L = 10, K = 7 at L = 11, K = 6 at L = 12) run in
    FP64 and in split precision and match the oracle; one more primitive per
    shell is refused with ERI_EINVAL (no tile holds it, or K > ERI_KMAX)."""
    basis, bra, ket, q = synth.small_random_batch(cls, K=(K,) * 4, nq=2, seed=5)
    ref = oracle_blocks(cls, basis, bra, ket, q, prec="d")
    assert_close(gpu_list(cls, basis, bra, ket, q), ref, what=f"fp64 {cls} K={K}")
    assert_close(gpu_list(cls, basis, bra, ket, q, precision=eri.ERI_PREC_SPLIT), ref, atol=1e-10, rtol=1e-10,
                 what=f"split {cls} K={K}")
    basis, bra, ket, q = synth.small_random_batch(cls, K=(K + 1,) * 4, nq=2, seed=5)
    for prec in (eri.ERI_PREC_FP64, eri.ERI_PREC_SPLIT):
        with pytest.raises(eri.EriError) as e:
            gpu_list(cls, basis, bra, ket, q, precision=prec)
        assert e.value.code == eri.ERI_EINVAL
