"""3-centre integrals (eri_batch3): (x|cd) with a Cartesian or real
solid-harmonic x, against the oracle (4-centre oracle with a unit second
bra function; the oracle's closed-form solid harmonics), element by element."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2506_12501_gb300 as eri
from gpu_helpers import THREADS, assert_close, nc

pytestmark = pytest.mark.gpu

CLASSES3 = [(lx, lc, ld) for lx in range(4) for lc, ld in ((0, 0), (1, 0), (1, 1), (2, 1), (2, 2))]


@pytest.fixture(scope="module")
def pools():
    return synth.three_centre_pools(seed=0, pool=64)


def gpu3(cls3, basis, x, ket, t, pure, precision=eri.ERI_PREC_FP64, db=None):
    lx, lc, ld = cls3
    db = db or eri.DeviceBasis(basis)
    out = eri.eri_batch3(lx, lc, ld, db, torch.as_tensor(x, device="cuda"), torch.as_tensor(ket, device="cuda"),
                         torch.as_tensor(t, device="cuda"), pure=pure, precision=precision)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(-1, len(t)).T  # [t][x*ncd + cd]


def ref3(cls3, basis, x, ket, t, pure):
    triples = np.stack([x[t[:, 0]], ket[t[:, 1], 0], ket[t[:, 1], 1]], axis=1)
    return oracle.solid.eri3(basis, triples, pure=pure, prec="d", threads=THREADS).reshape(len(t), -1)


@pytest.mark.parametrize("cls3", CLASSES3)
@pytest.mark.parametrize("pure", [True, False])
def test_three_centre_against_oracle(cuda, pools, cls3, pure):
    basis, orb, aux = pools
    L = sum(cls3)
    x, ket, t = synth.three_centre_batch(orb, aux, cls3, seed=1, nx=48, npairs=48, nt=211 if L <= 4 else 67)
    assert_close(gpu3(cls3, basis, x, ket, t, pure), ref3(cls3, basis, x, ket, t, pure), what=f"{cls3} pure={pure}")


@pytest.mark.parametrize("cls3", [(3, 2, 2), (2, 1, 0), (3, 0, 0), (1, 2, 1)])
def test_three_centre_both_orders_and_split(cuda, pools, cls3):
    """Either side transformed first (forced), and the split-precision transforms."""
    basis, orb, aux = pools
    x, ket, t = synth.three_centre_batch(orb, aux, cls3, seed=2, nx=32, npairs=32, nt=97)
    db = eri.DeviceBasis(basis)
    for pure in (True, False):
        ref = ref3(cls3, basis, x, ket, t, pure)
        try:
            for form in (0, 1):
                eri.eri_set_forms(1 << form)
                assert_close(gpu3(cls3, basis, x, ket, t, pure, db=db), ref, what=f"{cls3} pure={pure} form {form}")
                assert eri.eri_last_form() == (bool(form), False)
        finally:
            eri.eri_set_forms(0)
        spl = gpu3(cls3, basis, x, ket, t, pure, precision=eri.ERI_PREC_SPLIT, db=db)
        assert_close(spl, ref, atol=1e-10, what=f"{cls3} pure={pure} split")


def test_three_centre_product_form_and_errors(cuda, pools):
    basis, orb, aux = pools
    cls3 = (2, 1, 1)
    rng = np.random.default_rng(5)
    x = rng.choice(aux[2], 5).astype(np.int32)
    ket = np.stack([rng.choice(orb[1], 4), rng.choice(orb[1], 4)], axis=1).astype(np.int32)
    db = eri.DeviceBasis(basis)
    xd, kd = torch.as_tensor(x, device=cuda), torch.as_tensor(ket, device=cuda)
    out = eri.eri_batch3(2, 1, 1, db, xd, kd, None, pure=True).cpu().numpy()
    t = np.array([(i, k) for k in range(4) for i in range(5)], dtype=np.int64)
    ref = ref3(cls3, basis, x, ket, t, True).reshape(4, 5, 5, 9)   # [k][i][m][cd]
    assert_close(out.reshape(4, 9, 5, 5), ref.transpose(0, 3, 2, 1), what="product form")
    # an x shell of the wrong l, an index out of range, a short output
    with pytest.raises(eri.EriError) as ex:
        eri.eri_batch3(2, 1, 1, db, torch.as_tensor(aux[1][:5], device=cuda), kd, None)
    assert ex.value.code == eri.ERI_ECLASS
    with pytest.raises(eri.EriError) as ex:
        eri.eri_batch3(2, 1, 1, db, xd, kd, torch.as_tensor([[0, 9]], dtype=torch.int64, device=cuda))
    assert ex.value.code == eri.ERI_EINVAL
    with pytest.raises(eri.EriError):
        eri.eri_batch3(2, 1, 1, db, xd, kd, None, out=torch.empty(10, dtype=torch.float64, device=cuda))
    assert eri.eri_last_status() == eri.ERI_OK


def test_three_centre_full_size_sampled(cuda):
    """The measured workload size (2048 x shells, 2048 ket pairs, 1e5 triples,
    K = 3 orbital shells) for the heaviest class, in the launch configuration
    the benchmark times (timed form and tile choice); 48 sampled triples."""
    basis, orb, aux = synth.three_centre_pools(seed=0, pool=512)
    cls3 = (3, 2, 2)
    x, ket, t = synth.three_centre_batch(orb, aux, cls3, seed=0)
    db = eri.DeviceBasis(basis)
    out = eri.eri_batch3(3, 2, 2, db, torch.as_tensor(x, device=cuda), torch.as_tensor(ket, device=cuda),
                         torch.as_tensor(t, device=cuda), pure=True)
    torch.cuda.synchronize()
    nt = len(t)
    sample = np.random.default_rng(3).choice(nt, 48, replace=False)
    sample[:2] = [0, nt - 1]
    got = out.view(-1, nt)[:, torch.as_tensor(sample, device=cuda)].T.cpu().numpy()
    assert_close(got, ref3(cls3, basis, x, ket, t[sample], True), what="full (fd|dd)")
    assert torch.isfinite(out).all()
