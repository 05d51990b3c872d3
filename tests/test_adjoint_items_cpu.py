"""The adjoint's channel items (Section 2.1 derivatives of a primitive
Gaussian): the (ab, p') pairs with non-zero weight in some channel, and the
channels each kind of item can reach, checked on the oracle's one-dimensional
Hermite expansion coefficients (Eqs. E2rr1/E2rr2) for random primitive pairs.

With E_i = E^{a_i b_i}_{t_i} per axis, the bra channels of (ab, p') are
  d/dA_i:    (2 z_a E^{a+1_i,b} - a_i E^{a-1_i,b})_{t_i} E_j E_k
  d/dB_i:    (2 z_b E^{a,b+1_i} - b_i E^{a,b-1_i})_{t_i} E_j E_k
  d/dz_a:    -sum_i E^{a+2_i,b}_{t_i} E_j E_k   (z_b likewise)
The library visits only the pairs with t_i <= a_i + b_i on all axes but at
most one, which may exceed it by 1 (then only the channels A_i, B_i, z_a,
z_b are non-zero) or by 2 (only z_a, z_b); every one of them carries some
weight for a generic geometry."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2506_12501_gb300 import opcount


def herm(N):
    return [(t, u, n - t - u) for n in range(N + 1) for t in range(n, -1, -1) for u in range(n - t, -1, -1)]


def channel_weights(la, lb, za, zb, A, B):
    """{(ab, p'): 8 channel weights} over every component pair and every
    Hermite function of order <= la + lb + 2."""
    E = [np.asarray(oracle.hermite_E(la + 2, lb + 2, za, zb, A[x], B[x], prec="d"), dtype=np.float64)
         for x in range(3)]

    def e(x, i, j, t):
        if i < 0 or j < 0 or t > i + j:
            return 0.0
        return E[x][i, j, t]

    out = {}
    ca, cb = oracle.cart_components(la), oracle.cart_components(lb)
    for ia, a in enumerate(ca):
        for ib, b in enumerate(cb):
            for p in herm(la + lb + 2):
                base = [e(x, a[x], b[x], p[x]) for x in range(3)]
                w = np.zeros(8)
                for x in range(3):
                    rest = np.prod([base[y] for y in range(3) if y != x])
                    w[x] = (2 * za * e(x, a[x] + 1, b[x], p[x]) - a[x] * e(x, a[x] - 1, b[x], p[x])) * rest
                    w[3 + x] = (2 * zb * e(x, a[x], b[x] + 1, p[x]) - b[x] * e(x, a[x], b[x] - 1, p[x])) * rest
                    w[6] -= e(x, a[x] + 2, b[x], p[x]) * rest
                    w[7] -= e(x, a[x], b[x] + 2, p[x]) * rest
                out[(ia * len(cb) + ib, p)] = (a, b, w)
    return out


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (1, 1), (2, 1), (2, 2), (3, 1)])
def test_channel_items_cover_every_nonzero_weight(la, lb):
    rng = np.random.default_rng([la, lb])
    counts = None
    for _ in range(3):
        za, zb = 10 ** rng.uniform(-1, 1, 2)
        A, B = rng.uniform(-1.5, 1.5, 3), rng.uniform(-1.5, 1.5, 3)
        n = [0, 0, 0]
        for (ab, p), (a, b, w) in channel_weights(la, lb, za, zb, A, B).items():
            over = [p[x] - a[x] - b[x] for x in range(3)]
            item = max(over) <= 2 and sum(1 for o in over if o > 0) <= 1
            if not item:
                assert np.all(w == 0.0), (ab, p, w)
                continue
            kind = max(0, max(over))
            n[kind] += 1
            assert np.any(w != 0.0), (ab, p)  # no item is dead weight for a generic geometry
            if kind > 0:
                i = int(np.argmax(over))
                live = {i, 3 + i, 6, 7} if kind == 1 else {6, 7}
                for c in range(8):
                    if c not in live:
                        assert w[c] == 0.0, (ab, p, c, w)
        counts = tuple(n)
    assert counts == opcount.grad_item_kinds(la, lb)
