"""The term counts behind the benchmark's operation counts (and so its
roofline fractions), checked against the oracle's Hermite expansion
coefficients (Eqs. E2rr1/E2rr2) for a generic geometry: a term is a
(Cartesian pair, Hermite function) whose product of one-dimensional
coefficients is non-zero."""
import numpy as np
import pytest

import oracle
from paper_2506_12501_gb300 import opcount


def hermite_functions(L):
    return [(t, u, v) for t in range(L + 1) for u in range(L + 1 - t) for v in range(L + 1 - t - u)]


@pytest.mark.parametrize("L", range(0, 11))
def test_hermite_function_counts(L):
    assert opcount.nh(L) == len(hermite_functions(L))
    assert sorted(opcount._herm(L)) == sorted(hermite_functions(L))


def axis_tables(l1, l2, seed):
    rng = np.random.default_rng(seed)
    za, zb = 10 ** rng.uniform(-1, 1, 2)
    A, B = rng.uniform(-2, 2, 3), rng.uniform(-2, 2, 3)
    return [np.asarray(oracle.hermite_E(l1, l2, za, zb, A[x], B[x], prec="d"), dtype=np.float64) for x in range(3)]


@pytest.mark.parametrize("l1,l2", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 2), (3, 3)])
def test_sparse_terms_of_a_pair(l1, l2):
    """opcount.terms: the non-zero products E^x E^y E^z over every component
    pair (a, b) and Hermite function of order <= l1 + l2."""
    E = axis_tables(l1, l2, seed=[l1, l2])
    n = 0
    for a in oracle.cart_components(l1):
        for b in oracle.cart_components(l2):
            for p in hermite_functions(l1 + l2):
                if all(p[i] <= a[i] + b[i] for i in range(3)):  # beyond, the table holds no entry
                    n += np.prod([E[i][a[i], b[i], p[i]] for i in range(3)]) != 0.0
    assert n == opcount.terms(l1, l2)


@pytest.mark.parametrize("l1,l2", [(0, 0), (1, 0), (1, 1), (2, 1), (2, 2), (3, 3)])
def test_sparse_terms_of_the_recursion_form(l1, l2):
    """opcount.terms_hrr: the non-zero products of E_{e,0} over the functions e
    with l1 <= |e| <= l1 + l2 (one centre's polynomial about the pair's)."""
    L = l1 + l2
    E = axis_tables(L, 0, seed=[l1, l2, 1])
    n = 0
    for l in range(l1, l1 + l2 + 1):
        for e in oracle.cart_components(l):
            for p in hermite_functions(L):
                if all(p[i] <= e[i] for i in range(3)):
                    n += np.prod([E[i][e[i], 0, p[i]] for i in range(3)]) != 0.0
    assert n == opcount.terms_hrr(l1, l2)
    assert opcount.ncols_hrr(l1, l2) == sum(opcount.nc(l) for l in range(l1, l1 + l2 + 1))


@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 2, 2), (2, 1, 0, 0), (3, 3, 3, 3)])
def test_sparse_count_below_dense(cls):
    """The sparse sequence skips work; it never exceeds the dense formulation
    by more than the per-primitive setup the dense figure books as 50."""
    for K in (1, 9):
        s = opcount.sparse_flops(cls, K, K)
        d = opcount.dense_flops(cls, K, K)
        assert s > 0 and d > 0
        if sum(cls) >= 4:
            assert s < d
