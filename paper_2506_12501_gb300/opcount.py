"""Operation counts of one contracted quartet (host-side bookkeeping for the
benchmark's roofline; no integral arithmetic).

``sparse_flops`` counts the FP64 floating-point operations the library's
forward path performs (FMA = 2, MUL/ADD = 1, one square root and one
division counted for the reciprocal square root): the MD sequence of
Eq. md-2body with the structural zeros of the Hermite expansion coefficients
skipped.  ``dense_flops`` is the dense-GEMM formulation of the same sequence
(every Hermite pair of a class taken as nonzero, Boys and prefactor as a
nominal 50), the per-quartet figure used in the measurement plan.
"""
from __future__ import annotations

import math


def nh(l: int) -> int:
    return (l + 1) * (l + 2) * (l + 3) // 6


def nc(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def carts(l: int):
    return [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]


def terms(l1: int, l2: int) -> int:
    """number of nonzero (Cartesian pair, Hermite function) terms of E"""
    return sum(math.prod(a[i] + b[i] + 1 for i in range(3)) for a in carts(l1) for b in carts(l2))


def _herm(L):
    out = []
    for N in range(L + 1):
        for t in range(N, -1, -1):
            for u in range(N - t, -1, -1):
                out.append((t, u, N - t - u))
    return out


def r_recursion_flops(L: int) -> int:
    """FP64 operations of the in-place auxiliary recursion (Eq. r-rr):
    a multiply per entry and level, plus an FMA where the coefficient
    r_i - 1 of the chosen axis is nonzero (axis with r_i = 1 preferred)."""
    H = _herm(L)
    cost = []
    for (t, u, v) in H:
        r = (t, u, v)
        if max(r) == 0:
            cost.append(0)
            continue
        if 1 in r:
            cost.append(1)
        else:
            cost.append(3)
    total = 0
    for n in range(L - 1, -1, -1):
        total += sum(cost[1:nh(L - n)])
    return total


def prim_quartet_flops(L: int) -> int:
    """setup (rho, T, prefactor: 15 + rsqrt counted as 2), Boys (Taylor 12;
    for L > 0 also exp(-T) 13, 2T 1 and the downward recursion, 3 per
    order), scaling 2 per order, recursion"""
    boys = 12 + (14 + 3 * L if L > 0 else 0)
    return 17 + boys + 2 * (L + 1) + r_recursion_flops(L)


def terms_hrr(l1: int, l2: int) -> int:
    """nonzero terms of E_{e,0} over the functions e with l1 <= |e| <= l1 + l2"""
    return sum(math.prod(e[i] + 1 for i in range(3)) for l in range(l1, l1 + l2 + 1) for e in carts(l))


def ncols_hrr(l1: int, l2: int) -> int:
    return sum(nc(l) for l in range(l1, l1 + l2 + 1))


def hrr_steps(l1: int, l2: int) -> int:
    """FMA steps of the horizontal recursion building (l1 l2| from (e0|"""
    return sum(nc(j) * sum(nc(l) for l in range(l1, l1 + l2 - j + 1)) for j in range(1, l2 + 1))


def _form(cls, hrr: bool):
    """(rows, cols, bra terms, ket terms, HRR FMAs per quartet) of one form"""
    la, lb, lc, ld = cls
    if not hrr:
        return nc(la) * nc(lb), nc(lc) * nc(ld), terms(la, lb), terms(lc, ld), 0
    rows, cols = ncols_hrr(la, lb), ncols_hrr(lc, ld)
    return rows, cols, terms_hrr(la, lb), terms_hrr(lc, ld), rows * hrr_steps(lc, ld) + nc(lc) * nc(ld) * hrr_steps(la, lb)


def choice(cls, Kbra: int, Kket: int, allow_hrr: bool = True):
    """The library's modelled choice of form for eri_batch (before any timing
    of forms): (swapped, hrr), the cheapest by the same cost model (transform terms, half an operation per R entry,
    the recursions), the horizontal-recursion form only when its (f0|e0)
    accumulators fit (rows * cols <= 4096)."""
    best, best_cost = None, None
    for o in range(4 if allow_hrr else 2):
        sw, hrr = bool(o & 1), o >= 2
        c = (cls[2], cls[3], cls[0], cls[1]) if sw else cls
        kb, kk = (Kket, Kbra) if sw else (Kbra, Kket)
        rows, cols, tb, tk, hs = _form(c, hrr)
        if hrr and rows * cols > 4096:
            continue
        L = sum(c)
        cost = kb * kk * (nh(c[0] + c[1]) * tk + 0.5 * nh(L)) + kb * cols * tb + hs
        if best is None or cost < best_cost:
            best, best_cost = (sw, hrr), cost
    return best


def swapped(cls, Kbra: int, Kket: int) -> bool:
    return choice(cls, Kbra, Kket)[0]


def sparse_flops(cls, Kbra: int, Kket: int, orient: str = "auto", allow_hrr: bool = True, form=None) -> int:
    """FP64 flops of one form: `form` = (swapped, hrr) as the library reports
    it (eri_last_form), else the modelled choice (orient='auto'), else the
    ket-first plain form (orient='as-is')."""
    if form is not None:
        sw, hrr = bool(form[0]), bool(form[1])
    else:
        sw, hrr = choice(cls, Kbra, Kket, allow_hrr) if orient == "auto" else (False, False)
    if sw:
        cls = (cls[2], cls[3], cls[0], cls[1])
        Kbra, Kket = Kket, Kbra
    la, lb, lc, ld = cls
    L = la + lb + lc + ld
    rows, cols, tb, tk, hs = _form(cls, hrr)
    ket = 2 * nh(la + lb) * tk                       # per primitive quartet
    bra = 2 * cols * tb                              # per bra primitive (each chain starts from the accumulator)
    return Kbra * Kket * (prim_quartet_flops(L) + ket) + Kbra * bra + 2 * hs


def dense_flops(cls, Kbra: int, Kket: int) -> int:
    la, lb, lc, ld = cls
    L = la + lb + lc + ld
    ncd = nc(lc) * nc(ld)
    per_prim = 50 + 3 * (math.comb(L + 4, 4) - (L + 1)) + 2 * nh(la + lb) * nh(lc + ld) * ncd
    return Kbra * Kket * per_prim + Kbra * 2 * nh(la + lb) * nc(la) * nc(lb) * ncd


def sparse_flops3(cls3, Kx: int, Kket: int, pure: bool, swapped: bool, pure_terms: int = 0) -> int:
    """FP64 flops of one 3-centre triple (x|cd) = (x 1|cd), 1 the unit
    function, in the form the library ran: swapped = False transforms the cd
    ket first over the x side's Hermite functions (only those of order lx for
    a solid-harmonic x), swapped = True transforms x first.  pure_terms: the
    number of nonzero Cartesian coefficients of the lx solid harmonics."""
    lx, lc, ld = cls3
    L = lx + lc + ld
    tx = pure_terms if pure else terms(lx, 0)
    nx = 2 * lx + 1 if pure else nc(lx)
    tcd, ncd = terms(lc, ld), nc(lc) * nc(ld)
    if not swapped:
        kb, kk = Kx, Kket
        ket = 2 * (nc(lx) if pure else nh(lx)) * tcd
        bra = 2 * ncd * tx
    else:
        kb, kk = Kket, Kx
        ket = 2 * nh(lc + ld) * tx
        bra = 2 * nx * tcd
    return kb * kk * (prim_quartet_flops(L) + ket) + kb * bra


def grad_item_kinds(la: int, lb: int):
    """Channel items of a bra class by kind: the (ab, p') pairs, p' = (t, u, v)
    of order <= la + lb + 2, with t_i <= a_i + b_i on all axes but at most one,
    which may exceed it by 1 or 2 (every other pair has zero weight in all
    8 channels, the one-dimensional E^{ij}_t vanishing for t > i + j).
    Returns (within on every axis, above by 1 on one axis, above by 2)."""
    n = [0, 0, 0]
    for a in carts(la):
        for b in carts(lb):
            for N in range(la + lb + 3):
                for t in range(N, -1, -1):
                    for u in range(N - t, -1, -1):
                        over = [h - a[i] - b[i] for i, h in enumerate((t, u, N - t - u))]
                        if max(over) <= 2 and sum(1 for e in over if e > 0) <= 1:
                            n[max(0, max(over))] += 1
    return tuple(n)


def grad_items(la: int, lb: int) -> int:
    """All channel items of a bra class (see grad_item_kinds)."""
    return sum(grad_item_kinds(la, lb))


def _grad_launch_flops(cls, Kbra: int, Kket: int, vform: int = 0) -> int:
    """FP64 flops of one adjoint launch (the channels of the kernel's bra):
    per primitive quartet the auxiliary integrals to order L+2; per bra
    primitive the derived per-axis tables (3 (la+1)(lb+1)(la+lb+3) entries,
    6 flops each) and, per channel item, T[ab][p'] and the channel terms: all
    8 (5 multiplies and 12 FMAs, 29 flops), or, for an item above a_i + b_i on
    one axis, the 4 (2 multiplies and 4 FMAs, 10 flops) or 2 (6 flops) with
    non-zero weight.  T comes from
      the X form (vform 0): per primitive quartet the ket transform over the
        raised bra Hermite range, then 2 ncd per channel item;
      the V form (vform 1): per quartet and ket primitive V[ab][q] (2 nab Tcd),
        then 2 Nh(lc+ld) per channel item and ket primitive."""
    la, lb, lc, ld = cls
    L = la + lb + lc + ld
    nhb2 = nh(la + lb + 2)
    ncd = nc(lc) * nc(ld)
    nab = nc(la) * nc(lb)
    n0, n1, n2 = grad_item_kinds(la, lb)
    nit = n0 + n1 + n2
    nd = (la + 1) * (lb + 1) * (la + lb + 3)
    channels = 18 * nd + 29 * n0 + 10 * n1 + 6 * n2
    if vform:
        return Kbra * Kket * prim_quartet_flops(L + 2) + Kket * 2 * nab * terms(lc, ld) + \
            Kbra * (channels + nit * 2 * nh(lc + ld) * Kket)
    return Kbra * Kket * (prim_quartet_flops(L + 2) + 2 * nhb2 * terms(lc, ld)) + \
        Kbra * (channels + nit * 2 * ncd)


def _grad_ket_flops(cls, Kbra: int, Kket: int) -> int:
    """FP64 flops of the ket channels in the single launch (eri_last_grad_forms
    reports ERI_GRAD_ONE): per primitive quartet Y'[ab][q'] over the raised
    ket range (2 Nh(lc+ld+2) Tab); per ket primitive the derived tables
    (18 (lc+1)(ld+1)(lc+ld+3)) and, per ket channel item, T (2 nab) and its
    channel terms (29, 10 or 6 flops by kind)."""
    la, lb, lc, ld = cls
    nab = nc(la) * nc(lb)
    n0, n1, n2 = grad_item_kinds(lc, ld)
    nd = (lc + 1) * (ld + 1) * (lc + ld + 3)
    per_k = 18 * nd + 29 * n0 + 10 * n1 + 6 * n2 + (n0 + n1 + n2) * 2 * nab
    return Kbra * Kket * 2 * nh(lc + ld + 2) * terms(la, lb) + Kket * per_k


def grad_flops(cls, Kbra: int, Kket: int, forms=(0, 0)) -> int:
    """FP64 flops of the adjoint of one quartet in the forms of
    eri_last_grad_forms: the bra channels in form forms[0]; the ket channels
    either from the same launch (forms[1] = 2, ERI_GRAD_ONE: the auxiliary
    integrals are computed once; 4, ERI_GRAD_ONE_SWAPPED: the same with the
    sides exchanged, forms[0] then being the form of the ket's channels) or
    from a second launch with the sides exchanged, in form forms[1]."""
    la, lb, lc, ld = cls
    if forms[1] == 2:
        return _grad_launch_flops(cls, Kbra, Kket, forms[0]) + _grad_ket_flops(cls, Kbra, Kket)
    if forms[1] == 4:  # ERI_GRAD_ONE_SWAPPED: the single launch with the sides exchanged
        sw = (lc, ld, la, lb)
        return _grad_launch_flops(sw, Kket, Kbra, forms[0]) + _grad_ket_flops(sw, Kket, Kbra)
    return _grad_launch_flops(cls, Kbra, Kket, forms[0]) + _grad_launch_flops((lc, ld, la, lb), Kket, Kbra, forms[1])
