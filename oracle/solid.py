"""TEST INFRASTRUCTURE ONLY: real solid harmonics as Cartesian polynomials,
and the 3-centre integrals the library's eri_batch3 computes.

Solid harmonics.  S_lm(x, y, z), m = -l..l, are the real regular solid
harmonics with Racah normalisation: S_l0(0, 0, 1) = 1, and over the unit
sphere  int S_lm S_lm' dOmega = 4 pi / (2l + 1) delta_mm'.  S_lm for m > 0
goes as cos(m phi) and for m < 0 as sin(|m| phi), with positive coefficients
of x^|m| z^(l-|m|) and x^(|m|-1) y z^(l-|m|) respectively.  The polynomial
coefficients come from the closed form of these functions as a triple sum
over monomials x^(2t+|m|-2(u+v)) y^(2(u+v)) z^(l-2t-|m|):

    S_lm = N_lm sum_t sum_u sum_v (-1)^(t+v-v_m) 4^-t C(l,t) C(l-t,|m|+t) C(t,u) C(|m|,2v)
    N_lm = sqrt(2 (l+|m|)! (l-|m|)! / 2^delta_m0) / (2^|m| l!),

with t = 0..floor((l-|m|)/2), u = 0..t, and 2v running over the even
(m >= 0, v_m = 0) or odd (m < 0, v_m = 1/2) integers up to |m|.  The paper
uses such Cartesian-to-solid coefficients for its H matrices (Section 2.1,
Eqs. solid2herm-1 and -2) and for its solid-harmonic 3-centre bra
(Section 2.2.3).  Every property above is checked independently in
tests/test_oracle_solid.py.

3-centre integrals.  (x|cd) = int int phi_x(r1) r12^-1 phi_c(r2) phi_d(r2) is
the 4-centre integral with the second bra function equal to 1, i.e. an s
Gaussian of exponent 0 and coefficient 1.  eri3 evaluates exactly that with
the 4-centre oracle, then, for a solid-harmonic x, applies the table above.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import oracle as _o


def _cart_index(l: int) -> dict:
    return {c: i for i, c in enumerate(_o.cart_components(l))}


def c2s(l: int) -> np.ndarray:
    """[2l+1][nc(l)] coefficients: S_lm = sum_a c2s[m+l][a] x^ax y^ay z^az,
    rows m = -l..l, columns the Cartesian components x^l first."""
    idx = _cart_index(l)
    out = np.zeros((2 * l + 1, len(idx)), dtype=np.float64)
    for m in range(-l, l + 1):
        am = abs(m)
        norm = math.sqrt(2.0 * math.factorial(l + am) * math.factorial(l - am) / (2.0 if m == 0 else 1.0)) \
            / (2 ** am * math.factorial(l))
        coef = {}
        for t in range((l - am) // 2 + 1):
            for u in range(t + 1):
                for v2 in range(1 if m < 0 else 0, am + 1, 2):  # v2 = 2v
                    sign = -1 if (t + (v2 - (1 if m < 0 else 0)) // 2) % 2 else 1
                    c = Fraction(sign) * Fraction(1, 4 ** t) * math.comb(l, t) * math.comb(l - t, am + t) \
                        * math.comb(t, u) * math.comb(am, v2)
                    ex = (2 * t + am - 2 * u - v2, 2 * u + v2, l - 2 * t - am)
                    coef[ex] = coef.get(ex, Fraction(0)) + c
        for ex, c in coef.items():
            out[m + l, idx[ex]] += float(c) * norm
    return out


def eri3(basis, triples, pure: bool, prec: str = "d", threads: int = 1) -> np.ndarray:
    """3-centre shellsets for (x, c, d) shell triples.  Returns [ntriples][nx][nc*nd]
    as one array per triple concatenated in a list (shapes differ), or, when all
    triples share one class, a single array [ntriples, nx, ncd]."""
    tr = np.asarray(triples, dtype=np.int64).reshape(-1, 3)
    # append the unit s function: exponent 0, coefficient 1 (its centre is irrelevant)
    b = {k: np.asarray(basis[k]) for k in ("centres", "shell_atom", "shell_l", "shell_K", "shell_off", "exps", "coefs")}
    unit = len(b["shell_l"])
    aug = {
        "centres": b["centres"],
        "shell_atom": np.concatenate([b["shell_atom"], [0]]).astype(np.int32),
        "shell_l": np.concatenate([b["shell_l"], [0]]).astype(np.int32),
        "shell_K": np.concatenate([b["shell_K"], [1]]).astype(np.int32),
        "shell_off": np.concatenate([b["shell_off"], [len(b["exps"])]]).astype(np.int32),
        "exps": np.concatenate([b["exps"], [0.0]]),
        "coefs": np.concatenate([b["coefs"], [1.0]]),
    }
    quartets = np.stack([tr[:, 0], np.full(len(tr), unit), tr[:, 1], tr[:, 2]], axis=1).astype(np.int32)
    vals = _o.eri_quartets(aug, quartets, prec=prec, threads=threads).astype(np.float64)
    sizes = _o.shellset_size(aug, quartets)
    pos = np.concatenate([[0], np.cumsum(sizes)])
    l = b["shell_l"]
    blocks = []
    for i, (x, c, d) in enumerate(tr):
        nx = _o.ncart(l[x])
        blk = vals[pos[i]:pos[i + 1]].reshape(nx, -1)
        if pure:
            blk = c2s(int(l[x])) @ blk
        blocks.append(blk)
    if len({bk.shape for bk in blocks}) == 1:
        return np.stack(blocks) if blocks else np.zeros((0, 0, 0))
    return blocks
