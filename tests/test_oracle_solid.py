"""Pins of the oracle's solid harmonics and 3-centre integrals (oracle/solid.py)
against mathematics that does not use them: harmonicity, the sphere norms
and orthogonality (Racah normalisation), the stated sign and phase
conventions, the (s|ss) closed form, the independence of the unit function's
centre and exponent limit, and rotation invariance of the sum over m."""
import math

import mpmath
import numpy as np
import pytest

import oracle
import synth


def poly(l, row):
    """{(ax, ay, az): coefficient} of one solid harmonic."""
    return {c: row[i] for i, c in enumerate(oracle.cart_components(l)) if row[i] != 0.0}


def laplacian(p):
    out = {}
    for (a, b, c), v in p.items():
        for k, e in ((0, a), (1, b), (2, c)):
            if e >= 2:
                ex = [a, b, c]
                ex[k] -= 2
                out[tuple(ex)] = out.get(tuple(ex), 0.0) + v * e * (e - 1)
    return out


def sphere_integral(a, b, c):
    """int over the unit sphere of x^a y^b z^c."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    return 2.0 * math.gamma((a + 1) / 2) * math.gamma((b + 1) / 2) * math.gamma((c + 1) / 2) / math.gamma(
        (a + b + c + 3) / 2)


@pytest.mark.parametrize("l", range(0, 6))
def test_solid_harmonics_are_harmonic_and_orthonormal(l):
    T = oracle.solid.c2s(l)
    assert T.shape == (2 * l + 1, (l + 1) * (l + 2) // 2)
    for m in range(2 * l + 1):
        lap = laplacian(poly(l, T[m]))
        assert all(abs(v) < 1e-12 for v in lap.values()), (l, m, lap)
    G = np.zeros((2 * l + 1, 2 * l + 1))
    comps = oracle.cart_components(l)
    for i, ci in enumerate(comps):
        for j, cj in enumerate(comps):
            G += np.outer(T[:, i], T[:, j]) * sphere_integral(ci[0] + cj[0], ci[1] + cj[1], ci[2] + cj[2])
    assert np.allclose(G, 4 * math.pi / (2 * l + 1) * np.eye(2 * l + 1), rtol=0, atol=1e-12)


@pytest.mark.parametrize("l", range(1, 6))
def test_solid_harmonic_conventions(l):
    T = oracle.solid.c2s(l)
    idx = {c: i for i, c in enumerate(oracle.cart_components(l))}
    assert T[l, idx[(0, 0, l)]] == pytest.approx(1.0, abs=1e-14)          # S_l0(0,0,1) = 1
    for am in range(1, l + 1):
        assert T[l + am, idx[(am, 0, l - am)]] > 0                           # cos(m phi), m > 0
        assert T[l - am, idx[(am - 1, 1, l - am)]] > 0                       # sin(|m| phi), m < 0
        # azimuthal dependence: S_{l,am} at (cos p, sin p, 0)-type points goes as cos(am p) (resp. sin)
        p = 0.37
        r = np.array([math.cos(p), math.sin(p), 0.3])
        rr = np.array([math.cos(p + math.pi / am), math.sin(p + math.pi / am), 0.3])
        val = lambda row, x: sum(v * x[0] ** a * x[1] ** b * x[2] ** c for (a, b, c), v in poly(l, row).items())
        assert val(T[l + am], rr) == pytest.approx(-val(T[l + am], r), abs=1e-12)
        assert val(T[l - am], rr) == pytest.approx(-val(T[l - am], r), abs=1e-12)


def _three_centre_basis():
    rng = np.random.default_rng(5)
    centres = rng.uniform(0, 3, (3, 3))
    shells = [(0, 0, [0.7], [1.3]), (1, 0, [1.1, 0.3], [0.6, 0.4]), (2, 0, [0.5], [0.8]),
              (0, 2, [0.9], [1.0]), (0, 3, [0.45], [0.7]), (1, 1, [0.8, 0.2], [0.5, 0.7]), (2, 1, [1.3], [1.1])]
    return synth.basis_from_shells(centres, shells)


def test_three_centre_s_closed_form():
    """(s|ss) = 2 pi^(5/2) / (p q sqrt(p+q)) c_x K_cd F_0(T), p = zeta_x, T = p q/(p+q) |X-Q|^2."""
    b = _three_centre_basis()
    got = oracle.solid.eri3(b, [(0, 1, 2)], pure=False, prec="ld")[0, 0, 0]
    mpmath.mp.dps = 40
    X = [mpmath.mpf(v) for v in b.centres[0]]
    C = [mpmath.mpf(v) for v in b.centres[1]]
    D = [mpmath.mpf(v) for v in b.centres[2]]
    ref = mpmath.mpf(0)
    zx, cx = mpmath.mpf(0.7), mpmath.mpf(1.3)
    for zc, cc in ((1.1, 0.6), (0.3, 0.4)):
        zc, cc = mpmath.mpf(zc), mpmath.mpf(cc)
        zd, cd = mpmath.mpf(0.5), mpmath.mpf(0.8)
        q = zc + zd
        Q = [(zc * C[i] + zd * D[i]) / q for i in range(3)]
        Kcd = mpmath.exp(-zc * zd / q * sum((C[i] - D[i]) ** 2 for i in range(3)))
        T = zx * q / (zx + q) * sum((X[i] - Q[i]) ** 2 for i in range(3))
        F0 = mpmath.sqrt(mpmath.pi / T) * mpmath.erf(mpmath.sqrt(T)) / 2
        ref += 2 * mpmath.pi ** 2.5 / (zx * q * mpmath.sqrt(zx + q)) * cx * cc * cd * Kcd * F0
    assert abs(float(got) - float(ref)) <= 1e-15 * abs(float(ref))


def test_three_centre_unit_function_reading():
    """The unit second bra function is position-independent, and the limit of
    an s function of vanishing exponent."""
    b = _three_centre_basis()
    base = oracle.solid.eri3(b, [(4, 5, 6)], pure=False, prec="ld")[0]
    for atom, eps in ((1, 0.0), (2, 0.0), (0, 1e-9)):
        aug = b.copy()
        aug.shell_atom = np.concatenate([b.shell_atom, [atom]]).astype(np.int32)
        aug.shell_l = np.concatenate([b.shell_l, [0]]).astype(np.int32)
        aug.shell_K = np.concatenate([b.shell_K, [1]]).astype(np.int32)
        aug.shell_off = np.concatenate([b.shell_off, [len(b.exps)]]).astype(np.int32)
        aug.exps = np.concatenate([b.exps, [eps]])
        aug.coefs = np.concatenate([b.coefs, [1.0]])
        v = oracle.eri_quartets(aug, [(4, b.nshell, 5, 6)], prec="ld").astype(np.float64).reshape(base.shape)
        assert np.allclose(v, base, rtol=0, atol=(1e-16 if eps == 0 else 1e-7) * np.abs(base).max())


def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


@pytest.mark.parametrize("l", [1, 2, 3])
def test_three_centre_pure_rotation_invariance(l):
    """With an s-type ket, sum_m (x_lm|ss)^2 is invariant under rotations of the
    geometry (the real solid harmonics of one l are an orthonormal set up to a
    common factor); the Cartesian sum is not, in general."""
    rng = np.random.default_rng(l)
    centres = rng.uniform(-1.5, 1.5, (3, 3))
    shells = [(0, l, [0.6], [1.0]), (1, 0, [0.9, 0.25], [0.7, 0.5]), (2, 0, [0.4], [1.0])]
    b = synth.basis_from_shells(centres, shells)
    v0 = oracle.solid.eri3(b, [(0, 1, 2)], pure=True, prec="ld")[0, :, 0]
    c0 = oracle.solid.eri3(b, [(0, 1, 2)], pure=False, prec="ld")[0, :, 0]
    for seed in (1, 2):
        R = _rotation(seed)
        br = synth.basis_from_shells(centres @ R.T, shells)
        v = oracle.solid.eri3(br, [(0, 1, 2)], pure=True, prec="ld")[0, :, 0]
        assert np.sum(v ** 2) == pytest.approx(np.sum(v0 ** 2), rel=1e-12)
        if l >= 2:
            c = oracle.solid.eri3(br, [(0, 1, 2)], pure=False, prec="ld")[0, :, 0]
            assert abs(np.sum(c ** 2) - np.sum(c0 ** 2)) > 1e-8 * np.sum(c0 ** 2)
