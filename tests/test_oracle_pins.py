"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks the oracle (oracle/md_oracle.c, long double) against a fact
the mathematics or the paper fixes: closed forms evaluated by an independent
high-precision library, the defining expansions, physical limits, exact
symmetries, and the independent Obara-Saika recursion (oracle/os_oracle.c).
"""
import math

import numpy as np
import pytest

import oracle
import synth

mpmath = pytest.importorskip("mpmath")


# ---------------------------------------------------------------- Boys (Eq. boys)
def test_boys_at_zero():
    """F_m(0) = int_0^1 y^{2m} dy = 1/(2m+1) exactly."""
    F = oracle.boys(24, [0.0])[0]
    for m in range(25):
        assert abs(float(F[m] * (2 * m + 1) - 1)) < 1e-18


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.1, 0.5, 1.0, 5.0, 10.0, 20.0, 35.0, 59.99, 60.0, 60.01, 80.0, 120.0,
                               500.0, 1e4])
def test_boys_incomplete_gamma(T):
    """F_m(T) = gamma(m+1/2, T) / (2 T^{m+1/2}) (substitution t = T y^2 in Eq. boys),
    evaluated by mpmath at 40 digits.  Covers both oracle branches (series below
    T = 60, erf + upward recursion above)."""
    mpmath.mp.dps = 40
    F = oracle.boys(20, [T])[0]
    Tm = mpmath.mpf(T)
    for m in (0, 1, 2, 5, 10, 16, 20):
        ref = mpmath.gammainc(m + mpmath.mpf(1) / 2, 0, Tm) / (2 * Tm ** (m + mpmath.mpf(1) / 2))
        rel = abs((mpmath.mpf(str(F[m])) - ref) / ref)
        assert rel < 2e-17, (T, m, rel)


@pytest.mark.parametrize("T,m", [(0.7, 0), (3.3, 4), (27.0, 9)])
def test_boys_quadrature_of_definition(T, m):
    """Eq. boys integrated numerically (mpmath.quad, 30 digits)."""
    mpmath.mp.dps = 30
    ref = mpmath.quad(lambda y: y ** (2 * m) * mpmath.exp(-T * y * y), [0, 1])
    got = mpmath.mpf(str(oracle.boys(m, [T])[0][m]))
    assert abs((got - ref) / ref) < 1e-17


def test_boys_large_T_asymptote():
    """F_m(T) -> (2m-1)!! / 2^{m+1} sqrt(pi / T^{2m+1}) as T -> inf (the
    exp(-T) and erfc terms vanish); at T = 1e4 the correction is ~e^{-1e4}."""
    T = 1e4
    F = oracle.boys(12, [T])[0]
    for m in range(13):
        dfact = math.prod(range(2 * m - 1, 0, -2)) if m > 0 else 1
        ref = dfact / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(float(F[m]) / ref - 1) < 1e-15


def test_boys_double_build_matches_long_double():
    T = np.concatenate([np.linspace(0, 80, 401), np.geomspace(1e-6, 1e4, 200)])
    Fl = oracle.boys(16, T, prec="ld").astype(np.float64)
    Fd = oracle.boys(16, T, prec="d")
    assert np.max(np.abs(Fd / Fl - 1)) < 5e-15


# ------------------------------------------------- Hermite expansion (Eqs. E2rr*)
@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 1), (3, 2), (3, 3)])
def test_E_defining_expansion(la, lb):
    """Eq. cart2herm-2 along one axis:
    (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) = sum_t E_ij^t Lambda_t(x),
    Lambda_t = (d/dP)^t exp(-p (x-P)^2) = p^{t/2} H_t(sqrt(p)(x-P)) exp(-p(x-P)^2)
    with physicists' Hermite polynomials H_t (mpmath)."""
    mpmath.mp.dps = 30
    a, b, A, B = 0.7, 1.9, 0.3, -0.8
    E = oracle.hermite_E(la, lb, a, b, A, B)
    a, b, A, B = (mpmath.mpf(v) for v in (a, b, A, B))
    p = a + b
    P = (a * A + b * B) / p
    for x in (-1.3, -0.2, 0.05, 0.9, 1.7):
        X = mpmath.mpf(x)
        for i in range(la + 1):
            for j in range(lb + 1):
                lhs = (X - A) ** i * (X - B) ** j * mpmath.exp(-a * (X - A) ** 2 - b * (X - B) ** 2)
                rhs = 0
                for t in range(i + j + 1):
                    rhs += mpmath.mpf(str(E[i, j, t])) * mpmath.mpf(p) ** (mpmath.mpf(t) / 2) * \
                        mpmath.hermite(t, mpmath.sqrt(p) * (X - P)) * mpmath.exp(-p * (X - P) ** 2)
                assert abs(lhs - rhs) < 1e-17 * (1 + abs(lhs))


def test_E_overlap_integral():
    """E_ij^0 sqrt(pi/p) is the 1-D overlap integral (only Lambda_0 has a
    nonzero integral); compared with mpmath.quad."""
    mpmath.mp.dps = 30
    a, b, A, B = 1.3, 0.45, 0.2, 1.1
    E = oracle.hermite_E(3, 3, a, b, A, B)
    a, b, A, B = (mpmath.mpf(v) for v in (a, b, A, B))
    p = a + b
    for i in range(4):
        for j in range(4):
            ref = mpmath.quad(lambda x: (x - A) ** i * (x - B) ** j * mpmath.exp(-a * (x - A) ** 2 - b * (x - B) ** 2),
                              [-mpmath.inf, mpmath.inf])
            got = mpmath.mpf(str(E[i, j, 0])) * mpmath.sqrt(mpmath.pi / p)
            assert abs(got - ref) < 1e-17 * (1 + abs(ref))


def test_E_terminal_closed_form():
    """Eq. E2-abab: E_ij^{i+j} = E_00^0 / (2p)^{i+j}."""
    a, b, A, B = 0.8, 2.2, -0.4, 0.9
    E = oracle.hermite_E(3, 3, a, b, A, B)
    p = np.longdouble(a) + np.longdouble(b)
    for i in range(4):
        for j in range(4):
            assert abs(float(E[i, j, i + j] * (2 * p) ** (i + j) / E[0, 0, 0]) - 1) < 1e-17


def test_E_two_centre_parity_reading():
    """Eq. E2-abp's parity clause would make E_10^0 vanish; the recursion
    Eq. E2rr1 gives E_10^0 = (P-A) E_00^0, confirmed by the 1-D overlap of
    (x-A) times an s function on B, which is nonzero.  The oracle applies only
    the range rule."""
    a, b, A, B = 1.0, 1.0, 0.0, 1.0
    E = oracle.hermite_E(1, 0, a, b, A, B)
    P = (a * A + b * B) / (a + b)
    assert abs(float(E[1, 0, 0]) - (P - A) * float(E[0, 0, 0])) < 1e-17
    assert abs(float(E[1, 0, 0])) > 0.1


# ---------------------------------------------------------- 4-centre integrals
def _ssss_fourier(za, zb, zc, zd, A, B, C, D):
    """(ss|ss) from the Coulomb energy of two Gaussian charge distributions in
    Fourier space: (2/pi) K_AB K_CD (pi^2/(pq))^{3/2} int_0^inf exp(-s k^2) sinc(kR) dk,
    s = 1/(4p) + 1/(4q) -- independent of the Boys function and of Eq. 0m."""
    mpmath.mp.dps = 30
    za, zb, zc, zd = (mpmath.mpf(float(v)) for v in (za, zb, zc, zd))
    A, B, C, D = ([mpmath.mpf(float(c)) for c in x] for x in (A, B, C, D))
    p, q = za + zb, zc + zd
    P = [(za * a + zb * b) / p for a, b in zip(A, B)]
    Q = [(zc * c + zd * d) / q for c, d in zip(C, D)]
    KAB = mpmath.exp(-za * zb / p * sum((a - b) ** 2 for a, b in zip(A, B)))
    KCD = mpmath.exp(-zc * zd / q * sum((c - d) ** 2 for c, d in zip(C, D)))
    R = mpmath.sqrt(sum((x - y) ** 2 for x, y in zip(P, Q)))
    s = mpmath.mpf(1) / (4 * p) + mpmath.mpf(1) / (4 * q)
    if R == 0:
        I = mpmath.quad(lambda k: mpmath.exp(-s * k * k), [0, mpmath.inf])
    else:
        I = mpmath.quad(lambda k: mpmath.exp(-s * k * k) * mpmath.sin(k * R) / (k * R), [0, mpmath.inf])
    return 2 / mpmath.pi * KAB * KCD * (mpmath.pi ** 2 / (p * q)) ** mpmath.mpf(1.5) * I


@pytest.mark.parametrize("geom", [0, 1, 2])
def test_ssss_fourier_space(geom):
    rng = np.random.default_rng(geom)
    z = 10 ** rng.uniform(-1, 1, 4)
    X = rng.uniform(0, 2.0 + 3 * geom, size=(4, 3))
    if geom == 0:
        X[:] = X[0]
    got = oracle.prim_eri([0, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 0], *z, *X)
    ref = _ssss_fourier(*z, *X)
    assert abs((mpmath.mpf(str(got)) - ref) / ref) < 1e-17


def test_far_field_dipole_sign():
    """(p_x s | s s) with the bra at A and the ket far away at C = A + R x:
    the bra distribution x_A exp(-p r_A^2) has dipole mu_x = (pi/p)^{3/2}/(2p),
    so the integral -> S_cd mu_x R / R^3 > 0 (pins the derivative direction and
    the (-1)^{l_q} sign of Eq. pq-from-r)."""
    za, zb, zc, zd = 0.9, 0.6, 0.7, 1.1
    A = np.zeros(3)
    R = 300.0
    C = np.array([R, 0.0, 0.0])
    got = float(oracle.prim_eri([1, 0, 0], [0, 0, 0], [0, 0, 0], [0, 0, 0], za, zb, zc, zd, A, A, C, C))
    p, q = za + zb, zc + zd
    mu = (math.pi / p) ** 1.5 / (2 * p)
    S = (math.pi / q) ** 1.5
    ref = S * mu / R ** 2
    assert got > 0 and abs(got / ref - 1) < 1e-4


def test_p_function_is_centre_derivative():
    """phi_{1x} = (1/(2 zeta_a)) d/dA_x exp(-zeta_a r_A^2): (p_x s|ss) equals the
    central finite difference (Richardson, long double) of (ss|ss)."""
    za, zb, zc, zd = 0.8, 1.3, 0.5, 2.0
    A, B, C, D = [0.1, 0.2, -0.3], [0.9, -0.4, 0.2], [-0.5, 0.7, 1.1], [0.3, 0.3, 0.6]
    s = [0, 0, 0]

    def f(dx):
        Ah = [A[0] + dx, A[1], A[2]]
        return oracle.prim_eri(s, s, s, s, za, zb, zc, zd, Ah, B, C, D)

    h = 1e-3
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    deriv = (4 * d2 - d1) / 3
    got = oracle.prim_eri([1, 0, 0], s, s, s, za, zb, zc, zd, A, B, C, D)
    assert abs(float(got - deriv / (2 * za))) < 1e-12


CLASSES_L2 = synth.all_classes(2)


@pytest.mark.parametrize("cls", CLASSES_L2 + [(3, 0, 0, 0), (3, 3, 1, 0), (2, 3, 3, 1), (3, 2, 3, 3), (3, 3, 3, 3)])
def test_md_equals_obara_saika(cls):
    """The MD oracle and the independent Obara-Saika recursion agree on contracted
    shellsets of every class with l <= 2 and several with l = 3."""
    K = (2, 1, 1, 2) if max(cls) < 3 else (1, 1, 1, 1)
    nq = 2 if sum(cls) < 10 else 1
    b, bra, ket, q = synth.small_random_batch(cls, K=K, nq=nq, seed=sum(cls))
    qs = synth.quartet_shells(bra, ket, q)
    md = oracle.eri_quartets(b, qs)
    os_ = oracle.eri_quartets(b, qs, method="os")
    scale = float(np.max(np.abs(os_)))
    assert float(np.max(np.abs(md - os_))) <= 1e-16 * scale


def _component_map(l, perm):
    """index of component a in the shell after relabelling axes by perm"""
    comps = oracle.cart_components(l)
    pos = {c: i for i, c in enumerate(comps)}
    return [pos[tuple(c[perm[i]] for i in range(3))] for c in comps]


@pytest.mark.parametrize("cls", [(1, 0, 2, 1), (2, 2, 1, 1), (2, 1, 2, 2)])
def test_symmetries(cls):
    """8-fold permutational symmetry of (ab|cd) (Eq. def-abcd is symmetric under
    a<->b, c<->d and bra<->ket), translation invariance, a cyclic relabelling of
    the axes and the reflection x -> -x."""
    b, bra, ket, q = synth.small_random_batch(cls, K=(2, 1, 2, 1), nq=1, seed=7)
    sh = synth.quartet_shells(bra, ket, q)[0]
    la, lb, lc, ld = cls
    nc = [oracle.ncart(l) for l in cls]
    ref = oracle.eri_quartets(b, [sh]).reshape(nc)
    scale = float(np.max(np.abs(ref)))
    sw = oracle.eri_quartets(b, [[sh[1], sh[0], sh[2], sh[3]]]).reshape(nc[1], nc[0], nc[2], nc[3])
    assert float(np.max(np.abs(sw.transpose(1, 0, 2, 3) - ref))) < 1e-17 * scale
    sw = oracle.eri_quartets(b, [[sh[0], sh[1], sh[3], sh[2]]]).reshape(nc[0], nc[1], nc[3], nc[2])
    assert float(np.max(np.abs(sw.transpose(0, 1, 3, 2) - ref))) < 1e-17 * scale
    sw = oracle.eri_quartets(b, [[sh[2], sh[3], sh[0], sh[1]]]).reshape(nc[2], nc[3], nc[0], nc[1])
    assert float(np.max(np.abs(sw.transpose(2, 3, 0, 1) - ref))) < 1e-17 * scale
    # translation
    b2 = b.copy()
    b2.centres = b.centres + np.array([0.375, -1.25, 2.5])
    tr = oracle.eri_quartets(b2, [sh]).reshape(nc)
    assert float(np.max(np.abs(tr - ref))) < 1e-14 * scale
    # cyclic relabelling x' = z, y' = x, z' = y  (r'_i = r_{perm[i]})
    perm = (2, 0, 1)
    b3 = b.copy()
    b3.centres = b.centres[:, list(perm)]
    rot = oracle.eri_quartets(b3, [sh]).reshape(nc)
    # component a' in the new frame equals component a with a_{perm[i]} = a'_i in the old frame
    maps = []
    for l in cls:
        comps = oracle.cart_components(l)
        pos = {c: i for i, c in enumerate(comps)}
        m = []
        for c in comps:
            old = [0, 0, 0]
            for i in range(3):
                old[perm[i]] = c[i]
            m.append(pos[tuple(old)])
        maps.append(m)
    back = ref[np.ix_(*maps)]
    assert float(np.max(np.abs(rot - back))) < 1e-15 * scale
    # reflection x -> -x: sign (-1)^{sum of x quanta}
    b4 = b.copy()
    b4.centres = b.centres * np.array([-1.0, 1.0, 1.0])
    refl = oracle.eri_quartets(b4, [sh]).reshape(nc)
    sign = np.ones(nc)
    for ax_, l in enumerate(cls):
        xs = np.array([c[0] for c in oracle.cart_components(l)])
        shape = [1, 1, 1, 1]
        shape[ax_] = -1
        sign = sign * ((-1.0) ** xs).reshape(shape)
    assert float(np.max(np.abs(refl - sign * ref))) < 1e-15 * scale


# ------------------------------------------------------------------ gradients
def _energy(b, qs, W):
    return float(np.sum(oracle.eri_quartets(b, qs).astype(np.float64) * W))


@pytest.mark.parametrize("cls", [(1, 0, 1, 0), (2, 1, 1, 0), (1, 1, 2, 0)])
def test_gradient_translation_invariance_and_fd(cls):
    """sum over atoms of dE/dX = 0 (translation invariance), and the analytic
    centre and exponent derivatives match central finite differences
    (Richardson-extrapolated) of the oracle energy."""
    b, bra, ket, q = synth.small_random_batch(cls, K=(2, 1, 1, 2), nq=2, seed=3)
    qs = synth.quartet_shells(bra, ket, q)
    n = int(np.sum(oracle.shellset_size(b, qs)))
    W = np.random.default_rng(5).uniform(-1, 1, n)
    gc, ge = oracle.eri_grad_quartets(b, qs, W)
    gc = gc.astype(np.float64)
    ge = ge.astype(np.float64)
    assert np.max(np.abs(gc.sum(axis=0))) < 1e-14 * np.max(np.abs(gc))

    def fd(mutate, h):
        def e(s):
            bb = b.copy()
            mutate(bb, s)
            return _energy(bb, qs, W)
        d1 = (e(h) - e(-h)) / (2 * h)
        d2 = (e(h / 2) - e(-h / 2)) / h
        return (4 * d2 - d1) / 3

    for atom in (0, 5):
        for ax in range(3):
            def mut(bb, s, atom=atom, ax=ax):
                bb.centres[atom, ax] += s
            assert abs(fd(mut, 1e-3) - gc[atom, ax]) < 1e-9 * max(1.0, abs(gc[atom, ax]))
    for prim in (0, 1, 3):
        def mut(bb, s, prim=prim):
            bb.exps[prim] += s
        assert abs(fd(mut, 1e-4) - ge[prim]) < 1e-8 * max(1.0, abs(ge[prim]))


# ------------------------------------------------ double build vs long double
@pytest.mark.parametrize("cls", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 1, 2, 0), (2, 2, 2, 2)])
def test_double_oracle_close_to_long_double(cls):
    """The double-precision build of the same source stays far inside the
    parity tolerance of the GPU tests (1e-11 abs + 1e-10 rel)."""
    basis, pools = synth.class_sweep_pools(seed=0, pool=64, K=3)
    bra, ket, q = synth.class_sweep_batch(pools, cls, nq=6 if sum(cls) < 8 else 2, npairs=64)
    qs = synth.quartet_shells(bra, ket, q)
    ld = oracle.eri_quartets(basis, qs, prec="ld").astype(np.float64)
    d = oracle.eri_quartets(basis, qs, prec="d")
    assert np.max(np.abs(d - ld) - 1e-13 * np.abs(ld)) < 1e-14


@pytest.mark.parametrize("cls", [(2, 2, 2, 2), (3, 3, 2, 2), (3, 3, 3, 3)])
def test_double_oracle_close_to_long_double_high_l_k5(cls):
    """The same on the high angular momentum workload the split-precision
    tests use (exponents log-uniform in [0.05, 50], centres in a 12-bohr
    cube, K = 5 on every shell, L up to 12): the GPU tests of those classes
    compare with the double build."""
    basis, bra, ket, q = synth.split_batch(cls, K=5, seed=7, nq=64, pool=16, npairs=8)
    qs = synth.quartet_shells(bra, ket, q)
    # the most compact candidate (shortest |A-B| + |C-D|): integrals of order one
    c = basis.centres[basis.shell_atom]
    spread = np.linalg.norm(c[qs[:, 0]] - c[qs[:, 1]], axis=1) + np.linalg.norm(c[qs[:, 2]] - c[qs[:, 3]], axis=1)
    qs = qs[np.argsort(spread)[:1]]
    ld = oracle.eri_quartets(basis, qs, prec="ld").astype(np.float64)
    d = oracle.eri_quartets(basis, qs, prec="d")
    print(f"{cls} K=5: max |d - ld| = {np.max(np.abs(d - ld)):.2e}, max |ld| = {np.max(np.abs(ld)):.2e}")
    assert np.max(np.abs(d - ld) - 1e-13 * np.abs(ld)) < 1e-14
