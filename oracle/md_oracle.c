/*
 * md_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, serial, deliberately slow CPU implementation of the 4-centre
 * electron-repulsion integrals (ab|cd) over contracted Cartesian Gaussians,
 * written straight from the McMurchie-Davidson (MD) formalism of
 * arXiv 2506.12501 Section 2.1.  It exists to check the CUDA library; only
 * the tests, the smoke entry point and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant with the CUDA
 * path.
 *
 * The file is compiled twice: with REAL = long double (the parity oracle,
 * used by the pins) and with REAL = double (same source; used where the
 * long-double build is too slow, e.g. large parity samples on a host whose
 * long double is software binary128).  Select with -DORACLE_REAL_DOUBLE.
 *
 * Method, step by step (no GEMM, no ket-first ordering, no early
 * contraction, no reuse beyond one R table per primitive quartet):
 *   1. pair quantities  zeta_p = zeta_a + zeta_b,  P = (zeta_a A + zeta_b B)/zeta_p,
 *      same for the ket (Section 2.1, text after Eq. cart2herm-2);
 *   2. Hermite expansion coefficients per axis by Eqs. E2rr1/E2rr2 from
 *      E_00^0 = exp(-zeta_a zeta_b (A_i-B_i)^2 / zeta_p)  (Eq. E2-000), zero
 *      outside 0 <= t <= a+b (Eq. E2-abp, range part; see the parity note);
 *   3. Boys function F_m(T) from its definition (Eq. boys);
 *   4. [0]^(m) = 2 pi^(5/2) / (zeta_p zeta_q sqrt(zeta_p+zeta_q)) (-2 rho)^m F_m(rho |P-Q|^2)
 *      (Eq. 0m) and the auxiliary recursion Eq. r-rr down to m = 0;
 *   5. [p|q] = (-1)^{l_q} [p+q]^(0)  (Eq. pq-from-r);
 *   6. [ab|cd] = sum_p sum_q E_ab^p E_cd^q [p|q]  (Eqs. cart2herm-2, ket- and
 *      bra-from-hermite with Cartesian H = E), then the primitive sum of the
 *      contraction (Section 2.1, contracted Gaussians).
 *
 * Readings taken where the paper is silent or garbled:
 *   - The F_0 formula printed in Section 3.2.1 lacks a factor 1/2; the
 *     definition Eq. boys gives F_0(x) = (1/2) sqrt(pi/x) erf(sqrt x).
 *   - Eq. E2-abp also states a parity rule for the two-centre E; the
 *     recursion Eq. E2rr1 contradicts it (E_10^0 = (P_x - A_x) E_00^0), so
 *     only the range rule is applied.
 *   - Cartesian components of a shell are ordered lexicographically
 *     (x^l first: xx, xy, xz, yy, yz, zz); a pair index is ab = a*nc(lb) + b.
 *   - Contraction coefficients are used verbatim (no normalisation here).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_REAL_DOUBLE
typedef double REAL;
#define RX(f) f
#define ORACLE_SYM(name) oracle_d_##name
#else
typedef long double REAL;
#define RX(f) f##l
#define ORACLE_SYM(name) oracle_ld_##name
#endif

#define PI_R ((REAL)3.14159265358979323846264338327950288L)

/* ORACLE_MUTANT (default 0) plants one deliberate mistake so that a test can
 * show that the pins catch it; the oracle proper is built with 0. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* largest total angular momentum handled (4 shells of l <= 5, plus 2 for
 * the exponent derivative) */
#define OMAX_L 24
#define OMAX_M (OMAX_L + 1)
/* largest quantum along one axis of one function */
#define OMAX_AX 10

/* ------------------------------------------------------------------ */
/* Boys function, Eq. boys: F_m(T) = int_0^1 y^{2m} exp(-T y^2) dy      */
/* ------------------------------------------------------------------ */
/*
 * For T < 60: the series obtained from the definition by repeated
 * integration by parts,
 *     F_m(T) = exp(-T) * sum_{k>=0} (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)),
 * whose terms are all positive (no cancellation).  For T >= 60:
 *     F_0(T) = (1/2) sqrt(pi/T) erf(sqrt T)
 * followed by the upward recursion of Section 3.2.1,
 *     F_{m+1}(T) = ((2m+1) F_m(T) - exp(-T)) / (2T),
 * which is stable there because exp(-T) is negligible against (2m+1) F_m.
 */
void ORACLE_SYM(boys)(int mmax, REAL T, REAL* F)
{
    if (T < (REAL)60) {
        for (int m = 0; m <= mmax; ++m) {
            REAL term = (REAL)1 / (REAL)(2 * m + 1);
            REAL sum = term;
            for (int k = 1; k < 100000; ++k) {
                term *= (REAL)2 * T / (REAL)(2 * m + 2 * k + 1 - (ORACLE_MUTANT == 6 ? 2 : 0));
                sum += term;
                if (term < sum * (REAL)1e-40L) break;
            }
            F[m] = RX(exp)(-T) * sum;
        }
    } else {
        REAL eT = RX(exp)(-T);
        F[0] = (REAL)0.5 * RX(sqrt)(PI_R / T) * RX(erf)(RX(sqrt)(T));
        for (int m = 0; m < mmax; ++m)
            F[m + 1] = ((REAL)(2 * m + 1) * F[m] - eT) / ((REAL)2 * T);
    }
}

/* batch wrapper for the tests: F[i*(mmax+1) + m] = F_m(T[i]) */
void ORACLE_SYM(boys_batch)(int mmax, const double* T, long n, REAL* F)
{
    for (long i = 0; i < n; ++i) ORACLE_SYM(boys)(mmax, (REAL)T[i], F + i * (mmax + 1));
}

/* ------------------------------------------------------------------ */
/* Hermite expansion coefficients, Eqs. E2rr1, E2rr2, E2-000            */
/* ------------------------------------------------------------------ */
/*
 * E[(i*(lb+1) + j)*(la+lb+1) + t] = (E_x)_{i j}^{t} for 0<=i<=la, 0<=j<=lb,
 * 0<=t<=la+lb along one axis with coordinates Ax, Bx and exponents za, zb.
 */
static void hermite_E(int la, int lb, REAL za, REAL zb, REAL Ax, REAL Bx, REAL* E)
{
    const int nt = la + lb + 1;
    const REAL p = za + zb;
    const REAL Px = (za * Ax + zb * Bx) / p;
    const REAL PA = Px - Ax, PB = Px - Bx;
    const REAL inv2p = (REAL)1 / ((REAL)2 * p);
    memset(E, 0, sizeof(REAL) * (size_t)(la + 1) * (lb + 1) * nt);
#define EIDX(i, j, t) (((i) * (lb + 1) + (j)) * nt + (t))
    E[EIDX(0, 0, 0)] = RX(exp)(-za * zb * (Ax - Bx) * (Ax - Bx) / p);
    /* raise a at b = 0 (Eq. E2rr1) */
    for (int i = 0; i < la; ++i)
        for (int t = 0; t <= i + 1; ++t) {
            REAL v = 0;
            if (t >= 1) v += inv2p * E[EIDX(i, 0, t - 1)];
            if (t <= i) v += (ORACLE_MUTANT == 2 ? PB : PA) * E[EIDX(i, 0, t)];
            if (t + 1 <= i && ORACLE_MUTANT != 1) v += (REAL)(t + 1) * E[EIDX(i, 0, t + 1)];
            E[EIDX(i + 1, 0, t)] = v;
        }
    /* raise b for every a (Eq. E2rr2) */
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j < lb; ++j)
            for (int t = 0; t <= i + j + 1; ++t) {
                REAL v = 0;
                if (t >= 1) v += inv2p * E[EIDX(i, j, t - 1)];
                if (t <= i + j) v += PB * E[EIDX(i, j, t)];
                if (t + 1 <= i + j) v += (REAL)(t + 1) * E[EIDX(i, j, t + 1)];
                E[EIDX(i, j + 1, t)] = v;
            }
#undef EIDX
}

/* test hook: the same table for one axis, written to E */
void ORACLE_SYM(hermite_E)(int la, int lb, double za, double zb, double Ax, double Bx, REAL* E)
{
    hermite_E(la, lb, (REAL)za, (REAL)zb, (REAL)Ax, (REAL)Bx, E);
}

/* ------------------------------------------------------------------ */
/* Auxiliary integrals [r]^(0), Eqs. 0m and r-rr                        */
/* ------------------------------------------------------------------ */
/*
 * R table for one primitive quartet: Rt[(t*(L+1) + u)*(L+1) + v] = [t u v]^(0)
 * for t+u+v <= L, computed by the recursion Eq. r-rr
 *   [r + 1_i]^(m) = r_i [r - 1_i]^(m+1) + (P_i - Q_i) [r]^(m+1)
 * from [0]^(m) of Eq. 0m.  The whole (m, t, u, v) cube is kept.
 */
typedef struct {
    int L;
    REAL* R0; /* (L+1)^3 values of [tuv]^(0) */
} rtable;

static void build_rtable(int L, REAL p, REAL q, const REAL P[3], const REAL Q[3], rtable* rt)
{
    const int n = L + 1;
    const REAL rho = p * q / (p + q);
    const REAL sgn = ORACLE_MUTANT == 4 ? (REAL)-1 : (REAL)1;
    const REAL X[3] = {sgn * (P[0] - Q[0]), sgn * (P[1] - Q[1]), sgn * (P[2] - Q[2])};
    const REAL T = rho * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    REAL F[OMAX_M + 1];
    ORACLE_SYM(boys)(L, T, F);
    const REAL pref = (REAL)2 * RX(pow)(PI_R, ORACLE_MUTANT == 7 ? (REAL)2 : (REAL)2.5) / (p * q * RX(sqrt)(p + q));
    /* cube[m][t][u][v] */
    REAL* cube = (REAL*)calloc((size_t)n * n * n * n, sizeof(REAL));
#define CI(m, t, u, v) ((((size_t)(m) * n + (t)) * n + (u)) * n + (v))
    REAL f = pref;
    for (int m = 0; m <= L; ++m) {
        cube[CI(m, 0, 0, 0)] = f * F[m];
        f *= (REAL)-2 * rho;
    }
    /* increase total order N = t+u+v; level N needs m <= L - N */
    for (int N = 1; N <= L; ++N)
        for (int m = 0; m <= L - N; ++m)
            for (int t = 0; t <= N; ++t)
                for (int u = 0; u <= N - t; ++u) {
                    int v = N - t - u;
                    REAL val;
                    if (t > 0) {
                        val = X[0] * cube[CI(m + 1, t - 1, u, v)];
                        if (t > 1 && ORACLE_MUTANT != 3) val += (REAL)(t - 1) * cube[CI(m + 1, t - 2, u, v)];
                    } else if (u > 0) {
                        val = X[1] * cube[CI(m + 1, t, u - 1, v)];
                        if (u > 1) val += (REAL)(u - 1) * cube[CI(m + 1, t, u - 2, v)];
                    } else {
                        val = X[2] * cube[CI(m + 1, t, u, v - 1)];
                        if (v > 1) val += (REAL)(v - 1) * cube[CI(m + 1, t, u, v - 2)];
                    }
                    cube[CI(m, t, u, v)] = val;
                }
    rt->L = L;
    rt->R0 = (REAL*)malloc(sizeof(REAL) * (size_t)n * n * n);
    for (int t = 0; t < n; ++t)
        for (int u = 0; u < n; ++u)
            for (int v = 0; v < n; ++v) rt->R0[(t * n + u) * n + v] = cube[CI(0, t, u, v)];
#undef CI
    free(cube);
}

/* ------------------------------------------------------------------ */
/* One primitive integral over Cartesian monomials                      */
/* ------------------------------------------------------------------ */
typedef struct {
    REAL za, zb, zc, zd;
    REAL A[3], B[3], C[3], D[3];
    REAL P[3], Q[3];
    REAL p, q;
    rtable rt; /* built for the largest L needed by the caller */
} primquartet;

static void primquartet_init(primquartet* pq, REAL za, REAL zb, REAL zc, REAL zd,
                             const REAL A[3], const REAL B[3], const REAL C[3], const REAL D[3], int Lmax)
{
    pq->za = za; pq->zb = zb; pq->zc = zc; pq->zd = zd;
    for (int i = 0; i < 3; ++i) {
        pq->A[i] = A[i]; pq->B[i] = B[i]; pq->C[i] = C[i]; pq->D[i] = D[i];
    }
    pq->p = za + zb;
    pq->q = zc + zd;
    for (int i = 0; i < 3; ++i) {
        pq->P[i] = (za * A[i] + zb * B[i]) / pq->p;
        pq->Q[i] = (zc * C[i] + zd * D[i]) / pq->q;
    }
    build_rtable(Lmax, pq->p, pq->q, pq->P, pq->Q, &pq->rt);
}

static void primquartet_free(primquartet* pq) { free(pq->rt.R0); }

/*
 * [a b | c d] for monomial quanta a,b,c,d (any a_i >= 0), by the direct sum
 *   sum_{t u v} E^x_t E^y_u E^z_v  sum_{tau nu phi} (-1)^{tau+nu+phi}
 *        E'^x_tau E'^y_nu E'^z_phi  [t+tau, u+nu, v+phi]^(0)
 * (Eqs. cart2herm-2, pq-from-r, ket-/bra-from-hermite).  Returns 0 for a
 * negative quantum (the convention used by derivative formulas).
 */
static REAL prim_md(const primquartet* pq, const int a[3], const int b[3], const int c[3], const int d[3])
{
    for (int i = 0; i < 3; ++i)
        if (a[i] < 0 || b[i] < 0 || c[i] < 0 || d[i] < 0) return 0;
    int L = 0;
    for (int i = 0; i < 3; ++i) L += a[i] + b[i] + c[i] + d[i];
    if (L > pq->rt.L) abort();
    const int n = pq->rt.L + 1;
    /* per-axis E tables for the requested quanta */
    REAL Eb[3][2 * OMAX_AX + 1], Ek[3][2 * OMAX_AX + 1];
    REAL tb[(OMAX_AX + 1) * (OMAX_AX + 1) * (2 * OMAX_AX + 1)];
    for (int i = 0; i < 3; ++i) {
        if (a[i] > OMAX_AX || b[i] > OMAX_AX || c[i] > OMAX_AX || d[i] > OMAX_AX) abort();
        int nb = a[i] + b[i] + 1, nk = c[i] + d[i] + 1;
        hermite_E(a[i], b[i], pq->za, pq->zb, pq->A[i], pq->B[i], tb);
        for (int t = 0; t < nb; ++t) Eb[i][t] = tb[(a[i] * (b[i] + 1) + b[i]) * nb + t];
        hermite_E(c[i], d[i], pq->zc, pq->zd, ORACLE_MUTANT == 8 ? pq->D[i] : pq->C[i],
                  ORACLE_MUTANT == 8 ? pq->C[i] : pq->D[i], tb);
        for (int t = 0; t < nk; ++t) Ek[i][t] = tb[(c[i] * (d[i] + 1) + d[i]) * nk + t];
    }
    REAL sum = 0;
    for (int t = 0; t <= a[0] + b[0]; ++t)
        for (int u = 0; u <= a[1] + b[1]; ++u)
            for (int v = 0; v <= a[2] + b[2]; ++v) {
                REAL eb = Eb[0][t] * Eb[1][u] * Eb[2][v];
                REAL inner = 0;
                for (int tau = 0; tau <= c[0] + d[0]; ++tau)
                    for (int nu = 0; nu <= c[1] + d[1]; ++nu)
                        for (int phi = 0; phi <= c[2] + d[2]; ++phi) {
                            REAL sign = (((tau + nu + phi) & 1) && ORACLE_MUTANT != 5) ? (REAL)-1 : (REAL)1;
                            inner += sign * Ek[0][tau] * Ek[1][nu] * Ek[2][phi] *
                                     pq->rt.R0[((t + tau) * n + (u + nu)) * n + (v + phi)];
                        }
                sum += eb * inner;
            }
    return sum;
}

/* single primitive integral over monomials, for the tests (result in *res) */
void ORACLE_SYM(prim_eri)(const int* a, const int* b, const int* c, const int* d,
                          double za, double zb, double zc, double zd,
                          const double* A, const double* B, const double* C, const double* D, REAL* res)
{
    REAL Ar[3], Br[3], Cr[3], Dr[3];
    int L = 0;
    for (int i = 0; i < 3; ++i) {
        Ar[i] = A[i]; Br[i] = B[i]; Cr[i] = C[i]; Dr[i] = D[i];
        L += a[i] + b[i] + c[i] + d[i];
    }
    primquartet pq;
    primquartet_init(&pq, za, zb, zc, zd, Ar, Br, Cr, Dr, L);
    *res = prim_md(&pq, a, b, c, d);
    primquartet_free(&pq);
}

/* ------------------------------------------------------------------ */
/* Shells, Cartesian components                                        */
/* ------------------------------------------------------------------ */
static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* k-th Cartesian component of a shell of angular momentum l, x^l first */
static void cart_component(int l, int k, int q[3])
{
    int idx = 0;
    for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay) {
            if (idx == k) {
                q[0] = ax; q[1] = ay; q[2] = l - ax - ay;
                return;
            }
            ++idx;
        }
}

typedef struct {
    const double* centres;
    const int* shell_atom;
    const int* shell_l;
    const int* shell_K;
    const int* shell_off;
    const double* exps;
    const double* coefs;
} basis_t;

/* number of values in the Cartesian shellset of a quartet of shells */
static long shellset_size(const basis_t* bs, const int* sh)
{
    long n = 1;
    for (int i = 0; i < 4; ++i) n *= ncart(bs->shell_l[sh[i]]);
    return n;
}

/*
 * Contracted Cartesian shellset (ab|cd) for the shells sh[0..3]:
 *   (ab|cd) = sum_{i j k l} c_i c_j c_k c_l [a_i b_j | c_k d_l]
 * (Section 2.1, contracted Gaussians; Eq. def-abcd for each primitive),
 * written to out[(a*nb + b)*ncd + (c*nd + d)].
 */
static void shellset(const basis_t* bs, const int* sh, REAL* out)
{
    const int l[4] = {bs->shell_l[sh[0]], bs->shell_l[sh[1]], bs->shell_l[sh[2]], bs->shell_l[sh[3]]};
    const int nc[4] = {ncart(l[0]), ncart(l[1]), ncart(l[2]), ncart(l[3])};
    const long total = (long)nc[0] * nc[1] * nc[2] * nc[3];
    REAL X[4][3];
    for (int s = 0; s < 4; ++s)
        for (int i = 0; i < 3; ++i) X[s][i] = (REAL)bs->centres[3 * bs->shell_atom[sh[s]] + i];
    for (long i = 0; i < total; ++i) out[i] = 0;
    const int L = l[0] + l[1] + l[2] + l[3];
    for (int i = 0; i < bs->shell_K[sh[0]]; ++i)
        for (int j = 0; j < bs->shell_K[sh[1]]; ++j)
            for (int k = 0; k < bs->shell_K[sh[2]]; ++k)
                for (int m = 0; m < bs->shell_K[sh[3]]; ++m) {
                    const int pi = bs->shell_off[sh[0]] + i, pj = bs->shell_off[sh[1]] + j;
                    const int pk = bs->shell_off[sh[2]] + k, pm = bs->shell_off[sh[3]] + m;
                    const REAL w = (REAL)bs->coefs[pi] * (REAL)bs->coefs[pj] * (REAL)bs->coefs[pk] * (REAL)bs->coefs[pm];
                    primquartet pq;
                    primquartet_init(&pq, bs->exps[pi], bs->exps[pj], bs->exps[pk], bs->exps[pm],
                                     X[0], X[1], X[2], X[3], L);
                    long idx = 0;
                    for (int ia = 0; ia < nc[0]; ++ia)
                        for (int ib = 0; ib < nc[1]; ++ib)
                            for (int ic = 0; ic < nc[2]; ++ic)
                                for (int id = 0; id < nc[3]; ++id) {
                                    int qa[3], qb[3], qc[3], qd[3];
                                    cart_component(l[0], ia, qa);
                                    cart_component(l[1], ib, qb);
                                    cart_component(l[2], ic, qc);
                                    cart_component(l[3], id, qd);
                                    out[idx++] += w * prim_md(&pq, qa, qb, qc, qd);
                                }
                    primquartet_free(&pq);
                }
}

/*
 * Batch entry: quartets[4*q + s] are shell indices; the shellset of quartet
 * q is written contiguously at out + offset(q), offset(q) = sum of the sizes
 * of the earlier quartets.  Returns the total number of values written.
 */
long ORACLE_SYM(eri_quartets)(const double* centres, const int* shell_atom, const int* shell_l,
                              const int* shell_K, const int* shell_off, const double* exps,
                              const double* coefs, const int* quartets, long nq, REAL* out)
{
    basis_t bs = {centres, shell_atom, shell_l, shell_K, shell_off, exps, coefs};
    long off = 0;
    for (long q = 0; q < nq; ++q) {
        shellset(&bs, quartets + 4 * q, out + off);
        off += shellset_size(&bs, quartets + 4 * q);
    }
    return off;
}

/* ------------------------------------------------------------------ */
/* Gradient of sum W (ab|cd) wrt centres and exponents                  */
/* ------------------------------------------------------------------ */
/*
 * Differentiating a primitive Cartesian Gaussian (Section 2.1, first
 * equation) with respect to its centre and exponent, with the contraction
 * coefficients held fixed:
 *   d/dA_i  phi_a = 2 zeta_a phi_{a+1_i} - a_i phi_{a-1_i},
 *   d/dzeta phi_a = -(phi_{a+2x} + phi_{a+2y} + phi_{a+2z}),
 * so every derivative integral is a combination of primitive integrals over
 * shifted monomials, each evaluated with prim_md.  Accumulates (+=)
 *   gc[3*atom + i] += sum_q sum_abcd W_q[abcd] d(ab|cd)_q / dX_{atom,i}
 *   ge[prim]       += sum_q sum_abcd W_q[abcd] d(ab|cd)_q / dzeta_prim
 * where W uses the same per-quartet block layout as eri_quartets.
 */
void ORACLE_SYM(eri_grad_quartets)(const double* centres, const int* shell_atom, const int* shell_l,
                                   const int* shell_K, const int* shell_off, const double* exps,
                                   const double* coefs, const int* quartets, long nq, const double* W,
                                   REAL* gc, REAL* ge)
{
    basis_t bs = {centres, shell_atom, shell_l, shell_K, shell_off, exps, coefs};
    long off = 0;
    for (long qi = 0; qi < nq; ++qi) {
        const int* sh = quartets + 4 * qi;
        const int l[4] = {shell_l[sh[0]], shell_l[sh[1]], shell_l[sh[2]], shell_l[sh[3]]};
        const int nc[4] = {ncart(l[0]), ncart(l[1]), ncart(l[2]), ncart(l[3])};
        REAL X[4][3];
        for (int s = 0; s < 4; ++s)
            for (int i = 0; i < 3; ++i) X[s][i] = (REAL)centres[3 * shell_atom[sh[s]] + i];
        const int L = l[0] + l[1] + l[2] + l[3] + 2;
        int Ks[4], idx4[4];
        for (int s = 0; s < 4; ++s) Ks[s] = shell_K[sh[s]];
        for (idx4[0] = 0; idx4[0] < Ks[0]; ++idx4[0])
            for (idx4[1] = 0; idx4[1] < Ks[1]; ++idx4[1])
                for (idx4[2] = 0; idx4[2] < Ks[2]; ++idx4[2])
                    for (idx4[3] = 0; idx4[3] < Ks[3]; ++idx4[3]) {
                        int pr[4];
                        REAL z[4], w = 1;
                        for (int s = 0; s < 4; ++s) {
                            pr[s] = shell_off[sh[s]] + idx4[s];
                            z[s] = (REAL)exps[pr[s]];
                            w *= (REAL)coefs[pr[s]];
                        }
                        primquartet pq;
                        primquartet_init(&pq, z[0], z[1], z[2], z[3], X[0], X[1], X[2], X[3], L);
                        long idx = 0;
                        for (int ia = 0; ia < nc[0]; ++ia)
                            for (int ib = 0; ib < nc[1]; ++ib)
                                for (int ic = 0; ic < nc[2]; ++ic)
                                    for (int id = 0; id < nc[3]; ++id, ++idx) {
                                        int qq[4][3];
                                        cart_component(l[0], ia, qq[0]);
                                        cart_component(l[1], ib, qq[1]);
                                        cart_component(l[2], ic, qq[2]);
                                        cart_component(l[3], id, qq[3]);
                                        const REAL wq = w * (REAL)W[off + idx];
                                        if (wq == 0) continue;
                                        for (int s = 0; s < 4; ++s) {
                                            /* centre derivatives of function s */
                                            for (int i = 0; i < 3; ++i) {
                                                int up[4][3], dn[4][3];
                                                memcpy(up, qq, sizeof(up));
                                                memcpy(dn, qq, sizeof(dn));
                                                up[s][i] += 1;
                                                dn[s][i] -= 1;
                                                REAL g = (REAL)2 * z[s] * prim_md(&pq, up[0], up[1], up[2], up[3]);
                                                if (qq[s][i] > 0)
                                                    g -= (REAL)qq[s][i] * prim_md(&pq, dn[0], dn[1], dn[2], dn[3]);
                                                gc[3 * shell_atom[sh[s]] + i] += wq * g;
                                            }
                                            /* exponent derivative of function s */
                                            REAL gz = 0;
                                            for (int i = 0; i < 3; ++i) {
                                                int up[4][3];
                                                memcpy(up, qq, sizeof(up));
                                                up[s][i] += 2;
                                                gz -= prim_md(&pq, up[0], up[1], up[2], up[3]);
                                            }
                                            ge[pr[s]] += wq * gz;
                                        }
                                    }
                        primquartet_free(&pq);
                    }
        off += (long)nc[0] * nc[1] * nc[2] * nc[3];
    }
}
