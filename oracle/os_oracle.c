/*
 * os_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * An independent second oracle for the primitive 4-centre integrals,
 * following the Obara-Saika (1986) scheme that the paper contrasts with MD
 * (Section 1 and Section 2.1, reference "Obara and Saika 1986"), in the
 * vertical + horizontal form of Head-Gordon and Pople (1988).  It is written
 * from the published recursions and uses no MD quantity: no Hermite E
 * coefficients and no R_tuv recursion.  It serves only to pin the MD oracle
 * (md_oracle.c) on small inputs.  It calls that file's Boys function, which
 * is pinned on its own against the closed form of Eq. boys.
 *
 * Vertical recursion (W = (zeta_p P + zeta_q Q)/(zeta_p + zeta_q)):
 *   [e+1_i,0|f,0]^(m) = (P_i-A_i)[e0|f0]^(m) + (W_i-P_i)[e0|f0]^(m+1)
 *        + e_i/(2 zeta_p) ([e-1_i,0|f0]^(m) - rho/zeta_p [e-1_i,0|f0]^(m+1))
 *        + f_i/(2(zeta_p+zeta_q)) [e0|f-1_i,0]^(m+1)
 *   [e0|f+1_i,0]^(m)  = (Q_i-C_i)[e0|f0]^(m) + (W_i-Q_i)[e0|f0]^(m+1)
 *        + f_i/(2 zeta_q) ([e0|f-1_i,0]^(m) - rho/zeta_q [e0|f-1_i,0]^(m+1))
 *        + e_i/(2(zeta_p+zeta_q)) [e-1_i,0|f0]^(m+1)
 *   [00|00]^(m) = 2 pi^(5/2)/(zeta_p zeta_q sqrt(zeta_p+zeta_q))
 *                 K_AB K_CD F_m(rho |P-Q|^2),  K_AB = exp(-zeta_a zeta_b |A-B|^2/zeta_p)
 * Horizontal recursion (exact for any Gaussian, no exponent dependence):
 *   [a, b+1_i| = [a+1_i, b| + (A_i - B_i) [a, b|,   same on the ket with C, D.
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

void ORACLE_SYM(boys)(int mmax, REAL T, REAL* F);

typedef struct {
    int ne, nf, L;  /* max total quanta of the e and f functions, L = ne + nf */
    REAL* vrr;      /* memo over (e, f, m) */
    unsigned char* done;
    REAL PA[3], WP[3], QC[3], WQ[3], AB[3], CD[3];
    REAL p, q, rho;
    REAL F[64];
    REAL base; /* 2 pi^(5/2) / (p q sqrt(p+q)) K_AB K_CD */
} osctx;

static size_t vidx(const osctx* c, const int e[3], const int f[3], int m)
{
    const int de = c->ne + 1, df = c->nf + 1;
    size_t k = (size_t)e[0];
    k = k * de + e[1];
    k = k * de + e[2];
    k = k * df + f[0];
    k = k * df + f[1];
    k = k * df + f[2];
    return k * (c->L + 1) + m;
}

static REAL vrr(osctx* c, const int e[3], const int f[3], int m)
{
    for (int i = 0; i < 3; ++i)
        if (e[i] < 0 || f[i] < 0) return 0;
    const size_t k = vidx(c, e, f, m);
    if (c->done[k]) return c->vrr[k];
    REAL val;
    int i = -1;
    for (int j = 0; j < 3; ++j)
        if (e[j] > 0) { i = j; break; }
    if (i >= 0) {
        int e1[3] = {e[0], e[1], e[2]};
        e1[i] -= 1; /* e = e1 + 1_i */
        int e2[3] = {e1[0], e1[1], e1[2]};
        e2[i] -= 1;
        int f1[3] = {f[0], f[1], f[2]};
        f1[i] -= 1;
        val = c->PA[i] * vrr(c, e1, f, m) + c->WP[i] * vrr(c, e1, f, m + 1);
        if (e1[i] > 0)
            val += (REAL)e1[i] / ((REAL)2 * c->p) *
                   (vrr(c, e2, f, m) - c->rho / c->p * vrr(c, e2, f, m + 1));
        if (f[i] > 0) val += (REAL)f[i] / ((REAL)2 * (c->p + c->q)) * vrr(c, e1, f1, m + 1);
    } else {
        for (int j = 0; j < 3; ++j)
            if (f[j] > 0) { i = j; break; }
        if (i < 0) {
            val = c->base * c->F[m];
        } else {
            int f1[3] = {f[0], f[1], f[2]};
            f1[i] -= 1; /* f = f1 + 1_i ; e is zero here */
            int f2[3] = {f1[0], f1[1], f1[2]};
            f2[i] -= 1;
            val = c->QC[i] * vrr(c, e, f1, m) + c->WQ[i] * vrr(c, e, f1, m + 1);
            if (f1[i] > 0)
                val += (REAL)f1[i] / ((REAL)2 * c->q) *
                       (vrr(c, e, f2, m) - c->rho / c->q * vrr(c, e, f2, m + 1));
        }
    }
    c->vrr[k] = val;
    c->done[k] = 1;
    return val;
}

/* [a b | c0] from [e0|c0] by the bra horizontal recursion */
static REAL hrr_bra(osctx* c, const int a[3], const int b[3], const int e_ket[3])
{
    int i = -1;
    for (int j = 0; j < 3; ++j)
        if (b[j] > 0) { i = j; break; }
    if (i < 0) return vrr(c, a, e_ket, 0);
    int a1[3] = {a[0], a[1], a[2]}, b1[3] = {b[0], b[1], b[2]};
    a1[i] += 1;
    b1[i] -= 1;
    return hrr_bra(c, a1, b1, e_ket) + c->AB[i] * hrr_bra(c, a, b1, e_ket);
}

/* [a b | c d] by the ket horizontal recursion, then the bra one */
static REAL hrr(osctx* c, const int a[3], const int b[3], const int cc[3], const int d[3])
{
    int i = -1;
    for (int j = 0; j < 3; ++j)
        if (d[j] > 0) { i = j; break; }
    if (i < 0) return hrr_bra(c, a, b, cc);
    int c1[3] = {cc[0], cc[1], cc[2]}, d1[3] = {d[0], d[1], d[2]};
    c1[i] += 1;
    d1[i] -= 1;
    return hrr(c, a, b, c1, d1) + c->CD[i] * hrr(c, a, b, cc, d1);
}

/*
 * Primitive [a b | c d] over monomials by Obara-Saika.  All quanta >= 0.
 */
void ORACLE_SYM(os_prim_eri)(const int* a, const int* b, const int* cq, const int* d,
                             double za_, double zb_, double zc_, double zd_,
                             const double* A_, const double* B_, const double* C_, const double* D_, REAL* res)
{
    const REAL za = za_, zb = zb_, zc = zc_, zd = zd_;
    REAL A[3], B[3], C[3], D[3], P[3], Q[3], W[3];
    osctx c;
    c.p = za + zb;
    c.q = zc + zd;
    c.rho = c.p * c.q / (c.p + c.q);
    REAL AB2 = 0, CD2 = 0, PQ2 = 0;
    int la = 0, lb = 0, lc = 0, ld = 0;
    for (int i = 0; i < 3; ++i) {
        A[i] = A_[i]; B[i] = B_[i]; C[i] = C_[i]; D[i] = D_[i];
        P[i] = (za * A[i] + zb * B[i]) / c.p;
        Q[i] = (zc * C[i] + zd * D[i]) / c.q;
        W[i] = (c.p * P[i] + c.q * Q[i]) / (c.p + c.q);
        c.PA[i] = P[i] - A[i];
        c.WP[i] = W[i] - P[i];
        c.QC[i] = Q[i] - C[i];
        c.WQ[i] = W[i] - Q[i];
        c.AB[i] = A[i] - B[i];
        c.CD[i] = C[i] - D[i];
        AB2 += c.AB[i] * c.AB[i];
        CD2 += c.CD[i] * c.CD[i];
        PQ2 += (P[i] - Q[i]) * (P[i] - Q[i]);
        la += a[i]; lb += b[i]; lc += cq[i]; ld += d[i];
    }
    c.ne = la + lb;
    c.nf = lc + ld;
    c.L = c.ne + c.nf;
    ORACLE_SYM(boys)(c.L, c.rho * PQ2, c.F);
    c.base = (REAL)2 * RX(pow)(PI_R, (REAL)2.5) / (c.p * c.q * RX(sqrt)(c.p + c.q)) *
             RX(exp)(-za * zb / c.p * AB2) * RX(exp)(-zc * zd / c.q * CD2);
    size_t n = (size_t)(c.ne + 1) * (c.ne + 1) * (c.ne + 1) * (c.nf + 1) * (c.nf + 1) * (c.nf + 1) * (c.L + 1);
    c.vrr = (REAL*)malloc(n * sizeof(REAL));
    c.done = (unsigned char*)calloc(n, 1);
    *res = hrr(&c, a, b, cq, d);
    free(c.vrr);
    free(c.done);
}

/* ------------------------------------------------------------------ */
/* Contracted shellsets by Obara-Saika, one memo table per primitive   */
/* quartet; same inputs and output layout as the MD oracle's           */
/* eri_quartets.                                                        */
/* ------------------------------------------------------------------ */
static int os_ncart(int l) { return (l + 1) * (l + 2) / 2; }

static void os_cart(int l, int k, int q[3])
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

long ORACLE_SYM(os_eri_quartets)(const double* centres, const int* shell_atom, const int* shell_l,
                                 const int* shell_K, const int* shell_off, const double* exps,
                                 const double* coefs, const int* quartets, long nq, REAL* out)
{
    long off = 0;
    for (long qi = 0; qi < nq; ++qi) {
        const int* sh = quartets + 4 * qi;
        int l[4], nc[4];
        REAL X[4][3];
        for (int s = 0; s < 4; ++s) {
            l[s] = shell_l[sh[s]];
            nc[s] = os_ncart(l[s]);
            for (int i = 0; i < 3; ++i) X[s][i] = (REAL)centres[3 * shell_atom[sh[s]] + i];
        }
        const long total = (long)nc[0] * nc[1] * nc[2] * nc[3];
        for (long i = 0; i < total; ++i) out[off + i] = 0;
        int k4[4];
        for (k4[0] = 0; k4[0] < shell_K[sh[0]]; ++k4[0])
            for (k4[1] = 0; k4[1] < shell_K[sh[1]]; ++k4[1])
                for (k4[2] = 0; k4[2] < shell_K[sh[2]]; ++k4[2])
                    for (k4[3] = 0; k4[3] < shell_K[sh[3]]; ++k4[3]) {
                        REAL z[4], w = 1;
                        for (int s = 0; s < 4; ++s) {
                            int pr = shell_off[sh[s]] + k4[s];
                            z[s] = (REAL)exps[pr];
                            w *= (REAL)coefs[pr];
                        }
                        osctx c;
                        REAL P[3], Q[3], W[3], AB2 = 0, CD2 = 0, PQ2 = 0;
                        c.p = z[0] + z[1];
                        c.q = z[2] + z[3];
                        c.rho = c.p * c.q / (c.p + c.q);
                        for (int i = 0; i < 3; ++i) {
                            P[i] = (z[0] * X[0][i] + z[1] * X[1][i]) / c.p;
                            Q[i] = (z[2] * X[2][i] + z[3] * X[3][i]) / c.q;
                            W[i] = (c.p * P[i] + c.q * Q[i]) / (c.p + c.q);
                            c.PA[i] = P[i] - X[0][i];
                            c.WP[i] = W[i] - P[i];
                            c.QC[i] = Q[i] - X[2][i];
                            c.WQ[i] = W[i] - Q[i];
                            c.AB[i] = X[0][i] - X[1][i];
                            c.CD[i] = X[2][i] - X[3][i];
                            AB2 += c.AB[i] * c.AB[i];
                            CD2 += c.CD[i] * c.CD[i];
                            PQ2 += (P[i] - Q[i]) * (P[i] - Q[i]);
                        }
                        c.ne = l[0] + l[1];
                        c.nf = l[2] + l[3];
                        c.L = c.ne + c.nf;
                        ORACLE_SYM(boys)(c.L, c.rho * PQ2, c.F);
                        c.base = (REAL)2 * RX(pow)(PI_R, (REAL)2.5) / (c.p * c.q * RX(sqrt)(c.p + c.q)) *
                                 RX(exp)(-z[0] * z[1] / c.p * AB2) * RX(exp)(-z[2] * z[3] / c.q * CD2);
                        size_t n = (size_t)(c.ne + 1) * (c.ne + 1) * (c.ne + 1) * (c.nf + 1) * (c.nf + 1) *
                                   (c.nf + 1) * (c.L + 1);
                        c.vrr = (REAL*)malloc(n * sizeof(REAL));
                        c.done = (unsigned char*)calloc(n, 1);
                        long idx = 0;
                        for (int ia = 0; ia < nc[0]; ++ia)
                            for (int ib = 0; ib < nc[1]; ++ib)
                                for (int ic = 0; ic < nc[2]; ++ic)
                                    for (int id = 0; id < nc[3]; ++id, ++idx) {
                                        int qa[3], qb[3], qc[3], qd[3];
                                        os_cart(l[0], ia, qa);
                                        os_cart(l[1], ib, qb);
                                        os_cart(l[2], ic, qc);
                                        os_cart(l[3], id, qd);
                                        out[off + idx] += w * hrr(&c, qa, qb, qc, qd);
                                    }
                        free(c.vrr);
                        free(c.done);
                    }
        off += total;
    }
    return off;
}
