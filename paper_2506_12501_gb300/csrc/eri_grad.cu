// eri_grad.cu -- adjoint of eri_batch: derivatives of E = sum W (ab|cd)
// with respect to the atom centres and the primitive exponents.
//
// Differentiating a primitive Cartesian Gaussian (Section 2.1) gives
//   d/dA_x phi_a = 2 zeta_a phi_{a+1x} - a_x phi_{a-1x},
//   d/dzeta_a phi_a = -(phi_{a+2x} + phi_{a+2y} + phi_{a+2z}),
// so every derivative of the bra product phi_a phi_b expands in Hermite
// functions (Eq. cart2herm-2) with coefficients G^ch_{ab,p'} built from the
// E tables with raised indices (Hermite order up to l_bra + 2).  The kernel
// computes, per tile of quartets and per bra primitive i,
//   X'_i[p'][cd] = sum_k sum_q E^cd_{k,q} (-1)^{l_q} [p'+q]^(0)_{ik}
//                  (the forward ket transform, over the raised bra range),
//   T_i[ab][p']  = sum_cd W_abcd X'_i[p'][cd],
//   dE/dch      += sum_ab sum_p' G^ch_{i;ab,p'} T_i[ab][p']
// for the 8 channels of the bra (3 per centre, 2 exponents).  The ket's
// channels come from a second launch with the sides exchanged, since
// (ab|cd) = (cd|ab).  The auxiliary integrals [r]^(0) (order up to L+2) are
// recomputed, not stored.  Channel sums are reduced per quartet in shared
// memory and added atomically to the gradients (only the order of the
// additions varies).
#include <algorithm>
#include <cmath>

#include "eri_device.cuh"
#include "eri_internal.h"

namespace eri {

constexpr int kGT = 256;  // threads per CTA

struct GradArgs {
    ClassTables ct;            // kernel orientation: the channels are the kernel bra's
    const double* boys;        // Boys table for L+2
    const RStep* rsteps;
    PairTables pb, pk;         // bra: ps, ax, zz, kp; ket: ps, E, kp
    const int32_t* bra_sh;     // the kernel's bra pairs as shell indices [nbra_k][2]
    const int32_t* shell_atom;
    const int32_t* shell_off;
    const int32_t* shell_K;
    const int64_t* quartets;   // the caller's list (NULL: product form)
    int64_t nq, nbra, nket;    // the caller's counts
    int swap;                  // 1: the kernel's bra is the caller's ket
    int nab_o, ncd_o;          // the caller's component-pair counts
    const double* W;
    double* gc;                // [natom][3] or null
    double* ge;                // [nprim] or null
    int TQ, KB, KK, IC;
    int o_q, o_W, o_Pb, o_Pk, o_Ek, o_A, o_R, o_X, o_T, o_ch, o_che;
    int64_t ntiles;
};

__device__ __forceinline__ void g_pairs(const GradArgs& a, int64_t qq, int* b, int* k)
{
    int64_t ob, ok;
    if (a.quartets) {
        ob = a.quartets[2 * qq];
        ok = a.quartets[2 * qq + 1];
    } else {
        ob = qq % a.nbra;
        ok = qq / a.nbra;
    }
    *b = (int)(a.swap ? ok : ob);
    *k = (int)(a.swap ? ob : ok);
}

// W position of the kernel's (ab, cd) of quartet qq in the caller's layout.
__device__ __forceinline__ int64_t g_windex(const GradArgs& a, int64_t qq, int ab, int cd)
{
    const int abo = a.swap ? cd : ab, cdo = a.swap ? ab : cd;
    if (a.quartets) return qq + a.nq * ((int64_t)abo * a.ncd_o + cdo);
    const int64_t bra = qq % a.nbra, ket = qq / a.nbra;
    return bra + a.nbra * (abo + (int64_t)a.nab_o * (cdo + (int64_t)a.ncd_o * ket));
}

// Cartesian component k of a shell of angular momentum l (x^l first).
__device__ __forceinline__ void cart_of(int l, int k, int q[3])
{
    int idx = 0;
    for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay) {
            if (idx == k) {
                q[0] = ax;
                q[1] = ay;
                q[2] = l - ax - ay;
                return;
            }
            ++idx;
        }
}

// Hermite function (t, u, v) of tetrahedral index idx (order N, then t, u descending).
__device__ __forceinline__ void herm_of(int idx, int* t, int* u, int* v)
{
    int N = 0;
    while ((N + 1) * (N + 2) * (N + 3) / 6 <= idx) ++N;
    const int r = idx - N * (N + 1) * (N + 2) / 6;
    int d = 0;
    while ((d + 1) * (d + 2) / 2 <= r) ++d;
    const int e = r - d * (d + 1) / 2;
    *t = N - d;
    *u = d - e;
    *v = N - *t - *u;
}

// Small integers as doubles (the factors a_i of the lowering terms).
__constant__ double c_int_d[8] = {0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0};

// The 8 channel contributions of one Hermite function p' = (t,u,v) of the
// component pair (a, b) of one bra primitive pair, times y = T[ab][p'].
// Ax: the three per-axis tables E[i][j][t] (i <= l1+2, j <= l2+2);
// tz1, tz2: twice the two exponents.
__device__ __forceinline__ void channel_terms(int l1, int l2, const int qa[3], const int qb[3], const int tt[3],
                                              const double* __restrict__ Ax, int eax, double tz1, double tz2,
                                              double y, double ch[8])
{
    const int n2 = l2 + 3, nt = l1 + l2 + 5;
    auto Ev = [&](int x, int i, int j, int t) -> double {
        if (i < 0 || j < 0) return 0.0;
        return Ax[x * eax + (i * n2 + j) * nt + t];
    };
    double base[3], up1[3], dn1[3], up2[3], upb1[3], dnb1[3], upb2[3];
    for (int x = 0; x < 3; ++x) {
        base[x] = Ev(x, qa[x], qb[x], tt[x]);
        up1[x] = Ev(x, qa[x] + 1, qb[x], tt[x]);
        dn1[x] = Ev(x, qa[x] - 1, qb[x], tt[x]);
        up2[x] = Ev(x, qa[x] + 2, qb[x], tt[x]);
        upb1[x] = Ev(x, qa[x], qb[x] + 1, tt[x]);
        dnb1[x] = Ev(x, qa[x], qb[x] - 1, tt[x]);
        upb2[x] = Ev(x, qa[x], qb[x] + 2, tt[x]);
    }
    for (int x = 0; x < 3; ++x) {
        const int o1 = (x + 1) % 3, o2 = (x + 2) % 3;
        const double rest = base[o1] * base[o2] * y;
        const double ga = fma(tz1, up1[x], -c_int_d[qa[x]] * dn1[x]);
        const double gb = fma(tz2, upb1[x], -c_int_d[qb[x]] * dnb1[x]);
        ch[x] = fma(ga, rest, ch[x]);
        ch[3 + x] = fma(gb, rest, ch[3 + x]);
        ch[6] = fma(-up2[x], rest, ch[6]);
        ch[7] = fma(-upb2[x], rest, ch[7]);
    }
}

__global__ void __launch_bounds__(kGT, 2) grad_tile_kernel(GradArgs a)
{
    extern __shared__ __align__(16) double sm[];
    const ClassTables& ct = a.ct;
    const int tid = threadIdx.x;
    const int TQ = a.TQ, KB = a.KB, KK = a.KK, IC = a.IC;
    const int nab = ct.nab, ncd = ct.ncd, nhk = ct.nhk, nhb2 = ct.nhb2, nhl2 = ct.nhl2;
    const int L2 = ct.L + 2;
    const int NI = TQ * IC * KK;  // items of stage A
    const int NIs = NI | 1;       // R row stride (odd: spreads scattered rows over the banks)
    const int eax = a.pb.eax;
    const int AX = 3 * eax + 2;  // axis tables + the two exponents
    int* s_q = reinterpret_cast<int*>(sm + a.o_q);
    double* sW = sm + a.o_W;
    double* sPb = sm + a.o_Pb;
    double* sPk = sm + a.o_Pk;
    double* sEk = sm + a.o_Ek;
    double* sA = sm + a.o_A;
    double* sR = sm + a.o_R;
    double* sX = sm + a.o_X;
    double* sT = sm + a.o_T;
    double* sCh = sm + a.o_ch;
    double* sChE = sm + a.o_che;
    const int ncb = (ct.lb + 1) * (ct.lb + 2) / 2;

    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int64_t q0 = tile * TQ;
        const int nqt = (int)min((int64_t)TQ, a.nq - q0);
        __syncthreads();
        for (int q = tid; q < TQ; q += kGT) {
            int b = 0, k = 0, kb = 0, kk = 0;
            if (q < nqt) {
                g_pairs(a, q0 + q, &b, &k);
                kb = a.pb.kp[b];
                kk = a.pk.kp[k];
            }
            s_q[4 * q] = b;
            s_q[4 * q + 1] = k;
            s_q[4 * q + 2] = kb;
            s_q[4 * q + 3] = kk;
        }
        __syncthreads();
        for (int idx = tid; idx < TQ * KB * PS_N; idx += kGT) {
            const int q = idx / (KB * PS_N), r = idx - q * KB * PS_N, i = r / PS_N;
            sPb[idx] = i < s_q[4 * q + 2] ? a.pb.ps[(size_t)s_q[4 * q] * KB * PS_N + r] : 1.0;
        }
        for (int idx = tid; idx < TQ * KK * PS_N; idx += kGT) {
            const int q = idx / (KK * PS_N), r = idx - q * KK * PS_N, k = r / PS_N;
            sPk[idx] = k < s_q[4 * q + 3] ? a.pk.ps[(size_t)s_q[4 * q + 1] * KK * PS_N + r] : 1.0;
        }
        for (int idx = tid; idx < TQ * KK * ct.Tcd; idx += kGT) {
            const int nk = KK * ct.Tcd, q = idx / nk, r = idx - q * nk, k = r % KK;
            sEk[idx] = k < s_q[4 * q + 3] ? a.pk.E[(size_t)s_q[4 * q + 1] * nk + r] : 0.0;
        }
        for (int idx = tid; idx < TQ * nab * ncd; idx += kGT) {
            const int q = idx / (nab * ncd), r = idx - q * nab * ncd;
            sW[idx] = q < nqt ? a.W[g_windex(a, q0 + q, r / ncd, r % ncd)] : 0.0;
        }
        for (int idx = tid; idx < TQ * 8; idx += kGT) sCh[idx] = 0.0;
        for (int idx = tid; idx < TQ * IC * 2; idx += kGT) sChE[idx] = 0.0;

        for (int i0 = 0; i0 < KB; i0 += IC) {
            __syncthreads();
            // ---- A: auxiliary integrals up to order L+2 for (q, i0+ii, k);
            // with few items a warp shares each item's recursion
            const bool coop = NI * 4 < kGT;
            const int lane = tid & 31;
            for (int item = coop ? tid >> 5 : tid; item < NI; item += coop ? kGT / 32 : kGT) {
                const int q = item / (IC * KK), r = item - q * IC * KK, ii = r / KK, k = r - ii * KK;
                const int i = i0 + ii;
                struct S {
                    double* p;
                    int s;
                    __device__ double& operator[](int e) const { return p[(size_t)e * s]; }
                } R{sR + item, NIs};
                if (i < s_q[4 * q + 2] && k < s_q[4 * q + 3]) {
                    const double* pb = sPb + (q * KB + i) * PS_N;
                    const double* pk = sPk + (q * KK + k) * PS_N;
                    const double zp = pb[PS_P], zq = pk[PS_P];
                    const double rs = rsqrt(zp + zq);
                    const double rho = zp * zq * (rs * rs);
                    const double X = pb[PS_PX] - pk[PS_PX], Y = pb[PS_PY] - pk[PS_PY], Z = pb[PS_PZ] - pk[PS_PZ];
                    const double T = rho * fma(X, X, fma(Y, Y, Z * Z));
                    double base[kLtotMax + 1];
                    boys_eval(L2, T, a.boys, base);
                    double f = pb[PS_INVP] * pk[PS_INVP] * rs;
                    const double m2rho = -2.0 * rho;
                    for (int n = 0; n <= L2; ++n) {
                        base[n] *= f;
                        f *= m2rho;
                    }
                    if (coop)
                        r_recursion_warp(L2, base, X, Y, Z, a.rsteps, R, lane);
                    else
                        r_recursion(L2, base, X, Y, Z, a.rsteps, R);
                } else {
                    for (int e = coop ? lane : 0; e < nhl2; e += coop ? 32 : 1) R[e] = 0.0;
                }
            }
            // axis tables and exponents of the chunk's bra primitives
            for (int idx = tid; idx < TQ * IC * AX; idx += kGT) {
                const int q = idx / (IC * AX), r = idx - q * IC * AX, ii = r / AX, c = r - ii * AX;
                const int i = i0 + ii;
                double v = 0.0;
                if (i < s_q[4 * q + 2]) {
                    const size_t slot = (size_t)s_q[4 * q] * KB + i;
                    // the axis tables, then twice the two exponents
                    v = c < 3 * eax ? a.pb.ax[slot * 3 * eax + c] : 2.0 * a.pb.zz[slot * 2 + (c - 3 * eax)];
                }
                sA[idx] = v;
            }
            __syncthreads();
            const int ICe = min(IC, KB - i0);
            // ---- B': X'[ii][p'][cd][q] over the raised bra range (four chains)
            for (int item = tid; item < TQ * ICe * nhb2 * ncd; item += kGT) {
                const int q = item % TQ;
                int r = item / TQ;
                const int p = r % nhb2;
                r /= nhb2;
                const int cd = r % ncd, ii = r / ncd;
                const double* Ek = sEk + (size_t)q * KK * ct.Tcd;
                const double* Rc = sR + (q * IC + ii) * KK;
                const int16_t* row = ct.pq2b + (size_t)p * nhk;
                const int t0 = ct.ket_start[cd], t1 = ct.ket_start[cd + 1];
                double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
                int t = t0;
                for (; t + 1 < t1; t += 2) {
                    const double* Ra = Rc + (size_t)row[ct.ket_q[t]] * NIs;
                    const double* Rb = Rc + (size_t)row[ct.ket_q[t + 1]] * NIs;
                    const double* Ea = Ek + t * KK;
                    const double* Eb = Ea + KK;
                    int k = 0;
                    for (; k + 1 < KK; k += 2) {
                        v0 = fma(Ea[k], Ra[k], v0);
                        v1 = fma(Ea[k + 1], Ra[k + 1], v1);
                        v2 = fma(Eb[k], Rb[k], v2);
                        v3 = fma(Eb[k + 1], Rb[k + 1], v3);
                    }
                    if (k < KK) {
                        v0 = fma(Ea[k], Ra[k], v0);
                        v2 = fma(Eb[k], Rb[k], v2);
                    }
                }
                if (t < t1) {
                    const double* Ra = Rc + (size_t)row[ct.ket_q[t]] * NIs;
                    const double* Ea = Ek + t * KK;
                    for (int k = 0; k < KK; ++k) v0 = fma(Ea[k], Ra[k], v0);
                }
                sX[(((size_t)ii * nhb2 + p) * ncd + cd) * TQ + q] = (v0 + v1) + (v2 + v3);
            }
            __syncthreads();
            // ---- C'': T[ii][ab][p'][q] = sum_cd W[q][ab][cd] X'[ii][p'][cd][q]
            for (int item = tid; item < TQ * ICe * nab * nhb2; item += kGT) {
                const int q = item % TQ;
                int r = item / TQ;
                const int p = r % nhb2;
                r /= nhb2;
                const int ab = r % nab, ii = r / nab;
                const double* w = sW + (size_t)q * nab * ncd + (size_t)ab * ncd;
                const double* x = sX + ((size_t)ii * nhb2 + p) * ncd * TQ + q;
                double va = 0.0, vb = 0.0;
                int cd = 0;
                for (; cd + 1 < ncd; cd += 2) {
                    va = fma(w[cd], x[(size_t)cd * TQ], va);
                    vb = fma(w[cd + 1], x[(size_t)(cd + 1) * TQ], vb);
                }
                if (cd < ncd) va = fma(w[cd], x[(size_t)cd * TQ], va);
                sT[item] = va + vb;
            }
            __syncthreads();
            // ---- D: channel contributions.  A thread's items share q = tid % TQ
            // (TQ divides kGT) and run through the bra primitives in order: the
            // centre channels stay in registers for the whole tile, the two
            // exponent channels go to shared memory whenever ii changes.
            {
                double ch[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                const int q = tid % TQ;
                int cur = -1;
                for (int item = tid; item < TQ * ICe * nab * nhb2; item += kGT) {
                    int r = item / TQ;
                    const int p = r % nhb2;
                    r /= nhb2;
                    const int ab = r % nab, ii = r / nab;
                    if (ii != cur) {
                        if (cur >= 0) {
                            atomicAdd(&sChE[(q * IC + cur) * 2], ch[6]);
                            atomicAdd(&sChE[(q * IC + cur) * 2 + 1], ch[7]);
                        }
                        cur = ii;
                        ch[6] = ch[7] = 0.0;
                    }
                    if (i0 + ii >= s_q[4 * q + 2]) continue;  // padding bra primitive
                    int qa[3], qb[3], tt[3];
                    cart_of(ct.la, ab / ncb, qa);
                    cart_of(ct.lb, ab % ncb, qb);
                    herm_of(p, &tt[0], &tt[1], &tt[2]);
                    if (tt[0] > qa[0] + qb[0] + 2 || tt[1] > qa[1] + qb[1] + 2 || tt[2] > qa[2] + qb[2] + 2) continue;
                    const double* A = sA + ((size_t)q * IC + ii) * AX;
                    channel_terms(ct.la, ct.lb, qa, qb, tt, A, eax, A[3 * eax], A[3 * eax + 1], sT[item], ch);
                }
                if (cur >= 0) {
                    atomicAdd(&sChE[(q * IC + cur) * 2], ch[6]);
                    atomicAdd(&sChE[(q * IC + cur) * 2 + 1], ch[7]);
                }
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    if (ch[c] != 0.0) atomicAdd(&sCh[q * 8 + c], ch[c]);
            }
            __syncthreads();
            // exponent channels of the chunk's bra primitives
            for (int idx = tid; idx < TQ * ICe; idx += kGT) {
                const int q = idx % TQ, ii = idx / TQ, i = i0 + ii;
                double* e = sChE + (q * IC + ii) * 2;
                if (q < nqt && i < s_q[4 * q + 2] && a.ge) {
                    const int sa = a.bra_sh[2 * s_q[4 * q]], sb = a.bra_sh[2 * s_q[4 * q] + 1];
                    const int K2 = a.shell_K[sb], i1 = i / K2, i2 = i - i1 * K2;
                    atomicAdd(&a.ge[a.shell_off[sa] + i1], e[0]);
                    atomicAdd(&a.ge[a.shell_off[sb] + i2], e[1]);
                }
                e[0] = 0.0;
                e[1] = 0.0;
            }
        }
        __syncthreads();
        // centre channels of the tile's quartets
        if (a.gc)
            for (int q = tid; q < nqt; q += kGT) {
                const int sa = a.bra_sh[2 * s_q[4 * q]], sb = a.bra_sh[2 * s_q[4 * q] + 1];
                for (int x = 0; x < 3; ++x) {
                    atomicAdd(&a.gc[3 * a.shell_atom[sa] + x], sCh[q * 8 + x]);
                    atomicAdd(&a.gc[3 * a.shell_atom[sb] + x], sCh[q * 8 + 3 + x]);
                }
            }
    }
}

static bool grad_layout(const ClassTables& ct, int KB, int KK, int eax, int TQ, int IC, GradArgs* a, size_t* bytes)
{
    size_t off = 0;
    auto take = [&](size_t nd) {
        size_t o = off;
        off += (nd + 1) & ~size_t(1);
        return (int)o;
    };
    a->o_q = take((size_t)TQ * 2);
    a->o_W = take((size_t)TQ * ct.nab * ct.ncd);
    a->o_Pb = take((size_t)TQ * KB * PS_N);
    a->o_Pk = take((size_t)TQ * KK * PS_N);
    a->o_Ek = take((size_t)TQ * KK * ct.Tcd);
    a->o_A = take((size_t)TQ * IC * (3 * eax + 2));
    a->o_R = take((size_t)ct.nhl2 * ((TQ * IC * KK) | 1));
    a->o_X = take((size_t)ct.nhb2 * ct.ncd * TQ * IC);
    a->o_T = take((size_t)ct.nab * ct.nhb2 * TQ * IC);
    a->o_ch = take((size_t)TQ * 8);
    a->o_che = take((size_t)TQ * IC * 2);
    *bytes = off * 8;
    a->TQ = TQ;
    a->IC = IC;
    return *bytes <= (size_t)max_smem_optin();
}

// Tile shape (TQ quartets, IC bra primitives per stage pass): the feasible
// shape with the lowest modelled time per quartet.  Each stage pass costs its
// rounds of kGT items times the FP64 work of one item, plus a barrier; a
// tile makes ceil(KB / IC) passes of five stages.  Shapes that leave room for
// two CTAs per SM (so one CTA's barriers overlap the other's work) are
// preferred whenever one exists.
static bool grad_plan_within(const ClassTables& ct, int KB, int KK, int eax, int64_t nq, size_t limit, GradArgs* a,
                             size_t* bytes);

static bool grad_plan(const ClassTables& ct, int KB, int KK, int eax, int64_t nq, GradArgs* a, size_t* bytes)
{
    const size_t two_per_sm = (size_t)smem_per_sm() / 2 - 1024;
    for (int pass = 0; pass < 2; ++pass) {
        if (grad_plan_within(ct, KB, KK, eax, nq, pass == 0 ? two_per_sm : (size_t)max_smem_optin(), a, bytes))
            return true;
    }
    return false;
}

static bool grad_plan_within(const ClassTables& ct, int KB, int KK, int eax, int64_t nq, size_t limit, GradArgs* a,
                             size_t* bytes)
{
    double best = -1.0;
    GradArgs pick{};
    size_t pick_bytes = 0;
    for (int TQ = 32; TQ >= 1; TQ /= 2) {
        if (TQ > 1 && TQ > nq) continue;
        for (int IC = KB; IC >= 1; IC = IC == 1 ? 0 : (IC + 1) / 2) {
            GradArgs t = *a;
            size_t b = 0;
            if (!grad_layout(ct, KB, KK, eax, TQ, IC, &t, &b) || b > limit) continue;
            auto rounds = [](double n) { return std::ceil(n / kGT); };
            const double kBarrier = 60.0;
            const double pass = rounds((double)TQ * IC * KK) * (3.0 * ct.nhl2 + 60.0) +
                                rounds((double)TQ * IC * ct.nhb2 * ct.ncd) * (2.0 * KK * ct.Tcd / ct.ncd + 8.0) +
                                rounds((double)TQ * IC * ct.nab * ct.nhb2) * (2.0 * ct.ncd + 8.0) +
                                rounds((double)TQ * IC * ct.nab * ct.nhb2) * 50.0 + 5.0 * kBarrier;
            const double cost = std::ceil((double)KB / IC) * pass / TQ;
            if (best < 0 || cost < best) {
                best = cost;
                pick = t;
                pick_bytes = b;
            }
        }
    }
    if (best < 0) return false;
    *a = pick;
    *bytes = pick_bytes;
    return true;
}

// One launch: the channels of the kernel's bra.  bra/ket are the kernel's
// lists (the caller's ket/bra when swap = 1); nbra_o/nket_o are the caller's.
static int launch_grad(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                       int64_t nket, const int64_t* quartets, int64_t nq, const double* W, double* gc, double* ge,
                       int swap, int64_t nbra_o, int64_t nket_o, cudaStream_t st)
{
    const ClassTables* ct = nullptr;
    PairTables pb{}, pk{};
    int KB = 0, KK = 0, kmax[4];
    // the quartet indices refer to the caller's lists: validated on the first launch only
    int err = prepare_batch(cls, basis, bra, nbra, ket, nket, swap ? nullptr : quartets, swap ? 0 : nq, 2, st, &ct,
                            &pb, &pk, &KB, &KK, kmax, 0, nullptr);
    if (err != ERI_OK) return err;
    if (ct->L + 2 > kLtotMax) return ERI_EINVAL;
    GradArgs a{};
    a.ct = *ct;
    a.boys = get_boys_table(ct->L + 2, st, &err);
    a.rsteps = get_rsteps(st, &err);
    if (!a.boys || !a.rsteps) return err;
    a.pb = pb;
    a.pk = pk;
    a.bra_sh = bra;
    a.shell_atom = basis->shell_atom;
    a.shell_off = basis->shell_off;
    a.shell_K = basis->shell_K;
    a.quartets = quartets;
    a.nq = quartets ? nq : nbra_o * nket_o;
    a.nbra = nbra_o;
    a.nket = nket_o;
    a.swap = swap;
    a.nab_o = swap ? ct->ncd : ct->nab;
    a.ncd_o = swap ? ct->nab : ct->ncd;
    a.W = W;
    a.gc = gc;
    a.ge = ge;
    a.KB = KB;
    a.KK = KK;
    size_t bytes = 0;
    if (!grad_plan(*ct, KB, KK, pb.eax, a.nq, &a, &bytes)) return ERI_EINVAL;
    a.ntiles = (a.nq + a.TQ - 1) / a.TQ;
    if (cudaFuncSetAttribute(grad_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return ERI_ECUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_tile_kernel, kGT, bytes);
    const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)std::max(per_sm, 1) * sm_count());
    {
        ProfScope ps(PROF_GRAD, st);
        grad_tile_kernel<<<(int)grid, kGT, bytes, st>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_ECUDA;
}

}  // namespace eri

using namespace eri;

extern "C" int eri_batch_grad(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                              const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nq,
                              const double* W, int64_t w_len, double* grad_centres, double* grad_exps, void* stream)
{
    int err = check_batch_args(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, w_len);
    if (err != ERI_OK) return err;
    const int64_t nqq = quartets ? nq : nbra * nket;
    if (nqq == 0 || nbra == 0 || nket == 0) return ERI_OK;
    if (!W) return ERI_EINVAL;
    if (!grad_centres && !grad_exps) return ERI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // channels of the bra (a, b), then of the ket (c, d) with the sides exchanged
    err = launch_grad(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, W, grad_centres, grad_exps, 0, nbra,
                      nket, st);
    if (err != ERI_OK) return err;
    return launch_grad(eri_class_t{cls.lc, cls.ld, cls.la, cls.lb}, basis, ket_pairs, nket, bra_pairs, nbra, quartets,
                       nq, W, grad_centres, grad_exps, 1, nbra, nket, st);
}
