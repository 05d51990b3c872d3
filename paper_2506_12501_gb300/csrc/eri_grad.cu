// eri_grad.cu -- adjoint of eri_batch: derivatives of E = sum W (ab|cd)
// with respect to the atom centres and the primitive exponents.
//
// Differentiating a primitive Cartesian Gaussian (Section 2.1) gives
//   d/dA_x phi_a = 2 zeta_a phi_{a+1x} - a_x phi_{a-1x},
//   d/dzeta_a phi_a = -(phi_{a+2x} + phi_{a+2y} + phi_{a+2z}),
// so every derivative of the bra product phi_a phi_b expands in Hermite
// functions (Eq. cart2herm-2) with coefficients G^ch_{ab,p'} built from the
// same E tables with raised indices (Hermite order up to l_bra + 2).  With
//   V_k[ab][q]  = sum_cd W_abcd E^cd_{k,q} (-1)^{l_q}        (W back-transformed
//                                                             through the ket)
//   Y_i[ab][p'] = sum_k sum_q V_k[ab][q] [p'+q]^(0)_{ik}
// every bra channel is dE/dch = sum_i sum_ab sum_p' G^ch_{i;ab,p'} Y_i[ab][p'];
// the ket channels are the mirror image with
//   V'_i[cd][p] = sum_ab W_abcd E^ab_{i,p},
//   Z_k[cd][q'] = sum_i sum_p V'_i[cd][p] [p+q']^(0)_{ik},
//   dE/dch      = sum_k sum_cd sum_q' (-1)^{l_q'} G^ch_{k;cd,q'} Z_k[cd][q'].
// The auxiliary integrals [r]^(0) (up to order L+2) are recomputed, not
// stored: pass 1 walks bra primitives (all ket primitives at once), pass 2
// walks ket primitives (all bra primitives at once).
#include <algorithm>

#include "eri_device.cuh"
#include "eri_internal.h"

namespace eri {

constexpr int kGT = 128;  // threads per CTA

struct GradArgs {
    ClassTables ct;
    const double* boys;   // Boys table for L+2
    const RStep* rsteps;
    PairTables pb, pk;
    const int32_t* bra_pairs;
    const int32_t* ket_pairs;
    const int32_t* shell_atom;
    const int32_t* shell_off;
    const int32_t* shell_K;
    const int64_t* quartets;
    int64_t nq, nbra, nket;
    const double* W;
    double* gc;   // [natom][3] or null
    double* ge;   // [nprim] or null
    int KB, KK, KX;
    int o_W, o_Pb, o_Pk, o_Eb, o_Ek, o_A, o_R, o_V, o_Y, o_acc;
};

__device__ __forceinline__ int64_t w_index(const GradArgs& a, int64_t qq, int ab, int cd)
{
    if (a.quartets) return qq + a.nq * ((int64_t)ab * a.ct.ncd + cd);
    const int64_t bra = qq % a.nbra, ket = qq / a.nbra;
    return bra + a.nbra * (ab + (int64_t)a.ct.nab * (cd + (int64_t)a.ct.ncd * ket));
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

// Contraction of one side's derivative channels with Y (or Z) for one
// component pair (a, b) of a primitive pair.  Channels: 0..2 centre 1 (x,y,z),
// 3..5 centre 2, 6 exponent 1, 7 exponent 2.  Ax holds the three per-axis
// tables E[i][j][t] (i <= l1+2, j <= l2+2, t <= l1+l2+4).
__device__ void side_channels(int l1, int l2, const int qa[3], const int qb[3], const double* __restrict__ Ax, int eax,
                              double z1, double z2, const double* __restrict__ Yrow, const int16_t* __restrict__ herm3,
                              int ket, double ch[8])
{
    const int n2 = l2 + 3, nt = l1 + l2 + 5;
    const int H = kLtotMax + 1;
    auto Ev = [&](int x, int i, int j, int t) -> double {
        if (i < 0 || j < 0) return 0.0;
        return Ax[x * eax + (i * n2 + j) * nt + t];
    };
    // per-axis value of the function pair with quanta (i, j) at Hermite t
    // a channel raises one index by at most 2, so its Hermite functions
    // have order <= l1 + l2 + 2 (the rows of Y/Z hold exactly those)
    const int tmax[3] = {qa[0] + qb[0] + 2, qa[1] + qb[1] + 2, qa[2] + qb[2] + 2};
    const int omax = l1 + l2 + 2;
    for (int t = 0; t <= tmax[0]; ++t)
        for (int u = 0; u <= tmax[1] && t + u <= omax; ++u)
            for (int v = 0; v <= tmax[2] && t + u + v <= omax; ++v) {
                const int tt[3] = {t, u, v};
                const int h = herm3[(t * H + u) * H + v];
                double y = Yrow[h];
                if (ket && ((t + u + v) & 1)) y = -y;
                double base[3], up1[3], dn1[3], up2[3], upb1[3], dnb1[3], upb2[3];
                for (int x = 0; x < 3; ++x) {
                    base[x] = tt[x] <= qa[x] + qb[x] ? Ev(x, qa[x], qb[x], tt[x]) : 0.0;
                    up1[x] = Ev(x, qa[x] + 1, qb[x], tt[x]);
                    dn1[x] = Ev(x, qa[x] - 1, qb[x], tt[x]);
                    up2[x] = Ev(x, qa[x] + 2, qb[x], tt[x]);
                    upb1[x] = Ev(x, qa[x], qb[x] + 1, tt[x]);
                    dnb1[x] = Ev(x, qa[x], qb[x] - 1, tt[x]);
                    upb2[x] = Ev(x, qa[x], qb[x] + 2, tt[x]);
                }
                for (int x = 0; x < 3; ++x) {
                    const int o1 = (x + 1) % 3, o2 = (x + 2) % 3;
                    const double rest = base[o1] * base[o2];
                    const double ga = 2.0 * z1 * up1[x] - (double)(float)qa[x] * dn1[x];
                    const double gb = 2.0 * z2 * upb1[x] - (double)(float)qb[x] * dnb1[x];
                    ch[x] = fma(ga * rest, y, ch[x]);
                    ch[3 + x] = fma(gb * rest, y, ch[3 + x]);
                    ch[6] = fma(-up2[x] * rest, y, ch[6]);
                    ch[7] = fma(-upb2[x] * rest, y, ch[7]);
                }
            }
}

__global__ void __launch_bounds__(kGT) grad_kernel(GradArgs a)
{
    extern __shared__ __align__(16) double sm[];
    const ClassTables& ct = a.ct;
    const int tid = threadIdx.x;
    const int nab = ct.nab, ncd = ct.ncd, nhb = ct.nhb, nhk = ct.nhk;
    const int nhb2 = ct.nhb2, nhk2 = ct.nhk2;
    const int KB = a.KB, KK = a.KK, KX = a.KX;
    double* sW = sm + a.o_W;
    double* sPb = sm + a.o_Pb;
    double* sPk = sm + a.o_Pk;
    double* sEb = sm + a.o_Eb;
    double* sEk = sm + a.o_Ek;
    double* sA = sm + a.o_A;
    double* sR = sm + a.o_R;
    double* sV = sm + a.o_V;
    double* sY = sm + a.o_Y;
    double* sacc = sm + a.o_acc;  // 16 channel sums

    for (int64_t qq = blockIdx.x; qq < a.nq; qq += gridDim.x) {
        int bidx, kidx;
        if (a.quartets) {
            bidx = (int)a.quartets[2 * qq];
            kidx = (int)a.quartets[2 * qq + 1];
        } else {
            bidx = (int)(qq % a.nbra);
            kidx = (int)(qq / a.nbra);
        }
        const int Kb = a.pb.kp[bidx], Kk = a.pk.kp[kidx];
        const int sa = a.bra_pairs[2 * bidx], sb = a.bra_pairs[2 * bidx + 1];
        const int sc = a.ket_pairs[2 * kidx], sd = a.ket_pairs[2 * kidx + 1];
        const int K2b = a.shell_K[sb], K2k = a.shell_K[sd];
        __syncthreads();
        for (int i = tid; i < nab * ncd; i += kGT) sW[i] = a.W[w_index(a, qq, i / ncd, i % ncd)];
        for (int i = tid; i < KB * PS_N; i += kGT) sPb[i] = a.pb.ps[(size_t)bidx * KB * PS_N + i];
        for (int i = tid; i < KK * PS_N; i += kGT) sPk[i] = a.pk.ps[(size_t)kidx * KK * PS_N + i];
        for (int i = tid; i < KB * ct.Tab; i += kGT) sEb[i] = a.pb.E[(size_t)bidx * KB * ct.Tab + i];
        for (int i = tid; i < KK * ct.Tcd; i += kGT) sEk[i] = a.pk.E[(size_t)kidx * KK * ct.Tcd + i];
        if (tid < 16) sacc[tid] = 0.0;
        __syncthreads();

        for (int pass = 0; pass < 2; ++pass) {
            // side "s" is walked one primitive at a time, side "o" all at once
            const int Ks = pass == 0 ? Kb : Kk, Ko = pass == 0 ? Kk : Kb;
            const int nS = pass == 0 ? nab : ncd;     // components of the walked side
            const int nO = pass == 0 ? ncd : nab;     // components of the other side
            const int nhO = pass == 0 ? nhk : nhb;    // Hermite functions of the other side
            const int nhS2 = pass == 0 ? nhb2 : nhk2; // raised Hermite range of the walked side
            const int16_t* pq2 = pass == 0 ? ct.pq2b : ct.pq2k;
            // V_o[s-comp][h_o] = sum_{o-comp} W E^o_{o,h}  (all other-side primitives)
            for (int item = tid; item < Ko * nS; item += kGT) {
                const int ko = item / nS, cs = item - ko * nS;
                double* Vrow = sV + (size_t)item * nhO;
                for (int h = 0; h < nhO; ++h) Vrow[h] = 0.0;
                for (int co = 0; co < nO; ++co) {
                    const double w = pass == 0 ? sW[cs * ncd + co] : sW[co * ncd + cs];
                    if (pass == 0) {  // E stored term-major, primitive slot fastest
                        for (int t = ct.ket_start[co]; t < ct.ket_start[co + 1]; ++t)
                            Vrow[ct.ket_q[t]] = fma(w, sEk[t * KK + ko], Vrow[ct.ket_q[t]]);
                    } else {
                        for (int t = ct.bra_start[co]; t < ct.bra_start[co + 1]; ++t)
                            Vrow[ct.bra_p[t]] = fma(w, sEb[t * KB + ko], Vrow[ct.bra_p[t]]);
                    }
                }
            }
            for (int is = 0; is < Ks; ++is) {
                __syncthreads();
                // R for (is, every other-side primitive): layout sR[e * KX + ko]
                for (int ko = tid; ko < Ko; ko += kGT) {
                    const double* pb = pass == 0 ? sPb + is * PS_N : sPb + ko * PS_N;
                    const double* pk = pass == 0 ? sPk + ko * PS_N : sPk + is * PS_N;
                    const double zp = pb[PS_P], zq = pk[PS_P];
                    const double rs = rsqrt(zp + zq);
                    const double rho = zp * zq * (rs * rs);
                    const double X = pb[PS_PX] - pk[PS_PX], Y = pb[PS_PY] - pk[PS_PY], Z = pb[PS_PZ] - pk[PS_PZ];
                    const double T = rho * fma(X, X, fma(Y, Y, Z * Z));
                    double base[kLtotMax + 1];
                    boys_eval(ct.L + 2, T, a.boys, base);
                    double f = pb[PS_INVP] * pk[PS_INVP] * rs;
                    const double m2rho = -2.0 * rho;
                    for (int n = 0; n <= ct.L + 2; ++n) {
                        base[n] *= f;
                        f *= m2rho;
                    }
                    struct S {
                        double* p;
                        int s;
                        __device__ double& operator[](int e) const { return p[(size_t)e * s]; }
                    } R{sR + ko, KX};
                    r_recursion(ct.L + 2, base, X, Y, Z, a.rsteps, R);
                }
                // axis tables of the walked primitive
                const PairTables& PT = pass == 0 ? a.pb : a.pk;
                const int sidx = pass == 0 ? bidx : kidx;
                const int KSd = pass == 0 ? KB : KK;
                for (int i = tid; i < 3 * PT.eax; i += kGT) sA[i] = PT.ax[((size_t)sidx * KSd + is) * 3 * PT.eax + i];
                __syncthreads();
                // Y[s-comp][h'] = sum_ko sum_h V[ko][s-comp][h] R[h' + h]
                for (int item = tid; item < nS * nhS2; item += kGT) {
                    const int cs = item / nhS2, hs = item - cs * nhS2;
                    const int16_t* row = pq2 + (pass == 0 ? (size_t)hs * nhk : (size_t)hs);
                    double y = 0.0;
                    for (int ko = 0; ko < Ko; ++ko) {
                        const double* V = sV + ((size_t)ko * nS + cs) * nhO;
                        for (int h = 0; h < nhO; ++h) {
                            const int e = pass == 0 ? row[h] : row[(size_t)h * nhk2];
                            y = fma(V[h], sR[(size_t)e * KX + ko], y);
                        }
                    }
                    sY[item] = y;
                }
                __syncthreads();
                // channels of the walked primitive
                {
                    const double z1 = (pass == 0 ? a.pb.zz : a.pk.zz)[((size_t)sidx * KSd + is) * 2];
                    const double z2 = (pass == 0 ? a.pb.zz : a.pk.zz)[((size_t)sidx * KSd + is) * 2 + 1];
                    const int l1 = pass == 0 ? ct.la : ct.lc, l2 = pass == 0 ? ct.lb : ct.ld;
                    const int nc2 = (l2 + 1) * (l2 + 2) / 2;
                    double ch[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    for (int cs = tid; cs < nS; cs += kGT) {
                        int qa[3], qb[3];
                        cart_of(l1, cs / nc2, qa);
                        cart_of(l2, cs % nc2, qb);
                        side_channels(l1, l2, qa, qb, sA, PT.eax, z1, z2, sY + (size_t)cs * nhS2, ct.herm3, pass,
                                      ch);
                    }
                    // block reduction of the 8 channels (warp shuffles, then shared atomics)
                    for (int c = 0; c < 8; ++c) {
                        double v = ch[c];
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                        if ((tid & 31) == 0) atomicAdd(&sacc[8 * pass + c], v);
                    }
                    __syncthreads();
                    if (tid == 0) {
                        const int s1 = pass == 0 ? sa : sc, s2 = pass == 0 ? sb : sd;
                        const int K2 = pass == 0 ? K2b : K2k;
                        const int i1 = is / K2, i2 = is - i1 * K2;
                        if (a.ge) {
                            atomicAdd(&a.ge[a.shell_off[s1] + i1], sacc[8 * pass + 6]);
                            atomicAdd(&a.ge[a.shell_off[s2] + i2], sacc[8 * pass + 7]);
                        }
                        if (a.gc) {
                            for (int x = 0; x < 3; ++x) {
                                atomicAdd(&a.gc[3 * a.shell_atom[s1] + x], sacc[8 * pass + x]);
                                atomicAdd(&a.gc[3 * a.shell_atom[s2] + x], sacc[8 * pass + 3 + x]);
                            }
                        }
                        for (int c = 0; c < 8; ++c) sacc[8 * pass + c] = 0.0;
                    }
                }
            }
            __syncthreads();
        }
    }
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
    const ClassTables* ct = nullptr;
    PairTables pb{}, pk{};
    int KB = 0, KK = 0, kmax[4];
    err = prepare_batch(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, 2, st, &ct, &pb, &pk, &KB, &KK,
                        kmax, 0, nullptr);
    if (err != ERI_OK) return err;
    if (ct->L + 2 > kLtotMax) return ERI_EINVAL;
    const double* boys = get_boys_table(ct->L + 2, st, &err);
    if (!boys) return err;
    const RStep* rs = get_rsteps(st, &err);
    if (!rs) return err;
    GradArgs a{};
    a.ct = *ct;
    a.boys = boys;
    a.rsteps = rs;
    a.pb = pb;
    a.pk = pk;
    a.bra_pairs = bra_pairs;
    a.ket_pairs = ket_pairs;
    a.shell_atom = basis->shell_atom;
    a.shell_off = basis->shell_off;
    a.shell_K = basis->shell_K;
    a.quartets = quartets;
    a.nq = nqq;
    a.nbra = nbra;
    a.nket = nket;
    a.W = W;
    a.gc = grad_centres;
    a.ge = grad_exps;
    a.KB = KB;
    a.KK = KK;
    a.KX = std::max(KB, KK);
    size_t off = 0;
    auto take = [&](size_t nd) {
        size_t o = off;
        off += (nd + 1) & ~size_t(1);
        return (int)o;
    };
    a.o_W = take((size_t)ct->nab * ct->ncd);
    a.o_Pb = take((size_t)KB * PS_N);
    a.o_Pk = take((size_t)KK * PS_N);
    a.o_Eb = take((size_t)KB * ct->Tab);
    a.o_Ek = take((size_t)KK * ct->Tcd);
    a.o_A = take((size_t)3 * std::max(pb.eax, pk.eax));
    a.o_R = take((size_t)ct->nhl2 * a.KX);
    a.o_V = take(std::max((size_t)KK * ct->nab * ct->nhk, (size_t)KB * ct->ncd * ct->nhb));
    a.o_Y = take(std::max((size_t)ct->nab * ct->nhb2, (size_t)ct->ncd * ct->nhk2));
    a.o_acc = take(16);
    const size_t bytes = off * 8;
    if (bytes > (size_t)max_smem_optin()) return ERI_EINVAL;
    if (cudaFuncSetAttribute(grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return ERI_ECUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_kernel, kGT, bytes);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(nqq, (int64_t)per_sm * sm_count());
    {
        ProfScope ps(PROF_GRAD, st);
        grad_kernel<<<(int)grid, kGT, bytes, st>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_ECUDA;
}
