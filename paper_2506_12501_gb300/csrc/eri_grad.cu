// eri_grad.cu -- adjoint of eri_batch: derivatives of E = sum W (ab|cd)
// with respect to the atom centres and the primitive exponents.
//
// Differentiating a primitive Cartesian Gaussian (Section 2.1) gives
//   d/dA_x phi_a = 2 zeta_a phi_{a+1x} - a_x phi_{a-1x},
//   d/dzeta_a phi_a = -(phi_{a+2x} + phi_{a+2y} + phi_{a+2z}),
// so every derivative of the bra product phi_a phi_b expands in Hermite
// functions (Eq. cart2herm-2) with coefficients G^ch_{ab,p'} built from the
// E tables with raised indices (Hermite order up to l_bra + 2).  Per tile of
// quartets and per bra primitive i the kernel forms
//   T_i[ab][p']  = sum_cd W_abcd sum_k sum_q E^cd_{k,q} (-1)^{l_q} [p'+q]^(0)_{ik}
//   dE/dch      += sum_ab sum_p' G^ch_{i;ab,p'} T_i[ab][p']
// for the 8 channels of the bra (3 per centre, 2 exponents), in one of two
// orders chosen per launch by a cost model:
//   X form: X'_i[p'][cd] = sum_k sum_q E^cd_{k,q} [p'+q]_ik (the forward ket
//           transform over the raised bra range), then T = sum_cd W X';
//   V form: V_k[ab][q] = sum_cd W_abcd E^cd_{k,q} once per quartet, then
//           T = sum_k sum_q V_k[ab][q] [p'+q]_ik.
// G^ch is a product of one-dimensional tables, so T is formed only for the
// channel items, the (ab, p') where some channel's G is non-zero, and each T
// value is folded at once into the channels its item can reach.  The ket's
// channels come from a second launch with the sides exchanged, since
// (ab|cd) = (cd|ab).  The auxiliary integrals [r]^(0) (order up to L+2) are
// recomputed, not stored.  A batch that mixes contraction degrees runs its
// quartets sorted by primitive-pair counts; CTAs take tiles from a queue.
// Channel sums are reduced per (quartet, bra primitive) by lane groups and
// added atomically to the gradients (only the order of the additions varies).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

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
    const int64_t* order;      // processing order of the caller's quartet indices (NULL: identity)
    unsigned long long* next;  // tile queue (zero at launch)
    int64_t nq, nbra, nket;    // the caller's counts
    int swap;                  // 1: the kernel's bra is the caller's ket
    int nab_o, ncd_o;          // the caller's component-pair counts
    const double* W;
    double* gc;                // [natom][3] or null
    double* ge;                // [nprim] or null
    const int2* items;         // channel items of the bra class (see ItemTable)
    int nit;                   // their number
    int ND, PST;               // derived-table entries per axis and value; doubles per bra primitive
    int Ws, Eks;               // shared-memory row strides of W and of the ket E products (odd)
    int TQ, KB, KK, IC;
    int Xs, XQ;                // X' strides: per Hermite function p' and per (ii, q) (odd)
    // V form (vform = 1): V_k[ab][q] = sum_cd W_abcd E^cd_{k,q} per quartet,
    // then T[ab][p'] = sum_k sum_q V_k[ab][q] [p'+q]_{ik} per channel item
    int vform;
    const int* vstart;         // [nhk+1] terms of each ket Hermite function q
    const int* vlist;          // [Tcd] term t | cd << 16, grouped by q
    int Vs;                    // per-quartet stride of V (odd)
    int o_V, o_pq;
    int o_q, o_W, o_Pb, o_Pk, o_Ek, o_D, o_R, o_X, o_ch;
    int64_t ntiles;
    // one launch for every channel (both = 1): the ket's channels from the
    // same auxiliary integrals, through
    //   Y'_k[ab][q'] = sum_i sum_p E^ab_{i,p} [p+q']^(0)_{ik}   (q' over the raised ket range)
    //   T_k[cd][q']  = (-1)^{|q'|} sum_ab W_abcd Y'_k[ab][q'],
    // folded into the ket channels per (quartet, ket primitive) at the end of a tile
    int both;
    const int32_t* ket_sh;     // the kernel's ket pairs as shell indices [nket_k][2]
    const int2* kitems;        // channel items of the ket class (lc, ld)
    int nitk;
    int NDk, PSTk;             // ket derived-table entries per axis and value; doubles per (quartet, ket primitive)
    int Ebs, Ys;               // strides: staged bra E products per quartet, Y' per (quartet, ket primitive) (odd)
    int o_Eb, o_Y, o_Dk, o_chk;
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

// ---------------------------------------------------------------------------
// Channel items.  The bra channels of one (ab, p') with p' = (t, u, v) are
//   d/dA_i:    (2 zeta_a E^{a+1_i,b} - a_i E^{a-1_i,b})_{t_i} * prod_{j != i} E^{ab}_{t_j}
//   d/dB_i:    (2 zeta_b E^{a,b+1_i} - b_i E^{a,b-1_i})_{t_i} * prod_{j != i} E^{ab}_{t_j}
//   d/dzeta_a: -sum_i E^{a+2_i,b}_{t_i} prod_{j != i} E^{ab}_{t_j}   (zeta_b likewise)
// per axis.  A one-dimensional E^{ij}_t vanishes for t > i + j, so (ab, p')
// contributes only if t_j <= a_j + b_j on all axes but at most one, which may
// exceed it by 1 or 2.  The item list holds exactly those pairs of a class
// (46 % of all (ab, p') for d-d).  A pair that exceeds on axis i has zero
// weight in every channel but those of axis i and the exponents (E^{ab} of
// axis i vanishes there), and by 2 also in the A_i and B_i channels: such
// items get their own, shorter channel code.  Each item is
//   .x = ab | p' << 10 | kind << 20, kind 0: within a_j + b_j on every axis,
//        1 + i: above by 1 on axis i, 4 + i: above by 2 on axis i;
//   .y = the per-axis derived-table offsets (a_i (lb+1) + b_i) nt + t_i,
//        nt = la + lb + 3, at bits 0, 10 and 20,
// ordered by kind, so that neighbouring lanes mostly take the same code.
// ---------------------------------------------------------------------------
struct ItemTable {
    const int2* list[kLmax + 1][kLmax + 1];
    int n[kLmax + 1][kLmax + 1];
};

static std::vector<std::array<int, 3>> cart_list(int l)
{
    std::vector<std::array<int, 3>> r;
    for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay) r.push_back({ax, ay, l - ax - ay});
    return r;
}

static const ItemTable* get_items(cudaStream_t s, int* err)
{
    static std::map<int, ItemTable> tabs;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = tabs.find(dev);
    if (it != tabs.end()) return &it->second;
    std::vector<int2> all;
    int start[kLmax + 1][kLmax + 1];
    ItemTable t{};
    for (int la = 0; la <= kLmax; ++la)
        for (int lb = 0; lb <= kLmax; ++lb) {
            start[la][lb] = (int)all.size();
            std::vector<int2> by_kind[7];
            const auto ca = cart_list(la), cb = cart_list(lb);
            const int nt = la + lb + 3, N2 = la + lb + 2;
            for (int ia = 0; ia < (int)ca.size(); ++ia)
                for (int ib = 0; ib < (int)cb.size(); ++ib) {
                    const int ab = ia * (int)cb.size() + ib;
                    for (int N = 0; N <= N2; ++N)
                        for (int tt = N; tt >= 0; --tt)
                            for (int uu = N - tt; uu >= 0; --uu) {
                                const int h[3] = {tt, uu, N - tt - uu};
                                int over = 0, ok = 1, kind = 0, off[3];
                                for (int x = 0; x < 3; ++x) {
                                    const int e = h[x] - ca[ia][x] - cb[ib][x];
                                    if (e > 2) ok = 0;
                                    if (e > 0) {
                                        ++over;
                                        kind = (e == 1 ? 1 : 4) + x;
                                    }
                                    off[x] = (ca[ia][x] * (lb + 1) + cb[ib][x]) * nt + h[x];
                                }
                                if (!ok || over > 1) continue;
                                const int p = herm_index(h[0], h[1], h[2]);
                                by_kind[kind].push_back(
                                    make_int2(ab | (p << 10) | (kind << 20), off[0] | (off[1] << 10) | (off[2] << 20)));
                            }
                }
            for (const auto& v : by_kind) all.insert(all.end(), v.begin(), v.end());
            t.n[la][lb] = (int)all.size() - start[la][lb];
        }
    int2* d = nullptr;
    if (cudaMalloc(&d, sizeof(int2) * all.size()) != cudaSuccess) {
        *err = ERI_ENOMEM;
        return nullptr;
    }
    if (cudaMemcpyAsync(d, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(d);
        *err = ERI_ECUDA;
        return nullptr;
    }
    for (int la = 0; la <= kLmax; ++la)
        for (int lb = 0; lb <= kLmax; ++lb) t.list[la][lb] = d + start[la][lb];
    tabs[dev] = t;
    return &tabs[dev];
}

// Small integers as doubles (the factors a_i of the lowering terms).
__constant__ double c_int_d[8] = {0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0};

// Forms of the last eri_batch_grad call's two launches (eri_last_grad_forms),
// and the forms the planner may pick (eri_set_grad_forms): bit f allows form f.
static int g_last_grad_form[2] = {-1, -1};
// bits: ERI_GRAD_X, ERI_GRAD_V (forms of a launch's own channels), 2: the
// single launch, 3: two launches; a mask without bits 2 and 3 means two launches
static std::atomic<int> g_grad_form_mask{0xF};
// The scheme a call runs: 0, the cost model's pick; 1, one launch; 2, two
// launches (set by the timed choice of eri_batch_grad for the call).
static thread_local int g_grad_force = 0;

// Derived-table entries per axis and value: (la+1)(lb+1)(la+lb+3).
static int derived_entries(int la, int lb) { return (la + 1) * (lb + 1) * (la + lb + 3); }

// Total order N = t+u+v of Hermite function e (tetrahedral numbering).
__device__ __forceinline__ int herm_order(int e)
{
    int N = 0;
    while ((N + 1) * (N + 2) * (N + 3) / 6 <= e) ++N;
    return N;
}

// Folds one channel item's T value y into the 8 channel sums of its side:
// Dx, Dy, Dz point at the item's entry of the per-axis derived tables
// (components 0..4 at strides ND: E, the two centre-derivative factors, the
// two exponent-derivative factors); kind as in the item table.
__device__ __forceinline__ void fold_item(double y, const double* Dx, const double* Dy, const double* Dz, int ND,
                                          int kind, double (&ch)[8])
{
    switch (kind) {
        case 0: {  // every channel
            const double ex = Dx[0], ey = Dy[0], ez = Dz[0];
            const double yx = y * ex;
            const double pyz = y * ey * ez, pxz = yx * ez, pxy = yx * ey;
            ch[0] = fma(Dx[ND], pyz, ch[0]);
            ch[3] = fma(Dx[2 * ND], pyz, ch[3]);
            ch[6] = fma(Dx[3 * ND], pyz, ch[6]);
            ch[7] = fma(Dx[4 * ND], pyz, ch[7]);
            ch[1] = fma(Dy[ND], pxz, ch[1]);
            ch[4] = fma(Dy[2 * ND], pxz, ch[4]);
            ch[6] = fma(Dy[3 * ND], pxz, ch[6]);
            ch[7] = fma(Dy[4 * ND], pxz, ch[7]);
            ch[2] = fma(Dz[ND], pxy, ch[2]);
            ch[5] = fma(Dz[2 * ND], pxy, ch[5]);
            ch[6] = fma(Dz[3 * ND], pxy, ch[6]);
            ch[7] = fma(Dz[4 * ND], pxy, ch[7]);
            break;
        }
        case 1: {  // above by 1 on x: the x centre channels and the exponents
            const double r = y * Dy[0] * Dz[0];
            ch[0] = fma(Dx[ND], r, ch[0]);
            ch[3] = fma(Dx[2 * ND], r, ch[3]);
            ch[6] = fma(Dx[3 * ND], r, ch[6]);
            ch[7] = fma(Dx[4 * ND], r, ch[7]);
            break;
        }
        case 2: {
            const double r = y * Dx[0] * Dz[0];
            ch[1] = fma(Dy[ND], r, ch[1]);
            ch[4] = fma(Dy[2 * ND], r, ch[4]);
            ch[6] = fma(Dy[3 * ND], r, ch[6]);
            ch[7] = fma(Dy[4 * ND], r, ch[7]);
            break;
        }
        case 3: {
            const double r = y * Dx[0] * Dy[0];
            ch[2] = fma(Dz[ND], r, ch[2]);
            ch[5] = fma(Dz[2 * ND], r, ch[5]);
            ch[6] = fma(Dz[3 * ND], r, ch[6]);
            ch[7] = fma(Dz[4 * ND], r, ch[7]);
            break;
        }
        case 4: {  // above by 2 on x: the exponents only
            const double r = y * Dy[0] * Dz[0];
            ch[6] = fma(Dx[3 * ND], r, ch[6]);
            ch[7] = fma(Dx[4 * ND], r, ch[7]);
            break;
        }
        case 5: {
            const double r = y * Dx[0] * Dz[0];
            ch[6] = fma(Dy[3 * ND], r, ch[6]);
            ch[7] = fma(Dy[4 * ND], r, ch[7]);
            break;
        }
        default: {
            const double r = y * Dx[0] * Dy[0];
            ch[6] = fma(Dz[3 * ND], r, ch[6]);
            ch[7] = fma(Dz[4 * ND], r, ch[7]);
            break;
        }
    }
}

// The per-axis derived tables of one primitive pair (a side's 5 components
// per axis, see the bra's stage in the kernel) from its raised E tables:
// out[(x 5 + c) ND + e], e = (i nbd + j) ntd + t.
__device__ __forceinline__ void derived_entry(const double* __restrict__ ax, const double* __restrict__ zz, int eax,
                                              int l1, int l2, int x, int e, double* o, int ND)
{
    const int n2 = l2 + 3, nte = l1 + l2 + 5, nbd = l2 + 1, ntd = l1 + l2 + 3;
    const int t = e % ntd, ij = e / ntd, jj = ij % nbd, ii = ij / nbd;
    const double* A = ax + (size_t)x * eax + t;
    const double tz1 = 2.0 * zz[0], tz2 = 2.0 * zz[1];
    const int r0 = ii * n2 + jj;
    double v1 = tz1 * A[(r0 + n2) * nte];
    if (ii) v1 = fma(-c_int_d[ii], A[(r0 - n2) * nte], v1);
    double v2 = tz2 * A[(r0 + 1) * nte];
    if (jj) v2 = fma(-c_int_d[jj], A[(r0 - 1) * nte], v2);
    o[0] = A[r0 * nte];
    o[ND] = v1;
    o[2 * ND] = v2;
    o[3 * ND] = -A[(r0 + 2 * n2) * nte];
    o[4 * ND] = -A[(r0 + 2) * nte];
}

__global__ void __launch_bounds__(kGT, 2) grad_tile_kernel(GradArgs a)
{
    extern __shared__ __align__(16) double sm[];
    const ClassTables& ct = a.ct;
    const int tid = threadIdx.x;
    const int TQ = a.TQ, KB = a.KB, KK = a.KK, IC = a.IC;
    const int nab = ct.nab, ncd = ct.ncd, nhk = ct.nhk, nhb2 = ct.nhb2, nhl2 = ct.nhl2;
    const int L2 = ct.L + 2;
    const int NI = TQ * IC * KK;  // items of stage A, ordered (k, ii, q) with q fastest
    const int NIs = NI | 1;       // R row stride (odd: spreads scattered rows over the banks)
    const int ICT = IC * TQ;
    const int Ws = a.Ws, Eks = a.Eks, ND = a.ND, PST = a.PST, nit = a.nit, Xs = a.Xs, XQ = a.XQ;
    const int eax = a.pb.eax;
    const int n2 = ct.lb + 3, nte = ct.la + ct.lb + 5;  // strides of the raised E tables
    const int nbd = ct.lb + 1, ntd = ct.la + ct.lb + 3; // strides of the derived tables
    int* s_q = reinterpret_cast<int*>(sm + a.o_q);
    int64_t* s_qq = reinterpret_cast<int64_t*>(sm + a.o_q + 2 * TQ);
    __shared__ int s_kmax[2];
    __shared__ int64_t s_tile;
    double* sW = sm + a.o_W;
    double* sPb = sm + a.o_Pb;
    double* sPk = sm + a.o_Pk;
    double* sEk = sm + a.o_Ek;
    double* sD = sm + a.o_D;
    double* sR = sm + a.o_R;
    double* sX = sm + a.o_X;
    double* sC8 = sm + a.o_ch;
    double* sV = sm + a.o_V;
    double* sEb = sm + a.o_Eb;
    double* sY = sm + a.o_Y;
    double* sCk = sm + a.o_chk;
    int16_t* s_pq = reinterpret_cast<int16_t*>(sm + a.o_pq);
    const int Vs = a.Vs;
    if (a.vform) {  // the p'+q table, read for every V-form term
        for (int i = tid; i < nhb2 * nhk; i += kGT) s_pq[i] = ct.pq2b[i];
    }

    // tiles from a queue: the sorted order puts the heaviest first, so the
    // CTAs that finish early take the lighter tiles of the tail
    for (;;) {
        __syncthreads();  // the previous tile is done with shared memory
        if (tid == 0) {
            s_tile = (int64_t)atomicAdd(a.next, 1ULL);
            s_kmax[0] = s_kmax[1] = 0;
        }
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= a.ntiles) break;
        const int64_t q0 = tile * TQ;
        const int nqt = (int)min((int64_t)TQ, a.nq - q0);
        {
            int mkb = 0, mkk = 0;
            for (int q = tid; q < TQ; q += kGT) {
                int b = 0, k = 0, kb = 0, kk = 0;
                int64_t qq = 0;
                if (q < nqt) {
                    qq = a.order ? a.order[q0 + q] : q0 + q;
                    g_pairs(a, qq, &b, &k);
                    kb = a.pb.kp[b];
                    kk = a.pk.kp[k];
                }
                s_q[4 * q] = b;
                s_q[4 * q + 1] = k;
                s_q[4 * q + 2] = kb;
                s_q[4 * q + 3] = kk;
                s_qq[q] = qq;
                mkb = max(mkb, kb);
                mkk = max(mkk, kk);
            }
            mkb = __reduce_max_sync(0xffffffffu, mkb);
            mkk = __reduce_max_sync(0xffffffffu, mkk);
            if ((tid & 31) == 0 && mkb > 0) {
                atomicMax(&s_kmax[0], mkb);
                atomicMax(&s_kmax[1], mkk);
            }
        }
        __syncthreads();
        // the tile's own contraction degrees (its quartets share them when sorted)
        const int KBt = s_kmax[0], KKt = s_kmax[1];
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
            sEk[(size_t)q * Eks + r] = k < s_q[4 * q + 3] ? a.pk.E[(size_t)s_q[4 * q + 1] * nk + r] : 0.0;
        }
        for (int idx = tid; idx < TQ * nab * ncd; idx += kGT) {
            const int q = idx / (nab * ncd), r = idx - q * nab * ncd;
            sW[(size_t)q * Ws + r] = q < nqt ? a.W[g_windex(a, s_qq[q], r / ncd, r % ncd)] : 0.0;
        }
        for (int idx = tid; idx < TQ * IC * 8; idx += kGT) sC8[idx] = 0.0;
        if (a.both) {
            // the bra E products of the tile ([q][t][i], no sign), zeroed Y'
            // and ket channel sums
            const int nb = KB * ct.Tab;
            for (int idx = tid; idx < TQ * nb; idx += kGT) {
                const int q = idx / nb, r = idx - q * nb, i = r % KB;
                sEb[(size_t)q * a.Ebs + r] = i < s_q[4 * q + 2] ? a.pb.E[(size_t)s_q[4 * q] * nb + r] : 0.0;
            }
            for (int idx = tid; idx < TQ * KK * a.Ys; idx += kGT) sY[idx] = 0.0;
            for (int idx = tid; idx < TQ * KK * 8; idx += kGT) sCk[idx] = 0.0;
        }
        if (a.vform) {
            // ---- V: V[q][k][ab][qh] = sum over the terms t = (cd, qh) of
            // W[q][ab][cd] E[q][t][k] (the caller's W met with the ket transform)
            __syncthreads();
            const int nV = TQ * KKt * nab * nhk;
            for (int item = tid; item < nV; item += kGT) {
                const int q = item % TQ;
                int r = item / TQ;
                const int qh = r % nhk;
                r /= nhk;
                const int ab = r % nab, k = r / nab;
                const double* w = sW + (size_t)q * Ws + ab * ncd;
                const double* Ek = sEk + (size_t)q * Eks + k;
                // one accumulator chain: a dependent DFMA chain runs at the
                // FP64 pipe's full rate, and needs no DADD to join
                double v = 0.0;
                const int e1 = __ldg(a.vstart + qh + 1);
                for (int e = __ldg(a.vstart + qh); e < e1; ++e) {
                    const int g0 = __ldg(a.vlist + e);
                    v = fma(w[g0 >> 16], Ek[(g0 & 0xffff) * KK], v);
                }
                sV[(size_t)q * Vs + (k * nab + ab) * nhk + qh] = v;
            }
        }

        const int NIt = TQ * IC * KKt;  // stage-A items of this tile (k < KKt)
        for (int i0 = 0; i0 < KBt; i0 += IC) {
            __syncthreads();
            // ---- A: auxiliary integrals up to order L+2 for (q, i0+ii, k);
            // with few items a warp shares each item's recursion
            const bool coop = NIt * 4 < kGT;
            const int lane = tid & 31;
            for (int item = coop ? tid >> 5 : tid; item < NIt; item += coop ? kGT / 32 : kGT) {
                const int q = item % TQ, r = item / TQ, ii = r % IC, k = r / IC;
                const int i = i0 + ii;
                struct S {
                    double* p;
                    int s;
                    __device__ double& operator[](int e) const { return p[(size_t)e * s]; }
                } R{sR + item, NIs};
                if (i < s_q[4 * q + 2] && k < s_q[4 * q + 3]) {
                    const double* pb = sPb + (q * KB + i) * PS_N;
                    const double* pk = sPk + (q * KK + k) * PS_N;
                    // the compile-time path for low orders
                    if (!coop && aux_integrals_fixed(L2, pb, pk, a.boys, R)) continue;
                    const double zp = pb[PS_P], zq = pk[PS_P];
                    const double rs = rsqrt_fp64(zp + zq);
                    const double rho = zp * zq * (rs * rs);
                    const double X = pb[PS_PX] - pk[PS_PX], Y = pb[PS_PY] - pk[PS_PY], Z = pb[PS_PZ] - pk[PS_PZ];
                    const double T = rho * fma(X, X, fma(Y, Y, Z * Z));
                    double base[kLtotMax + 1];
                    boys_eval(L2, T, a.boys, base);
                    double f = rs;  // the pair factors of Eq. 0m are in the E tables
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
            // derived per-axis tables of the chunk's bra primitives,
            // sD[(ii TQ + q) PST + (x 5 + c) ND + e], e = (a nbd + b) ntd + t:
            // c = 0: E^{ab}_t; 1: 2 zeta_a E^{a+1,b}_t - a E^{a-1,b}_t;
            // 2: 2 zeta_b E^{a,b+1}_t - b E^{a,b-1}_t; 3: -E^{a+2,b}_t; 4: -E^{a,b+2}_t
            for (int idx = tid; idx < ICT * 3 * ND; idx += kGT) {
                const int e = idx % ND;
                int r = idx / ND;
                const int x = r % 3;
                r /= 3;
                const int q = r % TQ, ii = r / TQ, i = i0 + ii;
                double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0;
                if (i < s_q[4 * q + 2]) {
                    const int t = e % ntd, ab2 = e / ntd, bb = ab2 % nbd, aa = ab2 / nbd;
                    const size_t slot = (size_t)s_q[4 * q] * KB + i;
                    const double* Ax = a.pb.ax + (slot * 3 + x) * eax + t;
                    const double tz1 = 2.0 * a.pb.zz[2 * slot], tz2 = 2.0 * a.pb.zz[2 * slot + 1];
                    const int r0 = aa * n2 + bb;
                    v0 = Ax[r0 * nte];
                    v1 = tz1 * Ax[(r0 + n2) * nte];
                    if (aa) v1 = fma(-c_int_d[aa], Ax[(r0 - n2) * nte], v1);
                    v2 = tz2 * Ax[(r0 + 1) * nte];
                    if (bb) v2 = fma(-c_int_d[bb], Ax[(r0 - 1) * nte], v2);
                    v3 = -Ax[(r0 + 2 * n2) * nte];
                    v4 = -Ax[(r0 + 2) * nte];
                }
                double* o = sD + (size_t)(ii * TQ + q) * PST + x * 5 * ND + e;
                o[0] = v0;
                o[ND] = v1;
                o[2 * ND] = v2;
                o[3 * ND] = v3;
                o[4 * ND] = v4;
            }
            __syncthreads();
            const int ICe = min(IC, KBt - i0);
            // ---- B': X'[ii][q][p'][cd] over the raised bra range (one chain)
            for (int item = tid; item < (a.vform ? 0 : TQ * ICe * nhb2 * ncd); item += kGT) {
                const int q = item % TQ;
                int r = item / TQ;
                const int p = r % nhb2;
                r /= nhb2;
                const int cd = r % ncd, ii = r / ncd;
                const double* Ek = sEk + (size_t)q * Eks;
                const double* Rc = sR + ii * TQ + q;
                const int16_t* row = ct.pq2b + (size_t)p * nhk;
                const int t0 = ct.ket_start[cd], t1 = ct.ket_start[cd + 1];
                double v = 0.0;
                for (int t = t0; t < t1; ++t) {
                    const double* Ra = Rc + (size_t)row[ct.ket_q[t]] * NIs;
                    const double* Ea = Ek + t * KK;
                    for (int k = 0; k < KKt; ++k) v = fma(Ea[k], Ra[k * ICT], v);
                }
                sX[(size_t)(ii * TQ + q) * XQ + p * Xs + cd] = v;
            }
            if (!a.vform) __syncthreads();
            // ---- C+D.  Each (q, ii) of the chunk is taken by a group of G
            // consecutive lanes.  The group's lanes split its channel items
            // (ab, p'), form y = T[ab][p'] = sum_cd W[q][ab][cd] X'[ii][q][p'][cd]
            // and fold y into the 8 channel sums, which are then reduced over
            // the group by shuffles.  G: the fewest rounds of items, with
            // log2(G) shuffle steps counted.
            {
                int G = 1;
                {
                    int best = -1;
                    for (int g = 1; g <= 32; g *= 2) {
                        const int c = ((TQ * ICe * g + kGT - 1) / kGT) * ((nit + g - 1) / g) * (ncd + 20) +
                                      24 * (__ffs(g) - 1);
                        if (best < 0 || c < best) {
                            best = c;
                            G = g;
                        }
                    }
                }
                const int s = tid & (G - 1), NG = kGT / G;
                const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << ((tid & 31) & ~(G - 1));
                for (int combo = tid / G; combo < TQ * ICe; combo += NG) {
                    const int q = combo % TQ, ii = combo / TQ;
                    const bool live = i0 + ii < s_q[4 * q + 2];  // the same for the whole group
                    double ch[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (live) {
                        const double* wq = sW + (size_t)q * Ws;
                        const double* xq = sX + (size_t)(ii * TQ + q) * XQ;
                        const double* Dq = sD + (size_t)(ii * TQ + q) * PST;
                        for (int j = s; j < nit; j += G) {
                            const int2 g = __ldg(a.items + j);
                            double y = 0.0;  // one chain (see stage V)
                            if (!a.vform) {
                                const double* w = wq + (g.x & 1023) * ncd;
                                const double* xv = xq + ((g.x >> 10) & 1023) * Xs;
                                for (int cd = 0; cd < ncd; ++cd) y = fma(w[cd], xv[cd], y);
                            } else {
                                // T = sum_qh sum_k V[q][k][ab][qh] R_{ii,k}[p'+qh]
                                const double* vq = sV + (size_t)q * Vs + (g.x & 1023) * nhk;
                                const int16_t* pqr = s_pq + ((g.x >> 10) & 1023) * nhk;
                                const double* Rq = sR + ii * TQ + q;
                                const int VK = nab * nhk;
                                for (int qh = 0; qh < nhk; ++qh) {
                                    const double* Ra = Rq + (size_t)pqr[qh] * NIs;
                                    for (int k = 0; k < KKt; ++k) y = fma(vq[k * VK + qh], Ra[k * ICT], y);
                                }
                            }
                            const double* Dx = Dq + (g.y & 1023);
                            const double* Dy = Dq + 5 * ND + ((g.y >> 10) & 1023);
                            const double* Dz = Dq + 10 * ND + (g.y >> 20);
                            fold_item(y, Dx, Dy, Dz, ND, g.x >> 20, ch);
                        }
                    }
                    for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
                        for (int c = 0; c < 8; ++c) ch[c] += __shfl_xor_sync(gmask, ch[c], o);
                    if (live && s == 0) {
                        // centre channels accumulate over the chunks; the exponent
                        // channels belong to this chunk's primitive i0 + ii
                        double* o8 = sC8 + (size_t)(q * IC + ii) * 8;
#pragma unroll
                        for (int c = 0; c < 6; ++c) o8[c] += ch[c];
                        o8[6] = ch[6];
                        o8[7] = ch[7];
                    }
                }
            }
            __syncthreads();
            // exponent channels of the chunk's bra primitives
            if (a.ge)
                for (int idx = tid; idx < TQ * ICe; idx += kGT) {
                    const int q = idx % TQ, ii = idx / TQ, i = i0 + ii;
                    if (q < nqt && i < s_q[4 * q + 2]) {
                        const double* e = sC8 + (size_t)(q * IC + ii) * 8 + 6;
                        const int sa = a.bra_sh[2 * s_q[4 * q]], sb = a.bra_sh[2 * s_q[4 * q] + 1];
                        const int K2 = a.shell_K[sb], i1 = i / K2, i2 = i - i1 * K2;
                        atomicAdd(&a.ge[a.shell_off[sa] + i1], e[0]);
                        atomicAdd(&a.ge[a.shell_off[sb] + i2], e[1]);
                    }
                }
            if (a.both) {
                // ---- K1: Y'[q][k][ab][q'] += sum_ii sum_{p in nz(ab)} E^ab_{i0+ii,p}
                // R_{ii,k}[p+q'], q' over the raised ket range (the auxiliary
                // integrals of this chunk are still in place).  A thread takes
                // four ket primitives of one (q, ab, q'): each term's index
                // lookups and E value serve four products.
                const int nhk2 = ct.nhk2, Ys = a.Ys;
                const int nkb = (KKt + 3) >> 2;
                const int nK1 = TQ * nhk2 * nab * nkb;
                for (int item = tid; item < nK1; item += kGT) {
                    const int q = item % TQ;
                    int r = item / TQ;
                    const int qp = r % nhk2;
                    r /= nhk2;
                    const int ab = r % nab, k0 = 4 * (r / nab);
                    const int kq = s_q[4 * q + 3];
                    if (k0 >= kq) continue;
                    const int nk = min(4, kq - k0);
                    const double* Eq = sEb + (size_t)q * a.Ebs + i0;  // + t KB + ii
                    const double* Rq = sR + q + (size_t)TQ * IC * k0;  // + e NIs + ii TQ + j TQ IC
                    const int kst = TQ * IC;
                    double y[4] = {0.0, 0.0, 0.0, 0.0};
                    const int t0 = __ldg(ct.bra_start + ab), t1 = __ldg(ct.bra_start + ab + 1);
                    for (int t = t0; t < t1; ++t) {
                        const int e = __ldg(ct.pq2k + (int)__ldg(ct.bra_p + t) * nhk2 + qp);
                        const double* Et = Eq + t * KB;
                        const double* Re = Rq + (size_t)e * NIs;
                        for (int ii = 0; ii < ICe; ++ii) {
                            const double ev = Et[ii];
                            const double* Ri = Re + ii * TQ;
                            // only the quartet's own ket primitives (nk of the four)
                            y[0] = fma(ev, Ri[0], y[0]);
                            if (nk > 1) y[1] = fma(ev, Ri[kst], y[1]);
                            if (nk > 2) y[2] = fma(ev, Ri[2 * kst], y[2]);
                            if (nk > 3) y[3] = fma(ev, Ri[3 * kst], y[3]);
                        }
                    }
                    double* yo = sY + ((size_t)q * KK + k0) * Ys + ab * nhk2 + qp;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (j < nk) yo[(size_t)j * Ys] += y[j];
                }
            }
        }
        __syncthreads();
        if (a.both) {
            // ---- K2: the ket's derived tables per (quartet, ket primitive), in
            // the auxiliary-integral region (dead now)
            const int NDk = a.NDk, PSTk = a.PSTk;
            double* sDk = sR;
            for (int idx = tid; idx < TQ * KKt * 3 * NDk; idx += kGT) {
                const int e = idx % NDk;
                int r = idx / NDk;
                const int x = r % 3;
                r /= 3;
                const int q = r % TQ, k = r / TQ;
                double* o = sDk + ((size_t)q * KK + k) * PSTk + x * 5 * NDk + e;
                if (k < s_q[4 * q + 3]) {
                    const size_t slot = (size_t)s_q[4 * q + 1] * KK + k;
                    derived_entry(a.pk.ax + slot * 3 * a.pk.eax, a.pk.zz + 2 * slot, a.pk.eax, ct.lc, ct.ld, x, e,
                                  o, NDk);
                } else {
                    for (int c = 0; c < 5; ++c) o[c * NDk] = 0.0;
                }
            }
            __syncthreads();
            // ---- K3: the ket's channel items per (quartet, ket primitive):
            // T = (-1)^{|q'|} sum_ab W[q][ab][cd] Y'[q][k][ab][q'], folded into
            // the 8 ket channels by lane groups as in C+D
            const int nhk2 = ct.nhk2, Ys = a.Ys, nitk = a.nitk;
            int G = 1;
            {
                int best = -1;
                for (int g = 1; g <= 32; g *= 2) {
                    const int c = ((TQ * KKt * g + kGT - 1) / kGT) * ((nitk + g - 1) / g) * (nab + 20) +
                                  24 * (__ffs(g) - 1);
                    if (best < 0 || c < best) {
                        best = c;
                        G = g;
                    }
                }
            }
            const int sl = tid & (G - 1), NG = kGT / G;
            const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << ((tid & 31) & ~(G - 1));
            for (int combo = tid / G; combo < TQ * KKt; combo += NG) {
                const int q = combo % TQ, k = combo / TQ;
                const bool live = k < s_q[4 * q + 3];  // the same for the whole group
                double ch[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (live) {
                    const double* wq = sW + (size_t)q * Ws;
                    const double* yq = sY + ((size_t)q * KK + k) * Ys;
                    const double* Dq = sDk + ((size_t)q * KK + k) * PSTk;
                    for (int j = sl; j < nitk; j += G) {
                        const int2 g = __ldg(a.kitems + j);
                        const int cd = g.x & 1023, qp = (g.x >> 10) & 1023;
                        const double* yv = yq + qp;
                        double ya = 0.0;
                        for (int ab = 0; ab < nab; ++ab) ya = fma(wq[ab * ncd + cd], yv[ab * nhk2], ya);
                        const double y = (herm_order(qp) & 1) ? -ya : ya;
                        fold_item(y, Dq + (g.y & 1023), Dq + 5 * NDk + ((g.y >> 10) & 1023),
                                  Dq + 10 * NDk + (g.y >> 20), NDk, g.x >> 20, ch);
                    }
                }
                for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
                    for (int c = 0; c < 8; ++c) ch[c] += __shfl_xor_sync(gmask, ch[c], o);
                if (live && sl == 0) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) sCk[((size_t)q * KK + k) * 8 + c] = ch[c];
                    if (a.ge) {  // exponent channels of ket primitive k
                        const int sc = a.ket_sh[2 * s_q[4 * q + 1]], sd = a.ket_sh[2 * s_q[4 * q + 1] + 1];
                        const int K2 = a.shell_K[sd], k1 = k / K2, k2 = k - k1 * K2;
                        atomicAdd(&a.ge[a.shell_off[sc] + k1], ch[6]);
                        atomicAdd(&a.ge[a.shell_off[sd] + k2], ch[7]);
                    }
                }
            }
            __syncthreads();
            // centre channels of the ket (summed over the ket primitives)
            if (a.gc)
                for (int q = tid; q < nqt; q += kGT) {
                    const int sc = a.ket_sh[2 * s_q[4 * q + 1]], sd = a.ket_sh[2 * s_q[4 * q + 1] + 1];
                    double c6[6] = {0, 0, 0, 0, 0, 0};
                    for (int k = 0; k < KKt; ++k)
#pragma unroll
                        for (int c = 0; c < 6; ++c) c6[c] += sCk[((size_t)q * KK + k) * 8 + c];
                    for (int x = 0; x < 3; ++x) {
                        atomicAdd(&a.gc[3 * a.shell_atom[sc] + x], c6[x]);
                        atomicAdd(&a.gc[3 * a.shell_atom[sd] + x], c6[3 + x]);
                    }
                }
        }
        // centre channels of the tile's quartets (summed over the IC slots)
        if (a.gc)
            for (int q = tid; q < nqt; q += kGT) {
                const int sa = a.bra_sh[2 * s_q[4 * q]], sb = a.bra_sh[2 * s_q[4 * q] + 1];
                double c6[6] = {0, 0, 0, 0, 0, 0};
                for (int ii = 0; ii < IC; ++ii)
#pragma unroll
                    for (int c = 0; c < 6; ++c) c6[c] += sC8[(size_t)(q * IC + ii) * 8 + c];
                for (int x = 0; x < 3; ++x) {
                    atomicAdd(&a.gc[3 * a.shell_atom[sa] + x], c6[x]);
                    atomicAdd(&a.gc[3 * a.shell_atom[sb] + x], c6[3 + x]);
                }
            }
    }
}

static bool grad_layout(const ClassTables& ct, int KB, int KK, int TQ, int IC, int vform, int both, GradArgs* a,
                        size_t* bytes)
{
    size_t off = 0;
    auto take = [&](size_t nd) {
        size_t o = off;
        off += (nd + 1) & ~size_t(1);
        return (int)o;
    };
    a->ND = derived_entries(ct.la, ct.lb);
    a->PST = (15 * a->ND) | 1;
    a->Ws = (ct.nab * ct.ncd) | 1;
    a->Eks = (KK * ct.Tcd) | 1;
    a->NDk = derived_entries(ct.lc, ct.ld);
    a->PSTk = (15 * a->NDk) | 1;
    a->Ebs = both ? (KB * ct.Tab) | 1 : 0;
    a->Ys = both ? (ct.nab * ct.nhk2) | 1 : 0;
    a->o_q = take((size_t)TQ * 3);  // (b, k, kb, kk) as int32, then the quartet index
    a->o_W = take((size_t)TQ * a->Ws);
    a->o_Pb = take((size_t)TQ * KB * PS_N);
    a->o_Pk = take((size_t)TQ * KK * PS_N);
    a->o_Ek = take((size_t)TQ * a->Eks);
    a->o_D = take((size_t)TQ * IC * a->PST);
    // the auxiliary integrals; at the end of a tile the ket's derived tables
    // take their place (single launch)
    a->o_R = take(std::max((size_t)ct.nhl2 * ((TQ * IC * KK) | 1), both ? (size_t)TQ * KK * a->PSTk : 0));
    a->Xs = ct.ncd | 1;
    a->XQ = (ct.nhb2 * a->Xs) | 1;
    a->o_X = take(vform ? 0 : (size_t)a->XQ * TQ * IC);
    a->o_ch = take((size_t)TQ * IC * 8);
    a->Vs = (KK * ct.nab * ct.nhk) | 1;
    a->o_V = take(vform ? (size_t)TQ * a->Vs : 0);
    a->o_pq = take(vform ? ((size_t)ct.nhb2 * ct.nhk * 2 + 7) / 8 : 0);
    a->o_Eb = take((size_t)TQ * a->Ebs);
    a->o_Y = take((size_t)TQ * KK * a->Ys);
    a->o_chk = take(both ? (size_t)TQ * KK * 8 : 0);
    a->o_Dk = a->o_R;
    *bytes = off * 8;
    a->TQ = TQ;
    a->IC = IC;
    a->vform = vform;
    a->both = both;
    return *bytes <= (size_t)max_smem_optin();
}

// Form and tile shape (TQ quartets, IC bra primitives per stage pass): the
// feasible pair with the lowest modelled time per quartet.  Each stage pass
// costs its rounds of kGT items times the FP64 work of one item, plus a
// barrier; a tile makes ceil(KB / IC) passes.  The X form's pass forms X'
// over every (p', cd) and contracts it with W per channel item; the V form
// contracts W with the ket E products once per tile and forms each channel
// item's T from V and the auxiliary integrals.  A single launch (both = 1)
// adds, per pass, Y' over (k, ab, q') and, per tile, the ket's derived tables
// and channel items.  Shapes that leave room for two CTAs per SM (so one
// CTA's barriers overlap the other's work) are preferred whenever one exists.
// *cost_out: the modelled time per quartet of the pick.
static bool grad_plan_within(const ClassTables& ct, int KB, int KK, int nit, int nitk, int64_t nq, int both,
                             size_t limit, GradArgs* a, size_t* bytes, double* cost_out);

static bool grad_plan(const ClassTables& ct, int KB, int KK, int nit, int nitk, int64_t nq, int both, GradArgs* a,
                      size_t* bytes, double* cost_out)
{
    const size_t two_per_sm = (size_t)smem_per_sm() / 2 - 1024;
    for (int pass = 0; pass < 2; ++pass) {
        if (grad_plan_within(ct, KB, KK, nit, nitk, nq, both, pass == 0 ? two_per_sm : (size_t)max_smem_optin(), a,
                             bytes, cost_out))
            return true;
    }
    return false;
}

static bool grad_plan_within(const ClassTables& ct, int KB, int KK, int nit, int nitk, int64_t nq, int both,
                             size_t limit, GradArgs* a, size_t* bytes, double* cost_out)
{
    double best = -1.0;
    GradArgs pick{};
    size_t pick_bytes = 0;
    const int ND = derived_entries(ct.la, ct.lb), NDk = derived_entries(ct.lc, ct.ld);
    const int forms = (g_grad_form_mask.load() & 3) ? (g_grad_form_mask.load() & 3) : 3;  // neither bit: both
    for (int vform = 0; vform < 2; ++vform)
    for (int TQ = 32; TQ >= 1; TQ /= 2) {
        if (!(forms >> vform & 1)) break;
        if (TQ > 1 && TQ > nq) continue;
        for (int IC = KB; IC >= 1; IC = IC == 1 ? 0 : (IC + 1) / 2) {
            GradArgs t = *a;
            size_t b = 0;
            if (!grad_layout(ct, KB, KK, TQ, IC, vform, both, &t, &b) || b > limit) continue;
            auto rounds = [](double n) { return std::ceil(n / kGT); };
            const double kBarrier = 60.0;
            double common = rounds((double)TQ * IC * KK) * (3.0 * ct.nhl2 + 60.0) +
                            rounds((double)TQ * IC * 3 * ND) * 14.0;
            if (both)  // Y' of the chunk: per (q, ab, q') and four ket primitives, its terms over the chunk's
                       // bra primitives (two lookups per term, an E value and four products per primitive)
                common += rounds((double)TQ * ((KK + 3) / 4) * ct.nab * ct.nhk2) *
                              ((3.0 + 6.0 * IC) * ct.Tab / ct.nab + 12.0) +
                          kBarrier;
            double cost;
            // a term's index lookup and scattered load cost about as much as
            // its FMAs over the ket primitives: weight 2 KK + 1.5 (X's ket
            // transform) and 2 KK + 2.5 (V's T, one p'+q lookup per term)
            if (!vform) {
                const double pass =
                    common + rounds((double)TQ * IC * ct.nhb2 * ct.ncd) * ((2.0 * KK + 1.5) * ct.Tcd / ct.ncd + 8.0) +
                    rounds((double)TQ * IC * nit) * (2.0 * ct.ncd + 40.0) + 4.0 * kBarrier;
                cost = std::ceil((double)KB / IC) * pass;
            } else {
                const double pass =
                    common + rounds((double)TQ * IC * nit) * ((2.0 * KK + 2.5) * ct.nhk + 40.0) + 3.0 * kBarrier;
                const double vstage =
                    rounds((double)TQ * KK * ct.nab * ct.nhk) * (3.5 * ct.Tcd / ct.nhk + 8.0) + kBarrier;
                cost = vstage + std::ceil((double)KB / IC) * pass;
            }
            if (both)  // the ket's derived tables and channel items, once per tile
                cost += rounds((double)TQ * KK * 3 * NDk) * 16.0 + rounds((double)TQ * KK * nitk) * (2.0 * ct.nab + 40.0) +
                        3.0 * kBarrier;
            cost /= TQ;
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
    if (cost_out) *cost_out = best;
    return true;
}

// The ket terms of a class grouped by their Hermite function q (for the V
// form): vstart[q]..vstart[q+1] index vlist, whose entries are t | cd << 16.
// Built from the class tables' own term list, once per class table.
struct VList {
    int* vstart = nullptr;
    int* vlist = nullptr;
};

static const VList* get_vlist(const ClassTables& ct, cudaStream_t st, int* err)
{
    static std::map<std::pair<int, const void*>, VList> tabs;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(dev, (const void*)ct.ket_q);
    auto it = tabs.find(key);
    if (it != tabs.end()) return &it->second;
    std::vector<int> start(ct.ncd + 1);
    std::vector<int16_t> q(ct.Tcd);
    if (cudaMemcpyAsync(start.data(), ct.ket_start, sizeof(int) * (ct.ncd + 1), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(q.data(), ct.ket_q, sizeof(int16_t) * ct.Tcd, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *err = ERI_ECUDA;
        return nullptr;
    }
    std::vector<int> vstart(ct.nhk + 1, 0), vlist(ct.Tcd);
    for (int t = 0; t < ct.Tcd; ++t) ++vstart[q[t] + 1];
    for (int h = 0; h < ct.nhk; ++h) vstart[h + 1] += vstart[h];
    std::vector<int> fill(vstart.begin(), vstart.end() - 1);
    for (int cd = 0; cd < ct.ncd; ++cd)
        for (int t = start[cd]; t < start[cd + 1]; ++t) vlist[fill[q[t]]++] = t | (cd << 16);
    VList v;
    if (cudaMalloc(&v.vstart, sizeof(int) * (ct.nhk + 1)) != cudaSuccess ||
        cudaMalloc(&v.vlist, sizeof(int) * std::max(ct.Tcd, 1)) != cudaSuccess) {
        *err = ERI_ENOMEM;
        return nullptr;
    }
    if (cudaMemcpyAsync(v.vstart, vstart.data(), sizeof(int) * (ct.nhk + 1), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(v.vlist, vlist.data(), sizeof(int) * ct.Tcd, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *err = ERI_ECUDA;
        return nullptr;
    }
    return &(tabs[key] = v);
}

// The quartet order and the two tile queues, shared by the two launches.
struct GradOrder {
    int64_t* order = nullptr;            // NULL: the identity
    unsigned long long* queue = nullptr;
};

// One launch: the channels of the kernel's bra.  bra/ket are the kernel's
// lists (the caller's ket/bra when swap = 1); nbra_o/nket_o are the caller's.
// What a launch_grad call did or leaves to do (its `next`).
enum { GRAD_DONE = 0, GRAD_SECOND = 1, GRAD_ONE_SWAPPED = 2 };

// One adjoint launch.  bra/ket are the kernel's lists (the caller's ket/bra
// when swap = 1); nbra_o/nket_o are the caller's.  mode 0 (the call's first
// launch, caller's orientation): picks, by the cost model, one launch for
// every channel in this orientation (launched here), one in the other
// orientation (*next = GRAD_ONE_SWAPPED, nothing launched), or two launches
// (this side's channels here, *next = GRAD_SECOND).  mode 1: the second of
// two launches; mode 2: one launch for every channel, in this orientation.
static int launch_grad(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                       int64_t nket, const int64_t* quartets, int64_t nq, const double* W, double* gc, double* ge,
                       int swap, int64_t nbra_o, int64_t nket_o, GradOrder* ord, cudaStream_t st, int mode, int* next)
{
    const ClassTables* ct = nullptr;
    PairTables pb{}, pk{};
    int KB = 0, KK = 0, kmax[4];
    // a single launch needs the pair tables of both sides raised and the E
    // products of both; otherwise the kernel bra's raised tables suffice
    const int mask = g_grad_form_mask.load();
    const bool allow_one = (mask & 4) != 0 && g_grad_force != 2,
               allow_two = ((mask & 8) || !(mask & 12)) && g_grad_force != 1;
    const bool may_one = mode == 2 || (mode == 0 && allow_one);
    // the quartet indices refer to the caller's lists: validated by the first call only
    int mixed = 0;
    int err = prepare_batch(cls, basis, bra, nbra, ket, nket, mode == 0 ? quartets : nullptr, mode == 0 ? nq : 0,
                            may_one ? 2 : 1, st, &ct, &pb, &pk, &KB, &KK, kmax, 0, nullptr, 0, 0, &mixed);
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
    a.ket_sh = ket;
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
    const ItemTable* items = get_items(st, &err);
    if (!items) return err;
    a.items = items->list[ct->la][ct->lb];
    a.nit = items->n[ct->la][ct->lb];
    a.kitems = items->list[ct->lc][ct->ld];
    a.nitk = items->n[ct->lc][ct->ld];
    const VList* vl = get_vlist(*ct, st, &err);
    if (!vl) return err;
    a.vstart = vl->vstart;
    a.vlist = vl->vlist;
    size_t bytes = 0;
    bool one = false;
    if (next) *next = GRAD_DONE;
    if (mode == 2) {
        one = grad_plan(*ct, KB, KK, a.nit, a.nitk, a.nq, 1, &a, &bytes, nullptr);
        if (!one) return ERI_EINVAL;
    } else if (mode == 0 && allow_one) {
        // modelled cost per quartet of: one launch in this orientation, one in
        // the other (the sides exchanged), two launches
        const ClassTables* ctk = get_class_tables(cls.lc, cls.ld, cls.la, cls.lb, st, &err);
        if (!ctk) return err;
        GradArgs a1 = a, a0 = a, as = a, aw = a;
        size_t b1 = 0, b0 = 0, bs = 0, bw = 0;
        double c1 = 0.0, c0 = 0.0, cs = 0.0, cw = 0.0;
        const bool ok1 = grad_plan(*ct, KB, KK, a.nit, a.nitk, a.nq, 1, &a1, &b1, &c1);
        const bool okw = grad_plan(*ctk, KK, KB, a.nitk, a.nit, a.nq, 1, &aw, &bw, &cw);
        const bool ok2 = allow_two && grad_plan(*ct, KB, KK, a.nit, a.nitk, a.nq, 0, &a0, &b0, &c0) &&
                         grad_plan(*ctk, KK, KB, a.nitk, a.nit, a.nq, 0, &as, &bs, &cs);
        double best = 1e300;
        int pick = -1;  // 0: one here, 1: one swapped, 2: two
        if (ok1 && c1 < best) { best = c1; pick = 0; }
        if (okw && cw < best) { best = cw; pick = 1; }
        if (ok2 && c0 + cs < best) { best = c0 + cs; pick = 2; }
        if (pick == 1) {
            if (next) *next = GRAD_ONE_SWAPPED;
            return ERI_OK;  // validated; the swapped call builds its own tables and order
        }
        if (pick == 0) {
            one = true;
            a = a1;
            bytes = b1;
        }
    }
    if (!one) {
        if (!grad_plan(*ct, KB, KK, a.nit, a.nitk, a.nq, 0, &a, &bytes, nullptr)) return ERI_EINVAL;
        if (mode == 0 && next) *next = GRAD_SECOND;
    }
    if (one) {
        g_last_grad_form[0] = a.vform;
        g_last_grad_form[1] = swap ? ERI_GRAD_ONE_SWAPPED : ERI_GRAD_ONE;
    } else {
        g_last_grad_form[swap] = a.vform;
    }
    a.ntiles = (a.nq + a.TQ - 1) / a.TQ;
    if (!ord->queue) {  // the call's first kernel launch: order (sorted if the batch mixes degrees); a second reuses it
        err = build_order(quartets, a.nq, nbra_o, pb.kp, pk.kp, KB, KK, swap, mixed, st, &ord->order, &ord->queue);
        if (err != ERI_OK) return err;
    }
    a.order = ord->order;
    a.next = ord->queue + swap;
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

// One adjoint call (arguments validated): the bra's channels, then, unless
// that launch covered every channel, the ket's with the sides exchanged.
static int run_grad(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                    const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nq, const double* W,
                    double* grad_centres, double* grad_exps, cudaStream_t st)
{
    int err = ERI_OK;
    GradOrder order;
    g_last_grad_form[0] = g_last_grad_form[1] = -1;
    int next = GRAD_DONE;
    err = launch_grad(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, W, grad_centres, grad_exps, 0, nbra,
                      nket, &order, st, 0, &next);
    if (err != ERI_OK || next == GRAD_DONE) return err;
    return launch_grad(eri_class_t{cls.lc, cls.ld, cls.la, cls.lb}, basis, ket_pairs, nket, bra_pairs, nbra, quartets,
                       nq, W, grad_centres, grad_exps, 1, nbra, nket, &order, st, next == GRAD_ONE_SWAPPED ? 2 : 1,
                       nullptr);
}

// Timed choice between one launch and two, on the first large list-form
// batch of a class (per device): each scheme runs twice on the batch's first
// kGradTuneQuartets quartets, into scratch gradients (the weights read are
// the caller's, in range, whatever they mean for the shorter list), and the
// faster second run decides for the class.  The cost model still picks the
// single launch's orientation and each launch's form.  Returns 1 (one
// launch), 2 (two), or 0 (no decision: the model's pick).
constexpr int64_t kGradTuneMin = 65536, kGradTuneQuartets = 32768;
static std::map<std::tuple<int, int, int, int, int>, int> g_grad_scheme;
static std::mutex g_grad_scheme_mu;

static int timed_grad_scheme(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                             const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nq,
                             const double* W, cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const auto key = std::make_tuple(dev, cls.la, cls.lb, cls.lc, cls.ld);
    {
        std::lock_guard<std::mutex> lk(g_grad_scheme_mu);
        auto it = g_grad_scheme.find(key);
        if (it != g_grad_scheme.end()) return it->second;
    }
    int err = ERI_OK;
    const size_t ng = 3 * (size_t)basis->natom + (size_t)basis->nprim;
    double* scratch = (double*)aux_workspace(sizeof(double) * ng, &err);
    if (!scratch) return 0;
    const int64_t n = std::min(nq, kGradTuneQuartets);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0;
    }
    float ms[3] = {0.f, 0.f, 0.f};
    bool ok = true;
    for (int scheme = 1; scheme <= 2 && ok; ++scheme) {
        g_grad_force = scheme;
        for (int rep = 0; rep < 2 && ok; ++rep) {
            ok &= cudaEventRecord(e0, st) == cudaSuccess;
            ok &= run_grad(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, n, W, scratch,
                           scratch + 3 * basis->natom, st) == ERI_OK;
            ok &= cudaEventRecord(e1, st) == cudaSuccess;
            ok &= cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms[scheme], e0, e1) == cudaSuccess;
        }
    }
    g_grad_force = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) {
        cudaGetLastError();
        return 0;
    }
    const int pick = ms[1] <= ms[2] ? 1 : 2;
    std::lock_guard<std::mutex> lk(g_grad_scheme_mu);
    g_grad_scheme[key] = pick;
    return pick;
}

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
    const int mask = g_grad_form_mask.load();
    const bool both = (mask & 4) && ((mask & 8) || !(mask & 12));
    int scheme = 0;
    if (both && quartets && nqq >= kGradTuneMin)
        scheme = timed_grad_scheme(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, W, st);
    g_grad_force = scheme;
    err = run_grad(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, W, grad_centres, grad_exps, st);
    g_grad_force = 0;
    return err;
}

extern "C" int eri_last_grad_forms(int32_t* bra_form, int32_t* ket_form)
{
    if (!bra_form || !ket_form) return ERI_EINVAL;
    if (g_last_grad_form[0] < 0 || g_last_grad_form[1] < 0) return ERI_EINVAL;
    *bra_form = g_last_grad_form[0];
    *ket_form = g_last_grad_form[1];
    return ERI_OK;
}

extern "C" int eri_set_grad_forms(int32_t mask)
{
    if (mask < 0 || mask > 0xF) return ERI_EINVAL;
    return g_grad_form_mask.exchange(mask ? mask : 0xF);
}
