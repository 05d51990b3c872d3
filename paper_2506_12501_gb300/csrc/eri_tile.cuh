// eri_tile.cuh -- the forward tile of quartets, shared by the per-class
// kernel (eri_fwd.cu) and the plan's persistent kernel (eri_plan.cu).
//
// A tile is TQ quartets of one class.  Staged through shared memory:
//   A. [r]^(0) for every primitive quartet (Boys function, Eq. 0m, Eq. r-rr);
//   B. ket transform and ket contraction (Eq. ket-from-hermite):
//      X[p][cd] = sum_k sum_q E^cd_{k,q} [p+q]^(0)_{ik};
//   C. bra transform and bra contraction (Eq. bra-from-hermite):
//      (ab|cd) += sum_p E^ab_{i,p} X[p][cd], over bra primitives i,
// then coalesced stores of the quartet-fastest output, or digestion into
// sum W (ab|cd) with W_abcd = D_ab D_cd.
#pragma once

#include "eri_device.cuh"
#include "eri_internal.h"

namespace eri {

constexpr int kNT = 256;   // threads per CTA of the tile kernels (plans; most eri_batch tiles)
constexpr int kNTWide = 512;  // eri_batch tiles that fill an SM's shared memory alone
constexpr int kNACC = 16;  // outputs per thread held in registers

// Split form: bra Hermite functions per lane in the blocked ket stage (one
// warp per (quartet, cd)) for a bra range of nhbu functions; 0: not blocked.
__host__ __device__ constexpr int split_block_width(int nhbu)
{
    return nhbu >= 72 && nhbu <= 96 ? 3 : (nhbu >= 48 && nhbu <= 64 ? 2 : 0);
}
// ket E rows per warp in the ring of the blocked split stage
constexpr int kRingRows = 3;

// ---- split precision: a double x is carried as hi + lo with hi = fl32(x),
// lo = fl32(x - hi) (about 48 significant bits); products of two such pairs
// keep the exact error of hi*hi (from an FMA) and the two cross terms, and
// sums are compensated (TwoSum), so a long sum keeps about 44 bits.  The
// rounded intrinsics keep the compiler from contracting the error terms.
__device__ __forceinline__ float2 split_f64(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// (S, c) += a * b with a, b split pairs
__device__ __forceinline__ void ff_mac(float2 a, float2 b, float& S, float& c)
{
    const float p = __fmul_rn(a.x, b.x);
    const float pe = __fmaf_rn(a.x, b.x, -p);
    const float t = __fadd_rn(S, p);
    const float z = __fsub_rn(t, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(p, z));
    S = t;
    c = __fadd_rn(c, __fadd_rn(err, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, pe))));
}

// ---- the same arithmetic on two independent chains at once: packed FP32
// pairs (PTX f32x2, one 64-bit register holding two floats)
__device__ __forceinline__ uint64_t f2_pack(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ff_mac on two chains: (S, c) += a * b lane-wise, with a = (ah, al) and
// b = (bh, bl) split pairs of each chain, nah = -ah.  The same operations as
// ff_mac: q = fl(-ah bh) is the rounded product negated (exact), so the
// exact product error is fma(ah, bh, q), and the TwoSum of S and -q is
// written with q.
__device__ __forceinline__ void ff_mac2(uint64_t ah, uint64_t al, uint64_t nah, uint64_t bh, uint64_t bl,
                                        uint64_t& S, uint64_t& c)
{
    const uint64_t q = f2_mul(nah, bh);
    const uint64_t pe = f2_fma(ah, bh, q);
    const uint64_t t = f2_sub(S, q);
    const uint64_t z = f2_sub(t, S);
    const uint64_t err = f2_sub(f2_sub(S, f2_sub(t, z)), f2_add(q, z));
    S = t;
    c = f2_add(c, f2_add(err, f2_fma(ah, bl, f2_fma(al, bh, pe))));
}

// Loads and stores with an L2 eviction priority (a cache policy made by
// createpolicy).  A large quartet's ket E products are re-read for every bra
// primitive while its bra E products and its accumulating outputs stream
// through: the first are marked to stay in L2, the others to leave it first.
__device__ __forceinline__ uint64_t policy_keep()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_stream()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ld_hint(const float2* p, uint64_t pol)
{
    float2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_hint(const double* p, uint64_t pol)
{
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void prefetch_l1(const void* p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
// 8-byte asynchronous copy global -> shared (completes per commit group)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, uint64_t pol)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void st_hint(double* p, double v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}

struct FwdArgs {
    ClassTables ct;
    const double* boys;
    const RStep* rsteps;
    const double* bra_ps;
    const double* bra_E;
    const int32_t* bra_kp;
    const double* ket_ps;
    const double* ket_E;
    const int32_t* ket_kp;
    const int64_t* quartets;  // NULL: product form
    const int64_t* order;     // processing order of the quartet indices (NULL: identity)
    int64_t nq, nbra, nket;   // nbra/nket: the caller's lists (before any swap)
    int swap;                 // 1: the kernel's bra is the caller's ket
    int nab_o, ncd_o;         // component-pair counts of the caller's class
    double* out;
    int TQ, KB, KK, IC;
    int e_smem, acc_regs;
    int sEbS, sEkS;           // per-quartet strides of staged E (doubles)
    int o_Eb, o_Ek, o_Pb, o_Pk, o_R, o_X, o_tab, o_q;  // smem offsets (doubles)
    int o_hB, o_geo;          // horizontal-recursion form: second buffer, A-B and C-D per quartet
    int o_dj;                 // Coulomb digestion scratch: [TQ] weights, [nab] bra sums
    int o_Ei;                 // one-quartet tile with E not staged: the bra E products of the current bra primitive, [Tab] (-1: none)
    int o_Er;                 // split blocked ket stage with E not staged: a ring of three ket E rows per warp (-1: none)
    int r_pairs;              // auxiliary integrals in the paired layout (split form, blocked ket stage)
    int64_t ntiles;
    // work-queue mode (plans): one bra pair, consecutive ket pairs
    int mode;                 // 0: list/product batch, 1: ranged (bra rbra, kets rk0..)
    int64_t rbra, rk0, rq0;   // ranged: bra index, first ket index, list index of that quartet
    // digestion (energy = sum W (ab|cd), W_abcd = D_ab D_cd) instead of stores
    double* energy;           // non-null: digest; out is not written
    double* Jmat;             // non-null (plans): Coulomb digestion into J' [nbf][nbf]; out is not written
    double* Kmat;             // non-null (plans): exchange digestion into K' [nbf][nbf]; out is not written
    const double* D;          // [nbf][nbf]
    int nbf;
    const int32_t* bf_off;    // [nshell] first Cartesian function of each shell
    const int32_t* bra_sh;    // kernel's bra pairs as shell indices [nbra][2]
    const int32_t* ket_sh;    // kernel's ket pairs [nket][2]
    // horizontal-recursion form: A-B and C-D from the shell centres
    const double* centres;
    const int32_t* shell_atom;
};

// Copy a tile shape into the kernel arguments.
inline void set_tile(FwdArgs& a, const TilePlan& tp)
{
    a.TQ = tp.TQ;
    a.IC = tp.IC;
    a.e_smem = tp.e_smem;
    a.acc_regs = tp.acc_regs;
    a.sEbS = tp.sEbS;
    a.sEkS = tp.sEkS;
    a.o_Eb = tp.o_Eb;
    a.o_Ek = tp.o_Ek;
    a.o_Pb = tp.o_Pb;
    a.o_Pk = tp.o_Pk;
    a.o_R = tp.o_R;
    a.o_X = tp.o_X;
    a.o_tab = tp.o_tab;
    a.o_q = tp.o_q;
    a.o_hB = tp.o_hB;
    a.o_geo = tp.o_geo;
    a.o_dj = tp.o_dj;
    a.o_Ei = tp.o_Ei;
    a.o_Er = tp.o_Er;
    a.r_pairs = tp.r_pairs;
}

struct Strided {
    double* p;
    int s;
    __device__ __forceinline__ double& operator[](int e) const { return p[(size_t)e * s]; }
};

// Output position of the kernel's component pair (ab, cd) of quartet qq, in
// the caller's layout (ab and cd exchange roles when the sides were swapped).
__device__ __forceinline__ int64_t out_index(const FwdArgs& a, int64_t qq, int ab, int cd)
{
    const int abo = a.swap ? cd : ab, cdo = a.swap ? ab : cd;
    if (a.quartets || a.mode == 1) return qq + a.nq * ((int64_t)abo * a.ncd_o + cdo);
    const int64_t bra = qq % a.nbra, ket = qq / a.nbra;
    return bra + a.nbra * (abo + (int64_t)a.nab_o * (cdo + (int64_t)a.ncd_o * ket));
}

// The kernel's (bra, ket) pair indices of quartet qq.
__device__ __forceinline__ void quartet_pairs(const FwdArgs& a, int64_t qq, int* b, int* k)
{
    int64_t ob, ok;
    if (a.mode == 1) {
        *b = (int)a.rbra;
        *k = (int)(a.rk0 + (qq - a.rq0));
        return;
    }
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

// Stage C inner sum: acc + sum_{u in [u0,u1)} E^ab_u X[p_u][cd] of one
// quartet and one bra primitive (E term u at Eb[u * KB]).  FP64: one chain
// from the accumulator (no DADD); the split form adds its compensated float
// sum to acc as a double (3 FP64 ops).
template <bool SPLIT>
__device__ __forceinline__ double bra_sum(const double* Eb, int KB, const double* sX, int u0, int u1,
                                          const int16_t* s_bp, int ncd, int cd, int TQ, int q, double acc)
{
    if (!SPLIT) {
        double v = acc;
        for (int u = u0; u < u1; ++u) v = fma(Eb[(size_t)u * KB], sX[(s_bp[u] * ncd + cd) * TQ + q], v);
        return v;
    } else {
        const float2* E2 = reinterpret_cast<const float2*>(Eb);
        const float2* X2 = reinterpret_cast<const float2*>(sX);
        float Sa = 0.f, ca = 0.f, Sb = 0.f, cb = 0.f;
        int u = u0;
        for (; u + 1 < u1; u += 2) {
            ff_mac(E2[(size_t)u * KB], X2[(s_bp[u] * ncd + cd) * TQ + q], Sa, ca);
            ff_mac(E2[(size_t)(u + 1) * KB], X2[(s_bp[u + 1] * ncd + cd) * TQ + q], Sb, cb);
        }
        if (u < u1) ff_mac(E2[(size_t)u * KB], X2[(s_bp[u] * ncd + cd) * TQ + q], Sa, ca);
        return acc + (((double)Sa + (double)Sb) + ((double)ca + (double)cb));
    }
}

// Class tables into shared memory (each CTA, whenever the class changes).
template <int NT>
__device__ __forceinline__ void stage_class_tables(const FwdArgs& a, double* sm)
{
    const ClassTables& ct = a.ct;
    const int tid = threadIdx.x;
    int* s_bstart = reinterpret_cast<int*>(sm + a.o_tab);
    int* s_kstart = s_bstart + ct.nab + 1;
    int16_t* s_bp = reinterpret_cast<int16_t*>(s_kstart + ct.ncd + 1);
    int16_t* s_kq = s_bp + ct.Tab;
    int16_t* s_pq = s_kq + ct.Tcd;
    for (int i = tid; i <= ct.nab; i += NT) s_bstart[i] = ct.bra_start[i];
    for (int i = tid; i <= ct.ncd; i += NT) s_kstart[i] = ct.ket_start[i];
    for (int i = tid; i < ct.Tab; i += NT) s_bp[i] = ct.bra_p[i];
    for (int i = tid; i < ct.Tcd; i += NT) s_kq[i] = ct.ket_q[i];
    for (int i = tid; i < ct.nhb * ct.nhk; i += NT) s_pq[i] = ct.pq[i];
}

// W_abcd = D_ab D_cd for the kernel's component pair (ab, cd) of quartet
// (b, k); W is symmetric in bra and ket, so the side order does not matter.
__device__ __forceinline__ double digest_weight(const FwdArgs& a, int b, int k, int ab, int cd)
{
    const ClassTables& ct = a.ct;
    const int ncb = (ct.lb + 1) * (ct.lb + 2) / 2, ncd2 = (ct.ld + 1) * (ct.ld + 2) / 2;
    const int ia = a.bf_off[a.bra_sh[2 * b]] + ab / ncb, ib = a.bf_off[a.bra_sh[2 * b + 1]] + ab % ncb;
    const int ic = a.bf_off[a.ket_sh[2 * k]] + cd / ncd2, id = a.bf_off[a.ket_sh[2 * k + 1]] + cd % ncd2;
    return a.D[(size_t)ia * a.nbf + ib] * a.D[(size_t)ic * a.nbf + id];
}

// Coulomb digestion of one tile of a plan work item (one bra pair, the
// tile's ket pairs).  V[ab][cd][q] (index q + TQ (cd + ncd ab)) holds the
// tile's contracted integrals.  Every unique shell quartet stands for its
// distinct images under the 8 index permutations; with s = 1/2 for each of
// a == b, c == d and (ab) == (cd) (shells), and D symmetric,
//   J'[a][b] += 2s sum_cd (ab|cd) D[c][d],   J'[c][d] += 2s sum_ab (ab|cd) D[a][b],
// and J = J' + J'^T afterwards gives J_uv = sum over all (ls) of (uv|ls) D_ls.
// The bra sums are reduced over the tile in shared memory first (one global
// atomic per ab), the ket sums take one global atomic per (q, cd).
template <int NT>
static __device__ void digest_coulomb(const FwdArgs& a, const double* V, int nqt, const int* s_q, double* s_dj)
{
    const ClassTables& ct = a.ct;
    const int TQ = a.TQ, nab = ct.nab_f, ncd = ct.ncd_f, tid = threadIdx.x;
    const int ncb = (ct.lb + 1) * (ct.lb + 2) / 2, ncdd = (ct.ld + 1) * (ct.ld + 2) / 2;
    double* s_w = s_dj;        // [TQ]
    double* s_jb = s_dj + TQ;  // [nab]
    const int b = s_q[0];
    const int sa = a.bra_sh[2 * b], sb = a.bra_sh[2 * b + 1];
    const int oa = a.bf_off[sa], ob = a.bf_off[sb];
    for (int q = tid; q < TQ; q += NT) {
        double w = 0.0;
        if (q < nqt) {
            const int k = s_q[4 * q + 1];
            const int sc = a.ket_sh[2 * k], sd = a.ket_sh[2 * k + 1];
            w = 2.0;
            if (sa == sb) w *= 0.5;
            if (sc == sd) w *= 0.5;
            if ((sa == sc && sb == sd) || (sa == sd && sb == sc)) w *= 0.5;
        }
        s_w[q] = w;
    }
    for (int i = tid; i < nab; i += NT) s_jb[i] = 0.0;
    __syncthreads();
    for (int item = tid; item < TQ * ncd; item += NT) {
        const int q = item % TQ, cd = item / TQ;
        if (q >= nqt) continue;
        double sum = 0.0;
        for (int ab = 0; ab < nab; ++ab)
            sum = fma(V[q + TQ * (cd + ncd * ab)], a.D[(size_t)(oa + ab / ncb) * a.nbf + ob + ab % ncb], sum);
        const int k = s_q[4 * q + 1];
        const int ic = a.bf_off[a.ket_sh[2 * k]] + cd / ncdd, id = a.bf_off[a.ket_sh[2 * k + 1]] + cd % ncdd;
        atomicAdd(&a.Jmat[(size_t)ic * a.nbf + id], s_w[q] * sum);
    }
    for (int item = tid; item < TQ * nab; item += NT) {
        const int q = item % TQ, ab = item / TQ;
        if (q >= nqt) continue;
        const int k = s_q[4 * q + 1];
        const int oc = a.bf_off[a.ket_sh[2 * k]], od = a.bf_off[a.ket_sh[2 * k + 1]];
        double sum = 0.0;
        for (int cd = 0; cd < ncd; ++cd)
            sum = fma(V[q + TQ * (cd + ncd * ab)], a.D[(size_t)(oc + cd / ncdd) * a.nbf + od + cd % ncdd], sum);
        atomicAdd(&s_jb[ab], s_w[q] * sum);
    }
    __syncthreads();
    for (int ab = tid; ab < nab; ab += NT)
        atomicAdd(&a.Jmat[(size_t)(oa + ab / ncb) * a.nbf + ob + ab % ncb], s_jb[ab]);
}

// Exchange digestion of one tile of a plan work item, from the same V as
// digest_coulomb.  With s as there (1/2 per coincident shell pair or pair
// of pairs), every unique quartet adds
//   K'[a][c] += s sum_bd (ab|cd) D[b][d],   K'[b][c] += s sum_ad (ab|cd) D[a][d],
//   K'[a][d] += s sum_bc (ab|cd) D[b][c],   K'[b][d] += s sum_ac (ab|cd) D[a][c],
// (its images with the bra and ket exchanged are the transposes), and
// K = K' + K'^T afterwards gives K_ul = sum over all (vs) of (uv|ls) D_vs.
// One global atomic per (quartet, target element).
template <int NT>
static __device__ void digest_exchange(const FwdArgs& a, const double* V, int nqt, const int* s_q, double* s_dj)
{
    const ClassTables& ct = a.ct;
    const int TQ = a.TQ, ncd = ct.ncd_f, tid = threadIdx.x;
    const int na = (ct.la + 1) * (ct.la + 2) / 2, nb = (ct.lb + 1) * (ct.lb + 2) / 2;
    const int nc = (ct.lc + 1) * (ct.lc + 2) / 2, nd = (ct.ld + 1) * (ct.ld + 2) / 2;
    double* s_w = s_dj;  // [TQ]
    const int b0 = s_q[0];
    const int sa = a.bra_sh[2 * b0], sb = a.bra_sh[2 * b0 + 1];
    const int oa = a.bf_off[sa], ob = a.bf_off[sb];
    const double* D = a.D;
    const size_t n = (size_t)a.nbf;
    __syncthreads();  // the Coulomb digestion may still read s_dj
    for (int q = tid; q < TQ; q += NT) {
        double w = 0.0;
        if (q < nqt) {
            const int k = s_q[4 * q + 1];
            const int sc = a.ket_sh[2 * k], sd = a.ket_sh[2 * k + 1];
            w = 1.0;
            if (sa == sb) w *= 0.5;
            if (sc == sd) w *= 0.5;
            if ((sa == sc && sb == sd) || (sa == sd && sb == sc)) w *= 0.5;
        }
        s_w[q] = w;
    }
    __syncthreads();
    const int n0 = na * nc, n1 = n0 + nb * nc, n2 = n1 + na * nd, n3 = n2 + nb * nd;
    for (int item = tid; item < TQ * n3; item += NT) {
        const int q = item % TQ, r = item / TQ;
        if (q >= nqt) continue;
        const int k = s_q[4 * q + 1];
        const int oc = a.bf_off[a.ket_sh[2 * k]], od = a.bf_off[a.ket_sh[2 * k + 1]];
        const double* Vq = V + q;  // V[ab][cd] at Vq[TQ * (cd + ncd * ab)]
        double sum = 0.0;
        size_t tgt;
        if (r < n0) {  // (a, c): over b, d
            const int x = r / nc, y = r % nc;
            for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nd; ++j)
                    sum = fma(Vq[TQ * ((y * nd + j) + ncd * (x * nb + i))], D[(ob + i) * n + od + j], sum);
            tgt = (oa + x) * n + oc + y;
        } else if (r < n1) {  // (b, c): over a, d
            const int x = (r - n0) / nc, y = (r - n0) % nc;
            for (int i = 0; i < na; ++i)
                for (int j = 0; j < nd; ++j)
                    sum = fma(Vq[TQ * ((y * nd + j) + ncd * (i * nb + x))], D[(oa + i) * n + od + j], sum);
            tgt = (ob + x) * n + oc + y;
        } else if (r < n2) {  // (a, d): over b, c
            const int x = (r - n1) / nd, y = (r - n1) % nd;
            for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nc; ++j)
                    sum = fma(Vq[TQ * ((j * nd + y) + ncd * (x * nb + i))], D[(ob + i) * n + oc + j], sum);
            tgt = (oa + x) * n + od + y;
        } else {  // (b, d): over a, c
            const int x = (r - n2) / nd, y = (r - n2) % nd;
            for (int i = 0; i < na; ++i)
                for (int j = 0; j < nc; ++j)
                    sum = fma(Vq[TQ * ((j * nd + y) + ncd * (i * nb + x))], D[(oa + i) * n + oc + j], sum);
            tgt = (ob + x) * n + od + y;
        }
        atomicAdd(&a.Kmat[tgt], s_w[q] * sum);
    }
}

// One index of the contracted block mapped to solid harmonics:
// out[(o nout + m) inner + i] = sum_k M[m][k] in[(o nin + k) inner + i].
template <int NT>
static __device__ void contract_index(const double* in, double* out, const double* __restrict__ M, int outer,
                                      int nin, int nout, int inner)
{
    for (int item = threadIdx.x; item < outer * nout * inner; item += NT) {
        const int i = item % inner, r = item / inner, m = r % nout, o = r / nout;
        const double* row = M + m * nin;
        const double* src = in + (size_t)o * nin * inner + i;
        double v = 0.0;
        for (int k = 0; k < nin; ++k) {
            const double c = row[k];
            if (c != 0.0) v = fma(c, src[(size_t)k * inner], v);
        }
        out[item] = v;
    }
    __syncthreads();
}

// Solid-harmonic output: the Cartesian block [ab][cd][q] in buf[cur] becomes
// [ma mb][mc md][q] (m = -l..l on every centre), one centre at a time,
// alternating between buf[0] and buf[1]; returns the final buffer.
template <int NT>
static __device__ const double* to_solid_harmonics(const FwdArgs& a, double* const buf[2], int cur)
{
    const ClassTables& ct = a.ct;
    const int TQ = a.TQ;
    const int na = (ct.la + 1) * (ct.la + 2) / 2, nb = (ct.lb + 1) * (ct.lb + 2) / 2;
    const int nc = (ct.lc + 1) * (ct.lc + 2) / 2, nd = (ct.ld + 1) * (ct.ld + 2) / 2;
    const int sa = 2 * ct.la + 1, sb = 2 * ct.lb + 1, sc = 2 * ct.lc + 1, sd = 2 * ct.ld + 1;
    // (outer, nin, nout, inner) of the four steps: a, b, then c, d
    const int steps[4][4] = {{1, na, sa, nb * nc * nd * TQ},
                             {sa, nb, sb, nc * nd * TQ},
                             {sa * sb, nc, sc, nd * TQ},
                             {sa * sb * sc, nd, sd, TQ}};
    for (int i = 0; i < 4; ++i) {
        if (!ct.c2s[i]) continue;  // l = 0: the identity
        contract_index<NT>(buf[cur], buf[cur ^ 1], ct.c2s[i], steps[i][0], steps[i][1], steps[i][2], steps[i][3]);
        cur ^= 1;
    }
    return buf[cur];
}

// Stage B of the split form for a wide bra Hermite range (32 < nhbu <= 32 P):
// one warp per (quartet, cd); lane l carries the bra Hermite functions
// p = pb0 + l + 32 j, j < P, so that every ket E value loaded (the same for
// the whole warp) feeds P products and the loop trip counts are uniform.
template <int P, int NT>
__device__ __forceinline__ void split_ket_blocked(const FwdArgs& a, int TQ, int IC, int ii, int KK, int KKt,
                                                  int NIs, int ncd, int nhk, const double* sEk, const double* sR,
                                                  double* sX, const int* s_q, const int* s_kstart,
                                                  const int16_t* s_kq, const int16_t* s_pq, float2* ring)
{
    const ClassTables& ct = a.ct;
    const int lane = threadIdx.x & 31, nhb = ct.nhb;
    const uint64_t keep = policy_keep();
    for (int w = threadIdx.x >> 5; w < TQ * ncd; w += NT / 32) {
        const int q = w % TQ, cd = w / TQ;
        const float2* Ek = reinterpret_cast<const float2*>(
            a.e_smem ? sEk + q * a.sEkS : a.ket_E + (size_t)s_q[4 * q + 1] * KK * ct.Tcd);
        const double* Rc = sR + (q * IC + ii) * KK;
        int prow[P];
        float S[P][2], c[P][2];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int p = ct.pb0 + lane + 32 * j;
            prow[j] = (p < nhb ? p : ct.pb0) * nhk;  // lanes past the range read a valid row, results dropped
            S[j][0] = S[j][1] = c[j][0] = c[j][1] = 0.f;
        }
        const int t0 = s_kstart[cd], t1 = s_kstart[cd + 1];
        const bool gl = !a.e_smem;
        if (ring) {
            // the warp's ring of three ket E rows in shared memory: the rows of
            // terms t+1 and t+2 are in flight (asynchronous copies, one commit
            // group per row, possibly empty) while the warp works on term t
            auto issue = [&](int t, int slot) {
                if (t < t1)
                    for (int k = lane; k < KKt; k += 32) cp_async8(ring + slot * KK + k, Ek + (size_t)t * KK + k, keep);
                cp_async_commit();
            };
            issue(t0, 0);
            issue(t0 + 1, 1);
            int slot = 0;
            for (int t = t0; t < t1; ++t) {
                // the slot of term t+2 held term t-1, whose readers passed the
                // warp barrier at the end of the previous term
                issue(t + 2, slot == 0 ? 2 : slot - 1);
                cp_async_wait<2>();
                __syncwarp();
                const int qv = s_kq[t];
                const float2* Rj[P];
#pragma unroll
                for (int j = 0; j < P; ++j)
                    Rj[j] = reinterpret_cast<const float2*>(Rc + (size_t)s_pq[prow[j] + qv] * NIs);
                const float2* Ea = ring + slot * KK;
                int k = 0;
                for (; k + 1 < KKt; k += 2) {
                    const float2 e0 = Ea[k], e1 = Ea[k + 1];
#pragma unroll
                    for (int j = 0; j < P; ++j) {
                        ff_mac(e0, Rj[j][k], S[j][0], c[j][0]);
                        ff_mac(e1, Rj[j][k + 1], S[j][1], c[j][1]);
                    }
                }
                if (k < KKt) {
                    const float2 e0 = Ea[k];
#pragma unroll
                    for (int j = 0; j < P; ++j) ff_mac(e0, Rj[j][k], S[j][0], c[j][0]);
                }
                __syncwarp();
                slot = slot == 2 ? 0 : slot + 1;
            }
            cp_async_wait<0>();  // only empty groups can remain
        }
        // without a ring (or with E staged) the ket E rows of a term (KK float
        // pairs) are read in place; from L2 or DRAM, the lanes prefetch the
        // rows of the next two terms into L1 while the warp works on the
        // current one
        // (each prefetched address lies inside its row: the line of byte
        // min(128 l, 8 KK - 8) for lane l; a row spans at most nline lines)
        const int nline = (KK * 8 + 127) / 128 + 1;
        if (!ring && gl && lane < 2 * nline && t0 + lane / nline < t1)
            prefetch_l1(reinterpret_cast<const char*>(Ek + (t0 + lane / nline) * KK) +
                        min(128 * (lane % nline), 8 * KK - 8));
        for (int t = ring ? t1 : t0; t < t1; ++t) {
            if (gl && lane < nline && t + 2 < t1)
                prefetch_l1(reinterpret_cast<const char*>(Ek + (t + 2) * KK) + min(128 * lane, 8 * KK - 8));
            const int qv = s_kq[t];
            const float2* Rj[P];
#pragma unroll
            for (int j = 0; j < P; ++j) Rj[j] = reinterpret_cast<const float2*>(Rc + (size_t)s_pq[prow[j] + qv] * NIs);
            const float2* Ea = Ek + t * KK;
            int k = 0;
            for (; k + 1 < KKt; k += 2) {
                const float2 e0 = gl ? ld_hint(Ea + k, keep) : Ea[k], e1 = gl ? ld_hint(Ea + k + 1, keep) : Ea[k + 1];
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    ff_mac(e0, Rj[j][k], S[j][0], c[j][0]);
                    ff_mac(e1, Rj[j][k + 1], S[j][1], c[j][1]);
                }
            }
            if (k < KKt) {
                const float2 e0 = gl ? ld_hint(Ea + k, keep) : Ea[k];
#pragma unroll
                for (int j = 0; j < P; ++j) ff_mac(e0, Rj[j][k], S[j][0], c[j][0]);
            }
        }
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int p = ct.pb0 + lane + 32 * j;
            if (p >= nhb) continue;
            // fold the two chains into one split pair (error-free sum of the highs)
            const float t2 = __fadd_rn(S[j][0], S[j][1]), z = __fsub_rn(t2, S[j][0]);
            const float err = __fadd_rn(__fsub_rn(S[j][0], __fsub_rn(t2, z)), __fsub_rn(S[j][1], z));
            const float ch = __fadd_rn(__fadd_rn(c[j][0], c[j][1]), err);
            reinterpret_cast<float2*>(sX)[(p * ncd + cd) * TQ + q] = make_float2(t2, ch);
        }
    }
}

// split_ket_blocked on the paired layout of the auxiliary integrals (r_row_stride):
// each lane's two accumulator chains per bra function run as one packed
// pair, chain 0 over the even ket primitives k and chain 1 over k + 1, so
// one 16-byte load of a row gives both chains' (hi) and (lo) operands and
// each FP32 instruction serves two products.  A tile whose own ket count
// KKt is odd pairs its last primitive with a zero (its paired column is
// zero, and so is the E value taken for it).
template <int P, int NT>
__device__ __forceinline__ void split_ket_paired(const FwdArgs& a, int TQ, int IC, int ii, int KK, int KKr,
                                                 int KKt, int NIs, int ncd, int nhk, const double* sEk,
                                                 const double* sR, double* sX, const int* s_q, const int* s_kstart,
                                                 const int16_t* s_kq, const int16_t* s_pq, float2* ring)
{
    const ClassTables& ct = a.ct;
    const int lane = threadIdx.x & 31, nhb = ct.nhb;
    const uint64_t keep = policy_keep();
    const uint64_t m1 = f2_pack(-1.f, -1.f);
    const int KKe = KKt & ~1;  // ket primitives in full pairs
    for (int w = threadIdx.x >> 5; w < TQ * ncd; w += NT / 32) {
        const int q = w % TQ, cd = w / TQ;
        const float2* Ek = reinterpret_cast<const float2*>(
            a.e_smem ? sEk + q * a.sEkS : a.ket_E + (size_t)s_q[4 * q + 1] * KK * ct.Tcd);
        const double* Rc = sR + (q * IC + ii) * KKr;
        int prow[P];
        uint64_t S[P], c[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int p = ct.pb0 + lane + 32 * j;
            prow[j] = (p < nhb ? p : ct.pb0) * nhk;  // lanes past the range read a valid row, results dropped
            S[j] = c[j] = 0ull;
        }
        const int t0 = s_kstart[cd], t1 = s_kstart[cd + 1];
        const bool gl = !a.e_smem && !ring;
        // one term: the ket E row Ea (KK float pairs) against the rows of p + q_t
        auto term = [&](int t, const float2* Ea, bool from_global) {
            const int qv = s_kq[t];
            const ulonglong2* Rj[P];
#pragma unroll
            for (int j = 0; j < P; ++j)
                Rj[j] = reinterpret_cast<const ulonglong2*>(Rc + (size_t)s_pq[prow[j] + qv] * NIs);
            auto ld = [&](int k) { return from_global ? ld_hint(Ea + k, keep) : Ea[k]; };
            for (int k = 0; k < KKe; k += 2) {
                const float2 e0 = ld(k), e1 = ld(k + 1);
                const uint64_t ah = f2_pack(e0.x, e1.x), al = f2_pack(e0.y, e1.y), nah = f2_mul(ah, m1);
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const ulonglong2 b = Rj[j][k >> 1];
                    ff_mac2(ah, al, nah, b.x, b.y, S[j], c[j]);
                }
            }
            if (KKe < KKt) {
                const float2 e0 = ld(KKe);
                const uint64_t ah = f2_pack(e0.x, 0.f), al = f2_pack(e0.y, 0.f), nah = f2_mul(ah, m1);
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    const ulonglong2 b = Rj[j][KKe >> 1];
                    ff_mac2(ah, al, nah, b.x, b.y, S[j], c[j]);
                }
            }
        };
        if (ring) {
            // the warp's ring of three ket E rows, as in split_ket_blocked
            auto issue = [&](int t, int slot) {
                if (t < t1)
                    for (int k = lane; k < KKt; k += 32) cp_async8(ring + slot * KK + k, Ek + (size_t)t * KK + k, keep);
                cp_async_commit();
            };
            issue(t0, 0);
            issue(t0 + 1, 1);
            int slot = 0;
            for (int t = t0; t < t1; ++t) {
                issue(t + 2, slot == 0 ? 2 : slot - 1);
                cp_async_wait<2>();
                __syncwarp();
                term(t, ring + slot * KK, false);
                __syncwarp();
                slot = slot == 2 ? 0 : slot + 1;
            }
            cp_async_wait<0>();
        } else {
            const int nline = (KK * 8 + 127) / 128 + 1;
            if (gl && lane < 2 * nline && t0 + lane / nline < t1)
                prefetch_l1(reinterpret_cast<const char*>(Ek + (t0 + lane / nline) * KK) +
                            min(128 * (lane % nline), 8 * KK - 8));
            for (int t = t0; t < t1; ++t) {
                if (gl && lane < nline && t + 2 < t1)
                    prefetch_l1(reinterpret_cast<const char*>(Ek + (t + 2) * KK) + min(128 * lane, 8 * KK - 8));
                term(t, Ek + t * KK, gl);
            }
        }
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int p = ct.pb0 + lane + 32 * j;
            if (p >= nhb) continue;
            float s0, s1, c0, c1;
            f2_unpack(S[j], s0, s1);
            f2_unpack(c[j], c0, c1);
            // fold the two chains into one split pair (error-free sum of the highs)
            const float t2 = __fadd_rn(s0, s1), z = __fsub_rn(t2, s0);
            const float err = __fadd_rn(__fsub_rn(s0, __fsub_rn(t2, z)), __fsub_rn(s1, z));
            const float ch = __fadd_rn(__fadd_rn(c0, c1), err);
            reinterpret_cast<float2*>(sX)[(p * ncd + cd) * TQ + q] = make_float2(t2, ch);
        }
    }
}

// One tile: quartets q0 .. q0+nqt-1 (the class tables are already staged).
// s_red: one shared double for the digestion sum.
template <bool SPLIT, int NT = kNT>
__device__ void tile_body(const FwdArgs& a, int64_t q0, int nqt, double* sm, double* s_red)
{
    const ClassTables& ct = a.ct;
    const int tid = threadIdx.x;
    const int TQ = a.TQ, KB = a.KB, KK = a.KK, IC = a.IC;
    const int nhl = ct.nhl, nhb = ct.nhb, nhk = ct.nhk, ncd = ct.ncd, nab = ct.nab;
    // R columns (items of stage A): a block of KKr ket primitives per (quartet,
    // bra primitive), KKr = KK rounded up to even in the paired layout
    const int KKr = a.r_pairs ? (KK + 1) & ~1 : KK;
    const int NI = TQ * IC * KKr;
    const int NIs = r_row_stride(NI, a.r_pairs);  // see r_row_stride
    const int* s_bstart = reinterpret_cast<const int*>(sm + a.o_tab);
    const int* s_kstart = s_bstart + nab + 1;
    const int16_t* s_bp = reinterpret_cast<const int16_t*>(s_kstart + ncd + 1);
    const int16_t* s_kq = s_bp + ct.Tab;
    const int16_t* s_pq = s_kq + ct.Tcd;
    int* s_q = reinterpret_cast<int*>(sm + a.o_q);  // [TQ][4]: bra, ket, Kbra, Kket
    // [TQ] quartet indices of a sorted batch (order != NULL, eri_batch only),
    // kept in the Coulomb-digestion scratch, which only plans (never sorted) use
    int64_t* s_qq = reinterpret_cast<int64_t*>(sm + a.o_dj);
    __shared__ int s_kmax[2];
    double* sEb = sm + a.o_Eb;
    double* sEk = sm + a.o_Ek;
    double* sPb = sm + a.o_Pb;
    double* sPk = sm + a.o_Pk;
    double* sR = sm + a.o_R;
    double* sX = sm + a.o_X;
    if (tid == 0) s_kmax[0] = s_kmax[1] = 0;
    __syncthreads();
    {
        int mkb = 0, mkk = 0;
        for (int q = tid; q < TQ; q += NT) {
            int b = 0, k = 0, kb = 0, kk = 0;
            const int64_t qq = q < nqt && a.order ? a.order[q0 + q] : q0 + q;
            if (q < nqt) {
                quartet_pairs(a, qq, &b, &k);
                kb = a.bra_kp[b];
                kk = a.ket_kp[k];
            }
            s_q[4 * q] = b;
            s_q[4 * q + 1] = k;
            s_q[4 * q + 2] = kb;
            s_q[4 * q + 3] = kk;
            if (a.order) s_qq[q] = qq;
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
    // the tile's own largest primitive-pair counts (a sorted batch's tiles share them)
    const int KBt = s_kmax[0], KKt = s_kmax[1];
    const int NIt = TQ * IC * KKt;  // stage-A items of this tile
    // stage primitive-pair scalars (and E products) of the tile
    for (int idx = tid; idx < TQ * KB * PS_N; idx += NT) {
        const int q = idx / (KB * PS_N), r = idx - q * KB * PS_N, i = r / PS_N;
        sPb[idx] = i < s_q[4 * q + 2] ? a.bra_ps[(size_t)s_q[4 * q] * KB * PS_N + r] : 1.0;
    }
    for (int idx = tid; idx < TQ * KK * PS_N; idx += NT) {
        const int q = idx / (KK * PS_N), r = idx - q * KK * PS_N, k = r / PS_N;
        sPk[idx] = k < s_q[4 * q + 3] ? a.ket_ps[(size_t)s_q[4 * q + 1] * KK * PS_N + r] : 1.0;
    }
    if (a.e_smem) {
        const int nb = KB * ct.Tab, nk = KK * ct.Tcd;
        for (int idx = tid; idx < TQ * nb; idx += NT) {
            const int q = idx / nb, r = idx - q * nb, i = r % KB;
            sEb[q * a.sEbS + r] = i < s_q[4 * q + 2] ? a.bra_E[(size_t)s_q[4 * q] * nb + r] : 0.0;
        }
        for (int idx = tid; idx < TQ * nk; idx += NT) {
            const int q = idx / nk, r = idx - q * nk, k = r % KK;
            sEk[q * a.sEkS + r] = k < s_q[4 * q + 3] ? a.ket_E[(size_t)s_q[4 * q + 1] * nk + r] : 0.0;
        }
    }
    // output accumulators
    double acc[kNACC];
#pragma unroll
    for (int s = 0; s < kNACC; ++s) acc[s] = 0.0;

    for (int i0 = 0; i0 < KBt; i0 += IC) {
        __syncthreads();
        // ---- A: auxiliary integrals of the primitive quartets (q, i0+ii, k),
        // k < KKt; few items (small tiles of high-l classes with K = 1): a warp
        // shares each item's recursion instead of leaving most threads idle
        const bool coop = NIt * 4 < NT;
        const int lane = tid & 31;
        auto stage_a_item = [&](int q, int ii, int k) {
            const int i = i0 + ii;
            Strided R{sR + (q * IC + ii) * KKr + k, NIs};
            const int e0 = coop ? lane : 0, de = coop ? 32 : 1;
            if (i < s_q[4 * q + 2] && k < s_q[4 * q + 3]) {
                const double* pb = sPb + (q * KB + i) * PS_N;
                const double* pk = sPk + (q * KK + k) * PS_N;
                // the compile-time path for low orders; the general one above them
                // and for the warp-shared recursion of small tiles
                if (coop || !aux_integrals_fixed(ct.L, pb, pk, a.boys, R)) {
                    const double zp = pb[PS_P], zq = pk[PS_P];
                    const double rs = rsqrt_fp64(zp + zq);
                    const double rho = zp * zq * (rs * rs);
                    const double X = pb[PS_PX] - pk[PS_PX], Y = pb[PS_PY] - pk[PS_PY], Z = pb[PS_PZ] - pk[PS_PZ];
                    const double PQ2 = fma(X, X, fma(Y, Y, Z * Z));
                    const double T = rho * PQ2;
                    double base[kLtotMax + 1];
                    boys_eval(ct.L, T, a.boys, base);
                    double f = rs;  // 2 pi^(5/2) / (zp zq sqrt(zp+zq)) less the pair factors in E
                    const double m2rho = -2.0 * rho;
                    for (int n = 0; n <= ct.L; ++n) {
                        base[n] *= f;
                        f *= m2rho;
                    }
                    if (coop)
                        r_recursion_warp(ct.L, base, X, Y, Z, a.rsteps, R, lane);
                    else
                        r_recursion(ct.L, base, X, Y, Z, a.rsteps, R);
                }
                if (SPLIT && !a.r_pairs)  // each entry becomes its (hi, lo) float pair, in place
                    for (int e = e0; e < nhl; e += de) {
                        double& slot = R[e];
                        const float2 f = split_f64(slot);
                        reinterpret_cast<float2&>(slot) = f;
                    }
            } else {
                for (int e = e0; e < nhl; e += de) R[e] = 0.0;
            }
        };
        // the decode divides by the tile's ket count; a tile at the batch's
        // own counts (every tile of a uniform batch) divides by the kernel
        // argument instead, which the compiler keeps in uniform registers
        if (KKt == KK) {
            for (int item = coop ? tid >> 5 : tid; item < NIt; item += coop ? NT / 32 : NT) {
                const int q = item / (IC * KK), r = item - q * IC * KK, ii = r / KK, k = r - ii * KK;
                stage_a_item(q, ii, k);
            }
        } else {
            for (int item = coop ? tid >> 5 : tid; item < NIt; item += coop ? NT / 32 : NT) {
                const int q = item / (IC * KKt), r = item - q * IC * KKt, ii = r / KKt, k = r - ii * KKt;
                stage_a_item(q, ii, k);
            }
        }
        __syncthreads();
        if (SPLIT && a.r_pairs) {
            // into the paired layout: columns k, k+1 of a block become (hi_k,
            // hi_k+1, lo_k, lo_k+1); a column at or past the tile's ket count
            // (the block's padding, or one stage A left untouched) pairs as zero
            const int npr = NI >> 1, hb = KKr >> 1;
            for (int idx = tid; idx < nhl * npr; idx += NT) {
                const int e = idx / npr, m = idx - e * npr, k0 = 2 * (m % hb);
                if (k0 >= KKt) continue;
                double* d = sR + (size_t)e * NIs + 2 * m;
                const float2 f0 = split_f64(d[0]), f1 = split_f64(k0 + 1 < KKt ? d[1] : 0.0);
                *reinterpret_cast<float4*>(d) = make_float4(f0.x, f1.x, f0.y, f1.y);
            }
            __syncthreads();
        }
        for (int ii = 0; ii < IC && i0 + ii < KBt; ++ii) {
            const int i = i0 + ii;
            // ---- B: ket transform + ket contraction
            // only the bra Hermite functions the bra transform reads (all of
            // them, or those of order la for a solid-harmonic bra)
            const bool e_row = a.o_Ei >= 0;  // one-quartet tile with unstaged E (where the row fits)
            if (e_row) {
                // the bra E products of primitive i, gathered once (strided in
                // global memory: one slot of every term) for stage C
                double* sEi = sm + a.o_Ei;
                for (int t = tid; t < ct.Tab; t += NT)
                    sEi[t] = i < s_q[2] ? a.bra_E[((size_t)s_q[0] * ct.Tab + t) * KB + i] : 0.0;
            }
            const int nhbu = nhb - ct.pb0;
            // split form, wide bra Hermite range: warp per (quartet, cd), P functions per lane
            const int blocked = SPLIT ? split_block_width(nhbu) : 0;
            float2* ring = a.o_Er >= 0 && !a.e_smem
                               ? reinterpret_cast<float2*>(sm + a.o_Er) + (size_t)(tid >> 5) * kRingRows * KK
                               : nullptr;
            if (a.r_pairs && blocked == 3)
                split_ket_paired<3, NT>(a, TQ, IC, ii, KK, KKr, KKt, NIs, ncd, nhk, sEk, sR, sX, s_q, s_kstart, s_kq,
                                        s_pq, ring);
            else if (a.r_pairs && blocked == 2)
                split_ket_paired<2, NT>(a, TQ, IC, ii, KK, KKr, KKt, NIs, ncd, nhk, sEk, sR, sX, s_q, s_kstart, s_kq,
                                        s_pq, ring);
            else if (blocked == 3)
                split_ket_blocked<3, NT>(a, TQ, IC, ii, KK, KKt, NIs, ncd, nhk, sEk, sR, sX, s_q, s_kstart, s_kq, s_pq,
                                     ring);
            else if (blocked == 2)
                split_ket_blocked<2, NT>(a, TQ, IC, ii, KK, KKt, NIs, ncd, nhk, sEk, sR, sX, s_q, s_kstart, s_kq, s_pq,
                                     ring);
            const int nB = blocked ? 0 : TQ * nhbu * ncd;
            for (int item = tid; item < nB; item += NT) {
                const int q = item % TQ, r = item / TQ, p = ct.pb0 + r % nhbu, cd = r / nhbu;
                const double* Ek = a.e_smem ? sEk + q * a.sEkS : a.ket_E + (size_t)s_q[4 * q + 1] * KK * ct.Tcd;
                const double* Rc = sR + (q * IC + ii) * KKr;  // + e * NIs + k
                const int16_t* pqrow = s_pq + p * nhk;
                const int t0 = s_kstart[cd], t1 = s_kstart[cd + 1];
                // terms outer, ket primitives inner: one p+q lookup per term
                // serves all KK primitives (E is stored slot-fastest).  FP64:
                // one accumulator chain, since the FP64 pipe keeps a dependent
                // DFMA chain at its full rate with one warp per scheduler
                // (measured: 1.06 TFLOP/s with one chain and 4 warps per SM),
                // and a single chain needs no DADD to join partial sums.
                // Split: two terms and two primitives at a time feed four
                // chains, which hides the TwoSum latency.
                if (!SPLIT) {
                    double v = 0.0;
                    for (int t = t0; t < t1; ++t) {
                        const double* Ra = Rc + (size_t)pqrow[s_kq[t]] * NIs;
                        const double* Ea = Ek + t * KK;
                        for (int k = 0; k < KKt; ++k) v = fma(Ea[k], Ra[k], v);
                    }
                    sX[(p * ncd + cd) * TQ + q] = v;
                } else {
                    float S[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
                    int t = t0;
                    for (; t + 1 < t1; t += 2) {
                        const float2* Ra = reinterpret_cast<const float2*>(Rc + (size_t)pqrow[s_kq[t]] * NIs);
                        const float2* Rb = reinterpret_cast<const float2*>(Rc + (size_t)pqrow[s_kq[t + 1]] * NIs);
                        const float2* Ea = reinterpret_cast<const float2*>(Ek + t * KK);
                        const float2* Eb2 = Ea + KK;
                        int k = 0;
                        for (; k + 1 < KKt; k += 2) {
                            ff_mac(Ea[k], Ra[k], S[0], c[0]);
                            ff_mac(Ea[k + 1], Ra[k + 1], S[1], c[1]);
                            ff_mac(Eb2[k], Rb[k], S[2], c[2]);
                            ff_mac(Eb2[k + 1], Rb[k + 1], S[3], c[3]);
                        }
                        if (k < KKt) {
                            ff_mac(Ea[k], Ra[k], S[0], c[0]);
                            ff_mac(Eb2[k], Rb[k], S[2], c[2]);
                        }
                    }
                    if (t < t1) {
                        const float2* Ra = reinterpret_cast<const float2*>(Rc + (size_t)pqrow[s_kq[t]] * NIs);
                        const float2* Ea = reinterpret_cast<const float2*>(Ek + t * KK);
                        int k = 0;
                        for (; k + 1 < KKt; k += 2) {
                            ff_mac(Ea[k], Ra[k], S[0], c[0]);
                            ff_mac(Ea[k + 1], Ra[k + 1], S[1], c[1]);
                        }
                        if (k < KKt) ff_mac(Ea[k], Ra[k], S[0], c[0]);
                    }
                    // fold the four chains into one split pair (error-free sums of the highs)
                    float Sh = S[0], ch = c[0];
#pragma unroll
                    for (int j = 1; j < 4; ++j) {
                        const float t2 = __fadd_rn(Sh, S[j]), z = __fsub_rn(t2, Sh);
                        const float err = __fadd_rn(__fsub_rn(Sh, __fsub_rn(t2, z)), __fsub_rn(S[j], z));
                        Sh = t2;
                        ch = __fadd_rn(__fadd_rn(ch, c[j]), err);
                    }
                    reinterpret_cast<float2*>(sX)[(p * ncd + cd) * TQ + q] = make_float2(Sh, ch);
                }
            }
            __syncthreads();
            // ---- C: bra transform + bra contraction
            const int nC = TQ * nab * ncd;
            if (a.acc_regs) {
#pragma unroll
                for (int s = 0; s < kNACC; ++s) {
                    const int item = tid + s * NT;
                    if (item < nC) {
                        const int q = item % TQ, r = item / TQ, cd = r % ncd, ab = r / ncd;
                        const double* Eb = a.e_smem ? sEb + q * a.sEbS + i
                                                    : (e_row ? sm + a.o_Ei
                                                             : a.bra_E + (size_t)s_q[4 * q] * KB * ct.Tab + i);
                        acc[s] = bra_sum<SPLIT>(Eb, e_row ? 1 : KB, sX, s_bstart[ab], s_bstart[ab + 1], s_bp, ncd, cd,
                                                TQ, q, acc[s]);
                    }
                }
            } else {
                const uint64_t stream = policy_stream();
                for (int item = tid; item < nC; item += NT) {
                    const int q = item % TQ, r = item / TQ, cd = r % ncd, ab = r / ncd;
                    if (q >= nqt) continue;
                    const double* Eb = a.e_smem ? sEb + q * a.sEbS + i
                                                : (e_row ? sm + a.o_Ei : a.bra_E + (size_t)s_q[4 * q] * KB * ct.Tab + i);
                    const int64_t o = out_index(a, a.order ? s_qq[q] : q0 + q, ab, cd);
                    const double prev = (i == 0) ? 0.0 : ld_hint(a.out + o, stream);
                    st_hint(a.out + o,
                            bra_sum<SPLIT>(Eb, e_row ? 1 : KB, sX, s_bstart[ab], s_bstart[ab + 1], s_bp, ncd, cd, TQ,
                                           q, prev),
                            stream);
                }
            }
            __syncthreads();
        }
    }
    if (a.acc_regs) {
        const int nC = TQ * nab * ncd;
        double esum = 0.0;
        if (!ct.hrr && ct.sph) {
            double* buf[2] = {sm, sm + a.o_hB};
#pragma unroll
            for (int s = 0; s < kNACC; ++s) {
                const int item = tid + s * NT;
                if (item < nC) buf[0][item] = acc[s];
            }
            __syncthreads();
            const double* fin = to_solid_harmonics<NT>(a, buf, 0);
            for (int item = tid; item < TQ * ct.nab_s * ct.ncd_s; item += NT) {
                const int q = item % TQ, r = item / TQ, cd = r % ct.ncd_s, ab = r / ct.ncd_s;
                if (q < nqt) a.out[out_index(a, a.order ? s_qq[q] : q0 + q, ab, cd)] = fin[item];
            }
        } else if (!ct.hrr && (a.Jmat || a.Kmat)) {
            // the values go to shared memory (the staging regions are dead)
#pragma unroll
            for (int s = 0; s < kNACC; ++s) {
                const int item = tid + s * NT;
                if (item < nC) sm[item] = acc[s];
            }
            __syncthreads();
            if (a.Jmat) digest_coulomb<NT>(a, sm, nqt, s_q, sm + a.o_dj);
            if (a.Kmat) digest_exchange<NT>(a, sm, nqt, s_q, sm + a.o_dj);
        } else if (!ct.hrr) {
#pragma unroll
            for (int s = 0; s < kNACC; ++s) {
                const int item = tid + s * NT;
                if (item < nC) {
                    const int q = item % TQ, r = item / TQ, cd = r % ncd, ab = r / ncd;
                    if (q < nqt) {
                        if (a.energy)
                            esum = fma(acc[s], digest_weight(a, s_q[4 * q], s_q[4 * q + 1], ab, cd), esum);
                        else
                            a.out[out_index(a, a.order ? s_qq[q] : q0 + q, ab, cd)] = acc[s];
                    }
                }
            }
        } else {
            // horizontal recursions on the contracted (f0|e0), one level at a
            // time over the whole tile, ping-ponging between two buffers that
            // alias the dead staging regions: ket levels on every f row
            // ([f][e][q]), then bra levels on every (cd) column ([f][cd][q])
            double* hbuf[2] = {sm, sm + a.o_hB};
            double* s_geo = sm + a.o_geo;  // [q][6]: A-B, C-D
#pragma unroll
            for (int s = 0; s < kNACC; ++s) {
                const int item = tid + s * NT;
                if (item < nC) hbuf[0][item] = acc[s];
            }
            for (int q = tid; q < TQ; q += NT) {
                const int b = s_q[4 * q], k = s_q[4 * q + 1];
                const double* A = a.centres + 3 * a.shell_atom[a.bra_sh[2 * b]];
                const double* B = a.centres + 3 * a.shell_atom[a.bra_sh[2 * b + 1]];
                const double* C = a.centres + 3 * a.shell_atom[a.ket_sh[2 * k]];
                const double* D = a.centres + 3 * a.shell_atom[a.ket_sh[2 * k + 1]];
                for (int i = 0; i < 3; ++i) {
                    s_geo[6 * q + i] = A[i] - B[i];
                    s_geo[6 * q + 3 + i] = C[i] - D[i];
                }
            }
            __syncthreads();
            int g = 0;
            for (int j = 1; j <= ct.ld; ++j, ++g) {
                const double* src = hbuf[g & 1];
                double* dst = hbuf[(g + 1) & 1];
                const int np = ct.kn[j - 1], nn = ct.kn[j];
                const int16_t* st = ct.ksteps + 3 * ct.koff[j];
                for (int item = tid; item < TQ * nab * nn; item += NT) {
                    const int q = item % TQ, r = item / TQ, o = r % nn, f = r / nn;
                    const int16_t* s3 = st + 3 * o;
                    const double* row = src + (size_t)f * np * TQ + q;
                    dst[item] = fma(s_geo[6 * q + 3 + s3[2]], row[s3[1] * TQ], row[s3[0] * TQ]);
                }
                __syncthreads();
            }
            const int ncf = ct.ncd_f;
            for (int j = 1; j <= ct.lb; ++j, ++g) {
                const double* src = hbuf[g & 1];
                double* dst = hbuf[(g + 1) & 1];
                const int16_t* st = ct.bsteps + 3 * ct.boff[j];
                for (int item = tid; item < TQ * ncf * ct.bn[j]; item += NT) {
                    const int q = item % TQ, r = item / TQ, cd = r % ncf, o = r / ncf;
                    const int16_t* s3 = st + 3 * o;
                    const double* col = src + (size_t)cd * TQ + q;
                    dst[item] = fma(s_geo[6 * q + s3[2]], col[(size_t)s3[1] * ncf * TQ], col[(size_t)s3[0] * ncf * TQ]);
                }
                __syncthreads();
            }
            const double* fin = hbuf[g & 1];  // [ab][cd][q]
            if (ct.sph) {
                const double* fs = to_solid_harmonics<NT>(a, hbuf, g & 1);
                for (int item = tid; item < TQ * ct.nab_s * ct.ncd_s; item += NT) {
                    const int q = item % TQ, r = item / TQ, cd = r % ct.ncd_s, ab = r / ct.ncd_s;
                    if (q < nqt) a.out[out_index(a, a.order ? s_qq[q] : q0 + q, ab, cd)] = fs[item];
                }
            } else if (a.Jmat || a.Kmat) {
                if (a.Jmat) digest_coulomb<NT>(a, fin, nqt, s_q, sm + a.o_dj);
                if (a.Kmat) digest_exchange<NT>(a, fin, nqt, s_q, sm + a.o_dj);
            } else {
                for (int item = tid; item < TQ * ct.nab_f * ncf; item += NT) {
                    const int q = item % TQ, r = item / TQ, cd = r % ncf, ab = r / ncf;
                    if (q >= nqt) continue;
                    if (a.energy)
                        esum = fma(fin[item], digest_weight(a, s_q[4 * q], s_q[4 * q + 1], ab, cd), esum);
                    else
                        a.out[out_index(a, a.order ? s_qq[q] : q0 + q, ab, cd)] = fin[item];
                }
            }
        }
        if (a.energy) {
            for (int o = 16; o > 0; o >>= 1) esum += __shfl_down_sync(0xffffffffu, esum, o);
            if ((tid & 31) == 0) atomicAdd(s_red, esum);
            __syncthreads();
            if (tid == 0) {
                atomicAdd(a.energy, *s_red);
                *s_red = 0.0;
            }
        }
    }
}

// NT = kNT: two CTAs per SM (128 registers a thread); kNTWide: one.
template <bool SPLIT, int NT>
__global__ void __launch_bounds__(NT, NT == kNT ? 2 : 1) fwd_kernel_t(FwdArgs a)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ double s_red;
    if (threadIdx.x == 0) s_red = 0.0;
    stage_class_tables<NT>(a, sm);
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int64_t q0 = tile * a.TQ;
        tile_body<SPLIT, NT>(a, q0, (int)min((int64_t)a.TQ, a.nq - q0), sm, &s_red);
    }
}

}  // namespace eri
