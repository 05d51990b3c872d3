// eri_fwd.cu -- forward ERI batches: eri_boys and eri_batch.
//
// Per class and batch (Section 3.1: bra pair list x ket pair list):
//  1. prepass_kernel   validates indices, angular momenta and contraction
//                      degrees and finds the largest K on each centre;
//  2. pair_kernel      per primitive pair: zeta_p, P, 2pi^(5/2)/zeta_p or
//                      1/zeta_q, and the products E^x E^y E^z of the
//                      Hermite expansion coefficients (Eqs. E2rr1/E2rr2/
//                      E2-000) for every nonzero (Cartesian pair, Hermite)
//                      term, with c_a c_b folded in and, on the ket, the
//                      sign (-1)^{l_q} of Eq. pq-from-r;
//  3. fwd_kernel       per tile of quartets, staged through shared memory:
//       A. [r]^(0) for every primitive quartet of the tile (Boys function,
//          Eq. 0m, Eq. r-rr);
//       B. ket transform and ket contraction (Eq. ket-from-hermite):
//          X[p][cd] = sum_k sum_q E^cd_{k,q} [p+q]^(0)_{ik};
//       C. bra transform and bra contraction (Eq. bra-from-hermite):
//          (ab|cd) += sum_p E^ab_{i,p} X[p][cd], accumulated over bra
//          primitives i in registers (or in `out` for very large shellsets),
//     then coalesced stores of the quartet-fastest output.
// Every FP64 operation of the path runs in these kernels.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "eri_device.cuh"
#include "eri_internal.h"
#include "eri_tile.cuh"

namespace eri {

// ---------------------------------------------------------------------------
// 1. prepass
// ---------------------------------------------------------------------------
struct PrepassArgs {
    const int32_t* shell_l;
    const int32_t* shell_K;
    int32_t nshell;
    const int32_t* bra;
    int64_t nbra;
    const int32_t* ket;
    int64_t nket;
    const int64_t* quartets;
    int64_t nq;
    int l[4];
    int unit_b;  // 1: every bra pair's second shell is -1, the unit function (3-centre)
    int* info;   // [0..3] max K per centre, [4] error, [5..6] recursion risk (float bits)
    // recursion risk (risk = 1): per pair (2|A-B|)^l2 max_ij exp(-mu_ij |A-B|^2),
    // the factor by which the horizontal recursion can magnify the pair's
    // rounding relative to its integrals; the largest over bra (ket) pairs
    int risk;
    const double* centres;
    const int32_t* shell_atom;
    const int32_t* shell_off;
    const double* exps;
    int* kmin;   // optional [2]: the smallest primitive-pair count K1 K2 over bra (ket) pairs
};

// Copies the prepass results to mapped host memory.
__global__ void info_to_host_kernel(const int* __restrict__ src, int n, int* dst)
{
    if ((int)threadIdx.x < n) dst[threadIdx.x] = src[threadIdx.x];
}

// (2|A-B|)^l2 max over primitive pairs of exp(-z1 z2 / (z1 + z2) |A-B|^2)
__device__ float pair_recursion_risk(const PrepassArgs& a, int s1, int s2, int l2)
{
    if (l2 == 0) return 1.0f;
    const double* A = a.centres + 3 * a.shell_atom[s1];
    const double* B = a.centres + 3 * a.shell_atom[s2];
    const double d2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
    double mu = 1e300;
    for (int i = 0; i < a.shell_K[s1]; ++i)
        for (int j = 0; j < a.shell_K[s2]; ++j) {
            const double z1 = a.exps[a.shell_off[s1] + i], z2 = a.exps[a.shell_off[s2] + j];
            mu = fmin(mu, z1 * z2 / (z1 + z2));
        }
    const double amp = pow(2.0 * sqrt(d2), (double)l2);
    return (float)fmin(amp * exp(-mu * d2), 3.0e38);
}

__device__ __forceinline__ void set_err(int* p, int code) { atomicCAS(p, 0, code); }

__global__ void prepass_kernel(PrepassArgs a)
{
    const int64_t n = max(max(a.nbra, a.nket), a.nq);
    int kmin[2] = {0x7fffffff, 0x7fffffff};  // this thread's smallest pair counts, reduced per warp at the end
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int side = 0; side < 2; ++side) {
            const int32_t* pr = side == 0 ? a.bra : a.ket;
            const int64_t np = side == 0 ? a.nbra : a.nket;
            if (i >= np) continue;
            for (int c = 0; c < 2; ++c) {
                const int32_t s = pr[2 * i + c];
                if (a.unit_b && side == 0 && c == 1) {
                    if (s != -1) set_err(&a.info[4], DEV_EINDEX);
                    atomicMax(&a.info[1], 1);
                    continue;
                }
                if (s < 0 || s >= a.nshell) {
                    set_err(&a.info[4], DEV_EINDEX);
                    continue;
                }
                const int l = a.shell_l[s], K = a.shell_K[s];
                if (l != a.l[2 * side + c]) set_err(&a.info[4], DEV_ECLASS);
                if (K < 1 || K > kKmax) {
                    set_err(&a.info[4], DEV_EK);
                    continue;
                }
                atomicMax(&a.info[2 * side + c], K);
            }
            if (a.kmin) {
                const int s1 = pr[2 * i], s2 = pr[2 * i + 1];
                const bool unit = a.unit_b && side == 0;
                if (s1 >= 0 && s1 < a.nshell && (unit || (s2 >= 0 && s2 < a.nshell)))
                    kmin[side] = min(kmin[side], a.shell_K[s1] * (unit ? 1 : a.shell_K[s2]));
            }
            if (a.risk) {
                const int s1 = pr[2 * i], s2 = pr[2 * i + 1];
                if (s1 >= 0 && s1 < a.nshell && s2 >= 0 && s2 < a.nshell) {
                    const int K1 = a.shell_K[s1], K2 = a.shell_K[s2];
                    if (K1 >= 1 && K1 <= kKmax && K2 >= 1 && K2 <= kKmax) {
                        const float r = pair_recursion_risk(a, s1, s2, a.l[2 * side + 1]);
                        atomicMax(&a.info[5 + side], __float_as_int(r));  // r >= 0: int order = float order
                    }
                }
            }
        }
        if (a.quartets && i < a.nq) {
            const int64_t b = a.quartets[2 * i], k = a.quartets[2 * i + 1];
            if (b < 0 || b >= a.nbra || k < 0 || k >= a.nket) set_err(&a.info[4], DEV_EINDEX);
        }
    }
    if (a.kmin) {  // every thread of the block reaches this point
        const int m0 = __reduce_min_sync(0xffffffffu, kmin[0]), m1 = __reduce_min_sync(0xffffffffu, kmin[1]);
        if ((threadIdx.x & 31) == 0) {
            if (m0 != 0x7fffffff) atomicMin(&a.kmin[0], m0);
            if (m1 != 0x7fffffff) atomicMin(&a.kmin[1], m1);
        }
    }
}

// ---------------------------------------------------------------------------
// 2. primitive-pair tables
// ---------------------------------------------------------------------------
struct PairArgs {
    const double* centres;
    const int32_t* shell_atom;
    const int32_t* shell_K;
    const int32_t* shell_off;
    const double* exps;
    const double* coefs;
    const int32_t* pairs;
    int64_t npairs;
    int l1, l2;
    int KS;                 // primitive-pair slots per pair
    int T;                  // terms
    const uint8_t* fac;     // [T][3] per-axis E-table indices
    int ket;                // 1: ket side (sign (-1)^{l_q}, scale 1/zeta_q)
    double* ps;             // [npairs][KS][PS_N]
    double* E;              // [npairs][T][KS] (slot fastest)
    int32_t* kprim;         // [npairs] number of valid slots K1*K2
    // adjoint only (ax == nullptr otherwise): per-axis tables with both
    // indices raised by up to 2, ax[(g*3 + axis)*eax + (i*(l2+3) + j)*(l1+l2+5) + t]
    double* ax;
    int eax;
    double* zz;             // [npairs][KS][2]: the two exponents
    int split;              // 1: E products stored as float pairs (hi, lo) in the double slots
    int hrr;                // 1: terms of E_{e,0}, |e| = l1..l1+l2 (horizontal-recursion form)
    const double* scale;    // [T] per-term factors (solid-harmonic side), or null
};

constexpr int kEax = (kLmax + 3) * (kLmax + 3) * (2 * kLmax + 5);  // per-axis E table bound (adjoint shifts)
constexpr int kEfw = (kLmax + 1) * (kLmax + 1) * (2 * kLmax + 1);  // without the shifts (also the HRR form's)

// RAISED: the adjoint's tables (a.ax != NULL): the per-axis E tables with
// both indices raised by 2, one thread per (slot, axis).  The adjoint reads
// no E products of that side, so none are formed.  Otherwise one thread per
// slot forms the three tables and the E products of the class's terms.
template <bool RAISED>
__global__ void pair_kernel_t(PairArgs a)
{
    constexpr int NX = RAISED ? 1 : 3;  // axes per thread
    const int64_t total = a.npairs * a.KS * (RAISED ? 3 : 1);
    for (int64_t gg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gg < total;
         gg += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = RAISED ? gg / 3 : gg;       // the slot
        const int x0 = RAISED ? (int)(gg - g * 3) : 0;  // its first axis
        const int64_t j = g / a.KS;
        const int s = (int)(g - j * a.KS);
        // s2 = -1: the unit function (exponent 0, coefficient 1) of a 3-centre
        // bra; its centre is immaterial and taken as the first shell's
        const int s1 = a.pairs[2 * j], s2 = a.pairs[2 * j + 1];
        const int K1 = a.shell_K[s1], K2 = s2 < 0 ? 1 : a.shell_K[s2];
        if (s == 0 && x0 == 0) a.kprim[j] = K1 * K2;
        if (s >= K1 * K2) {  // padding slot: finite zeros, never contributes
            if (RAISED) {
                for (int q = 0; q < a.eax; ++q) a.ax[((size_t)g * 3 + x0) * a.eax + q] = 0.0;
                if (x0 != 0) continue;
                a.zz[2 * g] = a.zz[2 * g + 1] = 1.0;
            } else {
                for (int t = 0; t < a.T; ++t) a.E[((size_t)j * a.T + t) * a.KS + s] = 0.0;
            }
            double* o = a.ps + (size_t)g * PS_N;
            o[PS_P] = 1.0;
            o[PS_PX] = o[PS_PY] = o[PS_PZ] = 0.0;
            continue;
        }
        const int i1 = s / K2, i2 = s - i1 * K2;
        const int p1 = a.shell_off[s1] + i1, p2 = s2 < 0 ? -1 : a.shell_off[s2] + i2;
        const double z1 = a.exps[p1], z2 = s2 < 0 ? 0.0 : a.exps[p2];
        const double c2 = s2 < 0 ? 1.0 : a.coefs[p2];
        const double* A = a.centres + 3 * a.shell_atom[s1];
        const double* B = s2 < 0 ? A : a.centres + 3 * a.shell_atom[s2];
        const double p = z1 + z2;
        const double invp = 1.0 / p;
        const double inv2p = 0.5 * invp;
        double PA[3], PB[3], P[3], AB2 = 0.0;
        for (int x = 0; x < 3; ++x) {
            P[x] = (z1 * A[x] + z2 * B[x]) * invp;
            PA[x] = P[x] - A[x];
            PB[x] = P[x] - B[x];
            const double d = A[x] - B[x];
            AB2 = fma(d, d, AB2);
        }
        // K_AB c_1 c_2 carried by the x-axis bootstrap E_00^0 (Eq. E2-000),
        // 1 on y and z: the products E^x E^y E^z are unchanged.  So is the
        // pair's factor of the Eq. 0m prefactor, 2 pi^(5/2) / zeta_p on the
        // bra and 1 / zeta_q on the ket: every E of the pair (per-axis tables
        // and products alike) carries it once, and [0]^(m) needs only the
        // quartet's 1/sqrt(zeta_p + zeta_q).
        const double e00x = a.coefs[p1] * c2 * exp(-z1 * z2 * invp * AB2) * (a.ket ? invp : kTwoPi52 * invp);
        const int ext = RAISED ? 2 : 0;
        // largest raised indices: the adjoint raises both by 2; the
        // horizontal-recursion form needs E_{i,0} for i <= l1 + l2
        const int m1 = a.hrr ? a.l1 + a.l2 : a.l1 + ext, m2 = a.hrr ? 0 : a.l2 + ext;
        const int L12 = a.l1 + a.l2, n2 = m2 + 1, nt = m1 + m2 + 1;
        double E[NX][RAISED ? kEax : kEfw];
        for (int xi = 0; xi < NX; ++xi) {
            const int x = x0 + xi;
            double* Ex = E[xi];
            for (int q = 0; q < (m1 + 1) * n2 * nt; ++q) Ex[q] = 0.0;
            Ex[0] = x == 0 ? e00x : 1.0;
            // raise the first index at j = 0 (Eq. E2rr1)
            for (int i = 0; i < m1; ++i)
                for (int t = 0; t <= i + 1; ++t) {
                    double v = 0.0;
                    if (t >= 1) v = inv2p * Ex[(i * n2) * nt + t - 1];
                    if (t <= i) v = fma(PA[x], Ex[(i * n2) * nt + t], v);
                    if (t + 1 <= i) v = fma((double)(float)(t + 1), Ex[(i * n2) * nt + t + 1], v);
                    Ex[((i + 1) * n2) * nt + t] = v;
                }
            // raise the second index for every first index (Eq. E2rr2)
            for (int i = 0; i <= m1; ++i)
                for (int jj = 0; jj < m2; ++jj)
                    for (int t = 0; t <= i + jj + 1; ++t) {
                        const int b0 = (i * n2 + jj) * nt;
                        double v = 0.0;
                        if (t >= 1) v = inv2p * Ex[b0 + t - 1];
                        if (t <= i + jj) v = fma(PB[x], Ex[b0 + t], v);
                        if (t + 1 <= i + jj) v = fma((double)(float)(t + 1), Ex[b0 + t + 1], v);
                        Ex[(i * n2 + jj + 1) * nt + t] = v;
                    }
        }
        if (RAISED) {
            double* o = a.ax + ((size_t)g * 3 + x0) * a.eax;
            for (int q = 0; q < (m1 + 1) * n2 * nt; ++q) o[q] = E[0][q];
            if (x0 != 0) continue;
            a.zz[2 * g] = z1;
            a.zz[2 * g + 1] = z2;
        } else {
            double* Eout = a.E + (size_t)j * a.T * a.KS + s;  // term t at Eout[t * KS]
            const int ntc = L12 + 1, n2c = a.hrr ? 1 : a.l2 + 1;  // dims the class-table indices use
            for (int t = 0; t < a.T; ++t) {
                int idx[3], lq = 0;
                for (int x = 0; x < 3; ++x) {
                    const int f = a.fac[3 * t + x];
                    const int tt = f % ntc, bb = (f / ntc) % n2c, aa = f / (ntc * n2c);
                    idx[x] = (aa * n2 + bb) * nt + tt;
                    lq += tt;
                }
                double v = E[0][idx[0]] * E[NX > 1 ? 1 : 0][idx[1]] * E[NX > 2 ? 2 : 0][idx[2]];
                if (a.scale) v *= a.scale[t];
                if (a.ket && (lq & 1)) v = -v;
                if (a.split)
                    reinterpret_cast<float2*>(Eout)[(size_t)t * a.KS] = split_f64(v);
                else
                    Eout[(size_t)t * a.KS] = v;
            }
        }
        double* o = a.ps + (size_t)g * PS_N;
        o[PS_P] = p;
        o[PS_PX] = P[0];
        o[PS_PY] = P[1];
        o[PS_PZ] = P[2];
    }
}

// grid: blocks of 128 threads for one thread per slot; the raised kernel
// takes three per slot
static void launch_pair(const PairArgs& p, int grid, cudaStream_t st)
{
    if (p.ax)
        pair_kernel_t<true><<<(int)std::min<int64_t>(3LL * grid, 24LL * sm_count()), 128, 0, st>>>(p);
    else
        pair_kernel_t<false><<<grid, 128, 0, st>>>(p);
}

static const auto fwd_kernel = fwd_kernel_t<false, kNT>;
static const auto fwd_kernel_split = fwd_kernel_t<true, kNT>;

// A tile whose shared memory leaves room for one CTA per SM (each CTA also
// takes a 1 KB system reserve and a few bytes of static shared memory).
static bool one_cta_per_sm(size_t bytes) { return 2 * (bytes + 1024 + 64) > (size_t)smem_per_sm(); }

// The forward kernel for a precision and a CTA width (kNT or kNTWide).
static void (*fwd_kern(int split, int nt))(FwdArgs)
{
    if (nt == kNTWide) return split ? fwd_kernel_t<true, kNTWide> : fwd_kernel_t<false, kNTWide>;
    return split ? fwd_kernel_split : fwd_kernel;
}

// ---------------------------------------------------------------------------
// Boys entry kernel
// ---------------------------------------------------------------------------
__global__ void boys_kernel(int mmax, const double* T, int64_t n, const double* tab, double* F)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double f[ERI_BOYS_MMAX + 1];
        boys_eval(mmax, T[i], tab, f);
        for (int m = 0; m <= mmax; ++m) F[i * (mmax + 1) + m] = f[m];
    }
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int smem_per_sm()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (n <= 0) n = 64 * 1024;
    }
    return n;
}

int max_smem_optin()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (n <= 0) n = 48 * 1024;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Tile planning: pick (TQ, IC, e_smem, acc_regs) so that shared memory fits
// and the auxiliary-integral stage has enough independent items.
// ---------------------------------------------------------------------------
static int odd_up(int n) { return n | 1; }

// Ping-pong buffers of the epilogue's horizontal recursions: level g of the
// combined sequence (ket levels 0..ld, then bra levels 1..lb) lives in
// buffer g % 2; *A and *B are the largest even and odd level (doubles).
static void hrr_buffers(const ClassTables& ct, int TQ, size_t* A, size_t* B)
{
    *A = *B = 0;
    for (int g = 0; g <= ct.ld + ct.lb; ++g) {
        const size_t n = g <= ct.ld ? (size_t)TQ * ct.nab * ct.kn[g] : (size_t)TQ * ct.ncd_f * ct.bn[g - ct.ld];
        size_t& m = (g & 1) ? *B : *A;
        m = std::max(m, n);
    }
}

bool tile_layout(const ClassTables& ct, int KB, int KK, int TQ, int IC, int e_smem, TilePlan* tp, int split)
{
    size_t off = 0;
    auto take = [&](size_t nd) {
        size_t o = off;
        off += (nd + 1) & ~size_t(1);  // keep 16-byte alignment
        return (int)o;
    };
    auto even = [](size_t nd) { return (nd + 1) & ~size_t(1); };
    tp->TQ = TQ;
    tp->IC = IC;
    tp->e_smem = e_smem;
    tp->sEbS = e_smem ? odd_up(KB * ct.Tab) : 0;
    tp->sEkS = e_smem ? odd_up(KK * ct.Tcd) : 0;
    // the paired layout of the auxiliary integrals where the split form's
    // blocked ket stage packs two ket primitives per FP32 instruction, for
    // tiles that accumulate in memory: with register accumulators live
    // through the ket stage the packed loop runs short of registers (measured
    // on (ff|dd), K = 5: 1.27 times slower than the unpacked loop; (ff|ff),
    // K = 5, accumulating in memory: 1.06 times faster)
    const bool acc_regs = TQ * ct.nab * ct.ncd <= kNT * kNACC;
    tp->r_pairs = split && split_block_width(ct.nhb - ct.pb0) && KK >= 2 && !acc_regs ? 1 : 0;
    const int KKr = tp->r_pairs ? (KK + 1) & ~1 : KK;
    size_t r_need = (size_t)r_row_stride(TQ * IC * KKr, tp->r_pairs) * ct.nhl;
    size_t hA = 0, hB = 0;
    if (ct.hrr || ct.sph) {
        // the recursion (and solid-harmonic) buffers alias every staging
        // region before the tables (E, pair scalars, R, X are dead in the
        // epilogue); grow R if short
        if (ct.hrr) hrr_buffers(ct, TQ, &hA, &hB);
        if (ct.sph) {  // each solid-harmonic step reads one buffer and writes the other
            const size_t nf = (size_t)TQ * ct.nab_f * ct.ncd_f;
            hA = std::max(hA, nf);
            hB = std::max(hB, nf);
        }
        const size_t staged = even((size_t)TQ * tp->sEbS) + even((size_t)TQ * tp->sEkS) +
                              even((size_t)TQ * KB * PS_N) + even((size_t)TQ * KK * PS_N) + even(r_need) +
                              even((size_t)TQ * ct.nhb * ct.ncd);
        const size_t need = even(hA) + even(hB);
        if (staged < need) r_need += need - staged;
    }
    {
        // the Coulomb digestion of plans stages the tile's values there too
        const size_t staged = even((size_t)TQ * tp->sEbS) + even((size_t)TQ * tp->sEkS) +
                              even((size_t)TQ * KB * PS_N) + even((size_t)TQ * KK * PS_N) + even(r_need) +
                              even((size_t)TQ * ct.nhb * ct.ncd);
        const size_t need = even((size_t)TQ * ct.nab * ct.ncd);
        if (TQ * ct.nab * ct.ncd <= kNT * kNACC && staged < need) r_need += need - staged;
    }
    tp->o_Eb = take((size_t)TQ * tp->sEbS);
    tp->o_Ek = take((size_t)TQ * tp->sEkS);
    tp->o_Pb = take((size_t)TQ * KB * PS_N);
    tp->o_Pk = take((size_t)TQ * KK * PS_N);
    tp->o_R = take(r_need);
    tp->o_X = take((size_t)TQ * ct.nhb * ct.ncd);
    tp->o_hB = (int)even(hA);
    const size_t tab_bytes = 4 * (ct.nab + ct.ncd + 2) + 2 * (ct.Tab + ct.Tcd + ct.nhb * ct.nhk);
    tp->o_tab = take((tab_bytes + 7) / 8);
    tp->o_q = take((size_t)TQ * 2);
    tp->o_geo = take(ct.hrr ? (size_t)TQ * 6 : 0);
    tp->o_dj = take((size_t)TQ + ct.nab_f);  // also the quartet indices of a sorted batch
    // one-quartet tiles only, and only where it fits: a tile without it
    // reads the bra E products from global memory
    tp->o_Ei = -1;
    if (!e_smem && TQ == 1 && (off + even(ct.Tab)) * 8 <= (size_t)max_smem_optin()) tp->o_Ei = take(ct.Tab);
    tp->o_Er = -1;  // added for the split form by add_e_ring
    tp->bytes = off * 8;
    tp->nt = kNT;
    tp->acc_regs = (TQ * ct.nab * ct.ncd <= kNT * kNACC) ? 1 : 0;
    if (ct.hrr && !tp->acc_regs) return false;
    return tp->bytes <= (size_t)max_smem_optin();
}

// Split form: when the blocked ket stage reads its ket E rows from global
// memory, give every warp (tp->nt / 32 of them) a ring of kRingRows rows (KK
// float pairs each) at the end of the tile's shared memory, if it fits.
static void add_e_ring(const ClassTables& ct, int KK, TilePlan* tp)
{
    tp->o_Er = -1;
    if (tp->e_smem || !split_block_width(ct.nhb - ct.pb0)) return;
    const size_t off = (tp->bytes / 8 + 1) & ~size_t(1), nd = (size_t)(tp->nt / 32) * kRingRows * KK;
    if ((off + nd) * 8 > (size_t)max_smem_optin()) return;
    tp->o_Er = (int)off;
    tp->bytes = (off + nd) * 8;
}

bool plan_tiles(const ClassTables& ct, int KB, int KK, int64_t nq, TilePlan* best, size_t max_bytes, int split)
{
    bool found = false;
    double best_score = -1.0;
    for (int e_smem = 1; e_smem >= 0; --e_smem) {
        for (int TQ = 128; TQ >= 1; TQ /= 2) {
            if (TQ > 1 && TQ * ct.nab * ct.ncd > kNT * kNACC) continue;  // prefer register accumulation
            if (TQ > 1 && (int64_t)TQ > 2 * nq) continue;
            for (int IC = KB; IC >= 1; IC = (IC + 1) / 2 - (IC == 1)) {
                TilePlan tp;
                if (!tile_layout(ct, KB, KK, TQ, IC, e_smem, &tp, split) || (max_bytes && tp.bytes > max_bytes)) {
                    if (IC == 1) break;
                    continue;
                }
                // score: utilisation of the stage-A items, the ket-stage items
                // and the bra-stage items (fraction of kNT-wide rounds used)
                auto util = [](int64_t n) {
                    const int64_t rounds = (n + kNT - 1) / kNT;
                    return rounds ? (double)n / (double)(rounds * kNT) : 0.0;
                };
                const int64_t nA = (int64_t)TQ * IC * KK;
                const double wA = (double)ct.nhl * 2.0 + 40.0;
                const double wB = (double)ct.nhb * ct.Tcd * KK;
                const double wC = (double)ct.ncd * ct.Tab;
                const double score = (wA + wB + wC) /
                                     (wA / util(nA) + wB / util((int64_t)TQ * ct.nhb * ct.ncd) +
                                      wC / util((int64_t)TQ * ct.nab * ct.ncd)) +
                                     1e-3 * TQ * IC + (e_smem ? 0.05 : 0.0);
                if (score > best_score) {
                    best_score = score;
                    *best = tp;
                    found = true;
                }
                if (IC == 1) break;
            }
        }
        if (found) break;
    }
    return found;
}

static int dev_err_to_code(int e)
{
    switch (e) {
        case DEV_OK: return ERI_OK;
        case DEV_ECLASS: return ERI_ECLASS;
        case DEV_EINDEX: return ERI_EINVAL;
        case DEV_EK: return ERI_EINVAL;
        case DEV_ETIMEOUT: return ERI_ETIMEOUT;
        default: return ERI_ECUDA;
    }
}

static size_t align_up(size_t n) { return (n + 255) & ~size_t(255); }

// Prepass + pair tables shared by the forward and adjoint entry points.
// On success fills the pair tables and the largest K on each centre.
// Largest product of bra and ket recursion risks for which the recursion
// forms are offered (see prepass_kernel): 1.1e-16 x 900 x O(10) ~ 1e-12.
constexpr double kRecursionRisk = 900.0;

// Forms eri_batch may use (eri_set_forms): bit o allows form o.
static std::atomic<int> g_form_mask{0xF};

// Forms chosen by timing, per (device, class, K_bra, K_ket, precision).
static std::map<std::tuple<int, int, int, int, int, int, int, int, int>, int> g_forms;
static std::mutex g_forms_mu;

static std::tuple<int, int, int, int, int, int, int, int, int> form_key(eri_class_t cls, int KB, int KK, int split,
                                                                        int kind)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return std::make_tuple(dev, cls.la, cls.lb, cls.lc, cls.ld, KB, KK, split, kind);
}

static int lookup_form(eri_class_t cls, int KB, int KK, int split, int kind)
{
    std::lock_guard<std::mutex> lk(g_forms_mu);
    auto it = g_forms.find(form_key(cls, KB, KK, split, kind));
    return it == g_forms.end() ? -1 : it->second;
}

void remember_form(eri_class_t cls, int KB, int KK, int split, int kind, int form)
{
    std::lock_guard<std::mutex> lk(g_forms_mu);
    g_forms[form_key(cls, KB, KK, split, kind)] = form;
}

int prepare_batch(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                  int64_t nket, const int64_t* quartets, int64_t nq, int ldelta, cudaStream_t st,
                  const ClassTables** ct_out, PairTables* pb, PairTables* pk, int* KB, int* KK, int kmax[4],
                  int allow_swap, FormChoice* fc, int split, int kind, int* mixed)
{
    int err = ERI_OK;
    // kind 2: the caller's bra side (x, unit) is a solid harmonic
    // kind 3: solid-harmonic output on every centre (plain or recursion form)
    auto tables = [&](int la, int lb, int lc, int ld, int x_first, int hrr) {
        if (kind == 2) return get_class_tables_pure(la, lb, lc, ld, x_first ? 1 : 2, st, &err);
        if (kind == 3) return get_class_tables_sph(la, lb, lc, ld, hrr, st, &err);
        return hrr ? get_class_tables_hrr(la, lb, lc, ld, st, &err) : get_class_tables(la, lb, lc, ld, st, &err);
    };
    const ClassTables* ct = tables(cls.la, cls.lb, cls.lc, cls.ld, 1, 0);
    if (!ct) return err;
    *ct_out = ct;
    const int forced = fc ? fc->form : -1;
    if (fc) {
        fc->form = 0;
        fc->alt = -1;
        fc->cached = 0;
    }
    int* status = device_status();
    if (!status) return ERI_ECUDA;
    int32_t* hinfo = host_pinned_i32(16);
    if (!hinfo) return ERI_ENOMEM;
    // info lives in the status block (slots 8..16), separate from the error word:
    // [0..6] as PrepassArgs::info, [7..8] the smallest pair counts per side
    int* dinfo = status + 8;
    if (cudaMemsetAsync(dinfo, 0, 7 * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(dinfo + 7, 0x7f, 2 * sizeof(int), st) != cudaSuccess)
        return ERI_ECUDA;
    PrepassArgs pa{basis->shell_l, basis->shell_K, basis->nshell, bra, nbra, ket, nket, quartets,
                   quartets ? nq : (int64_t)0,
                   {cls.la, cls.lb, cls.lc, cls.ld}, (kind == 1 || kind == 2) ? 1 : 0, dinfo,
                   allow_swap > 1 ? 1 : 0, basis->centres, basis->shell_atom, basis->shell_off, basis->exps,
                   dinfo + 7};
    const int64_t n = std::max(std::max(nbra, nket), quartets ? nq : (int64_t)0);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * sm_count());
    {
        ProfScope ps(PROF_PREPASS, st);
        prepass_kernel<<<std::max(grid, 1), 256, 0, st>>>(pa);
    }
    if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    // the info goes to the pinned host buffer through its mapped device
    // address, written by a kernel: a device-to-host copy would queue behind
    // any large read-back the caller has put on that copy engine
    int32_t* hmapped = nullptr;
    if (cudaHostGetDevicePointer((void**)&hmapped, hinfo, 0) == cudaSuccess && hmapped) {
        count_launch();
        info_to_host_kernel<<<1, 32, 0, st>>>(dinfo, 9, hmapped);
        if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    } else {
        cudaGetLastError();
        if (cudaMemcpyAsync(hinfo, dinfo, 9 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return ERI_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return ERI_ECUDA;
    if (hinfo[4] != 0) return dev_err_to_code(hinfo[4]);
    for (int c = 0; c < 4; ++c) kmax[c] = hinfo[c];
    *KB = kmax[0] * kmax[1];
    *KK = kmax[2] * kmax[3];
    if (mixed) *mixed = (hinfo[7] < *KB || hinfo[8] < *KK) ? 1 : 0;
    if (allow_swap) {
        // Four forms: which side is transformed first (Section 3.2.2
        // transforms the ket first, assuming it has the lower l) and whether
        // the transforms run on (e0) functions followed by horizontal
        // recursions in the contracted basis.  The FP64-work model picks one
        // unless a form is forced or an earlier timing chose one.
        const ClassTables* opt[4] = {ct, tables(cls.lc, cls.ld, cls.la, cls.lb, 0, 0), nullptr, nullptr};
        if (!opt[1]) return err;
        // The recursion forms must keep their magnified rounding, about
        // 1.1e-16 x (bra risk) x (ket risk) x the integrals' scale, well
        // inside the 1e-11 absolute bar: they are offered only while the
        // product of the largest pair risks stays below kRecursionRisk.
        float rb, rk;
        std::memcpy(&rb, &hinfo[5], 4);
        std::memcpy(&rk, &hinfo[6], 4);
        const bool hrr_ok = (double)rb * (double)rk <= kRecursionRisk;
        if (allow_swap > 1 && (kind == 0 || kind == 3) && hrr_ok) {
            opt[2] = tables(cls.la, cls.lb, cls.lc, cls.ld, 1, 1);
            opt[3] = tables(cls.lc, cls.ld, cls.la, cls.lb, 0, 1);
            if (!opt[2] || !opt[3]) return err;
        }
        const int64_t nqq = quartets ? nq : nbra * nket;
        double cost[4];
        for (int o = 0; o < 4; ++o) {
            cost[o] = -1.0;  // infeasible
            const ClassTables* c = opt[o];
            if (!c) continue;
            const double kb = (o & 1) ? *KK : *KB, kk = (o & 1) ? *KB : *KK;
            if (c->hrr) {
                // (f0|e0) must fit the register accumulators and the
                // recursion buffers of the epilogue the shared memory
                TilePlan tp;
                if (c->nab * c->ncd > kNT * kNACC || !plan_tiles(*c, (int)kb, (int)kk, nqq, &tp)) continue;
            }
            cost[o] = kb * kk * ((c->nhb - c->pb0) * c->Tcd + 0.5 * c->nhl) + kb * c->ncd * c->Tab +
                      (c->hrr ? c->nab * c->nks + c->ncd_f * c->nbs : 0);
        }
        {
            // the caller's form mask (eri_set_forms), unless it leaves no feasible form
            const int mask = g_form_mask.load();
            bool any = false;
            for (int o = 0; o < 4; ++o) any |= cost[o] >= 0 && (mask >> o & 1);
            if (any)
                for (int o = 0; o < 4; ++o)
                    if (!(mask >> o & 1)) cost[o] = -1.0;
        }
        auto cheapest = [&](int lo, int hi) {
            int b = -1;
            for (int o = lo; o < hi; ++o)
                if (cost[o] >= 0 && (b < 0 || cost[o] < cost[b])) b = o;
            return b;
        };
        int best = -1;
        if (forced >= 0) {
            if (forced > 3 || cost[forced] < 0) return ERI_EINVAL;
            best = forced;
        } else {
            best = lookup_form(cls, *KB, *KK, split, kind);
            if (best >= 0 && cost[best] >= 0) {
                if (fc) fc->cached = 1;
            } else {
                best = cheapest(0, 4);
            }
        }
        if (fc) {
            fc->form = best;
            fc->alt = best >= 2 ? cheapest(0, 2) : cheapest(2, 4);
        }
        ct = opt[best];
        *ct_out = ct;
        if (best & 1) {
            cls = eri_class_t{cls.lc, cls.ld, cls.la, cls.lb};
            std::swap(bra, ket);
            std::swap(nbra, nket);
            std::swap(*KB, *KK);
            std::swap(kmax[0], kmax[2]);
            std::swap(kmax[1], kmax[3]);
        }
    }
    // workspace: pair tables of both sides
    const size_t nb_ps = align_up(sizeof(double) * nbra * *KB * PS_N), nb_E = align_up(sizeof(double) * nbra * *KB * ct->Tab);
    const size_t nk_ps = align_up(sizeof(double) * nket * *KK * PS_N), nk_E = align_up(sizeof(double) * nket * *KK * ct->Tcd);
    const size_t nb_k = align_up(sizeof(int32_t) * nbra), nk_k = align_up(sizeof(int32_t) * nket);
    // ldelta 1: the raised tables of the kernel bra only (the adjoint launch
    // for one side's channels); 2: of both sides, with the E products of
    // both (the adjoint launch for every channel)
    const int grad = ldelta > 0, grad_both = ldelta > 1;
    const int eaxb = (cls.la + 3) * (cls.lb + 3) * (cls.la + cls.lb + 5);
    const int eaxk = (cls.lc + 3) * (cls.ld + 3) * (cls.lc + cls.ld + 5);
    const size_t nb_ax = grad ? align_up(sizeof(double) * nbra * *KB * 3 * eaxb) : 0;
    const size_t nk_ax = grad_both ? align_up(sizeof(double) * nket * *KK * 3 * eaxk) : 0;
    const size_t nb_z = grad ? align_up(sizeof(double) * nbra * *KB * 2) : 0;
    const size_t nk_z = grad_both ? align_up(sizeof(double) * nket * *KK * 2) : 0;
    uint8_t* ws = (uint8_t*)workspace(nb_ps + nb_E + nk_ps + nk_E + nb_k + nk_k + nb_ax + nk_ax + nb_z + nk_z, &err);
    if (!ws) return err;
    {
        uint8_t* g0 = ws + nb_ps + nb_E + nk_ps + nk_E + nb_k + nk_k;
        pb->ax = grad ? (double*)g0 : nullptr;
        pk->ax = grad_both ? (double*)(g0 + nb_ax) : nullptr;
        pb->zz = grad ? (double*)(g0 + nb_ax + nk_ax) : nullptr;
        pk->zz = grad_both ? (double*)(g0 + nb_ax + nk_ax + nb_z) : nullptr;
        pb->eax = eaxb;
        pk->eax = eaxk;
    }
    pb->ps = (double*)ws;
    pb->E = (double*)(ws + nb_ps);
    pk->ps = (double*)(ws + nb_ps + nb_E);
    pk->E = (double*)(ws + nb_ps + nb_E + nk_ps);
    pb->kp = (int32_t*)(ws + nb_ps + nb_E + nk_ps + nk_E);
    pk->kp = (int32_t*)(ws + nb_ps + nb_E + nk_ps + nk_E + nb_k);
    for (int side = 0; side < 2; ++side) {
        PairArgs p{};
        p.centres = basis->centres;
        p.shell_atom = basis->shell_atom;
        p.shell_K = basis->shell_K;
        p.shell_off = basis->shell_off;
        p.exps = basis->exps;
        p.coefs = basis->coefs;
        p.pairs = side ? ket : bra;
        p.npairs = side ? nket : nbra;
        p.l1 = side ? cls.lc : cls.la;
        p.l2 = side ? cls.ld : cls.lb;
        p.KS = side ? *KK : *KB;
        p.T = side ? ct->Tcd : ct->Tab;
        p.fac = side ? ct->ket_fac : ct->bra_fac;
        p.ket = side;
        PairTables& t = side ? *pk : *pb;
        p.ps = t.ps;
        p.E = t.E;
        p.kprim = t.kp;
        p.ax = t.ax;
        p.eax = t.eax;
        p.zz = t.zz;
        p.split = split;
        p.hrr = ct->hrr;
        p.scale = side ? ct->ket_scale : ct->bra_scale;
        const int64_t tot = p.npairs * p.KS;
        const int g = (int)std::min<int64_t>((tot + 127) / 128, 8 * sm_count());
        ProfScope ps(PROF_PAIR, st);
        if (grad_both) {  // the E products as well as the raised tables (both write the same pair scalars)
            PairArgs pe = p;
            pe.ax = nullptr;
            pe.zz = nullptr;
            launch_pair(pe, std::max(g, 1), st);
        }
        launch_pair(p, std::max(g, 1), st);
        if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    }
    return ERI_OK;
}

static int check_basis(const eri_basis_t* b)
{
    if (!b || !b->centres || !b->shell_atom || !b->shell_l || !b->shell_K || !b->shell_off || !b->exps || !b->coefs)
        return ERI_EINVAL;
    if (b->natom < 0 || b->nshell < 0 || b->nprim < 0) return ERI_EINVAL;
    return ERI_OK;
}

static int check_class(eri_class_t c)
{
    const int l[4] = {c.la, c.lb, c.lc, c.ld};
    for (int i = 0; i < 4; ++i)
        if (l[i] < 0 || l[i] > kLmax) return ERI_EINVAL;
    return ERI_OK;
}

int check_batch_args(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                     int64_t nket, const int64_t* quartets, int64_t nq, int64_t len)
{
    if (check_class(cls) != ERI_OK || check_basis(basis) != ERI_OK) return ERI_EINVAL;
    if (nbra < 0 || nket < 0 || (quartets && nq < 0)) return ERI_EINVAL;
    if ((nbra > 0 && !bra) || (nket > 0 && !ket)) return ERI_EINVAL;
    if (nbra > INT32_MAX || nket > INT32_MAX) return ERI_EINVAL;
    const int64_t nqq = quartets ? nq : nbra * nket;
    const int64_t nab = host_nc(cls.la) * host_nc(cls.lb), ncd = host_nc(cls.lc) * host_nc(cls.ld);
    if (len < nqq * nab * ncd) return ERI_EINVAL;
    return ERI_OK;
}

// Autotuner of eri_batch: on the first large batch of a (class, form, K_bra,
// K_ket, precision) signature, time every feasible tile shape (TQ in 1..128 with
// register accumulation, IC in {K_bra, K_bra/2, 1}, E staged when it fits)
// on the batch's leading quartets (about four waves of tiles, at least
// kTuneQuartets) and remember the fastest with its time per quartet
// (eri_batch compares forms by it).  The trial launches write (part
// of) `out`; the real launch overwrites it.
constexpr int64_t kTuneMinQuartets = 16384;
constexpr int64_t kTuneQuartets = 8192;
static std::map<std::tuple<int, int, int, int, int, int, int, int, int, int>, std::pair<TilePlan, float>> g_tuned;
static std::mutex g_tuned_mu;

static bool tuned_tile(const FwdArgs& base, int split, cudaStream_t st, TilePlan* best, float* best_ms_out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const ClassTables& ct = base.ct;
    const auto key = std::make_tuple(dev, ct.la, ct.lb, ct.lc, ct.ld, ct.hrr, ct.pure, base.KB, base.KK, split);
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *best = it->second.first;
            *best_ms_out = it->second.second;
            return true;
        }
    }
    std::vector<TilePlan> cands;
    for (int TQ = 1; TQ <= 128; TQ *= 2) {
        if (TQ * ct.nab * ct.ncd > kNT * kNACC) break;
        for (int IC : {base.KB, (base.KB + 1) / 2, 1}) {
            for (int es = 1; es >= 0; --es) {
                TilePlan tp;
                if (tile_layout(ct, base.KB, base.KK, TQ, IC, es, &tp, split) && tp.acc_regs) {
                    bool dup = false;
                    for (auto& c : cands) dup |= (c.TQ == TQ && c.IC == IC && c.e_smem == es);
                    if (dup) break;
                    // a tile that leaves room for one CTA per SM is also tried
                    // with 512 threads (twice the warps in the same memory)
                    const bool wide = one_cta_per_sm(tp.bytes);
                    TilePlan tw = tp;
                    tw.nt = kNTWide;
                    if (split) {
                        add_e_ring(ct, base.KK, &tp);
                        add_e_ring(ct, base.KK, &tw);
                    }
                    cands.push_back(tp);
                    if (wide && tw.bytes <= (size_t)max_smem_optin()) cands.push_back(tw);
                    break;
                }
            }
        }
    }
    if (cands.empty()) return false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 3e38f;  // per quartet
    bool ok = false;
    for (const TilePlan& tp : cands) {
        FwdArgs a = base;
        set_tile(a, tp);
        void (*kern)(FwdArgs) = fwd_kern(split, tp.nt);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp.bytes) != cudaSuccess)
            continue;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tp.nt, tp.bytes);
        const int64_t slots = (int64_t)std::max(per_sm, 1) * sm_count();
        // about four waves of tiles (steady state), at least kTuneQuartets quartets
        const int64_t nq = std::min(base.nq, std::max(kTuneQuartets, 4 * slots * tp.TQ));
        a.ntiles = (nq + tp.TQ - 1) / tp.TQ;
        const int64_t grid = std::min<int64_t>(a.ntiles, slots);
        // one warm-up launch, then the fastest of three timed ones: candidates
        // often lie within a few per cent of each other
        float ms = 3e38f;
        bool timed = true;
        count_launch();
        kern<<<(int)grid, tp.nt, tp.bytes, st>>>(a);
        for (int rep = 0; rep < 3 && timed; ++rep) {
            float t = 0.f;
            cudaEventRecord(e0, st);
            count_launch();
            kern<<<(int)grid, tp.nt, tp.bytes, st>>>(a);
            cudaEventRecord(e1, st);
            timed = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
            ms = std::min(ms, t);
        }
        if (!timed) {
            cudaGetLastError();
            continue;
        }
        ms /= (float)nq;
        if (ms < best_ms) {
            best_ms = ms;
            *best = tp;
            ok = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ok) {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        g_tuned[key] = std::make_pair(*best, best_ms);
        *best_ms_out = best_ms;
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Processing order (build_order).  A batch may mix contraction degrees (a
// molecule's s shells of K = 6, 3 and 1); the tile loops run to the tile's
// largest primitive-pair counts, so the quartets are counting-sorted by the
// key kb (KK + 1) + kk, descending: histogram, offsets, scatter.  Equal keys
// keep no particular order (only the positions the tiles read and write from
// depend on it, not the values).
// ---------------------------------------------------------------------------
struct OrderArgs {
    const int64_t* quartets;  // NULL: product form
    int64_t nq, nbra;
    const int32_t* kpb;
    const int32_t* kpk;
    int KK, swap;
};

__device__ __forceinline__ int order_key(const OrderArgs& o, int64_t qq)
{
    int64_t ob, ok;
    if (o.quartets) {
        ob = o.quartets[2 * qq];
        ok = o.quartets[2 * qq + 1];
    } else {
        ob = qq % o.nbra;
        ok = qq / o.nbra;
    }
    const int64_t b = o.swap ? ok : ob, k = o.swap ? ob : ok;
    return o.kpb[b] * (o.KK + 1) + o.kpk[k];
}

__global__ void order_hist_kernel(OrderArgs o, unsigned long long* cnt)
{
    for (int64_t qq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qq < o.nq; qq += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[order_key(o, qq)], 1ULL);
}

__global__ void order_scan_kernel(int nbins, unsigned long long* cnt)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long run = 0;
    for (int key = nbins - 1; key >= 0; --key) {
        const unsigned long long c = cnt[key];
        cnt[key] = run;
        run += c;
    }
}

__global__ void order_scatter_kernel(OrderArgs o, unsigned long long* off, int64_t* order)
{
    for (int64_t qq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qq < o.nq; qq += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd(&off[order_key(o, qq)], 1ULL)] = qq;
}

int build_order(const int64_t* quartets, int64_t nq, int64_t nbra, const int32_t* kpb, const int32_t* kpk, int KB,
                int KK, int swap, int sort, cudaStream_t st, int64_t** order, unsigned long long** queue)
{
    int err = ERI_OK;
    const int nbins = (KB + 1) * (KK + 1);
    // [2] tile-queue counters, then (sort) [nbins] key counts and [nq] order
    const size_t n64 = 2 + (sort ? (size_t)nbins + (size_t)nq : 0);
    unsigned long long* buf = (unsigned long long*)order_workspace(sizeof(unsigned long long) * n64, &err);
    if (!buf) return err;
    *queue = buf;
    *order = nullptr;
    if (cudaMemsetAsync(buf, 0, sizeof(unsigned long long) * (sort ? 2 + (size_t)nbins : 2), st) != cudaSuccess)
        return ERI_ECUDA;
    if (!sort) return ERI_OK;
    unsigned long long* cnt = buf + 2;
    int64_t* ord = reinterpret_cast<int64_t*>(cnt + nbins);
    const OrderArgs o{quartets, nq, nbra, kpb, kpk, KK, swap};
    const int g = (int)std::min<int64_t>((nq + 255) / 256, (int64_t)sm_count() * 8);
    count_launch();
    order_hist_kernel<<<std::max(g, 1), 256, 0, st>>>(o, cnt);
    count_launch();
    order_scan_kernel<<<1, 1, 0, st>>>(nbins, cnt);
    count_launch();
    order_scatter_kernel<<<std::max(g, 1), 256, 0, st>>>(o, cnt, ord);
    if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    *order = ord;
    return ERI_OK;
}

}  // namespace eri

using namespace eri;

extern "C" int eri_boys(int mmax, const double* T, int64_t n, double* F, void* stream)
{
    if (mmax < 0 || mmax > ERI_BOYS_MMAX || n < 0) return ERI_EINVAL;
    if (n == 0) return ERI_OK;
    if (!T || !F) return ERI_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int err = ERI_OK;
    const double* tab = get_boys_table(mmax, st, &err);
    if (!tab) return err;
    const int grid = (int)std::min<int64_t>((n + 127) / 128, 16 * sm_count());
    count_launch();
    boys_kernel<<<grid, 128, 0, st>>>(mmax, T, n, tab, F);
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_ECUDA;
}

// Kernel arguments of one forward batch in form fc (the pair tables pb, pk
// of that form are built); the tile shape from the planner.
static int forward_args(const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                        const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nqq, double* out,
                        const ClassTables* ct, const PairTables& pb, const PairTables& pk, int KB, int KK, int swapped,
                        int split, cudaStream_t st, FwdArgs* a, TilePlan* tp)
{
    int err = ERI_OK;
    const double* boys = get_boys_table(ct->L, st, &err);
    if (!boys) return err;
    const RStep* rs = get_rsteps(st, &err);
    if (!rs) return err;
    if (!plan_tiles(*ct, KB, KK, nqq, tp, 0, split)) return ERI_EINVAL;
    *a = FwdArgs{};
    a->ct = *ct;
    a->boys = boys;
    a->rsteps = rs;
    a->bra_ps = pb.ps;
    a->bra_E = pb.E;
    a->bra_kp = pb.kp;
    a->ket_ps = pk.ps;
    a->ket_E = pk.E;
    a->ket_kp = pk.kp;
    a->quartets = quartets;
    a->nq = nqq;
    a->nbra = nbra;  // original roles: output layout and product-form decoding
    a->nket = nket;
    a->swap = swapped;
    const int nab_out = ct->sph ? ct->nab_s : ct->nab_f, ncd_out = ct->sph ? ct->ncd_s : ct->ncd_f;
    a->nab_o = swapped ? ncd_out : nab_out;
    a->ncd_o = swapped ? nab_out : ncd_out;
    a->out = out;
    a->bra_sh = swapped ? ket_pairs : bra_pairs;  // the kernel's lists
    a->ket_sh = swapped ? bra_pairs : ket_pairs;
    a->centres = basis->centres;
    a->shell_atom = basis->shell_atom;
    a->KB = KB;
    a->KK = KK;
    set_tile(*a, *tp);
    a->ntiles = (nqq + tp->TQ - 1) / tp->TQ;
    return ERI_OK;
}

static thread_local int g_last_form = -1;
static thread_local TilePlan g_last_tile{};

// One forward batch of any kind (0: 4-centre; 1, 2: 3-centre with the unit
// function as the second bra shell, Cartesian or solid-harmonic x): form
// choice, pair tables, tile shape, launch.  Arguments already validated.
static int run_forward(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                       const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nq, double* out,
                       int split, int kind, cudaStream_t st)
{
    const int64_t nqq = quartets ? nq : nbra * nket;
    const ClassTables* ct = nullptr;
    PairTables pb{}, pk{};
    int KB = 0, KK = 0, kmax[4];
    FormChoice fc;
    // The recursion forms are FP64 only: the horizontal recursion multiplies
    // the (e0|f0) values by powers of A-B and C-D, which magnifies the split
    // transforms' rounding (about 1e-14 of those larger values) past the
    // 1e-10 bar when the centres are far apart.  3-centre batches have none.
    const int allow = (kind == 1 || kind == 2 || split) ? 1 : 2;
    // a batch that mixes contraction degrees runs its quartets sorted by
    // (kb, kk), each tile looping to its own largest counts; the order is
    // built once, in the first form's orientation (the grouping is the same
    // in the other)
    int mixed = 0;
    int64_t* order = nullptr;
    auto prepare = [&](FormChoice* f, FwdArgs* a, TilePlan* tp) -> int {
        int e = prepare_batch(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, 0, st, &ct, &pb, &pk, &KB,
                              &KK, kmax, allow, f, split, kind, &mixed);
        if (e != ERI_OK) return e;
        e = forward_args(basis, bra_pairs, nbra, ket_pairs, nket, quartets, nqq, out, ct, pb, pk, KB, KK,
                         f->form & 1, split, st, a, tp);
        if (e != ERI_OK) return e;
        if (mixed && !order && nqq > 1) {
            unsigned long long* queue = nullptr;
            e = build_order(quartets, nqq, nbra, pb.kp, pk.kp, KB, KK, f->form & 1, 1, st, &order, &queue);
            if (e != ERI_OK) return e;
        }
        a->order = order;
        return ERI_OK;
    };
    FwdArgs a;
    TilePlan tp;
    bool from_tuner = false;
    int err = prepare(&fc, &a, &tp);
    if (err != ERI_OK) return err;
    // large batches: tile shape from the autotuner (cached per kernel class,
    // form and signature); on the first such batch of a signature, the
    // cheapest plain and horizontal-recursion forms are both timed on the
    // batch's own leading quartets and the faster is remembered
    if (nqq >= kTuneMinQuartets) {
        TilePlan best;
        float ms = 0.f;
        bool tuned = tuned_tile(a, split, st, &best, &ms);
        if (!fc.cached && fc.alt >= 0) {
            const eri_class_t sig = cls;
            const int KB0 = (fc.form & 1) ? KK : KB, KK0 = (fc.form & 1) ? KB : KK;  // caller's orientation
            FormChoice f1;
            f1.form = fc.alt;
            FwdArgs a1;
            TilePlan tp1, best1;
            float ms1 = 0.f;
            bool tuned1 = false;
            if (prepare(&f1, &a1, &tp1) == ERI_OK) tuned1 = tuned_tile(a1, split, st, &best1, &ms1);
            const bool take_alt = tuned1 && (!tuned || ms1 < ms);
            remember_form(sig, KB0, KK0, split, kind, take_alt ? f1.form : fc.form);
            if (take_alt) {
                fc = f1;
                a = a1;
                tp = tp1;
                best = best1;
                tuned = tuned1;
            } else {
                // rebuild the pair tables of the first form (the workspace was reused)
                FormChoice f0;
                f0.form = fc.form;
                err = prepare(&f0, &a, &tp);
                if (err != ERI_OK) return err;
            }
        }
        if (tuned) {
            tp = best;
            set_tile(a, tp);
            a.ntiles = (nqq + tp.TQ - 1) / tp.TQ;
            from_tuner = true;
        }
    }
    if (!from_tuner) {
        // a tile the tuner did not choose (accumulation in memory, or a small
        // batch): 512 threads when the tile leaves room for one CTA per SM
        // only (measured on (ff|ff): FP64 1.07 and 1.14 times faster at K = 5
        // and 1, split 1.27 and 1.34), then, split, the ring of ket E rows;
        // the tuner's candidates come with both settled
        if (one_cta_per_sm(tp.bytes)) tp.nt = kNTWide;
        if (split) add_e_ring(a.ct, a.KK, &tp);
        set_tile(a, tp);
    }
    void (*kern)(FwdArgs) = fwd_kern(split, tp.nt);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp.bytes) != cudaSuccess)
        return ERI_ECUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tp.nt, tp.bytes);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)per_sm * sm_count());
    {
        ProfScope ps(PROF_FWD, st);
        kern<<<(int)grid, tp.nt, tp.bytes, st>>>(a);
    }
    if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    g_last_form = fc.form;
    g_last_tile = tp;
    return ERI_OK;
}

extern "C" int eri_batch(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                         const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nq, double* out,
                         int64_t out_len, int precision, void* stream)
{
    int err = check_batch_args(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, out_len);
    if (err != ERI_OK) return err;
    if (precision != ERI_PREC_FP64 && precision != ERI_PREC_SPLIT) return ERI_EINVAL;
    const int64_t nqq = quartets ? nq : nbra * nket;
    if (nqq == 0 || nbra == 0 || nket == 0) return ERI_OK;
    if (!out) return ERI_EINVAL;
    return run_forward(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, out,
                       precision == ERI_PREC_SPLIT, 0, (cudaStream_t)stream);
}

extern "C" int eri_solid_harmonics(int32_t l, double* out)
{
    if (l < 0 || l > ERI_LMAX || !out) return ERI_EINVAL;
    solid_harmonic_table(l, out);
    return ERI_OK;
}

extern "C" int eri_batch_sph(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                             const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nq,
                             double* out, int64_t out_len, int precision, void* stream)
{
    int err = check_batch_args(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, INT64_MAX);
    if (err != ERI_OK) return err;
    if (precision != ERI_PREC_FP64 && precision != ERI_PREC_SPLIT) return ERI_EINVAL;
    const int64_t nqq = quartets ? nq : nbra * nket;
    const int64_t ns = (int64_t)(2 * cls.la + 1) * (2 * cls.lb + 1) * (2 * cls.lc + 1) * (2 * cls.ld + 1);
    if (out_len < nqq * ns) return ERI_EINVAL;
    if (nqq == 0 || nbra == 0 || nket == 0) return ERI_OK;
    if (!out) return ERI_EINVAL;
    return run_forward(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, out,
                       precision == ERI_PREC_SPLIT, 3, (cudaStream_t)stream);
}

__global__ void unit_pairs_kernel(const int32_t* __restrict__ x, int64_t n, int32_t* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out[2 * i] = x[i];
        out[2 * i + 1] = -1;
    }
}

extern "C" int eri_batch3(int32_t lx, int32_t lc, int32_t ld, const eri_basis_t* basis, const int32_t* x_shells,
                          int64_t nx, const int32_t* ket_pairs, int64_t nket, const int64_t* triples, int64_t nt,
                          int32_t pure, double* out, int64_t out_len, int precision, void* stream)
{
    const eri_class_t cls{lx, 0, lc, ld};
    if (pure != 0 && pure != 1) return ERI_EINVAL;
    // the pair-list checks of eri_batch (x shells stand in for the bra pairs)
    int err = check_batch_args(cls, basis, x_shells, nx, ket_pairs, nket, triples, nt, INT64_MAX);
    if (err != ERI_OK) return err;
    if (precision != ERI_PREC_FP64 && precision != ERI_PREC_SPLIT) return ERI_EINVAL;
    const int64_t ntt = triples ? nt : nx * nket;
    const int64_t ncx = pure ? 2 * lx + 1 : host_nc(lx);
    if (out_len < ntt * ncx * host_nc(lc) * host_nc(ld)) return ERI_EINVAL;
    if (ntt == 0 || nx == 0 || nket == 0) return ERI_OK;
    if (!out) return ERI_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t* pairs = (int32_t*)aux_workspace(sizeof(int32_t) * 2 * (size_t)nx, &err);
    if (!pairs) return err;
    const int grid = (int)std::min<int64_t>((nx + 255) / 256, 4 * sm_count());
    unit_pairs_kernel<<<std::max(grid, 1), 256, 0, st>>>(x_shells, nx, pairs);
    if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    count_launch();
    return run_forward(cls, basis, pairs, nx, ket_pairs, nket, triples, nt, out, precision == ERI_PREC_SPLIT,
                       pure ? 2 : 1, st);
}

extern "C" int eri_set_forms(int32_t mask)
{
    if (mask < 0 || mask > 0xF) return ERI_EINVAL;
    return g_form_mask.exchange(mask ? mask : 0xF);
}

extern "C" int eri_last_tile(int32_t* tq, int32_t* ic, int32_t* threads, int32_t* smem_bytes)
{
    if (g_last_form < 0) return ERI_EINVAL;
    if (tq) *tq = g_last_tile.TQ;
    if (ic) *ic = g_last_tile.IC;
    if (threads) *threads = g_last_tile.nt;
    if (smem_bytes) *smem_bytes = (int32_t)g_last_tile.bytes;
    return ERI_OK;
}

extern "C" int eri_last_form(int32_t* swapped, int32_t* hrr)
{
    if (!swapped || !hrr) return ERI_EINVAL;
    if (g_last_form < 0) return ERI_EINVAL;
    *swapped = g_last_form & 1;
    *hrr = (g_last_form >> 1) & 1;
    return ERI_OK;
}

namespace eri {

// ---------------------------------------------------------------------------
// The forward batch on tables and scratch the caller supplies (no allocation,
// no swap of the sides): used by the allocation-free entry point.  `dinfo`
// is 5 device ints, `scratch` holds the pair tables of both sides.
// ---------------------------------------------------------------------------
int fwd_batch_on(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                 int64_t nket, const int64_t* quartets, int64_t nq, double* out, const ClassTables& ct,
                 const double* boys, const RStep* rs, int* dinfo, double* scratch, size_t scratch_doubles,
                 cudaStream_t st)
{
    if (cudaMemsetAsync(dinfo, 0, 5 * sizeof(int), st) != cudaSuccess) return ERI_ECUDA;
    PrepassArgs pa{basis->shell_l, basis->shell_K, basis->nshell, bra, nbra, ket, nket, quartets,
                   quartets ? nq : (int64_t)0, {cls.la, cls.lb, cls.lc, cls.ld}, 0, dinfo, 0,
                   nullptr, nullptr, nullptr, nullptr};
    const int64_t n = std::max(std::max(nbra, nket), quartets ? nq : (int64_t)0);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * sm_count());
    count_launch();
    prepass_kernel<<<std::max(grid, 1), 256, 0, st>>>(pa);
    if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    int hinfo[5] = {0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(hinfo, dinfo, sizeof(hinfo), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ERI_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ERI_ECUDA;
    if (hinfo[4] != 0) return dev_err_to_code(hinfo[4]);
    const int KB = hinfo[0] * hinfo[1], KK = hinfo[2] * hinfo[3];
    // carve the scratch: [ps_b | E_b | ps_k | E_k | kp_b | kp_k], 32-double aligned pieces
    auto up = [](size_t d) { return (d + 31) & ~size_t(31); };
    const size_t n_psb = up((size_t)nbra * KB * PS_N), n_Eb = up((size_t)nbra * KB * ct.Tab);
    const size_t n_psk = up((size_t)nket * KK * PS_N), n_Ek = up((size_t)nket * KK * ct.Tcd);
    const size_t n_kpb = up(((size_t)nbra + 1) / 2), n_kpk = up(((size_t)nket + 1) / 2);
    if (n_psb + n_Eb + n_psk + n_Ek + n_kpb + n_kpk > scratch_doubles) return ERI_EINVAL;
    PairTables pb{}, pk{};
    pb.ps = scratch;
    pb.E = pb.ps + n_psb;
    pk.ps = pb.E + n_Eb;
    pk.E = pk.ps + n_psk;
    pb.kp = reinterpret_cast<int32_t*>(pk.E + n_Ek);
    pk.kp = reinterpret_cast<int32_t*>(pk.E + n_Ek + n_kpb);
    for (int side = 0; side < 2; ++side) {
        PairArgs p{};
        p.centres = basis->centres;
        p.shell_atom = basis->shell_atom;
        p.shell_K = basis->shell_K;
        p.shell_off = basis->shell_off;
        p.exps = basis->exps;
        p.coefs = basis->coefs;
        p.pairs = side ? ket : bra;
        p.npairs = side ? nket : nbra;
        p.l1 = side ? cls.lc : cls.la;
        p.l2 = side ? cls.ld : cls.lb;
        p.KS = side ? KK : KB;
        p.T = side ? ct.Tcd : ct.Tab;
        p.fac = side ? ct.ket_fac : ct.bra_fac;
        p.ket = side;
        const PairTables& t = side ? pk : pb;
        p.ps = t.ps;
        p.E = t.E;
        p.kprim = t.kp;
        const int64_t tot = p.npairs * p.KS;
        const int g = (int)std::min<int64_t>((tot + 127) / 128, 8 * sm_count());
        count_launch();
        launch_pair(p, std::max(g, 1), st);
        if (cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    }
    const int64_t nqq = quartets ? nq : nbra * nket;
    TilePlan tp;
    if (!plan_tiles(ct, KB, KK, nqq, &tp)) return ERI_EINVAL;
    FwdArgs a{};
    a.ct = ct;
    a.boys = boys;
    a.rsteps = rs;
    a.bra_ps = pb.ps;
    a.bra_E = pb.E;
    a.bra_kp = pb.kp;
    a.ket_ps = pk.ps;
    a.ket_E = pk.E;
    a.ket_kp = pk.kp;
    a.quartets = quartets;
    a.nq = nqq;
    a.nbra = nbra;
    a.nket = nket;
    a.swap = 0;
    a.nab_o = ct.nab_f;
    a.ncd_o = ct.ncd_f;
    a.out = out;
    a.KB = KB;
    a.KK = KK;
    set_tile(a, tp);
    a.ntiles = (nqq + tp.TQ - 1) / tp.TQ;
    if (cudaFuncSetAttribute(fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp.bytes) != cudaSuccess)
        return ERI_ECUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd_kernel, kNT, tp.bytes);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid2 = std::min<int64_t>(a.ntiles, (int64_t)per_sm * sm_count());
    count_launch();
    fwd_kernel<<<(int)grid2, kNT, tp.bytes, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_ECUDA;
}

}  // namespace eri

namespace eri {

// Pair tables of one list of shell pairs with a uniform K1*K2 = KS, written
// into caller-provided buffers (plans own theirs).
int build_pair_tables_on(const eri_basis_t* basis, const int32_t* d_pairs, int64_t npairs, int l1, int l2, int KS,
                         int T, const uint8_t* fac, int ket, int split, PairTables* out, cudaStream_t st)
{
    PairArgs p{};
    p.centres = basis->centres;
    p.shell_atom = basis->shell_atom;
    p.shell_K = basis->shell_K;
    p.shell_off = basis->shell_off;
    p.exps = basis->exps;
    p.coefs = basis->coefs;
    p.pairs = d_pairs;
    p.npairs = npairs;
    p.l1 = l1;
    p.l2 = l2;
    p.KS = KS;
    p.T = T;
    p.fac = fac;
    p.ket = ket;
    p.ps = out->ps;
    p.E = out->E;
    p.kprim = out->kp;
    p.split = split;
    const int64_t tot = npairs * KS;
    const int g = (int)std::min<int64_t>((tot + 127) / 128, 8 * sm_count());
    count_launch();
    launch_pair(p, std::max(g, 1), st);
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_ECUDA;
}

}  // namespace eri
