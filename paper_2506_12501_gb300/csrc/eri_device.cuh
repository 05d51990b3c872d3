// eri_device.cuh -- device building blocks shared by the forward and adjoint
// kernels: the Boys function and the auxiliary integrals [r]^(0).
#pragma once

#include "eri_internal.h"

namespace eri {

// 1/(2n+1), n = 0..31 (exact to the last bit of a double division)
__constant__ double c_inv_odd[32] = {
    1.0 / 1,  1.0 / 3,  1.0 / 5,  1.0 / 7,  1.0 / 9,  1.0 / 11, 1.0 / 13, 1.0 / 15, 1.0 / 17, 1.0 / 19, 1.0 / 21,
    1.0 / 23, 1.0 / 25, 1.0 / 27, 1.0 / 29, 1.0 / 31, 1.0 / 33, 1.0 / 35, 1.0 / 37, 1.0 / 39, 1.0 / 41, 1.0 / 43,
    1.0 / 45, 1.0 / 47, 1.0 / 49, 1.0 / 51, 1.0 / 53, 1.0 / 55, 1.0 / 57, 1.0 / 59, 1.0 / 61, 1.0 / 63};

// 2 pi^(5/2), the constant of Eq. 0m
constexpr double kTwoPi52 = 34.986836655249725693;
// sqrt(pi)/2
constexpr double kHalfSqrtPi = 0.88622692545275801365;

// 1/sqrt(x) for x > 0, to within about one ulp, in five FP64 operations:
// a float seed, then one third-order step of the series
//   (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + O(e^3),   e = 1 - x y0^2
// (Householder's iteration of order 2 for x^(-1/2)).  The seed is the float
// reciprocal square root of x's float image (high bits, exponent rebiased),
// widened bitwise: |e| < 2^-20, so the truncated 5e^3/16 stays below 2^-61
// and the error is that of the roundings.  No 64-bit conversion is issued.
// x outside the float range [2^-126, 2^127] takes the library's rsqrt.
__device__ __forceinline__ double rsqrt_fp64(double x)
{
    const int hi = __double2hiint(x);
    if (hi < (897 << 20) || hi >= (1151 << 20)) return rsqrt(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const float xf = __int_as_float(((hi - (896 << 20)) << 3) | (int)(lo >> 29));
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    const int yb = __float_as_int(yf);
    const double y0 = __hiloint2double((yb >> 3) + (896 << 20), yb << 29);
    const double e = fma(-x, y0 * y0, 1.0);
    return fma(y0 * e, fma(0.375, e, 0.5), y0);
}

// Nearest grid point of T (0 <= T < kBoysTmax): returns j = rint(T/step)
// and sets md = T_j - T, with no 64-bit conversion (those share the FP64
// pipe): the float image of T comes from its high bits (exponent rebiased,
// mantissa truncated; 0 below the float range), the rounding from adding
// 1.5 * 2^23, and T_j = j * 2^-5 is assembled bitwise, exactly, so md costs
// one FP64 subtraction.  The truncated image is low by less than 2^-23 T,
// i.e. 2^-9 grid steps below kBoysTmax, so |md| <= 1/64 + 2^-14.
__device__ __forceinline__ int boys_grid(double T, double& md)
{
    const int hi = __double2hiint(T);
    const unsigned lo = (unsigned)__double2loint(T);
    const int fb = hi >= (897 << 20) ? (((hi - (896 << 20)) << 3) | (int)(lo >> 29)) : 0;
    const float s = __fmaf_rn(__int_as_float(fb), (float)kBoysInvStep, 12582912.0f);  // 1.5 * 2^23
    const int j = min(__float_as_int(s) - 0x4B400000, kBoysGrid - 1);
    const int e = 31 - __clz(j);  // j = 2^e (1 + m), 0 <= e <= 13 (j > 0)
    const int thi = j > 0 ? (((1023 - kBoysLog2InvStep + e) << 20) | ((j << (20 - e)) & 0xFFFFF)) : 0;
    md = __hiloint2double(thi, 0) - T;
    return j;
}

// Boys function F_0..F_L at T (Eq. boys), written to F[0..L].
// T < kBoysTmax: F_L by its Taylor expansion about the nearest grid point
//   F_L(T0 + d) = sum_{k<7} F_{L+k}(T0) (-d)^k / k!     (|d| <= 1/64 + 2^-14)
// (table rows hold F_{L+k}(T0)/k! and exp(-T0)), exp(-T) = exp(-T0) exp(-d)
// with exp(-d) by its own degree-6 Taylor polynomial, then the downward
// recursion F_n = (2T F_{n+1} + exp(-T)) / (2n+1).
// T >= kBoysTmax: F_0 = (1/2) sqrt(pi/T) (erf(sqrt T) = 1 to double
// precision) and the upward recursion F_{n+1} = (2n+1) F_n / (2T), the
// exp(-T) term being below double precision there (Section 3.2.1).
// FP64 cost: 6 + 7 + 2L (+1) below the grid end.
__device__ __forceinline__ void boys_eval(int L, double T, const double* __restrict__ tab, double* F)
{
    if (T < kBoysTmax) {
        double md;  // -d
        const int j = boys_grid(T, md);
        const double2* row = reinterpret_cast<const double2*>(tab + (size_t)j * 8);
        const double2 r01 = __ldg(row), r23 = __ldg(row + 1), r45 = __ldg(row + 2), r67 = __ldg(row + 3);
        double f = r67.x;
        f = fma(f, md, r45.y);
        f = fma(f, md, r45.x);
        f = fma(f, md, r23.y);
        f = fma(f, md, r23.x);
        f = fma(f, md, r01.y);
        f = fma(f, md, r01.x);
        F[L] = f;
        if (L == 0) return;  // exp(-T) only feeds the downward recursion
        double e = 1.0 / 720.0;
        e = fma(e, md, 1.0 / 120.0);
        e = fma(e, md, 1.0 / 24.0);
        e = fma(e, md, 1.0 / 6.0);
        e = fma(e, md, 0.5);
        e = fma(e, md, 1.0);
        e = fma(e, md, 1.0);
        const double eT = r67.y * e;
        const double twoT = T + T;
        for (int n = L - 1; n >= 0; --n) {
            f = fma(twoT, f, eT) * c_inv_odd[n];
            F[n] = f;
        }
    } else {
        const double rt = rsqrt_fp64(T);
        const double inv2T = 0.5 * rt * rt;
        double f = kHalfSqrtPi * rt;
        F[0] = f;
        for (int n = 0; n < L; ++n) {
            f = f * ((double)(2.0f * (float)n + 1.0f) * inv2T);
            F[n + 1] = f;
        }
    }
}

// Auxiliary integrals of one primitive quartet (Eqs. 0m and r-rr):
//   R[e] = [r_e]^(0) for every Hermite function e of order <= L (tetrahedral
//   numbering), given
//   base[n] = [0]^(n) = pref (-2 rho)^n F_n(T), n = 0..L (pref less the pair
//   factors that the E tables carry),
//   X = P - Q.
// The table `st` gives for each e >= 1 the axis i and the sources e-1_i and
// e-2_i.  Level by level, n = L-1 down to 0, all entries of order 1..L-n
// are rewritten in place from the level-(n+1) values (highest order first,
// so every source is read before it is overwritten).
// FP64 cost: one multiply per entry, plus one FMA where the coefficient
// e_i - 1 is nonzero.
// The same recursion for one primitive quartet shared by the 32 lanes of a
// warp (every lane holds the same base, X, Y, Z): each level is rewritten in
// chunks of 32 entries, highest first; a chunk's lanes read their sources
// (always of lower index) before any of them writes.  All lanes must call it.
template <typename RPtr>
__device__ __forceinline__ void r_recursion_warp(int L, const double* base, double X, double Y, double Z,
                                                 const RStep* __restrict__ st, RPtr R, int lane)
{
    if (lane == 0) R[0] = base[L];
    __syncwarp();
    for (int n = L - 1; n >= 0; --n) {
        const int N = L - n;
        const int top = (N + 1) * (N + 2) * (N + 3) / 6;  // Nh(N)
        for (int c0 = top - 1; c0 >= 1; c0 -= 32) {
            const int e = c0 - lane;
            double v = 0.0;
            if (e >= 1) {
                const RStep s = st[e];
                const double x = s.axis == 0 ? X : (s.axis == 1 ? Y : Z);
                v = x * R[s.src1];
                if (s.coef) v = fma(s.coefd, R[s.src2], v);
            }
            __syncwarp();
            if (e >= 1) R[e] = v;
            __syncwarp();
        }
        if (lane == 0) R[0] = base[n];
        __syncwarp();
    }
}

// One thread per primitive quartet.  The entries are rewritten four at a
// time, every load of a group before any of its stores: the sources of an
// entry have lower indices than the entry, so a group member that is the
// source of another is read at its old (level n+1) value, and no entry
// written earlier (a higher index) is a source of any later one.  The four
// independent steps overlap their latencies, which a one-at-a-time loop
// through shared memory (each load ordered after the previous store)
// cannot.
template <typename RPtr>
__device__ __forceinline__ void r_recursion(int L, const double* base, double X, double Y, double Z,
                                            const RStep* __restrict__ st, RPtr R)
{
    R[0] = base[L];
    for (int n = L - 1; n >= 0; --n) {
        const int N = L - n;
        const int top = (N + 1) * (N + 2) * (N + 3) / 6;  // Nh(N)
        int e = top - 1;
        for (; e >= 4; e -= 4) {
            RStep s[4];
            double v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) s[j] = st[e - j];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double x = s[j].axis == 0 ? X : (s[j].axis == 1 ? Y : Z);
                v[j] = x * R[s[j].src1];
                if (s[j].coef) v[j] = fma(s[j].coefd, R[s[j].src2], v[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) R[e - j] = v[j];
        }
        for (; e >= 1; --e) {
            const RStep s = st[e];
            const double x = s.axis == 0 ? X : (s.axis == 1 ? Y : Z);
            double v = x * R[s.src1];
            if (s.coef) v = fma(s.coefd, R[s.src2], v);
            R[e] = v;
        }
        R[0] = base[n];
    }
}

// ---- compile-time L: the same Boys evaluation, prefactor scaling and
// auxiliary recursion with every loop bound known, so that the per-order
// values stay in registers and the recursion steps fold into constants.

__host__ __device__ constexpr int herm_idx_c(int t, int u, int v)
{
    return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}

// (t, u, v) of Hermite index e (the tetrahedral numbering above)
__host__ __device__ constexpr void herm_tuv_c(int e, int& t, int& u, int& v)
{
    int N = 0;
    while ((N + 1) * (N + 2) * (N + 3) / 6 <= e) ++N;
    const int r = e - N * (N + 1) * (N + 2) / 6;
    int d = 0;
    while ((d + 1) * (d + 2) / 2 <= r) ++d;
    const int w = r - d * (d + 1) / 2;
    t = N - d;
    u = d - w;
    v = N - t - u;
}

// F_0..F_L at T into F[] (registers), as boys_eval.
template <int L>
__device__ __forceinline__ void boys_eval_c(double T, const double* __restrict__ tab, double (&F)[L + 1])
{
    if (T < kBoysTmax) {
        double md;
        const int j = boys_grid(T, md);
        const double2* row = reinterpret_cast<const double2*>(tab + (size_t)j * 8);
        const double2 r01 = __ldg(row), r23 = __ldg(row + 1), r45 = __ldg(row + 2), r67 = __ldg(row + 3);
        double f = r67.x;
        f = fma(f, md, r45.y);
        f = fma(f, md, r45.x);
        f = fma(f, md, r23.y);
        f = fma(f, md, r23.x);
        f = fma(f, md, r01.y);
        f = fma(f, md, r01.x);
        F[L] = f;
        if (L == 0) return;
        double e = 1.0 / 720.0;
        e = fma(e, md, 1.0 / 120.0);
        e = fma(e, md, 1.0 / 24.0);
        e = fma(e, md, 1.0 / 6.0);
        e = fma(e, md, 0.5);
        e = fma(e, md, 1.0);
        e = fma(e, md, 1.0);
        const double eT = r67.y * e;
        const double twoT = T + T;
#pragma unroll
        for (int n = L - 1; n >= 0; --n) {
            f = fma(twoT, f, eT) * (1.0 / (2 * n + 1));
            F[n] = f;
        }
    } else {
        const double rt = rsqrt_fp64(T);
        const double inv2T = 0.5 * rt * rt;
        double f = kHalfSqrtPi * rt;
        F[0] = f;
#pragma unroll
        for (int n = 0; n < L; ++n) {
            f = f * ((double)(2 * n + 1) * inv2T);
            F[n + 1] = f;
        }
    }
}

// The auxiliary recursion of r_recursion with L known: each step's axis,
// sources and coefficient are constants.
template <int L, typename RPtr>
__device__ __forceinline__ void r_recursion_c(const double (&base)[L + 1], double X, double Y, double Z, RPtr R)
{
    R[0] = base[L];
#pragma unroll
    for (int n = L - 1; n >= 0; --n) {
        const int N = L - n;
        const int top = (N + 1) * (N + 2) * (N + 3) / 6;
#pragma unroll
        for (int e = top - 1; e >= 1; --e) {
            int r[3] = {0, 0, 0};
            herm_tuv_c(e, r[0], r[1], r[2]);
            int axis = r[0] == 1 ? 0 : (r[1] == 1 ? 1 : (r[2] == 1 ? 2 : -1));
            if (axis < 0) {
                axis = 0;
                int best = 1 << 20;
                for (int i = 0; i < 3; ++i)
                    if (r[i] > 0 && r[i] < best) {
                        best = r[i];
                        axis = i;
                    }
            }
            const int c = r[axis] - 1;
            r[axis] -= 1;
            const int s1 = herm_idx_c(r[0], r[1], r[2]);
            const double x = axis == 0 ? X : (axis == 1 ? Y : Z);
            double v = x * R[s1];
            if (c > 0) {
                r[axis] -= 1;
                v = fma((double)c, R[herm_idx_c(r[0], r[1], r[2])], v);
            }
            R[e] = v;
        }
        R[0] = base[n];
    }
}

// The auxiliary integrals of one primitive quartet (Eqs. 0m and r-rr) with
// L known: pair scalars pb (bra) and pk (ket) as the pair kernel writes them.
template <int L, typename RPtr>
__device__ __forceinline__ void aux_integrals_c(const double* pb, const double* pk, const double* __restrict__ boys,
                                                RPtr R)
{
    const double zp = pb[PS_P], zq = pk[PS_P];
    const double rs = rsqrt_fp64(zp + zq);
    const double rho = zp * zq * (rs * rs);
    const double X = pb[PS_PX] - pk[PS_PX], Y = pb[PS_PY] - pk[PS_PY], Z = pb[PS_PZ] - pk[PS_PZ];
    const double T = rho * fma(X, X, fma(Y, Y, Z * Z));
    double base[L + 1];
    boys_eval_c<L>(T, boys, base);
    // 2 pi^(5/2) / (zp zq sqrt(zp+zq)), less the pair factors carried by E
    double f = rs;
    const double m2rho = -2.0 * rho;
#pragma unroll
    for (int n = 0; n <= L; ++n) {
        base[n] *= f;
        f *= m2rho;
    }
    r_recursion_c<L>(base, X, Y, Z, R);
}

// Orders with a compile-time path.  Measured on the class sweep: 5 % faster
// for L <= 1 and 1.4 % for L = 2, while unrolled recursions of L = 3..6
// (31 to 203 steps) made those classes 1.4 to 1.6 times slower, their code
// no longer fitting the instruction cache beside the transforms.
constexpr int kLFixed = 2;

// aux_integrals_c for the runtime L if L <= kLFixed (returns false otherwise).
template <typename RPtr>
__device__ __forceinline__ bool aux_integrals_fixed(int L, const double* pb, const double* pk,
                                                    const double* __restrict__ boys, RPtr R)
{
    switch (L) {
        case 0: aux_integrals_c<0>(pb, pk, boys, R); return true;
        case 1: aux_integrals_c<1>(pb, pk, boys, R); return true;
        case 2: aux_integrals_c<2>(pb, pk, boys, R); return true;
        default: return false;
    }
}

}  // namespace eri
