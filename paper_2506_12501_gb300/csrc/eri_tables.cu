// eri_tables.cu -- host-built tables of the ERI library: Hermite numbering,
// sparse Hermite<->Cartesian term lists per class, the auxiliary-recursion
// step table, the Boys-function tables, and the cached device workspace.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "eri_internal.h"

namespace eri {

// ---------------------------------------------------------------------------
// Hermite numbering (order by total N, then t descending, then u descending).
// Closed forms, no tables: the allocation-free entry point shares them.
// ---------------------------------------------------------------------------
int herm_index(int t, int u, int v)
{
    if (t < 0 || u < 0 || v < 0 || t + u + v > kLtotMax) return -1;
    const int N = t + u + v, d = N - t, e = N - t - u;
    return N * (N + 1) * (N + 2) / 6 + d * (d + 1) / 2 + e;
}

void herm_tuv(int idx, int* t, int* u, int* v)
{
    int N = 0;
    while ((N + 1) * (N + 2) * (N + 3) / 6 <= idx) ++N;
    const int r = idx - N * (N + 1) * (N + 2) / 6;
    int d = 0;  // d = N - t
    while ((d + 1) * (d + 2) / 2 <= r) ++d;
    const int e = r - d * (d + 1) / 2;  // e = N - t - u
    *t = N - d;
    *u = d - e;
    *v = N - *t - *u;
}

static std::vector<std::array<int, 3>> carts(int l)
{
    std::vector<std::array<int, 3>> r;
    for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay) r.push_back({ax, ay, l - ax - ay});
    return r;
}

// ---------------------------------------------------------------------------
// Auxiliary recursion steps, Eq. r-rr.  For each Hermite function e of order
// >= 1 pick the axis that needs the fewest FP64 operations: an axis with
// e_i = 1 needs only X_i * [e-1_i] (the e_i-1 coefficient vanishes).
// ---------------------------------------------------------------------------
void build_rstep_table(RStep* st)
{
    std::memset(st, 0, sizeof(RStep) * kNhMax);
    for (int e = 1; e < kNhMax; ++e) {
        int r[3];
        herm_tuv(e, &r[0], &r[1], &r[2]);
        int axis = -1;
        for (int i = 0; i < 3; ++i)
            if (r[i] == 1) { axis = i; break; }
        if (axis < 0)
            for (int i = 0; i < 3; ++i)
                if (r[i] > 0 && (axis < 0 || r[i] < r[axis])) axis = i;
        int d1[3] = {r[0], r[1], r[2]}, d2[3] = {r[0], r[1], r[2]};
        d1[axis] -= 1;
        d2[axis] -= 2;
        st[e].axis = (int8_t)axis;
        st[e].coef = (int8_t)(r[axis] - 1);
        st[e].coefd = (double)(r[axis] - 1);
        st[e].src1 = (int16_t)herm_index(d1[0], d1[1], d1[2]);
        st[e].src2 = (int16_t)(r[axis] >= 2 ? herm_index(d2[0], d2[1], d2[2]) : 0);
    }
}

const RStep* get_rsteps(cudaStream_t s, int* err)
{
    static std::map<int, RStep*> tabs;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = tabs.find(dev);
    if (it != tabs.end()) return it->second;
    std::vector<RStep> st(kNhMax);
    build_rstep_table(st.data());
    RStep* d = nullptr;
    if (cudaMalloc(&d, sizeof(RStep) * kNhMax) != cudaSuccess) {
        *err = ERI_ENOMEM;
        return nullptr;
    }
    if (cudaMemcpyAsync(d, st.data(), sizeof(RStep) * kNhMax, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(d);
        *err = ERI_ECUDA;
        return nullptr;
    }
    tabs[dev] = d;
    return d;
}

// Nonzero terms of a Cartesian pair (l1, l2): for every component pair
// (a, b) (a-major) every Hermite function t with t_i <= a_i + b_i on each
// axis.  start[ab]..start[ab+1]: the terms of pair ab; herm: the Hermite
// index of t; fac[3 n + i]: the per-axis E-table index (a_i, b_i, t_i).
// With null outputs only the count is returned.
int pair_term_list(int l1, int l2, int* start, int16_t* herm, uint8_t* fac)
{
    const int L12 = l1 + l2;
    int n = 0, k = 0;
    if (start) start[0] = 0;
    for (int ax = l1; ax >= 0; --ax)
        for (int ay = l1 - ax; ay >= 0; --ay)
            for (int bx = l2; bx >= 0; --bx)
                for (int by = l2 - bx; by >= 0; --by) {
                    const int a[3] = {ax, ay, l1 - ax - ay}, b[3] = {bx, by, l2 - bx - by};
                    for (int tx = 0; tx <= a[0] + b[0]; ++tx)
                        for (int ty = 0; ty <= a[1] + b[1]; ++ty)
                            for (int tz = 0; tz <= a[2] + b[2]; ++tz) {
                                if (herm) herm[n] = (int16_t)herm_index(tx, ty, tz);
                                const int tt[3] = {tx, ty, tz};
                                if (fac)
                                    for (int i = 0; i < 3; ++i)
                                        fac[3 * n + i] = (uint8_t)((a[i] * (l2 + 1) + b[i]) * (L12 + 1) + tt[i]);
                                ++n;
                            }
                    if (start) start[++k] = n;
                }
    return n;
}

// ---------------------------------------------------------------------------
// Class tables
// ---------------------------------------------------------------------------
struct ClassEntry {
    ClassTables t;
    void* blob = nullptr;
};
static std::map<std::tuple<int, int, int, int, int, int, int>, ClassEntry> g_classes;
static std::mutex g_class_mu;

// Horizontal-recursion levels of one side (l1, l2).  Level 0: the (e,0)
// functions, |e| = l1..l1+l2, in term-list order.  Level j = 1..l2: the
// pairs (c, d) with |d| = j and l1 <= |c| <= l1+l2-j, c-major, each built from
// level j-1 as (c + 1_ax, d - 1_ax) + X_ax (c, d - 1_ax), ax the first axis
// with d_ax > 0.  The last level is therefore in component-pair order.
struct HrrSide {
    std::vector<int16_t> steps;  // [n][3]: src1, src2, axis
    int n[4] = {0, 0, 0, 0};     // entries per level
    int off[4] = {0, 0, 0, 0};   // first step of each level
};

static HrrSide hrr_side(int l1, int l2)
{
    HrrSide h;
    std::vector<std::map<std::array<int, 6>, int>> idx(l2 + 1);
    for (int l = l1; l <= l1 + l2; ++l)
        for (auto& e : carts(l)) idx[0][{e[0], e[1], e[2], 0, 0, 0}] = h.n[0]++;
    for (int j = 1; j <= l2; ++j) {
        h.off[j] = (int)h.steps.size() / 3;
        for (int l = l1; l <= l1 + l2 - j; ++l)
            for (auto& c : carts(l))
                for (auto& d : carts(j)) {
                    const std::array<int, 6> key{c[0], c[1], c[2], d[0], d[1], d[2]};
                    int ax = 0;
                    while (d[ax] == 0) ++ax;
                    std::array<int, 6> s1 = key, s2 = key;
                    s1[ax] += 1;      // (c + 1_ax, d - 1_ax)
                    s1[3 + ax] -= 1;
                    s2[3 + ax] -= 1;  // (c, d - 1_ax)
                    h.steps.push_back((int16_t)idx[j - 1].at(s1));
                    h.steps.push_back((int16_t)idx[j - 1].at(s2));
                    h.steps.push_back((int16_t)ax);
                    idx[j][key] = h.n[j]++;
                }
    }
    return h;
}

// Real regular solid harmonics S_lm (Racah normalisation, m = -l..l) as
// polynomials in x, y, z, built by the recursions in l
//   S_{l+1,+(l+1)} = sqrt(2^d (2l+1)/(2l+2)) (x S_{l,l} - (1-d) y S_{l,-l}),
//   S_{l+1,-(l+1)} = sqrt(2^d (2l+1)/(2l+2)) (y S_{l,l} + (1-d) x S_{l,-l}),   d = [l == 0],
//   S_{l+1,m} = ((2l+1) z S_{l,m} - sqrt((l+m)(l-m)) r^2 S_{l-1,m}) / sqrt((l+m+1)(l-m+1)),
// from S_00 = 1; out[(m+l) * nc(l) + Cartesian index] (x^l first).
void solid_harmonic_table(int l, double* out)
{
    using Poly = std::map<std::array<int, 3>, long double>;
    auto mul = [](const Poly& P, int axis) {
        Poly R;
        for (auto& kv : P) {
            auto e = kv.first;
            ++e[axis];
            R[e] += kv.second;
        }
        return R;
    };
    auto axpy = [](Poly& Y, long double a, const Poly& X) {
        for (auto& kv : X) Y[kv.first] += a * kv.second;
    };
    std::vector<std::vector<Poly>> S(l + 1);  // S[k][m + k]
    S[0].assign(1, Poly{{{0, 0, 0}, 1.0L}});
    for (int k = 0; k < l; ++k) {
        S[k + 1].assign(2 * k + 3, Poly{});
        const long double d = k == 0 ? 1.0L : 0.0L;
        const long double f = sqrtl(powl(2.0L, d) * (2 * k + 1) / (long double)(2 * k + 2));
        const Poly& Skk = S[k][2 * k];
        const Poly& Skm = S[k][0];
        Poly top = mul(Skk, 0), bot = mul(Skk, 1);
        if (k > 0) {
            axpy(top, -1.0L, mul(Skm, 1));
            axpy(bot, 1.0L, mul(Skm, 0));
        }
        for (auto& kv : top) S[k + 1][2 * k + 2][kv.first] = f * kv.second;
        for (auto& kv : bot) S[k + 1][0][kv.first] = f * kv.second;
        for (int m = -k; m <= k; ++m) {
            Poly P;
            axpy(P, (long double)(2 * k + 1), mul(S[k][m + k], 2));
            if (k >= 1 && std::abs(m) <= k - 1) {
                const Poly& Q = S[k - 1][m + k - 1];
                const long double c = -sqrtl((long double)(k + m) * (k - m));
                for (int ax = 0; ax < 3; ++ax) axpy(P, c, mul(mul(Q, ax), ax));
            }
            const long double den = sqrtl((long double)(k + m + 1) * (k - m + 1));
            for (auto& kv : P) S[k + 1][m + k + 1][kv.first] = kv.second / den;
        }
    }
    const auto cs = carts(l);
    const int nc = (int)cs.size();
    for (int m = 0; m <= 2 * l; ++m)
        for (int i = 0; i < nc; ++i) {
            auto it = S[l][m].find({cs[i][0], cs[i][1], cs[i][2]});
            out[m * nc + i] = it == S[l][m].end() ? 0.0 : (double)it->second;
        }
}

static const ClassTables* class_tables_impl(int la, int lb, int lc, int ld, int hrr, int pure, cudaStream_t s,
                                            int* err, int sph = 0);

const ClassTables* get_class_tables(int la, int lb, int lc, int ld, cudaStream_t s, int* err)
{
    return class_tables_impl(la, lb, lc, ld, 0, 0, s, err);
}

const ClassTables* get_class_tables_hrr(int la, int lb, int lc, int ld, cudaStream_t s, int* err)
{
    return class_tables_impl(la, lb, lc, ld, 1, 0, s, err);
}

const ClassTables* get_class_tables_sph(int la, int lb, int lc, int ld, int hrr, cudaStream_t s, int* err)
{
    return class_tables_impl(la, lb, lc, ld, hrr, 0, s, err, 1);
}

const ClassTables* get_class_tables_pure(int la, int lb, int lc, int ld, int pure, cudaStream_t s, int* err)
{
    if ((pure == 1 && lb != 0) || (pure == 2 && ld != 0) || pure < 1 || pure > 2) {
        *err = ERI_EINVAL;
        return nullptr;
    }
    return class_tables_impl(la, lb, lc, ld, 0, pure, s, err);
}

static const ClassTables* class_tables_impl(int la, int lb, int lc, int ld, int hrr, int pure, cudaStream_t s,
                                            int* err, int sph)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_class_mu);
    auto key = std::make_tuple(dev, la, lb, lc, ld, hrr, pure * 2 + sph);
    auto it = g_classes.find(key);
    if (it != g_classes.end()) return &it->second.t;

    ClassTables t{};
    t.la = la; t.lb = lb; t.lc = lc; t.ld = ld;
    t.Lb = la + lb; t.Lk = lc + ld; t.L = t.Lb + t.Lk;
    t.nab = host_nc(la) * host_nc(lb);
    t.ncd = host_nc(lc) * host_nc(ld);
    t.nhb = host_nh(t.Lb); t.nhk = host_nh(t.Lk); t.nhl = host_nh(t.L);

    auto build_terms = [](int l1, int l2, std::vector<int>& start, std::vector<int16_t>& herm,
                          std::vector<uint8_t>& fac) {
        const int n = pair_term_list(l1, l2, nullptr, nullptr, nullptr);
        start.resize((size_t)host_nc(l1) * host_nc(l2) + 1);
        herm.resize(n);
        fac.resize(3 * (size_t)n);
        pair_term_list(l1, l2, start.data(), herm.data(), fac.data());
    };
    // E_{e,0} terms of the functions e with l1 <= |e| <= l1+l2 (table dims
    // (l1+l2+1) x 1 x (l1+l2+1)), in the order of the HRR level 0
    auto build_terms_hrr = [](int l1, int l2, std::vector<int>& start, std::vector<int16_t>& herm,
                              std::vector<uint8_t>& fac) {
        const int L12 = l1 + l2;
        start.push_back(0);
        for (int l = l1; l <= L12; ++l)
            for (auto& e : carts(l)) {
                for (int tx = 0; tx <= e[0]; ++tx)
                    for (int ty = 0; ty <= e[1]; ++ty)
                        for (int tz = 0; tz <= e[2]; ++tz) {
                            herm.push_back((int16_t)herm_index(tx, ty, tz));
                            const int tt[3] = {tx, ty, tz};
                            for (int i = 0; i < 3; ++i) fac.push_back((uint8_t)(e[i] * (L12 + 1) + tt[i]));
                        }
                start.push_back((int)herm.size());
            }
    };
    // a solid-harmonic side (l1, l2 = 0): row m holds the terminal Hermite
    // functions t = a, |a| = l1, of the Cartesians a in S_{l1 m}, each E
    // product (E_{a_i,0}^{a_i}) scaled by the coefficient of x^a in S_{l1 m}
    auto build_terms_pure = [](int l1, std::vector<int>& start, std::vector<int16_t>& herm,
                               std::vector<uint8_t>& fac, std::vector<double>& scale) {
        const auto cs = carts(l1);
        const int nc = (int)cs.size();
        std::vector<double> T((size_t)(2 * l1 + 1) * nc);
        solid_harmonic_table(l1, T.data());
        start.push_back(0);
        for (int m = 0; m <= 2 * l1; ++m) {
            for (int i = 0; i < nc; ++i) {
                const double c = T[(size_t)m * nc + i];
                if (std::fabs(c) < 1e-14) continue;
                herm.push_back((int16_t)herm_index(cs[i][0], cs[i][1], cs[i][2]));
                for (int x = 0; x < 3; ++x) fac.push_back((uint8_t)(cs[i][x] * (l1 + 1) + cs[i][x]));
                scale.push_back(c);
            }
            start.push_back((int)herm.size());
        }
    };
    std::vector<int> bs, ks;
    std::vector<int16_t> bp, kq, pq;
    std::vector<uint8_t> bf, kf;
    std::vector<double> bsc, ksc;
    t.pure = pure;
    t.pb0 = 0;
    if (pure) {
        if (pure == 1) {
            build_terms_pure(la, bs, bp, bf, bsc);
            build_terms(lc, ld, ks, kq, kf);
            t.nab = 2 * la + 1;
            t.pb0 = host_nh(la - 1);  // only the Hermite functions of order la
        } else {
            build_terms(la, lb, bs, bp, bf);
            build_terms_pure(lc, ks, kq, kf, ksc);
            t.ncd = 2 * lc + 1;
        }
        t.hrr = 0;
        t.nab_f = t.nab;
        t.ncd_f = t.ncd;
    } else if (hrr) {
        build_terms_hrr(la, lb, bs, bp, bf);
        build_terms_hrr(lc, ld, ks, kq, kf);
        t.hrr = 1;
        t.nab_f = t.nab;
        t.ncd_f = t.ncd;
        t.nab = (int)bs.size() - 1;
        t.ncd = (int)ks.size() - 1;
    } else {
        build_terms(la, lb, bs, bp, bf);
        build_terms(lc, ld, ks, kq, kf);
        t.hrr = 0;
        t.nab_f = t.nab;
        t.ncd_f = t.ncd;
    }
    HrrSide hb = hrr_side(la, lb), hk = hrr_side(lc, ld);
    t.nbs = (int)hb.steps.size() / 3;
    t.nks = (int)hk.steps.size() / 3;
    for (int j = 0; j < 4; ++j) {
        t.bn[j] = hb.n[j];
        t.kn[j] = hk.n[j];
        t.boff[j] = hb.off[j];
        t.koff[j] = hk.off[j];
    }
    t.Tab = (int)bp.size();
    t.Tcd = (int)kq.size();
    auto sum_table = [](int n1, int n2, std::vector<int16_t>& out) {
        out.resize((size_t)n1 * n2);
        for (int p = 0; p < n1; ++p)
            for (int q = 0; q < n2; ++q) {
                int a, b, c, x, y, z;
                herm_tuv(p, &a, &b, &c);
                herm_tuv(q, &x, &y, &z);
                out[(size_t)p * n2 + q] = (int16_t)herm_index(a + x, b + y, c + z);
            }
    };
    sum_table(t.nhb, t.nhk, pq);
    t.nhb2 = host_nh(t.Lb + 2);
    t.nhk2 = host_nh(t.Lk + 2);
    t.nhl2 = host_nh(t.L + 2);
    std::vector<int16_t> pq2b, pq2k, h3;
    sum_table(t.nhb2, t.nhk, pq2b);
    sum_table(t.nhb, t.nhk2, pq2k);
    {
        const int H = kLtotMax + 1;
        h3.assign((size_t)H * H * H, -1);
        for (int a = 0; a < H; ++a)
            for (int b = 0; b < H; ++b)
                for (int c = 0; c < H; ++c) h3[((size_t)a * H + b) * H + c] = (int16_t)herm_index(a, b, c);
    }
    // one blob: ints first (aligned), then int16, then uint8
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) & ~size_t(15);
        return o;
    };
    size_t o_bs = take(bs.size() * 4), o_ks = take(ks.size() * 4);
    size_t o_bp = take(bp.size() * 2), o_kq = take(kq.size() * 2), o_pq = take(pq.size() * 2);
    size_t o_pq2b = take(pq2b.size() * 2), o_pq2k = take(pq2k.size() * 2), o_h3 = take(h3.size() * 2);
    size_t o_bst = take(hb.steps.size() * 2 + 2), o_kst = take(hk.steps.size() * 2 + 2);
    // solid-harmonic output: the four centres' coefficient tables
    const int ls[4] = {la, lb, lc, ld};
    std::vector<double> c2s[4];
    size_t o_c2s[4] = {0, 0, 0, 0};
    t.sph = sph;
    t.nab_s = (2 * la + 1) * (2 * lb + 1);
    t.ncd_s = (2 * lc + 1) * (2 * ld + 1);
    for (int i = 0; i < 4; ++i) {
        if (!sph || ls[i] == 0) continue;
        c2s[i].resize((size_t)(2 * ls[i] + 1) * host_nc(ls[i]));
        solid_harmonic_table(ls[i], c2s[i].data());
        o_c2s[i] = take(c2s[i].size() * 8);
    }
    size_t o_bsc = take(bsc.size() * 8), o_ksc = take(ksc.size() * 8);
    size_t o_bf = take(bf.size()), o_kf = take(kf.size());
    std::vector<uint8_t> host(off);
    for (int i = 0; i < 4; ++i)
        if (!c2s[i].empty()) std::memcpy(host.data() + o_c2s[i], c2s[i].data(), c2s[i].size() * 8);
    if (!bsc.empty()) std::memcpy(host.data() + o_bsc, bsc.data(), bsc.size() * 8);
    if (!ksc.empty()) std::memcpy(host.data() + o_ksc, ksc.data(), ksc.size() * 8);
    std::memcpy(host.data() + o_bs, bs.data(), bs.size() * 4);
    std::memcpy(host.data() + o_ks, ks.data(), ks.size() * 4);
    std::memcpy(host.data() + o_bp, bp.data(), bp.size() * 2);
    std::memcpy(host.data() + o_kq, kq.data(), kq.size() * 2);
    std::memcpy(host.data() + o_pq, pq.data(), pq.size() * 2);
    std::memcpy(host.data() + o_pq2b, pq2b.data(), pq2b.size() * 2);
    std::memcpy(host.data() + o_pq2k, pq2k.data(), pq2k.size() * 2);
    std::memcpy(host.data() + o_h3, h3.data(), h3.size() * 2);
    if (!hb.steps.empty()) std::memcpy(host.data() + o_bst, hb.steps.data(), hb.steps.size() * 2);
    if (!hk.steps.empty()) std::memcpy(host.data() + o_kst, hk.steps.data(), hk.steps.size() * 2);
    std::memcpy(host.data() + o_bf, bf.data(), bf.size());
    std::memcpy(host.data() + o_kf, kf.data(), kf.size());
    void* blob = nullptr;
    if (cudaMalloc(&blob, off) != cudaSuccess) {
        *err = ERI_ENOMEM;
        return nullptr;
    }
    if (cudaMemcpyAsync(blob, host.data(), off, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(blob);
        *err = ERI_ECUDA;
        return nullptr;
    }
    uint8_t* b = (uint8_t*)blob;
    t.bra_start = (const int*)(b + o_bs);
    t.ket_start = (const int*)(b + o_ks);
    t.bra_p = (const int16_t*)(b + o_bp);
    t.ket_q = (const int16_t*)(b + o_kq);
    t.pq = (const int16_t*)(b + o_pq);
    t.pq2b = (const int16_t*)(b + o_pq2b);
    t.pq2k = (const int16_t*)(b + o_pq2k);
    t.herm3 = (const int16_t*)(b + o_h3);
    t.bsteps = (const int16_t*)(b + o_bst);
    t.ksteps = (const int16_t*)(b + o_kst);
    t.bra_fac = b + o_bf;
    t.ket_fac = b + o_kf;
    for (int i = 0; i < 4; ++i) t.c2s[i] = c2s[i].empty() ? nullptr : (const double*)(b + o_c2s[i]);
    t.bra_scale = bsc.empty() ? nullptr : (const double*)(b + o_bsc);
    t.ket_scale = ksc.empty() ? nullptr : (const double*)(b + o_ksc);
    ClassEntry& e = g_classes[key];
    e.t = t;
    e.blob = blob;
    return &e.t;
}

// ---------------------------------------------------------------------------
// Boys tables.  Master rows: F_m(T_j), m = 0..kBoysMtab, then exp(-T_j),
// computed in long double: the top order by the series
//   F_M(T) = exp(-T) sum_k (2T)^k / ((2M+1)(2M+3)...(2M+2k+1))
// (all terms positive) and the lower orders by the downward recursion
//   F_m(T) = (2T F_{m+1}(T) + exp(-T)) / (2m+1),
// which is stable for every T.
// Per-L rows (8 doubles, one 64-byte line): F_{L+k}(T_j)/k!, k = 0..6, and
// exp(-T_j): the coefficients of the Taylor expansion about T_j used by the
// kernels' Boys evaluation.
// ---------------------------------------------------------------------------
void build_boys_master(long double* rows)
{
    const int W = kBoysMtab + 2;
    for (int j = 0; j < kBoysGrid; ++j) {
        const long double T = (long double)j / kBoysInvStep;
        const long double eT = expl(-T);
        long double term = 1.0L / (2 * kBoysMtab + 1), sum = term;
        for (int k = 1; k < 10000; ++k) {
            term *= 2.0L * T / (long double)(2 * kBoysMtab + 2 * k + 1);
            sum += term;
            if (term < sum * 1e-22L) break;
        }
        long double* row = rows + (size_t)j * W;
        row[kBoysMtab] = eT * sum;
        for (int m = kBoysMtab - 1; m >= 0; --m) row[m] = (2.0L * T * row[m + 1] + eT) / (long double)(2 * m + 1);
        row[kBoysMtab + 1] = eT;
    }
}

void boys_taylor_rows(const long double* master, int L, double* out)
{
    const int W = kBoysMtab + 2;
    long double fact[kBoysOrder];
    fact[0] = 1;
    for (int k = 1; k < kBoysOrder; ++k) fact[k] = fact[k - 1] * k;
    for (int j = 0; j < kBoysGrid; ++j) {
        const long double* row = master + (size_t)j * W;
        for (int k = 0; k < kBoysOrder; ++k) out[(size_t)j * 8 + k] = (double)(row[L + k] / fact[k]);
        out[(size_t)j * 8 + 7] = (double)row[kBoysMtab + 1];
    }
}

static std::vector<long double> g_master_host;
static std::once_flag g_master_once;

static void build_master()
{
    g_master_host.assign((size_t)kBoysGrid * (kBoysMtab + 2), 0.0L);
    build_boys_master(g_master_host.data());
}

static std::map<std::pair<int, int>, double*> g_boys_tabs;
static std::mutex g_boys_mu;

const double* get_boys_table(int L, cudaStream_t s, int* err)
{
    std::call_once(g_master_once, build_master);
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_boys_mu);
    auto key = std::make_pair(dev, L);
    auto it = g_boys_tabs.find(key);
    if (it != g_boys_tabs.end()) return it->second;
    std::vector<double> tab((size_t)kBoysGrid * 8);
    boys_taylor_rows(g_master_host.data(), L, tab.data());
    double* d = nullptr;
    if (cudaMalloc(&d, tab.size() * sizeof(double)) != cudaSuccess) {
        *err = ERI_ENOMEM;
        return nullptr;
    }
    if (cudaMemcpyAsync(d, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(d);
        *err = ERI_ECUDA;
        return nullptr;
    }
    g_boys_tabs[key] = d;
    return d;
}

// ---------------------------------------------------------------------------
// Workspace, status word, pinned scratch
// ---------------------------------------------------------------------------
struct DevState {
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* aux = nullptr;
    size_t aux_bytes = 0;
    void* ord = nullptr;
    size_t ord_bytes = 0;
    int* status = nullptr;
};
static std::map<int, DevState> g_dev;
static std::mutex g_dev_mu;

void* workspace(size_t bytes, int* err)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevState& d = g_dev[dev];
    if (bytes <= d.ws_bytes) return d.ws;
    if (d.ws) {
        cudaDeviceSynchronize();
        cudaFree(d.ws);
        d.ws = nullptr;
        d.ws_bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&d.ws, want) != cudaSuccess) {
        cudaGetLastError();
        *err = ERI_ENOMEM;
        return nullptr;
    }
    d.ws_bytes = want;
    return d.ws;
}

void* aux_workspace(size_t bytes, int* err)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevState& d = g_dev[dev];
    if (bytes <= d.aux_bytes) return d.aux;
    if (d.aux) {
        cudaDeviceSynchronize();
        cudaFree(d.aux);
        d.aux = nullptr;
        d.aux_bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&d.aux, want) != cudaSuccess) {
        cudaGetLastError();
        *err = ERI_ENOMEM;
        return nullptr;
    }
    d.aux_bytes = want;
    return d.aux;
}

void* order_workspace(size_t bytes, int* err)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevState& d = g_dev[dev];
    if (bytes <= d.ord_bytes) return d.ord;
    if (d.ord) {
        cudaDeviceSynchronize();
        cudaFree(d.ord);
        d.ord = nullptr;
        d.ord_bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&d.ord, want) != cudaSuccess) {
        cudaGetLastError();
        *err = ERI_ENOMEM;
        return nullptr;
    }
    d.ord_bytes = want;
    return d.ord;
}

int* device_status()
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevState& d = g_dev[dev];
    if (!d.status) {
        if (cudaMalloc(&d.status, 128) != cudaSuccess) return nullptr;
        cudaMemset(d.status, 0, 128);
        cudaDeviceSynchronize();
    }
    return d.status;
}

int32_t* host_pinned_i32(int n)
{
    static int32_t* p = nullptr;
    static int cap = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (n > cap) {
        if (p) cudaFreeHost(p);
        if (cudaMallocHost(&p, sizeof(int32_t) * n) != cudaSuccess) {
            p = nullptr;
            cap = 0;
            return nullptr;
        }
        cap = n;
    }
    return p;
}

void release_all()
{
    {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        int dev = 0;
        cudaGetDevice(&dev);
        auto it = g_dev.find(dev);
        if (it != g_dev.end()) {
            if (it->second.ws) cudaFree(it->second.ws);
            if (it->second.aux) cudaFree(it->second.aux);
            if (it->second.ord) cudaFree(it->second.ord);
            if (it->second.status) cudaFree(it->second.status);
            g_dev.erase(it);
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_class_mu);
        for (auto& kv : g_classes) cudaFree(kv.second.blob);
        g_classes.clear();
    }
    {
        std::lock_guard<std::mutex> lk(g_boys_mu);
        for (auto& kv : g_boys_tabs) cudaFree(kv.second);
        g_boys_tabs.clear();
    }
}

}  // namespace eri
