// eri_internal.h -- shared host/device definitions of the GB300 ERI library.
//
// Index conventions used by every kernel:
//  * Hermite functions Lambda_(t,u,v) of total order N = t+u+v <= L are
//    numbered "tetrahedrally": all orders N = 0,1,2,... in turn, inside an
//    order by t descending then u descending.  The numbering of order <= L'
//    is a prefix of the numbering of order <= L for L' < L, so one table
//    serves every class.  Nh(L) = (L+1)(L+2)(L+3)/6 functions.
//  * Cartesian components of a shell: x^l first, then lexicographic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/eri.h"

namespace eri {

constexpr int kLmax = ERI_LMAX;            // per shell
constexpr int kKmax = ERI_KMAX;            // primitives per shell
constexpr int kLtotMax = 4 * kLmax + 2;    // largest L of an R table (gradient adds 2)
constexpr int kNhMax = (kLtotMax + 1) * (kLtotMax + 2) * (kLtotMax + 3) / 6;

// Boys-function table: grid T_j = j * kBoysStep, j = 0..kBoysGrid-1.
constexpr int kBoysInvStep = 32;           // 1/step (a power of two: T*32 is exact)
constexpr int kBoysLog2InvStep = 5;
static_assert(kBoysInvStep == 1 << kBoysLog2InvStep, "the grid step is a power of two");
constexpr double kBoysStep = 1.0 / kBoysInvStep;
// Beyond kBoysTmax the large-T form (Section 3.2.1).  The grid reaches past
// the arguments of most primitive quartets of compact basis sets (T = rho
// |P-Q|^2 up to a few hundred), so that the lanes of a warp seldom split
// between the two forms (a warp that does runs both).
constexpr double kBoysTmax = 320.0;
constexpr int kBoysGrid = (int)(kBoysTmax * kBoysInvStep) + 2;
constexpr int kBoysOrder = 7;              // Taylor terms k = 0..6, |delta| <= 1/64
constexpr int kBoysMtab = ERI_BOYS_MMAX + kBoysOrder;  // rows hold F_0..F_kBoysMtab

constexpr int host_nh(int l) { return (l + 1) * (l + 2) * (l + 3) / 6; }
constexpr int host_nc(int l) { return (l + 1) * (l + 2) / 2; }

// One step of the auxiliary recursion Eq. r-rr for Hermite function e:
//   [e]^(m) = X_axis [src1]^(m+1) + coef [src2]^(m+1)
// with src1 = e - 1_axis, src2 = e - 2_axis (coef = e_axis - 1, src2 unused if 0).
struct alignas(16) RStep {
    int16_t src1, src2;
    int8_t axis, coef;
    int16_t pad;
    double coefd;  // coef as a double (no int->double conversion on the device)
};

// Per-class tables (device copy lives in one blob; pointers into it).
struct ClassTables {
    int la, lb, lc, ld, L, Lb, Lk;
    int nab, ncd, nhb, nhk, nhl;
    int Tab, Tcd;                 // number of nonzero (component pair, Hermite) terms
    // bra terms, grouped by ab: [bra_start[ab], bra_start[ab+1])
    const int* bra_start;         // [nab+1]
    const int16_t* bra_p;         // [Tab] Hermite index of p (order <= Lb)
    const uint8_t* bra_fac;       // [Tab][6]: (ax,bx,t),(ay,by,u),(az,bz,v) -> E factor quanta
    // ket terms, grouped by cd
    const int* ket_start;         // [ncd+1]
    const int16_t* ket_q;         // [Tcd] Hermite index of q (order <= Lk)
    const uint8_t* ket_fac;       // [Tcd][6]
    const int16_t* pq;            // [nhb][nhk] Hermite index of p+q (order <= L)
    // adjoint: Hermite ranges widened by 2 on one side (shifted functions)
    int nhb2, nhk2, nhl2;         // Nh(Lb+2), Nh(Lk+2), Nh(L+2)
    const int16_t* pq2b;          // [nhb2][nhk] Hermite index of p'+q
    const int16_t* pq2k;          // [nhb][nhk2] Hermite index of p+q'
    const int16_t* herm3;         // [(t*H + u)*H + v] Hermite index, H = kLtotMax+1
    // Horizontal-recursion form (hrr = 1): the transforms produce (f0|e0)
    // with f over the Cartesians of orders la..la+lb on A and e over lc..lc+ld
    // on C (nab, ncd above then count f and e; the term lists are those of
    // E_{f,0} and E_{e,0}); after the contraction the recursions
    //   (c, d+1_i) = (c+1_i, d) + (C_i - D_i) (c, d)   on every f row,
    //   (a, b+1_i) = (a+1_i, b) + (A_i - B_i) (a, b)   on every (cd) column
    // give (ab|cd), one level |d| (|b|) = j at a time.  Level 0 of a side is
    // its (e0) list in term-list order; level j lists (c, d) with |d| = j and
    // l1 <= |c| <= l1 + l2 - j, each entry a step (src1, src2, axis) into
    // level j-1; the last level (j = l2) is in (c, d) component-pair order.
    // Solid-harmonic side (3-centre integrals): pure = 1 makes the kernel
    // bra (la, lb = 0) a real solid harmonic, pure = 2 the kernel ket
    // (lc, ld = 0).  Its rows are m = -l..l (2l+1 of them) and its terms
    // only the terminal Hermite functions |t| = l, each E product scaled by
    // the Cartesian coefficient of the harmonic (Section 2.2.3).
    int pure;
    // Solid-harmonic output (4-centre): the epilogue maps the contracted
    // Cartesian block to real solid harmonics on every centre, one index at
    // a time, with c2s[i] = [2l+1][nc(l)] of centre i (null for l = 0).
    int sph;
    int nab_s, ncd_s;             // (2la+1)(2lb+1), (2lc+1)(2ld+1)
    const double* c2s[4];
    int pb0;                      // first bra Hermite function the transforms need
    const double* bra_scale;      // [Tab] per-term factors, or null
    const double* ket_scale;      // [Tcd]
    int hrr;
    int nab_f, ncd_f;             // final component-pair counts
    int nbs, nks;                 // steps over all levels j >= 1
    int bn[4], kn[4];             // entries of level j (bn[0] = nab, kn[0] = ncd)
    int boff[4], koff[4];         // first step of level j in bsteps / ksteps
    const int16_t* bsteps;        // [nbs][3]: src1, src2, axis
    const int16_t* ksteps;        // [nks][3]
};

// Primitive-pair scalars written by the pair kernel.
// The prefactor 2 pi^(5/2) / zeta_p (bra) or 1 / zeta_q (ket) of Eq. 0m is
// not among them: it is folded into the pair's E tables (and so into its E
// products), so the kernels scale [0]^(m) by 1/sqrt(zeta_p + zeta_q) only.
enum { PS_P = 0, PS_PX, PS_PY, PS_PZ, PS_N };

// Device-side error word values (first error wins).
enum { DEV_OK = 0, DEV_ECLASS = 1, DEV_EINDEX = 2, DEV_EK = 3, DEV_ETIMEOUT = 4 };

// Host helpers implemented in eri_tables.cu
struct HostClassTables;
const ClassTables* get_class_tables(int la, int lb, int lc, int ld, cudaStream_t s, int* err);
const ClassTables* get_class_tables_hrr(int la, int lb, int lc, int ld, cudaStream_t s, int* err);
// pure: 1 = the (la, lb = 0) side a solid harmonic, 2 = the (lc, ld = 0) side
const ClassTables* get_class_tables_pure(int la, int lb, int lc, int ld, int pure, cudaStream_t s, int* err);
// Tables of the solid-harmonic output form (plain or recursion form).
const ClassTables* get_class_tables_sph(int la, int lb, int lc, int ld, int hrr, cudaStream_t s, int* err);
// Real solid harmonics (Racah normalisation) as [2l+1][nc(l)] Cartesian coefficients.
void solid_harmonic_table(int l, double* out);
const double* get_boys_table(int L, cudaStream_t s, int* err);    // rows of F_{L+k}(T_j)/k!, plus exp
const RStep* get_rsteps(cudaStream_t s, int* err);                 // recursion step table (device)
void release_all();

// Host table builders that allocate nothing (they fill the caller's
// buffers); the cached tables above and the allocation-free entry point's
// fixed tables both come from them.
//   build_boys_master: [kBoysGrid][kBoysMtab + 2] rows F_0..F_kBoysMtab(T_j), exp(-T_j);
//   boys_taylor_rows:  [kBoysGrid][8] rows F_{L+k}(T_j)/k!, k < kBoysOrder, exp(-T_j);
//   build_rstep_table: [kNhMax] steps of the auxiliary recursion;
//   pair_term_list:    nonzero (component pair, Hermite) terms of a Cartesian
//                      pair (l1, l2); returns their number (null outputs: count only).
void build_boys_master(long double* rows);
void boys_taylor_rows(const long double* master, int L, double* out);
void build_rstep_table(RStep* st);
int pair_term_list(int l1, int l2, int* start, int16_t* herm, uint8_t* fac);

// Hermite numbering helpers (host, closed forms)
int herm_index(int t, int u, int v);
void herm_tuv(int idx, int* t, int* u, int* v);

// Primitive-pair tables of one side of a batch (inside the workspace).
struct PairTables {
    double* ps;   // [npairs][KS][PS_N]
    double* E;    // [npairs][T][KS] E^x E^y E^z products, slot fastest (ket: times (-1)^{l_q})
    int32_t* kp;  // [npairs] number of primitive pairs
    double* ax;   // adjoint only: per-axis E tables with raised indices
    int eax;      // doubles per axis table
    double* zz;   // adjoint only: [npairs][KS][2] exponents
};

// Form of a forward batch: bit 0 = sides swapped (the caller's ket is the
// kernel's bra), bit 1 = horizontal-recursion form.
struct FormChoice {
    int form = -1;    // in: a form to force, or -1 (remembered, else modelled); out: the form used
    int alt = -1;     // out: the modelled-cheapest feasible form of the other kind (plain vs HRR), or -1
    int cached = 0;   // out: 1 when the form was remembered from an earlier timing
};
// Remember the measured-faster form of a (class, K_bra, K_ket, precision) signature.
void remember_form(eri_class_t cls, int KB, int KK, int split, int kind, int form);

// Prepass + pair tables shared by eri_batch, eri_batch3 and eri_batch_grad.
// ldelta = 1 also fills the adjoint tables of the bra side (pb->ax, pb->zz;
// the ket side's stay NULL, and the bra's E products are not formed);
// ldelta = 2 fills the adjoint tables and the E products of both sides.  Synchronises `st` once (reads
// the largest contraction degree of each centre).  allow_swap = 0: the plain
// form as given; 1: plain or swapped; 2: any of the four forms.  kind = 0:
// 4-centre; 1: 3-centre (the caller's bra pairs are (x, -1), -1 standing for
// the unit function, an s Gaussian of exponent 0 and coefficient 1);
// 2: 3-centre with x a real solid harmonic; 3: 4-centre with solid-harmonic
// output on every centre.
// mixed (optional out): 1 when the listed pairs of a side differ in their
// primitive-pair counts (the batch mixes contraction degrees).
int prepare_batch(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                  int64_t nket, const int64_t* quartets, int64_t nq, int ldelta, cudaStream_t st,
                  const ClassTables** ct_out, PairTables* pb, PairTables* pk, int* KB, int* KK, int kmax[4],
                  int allow_swap, FormChoice* fc, int split = 0, int kind = 0, int* mixed = nullptr);
// Processing order of a batch's quartets (list or product form, caller's
// indices): sorted by the kernel-orientation primitive-pair counts (kb, kk),
// descending, so that a tile's quartets share them (sort = 1; else *order =
// nullptr, the identity).  kpb/kpk: the kernel's per-pair counts (<= KB, KK);
// swap: the kernel's bra is the caller's ket.  *queue: two zeroed tile-queue
// counters.  Lives in order_workspace until the next call.
int build_order(const int64_t* quartets, int64_t nq, int64_t nbra, const int32_t* kpb, const int32_t* kpk, int KB,
                int KK, int swap, int sort, cudaStream_t st, int64_t** order, unsigned long long** queue);
int fwd_batch_on(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                 int64_t nket, const int64_t* quartets, int64_t nq, double* out, const ClassTables& ct,
                 const double* boys, const RStep* rs, int* dinfo, double* scratch, size_t scratch_doubles,
                 cudaStream_t st);
int check_batch_args(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra, int64_t nbra, const int32_t* ket,
                     int64_t nket, const int64_t* quartets, int64_t nq, int64_t len);
int sm_count();
int max_smem_optin();
int smem_per_sm();  // shared memory of one SM (bytes), for occupancy estimates

// Tile shape of the forward kernel for one class (eri_fwd.cu).
struct TilePlan {
    int TQ, IC, e_smem, acc_regs;
    int sEbS, sEkS;
    int o_Eb, o_Ek, o_Pb, o_Pk, o_R, o_X, o_tab, o_q;
    int o_hB, o_geo;  // horizontal-recursion form: second buffer (the first is at 0), A-B/C-D per quartet
    int o_dj;         // Coulomb digestion scratch (TQ + nab_f doubles)
    int o_Ei;         // one-quartet tile, E not staged: the bra E products of the current bra primitive ([Tab]), or -1
    int o_Er;         // split form, blocked ket stage, E not staged: three ket E rows per warp ([nt/32][3][KK] float pairs), or -1
    size_t bytes;
    int nt;           // threads per CTA: 256 (two CTAs per SM fit the registers) or 512 (one CTA per SM)
    int r_pairs;      // split form, blocked ket stage: auxiliary integrals in the paired layout (see r_row_stride)
};
// max_bytes > 0: only shapes whose shared memory stays within it; split: the
// tile runs the split-precision transforms
bool plan_tiles(const ClassTables& ct, int KB, int KK, int64_t nq, TilePlan* best, size_t max_bytes = 0,
                int split = 0);
bool tile_layout(const ClassTables& ct, int KB, int KK, int TQ, int IC, int e_smem, TilePlan* tp, int split = 0);

// The tile's auxiliary integrals [r]^(0) are a table of nhl rows (Hermite
// functions) by NI columns (quartet, bra primitive, ket primitive), ket
// primitive fastest.  Plain layout: a double per entry, the row stride odd so
// that the scattered 8-byte rows a warp reads spread over the banks.  Paired
// layout (split form, blocked ket stage): the per-(quartet, bra primitive)
// column blocks are rounded up to an even number of ket primitives, and each
// two columns k, k+1 (16 bytes) hold the float pairs as (hi_k, hi_k+1, lo_k,
// lo_k+1), so that one 16-byte load feeds two packed FP32 chains; the row
// stride is twice an odd number of such pairs.
__host__ __device__ constexpr int r_row_stride(int NI, int pairs)
{
    return pairs ? ((((NI + 1) >> 1) | 1) << 1) : (NI | 1);
}

// Measurement hook: events around launches of kernel `id` (eri_profile_*).
enum { PROF_FWD = 0, PROF_GRAD = 1, PROF_PAIR = 2, PROF_PREPASS = 3, PROF_N = 8 };
struct ProfScope {
    int id;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    ProfScope(int id, cudaStream_t st);
    ~ProfScope();
};
void count_launch();

// Device workspace (grows, cached per process; calls on one device serialise)
void* workspace(size_t bytes, int* err);
void* aux_workspace(size_t bytes, int* err);  // a second cached buffer (3-centre pair lists)
void* order_workspace(size_t bytes, int* err);  // a third (quartet processing orders, tile queues)
int* device_status();   // device error word
int32_t* host_pinned_i32(int n);

}  // namespace eri
