/*
 * eri.h -- C ABI of the GB300 McMurchie-Davidson 4-centre ERI library.
 *
 * The library evaluates batches of contracted Cartesian shellsets (ab|cd)
 * (Eq. def-abcd of arXiv 2506.12501, contracted as in Section 2.1) of one
 * angular-momentum class at a time, by the MD sequence of Eq. md-2body:
 *   [0]^(m) (Eq. 0m, Boys function Eq. boys)
 *     -> [r]^(0) (Eq. r-rr) -> [p|q] (Eq. pq-from-r)
 *     -> [p|cd] (Eq. ket-from-hermite, ket contracted first)
 *     -> [ab|cd] (Eq. bra-from-hermite, bra contracted),
 * with Cartesian transforms E built by Eqs. E2rr1/E2rr2/E2-000.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every array argument is DEVICE memory owned by the caller, except where
 *   a comment says "host".  The library never frees caller memory.
 * - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *   NULL = legacy default stream).  Pointers must stay valid until the work
 *   queued on the stream has completed (for plans: until eri_plan_destroy).
 * - Return value: ERI_OK (0) or a negative error code; eri_error_string()
 *   describes it.  Argument errors are detected on the host before any
 *   launch and leave outputs untouched.  ERI_ECUDA reports a failed CUDA
 *   call (launch or allocation).
 * - The library allocates only internal workspace (pair tables, class
 *   tables, the Boys table), cached per device and reused between calls;
 *   eri_finalize() releases it.  Calls on different streams of one device
 *   must not overlap in time (they share that workspace).
 * - Shells: angular momentum 0 <= l <= ERI_LMAX, contraction degree
 *   1 <= K <= ERI_KMAX.  Contraction coefficients are used verbatim (no
 *   normalisation is applied by the library).
 * - Cartesian components of a shell are ordered x^l first, then
 *   lexicographically (xx, xy, xz, yy, yz, zz for l = 2); a pair index is
 *   ab = a*nc(lb) + b with nc(l) = (l+1)(l+2)/2.
 */
#ifndef ERI_H
#define ERI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ERI_LMAX 3
#define ERI_KMAX 8

enum {
    ERI_OK = 0,
    ERI_EINVAL = -1,   /* bad argument: l or K out of range, NULL pointer, sizes */
    ERI_ECLASS = -2,   /* a pair's shell angular momenta disagree with the class */
    ERI_ECUDA = -3,    /* a CUDA call failed */
    ERI_ETIMEOUT = -4, /* a bounded device-side wait ran out (plan execution) */
    ERI_ENOMEM = -5,   /* workspace allocation failed */
    ERI_EPLAN = -6     /* plan misuse (wrong buffers for the plan's mode) */
};

/* Precision of the Hermite-to-Cartesian transforms. */
enum {
    ERI_PREC_FP64 = 0,  /* everything in FP64 */
    ERI_PREC_SPLIT = 1  /* transforms in FP32 hi+lo split products with FP64
                           accumulation; Boys, R and prefactors stay FP64;
                           plain (side-swapped or not) forms only, since the
                           horizontal recursion would magnify their rounding */
};

typedef struct {
    int32_t la, lb, lc, ld;
} eri_class_t;

/* A basis set: shells on atoms, primitives back to back (all DEVICE). */
typedef struct {
    const double* centres;     /* [natom][3] bohr */
    const int32_t* shell_atom; /* [nshell] atom of each shell */
    const int32_t* shell_l;    /* [nshell] angular momentum */
    const int32_t* shell_K;    /* [nshell] contraction degree */
    const int32_t* shell_off;  /* [nshell] first primitive of the shell */
    const double* exps;        /* [nprim] exponents (> 0) */
    const double* coefs;       /* [nprim] contraction coefficients */
    int32_t natom, nshell, nprim;
} eri_basis_t;

/*
 * eri_boys -- the Boys function F_m(T) = int_0^1 y^{2m} exp(-T y^2) dy
 * (Eq. boys), evaluated as the integral kernels do: Taylor interpolation of
 * F_mmax on a tabulated grid, then downward recursion
 *     F_m = (2T F_{m+1} + exp(-T)) / (2m+1);
 * for T beyond the grid the large-T form F_0 = (1/2) sqrt(pi/T) with the
 * upward recursion (Section 3.2.1).
 *   T: [n] arguments (T >= 0, finite); F: [n][mmax+1] results, F[i*(mmax+1)+m].
 *   0 <= mmax <= ERI_BOYS_MMAX.  n == 0 is a no-op.
 */
#define ERI_BOYS_MMAX 20
int eri_boys(int mmax, const double* T, int64_t n, double* F, void* stream);

/*
 * eri_batch -- contracted Cartesian shellsets (ab|cd) of class `cls` for a
 * batch (Section 3.1: bra shell-pair list x ket shell-pair list).
 *   bra_pairs: [nbra][2] shell indices (a, b) with l = (la, lb);
 *   ket_pairs: [nket][2] shell indices (c, d) with l = (lc, ld);
 *   quartets:  NULL => every (bra, ket) combination ("product form");
 *              else [nq][2] (bra index, ket index) ("list form").
 *   out: [out_len] doubles, written (not accumulated).  Layout, with
 *        nab = nc(la) nc(lb), ncd = nc(lc) nc(ld):
 *        product form  out[ij + nbra*(ab + nab*(cd + ncd*kl))]
 *                      (the [ij,ab,cd,kl] column-major layout of Section 3.1),
 *                      out_len >= nbra*nket*nab*ncd;
 *        list form     out[q + nq*(ab*ncd + cd)], out_len >= nq*nab*ncd.
 *   precision: ERI_PREC_FP64 or ERI_PREC_SPLIT.
 * Before any integral kernel runs, a validation kernel checks every shell
 * and quartet index (ERI_EINVAL if out of range), every contraction degree
 * (ERI_EINVAL if outside 1..ERI_KMAX) and every shell's angular momentum
 * against `cls` (ERI_ECLASS); its verdict and the largest contraction degree
 * per centre are read back, so each call synchronises `stream` once.  On an
 * error `out` is left untouched.
 * Shared memory bounds the primitive-pair counts: a tile holds the
 * auxiliary integrals of every ket primitive pair of one quartet.  With the
 * same K on all four shells, K = 8 fits for L = la+lb+lc+ld <= 10, K = 7 for
 * L = 11 and K = 6 for L = 12 (the cheaper side order is taken); beyond,
 * no tile fits and the call returns ERI_EINVAL.
 * nbra == 0, nket == 0 or nq == 0 is a no-op.
 */
int eri_batch(eri_class_t cls, const eri_basis_t* basis,
              const int32_t* bra_pairs, int64_t nbra,
              const int32_t* ket_pairs, int64_t nket,
              const int64_t* quartets, int64_t nq,
              double* out, int64_t out_len, int precision, void* stream);

/*
 * eri_batch_grad -- adjoint of eri_batch: accumulates the derivatives of
 *   E = sum_{quartets} sum_{abcd} W_abcd (ab|cd)
 * with respect to the atom centres and the primitive exponents (the
 * contraction coefficients are held fixed), by differentiating each
 * primitive Gaussian (Section 2.1) and recomputing the forward Hermite
 * intermediates.
 *   W: same layout and length as eri_batch's `out` for the same arguments;
 *   grad_centres: [natom][3], ACCUMULATED (+=);
 *   grad_exps:    [nprim],    ACCUMULATED (+=).
 * Either gradient pointer may be NULL to skip that part.
 * Its tiles hold the auxiliary integrals to order L+2 of every ket primitive
 * pair of a quartet, which bounds the contraction degrees more tightly than
 * the forward's: with the same K on all four shells, every class fits
 * K = 8 for L <= 4, K = 5 for L = 5, K = 3 for L = 6..9, K = 2 for L = 10
 * and K = 1 for L = 11, 12.  These bounds are reached by the classes with a
 * d-f or f-f pair; the others fit more.  Uncontracted d and f shells with s
 * and p shells of any K <= ERI_KMAX always fit.  Beyond, the call returns
 * ERI_EINVAL.
 */
int eri_batch_grad(eri_class_t cls, const eri_basis_t* basis,
                   const int32_t* bra_pairs, int64_t nbra,
                   const int32_t* ket_pairs, int64_t nket,
                   const int64_t* quartets, int64_t nq,
                   const double* W, int64_t w_len,
                   double* grad_centres, double* grad_exps, void* stream);

/*
 * eri_last_grad_forms -- the forms the last eri_batch_grad call ran.
 * The channels of a side come from one of two forms: ERI_GRAD_X (the
 * forward ket transform over the raised bra range, X'[p'][cd], contracted
 * with W per channel item) or ERI_GRAD_V (W contracted with the ket E
 * products once per quartet, V_k[ab][q], then each channel item's T from V
 * and the auxiliary integrals).  A call runs either one launch, whose bra
 * channels take the X or V form and whose ket channels come from the same
 * auxiliary integrals (Y'_k[ab][q'] = sum_i sum_p E^ab_{i,p} [p+q']_{ik}
 * over the raised ket range, accumulated over the bra primitives), or two
 * launches, the second with the sides exchanged.  *bra_form: the form of the
 * first launch's kernel-bra channels; *ket_form: ERI_GRAD_ONE for the single
 * launch with the caller's bra as its kernel bra, ERI_GRAD_ONE_SWAPPED for
 * the single launch with the caller's ket as its kernel bra (whose channels
 * *bra_form then describes), else the second launch's form.  All give the same derivatives to
 * round-off; a cost model picks per call, except that the first list-form
 * batch of at least 65536 quartets of a class (per device, with every scheme
 * allowed) times one launch against two on its first 32768 quartets, into
 * scratch gradients, and keeps the faster scheme for the class (the model
 * still picks the single launch's orientation and the forms).  ERI_EINVAL
 * before any call.
 * eri_set_grad_forms -- restrict the planner (process-wide; for testing):
 * bits ERI_GRAD_X and ERI_GRAD_V allow those forms, bit ERI_GRAD_ONE the
 * single launch, bit ERI_GRAD_TWO two launches; a mask with neither of the
 * last two bits means two launches; 0 allows everything.  Returns the
 * previous mask, or ERI_EINVAL for a mask outside 0..15.  A call for which
 * no tile of an allowed form fits in shared memory returns ERI_EINVAL (with
 * everything allowed, the two-launch X form's smallest tile always fits for
 * l <= ERI_LMAX and K <= ERI_KMAX).
 */
#define ERI_GRAD_X 0
#define ERI_GRAD_V 1
#define ERI_GRAD_ONE 2
#define ERI_GRAD_TWO 3
#define ERI_GRAD_ONE_SWAPPED 4  /* a form value of eri_last_grad_forms, not a mask bit */
int eri_last_grad_forms(int32_t* bra_form, int32_t* ket_form);
int eri_set_grad_forms(int32_t mask);

/*
 * eri_batch3 -- 3-centre integrals
 *   (x|cd) = int int phi_x(r1) |r1 - r2|^-1 phi_c(r2) phi_d(r2) dr1 dr2
 * of one class (lx | lc ld) for a batch: x from a list of single shells
 * (e.g. a density-fitting basis), cd from ket pairs as in eri_batch.
 *   x_shells: [nx] shell indices of angular momentum lx (DEVICE).
 *   triples:  NULL => every (x, ket) combination; else [nt][2] (x index,
 *             ket index), int64 (DEVICE).
 *   pure:     1 => x is a real solid harmonic (2 lx + 1 components,
 *             m = -lx..lx, Racah normalisation: S_l0(0,0,1) = 1, and
 *             S_lm over the unit sphere has norm 4 pi / (2l + 1)), whose
 *             transform uses only the terminal Hermite functions of order lx
 *             (Section 2.2.3); 0 => Cartesian x (nc(lx) components).
 *   out:      list form out[t + nt*(x*ncd + cd)]; product form
 *             out[i + nx*(x + nxc*(cd + ncd*k))], nxc the x component count.
 * The batch runs as the 4-centre kernel on (x 1|cd), 1 being the unit
 * function (an s Gaussian of exponent 0, coefficient 1), in the cheaper of
 * the two side orders.  precision as in eri_batch.  Synchronises `stream`
 * once.  Errors: ERI_EINVAL (l out of range, bad pointers, out_len too
 * small, a shell index out of range), ERI_ECLASS (an x shell's l is not lx
 * or a ket shell's l disagrees), ERI_ECUDA, ERI_ENOMEM.
 */
/*
 * eri_batch_sph -- the same batch as eri_batch with every centre in real
 * solid harmonics (the functions of eri_solid_harmonics, m = -l..l): each
 * shellset has (2la+1)(2lb+1)(2lc+1)(2ld+1) integrals,
 * (ma mb|mc md) = sum C^a_ma C^b_mb C^c_mc C^d_md (ab|cd), laid out as in
 * eri_batch with ab = (ma+la)(2lb+1) + (mb+lb) and likewise cd.  The
 * transforms run on Cartesians (in any of the four forms); the mapping to
 * solid harmonics is applied to the contracted block in the kernel's
 * epilogue, so only the smaller solid-harmonic block is stored (the paper
 * fuses these coefficients into its H matrices, Section 2.1).  Arguments,
 * errors and synchronisation as in eri_batch.
 */
int eri_batch_sph(eri_class_t cls, const eri_basis_t* basis,
                  const int32_t* bra_pairs, int64_t nbra,
                  const int32_t* ket_pairs, int64_t nket,
                  const int64_t* quartets, int64_t nq,
                  double* out, int64_t out_len, int precision, void* stream);

/*
 * eri_solid_harmonics -- the real solid harmonics eri_batch3 and eri_batch_sph use, as
 * Cartesian coefficients: S_lm = sum_a out[(m+l)*nc(l) + a] x^ax y^ay z^az,
 * m = -l..l, a in the library's Cartesian order.  out is a HOST buffer of
 * (2l+1) nc(l) doubles; no GPU work.  ERI_EINVAL for l outside 0..ERI_LMAX.
 */
int eri_solid_harmonics(int32_t l, double* out);

int eri_batch3(int32_t lx, int32_t lc, int32_t ld, const eri_basis_t* basis,
               const int32_t* x_shells, int64_t nx,
               const int32_t* ket_pairs, int64_t nket,
               const int64_t* triples, int64_t nt, int32_t pure,
               double* out, int64_t out_len, int precision, void* stream);

/*
 * eri_batch_noalloc -- the same integrals as eri_batch (FP64, list or
 * product form, same layout and errors), for callers that may not allocate
 * memory: the paper has no counterpart of this entry point.
 *
 * Who needs it: a process whose device memory belongs to another allocator
 * (a serving or training framework's caching pool, an MPI library's
 * registered pool) may not call cudaMalloc itself: memory that allocator
 * does not know about can make its own allocations fail or break its
 * accounting.  eri_batch caches its scratch (the primitive-pair tables) in
 * memory it allocates; this entry point instead keeps that scratch in a
 * fixed device array of ERI_NOALLOC_SCRATCH_BYTES, compiled into the
 * library, and its constant tables in fixed arrays as well.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * - The fixed arrays take ERI_NOALLOC_SCRATCH_BYTES (+ about 10 MB of
 *   tables) on every GPU that loads the library, until the process exits.
 * - A batch needs 8*(nbra*KB*(T_ab+4) + nket*KK*(T_cd+4)) bytes of scratch
 *   plus small padding (KB = largest K_a*K_b, T_ab = nonzero Hermite terms
 *   of the class); a larger batch is rejected with ERI_EINVAL before any
 *   integral kernel runs.  Split such batches.
 * - The first call on a device sets that device up (the device must be
 *   current): it fills the constant tables with synchronous copies and
 *   looks up the arrays' device addresses.
 * - Every call uses the same arrays, which keep the last call's contents;
 *   the call clears what must start at zero.  Calls whose GPU work overlaps
 *   in time (different streams, or several host threads) race on them:
 *   serialise them.
 * - Like eri_batch, each call synchronises `stream` once (validation).
 * - precision is always FP64; the sides are never swapped.  The bounds on
 *   the contraction degrees are therefore those of the side order given
 *   (the ket is transformed first, and a tile holds the auxiliary integrals
 *   of every ket primitive pair of a quartet), which can be tighter than
 *   eri_batch's, which takes the cheaper order: a batch no tile can hold in
 *   this order returns ERI_EINVAL.  Exchanging the bra and ket lists (and
 *   reading the output transposed) may make it fit.
 */
#define ERI_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int eri_batch_noalloc(eri_class_t cls, const eri_basis_t* basis,
                      const int32_t* bra_pairs, int64_t nbra,
                      const int32_t* ket_pairs, int64_t nket,
                      const int64_t* quartets, int64_t nq,
                      double* out, int64_t out_len, void* stream);

/*
 * Plans: the batched form over a whole basis.
 *
 * eri_plan_create -- every unique shell quartet (pair P >= pair Q over the
 * unique shell pairs i >= j) of `basis` whose Schwarz bound
 * Q_P Q_Q, Q_P = sqrt(max_ab |(ab|ab)|), reaches `threshold` (<= 0 keeps
 * every quartet), all classes together (batch-level screening, Section 3.1).
 * The plan copies the shell table to the host once (synchronising
 * `stream`), computes the Schwarz factors with eri_batch, buckets the pairs
 * by (class, contraction signature), sorts them by Q, builds the pair
 * tables and a device work queue, and owns all of it until
 * eri_plan_destroy.  The basis arrays must stay valid and unchanged for the
 * plan's lifetime.
 *   flags: ERI_PLAN_STORE  keep every integral (eri_plan_execute writes
 *                          them, job after job; for verification sizes);
 *          ERI_PLAN_SPLIT  split-precision transforms.
 * eri_plan_execute -- one persistent kernel over the queue, replayed as a
 * CUDA graph (captured on the first call).  Without ERI_PLAN_STORE it
 * writes *energy = sum over the plan's quartets of
 * sum_abcd D_ab D_cd (ab|cd) (D: [nbf][nbf] device, nbf = the number of
 * Cartesian functions of the basis, shells in order), and `out` must be
 * NULL.  With ERI_PLAN_STORE it writes the integrals to `out` (out_len >=
 * eri_plan_info's out_len): job j (see eri_plan_job) at offset out_off, in
 * the list-form layout of eri_batch for its own class and quartet order.
 * eri_plan_coulomb -- the same replay digesting into the Coulomb matrix:
 * J[u][v] = sum over all (l, s) of (uv|ls) D[l][s] for every Cartesian
 * function pair (u, v) of the basis, each unique screened quartet standing
 * for its distinct images under the 8 permutations of its indices (J is
 * overwritten, [nbf][nbf] device, symmetric).  D must be symmetric.  This
 * is a consumer of the integrals in the sense of Section 3.1: no integral is
 * stored.  Plans created with ERI_PLAN_STORE return ERI_EPLAN.
 * eri_plan_jk -- J as above and/or the exchange matrix
 * K[u][l] = sum over all (v, s) of (uv|ls) D[v][s], in one replay (either
 * output may be NULL, not both; they must not alias).  Same conditions.
 * eri_plan_set_budget -- bound each CTA of later executions to `cycles`
 * SM clock cycles (0 = no bound); a CTA over budget stops taking work and
 * the execution reports ERI_ETIMEOUT through eri_plan_status, which
 * synchronises `stream`.
 * eri_plan_info / eri_plan_job -- sizes; job j's class, quartet count,
 * output offset, and (if quartet_shells is a HOST buffer of 4*nq ints)
 * its quartets as shell indices (a, b, c, d) in output order.
 * eri_plan_job_degrees -- job j's pair contraction degrees K_a K_b and
 * K_c K_d in the order of its class (HOST pointers; for operation counts).
 */
typedef struct eri_plan eri_plan_t;
#define ERI_PLAN_STORE 1
#define ERI_PLAN_SPLIT 2
#define ERI_PLAN_NO_TUNE 4
int eri_plan_create(const eri_basis_t* basis, double threshold, int flags, void* stream, eri_plan_t** plan);
int eri_plan_execute(eri_plan_t* plan, const double* D, int32_t nbf, double* energy,
                     double* out, int64_t out_len, void* stream);
int eri_plan_coulomb(eri_plan_t* plan, const double* D, int32_t nbf, double* J, void* stream);
int eri_plan_jk(eri_plan_t* plan, const double* D, int32_t nbf, double* J, double* K, void* stream);
int eri_plan_set_budget(eri_plan_t* plan, int64_t cycles);
int eri_plan_status(eri_plan_t* plan, void* stream);
int eri_plan_info(eri_plan_t* plan, int64_t* nquartets, int32_t* njobs, int64_t* nitems, int64_t* out_len);
int eri_plan_job(eri_plan_t* plan, int32_t job, eri_class_t* cls, int64_t* nq, int64_t* out_off,
                 int32_t* quartet_shells);
int eri_plan_job_degrees(eri_plan_t* plan, int32_t job, int32_t* kbra, int32_t* kket);
int eri_plan_destroy(eri_plan_t* plan);

/*
 * Several GPUs on one plan (one process per GPU).  Quartets are independent
 * units, so ranks share a plan by partitioning its work items and need one
 * collective only for a digested result: each rank creates the same plan
 * (same basis, threshold and flags, hence the same work items), keeps its
 * own slice, executes it, and the per-rank energies (or J, K matrices) are
 * summed over ranks by the caller (one all-reduce).  J and K of a slice are
 * already symmetrised; the sum of the slices' J (K) is the plan's J (K).
 *
 * eri_partition -- host helper (no GPU work): longest processing time
 * first over `n` units of cost `cost` (HOST, finite, >= 0): units in
 * descending cost, ties in index order, each to the least-loaded rank (the
 * lowest on ties).  owner (HOST, [n]) receives each unit's rank; load
 * (HOST, [nranks], may be NULL) each rank's total cost.  The largest load
 * exceeds the smallest by at most the largest cost.  ERI_EINVAL for
 * nranks < 1, n < 0, NULL arrays with n > 0, or a negative or non-finite
 * cost.
 * eri_plan_set_slice -- keep the work items that eri_partition gives to
 * `rank` of `nranks` (each item's cost is its job's FP64-work estimate per
 * quartet times its quartet count); later eri_plan_execute, eri_plan_jk and
 * eri_plan_coulomb calls process that slice only.  (0, 1) restores the whole
 * plan.  Synchronises `stream`; the graph is captured again on the next
 * execution.  In ERI_PLAN_STORE mode only the slice's integrals are written.
 * eri_plan_slice_info -- the current slice's work items, quartets and total
 * cost estimate (HOST pointers, each may be NULL).
 */
int eri_partition(const double* cost, int64_t n, int32_t nranks, int32_t* owner, double* load);
int eri_plan_set_slice(eri_plan_t* plan, int32_t rank, int32_t nranks, void* stream);
int eri_plan_slice_info(eri_plan_t* plan, int64_t* nitems, int64_t* nquartets, double* cost);

/*
 * eri_last_form -- the form the calling thread's last successful eri_batch
 * launch ran (measurement support: operation counts depend on it).
 * *swapped = 1 when the kernel took the caller's ket as the side it
 * transforms last; *hrr = 1 when the transforms ran on the (e0| functions
 * with l_a <= |e| <= l_a + l_b (and likewise |f0) on the other side),
 * followed by the horizontal recursions (a, b + 1_i) = (a + 1_i, b) +
 * (A_i - B_i)(a, b) on the contracted integrals.  The form is chosen by an
 * operation-count model, or, from the first batch of at least 16384
 * quartets of a (class, K_bra, K_ket, precision) signature on, by timing the
 * cheapest plain and recursion forms on that batch.  Both arguments are HOST
 * pointers.  Returns ERI_EINVAL before the thread's first eri_batch launch.
 * The paper transforms the ket first and has no recursion form (Section 3.2.2).
 */
int eri_last_form(int32_t* swapped, int32_t* hrr);

/*
 * eri_last_tile -- the tile shape of the calling thread's last successful
 * eri_batch launch (measurement support): *tq quartets per tile, *ic bra
 * primitives per chunk of the auxiliary integrals, *threads per CTA (256, or
 * 512 for a tile that fills an SM's shared memory alone), *smem_bytes of
 * dynamic shared memory per CTA.  HOST pointers, each may be NULL.  Returns
 * ERI_EINVAL before the thread's first eri_batch launch.  No counterpart in
 * the paper, whose kernels run on CPU cores (Section 3).
 */
int eri_last_tile(int32_t* tq, int32_t* ic, int32_t* threads, int32_t* smem_bytes);

/*
 * eri_set_forms -- restrict the forms later eri_batch calls (all threads)
 * may choose from: bit 0 plain, bit 1 plain with the sides swapped, bit 2
 * recursion form, bit 3 recursion form swapped; 0 restores all four.  A
 * class for which no allowed form is feasible uses the feasible ones.
 * Returns the previous mask, or ERI_EINVAL for a mask outside 0..15.  For
 * tests and measurements of one form; the results agree to round-off.
 */
#define ERI_FORM_PLAIN 0x3
#define ERI_FORM_HRR 0xC
int eri_set_forms(int32_t mask);

/*
 * eri_last_status -- synchronises `stream` and returns ERI_OK or the first
 * error a kernel recorded since the previous call (then clears it).
 */
int eri_last_status(void* stream);

/*
 * Kernel timing hook (measurement support, not part of the method).
 * eri_profile_enable(1) makes every later launch of the dominant kernels
 * record CUDA events on its own stream; eri_profile_read() waits for them
 * and returns, per kernel id (0 = forward tile kernel, 1 = adjoint kernel,
 * 2 = pair kernel, 3 = prepass), the number of launches and their summed
 * duration in milliseconds since the last reset, then resets.  Arrays are
 * HOST memory of length n (n <= 8).  eri_launch_count() returns the number
 * of kernels the library has launched since load (all kernels).
 */
int eri_profile_enable(int on);
int eri_profile_read(int n, int64_t* launches, double* ms);
int64_t eri_launch_count(void);

/*
 * eri_peak_probe -- measurement support: the arithmetic throughput of the
 * current GPU, the denominator of the kernels' roofline fractions (the
 * paper quotes fractions of FP64 peak, Section 4).  kind 0: FP64 FMA
 * (DFMA), 1: FP64 tensor-core MMA (mma.sync m8n8k4 f64), 2: FP32 FMA.  A
 * launch of 2 to 8 CTAs per SM runs independent chains (4 to 16 per thread)
 * for about 100 ms; *gflops (HOST, GFLOP/s, FMA = 2 flops) is the best, over
 * those shapes, of three timed launches each on `stream` (CUDA events).
 * kind 3: DFMA with a single dependent chain per thread and one CTA of 256
 * threads per SM (whether FP64 latency needs more chains or warps).
 * sm_mhz (HOST, may be NULL): the SM clock during the best shape's last
 * launch, from the cycle counter and the global timer.
 * Synchronises `stream`.  ERI_EINVAL for another kind or a NULL gflops.
 */
int eri_peak_probe(int kind, double* gflops, double* sm_mhz, void* stream);

/* Human-readable text for an error code (static storage). */
const char* eri_error_string(int code);

/* Release every cached workspace of the current device. */
int eri_finalize(void);

#ifdef __cplusplus
}
#endif
#endif /* ERI_H */
