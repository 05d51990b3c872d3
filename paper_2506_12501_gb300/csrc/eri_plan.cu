// eri_plan.cu -- the batched form: every unique, Schwarz-screened shell
// quartet of a basis, all classes, in one persistent kernel fed by a device
// work queue and replayed as a CUDA graph.
//
// Plan creation (host, once):
//  1. unique shell pairs i >= j, ordered so that l_first >= l_second;
//  2. pair types = (l_a, l_b, K_a, K_b): pairs of one type share a class and
//     a contraction signature, so no primitive slot is padding;
//  3. Schwarz factors Q_P = sqrt(max_ab |(ab|ab)|) from the diagonal
//     integrals, computed by eri_batch (batch-level screening, Section 3.1);
//  4. each type's pairs sorted by Q descending: for a bra pair P the kets that
//     survive Q_P Q_Q >= threshold form a prefix of the other type's list (and,
//     within one type, the unique quartets are Q <= P), found by bisection;
//  5. one job per (type, type) with the cheaper side as the bra, its own pair
//     tables, class tables and tile shape (picked by a small autotuner that
//     times the candidate shapes on a sample of the job);
//  6. work items = (job, bra pair, range of ket positions), at most kChunk
//     quartets each, in one device array.
// Execution: a reset kernel and the persistent kernel, captured once into a
// CUDA graph.  Each CTA pops items with one atomicAdd on a counter (no other
// inter-CTA communication, so nothing waits); it runs the tile body of
// eri_tile.cuh on each tile of the item and either digests
//   energy = sum_quartets sum_abcd D_ab D_cd (ab|cd)
// or the Coulomb and exchange matrices J_uv = sum_ls (uv|ls) D_ls and
// K_ul = sum_vs (uv|ls) D_vs (every unique quartet standing for its
// permutation images; a last kernel symmetrises them), or stores the
// integrals (plans created with ERI_PLAN_STORE).  A cycle
// budget (eri_plan_set_budget) bounds the run: a CTA that exceeds it stops
// popping items and records ERI_ETIMEOUT in the plan's status word.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <queue>
#include <tuple>
#include <vector>

#include "eri_tile.cuh"

namespace eri {

constexpr int64_t kChunk = 512;  // quartets per work item (at most)
// Plan tile tuning: the heaviest jobs covering this share of the modelled
// work are timed, each on a sample of up to kTuneItemsPerSM items per SM cut
// to kTuneItemQ quartets; tuned shapes are kept per job signature.
constexpr double kTuneCover = 0.97;
constexpr int kTuneItemsPerSM = 4;
constexpr int64_t kTuneItemQ = 64;
// static shared memory of the plan kernel (job arguments and a few words),
// taken off the dynamic budget that lets two CTAs share an SM
constexpr size_t kPlanStaticSmem = 1024 + 256;
static_assert(sizeof(FwdArgs) + 64 <= kPlanStaticSmem, "plan kernel static shared memory budget");

struct WorkItem {
    int32_t job, bra;
    int64_t k0, k1, q0;  // ket positions [k0, k1); list index of (bra, k0) in the job
};

struct PlanParams {
    const double* D;
    int nbf;
    double* energy;
    double* J;            // Coulomb mode: [nbf][nbf], zeroed, accumulated, then symmetrised
    double* K;            // exchange mode: likewise
    double* out;          // store mode: base of the plan's output
    int64_t budget;       // clock64 cycles per CTA, 0 = unlimited
    int* counter;
    int* status;
};

// Tuned tile shapes per (device, class, K_bra, K_ket, split) of plan jobs.
static std::map<std::tuple<int, int, int, int, int, int, int, int>, TilePlan> g_plan_tuned;
static std::mutex g_plan_tuned_mu;

struct JobHost {
    eri_class_t cls;
    int typeA, typeB;     // bra type, ket type
    int64_t nq;           // quartets of the job
    int64_t out_off;      // store mode: offset of the job's output
    std::vector<int64_t> nket;   // per bra position: surviving kets (prefix length)
    std::vector<int64_t> qoff;   // per bra position: list index of its first quartet
    FwdArgs args;
    size_t smem;
    int split;
};

}  // namespace eri

struct eri_plan {
    int dev = 0;
    int flags = 0;
    double threshold = 0;
    int64_t nquartets = 0, out_len = 0;
    int nbf = 0;
    std::vector<eri::JobHost> jobs;
    std::vector<void*> owned;       // device buffers to free
    eri::FwdArgs* d_jobs = nullptr;
    eri::WorkItem* d_items = nullptr;
    int64_t nitems = 0;
    eri::PlanParams* d_params = nullptr;
    int* d_counter = nullptr;        // [0] queue counter, [1] status
    size_t smem = 0;
    int grid = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    eri::PlanParams params{};
    // every work item of the plan (host copy, heaviest first) with its
    // estimated cost, and the slice the device list currently holds
    std::vector<eri::WorkItem> items;
    std::vector<double> item_cost;
    int32_t slice_rank = 0, slice_n = 1;
    int64_t slice_q = 0;
    double slice_cost = 0.0;
    // host copies for eri_plan_job / tests
    std::vector<std::vector<int32_t>> type_pairs;  // per type: sorted pairs [n][2]
    std::vector<std::vector<double>> type_q;       // per type: Schwarz factors (sorted)
    std::vector<int32_t> bf_off;
};

namespace eri {

__global__ void plan_reset_kernel(const PlanParams* p)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        p->counter[0] = 0;
        p->status[0] = 0;
        if (p->energy) *p->energy = 0.0;
    }
    const size_t n = (size_t)p->nbf * p->nbf;
    for (double* M : {p->J, p->K})
        if (M)
            for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
                M[i] = 0.0;
}

// J = J' + J'^T and K = K' + K'^T in place: each unordered (u, v) by one thread.
__global__ void plan_finish_kernel(const PlanParams* p)
{
    const size_t nbf = (size_t)p->nbf, n = nbf * nbf;
    for (double* M : {p->J, p->K}) {
        if (!M) continue;
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            const size_t u = i / nbf, v = i % nbf;
            if (u < v) {
                const double t = M[u * nbf + v] + M[v * nbf + u];
                M[u * nbf + v] = t;
                M[v * nbf + u] = t;
            } else if (u == v) {
                M[i] *= 2.0;
            }
        }
    }
}

template <bool SPLIT>
__global__ void __launch_bounds__(kNT, 2)
    plan_kernel(const FwdArgs* __restrict__ jobs, const WorkItem* __restrict__ items, int64_t nitems,
                const PlanParams* __restrict__ pp)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ double s_red;
    __shared__ int64_t s_item;
    __shared__ int s_stop;
    // the current job's arguments, one copy per CTA (a per-thread copy would
    // live in local memory under the two-CTA register bound); thread 0
    // writes it between barriers, every thread reads it
    __shared__ FwdArgs a;
    const int tid = threadIdx.x;
    const PlanParams P = *pp;
    if (tid == 0) {
        s_red = 0.0;
        s_stop = 0;
    }
    const long long t_start = clock64();
    int cur = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            if (P.budget > 0 && clock64() - t_start > P.budget) {
                atomicCAS(P.status, 0, DEV_ETIMEOUT);
                s_stop = 1;
            }
            s_item = s_stop ? nitems : (int64_t)atomicAdd(P.counter, 1);
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= nitems) break;
        const WorkItem it = items[item];
        if (it.job != cur) {
            if (tid == 0) {
                a = jobs[it.job];
                a.energy = P.energy;
                a.Jmat = P.J;
                a.Kmat = P.K;
                a.D = P.D;
                a.nbf = P.nbf;
                if (P.out) a.out = P.out + (int64_t)(size_t)a.out;  // stored as an offset
            }
            __syncthreads();
            stage_class_tables<kNT>(a, sm);
            cur = it.job;
        }
        const int TQ = a.TQ;
        for (int64_t k = it.k0; k < it.k1; k += TQ) {
            __syncthreads();  // the previous tile no longer reads the range fields
            if (tid == 0) {
                a.rbra = it.bra;
                a.rk0 = k;
                a.rq0 = it.q0 + (k - it.k0);
            }
            // tile_body starts with a barrier, after which every thread sees them
            tile_body<SPLIT>(a, it.q0 + (k - it.k0), (int)min((int64_t)TQ, it.k1 - k), sm, &s_red);
        }
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

template <typename T>
static T* dev_upload(const std::vector<T>& v, std::vector<void*>& owned, cudaStream_t st, int* err)
{
    if (v.empty()) return nullptr;
    T* d = nullptr;
    if (cudaMalloc(&d, sizeof(T) * v.size()) != cudaSuccess) {
        *err = ERI_ENOMEM;
        return nullptr;
    }
    owned.push_back(d);
    if (cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        *err = ERI_ECUDA;
        return nullptr;
    }
    return d;
}

// Pair tables of one pair type in one role (bra or ket), plan-owned.
struct TypeTables {
    PairTables t[2];  // [0] bra form, [1] ket form
    bool built[2] = {false, false};
    int K1 = 0, K2 = 0;
};

int build_pair_tables_on(const eri_basis_t* basis, const int32_t* d_pairs, int64_t npairs, int l1, int l2, int KS,
                         int T, const uint8_t* fac, int ket, int split, PairTables* out, cudaStream_t st);

// The plan kernels' dynamic shared-memory limit (a per-device function
// attribute) only ever grows.  Every plan's graph launches the kernel with
// that plan's own size, and the creation of a later plan (its tile trials,
// its final size) must not lower the limit below a size an earlier plan's
// replay still uses.
static bool raise_smem_limit(bool split, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, size_t> cur;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(mu);
    size_t& c = cur[std::make_pair(dev, split ? 1 : 0)];
    if (bytes <= c) return true;
    auto kern = split ? plan_kernel<true> : plan_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return false;
    c = bytes;
    return true;
}

// Autotuner: time candidate tile shapes of one job on a sample of its own
// work items (the persistent kernel, digestion into a scratch energy with a
// zero density) and return the fastest.  Candidates: every TQ (powers of two
// up to 128) and bra-primitive chunk IC in {KB, KB/2, 1} that keeps the
// outputs in registers and fits shared memory.
static bool autotune_job(const FwdArgs& base, const std::vector<WorkItem>& sample, int64_t sample_q, bool split,
                         const double* zeroD, int nbf, double* d_scratch, int* d_ctr, PlanParams* d_prm,
                         cudaStream_t st, TilePlan* best)
{
    std::vector<TilePlan> cands;
    const size_t half_sm = (size_t)smem_per_sm() / 2 - 1024 - kPlanStaticSmem;
    for (int TQ = 1; TQ <= 128; TQ *= 2) {
        if (TQ * base.ct.nab * base.ct.ncd > kNT * kNACC) break;
        for (int IC : {base.KB, (base.KB + 1) / 2, 1}) {
            for (int es = 1; es >= 0; --es) {
                TilePlan tp;
                // shapes within half an SM's shared memory (two CTAs per SM)
                if (tile_layout(base.ct, base.KB, base.KK, TQ, IC, es, &tp, split) && tp.acc_regs &&
                    tp.bytes <= half_sm) {
                    bool dup = false;
                    for (auto& c : cands) dup |= (c.TQ == TQ && c.IC == IC && c.e_smem == es);
                    if (!dup) cands.push_back(tp);
                    break;  // prefer staged E when it fits
                }
            }
        }
    }
    if (cands.empty()) return false;
    if (cands.size() == 1) {
        *best = cands[0];
        return true;
    }
    std::vector<WorkItem> items = sample;
    for (auto& it : items) it.job = 0;
    WorkItem* d_items = nullptr;
    FwdArgs* d_job = nullptr;
    if (cudaMalloc(&d_items, sizeof(WorkItem) * items.size()) != cudaSuccess) return false;
    if (cudaMalloc(&d_job, sizeof(FwdArgs)) != cudaSuccess) {
        cudaFree(d_items);
        return false;
    }
    cudaMemcpyAsync(d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, st);
    PlanParams prm{};
    prm.D = zeroD;
    prm.nbf = nbf;
    prm.energy = d_scratch;
    prm.counter = d_ctr;
    prm.status = d_ctr + 1;
    cudaMemcpyAsync(d_prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, st);
    auto kern = split ? plan_kernel<true> : plan_kernel<false>;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_t = 1e300;
    bool ok = false;
    for (const TilePlan& tp : cands) {
        FwdArgs a = base;
        set_tile(a, tp);
        cudaMemcpyAsync(d_job, &a, sizeof(a), cudaMemcpyHostToDevice, st);
        if (!raise_smem_limit(split, tp.bytes)) continue;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, tp.bytes);
        const int grid = std::max(1, per_sm) * sm_count();
        float ms = 0.f;
        for (int rep = 0; rep < (&tp == &cands[0] ? 2 : 1); ++rep) {  // the first run warms the caches
            plan_reset_kernel<<<1, 32, 0, st>>>(d_prm);
            cudaEventRecord(e0, st);
            kern<<<grid, kNT, tp.bytes, st>>>(d_job, d_items, (int64_t)items.size(), d_prm);
            cudaEventRecord(e1, st);
        }
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (ms < best_t) {
            best_t = ms;
            *best = tp;
            ok = true;
        }
    }
    (void)sample_q;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_items);
    cudaFree(d_job);
    return ok;
}

}  // namespace eri

using namespace eri;

static int plan_fail(eri_plan* p, int code)
{
    if (p) {
        for (void* v : p->owned) cudaFree(v);
        delete p;
    }
    return code;
}

extern "C" int eri_plan_create(const eri_basis_t* basis, double threshold, int flags, void* stream,
                               eri_plan_t** plan_out)
{
    if (!plan_out || !basis || !basis->shell_l || !basis->shell_K || !basis->shell_atom || !basis->shell_off ||
        !basis->centres || !basis->exps || !basis->coefs || basis->nshell <= 0)
        return ERI_EINVAL;
    if (flags & ~(ERI_PLAN_STORE | ERI_PLAN_SPLIT | ERI_PLAN_NO_TUNE)) return ERI_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t half_sm = (size_t)smem_per_sm() / 2 - 1024 - kPlanStaticSmem;
    eri_plan* p = new eri_plan();
    p->flags = flags;
    p->threshold = threshold;
    cudaGetDevice(&p->dev);
    const int ns = basis->nshell;
    std::vector<int32_t> sl(ns), sk(ns);
    if (cudaMemcpyAsync(sl.data(), basis->shell_l, 4 * ns, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(sk.data(), basis->shell_K, 4 * ns, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return plan_fail(p, ERI_ECUDA);
    for (int s = 0; s < ns; ++s)
        if (sl[s] < 0 || sl[s] > kLmax || sk[s] < 1 || sk[s] > kKmax) return plan_fail(p, ERI_EINVAL);
    p->bf_off.resize(ns);
    int nbf = 0;
    for (int s = 0; s < ns; ++s) {
        p->bf_off[s] = nbf;
        nbf += ncart(sl[s]);
    }
    p->nbf = nbf;
    int err = ERI_OK;
    const int32_t* d_bf = dev_upload(p->bf_off, p->owned, st, &err);
    if (err) return plan_fail(p, err);

    // 1-2. unique pairs by type (la, lb, Ka, Kb), la >= lb (and Ka >= Kb if la == lb)
    std::map<std::tuple<int, int, int, int>, int> type_id;
    std::vector<std::tuple<int, int, int, int>> types;
    std::vector<std::vector<int32_t>> tpairs;
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j <= i; ++j) {
            int a = i, b = j;
            if (sl[a] < sl[b] || (sl[a] == sl[b] && sk[a] < sk[b])) std::swap(a, b);
            auto key = std::make_tuple(sl[a], sl[b], sk[a], sk[b]);
            auto it = type_id.find(key);
            int t;
            if (it == type_id.end()) {
                t = (int)types.size();
                type_id[key] = t;
                types.push_back(key);
                tpairs.emplace_back();
            } else {
                t = it->second;
            }
            tpairs[t].push_back(a);
            tpairs[t].push_back(b);
        }
    const int ntype = (int)types.size();

    // 3. Schwarz factors from the diagonal integrals (ab|ab)
    std::vector<std::vector<double>> tq(ntype);
    for (int t = 0; t < ntype; ++t) {
        const int la = std::get<0>(types[t]), lb = std::get<1>(types[t]);
        const int64_t n = (int64_t)tpairs[t].size() / 2;
        const int nab = ncart(la) * ncart(lb);
        std::vector<int64_t> diag(2 * n);
        for (int64_t i = 0; i < n; ++i) diag[2 * i] = diag[2 * i + 1] = i;
        int32_t* dp = nullptr;
        int64_t* dq = nullptr;
        double* dout = nullptr;
        if (cudaMalloc(&dp, 8 * n) != cudaSuccess || cudaMalloc(&dq, 16 * n) != cudaSuccess ||
            cudaMalloc(&dout, 8 * n * nab * nab) != cudaSuccess) {
            cudaFree(dp);
            cudaFree(dq);
            return plan_fail(p, ERI_ENOMEM);
        }
        cudaMemcpyAsync(dp, tpairs[t].data(), 8 * n, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dq, diag.data(), 16 * n, cudaMemcpyHostToDevice, st);
        int rc = eri_batch(eri_class_t{la, lb, la, lb}, basis, dp, n, dp, n, dq, n, dout, n * nab * nab,
                           ERI_PREC_FP64, stream);
        std::vector<double> h((size_t)n * nab * nab);
        if (rc == ERI_OK)
            rc = cudaMemcpyAsync(h.data(), dout, 8 * h.size(), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                         cudaStreamSynchronize(st) == cudaSuccess
                     ? ERI_OK
                     : ERI_ECUDA;
        cudaFree(dp);
        cudaFree(dq);
        cudaFree(dout);
        if (rc != ERI_OK) return plan_fail(p, rc);
        tq[t].resize(n);
        for (int64_t i = 0; i < n; ++i) {
            double m = 0.0;
            for (int ab = 0; ab < nab; ++ab) m = std::max(m, std::fabs(h[i + n * ((int64_t)ab * nab + ab)]));
            tq[t][i] = std::sqrt(m);
        }
        // 4. sort the type's pairs by Q descending
        std::vector<int64_t> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return tq[t][x] > tq[t][y]; });
        std::vector<int32_t> sp(2 * n);
        std::vector<double> sq(n);
        for (int64_t i = 0; i < n; ++i) {
            sp[2 * i] = tpairs[t][2 * ord[i]];
            sp[2 * i + 1] = tpairs[t][2 * ord[i] + 1];
            sq[i] = tq[t][ord[i]];
        }
        tpairs[t].swap(sp);
        tq[t].swap(sq);
    }
    p->type_pairs = tpairs;
    p->type_q = tq;
    std::vector<const int32_t*> d_tpairs(ntype);
    for (int t = 0; t < ntype; ++t) {
        d_tpairs[t] = dev_upload(tpairs[t], p->owned, st, &err);
        if (err) return plan_fail(p, err);
    }

    // 5. jobs
    std::vector<TypeTables> tt(ntype);
    const bool split = (flags & ERI_PLAN_SPLIT) != 0;
    std::vector<WorkItem> items;
    int64_t out_off = 0;
    for (int A = 0; A < ntype; ++A)
        for (int B = A; B < ntype; ++B) {
            const int la = std::get<0>(types[A]), lb = std::get<1>(types[A]);
            const int lc = std::get<0>(types[B]), ld = std::get<1>(types[B]);
            const int KA = std::get<2>(types[A]) * std::get<3>(types[A]);
            const int KBt = std::get<2>(types[B]) * std::get<3>(types[B]);
            const ClassTables* cAB = get_class_tables(la, lb, lc, ld, st, &err);
            const ClassTables* cBA = get_class_tables(lc, ld, la, lb, st, &err);
            if (!cAB || !cBA) return plan_fail(p, err);
            // the cheaper transform order decides which type is the bra
            const double costAB = (double)KA * KBt * cAB->nhb * cAB->Tcd + (double)KA * cAB->ncd * cAB->Tab;
            const double costBA = (double)KBt * KA * cBA->nhb * cBA->Tcd + (double)KBt * cBA->ncd * cBA->Tab;
            const int bt = (A != B && costBA < costAB) ? B : A, kt = bt == A ? B : A;
            const ClassTables* ct = bt == A ? cAB : cBA;
            const std::vector<double>& qb = tq[bt];
            const std::vector<double>& qk = tq[kt];
            JobHost J;
            J.cls = eri_class_t{ct->la, ct->lb, ct->lc, ct->ld};
            J.typeA = bt;
            J.typeB = kt;
            const int64_t nbp = (int64_t)qb.size();
            J.nket.assign(nbp, 0);
            J.qoff.assign(nbp, 0);
            int64_t nq = 0;
            for (int64_t i = 0; i < nbp; ++i) {
                int64_t n;
                if (threshold > 0) {
                    if (qb[i] <= 0) {
                        n = 0;
                    } else {
                        const double need = threshold / qb[i];
                        n = std::upper_bound(qk.begin(), qk.end(), need, [](double v, double x) { return v > x; }) -
                            qk.begin();
                    }
                } else {
                    n = (int64_t)qk.size();
                }
                if (A == B) n = std::min(n, i + 1);  // unique quartets: ket position <= bra position
                J.nket[i] = n;
                J.qoff[i] = nq;
                nq += n;
            }
            if (nq == 0) continue;
            J.nq = nq;
            J.out_off = out_off;
            if (flags & ERI_PLAN_STORE) out_off += nq * ct->nab * ct->ncd;
            // pair tables (bra form of bt, ket form of kt)
            for (int role = 0; role < 2; ++role) {
                const int ty = role == 0 ? bt : kt;
                if (!tt[ty].built[role]) {
                    const int l1 = std::get<0>(types[ty]), l2 = std::get<1>(types[ty]);
                    const ClassTables* c1 = get_class_tables(l1, l2, l1, l2, st, &err);
                    if (!c1) return plan_fail(p, err);
                    const int KS = std::get<2>(types[ty]) * std::get<3>(types[ty]);
                    const int64_t np = (int64_t)tq[ty].size();
                    PairTables& P = tt[ty].t[role];
                    double* ps = nullptr;
                    double* E = nullptr;
                    int32_t* kp = nullptr;
                    if (cudaMalloc(&ps, 8 * np * KS * PS_N) != cudaSuccess ||
                        cudaMalloc(&E, 8 * np * KS * (size_t)c1->Tab) != cudaSuccess ||
                        cudaMalloc(&kp, 4 * np) != cudaSuccess)
                        return plan_fail(p, ERI_ENOMEM);
                    p->owned.push_back(ps);
                    p->owned.push_back(E);
                    p->owned.push_back(kp);
                    P.ps = ps;
                    P.E = E;
                    P.kp = kp;
                    int rc = build_pair_tables_on(basis, d_tpairs[ty], np, l1, l2, KS, c1->Tab, c1->bra_fac, role,
                                                  split ? 1 : 0, &P, st);
                    if (rc != ERI_OK) return plan_fail(p, rc);
                    tt[ty].built[role] = true;
                }
            }
            const int KB = bt == A ? KA : KBt;  // primitive pairs of the bra type
            const int KK = bt == A ? KBt : KA;  // and of the ket type
            TilePlan tp;
            // the persistent kernel runs every job with the largest job's
            // shared memory: keep each job within half an SM so two CTAs fit
            if (!(plan_tiles(*ct, KB, KK, nq, &tp, half_sm, split) && tp.acc_regs) &&
                !(plan_tiles(*ct, KB, KK, nq, &tp, 0, split) && tp.acc_regs))
                return plan_fail(p, ERI_EINVAL);
            FwdArgs& a = J.args;
            a = FwdArgs{};
            a.ct = *ct;
            a.boys = get_boys_table(ct->L, st, &err);
            a.rsteps = get_rsteps(st, &err);
            if (!a.boys || !a.rsteps) return plan_fail(p, err);
            a.bra_ps = tt[bt].t[0].ps;
            a.bra_E = tt[bt].t[0].E;
            a.bra_kp = tt[bt].t[0].kp;
            a.ket_ps = tt[kt].t[1].ps;
            a.ket_E = tt[kt].t[1].E;
            a.ket_kp = tt[kt].t[1].kp;
            a.quartets = nullptr;
            a.nq = nq;
            a.nbra = nbp;
            a.nket = (int64_t)qk.size();
            a.swap = 0;
            a.nab_o = ct->nab_f;
            a.ncd_o = ct->ncd_f;
            a.out = reinterpret_cast<double*>((size_t)J.out_off);  // offset, rebased by the kernel
            a.KB = KB;
            a.KK = KK;
            set_tile(a, tp);
            a.mode = 1;
            a.bf_off = d_bf;
            a.bra_sh = d_tpairs[bt];
            a.ket_sh = d_tpairs[kt];
            J.smem = tp.bytes;
            p->smem = std::max(p->smem, tp.bytes);
            const int jid = (int)p->jobs.size();
            for (int64_t i = 0; i < nbp; ++i)
                for (int64_t k0 = 0; k0 < J.nket[i]; k0 += kChunk)
                    items.push_back(WorkItem{jid, (int32_t)i, k0, std::min(J.nket[i], k0 + kChunk), J.qoff[i] + k0});
            p->nquartets += nq;
            p->jobs.push_back(std::move(J));
        }
    p->out_len = out_off;
    // autotune the tile shape of every job with enough work to time
    if (!(flags & ERI_PLAN_NO_TUNE) && !p->jobs.empty()) {
        double* zeroD = nullptr;
        double* scratch = nullptr;
        int* ctr = nullptr;
        PlanParams* prm = nullptr;
        bool ok = cudaMalloc(&zeroD, 8 * (size_t)nbf * nbf) == cudaSuccess && cudaMalloc(&scratch, 64) == cudaSuccess &&
                  cudaMalloc(&ctr, 16) == cudaSuccess && cudaMalloc(&prm, sizeof(PlanParams)) == cudaSuccess;
        if (ok) cudaMemsetAsync(zeroD, 0, 8 * (size_t)nbf * nbf, st);
        // tune the heaviest jobs that together carry kTuneCover of the plan's
        // modelled FP64 work (the rest keep the planner's shape); a job whose
        // signature an earlier plan of this process tuned reuses that shape
        std::vector<double> jw(p->jobs.size());
        double total = 0.0;
        for (size_t j = 0; j < p->jobs.size(); ++j) {
            const FwdArgs& a = p->jobs[j].args;
            jw[j] = ((double)a.KB * a.KK * (a.ct.nhb * a.ct.Tcd + a.ct.nhl) + (double)a.KB * a.ct.ncd * a.ct.Tab) *
                    (double)p->jobs[j].nq;
            total += jw[j];
        }
        std::vector<size_t> byw(p->jobs.size());
        std::iota(byw.begin(), byw.end(), (size_t)0);
        std::stable_sort(byw.begin(), byw.end(), [&](size_t x, size_t y) { return jw[x] > jw[y]; });
        std::vector<std::vector<int64_t>> job_items(p->jobs.size());
        for (size_t i = 0; i < items.size(); ++i) job_items[(size_t)items[i].job].push_back((int64_t)i);
        double covered = 0.0;
        for (size_t j : byw) {
            if (!ok || covered >= kTuneCover * total) break;
            covered += jw[j];
            JobHost& J = p->jobs[j];
            const auto key = std::make_tuple(p->dev, J.args.ct.la, J.args.ct.lb, J.args.ct.lc, J.args.ct.ld,
                                             J.args.KB, J.args.KK, (int)split);
            {
                std::lock_guard<std::mutex> lk(g_plan_tuned_mu);
                auto it = g_plan_tuned.find(key);
                if (it != g_plan_tuned.end()) {
                    set_tile(J.args, it->second);
                    J.smem = it->second.bytes;
                    continue;
                }
            }
            // the sample: up to kTuneItemsPerSM items per SM spread over the
            // job, each cut to kTuneItemQ quartets, so that every CTA of the
            // persistent kernel takes part in the timed runs
            const std::vector<int64_t>& ji = job_items[j];
            const size_t want = std::min(ji.size(), (size_t)kTuneItemsPerSM * (size_t)sm_count());
            std::vector<WorkItem> sample;
            int64_t sq = 0;
            for (size_t s = 0; s < want; ++s) {
                WorkItem it = items[(size_t)ji[s * ji.size() / want]];
                it.k1 = std::min(it.k1, it.k0 + kTuneItemQ);
                sq += it.k1 - it.k0;
                sample.push_back(it);
            }
            TilePlan best;
            if (autotune_job(J.args, sample, sq, split, zeroD, nbf, scratch, ctr, prm, st, &best)) {
                set_tile(J.args, best);
                J.smem = best.bytes;
                std::lock_guard<std::mutex> lk(g_plan_tuned_mu);
                g_plan_tuned[key] = best;
            }
        }
        cudaStreamSynchronize(st);
        cudaFree(zeroD);
        cudaFree(scratch);
        cudaFree(ctr);
        cudaFree(prm);
        p->smem = 0;
        for (auto& J : p->jobs) p->smem = std::max(p->smem, J.smem);
    }
    // heavy items first: a job's cost per quartet ~ its FP64 work
    std::vector<double> jcost(p->jobs.size());
    for (size_t j = 0; j < p->jobs.size(); ++j) {
        const FwdArgs& a = p->jobs[j].args;
        jcost[j] = (double)a.KB * a.KK * (a.ct.nhb * a.ct.Tcd + a.ct.nhl) + (double)a.KB * a.ct.ncd * a.ct.Tab;
    }
    std::stable_sort(items.begin(), items.end(), [&](const WorkItem& x, const WorkItem& y) {
        return jcost[x.job] * (x.k1 - x.k0) > jcost[y.job] * (y.k1 - y.k0);
    });
    std::vector<FwdArgs> jargs;
    for (auto& J : p->jobs) jargs.push_back(J.args);
    p->d_jobs = dev_upload(jargs, p->owned, st, &err);
    p->d_items = dev_upload(items, p->owned, st, &err);
    if (err) return plan_fail(p, err);
    p->nitems = (int64_t)items.size();
    p->item_cost.resize(items.size());
    for (size_t i = 0; i < items.size(); ++i)
        p->item_cost[i] = jcost[items[i].job] * (double)(items[i].k1 - items[i].k0);
    p->slice_q = p->nquartets;
    p->slice_cost = std::accumulate(p->item_cost.begin(), p->item_cost.end(), 0.0);
    p->items = std::move(items);
    if (cudaMalloc(&p->d_params, sizeof(PlanParams)) != cudaSuccess ||
        cudaMalloc(&p->d_counter, 4 * sizeof(int)) != cudaSuccess)
        return plan_fail(p, ERI_ENOMEM);
    p->owned.push_back(p->d_params);
    p->owned.push_back(p->d_counter);
    auto kern = split ? plan_kernel<true> : plan_kernel<false>;
    if (p->smem > (size_t)max_smem_optin()) return plan_fail(p, ERI_EINVAL);
    if (!raise_smem_limit(split, p->smem)) return plan_fail(p, ERI_ECUDA);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, p->smem);
    p->grid = std::max(1, per_sm) * sm_count();
    if (cudaStreamSynchronize(st) != cudaSuccess) return plan_fail(p, ERI_ECUDA);
    *plan_out = p;
    return ERI_OK;
}

// Upload the parameters and replay the plan's graph (captured on the first
// call: reset, persistent kernel, J symmetrisation; every kernel reads its
// parameters from d_params, so one graph serves every mode and pointer).
static int plan_launch(eri_plan_t* p, const PlanParams& prm_in, cudaStream_t st)
{
    PlanParams prm = prm_in;
    prm.budget = p->params.budget;
    prm.counter = p->d_counter;
    prm.status = p->d_counter + 1;
    p->params = prm;
    if (cudaMemcpyAsync(p->d_params, &p->params, sizeof(PlanParams), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ERI_ECUDA;
    const int egrid = 2 * sm_count();
    if (!raise_smem_limit(p->flags & ERI_PLAN_SPLIT, p->smem)) return ERI_ECUDA;
    if (!p->exec) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return ERI_ECUDA;
        auto kern = (p->flags & ERI_PLAN_SPLIT) ? plan_kernel<true> : plan_kernel<false>;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            plan_reset_kernel<<<egrid, 256, 0, cs>>>(p->d_params);
            kern<<<p->grid, kNT, p->smem, cs>>>(p->d_jobs, p->d_items, p->nitems, p->d_params);
            plan_finish_kernel<<<egrid, 256, 0, cs>>>(p->d_params);
        }
        cudaGraph_t g = nullptr;
        ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && ok;
        cudaStreamDestroy(cs);
        if (!ok || cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return ERI_ECUDA;
        }
        p->graph = g;
    }
    count_launch();
    count_launch();
    count_launch();
    ProfScope ps(PROF_FWD, st);
    return cudaGraphLaunch(p->exec, st) == cudaSuccess ? ERI_OK : ERI_ECUDA;
}

extern "C" int eri_plan_execute(eri_plan_t* p, const double* D, int32_t nbf, double* energy, double* out,
                                int64_t out_len, void* stream)
{
    if (!p) return ERI_EINVAL;
    const bool store = (p->flags & ERI_PLAN_STORE) != 0;
    if (store ? (!out || out_len < p->out_len) : (!energy || !D || nbf != p->nbf)) return ERI_EPLAN;
    if (!store && out) return ERI_EPLAN;
    PlanParams prm{};
    prm.D = store ? nullptr : D;
    prm.nbf = p->nbf;
    prm.energy = store ? nullptr : energy;
    prm.out = store ? out : nullptr;
    return plan_launch(p, prm, (cudaStream_t)stream);
}

extern "C" int eri_plan_jk(eri_plan_t* p, const double* D, int32_t nbf, double* J, double* K, void* stream)
{
    if (!p) return ERI_EINVAL;
    if ((p->flags & ERI_PLAN_STORE) || !D || (!J && !K) || nbf != p->nbf || (J && J == K)) return ERI_EPLAN;
    PlanParams prm{};
    prm.D = D;
    prm.nbf = p->nbf;
    prm.J = J;
    prm.K = K;
    return plan_launch(p, prm, (cudaStream_t)stream);
}

extern "C" int eri_plan_coulomb(eri_plan_t* p, const double* D, int32_t nbf, double* J, void* stream)
{
    if (!J) return p ? ERI_EPLAN : ERI_EINVAL;
    return eri_plan_jk(p, D, nbf, J, nullptr, stream);
}

extern "C" int eri_plan_set_budget(eri_plan_t* p, int64_t cycles)
{
    if (!p || cycles < 0) return ERI_EINVAL;
    p->params.budget = cycles;
    return ERI_OK;
}

extern "C" int eri_plan_status(eri_plan_t* p, void* stream)
{
    if (!p) return ERI_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return ERI_ECUDA;
    int h = 0;
    if (cudaMemcpy(&h, p->d_counter + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ERI_ECUDA;
    return h == DEV_ETIMEOUT ? ERI_ETIMEOUT : (h ? ERI_ECUDA : ERI_OK);
}

extern "C" int eri_plan_info(eri_plan_t* p, int64_t* nquartets, int32_t* njobs, int64_t* nitems, int64_t* out_len)
{
    if (!p) return ERI_EINVAL;
    if (nquartets) *nquartets = p->nquartets;
    if (njobs) *njobs = (int32_t)p->jobs.size();
    if (nitems) *nitems = (int64_t)p->items.size();
    if (out_len) *out_len = p->out_len;
    return ERI_OK;
}

extern "C" int eri_plan_job(eri_plan_t* p, int32_t j, eri_class_t* cls, int64_t* nq, int64_t* out_off,
                            int32_t* quartet_shells)
{
    if (!p || j < 0 || j >= (int32_t)p->jobs.size()) return ERI_EINVAL;
    const JobHost& J = p->jobs[j];
    if (cls) *cls = J.cls;
    if (nq) *nq = J.nq;
    if (out_off) *out_off = J.out_off;
    if (quartet_shells) {
        const std::vector<int32_t>& bp = p->type_pairs[J.typeA];
        const std::vector<int32_t>& kp = p->type_pairs[J.typeB];
        for (size_t i = 0; i < J.nket.size(); ++i)
            for (int64_t k = 0; k < J.nket[i]; ++k) {
                int32_t* o = quartet_shells + 4 * (J.qoff[i] + k);
                o[0] = bp[2 * i];
                o[1] = bp[2 * i + 1];
                o[2] = kp[2 * k];
                o[3] = kp[2 * k + 1];
            }
    }
    return ERI_OK;
}

extern "C" int eri_plan_job_degrees(eri_plan_t* p, int32_t j, int32_t* kbra, int32_t* kket)
{
    if (!p || j < 0 || j >= (int32_t)p->jobs.size() || !kbra || !kket) return ERI_EINVAL;
    *kbra = p->jobs[j].args.KB;
    *kket = p->jobs[j].args.KK;
    return ERI_OK;
}

extern "C" int eri_partition(const double* cost, int64_t n, int32_t nranks, int32_t* owner, double* load)
{
    if (n < 0 || nranks < 1 || (n > 0 && (!cost || !owner))) return ERI_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return ERI_EINVAL;
    // longest processing time first: units by descending cost (ties keep
    // their order), each to the least-loaded rank (the lowest rank on ties)
    std::vector<int64_t> ord((size_t)n);
    std::iota(ord.begin(), ord.end(), (int64_t)0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return cost[x] > cost[y]; });
    using Slot = std::pair<double, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int32_t r = 0; r < nranks; ++r) heap.push(Slot(0.0, r));
    std::vector<double> ld((size_t)nranks, 0.0);
    for (int64_t i : ord) {
        Slot s = heap.top();
        heap.pop();
        owner[i] = s.second;
        s.first += cost[i];
        ld[(size_t)s.second] = s.first;
        heap.push(s);
    }
    if (load)
        for (int32_t r = 0; r < nranks; ++r) load[r] = ld[(size_t)r];
    return ERI_OK;
}

extern "C" int eri_plan_set_slice(eri_plan_t* p, int32_t rank, int32_t nranks, void* stream)
{
    if (!p || nranks < 1 || rank < 0 || rank >= nranks) return ERI_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)p->items.size();
    std::vector<int32_t> owner((size_t)n, 0);
    int rc = eri_partition(p->item_cost.data(), n, nranks, owner.data(), nullptr);
    if (rc != ERI_OK) return rc;
    // this rank's items, still heaviest first
    std::vector<WorkItem> mine;
    int64_t q = 0;
    double c = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (owner[(size_t)i] == rank) {
            mine.push_back(p->items[(size_t)i]);
            q += p->items[(size_t)i].k1 - p->items[(size_t)i].k0;
            c += p->item_cost[(size_t)i];
        }
    // the device list is the full list's buffer; earlier replays may still read it
    if (cudaStreamSynchronize(st) != cudaSuccess) return ERI_ECUDA;
    if (!mine.empty() &&
        cudaMemcpy(p->d_items, mine.data(), sizeof(WorkItem) * mine.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return ERI_ECUDA;
    p->nitems = (int64_t)mine.size();
    p->slice_rank = rank;
    p->slice_n = nranks;
    p->slice_q = q;
    p->slice_cost = c;
    // the graph holds the item count as a kernel argument: capture it again
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    if (p->graph) {
        cudaGraphDestroy(p->graph);
        p->graph = nullptr;
    }
    return ERI_OK;
}

extern "C" int eri_plan_slice_info(eri_plan_t* p, int64_t* nitems, int64_t* nquartets, double* cost)
{
    if (!p) return ERI_EINVAL;
    if (nitems) *nitems = p->nitems;
    if (nquartets) *nquartets = p->slice_q;
    if (cost) *cost = p->slice_cost;
    return ERI_OK;
}

extern "C" int eri_plan_destroy(eri_plan_t* p)
{
    if (!p) return ERI_OK;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (void* v : p->owned) cudaFree(v);
    delete p;
    return ERI_OK;
}
