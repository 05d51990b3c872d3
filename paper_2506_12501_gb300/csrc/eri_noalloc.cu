// eri_noalloc.cu -- eri_batch_noalloc: the forward batch without any device
// or host allocation.
//
// Some callers cannot allocate: a process whose device memory is owned by
// another allocator (a serving framework's pool, an MPI library's pinned
// pool) may not call cudaMalloc behind its back, and code that runs while a
// stream is being captured into a CUDA graph must not allocate.  For them
// the pair tables that eri_batch keeps in a cudaMalloc'ed workspace live
// here in a fixed, file-scope device array instead, next to fixed arrays for
// the constant tables (Boys function, recursion steps, class tables) and the
// validation words.  The arrays exist on every GPU that loads the library
// until the process exits.
//
// Set-up, once per device: the first call on a device, with that device
// current, computes the constant tables on the host into static host
// buffers, copies them into the static device arrays with synchronous
// cudaMemcpyToSymbol, and asks cudaGetSymbolAddress for the device address
// of every array (host code cannot use the array names as device
// addresses).  Later calls only upload the small class table of the
// requested class into its static array (stream-ordered) and launch.
#include <cmath>
#include <cstring>
#include <mutex>

#include "eri_internal.h"

namespace eri {

constexpr size_t kScratchDoubles = (size_t)ERI_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr int kMaxDev = 64;
constexpr int kMaxNc2 = 100;           // nc(3)^2
constexpr int kMaxTerms = 1920;        // most nonzero E terms of a pair of l <= 3 shells
constexpr int kMaxNh6 = 84;            // Nh(6)
constexpr int kBoysRows = kBoysGrid * 8;

static __device__ __align__(256) double g_scratch[kScratchDoubles];
static __device__ __align__(256) double g_boys[(kLtotMax + 1) * kBoysRows];
static __device__ __align__(256) RStep g_rsteps[kNhMax];
static __device__ __align__(256) uint8_t g_class[64 * 1024];
static __device__ __align__(256) int g_info[16];

struct DevPtrs {
    bool ready = false;
    double* scratch = nullptr;
    double* boys = nullptr;
    RStep* rsteps = nullptr;
    uint8_t* cls = nullptr;
    int* info = nullptr;
};
static DevPtrs g_dev_ptrs[kMaxDev];
static std::mutex g_mu;

// ---- host tables in static storage (no heap) --------------------------------
static long double h_master[kBoysGrid][kBoysMtab + 2];
static double h_boys[(kLtotMax + 1) * kBoysRows];
static RStep h_rsteps[kNhMax];

// Hermite numbering of (t,u,v), order by N = t+u+v then t, u descending.
static int hidx(int t, int u, int v)
{
    const int N = t + u + v;
    return N * (N + 1) * (N + 2) / 6 + (N - t) * (N - t + 1) / 2 + (N - t - u);
}

static void htuv(int idx, int* t, int* u, int* v)
{
    int N = 0;
    while ((N + 1) * (N + 2) * (N + 3) / 6 <= idx) ++N;
    int r = idx - N * (N + 1) * (N + 2) / 6;
    int d = 0;  // d = N - t
    while ((d + 1) * (d + 2) / 2 <= r) ++d;
    const int e = r - d * (d + 1) / 2;  // e = N - t - u
    *t = N - d;
    *u = d - e;
    *v = N - *t - *u;
}

static void build_constant_tables()
{
    // Boys: top order by its all-positive series, lower orders downward
    for (int j = 0; j < kBoysGrid; ++j) {
        const long double T = (long double)j / kBoysInvStep;
        const long double eT = expl(-T);
        long double term = 1.0L / (2 * kBoysMtab + 1), sum = term;
        for (int k = 1; k < 10000; ++k) {
            term *= 2.0L * T / (long double)(2 * kBoysMtab + 2 * k + 1);
            sum += term;
            if (term < sum * 1e-22L) break;
        }
        h_master[j][kBoysMtab] = eT * sum;
        for (int m = kBoysMtab - 1; m >= 0; --m) h_master[j][m] = (2.0L * T * h_master[j][m + 1] + eT) / (2 * m + 1);
        h_master[j][kBoysMtab + 1] = eT;
    }
    for (int L = 0; L <= kLtotMax; ++L) {
        long double fact = 1;
        for (int k = 0; k < kBoysOrder; ++k) {
            if (k > 0) fact *= k;
            for (int j = 0; j < kBoysGrid; ++j)
                h_boys[(size_t)L * kBoysRows + (size_t)j * 8 + k] = (double)(h_master[j][L + k] / fact);
        }
        for (int j = 0; j < kBoysGrid; ++j) h_boys[(size_t)L * kBoysRows + (size_t)j * 8 + 7] = (double)h_master[j][kBoysMtab + 1];
    }
    // auxiliary-recursion steps (axis with r_i = 1 preferred)
    std::memset(h_rsteps, 0, sizeof(h_rsteps));
    for (int e = 1; e < kNhMax; ++e) {
        int r[3];
        htuv(e, &r[0], &r[1], &r[2]);
        int axis = -1;
        for (int i = 0; i < 3; ++i)
            if (r[i] == 1) { axis = i; break; }
        if (axis < 0)
            for (int i = 0; i < 3; ++i)
                if (r[i] > 0 && (axis < 0 || r[i] < r[axis])) axis = i;
        int d1[3] = {r[0], r[1], r[2]}, d2[3] = {r[0], r[1], r[2]};
        d1[axis] -= 1;
        d2[axis] -= 2;
        h_rsteps[e].axis = (int8_t)axis;
        h_rsteps[e].coef = (int8_t)(r[axis] - 1);
        h_rsteps[e].coefd = (double)(r[axis] - 1);
        h_rsteps[e].src1 = (int16_t)hidx(d1[0], d1[1], d1[2]);
        h_rsteps[e].src2 = (int16_t)(r[axis] >= 2 ? hidx(d2[0], d2[1], d2[2]) : 0);
    }
}

static int setup_device(int dev, DevPtrs* out)
{
    static bool host_built = false;
    if (!host_built) {
        build_constant_tables();
        host_built = true;
    }
    DevPtrs d;
    if (cudaMemcpyToSymbol(g_boys, h_boys, sizeof(h_boys)) != cudaSuccess) return ERI_ECUDA;
    if (cudaMemcpyToSymbol(g_rsteps, h_rsteps, sizeof(h_rsteps)) != cudaSuccess) return ERI_ECUDA;
    if (cudaGetSymbolAddress((void**)&d.scratch, g_scratch) != cudaSuccess) return ERI_ECUDA;
    if (cudaGetSymbolAddress((void**)&d.boys, g_boys) != cudaSuccess) return ERI_ECUDA;
    if (cudaGetSymbolAddress((void**)&d.rsteps, g_rsteps) != cudaSuccess) return ERI_ECUDA;
    if (cudaGetSymbolAddress((void**)&d.cls, g_class) != cudaSuccess) return ERI_ECUDA;
    if (cudaGetSymbolAddress((void**)&d.info, g_info) != cudaSuccess) return ERI_ECUDA;
    (void)dev;
    d.ready = true;
    *out = d;
    return ERI_OK;
}

// ---- class tables in a static host blob, uploaded into g_class --------------
struct HostClassBlob {
    int bstart[kMaxNc2 + 1];
    int kstart[kMaxNc2 + 1];
    int16_t bp[kMaxTerms];
    int16_t kq[kMaxTerms];
    int16_t pq[kMaxNh6 * kMaxNh6];
    uint8_t bfac[3 * kMaxTerms];
    uint8_t kfac[3 * kMaxTerms];
};
static_assert(sizeof(HostClassBlob) <= sizeof(g_class), "class blob does not fit its static array");
static HostClassBlob h_blob;

static int terms_of(int l1, int l2, int* start, int16_t* herm, uint8_t* fac)
{
    const int L12 = l1 + l2;
    int n = 0, k = 0;
    start[0] = 0;
    for (int ax = l1; ax >= 0; --ax)
        for (int ay = l1 - ax; ay >= 0; --ay)
            for (int bx = l2; bx >= 0; --bx)
                for (int by = l2 - bx; by >= 0; --by) {
                    const int a[3] = {ax, ay, l1 - ax - ay}, b[3] = {bx, by, l2 - bx - by};
                    for (int tx = 0; tx <= a[0] + b[0]; ++tx)
                        for (int ty = 0; ty <= a[1] + b[1]; ++ty)
                            for (int tz = 0; tz <= a[2] + b[2]; ++tz) {
                                herm[n] = (int16_t)hidx(tx, ty, tz);
                                const int tt[3] = {tx, ty, tz};
                                for (int i = 0; i < 3; ++i)
                                    fac[3 * n + i] = (uint8_t)((a[i] * (l2 + 1) + b[i]) * (L12 + 1) + tt[i]);
                                ++n;
                            }
                    start[++k] = n;
                }
    return n;
}

static void class_tables(eri_class_t c, const uint8_t* dev_blob, ClassTables* t)
{
    std::memset(t, 0, sizeof(*t));
    t->la = c.la; t->lb = c.lb; t->lc = c.lc; t->ld = c.ld;
    t->Lb = c.la + c.lb; t->Lk = c.lc + c.ld; t->L = t->Lb + t->Lk;
    t->nab = host_nc(c.la) * host_nc(c.lb);
    t->ncd = host_nc(c.lc) * host_nc(c.ld);
    t->nhb = host_nh(t->Lb); t->nhk = host_nh(t->Lk); t->nhl = host_nh(t->L);
    t->nab_f = t->nab;
    t->ncd_f = t->ncd;
    t->Tab = terms_of(c.la, c.lb, h_blob.bstart, h_blob.bp, h_blob.bfac);
    t->Tcd = terms_of(c.lc, c.ld, h_blob.kstart, h_blob.kq, h_blob.kfac);
    for (int p = 0; p < t->nhb; ++p)
        for (int q = 0; q < t->nhk; ++q) {
            int a, b, cc, x, y, z;
            htuv(p, &a, &b, &cc);
            htuv(q, &x, &y, &z);
            h_blob.pq[p * t->nhk + q] = (int16_t)hidx(a + x, b + y, cc + z);
        }
    const HostClassBlob* d = reinterpret_cast<const HostClassBlob*>(dev_blob);
    t->bra_start = d->bstart;
    t->ket_start = d->kstart;
    t->bra_p = d->bp;
    t->ket_q = d->kq;
    t->pq = d->pq;
    t->bra_fac = d->bfac;
    t->ket_fac = d->kfac;
}

}  // namespace eri

using namespace eri;

extern "C" int eri_batch_noalloc(eri_class_t cls, const eri_basis_t* basis, const int32_t* bra_pairs, int64_t nbra,
                                 const int32_t* ket_pairs, int64_t nket, const int64_t* quartets, int64_t nq,
                                 double* out, int64_t out_len, void* stream)
{
    int err = check_batch_args(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, out_len);
    if (err != ERI_OK) return err;
    const int64_t nqq = quartets ? nq : nbra * nket;
    if (nqq == 0 || nbra == 0 || nket == 0) return ERI_OK;
    if (!out) return ERI_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return ERI_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    DevPtrs& d = g_dev_ptrs[dev];
    if (!d.ready) {
        err = setup_device(dev, &d);
        if (err != ERI_OK) return err;
    }
    ClassTables ct;
    class_tables(cls, d.cls, &ct);
    // stream-ordered upload of this call's class table (a pageable source is
    // staged before cudaMemcpyAsync returns, so h_blob may be reused at once)
    if (cudaMemcpyAsync(d.cls, &h_blob, sizeof(h_blob), cudaMemcpyHostToDevice, st) != cudaSuccess) return ERI_ECUDA;
    return fwd_batch_on(cls, basis, bra_pairs, nbra, ket_pairs, nket, quartets, nq, out, ct,
                        d.boys + (size_t)ct.L * kBoysRows, d.rsteps, d.info, d.scratch, kScratchDoubles, st);
}
