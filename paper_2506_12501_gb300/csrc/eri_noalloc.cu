// eri_noalloc.cu -- eri_batch_noalloc: the forward batch without any device
// or host allocation.
//
// Some callers cannot allocate: a process whose device memory is owned by
// another allocator (a serving or training framework's caching pool, an MPI
// library's registered pool) may not call cudaMalloc behind that
// allocator's back, since memory it does not know about can make it fail
// its own allocations or break its accounting.  For them the pair tables
// that eri_batch keeps in a cudaMalloc'ed workspace live here in a fixed,
// file-scope device array instead, next to fixed arrays for the constant
// tables (Boys function, recursion steps, class tables) and the validation
// words.  The arrays exist on every GPU that loads the library until the
// process exits.  The constant tables come from the same host builders as
// eri_batch's cached ones, which fill caller-given buffers and allocate
// nothing.
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

// ---- host tables in static storage (no heap), filled by the library's
// shared, allocation-free table builders
static long double h_master[kBoysGrid * (kBoysMtab + 2)];
static double h_boys[(kLtotMax + 1) * kBoysRows];
static RStep h_rsteps[kNhMax];

static void build_constant_tables()
{
    build_boys_master(h_master);
    for (int L = 0; L <= kLtotMax; ++L) boys_taylor_rows(h_master, L, h_boys + (size_t)L * kBoysRows);
    build_rstep_table(h_rsteps);
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
    t->Tab = pair_term_list(c.la, c.lb, h_blob.bstart, h_blob.bp, h_blob.bfac);
    t->Tcd = pair_term_list(c.lc, c.ld, h_blob.kstart, h_blob.kq, h_blob.kfac);
    for (int p = 0; p < t->nhb; ++p)
        for (int q = 0; q < t->nhk; ++q) {
            int a, b, cc, x, y, z;
            herm_tuv(p, &a, &b, &cc);
            herm_tuv(q, &x, &y, &z);
            h_blob.pq[p * t->nhk + q] = (int16_t)herm_index(a + x, b + y, cc + z);
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
