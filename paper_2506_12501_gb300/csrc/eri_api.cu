// eri_api.cu -- status, error strings and teardown of the ERI library.
#include <atomic>
#include <mutex>
#include <vector>

#include "eri_internal.h"

namespace eri {

static std::atomic<int> g_prof_on{0};
static std::atomic<int64_t> g_launches{0};
static std::mutex g_prof_mu;
struct ProfRec {
    int id;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_prof_pending;

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(int id_, cudaStream_t st_) : id(id_), st(st_)
{
    count_launch();
    if (g_prof_on.load()) {
        cudaEventCreate(&e0);
        cudaEventRecord(e0, st);
    }
}

ProfScope::~ProfScope()
{
    if (!e0) return;
    cudaEvent_t e1;
    cudaEventCreate(&e1);
    cudaEventRecord(e1, st);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.push_back({id, e0, e1});
}

}  // namespace eri

using namespace eri;

extern "C" int eri_profile_enable(int on)
{
    g_prof_on.store(on ? 1 : 0);
    return ERI_OK;
}

extern "C" int eri_profile_read(int n, int64_t* launches, double* ms)
{
    if (n < 0 || n > PROF_N || (n > 0 && (!launches || !ms))) return ERI_EINVAL;
    for (int i = 0; i < n; ++i) {
        launches[i] = 0;
        ms[i] = 0.0;
    }
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof_pending);
    }
    int rc = ERI_OK;
    for (auto& r : recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) rc = ERI_ECUDA;
        if (r.id >= 0 && r.id < n) {
            launches[r.id] += 1;
            ms[r.id] += t;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    return rc;
}

extern "C" int64_t eri_launch_count(void) { return g_launches.load(); }

extern "C" const char* eri_error_string(int code)
{
    switch (code) {
        case ERI_OK: return "ok";
        case ERI_EINVAL: return "invalid argument (class, contraction degree, index, size or pointer)";
        case ERI_ECLASS: return "a shell's angular momentum disagrees with the requested class";
        case ERI_ECUDA: return "a CUDA call failed";
        case ERI_ETIMEOUT: return "a bounded device-side wait ran out";
        case ERI_ENOMEM: return "device workspace allocation failed";
        case ERI_EPLAN: return "plan misuse";
        default: return "unknown error";
    }
}

extern "C" int eri_last_status(void* stream)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return ERI_ECUDA;
    int* st = device_status();
    if (!st) return ERI_ECUDA;
    int h = 0;
    if (cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ERI_ECUDA;
    if (h != 0) cudaMemset(st, 0, sizeof(int));
    switch (h) {
        case DEV_OK: return ERI_OK;
        case DEV_ECLASS: return ERI_ECLASS;
        case DEV_EINDEX: return ERI_EINVAL;
        case DEV_EK: return ERI_EINVAL;
        case DEV_ETIMEOUT: return ERI_ETIMEOUT;
        default: return ERI_ECUDA;
    }
}

extern "C" int eri_finalize(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return ERI_ECUDA;
    release_all();
    return ERI_OK;
}
