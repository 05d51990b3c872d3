// eri_peaks.cu -- measurement support: arithmetic-throughput probes of the
// GPU the library runs on (FP64 FMA, FP64 tensor-core MMA, FP32 FMA), the
// denominators of the kernels' roofline fractions.  Not part of the method.
//
// Each probe is one launch over every SM (a few CTAs per SM, each thread
// running independent FMA chains, or each warp independent MMA chains) whose
// duration is measured with CUDA events on the caller's stream.  Thread 0 of
// every CTA also reads the SM cycle counter and the global nanosecond timer
// at its start and end, which gives the SM clock during the probe.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "eri_internal.h"

namespace eri {

constexpr int kProbeThreads = 256;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// clk[blockIdx] = {cycles, ns} of the CTA; sink keeps the chains alive
template <typename T, int CH>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int64_t iters, T b, T c, T* sink,
                                                                  unsigned long long* clk)
{
    uint64_t c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        t0 = global_ns();
        c0 = clock64();
    }
    T v[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) v[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CH; ++j) v[j] = fma(v[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < CH; ++j) s += v[j];
    if (s == (T)-12345.0) sink[threadIdx.x] = s;  // never true; keeps the arithmetic
    if (threadIdx.x == 0) {
        const uint64_t c1 = clock64(), t1 = global_ns();
        clk[2 * blockIdx.x] = c1 - c0;
        clk[2 * blockIdx.x + 1] = t1 - t0;
    }
}

// FP64 MMA m8n8k4 (D = A B + C, 512 flops per warp instruction), four
// independent accumulators per warp
__global__ void __launch_bounds__(kProbeThreads) dmma_probe_kernel(int64_t iters, double* sink,
                                                                   unsigned long long* clk)
{
    uint64_t c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        t0 = global_ns();
        c0 = clock64();
    }
    const double a = 1e-3 * (threadIdx.x & 7), b = 0.5;
    double d[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j][0] = d[j][1] = 1e-6 * j;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[j][0]), "+d"(d[j][1])
                         : "d"(a), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += d[j][0] + d[j][1];
    if (s == -12345.0) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) {
        const uint64_t c1 = clock64(), t1 = global_ns();
        clk[2 * blockIdx.x] = c1 - c0;
        clk[2 * blockIdx.x + 1] = t1 - t0;
    }
}

}  // namespace eri

using namespace eri;

// One probe configuration: `per_sm` CTAs per SM, `chains` independent
// chains per thread (MMA: per warp).  Returns ERI_OK and the GFLOP/s of the
// best of three timed launches of about 100 ms, and the SM clock of the last.
static int probe_once(int kind, int chains, int per_sm, cudaStream_t st, double* gflops, double* sm_mhz)
{
    const int grid = per_sm * sm_count();
    int err = ERI_OK;
    // [grid][2] clock records, then a small sink
    uint8_t* ws = (uint8_t*)aux_workspace(sizeof(unsigned long long) * 2 * grid + 8 * kProbeThreads, &err);
    if (!ws) return err;
    unsigned long long* clk = (unsigned long long*)ws;
    double* sink = (double*)(ws + sizeof(unsigned long long) * 2 * grid);
    auto launch = [&](int64_t iters) {
        count_launch();
        if (kind == 1)
            dmma_probe_kernel<<<grid, kProbeThreads, 0, st>>>(iters, sink, clk);
        else if (kind == 3)
            fma_probe_kernel<double, 1><<<grid, kProbeThreads, 0, st>>>(iters, 0.999999, 1e-7, sink, clk);
        else if (kind == 0 && chains == 4)
            fma_probe_kernel<double, 4><<<grid, kProbeThreads, 0, st>>>(iters, 0.999999, 1e-7, sink, clk);
        else if (kind == 0 && chains == 8)
            fma_probe_kernel<double, 8><<<grid, kProbeThreads, 0, st>>>(iters, 0.999999, 1e-7, sink, clk);
        else if (kind == 0)
            fma_probe_kernel<double, 16><<<grid, kProbeThreads, 0, st>>>(iters, 0.999999, 1e-7, sink, clk);
        else if (chains == 4)
            fma_probe_kernel<float, 4><<<grid, kProbeThreads, 0, st>>>(iters, 0.9999f, 1e-4f, (float*)sink, clk);
        else if (chains == 8)
            fma_probe_kernel<float, 8><<<grid, kProbeThreads, 0, st>>>(iters, 0.9999f, 1e-4f, (float*)sink, clk);
        else
            fma_probe_kernel<float, 16><<<grid, kProbeThreads, 0, st>>>(iters, 0.9999f, 1e-4f, (float*)sink, clk);
    };
    // flops of one iteration of the whole grid
    const double per_iter = kind == 1 ? (double)grid * (kProbeThreads / 32) * 4 * 512.0
                                      : (double)grid * kProbeThreads * chains * 2.0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ERI_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ERI_ECUDA;
    }
    // calibrate on a short launch, then time launches of about 100 ms (best of 3)
    int64_t iters = 1 << 12;
    float ms = 0.f;
    bool ok = true;
    launch(iters);
    ok &= cudaEventRecord(e0, st) == cudaSuccess;
    launch(iters);
    ok &= cudaEventRecord(e1, st) == cudaSuccess;
    ok &= cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (ok) {
        iters = std::max<int64_t>(iters, (int64_t)((double)iters * 100.0 / std::max(ms, 1e-3f)));
        iters = std::min<int64_t>(iters, (int64_t)1 << 26);
        float best = 3e38f;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            ok &= cudaEventRecord(e0, st) == cudaSuccess;
            launch(iters);
            ok &= cudaEventRecord(e1, st) == cudaSuccess;
            ok &= cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            best = std::min(best, ms);
        }
        ms = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || cudaGetLastError() != cudaSuccess) return ERI_ECUDA;
    *gflops = per_iter * (double)iters / ((double)ms * 1e-3) / 1e9;
    // cycles over nanoseconds of the last launch, averaged over its CTAs
    std::vector<unsigned long long> h(2 * (size_t)grid);
    if (cudaMemcpy(h.data(), clk, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ERI_ECUDA;
    double cyc = 0, ns = 0;
    for (int i = 0; i < grid; ++i) {
        cyc += (double)h[2 * i];
        ns += (double)h[2 * i + 1];
    }
    *sm_mhz = ns > 0 ? 1e3 * cyc / ns : 0.0;
    return ERI_OK;
}

extern "C" int eri_peak_probe(int kind, double* gflops, double* sm_mhz, void* stream)
{
    if (kind < 0 || kind > 3 || !gflops) return ERI_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == 3) {  // one dependent DFMA chain per thread, one CTA (8 warps) per SM
        double g = 0.0, mhz = 0.0;
        const int rc = probe_once(3, 1, 1, st, &g, &mhz);
        if (rc != ERI_OK) return rc;
        *gflops = g;
        if (sm_mhz) *sm_mhz = mhz;
        return ERI_OK;
    }
    // the best over a few occupancies and chain counts (MMA: four
    // accumulators per warp, at two occupancies)
    const int shapes[][2] = {{4, 2}, {8, 2}, {16, 2}, {4, 4}, {8, 4}, {16, 4}, {8, 8}};
    double best = -1.0, best_mhz = 0.0;
    for (const auto& sh : shapes) {
        if (kind == 1 && sh[0] != 8) continue;
        double g = 0.0, mhz = 0.0;
        const int rc = probe_once(kind, sh[0], sh[1], st, &g, &mhz);
        if (rc != ERI_OK) return rc;
        if (g > best) {
            best = g;
            best_mhz = mhz;
        }
    }
    *gflops = best;
    if (sm_mhz) *sm_mhz = best_mhz;
    return ERI_OK;
}
