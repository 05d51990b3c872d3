// eri_api.cu -- status, error strings and teardown of the ERI library.
#include "eri_internal.h"

using namespace eri;

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
