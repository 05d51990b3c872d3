"""GB300-native McMurchie-Davidson 4-centre ERI library (arXiv 2506.12501).

The compute path is the CUDA library ``libmderi.so`` (C ABI in
``include/eri.h``); this package is its thin Python binding.
"""
from .binding import (  # noqa: F401
    DeviceBasis,
    EriError,
    ERI_OK, ERI_EINVAL, ERI_ECLASS, ERI_ECUDA, ERI_ETIMEOUT, ERI_ENOMEM, ERI_EPLAN,
    ERI_PREC_FP64, ERI_PREC_SPLIT, ERI_LMAX, ERI_KMAX, ERI_BOYS_MMAX,
    EXPORTS,
    eri_boys,
    eri_batch,
    eri_batch_grad,
    eri_batch3,
    eri_batch_sph,
    solid_harmonics,
    eri_batch_noalloc,
    Plan,
    ERI_PLAN_STORE, ERI_PLAN_SPLIT, ERI_PLAN_NO_TUNE,
    ERI_NOALLOC_SCRATCH_BYTES,
    eri_last_status,
    eri_last_form,
    eri_last_tile,
    eri_set_forms,
    ERI_FORM_PLAIN, ERI_FORM_HRR,
    eri_last_grad_forms,
    eri_set_grad_forms,
    ERI_GRAD_X, ERI_GRAD_V, ERI_GRAD_ONE, ERI_GRAD_TWO, ERI_GRAD_ONE_SWAPPED,
    eri_finalize,
    eri_profile_enable,
    eri_profile_read,
    eri_launch_count,
    eri_peak_probe,
    partition,
    PEAK_DFMA, PEAK_DMMA, PEAK_FFMA, PEAK_DFMA_ONE_CHAIN,
    PROF_FWD, PROF_GRAD, PROF_PAIR, PROF_PREPASS,
    error_string,
    lib,
    nc,
    out_len,
)
from .autograd import ERIFunction, eri  # noqa: F401,E402
