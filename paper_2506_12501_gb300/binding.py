"""ctypes binding of ``libmderi.so`` (include/eri.h).

Argument marshalling only: tensors are passed as raw device pointers and the
current torch CUDA stream as the ``stream`` argument; every integral is
computed by the library's kernels.  There is no CPU fallback: if the
library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

ERI_OK, ERI_EINVAL, ERI_ECLASS, ERI_ECUDA, ERI_ETIMEOUT, ERI_ENOMEM, ERI_EPLAN = 0, -1, -2, -3, -4, -5, -6
ERI_PREC_FP64, ERI_PREC_SPLIT = 0, 1
ERI_LMAX, ERI_KMAX, ERI_BOYS_MMAX = 3, 8, 20

_lock = threading.Lock()
_lib = None


class EriError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} (code {code})")


class eri_class_t(ctypes.Structure):
    _fields_ = [("la", ctypes.c_int32), ("lb", ctypes.c_int32), ("lc", ctypes.c_int32), ("ld", ctypes.c_int32)]


class eri_basis_t(ctypes.Structure):
    _fields_ = [("centres", ctypes.c_void_p), ("shell_atom", ctypes.c_void_p), ("shell_l", ctypes.c_void_p),
                ("shell_K", ctypes.c_void_p), ("shell_off", ctypes.c_void_p), ("exps", ctypes.c_void_p),
                ("coefs", ctypes.c_void_p), ("natom", ctypes.c_int32), ("nshell", ctypes.c_int32),
                ("nprim", ctypes.c_int32)]


EXPORTS = ["eri_boys", "eri_batch", "eri_batch_grad", "eri_last_status", "eri_error_string", "eri_finalize",
           "eri_profile_enable", "eri_profile_read", "eri_launch_count", "eri_batch_noalloc", "eri_plan_create",
           "eri_plan_execute", "eri_plan_set_budget", "eri_plan_status", "eri_plan_info", "eri_plan_job",
           "eri_plan_destroy", "eri_last_form", "eri_set_forms", "eri_plan_coulomb", "eri_plan_jk", "eri_plan_job_degrees", "eri_batch3", "eri_solid_harmonics", "eri_batch_sph",
           "eri_last_grad_forms", "eri_set_grad_forms", "eri_peak_probe",
           "eri_partition", "eri_plan_set_slice", "eri_plan_slice_info", "eri_last_tile"]
ERI_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024
ERI_PLAN_STORE, ERI_PLAN_SPLIT, ERI_PLAN_NO_TUNE = 1, 2, 4
ERI_FORM_PLAIN, ERI_FORM_HRR = 0x3, 0xC
ERI_GRAD_X, ERI_GRAD_V, ERI_GRAD_ONE, ERI_GRAD_TWO, ERI_GRAD_ONE_SWAPPED = 0, 1, 2, 3, 4
PROF_FWD, PROF_GRAD, PROF_PAIR, PROF_PREPASS = 0, 1, 2, 3


def lib() -> ctypes.CDLL:
    """Load the library, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.eri_boys.argtypes = [I, P, I64, P, P]
            L.eri_batch.argtypes = [eri_class_t, ctypes.POINTER(eri_basis_t), P, I64, P, I64, P, I64, P, I64, I, P]
            L.eri_solid_harmonics.argtypes = [ctypes.c_int32, P]
            L.eri_batch_sph.argtypes = [eri_class_t, ctypes.POINTER(eri_basis_t), P, I64, P, I64, P, I64, P, I64, I, P]
            L.eri_batch3.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(eri_basis_t), P,
                                     I64, P, I64, P, I64, ctypes.c_int32, P, I64, I, P]
            L.eri_batch_grad.argtypes = [eri_class_t, ctypes.POINTER(eri_basis_t), P, I64, P, I64, P, I64, P, I64,
                                         P, P, P]
            L.eri_last_status.argtypes = [P]
            L.eri_last_form.argtypes = [P, P]
            L.eri_last_tile.argtypes = [P, P, P, P]
            L.eri_set_forms.argtypes = [ctypes.c_int32]
            L.eri_last_grad_forms.argtypes = [P, P]
            L.eri_set_grad_forms.argtypes = [ctypes.c_int32]
            L.eri_error_string.argtypes = [I]
            L.eri_error_string.restype = ctypes.c_char_p
            L.eri_finalize.argtypes = []
            L.eri_batch_noalloc.argtypes = [eri_class_t, ctypes.POINTER(eri_basis_t), P, I64, P, I64, P, I64, P,
                                            I64, P]
            L.eri_batch_noalloc.restype = I
            L.eri_plan_create.argtypes = [ctypes.POINTER(eri_basis_t), ctypes.c_double, I, P, ctypes.POINTER(P)]
            L.eri_plan_execute.argtypes = [P, P, ctypes.c_int32, P, P, I64, P]
            L.eri_plan_coulomb.argtypes = [P, P, ctypes.c_int32, P, P]
            L.eri_plan_jk.argtypes = [P, P, ctypes.c_int32, P, P, P]
            L.eri_plan_set_budget.argtypes = [P, I64]
            L.eri_plan_status.argtypes = [P, P]
            L.eri_plan_info.argtypes = [P, P, P, P, P]
            L.eri_plan_job.argtypes = [P, ctypes.c_int32, P, P, P, P]
            L.eri_plan_destroy.argtypes = [P]
            L.eri_plan_job_degrees.argtypes = [P, ctypes.c_int32, P, P]
            for f in ("eri_plan_create", "eri_plan_execute", "eri_plan_set_budget", "eri_plan_status",
                      "eri_plan_info", "eri_plan_job", "eri_plan_destroy"):
                getattr(L, f).restype = I
            L.eri_profile_enable.argtypes = [I]
            L.eri_profile_enable.restype = I
            L.eri_profile_read.argtypes = [I, P, P]
            L.eri_profile_read.restype = I
            L.eri_partition.argtypes = [P, I64, ctypes.c_int32, P, P]
            L.eri_partition.restype = I
            L.eri_plan_set_slice.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P]
            L.eri_plan_set_slice.restype = I
            L.eri_plan_slice_info.argtypes = [P, P, P, P]
            L.eri_plan_slice_info.restype = I
            L.eri_peak_probe.argtypes = [I, P, P, P]
            L.eri_peak_probe.restype = I
            L.eri_launch_count.argtypes = []
            L.eri_launch_count.restype = I64
            for f in ("eri_boys", "eri_batch", "eri_batch_grad", "eri_last_status", "eri_finalize"):
                getattr(L, f).restype = I
            _lib = L
        return _lib


def error_string(code: int) -> str:
    return lib().eri_error_string(code).decode()


def _check(code: int, where: str):
    if code != ERI_OK:
        raise EriError(code, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor on the current device.
    With ``dtype`` the tensor's element type is checked too: the library reads
    and writes raw memory, so a tensor of the wrong type or on another GPU
    would be read or written past its end."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on {t.device}, but the current device is cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _pairs(t, name):
    """A [n][2] int32 pair list (or [n] int32 shell list when 1-D)."""
    p = _ptr(t, torch.int32, name)
    if t.dim() == 2 and t.shape[1] != 2:
        raise ValueError(f"{name}: expected shape [n][2], got {tuple(t.shape)}")
    return p


def _quartets(t, name="quartets"):
    if t is None:
        return None
    p = _ptr(t, torch.int64, name)
    if t.dim() != 2 or t.shape[1] != 2:
        raise ValueError(f"{name}: expected shape [n][2], got {tuple(t.shape)}")
    return p


def _f64(t, name):
    return _ptr(t, torch.float64, name)


def nc(l: int) -> int:
    return (l + 1) * (l + 2) // 2


class DeviceBasis:
    """A basis (see synth.Basis) copied to the current CUDA device."""

    def __init__(self, basis, device=None):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        f64 = dict(dtype=torch.float64, device=dev)
        i32 = dict(dtype=torch.int32, device=dev)
        self.centres = torch.as_tensor(basis["centres"], **f64).reshape(-1, 3).contiguous()
        self.shell_atom = torch.as_tensor(basis["shell_atom"], **i32).contiguous()
        self.shell_l = torch.as_tensor(basis["shell_l"], **i32).contiguous()
        self.shell_K = torch.as_tensor(basis["shell_K"], **i32).contiguous()
        self.shell_off = torch.as_tensor(basis["shell_off"], **i32).contiguous()
        self.exps = torch.as_tensor(basis["exps"], **f64).contiguous()
        self.coefs = torch.as_tensor(basis["coefs"], **f64).contiguous()

    def struct(self, centres=None, exps=None) -> eri_basis_t:
        c = self.centres if centres is None else centres
        e = self.exps if exps is None else exps
        if c.dim() != 2 or c.shape[1] != 3:
            raise ValueError(f"centres: expected shape [natom][3], got {tuple(c.shape)}")
        return eri_basis_t(_f64(c, "centres"), _ptr(self.shell_atom, torch.int32, "shell_atom"),
                           _ptr(self.shell_l, torch.int32, "shell_l"), _ptr(self.shell_K, torch.int32, "shell_K"),
                           _ptr(self.shell_off, torch.int32, "shell_off"), _f64(e, "exps"),
                           _f64(self.coefs, "coefs"), c.shape[0],
                           self.shell_l.shape[0], e.shape[0])


def eri_boys(mmax: int, T: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """F_m(T), m = 0..mmax, shape (n, mmax+1), by the library's Boys kernel."""
    T = T.contiguous()
    if out is None:
        out = torch.empty((T.numel(), mmax + 1), dtype=torch.float64, device=T.device)
    if out.numel() < T.numel() * (mmax + 1):
        raise ValueError(f"out: expected at least {T.numel() * (mmax + 1)} elements, got {out.numel()}")
    _check(lib().eri_boys(mmax, _f64(T, "T"), T.numel(), _f64(out, "out"), _stream(stream)), "eri_boys")
    return out


def out_len(cls, nbra: int, nket: int, nq: int | None) -> int:
    la, lb, lc, ld = cls
    nqq = nq if nq is not None else nbra * nket
    return nqq * nc(la) * nc(lb) * nc(lc) * nc(ld)


def eri_batch(cls, basis: DeviceBasis, bra_pairs: torch.Tensor, ket_pairs: torch.Tensor,
              quartets: torch.Tensor | None = None, out: torch.Tensor | None = None,
              precision: int = ERI_PREC_FP64, stream=None, centres=None, exps=None) -> torch.Tensor:
    """Contracted Cartesian shellsets of class ``cls`` (see include/eri.h for the layout)."""
    nbra, nket = bra_pairs.shape[0], ket_pairs.shape[0]
    nq = quartets.shape[0] if quartets is not None else None
    n = out_len(cls, nbra, nket, nq)
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=bra_pairs.device)
    if n == 0:  # an empty quartet list has no device pointer; nothing to compute
        return out
    b = basis.struct(centres, exps)
    code = lib().eri_batch(eri_class_t(*cls), ctypes.byref(b), _pairs(bra_pairs, "bra_pairs"), nbra,
                           _pairs(ket_pairs, "ket_pairs"), nket, _quartets(quartets), nq if nq is not None else 0,
                           _f64(out, "out"), out.numel(), precision, _stream(stream))
    _check(code, "eri_batch")
    return out


def eri_batch_sph(cls, basis: DeviceBasis, bra_pairs: torch.Tensor, ket_pairs: torch.Tensor,
                  quartets: torch.Tensor | None = None, out: torch.Tensor | None = None,
                  precision: int = ERI_PREC_FP64, stream=None) -> torch.Tensor:
    """Shellsets of class ``cls`` with every centre in real solid harmonics (see include/eri.h)."""
    nbra, nket = bra_pairs.shape[0], ket_pairs.shape[0]
    nq = quartets.shape[0] if quartets is not None else None
    ns = (2 * cls[0] + 1) * (2 * cls[1] + 1) * (2 * cls[2] + 1) * (2 * cls[3] + 1)
    n = (nq if nq is not None else nbra * nket) * ns
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=bra_pairs.device)
    if n == 0:
        return out
    b = basis.struct()
    code = lib().eri_batch_sph(eri_class_t(*cls), ctypes.byref(b), _pairs(bra_pairs, "bra_pairs"), nbra,
                               _pairs(ket_pairs, "ket_pairs"), nket, _quartets(quartets),
                               nq if nq is not None else 0, _f64(out, "out"), out.numel(), precision,
                               _stream(stream))
    _check(code, "eri_batch_sph")
    return out


def solid_harmonics(l: int):
    """[2l+1][nc(l)] Cartesian coefficients of the library's real solid harmonics (host)."""
    import numpy as np
    out = np.zeros((2 * l + 1, nc(l)), dtype=np.float64)
    _check(lib().eri_solid_harmonics(int(l), ctypes.c_void_p(out.ctypes.data)), "eri_solid_harmonics")
    return out


def eri_batch3(lx: int, lc: int, ld: int, basis: DeviceBasis, x_shells: torch.Tensor, ket_pairs: torch.Tensor,
               triples: torch.Tensor | None = None, pure: bool = True, out: torch.Tensor | None = None,
               precision: int = ERI_PREC_FP64, stream=None) -> torch.Tensor:
    """3-centre shellsets (x|cd) of class (lx | lc ld) (see include/eri.h for the layout)."""
    nx, nket = x_shells.shape[0], ket_pairs.shape[0]
    nt = triples.shape[0] if triples is not None else None
    ncx = 2 * lx + 1 if pure else nc(lx)
    n = (nt if nt is not None else nx * nket) * ncx * nc(lc) * nc(ld)
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=x_shells.device)
    if n == 0:
        return out
    b = basis.struct()
    code = lib().eri_batch3(lx, lc, ld, ctypes.byref(b), _ptr(x_shells, torch.int32, "x_shells"), nx,
                            _pairs(ket_pairs, "ket_pairs"), nket, _quartets(triples, "triples"),
                            nt if nt is not None else 0, 1 if pure else 0, _f64(out, "out"), out.numel(), precision,
                            _stream(stream))
    _check(code, "eri_batch3")
    return out


def eri_batch_grad(cls, basis: DeviceBasis, bra_pairs, ket_pairs, quartets, W: torch.Tensor,
                   grad_centres: torch.Tensor | None = None, grad_exps: torch.Tensor | None = None,
                   stream=None, centres=None, exps=None):
    """Accumulate d(sum W (ab|cd))/d(centres, exponents) into the given tensors."""
    nbra, nket = bra_pairs.shape[0], ket_pairs.shape[0]
    nq = quartets.shape[0] if quartets is not None else None
    if out_len(cls, nbra, nket, nq) == 0:
        return grad_centres, grad_exps
    b = basis.struct(centres, exps)
    W = W.contiguous()
    if grad_centres is not None and grad_centres.numel() != 3 * b.natom:
        raise ValueError(f"grad_centres: expected {3 * b.natom} elements, got {grad_centres.numel()}")
    if grad_exps is not None and grad_exps.numel() != b.nprim:
        raise ValueError(f"grad_exps: expected {b.nprim} elements, got {grad_exps.numel()}")
    code = lib().eri_batch_grad(eri_class_t(*cls), ctypes.byref(b), _pairs(bra_pairs, "bra_pairs"), nbra,
                                _pairs(ket_pairs, "ket_pairs"), nket, _quartets(quartets),
                                nq if nq is not None else 0, _f64(W, "W"), W.numel(),
                                _f64(grad_centres, "grad_centres"), _f64(grad_exps, "grad_exps"), _stream(stream))
    _check(code, "eri_batch_grad")
    return grad_centres, grad_exps


def eri_last_status(stream=None) -> int:
    return lib().eri_last_status(_stream(stream))


def eri_set_forms(mask: int) -> int:
    """Restrict eri_batch's forms (ERI_FORM_PLAIN, ERI_FORM_HRR, or 0 = all); returns the previous mask."""
    code = lib().eri_set_forms(int(mask))
    if code < 0:
        _check(code, "eri_set_forms")
    return code


def eri_last_form() -> tuple:
    """(swapped, hrr) of this thread's last eri_batch launch."""
    sw = ctypes.c_int32()
    hrr = ctypes.c_int32()
    _check(lib().eri_last_form(ctypes.byref(sw), ctypes.byref(hrr)), "eri_last_form")
    return bool(sw.value), bool(hrr.value)


def eri_last_tile() -> dict:
    """Tile shape of this thread's last eri_batch launch: quartets per tile, bra primitives per chunk,
    threads per CTA and dynamic shared memory (bytes)."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().eri_last_tile(*(ctypes.byref(x) for x in v)), "eri_last_tile")
    return {"tq": v[0].value, "ic": v[1].value, "threads": v[2].value, "smem_bytes": v[3].value}


def eri_set_grad_forms(mask: int) -> int:
    """Restrict eri_batch_grad's forms: bits ERI_GRAD_X / ERI_GRAD_V (a side's form), ERI_GRAD_ONE (single
    launch), ERI_GRAD_TWO (two launches); no launch bit = two launches; 0 = everything.  Returns the previous mask."""
    code = lib().eri_set_grad_forms(int(mask))
    if code < 0:
        _check(code, "eri_set_grad_forms")
    return code


def eri_last_grad_forms() -> tuple:
    """(bra-channel form, ket-channel form) of the last eri_batch_grad call: ERI_GRAD_X or ERI_GRAD_V, and
    ERI_GRAD_ONE (ERI_GRAD_ONE_SWAPPED) as the ket form when one launch with the caller's bra (ket) as its
    kernel bra produced every channel."""
    b = ctypes.c_int32()
    k = ctypes.c_int32()
    _check(lib().eri_last_grad_forms(ctypes.byref(b), ctypes.byref(k)), "eri_last_grad_forms")
    return b.value, k.value


def eri_finalize() -> int:
    return lib().eri_finalize()


def eri_profile_enable(on: bool = True) -> None:
    _check(lib().eri_profile_enable(1 if on else 0), "eri_profile_enable")


def eri_profile_read() -> dict:
    """{kernel id: (launches, total ms)} since the last read (waits for the events)."""
    n = 4
    launches = (ctypes.c_int64 * n)()
    ms = (ctypes.c_double * n)()
    _check(lib().eri_profile_read(n, ctypes.cast(launches, ctypes.c_void_p), ctypes.cast(ms, ctypes.c_void_p)),
           "eri_profile_read")
    return {i: (int(launches[i]), float(ms[i])) for i in range(n)}


def partition(costs, nranks: int):
    """(owner rank of each unit, load of each rank): the library's
    longest-processing-time-first partition (host only, no GPU work)."""
    import numpy as np
    c = np.ascontiguousarray(costs, dtype=np.float64)
    owner = np.zeros(c.size, dtype=np.int32)
    load = np.zeros(max(int(nranks), 1), dtype=np.float64)
    _check(lib().eri_partition(ctypes.c_void_p(c.ctypes.data), c.size, int(nranks),
                               ctypes.c_void_p(owner.ctypes.data), ctypes.c_void_p(load.ctypes.data)),
           "eri_partition")
    return owner, load


PEAK_DFMA, PEAK_DMMA, PEAK_FFMA, PEAK_DFMA_ONE_CHAIN = 0, 1, 2, 3


def eri_peak_probe(kind: int, stream=None) -> tuple:
    """(GFLOP/s, SM MHz during the probe) of one arithmetic-throughput probe
    (PEAK_DFMA, PEAK_DMMA or PEAK_FFMA) on the current device."""
    g = ctypes.c_double()
    mhz = ctypes.c_double()
    _check(lib().eri_peak_probe(int(kind), ctypes.byref(g), ctypes.byref(mhz), _stream(stream)), "eri_peak_probe")
    return g.value, mhz.value


def eri_launch_count() -> int:
    return int(lib().eri_launch_count())


def eri_batch_noalloc(cls, basis: DeviceBasis, bra_pairs: torch.Tensor, ket_pairs: torch.Tensor,
                      quartets: torch.Tensor | None, out: torch.Tensor, stream=None) -> torch.Tensor:
    """The allocation-free variant of eri_batch (FP64): the caller passes the
    output tensor, and the library uses only its fixed, compiled-in scratch
    (see include/eri.h).  Nothing is allocated by this call."""
    nbra, nket = bra_pairs.shape[0], ket_pairs.shape[0]
    nq = quartets.shape[0] if quartets is not None else None
    if out_len(cls, nbra, nket, nq) == 0:
        return out
    b = basis.struct()
    code = lib().eri_batch_noalloc(eri_class_t(*cls), ctypes.byref(b), _pairs(bra_pairs, "bra_pairs"), nbra,
                                   _pairs(ket_pairs, "ket_pairs"), nket, _quartets(quartets),
                                   nq if nq is not None else 0, _f64(out, "out"), out.numel(), _stream(stream))
    _check(code, "eri_batch_noalloc")
    return out


class Plan:
    """eri_plan_* over a DeviceBasis (kept alive with the plan)."""

    def __init__(self, basis: DeviceBasis, threshold: float = 1e-12, flags: int = 0, stream=None):
        self.basis = basis
        self._struct = basis.struct()
        self.ptr = ctypes.c_void_p()
        self.flags = flags
        _check(lib().eri_plan_create(ctypes.byref(self._struct), float(threshold), flags, _stream(stream),
                                     ctypes.byref(self.ptr)), "eri_plan_create")

    def info(self):
        nq, nj, ni, ol = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().eri_plan_info(self.ptr, ctypes.byref(nq), ctypes.byref(nj), ctypes.byref(ni), ctypes.byref(ol)),
               "eri_plan_info")
        return {"nquartets": nq.value, "njobs": nj.value, "nitems": ni.value, "out_len": ol.value}

    def job(self, j: int, with_quartets: bool = False):
        import numpy as np
        cls = eri_class_t()
        nq, off = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().eri_plan_job(self.ptr, j, ctypes.byref(cls), ctypes.byref(nq), ctypes.byref(off), None),
               "eri_plan_job")
        shells = None
        if with_quartets:
            shells = np.zeros((nq.value, 4), dtype=np.int32)
            _check(lib().eri_plan_job(self.ptr, j, None, None, None, ctypes.c_void_p(shells.ctypes.data)),
                   "eri_plan_job")
        return (cls.la, cls.lb, cls.lc, cls.ld), nq.value, off.value, shells

    @staticmethod
    def _square(D, *others):
        """D is [nbf][nbf]; every other matrix has D's shape."""
        if D.dim() != 2 or D.shape[0] != D.shape[1]:
            raise ValueError(f"D: expected a square matrix, got {tuple(D.shape)}")
        for name, M in others:
            if M is not None and tuple(M.shape) != tuple(D.shape):
                raise ValueError(f"{name}: expected shape {tuple(D.shape)}, got {tuple(M.shape)}")

    def execute(self, D: torch.Tensor | None = None, energy: torch.Tensor | None = None,
                out: torch.Tensor | None = None, stream=None):
        if D is not None:
            self._square(D)
        if energy is not None and energy.numel() < 1:
            raise ValueError("energy: expected at least one element")
        nbf = D.shape[0] if D is not None else 0
        _check(lib().eri_plan_execute(self.ptr, _f64(D, "D"), nbf, _f64(energy, "energy"), _f64(out, "out"),
                                      out.numel() if out is not None else 0, _stream(stream)), "eri_plan_execute")

    def coulomb(self, D: torch.Tensor, J: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """J_uv = sum_ls (uv|ls) D_ls over every quartet of the plan and its permutation images."""
        D = D.contiguous()
        if J is None:
            J = torch.empty_like(D)
        self._square(D, ("J", J))
        _check(lib().eri_plan_coulomb(self.ptr, _f64(D, "D"), D.shape[0], _f64(J, "J"), _stream(stream)),
               "eri_plan_coulomb")
        return J

    def jk(self, D: torch.Tensor, want_j: bool = True, want_k: bool = True, J: torch.Tensor | None = None,
           K: torch.Tensor | None = None, stream=None):
        """(J, K) in one replay: J_uv = sum_ls (uv|ls) D_ls, K_ul = sum_vs (uv|ls) D_vs (None where not wanted)."""
        D = D.contiguous()
        if want_j and J is None:
            J = torch.empty_like(D)
        if want_k and K is None:
            K = torch.empty_like(D)
        J = J if want_j else None
        K = K if want_k else None
        self._square(D, ("J", J), ("K", K))
        _check(lib().eri_plan_jk(self.ptr, _f64(D, "D"), D.shape[0], _f64(J, "J"), _f64(K, "K"), _stream(stream)),
               "eri_plan_jk")
        return J, K

    def job_degrees(self, j: int):
        """(K_a K_b, K_c K_d) of job j, in the order of its class."""
        kb = ctypes.c_int32()
        kk = ctypes.c_int32()
        _check(lib().eri_plan_job_degrees(self.ptr, int(j), ctypes.byref(kb), ctypes.byref(kk)), "eri_plan_job_degrees")
        return kb.value, kk.value

    def set_slice(self, rank: int, nranks: int, stream=None):
        """Keep the work items the cost-balanced partition gives to ``rank`` of ``nranks``."""
        _check(lib().eri_plan_set_slice(self.ptr, int(rank), int(nranks), _stream(stream)), "eri_plan_set_slice")

    def slice_info(self):
        n, q, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().eri_plan_slice_info(self.ptr, ctypes.byref(n), ctypes.byref(q), ctypes.byref(c)),
               "eri_plan_slice_info")
        return {"nitems": n.value, "nquartets": q.value, "cost": c.value}

    def set_budget(self, cycles: int):
        _check(lib().eri_plan_set_budget(self.ptr, int(cycles)), "eri_plan_set_budget")

    def status(self, stream=None) -> int:
        return lib().eri_plan_status(self.ptr, _stream(stream))

    def destroy(self):
        if self.ptr:
            lib().eri_plan_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
