"""ctypes front end of the CPU oracle (test infrastructure only).

The C sources are compiled here with plain ``gcc -O2`` (no fast-math, so the
IEEE semantics of every operation are kept) into ``oracle/_build``.  Two
libraries come out of ``md_oracle.c`` + ``os_oracle.c``:

* ``liboracle_ld.so`` -- REAL = long double (x86: 80-bit extended,
  aarch64: IEEE binary128 in software); the reference for all pins;
* ``liboracle_d.so``  -- REAL = double, the same source, used for large
  parity samples and for the timed CPU baseline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SOURCES = ["md_oracle.c", "os_oracle.c"]
_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}


def _lib_path(prec: str) -> str:
    return os.path.join(_BUILD, f"liboracle_{prec}.so")


def build(force: bool = False) -> None:
    """Compile both oracle libraries (idempotent unless ``force``)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    newest = max(os.path.getmtime(s) for s in srcs)
    for prec, flags in (("ld", []), ("d", ["-DORACLE_REAL_DOUBLE"])):
        out = _lib_path(prec)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math", *flags, *srcs, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, out)


def build_mutant(n: int, outdir: str) -> str:
    """Compile the long-double oracle with deliberate mistake number ``n``
    planted (ORACLE_MUTANT, see md_oracle.c) into ``outdir``; returns the
    library path.  Used only by the test that shows the pins catch mistakes."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    out = os.path.join(outdir, f"liboracle_mutant{n}.so")
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                           f"-DORACLE_MUTANT={n}", *srcs, "-o", out, "-lm"])
    return out


def use_library(prec: str, path: str | None) -> None:
    """Point the ``prec`` front end at another build (None: the normal one)."""
    with _lock:
        _libs.pop(prec, None)
        _override[prec] = path


_override: dict[str, str | None] = {}


def lib(prec: str = "ld") -> ctypes.CDLL:
    """Load (building first if needed) the oracle library for ``prec`` in {'ld','d'}."""
    if prec not in ("ld", "d"):
        raise ValueError(prec)
    with _lock:
        if prec not in _libs:
            path = _override.get(prec)
            if path is None:
                build()
                path = _lib_path(prec)
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            getattr(L, f"oracle_{prec}_boys_batch").argtypes = [ctypes.c_int, P, ctypes.c_long, P]
            getattr(L, f"oracle_{prec}_hermite_E").argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [P]
            for name in ("prim_eri", "os_prim_eri"):
                f = getattr(L, f"oracle_{prec}_{name}")
                f.argtypes = [P] * 4 + [ctypes.c_double] * 4 + [P] * 5
                f.restype = None
            f = getattr(L, f"oracle_{prec}_eri_quartets")
            f.argtypes = [P] * 7 + [P, ctypes.c_long, P]
            f.restype = ctypes.c_long
            f = getattr(L, f"oracle_{prec}_os_eri_quartets")
            f.argtypes = [P] * 7 + [P, ctypes.c_long, P]
            f.restype = ctypes.c_long
            f = getattr(L, f"oracle_{prec}_eri_grad_quartets")
            f.argtypes = [P] * 7 + [P, ctypes.c_long, P, P, P]
            f.restype = None
            _libs[prec] = L
        return _libs[prec]


def _real_dtype(prec: str):
    return np.longdouble if prec == "ld" else np.float64


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def cart_components(l: int) -> list[tuple[int, int, int]]:
    """Cartesian components of a shell, x^l first (xx, xy, xz, yy, yz, zz for l=2)."""
    return [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]


def boys(mmax: int, T, prec: str = "ld") -> np.ndarray:
    """F_m(T) for m = 0..mmax (Eq. boys); returns shape (len(T), mmax+1)."""
    T = np.ascontiguousarray(np.atleast_1d(np.asarray(T, dtype=np.float64)))
    out = np.zeros((T.size, mmax + 1), dtype=_real_dtype(prec))
    getattr(lib(prec), f"oracle_{prec}_boys_batch")(mmax, _ptr(T), T.size, _ptr(out))
    return out


def hermite_E(la: int, lb: int, za: float, zb: float, Ax: float, Bx: float, prec: str = "ld") -> np.ndarray:
    """(E_x)_{ij}^t table along one axis (Eqs. E2rr1/E2rr2); shape (la+1, lb+1, la+lb+1)."""
    out = np.zeros((la + 1, lb + 1, la + lb + 1), dtype=_real_dtype(prec))
    getattr(lib(prec), f"oracle_{prec}_hermite_E")(la, lb, za, zb, Ax, Bx, _ptr(out))
    return out


def _prim(name, a, b, c, d, za, zb, zc, zd, A, B, C, D, prec):
    ints = [np.ascontiguousarray(np.asarray(x, dtype=np.int32)) for x in (a, b, c, d)]
    cen = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in (A, B, C, D)]
    f = getattr(lib(prec), f"oracle_{prec}_{name}")
    res = np.zeros(1, dtype=_real_dtype(prec))
    f(*[_ptr(x) for x in ints], za, zb, zc, zd, *[_ptr(x) for x in cen], _ptr(res))
    return res[0]


def prim_eri(a, b, c, d, za, zb, zc, zd, A, B, C, D, prec: str = "ld"):
    """Primitive [ab|cd] over monomials by the MD oracle."""
    return _prim("prim_eri", a, b, c, d, za, zb, zc, zd, A, B, C, D, prec)


def os_prim_eri(a, b, c, d, za, zb, zc, zd, A, B, C, D, prec: str = "ld"):
    """Primitive [ab|cd] over monomials by the Obara-Saika oracle."""
    return _prim("os_prim_eri", a, b, c, d, za, zb, zc, zd, A, B, C, D, prec)


def _basis_arrays(basis):
    keys = ("centres", "shell_atom", "shell_l", "shell_K", "shell_off", "exps", "coefs")
    types = (np.float64, np.int32, np.int32, np.int32, np.int32, np.float64, np.float64)
    return [np.ascontiguousarray(np.asarray(basis[k], dtype=t)) for k, t in zip(keys, types)]


def shellset_size(basis, quartets) -> np.ndarray:
    l = np.asarray(basis["shell_l"])
    q = np.asarray(quartets).reshape(-1, 4)
    nc = (l + 1) * (l + 2) // 2
    return nc[q[:, 0]] * nc[q[:, 1]] * nc[q[:, 2]] * nc[q[:, 3]]


def eri_quartets(basis, quartets, prec: str = "ld", threads: int = 1, method: str = "md") -> np.ndarray:
    """Contracted Cartesian shellsets for a list of shell quartets.

    ``quartets``: int array (nq, 4) of shell indices.  Returns one flat array
    holding the shellsets back to back, each in [a][b][c][d] order.
    ``threads`` > 1 runs independent chunks of quartets on that many host
    threads (each chunk is the same serial oracle call).  ``method='os'``
    evaluates the same shellsets with the independent Obara-Saika oracle.
    """
    arrs = _basis_arrays(basis)
    q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
    sizes = shellset_size(basis, q)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    out = np.zeros(int(offs[-1]), dtype=_real_dtype(prec))
    f = getattr(lib(prec), f"oracle_{prec}_{'os_' if method == 'os' else ''}eri_quartets")
    itemsize = out.itemsize

    def run(lo, hi):
        lo, hi = int(lo), int(hi)
        if hi <= lo:
            return
        f(*[_ptr(a) for a in arrs], ctypes.c_void_p(q.ctypes.data + 16 * lo), hi - lo,
          ctypes.c_void_p(out.ctypes.data + itemsize * int(offs[lo])))

    nq = q.shape[0]
    if threads <= 1 or nq < 2:
        run(0, nq)
    else:
        bounds = np.linspace(0, nq, min(threads, nq) + 1).astype(int)
        with ThreadPoolExecutor(len(bounds) - 1) as ex:
            list(ex.map(lambda i: run(bounds[i], bounds[i + 1]), range(len(bounds) - 1)))
    return out


def eri_grad_quartets(basis, quartets, W, prec: str = "ld", threads: int = 1):
    """Gradient of sum_q sum_abcd W (ab|cd) with respect to the atom centres and
    the primitive exponents (coefficients fixed).  ``W`` uses the layout of
    :func:`eri_quartets`.  Returns (grad_centres (natom,3), grad_exps (nprim,))."""
    arrs = _basis_arrays(basis)
    q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
    sizes = shellset_size(basis, q)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    if W.size != offs[-1]:
        raise ValueError("W has the wrong length")
    natom = arrs[0].size // 3
    nprim = arrs[5].size
    f = getattr(lib(prec), f"oracle_{prec}_eri_grad_quartets")
    dt = _real_dtype(prec)
    nq = q.shape[0]
    nchunk = max(1, min(threads, nq))
    bounds = np.linspace(0, nq, nchunk + 1).astype(int)
    gcs = [np.zeros(natom * 3, dtype=dt) for _ in range(nchunk)]
    ges = [np.zeros(nprim, dtype=dt) for _ in range(nchunk)]

    def run(i):
        lo, hi = int(bounds[i]), int(bounds[i + 1])
        if hi <= lo:
            return
        f(*[_ptr(a) for a in arrs], ctypes.c_void_p(q.ctypes.data + 16 * lo), hi - lo,
          ctypes.c_void_p(W.ctypes.data + 8 * int(offs[lo])), _ptr(gcs[i]), _ptr(ges[i]))

    if nchunk == 1:
        run(0)
    else:
        with ThreadPoolExecutor(nchunk) as ex:
            list(ex.map(run, range(nchunk)))
    return sum(gcs).reshape(natom, 3), sum(ges)
