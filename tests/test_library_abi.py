"""The C-ABI library builds for sm_103a and exports every entry point that
include/*.h declares (CPU only: no kernel is launched)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(eri_[a-z_0-9]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("eri_boys", "eri_batch", "eri_last_status", "eri_error_string", "eri_finalize"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2506_12501_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_symbols() - exported
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_error_strings_without_gpu():
    import paper_2506_12501_gb300 as eri
    assert "class" in eri.error_string(eri.ERI_ECLASS)
    assert eri.error_string(eri.ERI_OK) == "ok"
    assert eri.error_string(12345) == "unknown error"


def test_kernels_compiled_for_sm103a():
    """Every translation unit is compiled with -gencode arch=compute_103a,code=sm_103a."""
    from paper_2506_12501_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_solid_harmonic_tables_agree_without_gpu():
    """The library builds its real solid harmonics by recursion in l (host
    code, no GPU work); the oracle writes them from their closed form.  The
    two independent constructions agree to round-off."""
    import numpy as np

    import oracle
    import paper_2506_12501_gb300 as eri
    for l in range(4):
        assert np.allclose(eri.solid_harmonics(l), oracle.solid.c2s(l), rtol=0, atol=1e-14), l
    with pytest.raises(eri.EriError):
        eri.solid_harmonics(4)


def test_form_selectors_without_gpu():
    """The form masks and form queries are host-only entry points: their
    argument checks and the not-yet-run answers need no GPU."""
    import paper_2506_12501_gb300 as eri
    L = eri.lib()
    assert L.eri_set_grad_forms(16) == eri.ERI_EINVAL
    assert L.eri_set_grad_forms(-1) == eri.ERI_EINVAL
    prev = L.eri_set_grad_forms(1 << eri.ERI_GRAD_V)
    assert 0 < prev <= 15
    assert L.eri_set_grad_forms(0) == 1 << eri.ERI_GRAD_V  # 0 restores everything
    assert L.eri_set_grad_forms((1 << eri.ERI_GRAD_X) | (1 << eri.ERI_GRAD_ONE)) == 15
    assert L.eri_set_grad_forms(0) == (1 << eri.ERI_GRAD_X) | (1 << eri.ERI_GRAD_ONE)
    assert L.eri_set_forms(16) == eri.ERI_EINVAL
    assert L.eri_last_grad_forms(None, None) == eri.ERI_EINVAL
    b, k = ctypes.c_int32(), ctypes.c_int32()
    r = L.eri_last_grad_forms(ctypes.byref(b), ctypes.byref(k))
    assert r == eri.ERI_EINVAL or (r == eri.ERI_OK and b.value in (0, 1) and k.value in (0, 1, 2, 4))


def test_tile_query_and_probe_kinds_without_gpu():
    """eri_last_tile answers ERI_EINVAL before the thread's first eri_batch
    launch (or a shape with a valid width after one), with NULL outputs
    allowed; eri_peak_probe rejects an unknown kind and a NULL rate before
    any GPU work."""
    import paper_2506_12501_gb300 as eri
    L = eri.lib()
    v = [ctypes.c_int32() for _ in range(4)]
    r = L.eri_last_tile(*(ctypes.byref(x) for x in v))
    assert r == eri.ERI_EINVAL or (r == eri.ERI_OK and v[0].value >= 1 and v[2].value in (256, 512))
    assert L.eri_last_tile(None, None, None, None) in (eri.ERI_EINVAL, eri.ERI_OK)
    g = ctypes.c_double()
    assert L.eri_peak_probe(4, ctypes.byref(g), None, None) == eri.ERI_EINVAL
    assert L.eri_peak_probe(-1, ctypes.byref(g), None, None) == eri.ERI_EINVAL
    assert L.eri_peak_probe(3, None, None, None) == eri.ERI_EINVAL
