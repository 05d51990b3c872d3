"""TEST INFRASTRUCTURE ONLY: the CPU oracle for the 4-centre ERI library.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never touches the CUDA library and
the CUDA library never touches it.

``md_oracle.c`` is a plain serial McMurchie-Davidson implementation
(arXiv 2506.12501, Section 2.1) built twice from one source: ``long double``
(``ld``) and ``double`` (``d``).  ``os_oracle.c`` is an independent
Obara-Saika recursion used to pin the MD oracle on small inputs.
``solid.py`` holds the real solid harmonics (closed form) and the 3-centre
integrals as 4-centre integrals with a unit second bra function.
"""
from . import oracle  # noqa: F401
from . import solid  # noqa: F401
from .oracle import (  # noqa: F401
    build,
    lib,
    boys,
    hermite_E,
    prim_eri,
    os_prim_eri,
    eri_quartets,
    eri_grad_quartets,
    shellset_size,
    ncart,
    cart_components,
)
