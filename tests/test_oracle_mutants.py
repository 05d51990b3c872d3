"""The oracle pins catch plausible mistakes (CPU only).

Each case builds the long-double oracle with one deliberate mistake planted
(ORACLE_MUTANT in oracle/md_oracle.c: a dropped term, a wrong operand, a
wrong sign, an off-by-one, a wrong constant, swapped centres) and checks
that at least one pin of tests/test_oracle_pins.py now fails.
"""
import pytest

import oracle
import test_oracle_pins as pins

MUTANTS = {
    1: "E recursion: (t+1) E^{t+1} term dropped",
    2: "E recursion: P-B used instead of P-A",
    3: "R recursion: (r_i - 1) term dropped",
    4: "R recursion: Q-P instead of P-Q",
    5: "sign (-1)^{l_q} of Eq. pq-from-r dropped",
    6: "Boys series: off-by-one in the odd denominators",
    7: "prefactor 2 pi^2 instead of 2 pi^(5/2)",
    8: "ket E built with the two centres swapped",
}

CHECKS = [
    lambda: pins.test_boys_incomplete_gamma(5.0),
    lambda: pins.test_E_defining_expansion(2, 1),
    lambda: pins.test_ssss_fourier_space(1),
    lambda: pins.test_far_field_dipole_sign(),
    lambda: pins.test_md_equals_obara_saika((1, 1, 1, 1)),
    lambda: pins.test_md_equals_obara_saika((2, 1, 2, 1)),
    lambda: pins.test_symmetries((2, 1, 2, 2)),
]


@pytest.mark.parametrize("n", sorted(MUTANTS))
def test_pins_catch_planted_mistake(n, tmp_path):
    path = oracle.oracle.build_mutant(n, str(tmp_path))
    oracle.oracle.use_library("ld", path)
    try:
        caught = []
        for i, check in enumerate(CHECKS):
            try:
                check()
            except AssertionError:
                caught.append(i)
        assert caught, f"mutant {n} ({MUTANTS[n]}) passed every pin"
    finally:
        oracle.oracle.use_library("ld", None)


def test_unmutated_build_passes_the_same_checks():
    for check in CHECKS:
        check()
