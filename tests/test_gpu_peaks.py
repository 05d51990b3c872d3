"""The library's arithmetic-throughput probes (measurement support): every
kind returns a positive rate at a plausible SM clock, an unknown kind is
rejected, and a single dependent DFMA chain per thread at 8 warps per SM runs
at the FP64 pipe's rate (the property that lets the FP64 transforms sum on
one accumulator chain)."""
import pytest

import paper_2506_12501_gb300 as eri

pytestmark = pytest.mark.gpu


def test_peak_probes(cuda):
    rates = {}
    for kind in (eri.PEAK_DFMA, eri.PEAK_DMMA, eri.PEAK_FFMA, eri.PEAK_DFMA_ONE_CHAIN):
        g, mhz = eri.eri_peak_probe(kind)
        assert g > 0 and 100 < mhz < 5000, (kind, g, mhz)
        rates[kind] = g
    assert rates[eri.PEAK_FFMA] > 10 * rates[eri.PEAK_DFMA]
    assert rates[eri.PEAK_DFMA_ONE_CHAIN] > 0.9 * rates[eri.PEAK_DFMA]
    with pytest.raises(eri.EriError):
        eri.eri_peak_probe(4)
