"""The throughput probe (ef_fp64_probe), whose DFMA rate is the peak of the
element kernels' roofline, and the integer-pipe multiply that the element and
adjoint kernels use for their products: plausible, positive rates through the
C ABI, and the integer multiply equal bit for bit to the FP64 multiply
instruction on generated operands (every pair it does not hand back)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op", [0, 1, 2, 3, 4, 5, 6])
def test_fp64_probe_rates(op):
    from paper_1409_4618_gb300 import edgefem as ef

    rate, ms = ef.ef_fp64_probe(op, 20_000)
    assert ms > 0
    # between a tenth and ten times the GPU's nominal FP64 rate (0.63 T lane operations / s)
    assert 0.06e12 < rate < 6.3e12, rate
    with pytest.raises(ef.EdgeFemError):
        ef.ef_fp64_probe(7, 10)


def test_int_mul_is_the_fp64_multiply():
    from paper_1409_4618_gb300 import edgefem as ef

    n = 1 << 26
    for seed in (1, 0x5eed):
        flagged, mismatched = ef.ef_int_mul_check(n, seed)
        assert mismatched == 0
        # the special-value pairs (a quarter of them) and the products that
        # leave the normal range go to the FP64 instruction; the rest do not
        assert n // 16 < flagged < n // 2, flagged
