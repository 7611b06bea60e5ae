"""The FP64 throughput probe (ef_fp64_probe), whose DFMA rate is the peak of
the element kernels' roofline: plausible, positive rates for the three
operations through the C ABI."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("op", [0, 1, 2])
def test_fp64_probe_rates(op):
    from paper_1409_4618_gb300 import edgefem as ef

    rate, ms = ef.ef_fp64_probe(op, 20_000)
    assert ms > 0
    # between a tenth and ten times the GPU's nominal FP64 rate (0.63 T lane operations / s)
    assert 0.06e12 < rate < 6.3e12, rate
    with pytest.raises(ef.EdgeFemError):
        ef.ef_fp64_probe(3, 10)
