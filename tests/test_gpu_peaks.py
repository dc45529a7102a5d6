"""The roofline denominators measured on the GPU by the benchmark's probe
library (random-row reads, shared-memory lookups): plausible magnitudes, the
L2-resident table no slower than the HBM-sized one, and argument checks."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra, probes
    build.build()
    probes.load()
    probes.CagraError = cagra.CagraError
    return probes


def test_row_gather_rates(C):
    l2 = C.measure_row_gather(128, 32 << 20)       # fits in L2
    hbm = C.measure_row_gather(128, 1 << 30)       # four times larger than any L2
    small = C.measure_row_gather(4, 32 << 20)
    for v in (l2, hbm, small):
        assert 1e10 < v < 1e14  # 10 GB/s .. 100 TB/s
    assert l2 >= 0.9 * hbm
    # a 4-byte read still moves a whole sector: far fewer useful bytes per second
    assert small < l2


def test_smem_lookups(C):
    v = C.measure_smem_lookups()
    assert 1e10 < v < 1e14


def test_measure_rejects_bad_arguments(C):
    with pytest.raises(C.CagraError, match="row_bytes"):
        C.measure_row_gather(64, 1 << 20)
    with pytest.raises(C.CagraError, match="table_bytes"):
        C.measure_row_gather(128, 128)
    with pytest.raises(C.CagraError, match="table_bytes"):
        C.measure_row_gather(4, 9 << 30)
