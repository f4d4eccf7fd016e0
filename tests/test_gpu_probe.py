"""The tensor-core peak probe (dgfs_probe_mma_rate) that gives the roofline
its measured denominator: it runs, its bounded wait does not expire, and the
rates are in the range of the GPU's tensor pipe (BF16 about twice TF32)."""
import pytest

from paper_1903_04670_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_probe_rates():
    tf32 = B.dgfs_probe_mma_rate(0, "tf32", 4096)
    bf16 = B.dgfs_probe_mma_rate(0, "bf16", 4096)
    print("tcgen05 probe: tf32 %.1f TFLOP/s, bf16 %.1f TFLOP/s" % (tf32, bf16))
    assert 200.0 < tf32 < 3000.0
    assert 1.5 < bf16 / tf32 < 2.5


def test_probe_rejects_bad_arguments():
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_probe_mma_rate(0, 2, 4096)
    assert e.value.status == 1
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_probe_mma_rate(0, "tf32", 10)
    assert e.value.status == 1
