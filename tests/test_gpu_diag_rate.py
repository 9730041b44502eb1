"""The FP32 FMA-rate diagnostic (the measured peak the FP32 direct form's roofline divides by): it
must report a rate that the SMs can reach. An FMA chain folded away by the compiler would show as
a rate far above SMs x 128 lanes x 2 flop x the clock ceiling; a stalled kernel as one far below."""

import pytest

torch = pytest.importorskip("torch")

import paper_1008_4370_gb300 as nb  # noqa: E402
from paper_1008_4370_gb300 import build as nbuild  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    nbuild.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("packed", [0, 1])
def test_fp32_rate_is_plausible(dev, packed):
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ceiling = sms * 128 * 2 * 2.2e9 / 1e12 * (2 if packed else 1)  # 2.2 GHz: above any clock seen
    t, ms = nb.nbfd_diag_fp32_rate(packed, 4, 1 << 18)
    print(f"packed={packed}: {t:.1f} TFLOP/s in {ms:.2f} ms")
    assert 0.2 * sms * 128 * 2 * 1.0e9 / 1e12 < t < ceiling
    with pytest.raises(nb.NbfdError):
        nb.nbfd_diag_fp32_rate(packed, 0, 1)
