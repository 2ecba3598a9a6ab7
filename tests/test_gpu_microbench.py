"""GPU: the measurement aids behind the rooflines -- the FMA rate of the FP64 and FP32 pipes and
the latency of one grid-barrier round and one cluster candidate exchange (with and without a
pivot column).  Checked for sane, finite values and the expected ordering, not for speed."""

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fma_rates(skel, dev):
    f64 = skel.debug_fma_rate(True, iters=1 << 12)
    f32 = skel.debug_fma_rate(False, iters=1 << 14)
    assert 0.05 < f64 < 200.0
    assert 1.0 < f32 < 500.0
    assert f32 > f64          # the FP32 pipes are far wider than FP64's on this part


def test_grid_barrier_round(skel, dev):
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ns = skel.debug_exchange_latency(0, sms, steps=500)
    assert 50.0 < ns < 1e5


@pytest.mark.parametrize("ctas,col_words", [(8, 0), (16, 0), (16, 24)])
def test_cluster_exchange_round(skel, dev, ctas, col_words):
    try:
        ns = skel.debug_exchange_latency(1, ctas, steps=2000, col_words=col_words)
    except skel.SkelError as e:
        if e.code == 7 and ctas == 16:      # 16-CTA clusters not offered by this device
            pytest.skip("non-portable cluster size unavailable")
        raise
    assert 20.0 < ns < 1e5
