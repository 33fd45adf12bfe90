"""The FMA throughput probe (vt_probe_fma) against the unit-count peak."""
import pytest
import torch

import paper_2412_04514_gb300 as vt

pytestmark = pytest.mark.gpu


def test_fma_probe_is_consistent_with_the_unit_counts():
    props = torch.cuda.get_device_properties(0)
    f32 = vt.probe_fma("fp32")
    f64 = vt.probe_fma("fp64")
    # 128 float32 lanes per SM, 2 flops per FMA, at most ~2.1 GHz
    upper = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.4 * upper < f32 < upper
    assert 0.0 < f64 < f32
    with pytest.raises(vt._lib.VtError):
        vt._lib.check(vt._lib.load().vt_probe_fma(7, None, None))
