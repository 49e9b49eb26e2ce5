"""The L2 reduction-rate calibration (inpc_l2_reduction_rate), which the
benchmark reports beside the grid adjoint's own reduction rate: every
reduction lands in the caller's region (the region's sum is exactly the
number of lane reductions times 4), and the rates are finite and positive."""
import pytest
import torch

from paper_2403_16862_gb300 import _binding as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("paired", [False, True])
def test_l2_reduction_rate(gpu, paired):
    rows = 1 << 16
    buf = torch.zeros(rows, 4, dtype=torch.float32, device=gpu)
    stream = torch.cuda.current_stream().cuda_stream
    gops = B.inpc_l2_reduction_rate(buf.data_ptr(), rows, paired, stream)
    torch.cuda.synchronize()
    assert 1.0 < gops < 1e5
    # 8 CTAs of 256 threads per SM, 128 reductions each, 2 warm-up + 5 timed
    # launches; each row holds an integer count below 2^24, exact in FP32
    sms = torch.cuda.get_device_properties(gpu).multi_processor_count
    lanes = sms * 8 * 256 * 128 * 7
    assert float(buf.double().sum()) == 4.0 * lanes
    assert float(buf.max()) < 2 ** 24
