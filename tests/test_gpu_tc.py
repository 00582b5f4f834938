"""The tcgen05 BF16 GEMM building block against a plain FP32 product of the
same BF16 values."""
import numpy as np
import pytest

import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,k", [(128, 16), (256, 64), (384, 288), (128, 512)])
def test_tc_gemm_matches_fp32_reference(m, k):
    import torch
    g = torch.Generator().manual_seed(m + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(32, k, generator=g).to(torch.bfloat16)
    ref = a.float() @ b.float().T
    da, db = a.cuda(), b.cuda()
    d = torch.full((m, 32), float("nan"), device="cuda")
    L.ac_tc_gemm_bf16_n32(da.data_ptr(), db.data_ptr(), d.data_ptr(), m, k,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_allclose(d.cpu().numpy(), ref.numpy(), rtol=1e-4, atol=1e-4)


def test_tc_gemm_rejects_bad_shapes():
    with pytest.raises(ac.AcError):
        L.ac_tc_gemm_bf16_n32(16, 16, 16, 100, 16, 0)
