"""A host-buffer batch of at least 6 x SMs items runs as two halves whose
copies overlap the other half's compute (ntu_batch_update_host).  Each half
keeps full ALS waves and the same kernels, so the outputs equal those of the
device-pointer call on the whole batch, bit for bit."""
import numpy as np
import pytest

from paper_2107_06635_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_host_halves_equal_one_device_launch():
    from paper_2107_06635_gb300 import ntu
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n, D = 6 * sms, 4
    Ta, Tb, G = I.batch_items(31, n, 2, D, I.zz_gate(0.01))
    ctx = ntu.Context(D, 2, 1, 2, 6, ntu.NTU_MIXED_BF16X3, 4, 8, n)
    a_h, b_h, i_h = ctx.batch_update_host(Ta, Tb, G)
    ta, tb, g = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (Ta, Tb, G))
    a_d, b_d = torch.empty_like(ta), torch.empty_like(tb)
    info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    ctx.batch_update_dev(n, ta, tb, g, a_d, b_d, info)
    ctx.sync()
    assert np.array_equal(a_h, a_d.cpu().numpy())
    assert np.array_equal(b_h, b_d.cpu().numpy())
    assert np.array_equal(i_h, info.cpu().numpy())
    # a second call on the same context (the copy stream exists by now)
    a2, b2, i2 = ctx.batch_update_host(Ta[::-1].copy(), Tb[::-1].copy(), G[::-1].copy())
    assert np.array_equal(a2, a_h[::-1]) and np.array_equal(i2, i_h[::-1])
    ctx.close()
