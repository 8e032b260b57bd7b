"""Failure detection on the GPU, made without faulting it: a non-finite input
must come back as NTU_ENUMERIC, and a device-side rendezvous that nothing
completes must give up after its poll budget and come back as NTU_ETIMEOUT.
In both cases the context stays usable and the next call is correct.

No wait here is unbounded and no kernel traps: the non-finite value is put
into the input on the host, and the rendezvous is made unreachable through
ntu_inject_wait_timeout (its target is one arrival more than the CTAs of an
item make), with a budget of a few thousand polls.
"""
import re

import numpy as np
import pytest

from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _pair(a, b):
    return np.einsum("plurn,qrvwx->plunqvwx", a, b)


@pytest.mark.parametrize("precision", [0, 2])
def test_non_finite_input_raises_numeric_and_context_recovers(precision):
    """Item 0 of a two-item batch carries a NaN: the call returns
    NTU_ENUMERIC; item 1, computed by its own CTAs, is still the oracle's;
    the next call on the same context with finite inputs succeeds."""
    from paper_2107_06635_gb300 import ntu
    D, n = 4, 2
    kmax = 15 if precision == 0 else 8
    Ta, Tb, G = I.batch_items(61, n, 2, D, I.zz_gate(0.01))
    bad = Ta.copy()
    bad[0, 1, 0, 1, 0, 1] = np.nan
    ctx = ntu.Context(D, 2, 1, 2, 10, precision, 4, kmax, n)
    with pytest.raises(ntu.NTUError) as e:
        ctx.batch_update_host(bad, Tb, G)
    assert e.value.status == 4, str(e.value)
    # a second NaN in the other operand position: the site tensor B
    badb = Tb.copy()
    badb[1, 0, 1, 1, 1, 0] = np.inf
    with pytest.raises(ntu.NTUError) as e:
        ctx.batch_update_host(Ta, badb, G)
    assert e.value.status == 4
    a, b, info = ctx.batch_update_host(Ta, Tb, G)
    cfg = O.Config(D=D, r=2, sweeps=10, tau_exponents=tuple(range(4, kmax + 1)))
    for i in range(n):
        A2, B2, ref = O.bond_update(Ta[i], Tb[i], G[i], cfg)
        if precision == 0:
            assert _rel(a[i], A2) < 1e-9 and abs(info[i, 1] - ref.delta) < 1e-8
        else:
            assert _rel(_pair(a[i], b[i]), _pair(A2, B2)) < 1e-4
    ctx.close()


def test_nan_item_does_not_touch_its_neighbours():
    """Per-item isolation: with a NaN in item 0, item 1's outputs (written
    before the status is read) equal those of a clean call bit for bit."""
    from paper_2107_06635_gb300 import ntu
    D, n = 3, 2
    Ta, Tb, G = I.batch_items(62, n, 2, D, I.zz_gate(0.02))
    ctx = ntu.Context(D, 2, 1, 2, 10, 0, 4, 15, n)
    a0, b0, i0 = ctx.batch_update_host(Ta, Tb, G)
    bad = Ta.copy()
    bad[0].flat[7] = np.nan
    ta, tb, gg = (torch.from_numpy(x).cuda() for x in (bad, Tb, G))
    oa, ob = torch.empty_like(ta), torch.empty_like(tb)
    info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    ctx.batch_update_dev(n, ta, tb, gg, oa, ob, info)
    with pytest.raises(ntu.NTUError) as e:
        ctx.sync()
    assert e.value.status == 4
    assert np.array_equal(oa[1].cpu().numpy(), a0[1])
    assert np.array_equal(ob[1].cpu().numpy(), b0[1])
    assert np.array_equal(info[1].cpu().numpy(), i0[1])
    ctx.sync()                                   # the status word was cleared
    ctx.close()


def test_rendezvous_that_never_completes_times_out():
    """A small split-BF16 batch (3 items, D=4, r=4) runs each item's ALS on a
    cluster of CTAs that meet at a rendezvous on a global counter.  With the
    rendezvous made unreachable and a budget of 4096 polls, every wait gives
    up, the call returns NTU_ETIMEOUT, and after switching the hook off the
    same context and a fresh one both give the correct update again."""
    from paper_2107_06635_gb300 import ntu
    n = 3
    rng = np.random.default_rng(63)
    Ta = np.stack([I.random_site_tensor(rng, 2, 4) for _ in range(n)])
    Tb = np.stack([I.random_site_tensor(rng, 2, 4) for _ in range(n)])
    G = np.stack([I.heisenberg_gate(0.01)] * n)
    ctx = ntu.Context(4, 2, 1, 4, 10, ntu.NTU_MIXED_BF16X3, 4, 8, n, wait_budget=4096)
    ref_a, ref_b, ref_i = ctx.batch_update_host(Ta, Tb, G)
    ctx.inject_wait_timeout(True)
    with pytest.raises(ntu.NTUError) as e:
        ctx.batch_update_host(Ta, Tb, G)
    assert e.value.status == 5, str(e.value)
    bits = int(re.search(r"reason bits 0x([0-9a-f]+)", str(e.value)).group(1), 16)
    assert bits & 64, str(e.value)              # 64: the ALS rendezvous ran out
    ctx.inject_wait_timeout(False)
    a, b, info = ctx.batch_update_host(Ta, Tb, G)
    assert np.array_equal(a, ref_a) and np.array_equal(b, ref_b) and np.array_equal(info, ref_i)
    ctx.close()
    fresh = ntu.Context(4, 2, 1, 4, 10, ntu.NTU_MIXED_BF16X3, 4, 8, n)
    a2, b2, i2 = fresh.batch_update_host(Ta, Tb, G)
    assert np.array_equal(a2, ref_a) and np.array_equal(i2, ref_i)
    cfg = O.Config(D=4, r=4, tau_exponents=tuple(range(4, 9)))
    A2, B2, inf = O.bond_update(Ta[0], Tb[0], G[0], cfg)
    assert abs(i2[0, 1] - inf.delta) <= 1e-2 * inf.delta
    fresh.close()


def test_timeout_hook_refused_without_a_rendezvous():
    """An FP64 context (one CTA per item, no rendezvous) refuses the hook."""
    from paper_2107_06635_gb300 import ntu
    ctx = ntu.Context(3, 2, 1, 2, 10, 0, 4, 15, 2)
    with pytest.raises(ntu.NTUError) as e:
        ctx.inject_wait_timeout(True)
    assert e.value.status == 6
    ctx.close()
