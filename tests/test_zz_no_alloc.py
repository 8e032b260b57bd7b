"""The allocation-free gate+QR entry point, for callers that cannot call
cudaMalloc (a framework that owns all device memory through its own pool,
or code that must not trigger the synchronisation of cudaMalloc/cudaFree).

ntu_gate_qr_noalloc keeps its scratch in a fixed device array instead of a
context's work space; its outputs must equal those of the context entry
point ntu_batch_gate_qr_dev on the same inputs, on consecutive calls (the
array keeps the previous call's contents).  This file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2107_06635_gb300 import inputs as I
from paper_2107_06635_gb300 import ntu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_gate_qr_matches_context_entry_point():
    lib = ntu.load()
    # two calls in a row, then the largest configuration the 4 MiB array
    # takes (D=8, r=4: 2.1 MB of scratch)
    cases = [(4, 2, 1, 2, 11), (3, 2, 2, 4, 12), (8, 2, 1, 4, 13)]
    for D, d, d_anc, r, seed in cases:
        rng = np.random.default_rng(seed)
        d_p, K = d * d_anc, D * r
        m = d_p * D ** 3
        Ta = I.random_site_tensor(rng, d_p, D)[None]
        Tb = I.random_site_tensor(rng, d_p, D)[None]
        G = I.random_gate(rng)[None]
        # reference: the context entry point
        ctx = ntu.Context(D, d, d_anc, r, 2, ntu.NTU_FP64, 4, 15, 1)
        ref = [torch.empty(s, dtype=torch.complex128, device="cuda")
               for s in ((1, m, K), (1, K, K), (1, m, K), (1, K, K))]
        ctx.batch_gate_qr_dev(1, _dev(Ta), _dev(Tb), _dev(G), *ref)
        ctx.sync()
        # allocation-free call on the same inputs
        out = [torch.full(s, float("nan"), dtype=torch.complex128, device="cuda")
               for s in ((m, K), (K, K), (m, K), (K, K))]
        ta, tb, gg = _dev(Ta[0]), _dev(Tb[0]), _dev(G[0])
        st = lib.ntu_gate_qr_noalloc(D, d, d_anc, r, ta.data_ptr(), tb.data_ptr(), gg.data_ptr(),
                                     *(o.data_ptr() for o in out), None)
        assert st == 0, lib.ntu_last_error(None)
        torch.cuda.synchronize()
        for o, rf in zip(out, ref):
            o, rf = o.cpu().numpy(), rf[0].cpu().numpy()
            assert np.all(np.isfinite(o))
            assert _rel(o, rf) < 1e-12
        ctx.close()


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    lib = ntu.load()
    buf = torch.zeros(16, dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())   # the size check rejects before any launch
    st = lib.ntu_gate_qr_noalloc(8, 4, 2, 4, p, p, p, p, p, p, p, None)
    assert st == 1
    assert b"scratch" in lib.ntu_last_error(None)
    # a gated matrix with fewer rows than columns (d_p D^2 < r) is refused too
    st = lib.ntu_gate_qr_noalloc(1, 2, 1, 4, p, p, p, p, p, p, p, None)
    assert st == 1
    assert b"unsupported" in lib.ntu_last_error(None)
