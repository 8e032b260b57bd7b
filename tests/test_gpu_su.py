"""GPU parity of the simple update (SU, Sec. II) of the two-site cell
against the oracle, through the C ABI: bond tensors lambda, the updated
site tensors and the SU error delta after every bond update, and whole
Trotter steps."""
import numpy as np
import pytest

from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _lams(rng, D):
    return [np.sort(rng.uniform(0.2, 1.0, D))[::-1].copy() for _ in range(4)]


@pytest.mark.parametrize("D,precision", [(3, 0), (5, 0), (4, 2)])
def test_su_bond_updates_match_oracle(D, precision):
    """Each of the four bonds in turn, a different site-asymmetric gate on
    each, random bond tensors: A', B' within 1e-10, lambda within 1e-12 and
    delta within 1e-12 of the oracle (the SU needs no environment; on the
    split-BF16 context its QR runs as double-FP32 CholeskyQR2)."""
    from paper_2107_06635_gb300 import ntu
    rng = np.random.default_rng(300 + D)
    A, B = I.random_pair(301 + D, 2, D)
    lam = _lams(rng, D)
    gates = [I.random_gate(rng) for _ in range(4)]
    ctx = ntu.Context(D, 2, 1, 2, 10, precision, 4, 15 if precision == 0 else 8, 1)
    ctx.set_state(A, B)
    ctx.su_set_lambdas(np.stack(lam))
    cfg = O.Config(D=D, r=2)
    for b in range(4):
        delta = ctx.su_update(b, gates[b])
        A, B, lam, dref = O.su_update_bond(A, B, lam, b, gates[b], cfg)
        Ag, Bg = ctx.get_state()
        tol = 1e-10 if precision == 0 else 1e-9
        assert _rel(Ag, A) < tol and _rel(Bg, B) < tol, b
        assert np.abs(ctx.su_get_lambdas() - np.stack(lam)).max() < 1e-12, b
        assert abs(delta - dref) < 1e-12, b
    ctx.close()


def test_su_step_trajectory_matches_oracle():
    """Three SU Trotter steps of the TFIM quench (h = 2.5, dt = 0.01, D = 4,
    the seeded start): <sigma_x> of both sites within 1e-9, lambda within
    1e-10 and delta per bond within 1e-12 of the oracle's SU step."""
    from paper_2107_06635_gb300 import ntu
    D = 4
    gates2, gate1 = I.tfim_real_time_gates(2.5, 0.01)
    A, B = I.quench_start(D)
    lam = [np.ones(D) for _ in range(4)]
    ctx = ntu.Context(D, 2, 1, 2, 10, 0, 4, 15, 1)
    ctx.set_state(A, B)
    cfg = O.Config(D=D, r=2)
    for _ in range(3):
        deltas = ctx.su_step(gates2, gate1)
        A, B, lam, dref = O.su_step(A, B, lam, gates2, gate1, cfg)
        assert np.abs(deltas - np.array(dref)).max() < 1e-12
        assert np.abs(ctx.su_get_lambdas() - np.stack(lam)).max() < 1e-10
        for site in (0, 1):
            assert abs(ctx.measure(site, I.pauli("X")) - O.measure(A, B, site, I.pauli("X"), 1)) < 1e-9
    ctx.close()


def test_su_rejects_bad_lambdas_and_bonds():
    from paper_2107_06635_gb300 import ntu
    ctx = ntu.Context(3, 2, 1, 2, 10, 0, 4, 15, 1)
    lam = np.ones((4, 3))
    lam[1, 2] = -1.0
    with pytest.raises(ntu.NTUError) as e:
        ctx.su_set_lambdas(lam)
    assert e.value.status == 1
    lam[1, 2] = np.nan
    with pytest.raises(ntu.NTUError):
        ctx.su_set_lambdas(lam)
    with pytest.raises(ntu.NTUError):
        ctx.su_update(4, I.zz_gate(0.1))
    assert np.array_equal(ctx.su_get_lambdas(), np.ones((4, 3)))     # unchanged, init value
    ctx.close()
