"""GPU runs of the real Hermitian iPEPO form of thermal states (Sec. IV):
the coefficient iPEPS (d^2 = 4 index over sigma_x, sigma_y, sigma_z, 1) with
the superoperator Trotter gates of rank 4, through the same C ABI as any
state with d = 4; against the oracle and against closed forms."""
import numpy as np
import pytest

from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_ipepo_field_only_exact_at_d1():
    """D = 1, identity bond gates, h = 0.7: <sigma_x>(beta) = tanh(beta h)."""
    from paper_2107_06635_gb300 import ntu
    h, db = 0.7, 0.05
    _, s1 = I.ipepo_thermal_gates(h, db)
    ctx = ntu.Context(1, 4, 1, 1, 2, 0, 4, 15, 1)
    ctx.set_state(I.ipepo_identity(1), I.ipepo_identity(1))
    Mx = I.ipepo_observable(I.pauli("X"))
    for step in range(1, 11):
        deltas = ctx.step([I.identity_gate(4)] * 4, s1)
        assert abs(ctx.measure(0, Mx).real - np.tanh(step * db * h)) < 1e-12
        assert np.all(deltas < 1e-14)
    ctx.close()


@pytest.mark.parametrize("D,precision,tol", [(3, 0, 1e-9), (4, 0, 1e-9), (4, 2, 1e-4)])
def test_ipepo_thermal_steps_match_oracle(D, precision, tol):
    """h = 2.5, dbeta = 0.005 from the seeded iPEPO start: per step
    <sigma_x>, <sigma_z> of both sites against the oracle (FP64 context
    1e-9; split-BF16 context 1e-4), and the tensors stay real to rounding."""
    from paper_2107_06635_gb300 import ntu
    gates2, s1 = I.ipepo_thermal_gates(2.5, 0.005)
    kmax = 15 if precision == 0 else 8
    cfg = O.Config(D=D, d=4, r=4, sweeps=10, tau_exponents=tuple(range(4, kmax + 1)))
    A, B = I.ipepo_start(D)
    ctx = ntu.Context(D, 4, 1, 4, 10, precision, 4, kmax, 1)
    ctx.set_state(A, B)
    Mx, Mz = I.ipepo_observable(I.pauli("X")), I.ipepo_observable(I.pauli("Z"))
    for _ in range(3):
        ctx.step(gates2, s1)
        A, B, _ = O.ntu_step(A, B, gates2, s1, cfg)
        for site in (0, 1):
            for M in (Mx, Mz):
                assert abs(ctx.measure(site, M) - O.measure(A, B, site, M, 1)) < tol
        Ag, Bg = ctx.get_state()
        for T in (Ag, Bg):
            assert np.abs(T.imag).max() < 1e-12 * np.abs(T).max()
    ctx.close()
