"""Pins of the real Hermitian iPEPO form of thermal states (Sec. IV) as fed
to the oracle: the operator-basis superoperators of the Trotter gates, exact
closed forms at D=1 and D=2, and that the parametrisation stays real.

rho(beta/2) is an iPEPO whose site tensors carry a d^2 = 4 index over the
Hermitian basis O^a = sigma_x, sigma_y, sigma_z, 1 with real coefficients;
a gate G acts as rho -> G rho G^dag, i.e. on the coefficients through the
real tensor G^{ab}_{a'b'} (Sec. IV).  The NTU then runs on the coefficient
iPEPS as on any state with d = 4.
"""
import numpy as np
import pytest

from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I


def _coeffs_two_site(rho):
    Ob = I.operator_basis()
    return np.array([[np.trace(np.kron(Ob[a], Ob[b]) @ rho) / 4 for b in range(4)]
                     for a in range(4)])


def _matrix_two_site(c):
    Ob = I.operator_basis()
    return sum(c[a, b] * np.kron(Ob[a], Ob[b]) for a in range(4) for b in range(4))


def test_superoperators_act_as_conjugation():
    """S applied to the coefficients of a random two-site Hermitian rho gives
    the coefficients of G rho G^dag (written as 4 x 4 matrix products), and
    they are real; likewise the single-site s for U O U^dag."""
    rng = np.random.default_rng(1)
    m = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    rho = m + m.conj().T
    G = np.eye(4) + np.tanh(0.3) * np.kron(I.pauli("Z"), I.pauli("Z"))
    S = I.superoperator_two_site(G)
    c = _coeffs_two_site(rho)
    assert np.abs(c.imag).max() < 1e-15
    c2 = np.einsum("xyab,ab->xy", S, c)
    assert np.abs(S.imag).max() == 0
    assert np.linalg.norm(_matrix_two_site(c2) - G @ rho @ G.conj().T) < 1e-13
    U = I.x_rotation_imag(0.2)
    s = I.superoperator_one_site(U)
    Ob = I.operator_basis()
    a = rng.standard_normal(4)
    one = sum(a[k] * Ob[k] for k in range(4))
    b = s @ a
    assert np.linalg.norm(sum(b[k] * Ob[k] for k in range(4)) - U @ one @ U.conj().T) < 1e-14


def test_observable_matrix_gives_the_thermal_average():
    """For a single site rho(beta/2) = sum_a c_a O^a (c real), the estimator's
    quadratic form c^T M c / c^T c equals Tr(rho^2 O) / Tr(rho^2)."""
    rng = np.random.default_rng(2)
    c = rng.standard_normal(4)
    rho = sum(c[k] * I.operator_basis()[k] for k in range(4))
    for name in ("X", "Y", "Z"):
        Op = I.pauli(name)
        M = I.ipepo_observable(Op)
        got = (c @ M @ c).real / (c @ c)
        ref = np.trace(rho @ rho @ Op).real / np.trace(rho @ rho).real
        assert abs(got - ref) < 1e-14


def test_ipepo_field_only_is_exact_at_d1():
    """H = -h sum X (identity bond gates), D = 1: every Trotter step is exact
    and <sigma_x>(beta) = tanh(beta h); <sigma_z> = 0."""
    h, db = 0.7, 0.05
    _, s1 = I.ipepo_thermal_gates(h, db)
    ident = I.identity_gate(4)
    cfg = O.Config(D=1, d=4, r=1, sweeps=2)
    A = B = I.ipepo_identity(1)
    Mx, Mz = I.ipepo_observable(I.pauli("X")), I.ipepo_observable(I.pauli("Z"))
    for step in range(1, 11):
        A, B, deltas = O.ntu_step(A, B, [ident] * 4, s1, cfg)
        beta = step * db
        assert abs(O.measure(A, B, 0, Mx, 1).real - np.tanh(beta * h)) < 1e-12
        assert abs(O.measure(A, B, 1, Mz, 1)) < 1e-14
        assert max(deltas) < 1e-14


def test_ipepo_classical_ising_is_exact_at_d2():
    """h = 0: rho(beta/2) = prod_bonds (cosh(beta/2) + sinh(beta/2) Z Z) has
    bond dimension 2 in the operator basis, so every NTU bond update at D=2
    with rank r=4 gates is exact (delta <= 1e-12), the coefficients stay real
    and only O^a in {sigma_z, 1} appear on the physical index (sigma_x and
    sigma_y only at rounding level: the QR completion of the rank-deficient
    padded start carries rounding noise, which the small kept singular value
    tanh(dbeta/4)^2 ~ 6e-4 amplifies to ~3e-8 of the largest entry)."""
    gates2, _ = I.ipepo_thermal_gates(0.0, 0.1)
    cfg = O.Config(D=2, d=4, r=4, sweeps=4)
    A = B = I.ipepo_identity(2)
    for _ in range(3):
        A, B, deltas = O.ntu_step(A, B, gates2, None, cfg)
        assert max(deltas) <= 1e-12
        for T in (A, B):
            assert np.abs(T.imag).max() < 1e-14 * np.abs(T).max()
            assert np.abs(T[:2]).max() < 1e-6 * np.abs(T).max()     # no sigma_x, sigma_y


@pytest.mark.parametrize("D", [2, 3])
def test_ipepo_ntu_stays_real(D):
    """The NTU of a real iPEPO with real gates keeps the tensors real (the
    Hermitian parametrisation of Sec. IV): three steps at h = 2.5 from the
    seeded start, imaginary parts below 1e-13 of the largest entry."""
    gates2, s1 = I.ipepo_thermal_gates(2.5, 0.05)
    cfg = O.Config(D=D, d=4, r=4, sweeps=4)
    A, B = I.ipepo_start(D)
    for _ in range(3):
        A, B, _ = O.ntu_step(A, B, gates2, s1, cfg)
        for T in (A, B):
            assert np.abs(T.imag).max() < 1e-13 * np.abs(T).max()
