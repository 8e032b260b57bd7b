"""Pins of the oracle's simple update (SU, Sec. II) against what the paper
fixes: its metric g_SU = 1_d (x) 1_d (x) prod_j lambda_j over the six outer
bonds, and its place in the SVDU < SU hierarchy.

* The SU result minimises the error in the metric g_SU: alternating least
  squares (Fig. 5) with the explicit separable metric built from the
  unweighted isometries reaches the same two-site tensor and the same
  relative error.
* The schematic form: the full two-site tensor of each of the four bonds,
  written out leg by leg with the outer legs weighted by lambda, gated and
  truncated by one SVD, equals the SU pair (Fig. 1(b,c) with the SU metric).
* With every lambda = 1, g_SU is the Frobenius norm and SU is the SVDU.
"""
import numpy as np
import pytest

from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I

LEGS = {0: (3, 1), 1: (2, 4), 2: (1, 3), 3: (4, 2)}   # axes of bond b on A and on B


def _lams(rng, D):
    """Four random bond tensors: distinct positive values, descending."""
    return [np.sort(rng.uniform(0.2, 1.0, D))[::-1].copy() for _ in range(4)]


def _weight_outer(T, lam, site, bond, power):
    """Multiply the three outer legs of T (site 'A' or 'B') by lambda ** power,
    written leg by leg from the bond table (independent of su_weight)."""
    bonds = {"A": {1: 2, 2: 1, 3: 0, 4: 3}, "B": {1: 0, 2: 3, 3: 2, 4: 1}}[site]
    T = T.copy()
    for axis, b in bonds.items():
        if b == bond:
            continue
        shape = [1] * 5
        shape[axis] = lam[b].size
        T = T * (lam[b] ** power).reshape(shape)
    return T


def _pair(A, B, bond):
    """The two-site tensor contracted over the legs of `bond`, as a matrix
    with rows (p_A, A's outer legs) and columns (p_B, B's outer legs)."""
    ja, jb = LEGS[bond]
    a = np.moveaxis(A, ja, -1)
    b = np.moveaxis(B, jb, -1)
    m = np.tensordot(a, b, axes=([4], [4]))          # [p, o, o, o, q, o, o, o]
    n = a.shape[0] * a.shape[1] ** 3
    return m.reshape(n, n)


def _schematic_su(A, B, lam, bond, G, D):
    """Fig. 1(b,c) with the SU metric: weight the outer legs by sqrt(lambda)
    (the symmetric-gauge tensors already carry the other sqrt(lambda)),
    contract the pair over the bond, apply the gate, SVD, keep D."""
    Aw = _weight_outer(A, lam, "A", bond, 0.5)
    Bw = _weight_outer(B, lam, "B", bond, 0.5)
    d_p, Dd = A.shape[0], A.shape[1]
    P = _pair(Aw, Bw, bond).reshape(d_p, Dd ** 3, d_p, Dd ** 3)
    Th = np.einsum("abst,sitj->aibj", G, P).reshape(d_p * Dd ** 3, d_p * Dd ** 3)
    U, s, Vh = np.linalg.svd(Th)
    return (U[:, :D] * s[:D]) @ Vh[:D], s


@pytest.mark.parametrize("bond", [0, 1, 2, 3])
def test_su_equals_the_schematic_weighted_truncation(bond):
    rng = np.random.default_rng(70 + bond)
    D = 2
    A, B = I.random_pair(71 + bond, 2, D)
    lam = _lams(rng, D)
    G = I.random_gate(rng)
    cfg = O.Config(D=D, r=4)
    A2, B2, lam2, delta = O.su_update_bond(A, B, lam, bond, G, cfg)
    ref, s = _schematic_su(A, B, lam, bond, G, D)
    got = _pair(_weight_outer(A2, lam, "A", bond, 0.5), _weight_outer(B2, lam, "B", bond, 0.5),
                bond)
    got = got / np.linalg.norm(got)
    ph = np.vdot(got.reshape(-1), ref.reshape(-1))
    assert np.linalg.norm(got * ph / abs(ph) - ref / np.linalg.norm(ref)) < 1e-12
    assert abs(delta - np.sum(s[D:] ** 2) / np.sum(s ** 2)) < 1e-13
    assert np.allclose(lam2[bond], s[:D] / np.linalg.norm(s[:D]), rtol=1e-12)
    for b in range(4):
        if b != bond:
            assert np.array_equal(lam2[b], lam[b])


def test_su_minimises_the_error_in_g_su():
    """Bond 0: the metric g_SU in the reduced space of the unweighted QR is
    separable, g_L (x) g_R with g_L = Q_A^H W_A Q_A (W_A the product of the
    lambdas on A's outer legs, per row of Q_A) and likewise g_R.  ALS with
    that explicit metric, from the SVDU start, converges to the SU pair and
    to the SU error delta."""
    rng = np.random.default_rng(80)
    D, r = 3, 2
    A, B = I.random_pair(81, 2, D)
    lam = _lams(rng, D)
    G = I.random_gate(rng)
    cfg = O.Config(D=D, r=r)
    A2, B2, _, delta = O.su_update_bond(A, B, lam, 0, G, cfg)
    GA, GB = O.gate_split(G, r)
    QA, RA = O.qr_positive(O.gated_matrix(A, GA, 1, "left"))
    QB, RB = O.qr_positive(O.gated_matrix(B, GB, 1, "right"))
    ones = np.ones(2)
    # rows (p, e, u, dn): A's e = l (bond 2), u (bond 1), dn (bond 3);
    # B's e = r (bond 2), u (bond 3), dn (bond 1)
    wA = np.einsum("p,e,u,n->peun", ones, lam[2], lam[1], lam[3]).reshape(-1)
    wB = np.einsum("p,e,u,n->peun", ones, lam[2], lam[3], lam[1]).reshape(-1)
    gL = QA.conj().T @ (wA[:, None] * QA)
    gR = QB.conj().T @ (wB[:, None] * QB)
    g = np.kron(gL, gR)
    MA, MB, eps, d_als, eps0, _ = O.als_truncate(g, RA, RB, D, 200, cfg.taus)
    Aa = O.recompose(QA, MA, 2, D, "left")
    Ba = O.recompose(QB, MB, 2, D, "right")
    p1 = _pair(A2, B2, 0)
    p2 = _pair(Aa, Ba, 0)
    p1, p2 = p1 / np.linalg.norm(p1), p2 / np.linalg.norm(p2)
    ph = np.vdot(p1.reshape(-1), p2.reshape(-1))
    assert np.linalg.norm(p1 * ph / abs(ph) - p2) < 1e-8
    assert abs(d_als - delta) < 1e-10 * delta


def test_su_with_unit_lambdas_is_the_svdu():
    """All lambda = 1: g_SU is the Frobenius norm, so the SU state equals the
    zero-sweep NTU update (the SVDU of Fig. 2(c,d)), and lambda_bond becomes
    the normalised singular values of R_A R_B^T."""
    D = 3
    A, B = I.random_pair(91, 2, D)
    G = I.random_gate(np.random.default_rng(92))
    lam = [np.ones(D) for _ in range(4)]
    cfg = O.Config(D=D, r=2, sweeps=0)
    for bond in range(4):
        A2, B2, lam2, _ = O.su_update_bond(A, B, lam, bond, G, cfg)
        A3, B3, _ = O.update_bond(A, B, bond, G, cfg)
        assert np.linalg.norm(A2 - A3) < 1e-12 and np.linalg.norm(B2 - B3) < 1e-12


def test_su_pins_catch_planted_mistakes(monkeypatch):
    """Full lambda instead of sqrt(lambda) on the outer legs, or the bond
    leg weighted too, breaks the schematic pin."""
    rng = np.random.default_rng(70)
    D = 2
    A, B = I.random_pair(71, 2, D)
    lam = _lams(rng, D)
    G = I.random_gate(rng)
    cfg = O.Config(D=D, r=4)
    ref, _ = _schematic_su(A, B, lam, 0, G, D)
    ref = ref / np.linalg.norm(ref)
    orig = O.su_weight

    def check(fake):
        monkeypatch.setattr(O, "su_weight", fake)
        A2, B2, _, _ = O.su_update_bond(A, B, lam, 0, G, cfg)
        monkeypatch.setattr(O, "su_weight", orig)
        got = _pair(_weight_outer(A2, lam, "A", 0, 0.5), _weight_outer(B2, lam, "B", 0, 0.5), 0)
        got = got / np.linalg.norm(got)
        ph = np.vdot(got.reshape(-1), ref.reshape(-1))
        return np.linalg.norm(got * ph / abs(ph) - ref)

    assert check(lambda T, l, bonds, skip, p: orig(T, l, bonds, skip, 2 * p)) > 1e-3
    assert check(lambda T, l, bonds, skip, p: orig(T, l, bonds, -1, p)) > 1e-3


def test_su_step_product_state_single_site_exact():
    """D=1, identity bond gates, field h (as P7): the SU step is exact and
    <sigma_z>(t) = cos(2 h t); the bond tensors stay 1."""
    h, dt = 0.7, 0.05
    cfg = O.Config(D=1, r=1)
    A = B = I.plus_z_state(1)
    lam = [np.ones(1) for _ in range(4)]
    for step in range(1, 11):
        A, B, lam, deltas = O.su_step(A, B, lam, [I.identity_gate()] * 4,
                                      I.x_rotation(h * dt / 2), cfg)
        assert abs(O.measure(A, B, 0, I.pauli("Z"), 1) - np.cos(2 * h * step * dt)) < 1e-12
        assert max(deltas) < 1e-14 and all(abs(l[0] - 1) < 1e-15 for l in lam)
