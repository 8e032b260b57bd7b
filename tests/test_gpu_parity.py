"""GPU parity of the CUDA NTU path against the CPU oracle, stage by stage and
end to end, through the C ABI.

Tolerances: FP64 path rel-Frobenius(g) <= 1e-10 (and bit-exact on small
integer inputs, where every partial sum is an exact integer), mixed FP32
environment rel(g) <= 1e-4; delta within 1e-8 of the oracle on the FP64
path and 1e-2 relative on the mixed path; <sigma_x> within 1e-6.
Gauge-dependent outputs (Q, R, g, M, A', B') are compared element by element
only on single calls with full-rank random inputs and gates with distinct
operator-Schmidt values, where QR with a positive diagonal and SVD with the
phase convention are unique.
"""
import os

import numpy as np
import pytest

from oracle import ntu_oracle as O
from paper_2107_06635_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _empty(shape):
    return torch.empty(shape, dtype=torch.complex128, device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _ctx(D, r=2, d_anc=1, sweeps=10, precision=0, max_batch=4, kmin=4, kmax=15):
    from paper_2107_06635_gb300 import ntu
    return ntu.Context(D, 2, d_anc, r, sweeps, precision, kmin, kmax, max_batch)


def _oracle_stage(Ta, Tb, G, cfg):
    GA, GB = O.gate_split(G, cfg.r)
    QA, RA = O.qr_positive(O.gated_matrix(Ta, GA, cfg.d_anc, "left"))
    QB, RB = O.qr_positive(O.gated_matrix(Tb, GB, cfg.d_anc, "right"))
    return QA, RA, QB, RB


def _items(seed, n, d_p, D):
    rng = np.random.default_rng(seed)
    Ta = np.stack([I.random_site_tensor(rng, d_p, D) for _ in range(n)])
    Tb = np.stack([I.random_site_tensor(rng, d_p, D) for _ in range(n)])
    G = np.stack([I.random_gate(rng) for _ in range(n)])
    return Ta, Tb, G


# ------------------------------------------------------------ gate + QR
@pytest.mark.parametrize("D,r,d_anc", [(2, 2, 1), (3, 2, 1), (5, 2, 1), (4, 4, 1), (3, 2, 2)])
def test_gate_qr_matches_oracle(D, r, d_anc):
    n = 3
    d_p = 2 * d_anc
    Ta, Tb, G = _items(100 + D, n, d_p, D)
    ctx = _ctx(D, r, d_anc, max_batch=n)
    m, K = d_p * D ** 3, D * r
    QA, RA, QB, RB = _empty((n, m, K)), _empty((n, K, K)), _empty((n, m, K)), _empty((n, K, K))
    ctx.batch_gate_qr_dev(n, _dev(Ta), _dev(Tb), _dev(G), QA, RA, QB, RB)
    ctx.sync()
    cfg = O.Config(D=D, r=r, d_anc=d_anc)
    for i in range(n):
        qa, ra, qb, rb = _oracle_stage(Ta[i], Tb[i], G[i], cfg)
        assert _rel(RA[i].cpu().numpy(), ra) < 1e-12
        assert _rel(RB[i].cpu().numpy(), rb) < 1e-12
        assert _rel(QA[i].cpu().numpy(), qa) < 1e-12
        assert _rel(QB[i].cpu().numpy(), qb) < 1e-12


@pytest.mark.parametrize("D,r,precision", [(3, 2, 1), (5, 2, 2), (8, 2, 2), (4, 4, 1)])
def test_gate_qr_cholesky_qr2_mixed_context(D, r, precision):
    """Mixed contexts factor the gated matrices by CholeskyQR2 in double-FP32
    arithmetic; the QR with positive real diag(R) is unique, so Q and R meet
    the oracle's Householder QR to near FP64 precision."""
    n = 3
    Ta, Tb, G = _items(120 + D, n, 2, D)
    ctx = _ctx(D, r, precision=precision, max_batch=n, kmax=8)
    m, K = 2 * D ** 3, D * r
    QA, RA, QB, RB = _empty((n, m, K)), _empty((n, K, K)), _empty((n, m, K)), _empty((n, K, K))
    ctx.solver_paths()
    ctx.batch_gate_qr_dev(n, _dev(Ta), _dev(Tb), _dev(G), QA, RA, QB, RB)
    ctx.sync()
    paths = ctx.solver_paths()
    assert paths["qr_cholesky2"] == 2 * n and paths["qr_householder"] == 0
    cfg = O.Config(D=D, r=r)
    for i in range(n):
        qa, ra, qb, rb = _oracle_stage(Ta[i], Tb[i], G[i], cfg)
        assert _rel(RA[i].cpu().numpy(), ra) < 1e-11
        assert _rel(RB[i].cpu().numpy(), rb) < 1e-11
        assert _rel(QA[i].cpu().numpy(), qa) < 1e-11
        assert _rel(QB[i].cpu().numpy(), qb) < 1e-11
        q = QA[i].cpu().numpy()
        assert np.abs(q.conj().T @ q - np.eye(K)).max() < 1e-12


def test_gate_qr_rank_deficient_falls_back_to_householder():
    """A zero-padded product state makes the gated matrices rank deficient:
    the Cholesky factorisation of M^H M fails and the mixed context hands the
    matrices to the Householder kernel, whose output is then bit-identical to
    the FP64 context's."""
    D, r, n = 3, 2, 2
    Ta = np.stack([I.plus_x_state(D), I.plus_z_state(D)])
    Tb = np.stack([I.plus_z_state(D), I.plus_x_state(D)])
    G = np.stack([I.zz_gate(0.3), I.zz_gate(0.7)])
    m, K = 2 * D ** 3, D * r
    outs = []
    for precision in (0, 2):
        ctx = _ctx(D, r, precision=precision, max_batch=n, kmax=8 if precision else 15)
        QA, RA, QB, RB = _empty((n, m, K)), _empty((n, K, K)), _empty((n, m, K)), _empty((n, K, K))
        ctx.solver_paths()
        ctx.batch_gate_qr_dev(n, _dev(Ta), _dev(Tb), _dev(G), QA, RA, QB, RB)
        ctx.sync()
        paths = ctx.solver_paths()
        assert paths["qr_householder"] == 2 * n and paths["qr_cholesky2"] == 0
        outs.append([x.cpu().numpy() for x in (QA, RA, QB, RB)])
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


# --------------------------------------------------------- environment
@pytest.mark.parametrize("D,r", [(2, 2), (3, 2), (4, 2), (5, 2), (3, 4)])
def test_env_matches_oracle_fp64(D, r):
    n = 2
    Ta, Tb, G = _items(200 + D, n, 2, D)
    cfg = O.Config(D=D, r=r)
    ctx = _ctx(D, r, max_batch=n)
    Q = [_oracle_stage(Ta[i], Tb[i], G[i], cfg) for i in range(n)]
    QA = np.stack([q[0] for q in Q])
    QB = np.stack([q[2] for q in Q])
    ng = (D * r) ** 2
    g = _empty((n, ng, ng))
    ctx.batch_env_dev(n, _dev(Ta), _dev(Tb), _dev(QA), _dev(QB), g)
    ctx.sync()
    for i in range(n):
        ref = O.metric_raw(Ta[i], Tb[i], QA[i], QB[i], 2, D)
        assert _rel(g[i].cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("D,r,dens", [(2, 2, 1.0), (3, 2, 0.3), (4, 2, 0.15), (5, 1, 0.1)])
def test_env_bit_exact_on_integer_inputs(D, r, dens):
    """Sparse small-integer tensors and isometries: contracting their
    absolute values bounds every partial sum below 2^53, so every partial sum
    is an exact integer in FP64 and any summation order gives the oracle's
    bits.  Checks the index bookkeeping of every contraction step."""
    rng = np.random.default_rng(300 + D)
    n, d_p, K = 2, 2, D * r
    m = d_p * D ** 3
    Ta = np.stack([I.sparse_integer_array(rng, (d_p, D, D, D, D), dens) for _ in range(n)])
    Tb = np.stack([I.sparse_integer_array(rng, (d_p, D, D, D, D), dens) for _ in range(n)])
    QA = np.stack([I.sparse_integer_array(rng, (m, K), dens) for _ in range(n)])
    QB = np.stack([I.sparse_integer_array(rng, (m, K), dens) for _ in range(n)])
    ctx = _ctx(D, r, max_batch=n)
    g = _empty((n, K * K, K * K))
    ctx.batch_env_dev(n, _dev(Ta), _dev(Tb), _dev(QA), _dev(QB), g)
    ctx.sync()
    ab = lambda x: (np.abs(x.real) + np.abs(x.imag)).astype(np.complex128)
    for i in range(n):
        bound = O.metric_raw(ab(Ta[i]), ab(Tb[i]), ab(QA[i]), ab(QB[i]), d_p, D)
        assert np.abs(bound).max() < 2 ** 53
        ref = O.metric_raw(Ta[i], Tb[i], QA[i], QB[i], d_p, D)
        assert np.count_nonzero(ref) > 0.9 * ref.size
        assert np.array_equal(g[i].cpu().numpy(), ref)


def test_env_mixed_fp32_within_budget():
    D, r, n = 5, 2, 2
    Ta, Tb, G = _items(400, n, 2, D)
    cfg = O.Config(D=D, r=r)
    ctx = _ctx(D, r, precision=1, max_batch=n)
    Q = [_oracle_stage(Ta[i], Tb[i], G[i], cfg) for i in range(n)]
    QA, QB = np.stack([q[0] for q in Q]), np.stack([q[2] for q in Q])
    ng = (D * r) ** 2
    g = _empty((n, ng, ng))
    ctx.batch_env_dev(n, _dev(Ta), _dev(Tb), _dev(QA), _dev(QB), g)
    ctx.sync()
    for i in range(n):
        ref = O.metric_raw(Ta[i], Tb[i], QA[i], QB[i], 2, D)
        assert _rel(g[i].cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("D,r", [(3, 2), (5, 2), (8, 2), (4, 4)])
def test_env_bf16x3_tensor_cores_within_budget(D, r):
    """Split-BF16 tcgen05 environment: rel-Frobenius(g) <= 1e-4 against the
    FP64 oracle, on full tiles (D=8), ragged tiles (D=5, D=3) and r=4."""
    n = 2
    Ta, Tb, G = _items(450 + D, n, 2, D)
    cfg = O.Config(D=D, r=r)
    ctx = _ctx(D, r, precision=2, max_batch=n)
    Q = [_oracle_stage(Ta[i], Tb[i], G[i], cfg) for i in range(n)]
    QA, QB = np.stack([q[0] for q in Q]), np.stack([q[2] for q in Q])
    ng = (D * r) ** 2
    g = _empty((n, ng, ng))
    ctx.batch_env_dev(n, _dev(Ta), _dev(Tb), _dev(QA), _dev(QB), g)
    ctx.sync()
    for i in range(n):
        ref = O.metric_raw(Ta[i], Tb[i], QA[i], QB[i], 2, D)
        assert _rel(g[i].cpu().numpy(), ref) < 1e-4


# --------------------------------------------------------------- repair
@pytest.mark.parametrize("kind", ["network", "dense"])
def test_repair_certified_paths_match_oracle(kind):
    """Positive definite input: nothing to clip.  Metrics of random site
    tensors are often diagonally dominant, so the Gershgorin discs certify
    them, else the Cholesky factorisation does; a dense positive definite
    matrix W diag(lam) W^H (Haar W, lam in [1, 30]) is far from diagonally
    dominant and needs the Cholesky factorisation."""
    D, r, n = 3, 2, 2
    raws, refs = [], []
    if kind == "network":
        Ta, Tb, G = _items(500, n, 2, D)
        cfg = O.Config(D=D, r=r)
        for i in range(n):
            qa, ra, qb, rb = _oracle_stage(Ta[i], Tb[i], G[i], cfg)
            raws.append(O.metric_raw(Ta[i], Tb[i], qa, qb, 2, D))
    else:
        rng = np.random.default_rng(11)
        ng = (D * r) ** 2
        for i in range(n):
            a = rng.standard_normal((ng, ng)) + 1j * rng.standard_normal((ng, ng))
            w, _ = np.linalg.qr(a)
            h = (w * np.geomspace(1.0, 30.0, ng)) @ w.conj().T
            raws.append(h + 1e-3 * rng.standard_normal((ng, ng)))    # small anti-Hermitian part
    refs = [O.hermitise_repair(x) for x in raws]
    ctx = _ctx(D, r, max_batch=n)
    g = _dev(np.stack(raws))
    diag = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.solver_paths()
    ctx.batch_repair_dev(n, g, diag)
    ctx.sync()
    paths = ctx.solver_paths()
    if kind == "network":
        # of these two metrics the first is diagonally dominant (min_i d_i - s_i
        # = +0.21 max d), the second is not (-0.19 max d)
        assert paths["repair_gershgorin"] == 1 and paths["repair_cholesky"] == 1
    else:
        assert paths["repair_cholesky"] == n
    for i in range(n):
        assert _rel(g[i].cpu().numpy(), refs[i][0]) < 1e-12
        dg = diag[i].cpu().numpy()
        assert abs(dg[0] - refs[i][1][0]) < 1e-12 * max(1.0, refs[i][1][0])
        assert abs(dg[2] - refs[i][1][2]) < 1e-12
        assert np.isnan(dg[1])          # certified positive definite, no repair


def test_repair_clips_negative_eigenvalues():
    """Indefinite Hermitian input: the eigen-repair fallback must match the
    oracle's clipping."""
    rng = np.random.default_rng(7)
    n, K = 2, 6
    ng = K * K
    raws = []
    for _ in range(n):
        a = rng.standard_normal((ng, ng)) + 1j * rng.standard_normal((ng, ng))
        h = a @ a.conj().T / ng
        lam, w = np.linalg.eigh(h)
        lam[:5] = -np.linspace(0.05, 0.2, 5)          # five negative modes
        raws.append((w * lam) @ w.conj().T + 1e-3 * (rng.standard_normal((ng, ng))))
    ctx = _ctx(3, 2, max_batch=n)
    g = _dev(np.stack(raws))
    diag = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.solver_paths()
    ctx.batch_repair_dev(n, g, diag)
    ctx.sync()
    assert ctx.solver_paths()["repair_eigen"] == n
    for i in range(n):
        ref, rd = O.hermitise_repair(raws[i])
        assert _rel(g[i].cpu().numpy(), ref) < 1e-11
        dg = diag[i].cpu().numpy()
        assert abs(dg[0] - rd[0]) < 1e-12 * max(1.0, rd[0])
        assert abs(dg[1] - rd[1]) < 1e-10


# ------------------------------------------------------------------ ALS
@pytest.mark.parametrize("D,r,sweeps,kmin", [(2, 2, 3, 4), (3, 2, 10, 4), (4, 2, 5, 4),
                                             (3, 4, 4, 4), (3, 2, 4, 0), (5, 2, 2, 0),
                                             (4, 2, 0, 4), (6, 4, 0, 4), (7, 4, 0, 4)])
def test_als_matches_oracle(D, r, sweeps, kmin):
    """kmin=4: g_A is well conditioned, the Cholesky certificate decides the
    tolerance selection.  kmin=0: the grid starts at tau=1, which drops every
    eigenpair, so the certificate cannot hold and every solve goes through
    the eigendecomposition and the full selection.  sweeps=0: the balanced
    SVDU truncation with no solve, reported tau NaN; at K = D r = 24 and 28
    its K x K SVD is the preconditioned one (QR, then Jacobi on R^H)."""
    n = 2
    Ta, Tb, G = _items(600 + D, n, 2, D)
    cfg = O.Config(D=D, r=r, sweeps=sweeps, tau_exponents=tuple(range(kmin, 16)))
    gs, RAs, RBs, refs = [], [], [], []
    for i in range(n):
        qa, ra, qb, rb = _oracle_stage(Ta[i], Tb[i], G[i], cfg)
        g, _ = O.hermitise_repair(O.metric_raw(Ta[i], Tb[i], qa, qb, 2, D))
        gs.append(g); RAs.append(ra); RBs.append(rb)
        refs.append(O.als_truncate(g, ra, rb, D, sweeps, cfg.taus))
    ctx = _ctx(D, r, sweeps=sweeps, max_batch=n, kmin=kmin)
    K = D * r
    MA, MB = _empty((n, K, D)), _empty((n, K, D))
    info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    ctx.solver_paths()
    ctx.batch_als_dev(n, _dev(np.stack(gs)), _dev(np.stack(RAs)), _dev(np.stack(RBs)), MA, MB, info)
    ctx.sync()
    paths = ctx.solver_paths()
    solves = n * 2 * sweeps
    if sweeps == 0:
        assert sum(paths[k] for k in ("als_gershgorin", "als_cholesky", "als_eigen")) == 0
    elif kmin == 4:
        # random-tensor metrics give diagonally dominant g_A: the discs decide
        assert paths["als_gershgorin"] + paths["als_cholesky"] == solves
        assert paths["als_gershgorin"] > 0 and paths["als_eigen"] == 0
    else:
        assert paths["als_gershgorin"] + paths["als_cholesky"] == 0
        assert paths["als_eigen"] == solves
    for i in range(n):
        ma, mb, eps, delta, eps0, tau = refs[i]
        inf = info[i].cpu().numpy()
        assert abs(inf[2] - eps0) < 1e-12 * eps0
        assert abs(inf[1] - delta) < 1e-8
        assert abs(inf[0] - eps) < 1e-8 * eps0
        if sweeps == 0:
            assert tau is None and np.isnan(inf[3])
        else:
            assert inf[3] == tau
        assert _rel(MA[i].cpu().numpy(), ma) < 1e-8
        assert _rel(MB[i].cpu().numpy(), mb) < 1e-8


@pytest.mark.parametrize("D,precision", [(3, 1), (4, 2), (6, 2)])
def test_als_double_fp32_build_matches_oracle(D, precision):
    """Mixed contexts build the reduced metric g_A in double-FP32 arithmetic
    (pairs of FP32 values, about 2^-48 relative) and solve in FP64.  On the
    same FP64 metric the result stays within 1e-9 of the FP64 oracle, far
    inside the mixed path's 1e-4 environment budget."""
    n, r, sweeps = 2, 2, 10
    Ta, Tb, G = _items(650 + D, n, 2, D)
    cfg = O.Config(D=D, r=r, sweeps=sweeps, tau_exponents=tuple(range(4, 9)))
    gs, RAs, RBs, refs = [], [], [], []
    for i in range(n):
        qa, ra, qb, rb = _oracle_stage(Ta[i], Tb[i], G[i], cfg)
        g, _ = O.hermitise_repair(O.metric_raw(Ta[i], Tb[i], qa, qb, 2, D))
        gs.append(g); RAs.append(ra); RBs.append(rb)
        refs.append(O.als_truncate(g, ra, rb, D, sweeps, cfg.taus))
    ctx = _ctx(D, r, sweeps=sweeps, precision=precision, max_batch=n, kmin=4, kmax=8)
    K = D * r
    MA, MB = _empty((n, K, D)), _empty((n, K, D))
    info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    ctx.batch_als_dev(n, _dev(np.stack(gs)), _dev(np.stack(RAs)), _dev(np.stack(RBs)), MA, MB, info)
    ctx.sync()
    for i in range(n):
        ma, mb, eps, delta, eps0, tau = refs[i]
        inf = info[i].cpu().numpy()
        assert abs(inf[2] - eps0) < 1e-12 * eps0
        assert abs(inf[1] - delta) < 1e-10
        assert inf[3] == tau
        assert _rel(MA[i].cpu().numpy(), ma) < 1e-9
        assert _rel(MB[i].cpu().numpy(), mb) < 1e-9


@pytest.mark.parametrize("D,r,precision", [(8, 2, 2), (4, 4, 2), (8, 2, 1), (8, 4, 2)])
def test_als_tensor_core_build_matches_oracle(D, r, precision):
    """K = D r = 16 or 32 on a mixed context with one CTA per item: the first
    stage of the reduced-metric build runs on the tensor cores with exact
    BF16 slicing (six slices, levels combined in double-FP32).  On the same
    FP64 metric the ALS result stays within 1e-9 of the FP64 oracle, like
    the double-FP32 lane build, and the two builds agree to 1e-11 at K = 16,
    where every level sum is exact in FP32, and to 1e-10 at K = 32, where the
    sums of the upper levels round at 2^-47 of the entry."""
    n, sweeps = 3, 10
    Ta, Tb, G = _items(660 + D, n, 2, D)
    cfg = O.Config(D=D, r=r, sweeps=sweeps, tau_exponents=tuple(range(4, 9)))
    gs, RAs, RBs, refs = [], [], [], []
    for i in range(n):
        qa, ra, qb, rb = _oracle_stage(Ta[i], Tb[i], G[i], cfg)
        g, _ = O.hermitise_repair(O.metric_raw(Ta[i], Tb[i], qa, qb, 2, D))
        gs.append(g); RAs.append(ra); RBs.append(rb)
        refs.append(O.als_truncate(g, ra, rb, D, sweeps, cfg.taus))
    ctx = _ctx(D, r, sweeps=sweeps, precision=precision, max_batch=n, kmin=4, kmax=8)
    K = D * r
    outs = {}
    # (split, build): one CTA per item with either build, and the
    # tensor-core build on 4-CTA clusters, which divide its tiles
    for split, build in ((1, 2), (1, 1), (4, 2)):
        ctx.set_tuning(als_split=split, als_build=build)
        MA, MB = _empty((n, K, D)), _empty((n, K, D))
        info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
        ctx.batch_als_dev(n, _dev(np.stack(gs)), _dev(np.stack(RAs)), _dev(np.stack(RBs)), MA,
                          MB, info)
        ctx.sync()
        outs[split, build] = (MA.cpu().numpy(), MB.cpu().numpy(), info.cpu().numpy())
    for a, b in zip(outs[4, 2], outs[1, 2]):
        assert np.array_equal(a, b)
    outs[2], outs[1] = outs[1, 2], outs[1, 1]
    MA, MB, info = outs[2]
    for i in range(n):
        ma, mb, eps, delta, eps0, tau = refs[i]
        assert abs(info[i, 2] - eps0) < 1e-12 * eps0
        assert abs(info[i, 1] - delta) < 1e-10
        assert info[i, 3] == tau
        assert _rel(MA[i], ma) < 1e-9 and _rel(MB[i], mb) < 1e-9
        tol = 1e-11 if K == 16 else 1e-10
        assert _rel(MA[i], outs[1][0][i]) < tol and _rel(MB[i], outs[1][1][i]) < tol


@pytest.mark.parametrize("spread,path", [(30.0, "als_cholesky"), (1e7, "als_eigen")])
def test_als_dense_metric_paths(spread, path):
    """A dense metric g = W diag(lam) W^H (W Haar-random, lam geometric on
    [1, spread]) makes g_A far from diagonally dominant.  With spread 30 the
    discs fail but the shifted Cholesky proves every tolerance of the grid
    keeps every eigenpair; with spread 1e7 the smallest eigenvalues fall below
    tau_max lambda_max and the full selection of Eq. 4 must run."""
    D, r, sweeps, n = 3, 2, 4, 2
    K = D * r
    ng = K * K
    rng = np.random.default_rng(4242)
    gs, RAs, RBs, refs = [], [], [], []
    cfg = O.Config(D=D, r=r, sweeps=sweeps)
    for _ in range(n):
        a = rng.standard_normal((ng, ng)) + 1j * rng.standard_normal((ng, ng))
        w, _ = np.linalg.qr(a)
        g = (w * np.geomspace(1.0, spread, ng)) @ w.conj().T
        g = 0.5 * (g + g.conj().T)
        RA = rng.standard_normal((K, K)) + 1j * rng.standard_normal((K, K))
        RB = rng.standard_normal((K, K)) + 1j * rng.standard_normal((K, K))
        gs.append(g); RAs.append(RA); RBs.append(RB)
        refs.append(O.als_truncate(g, RA, RB, D, sweeps, cfg.taus))
    ctx = _ctx(D, r, sweeps=sweeps, max_batch=n, kmin=4)
    MA, MB = _empty((n, K, D)), _empty((n, K, D))
    info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    ctx.solver_paths()
    ctx.batch_als_dev(n, _dev(np.stack(gs)), _dev(np.stack(RAs)), _dev(np.stack(RBs)), MA, MB, info)
    ctx.sync()
    assert ctx.solver_paths()[path] == n * 2 * sweeps
    for i in range(n):
        ma, mb, eps, delta, eps0, tau = refs[i]
        inf = info[i].cpu().numpy()
        assert abs(inf[2] - eps0) < 1e-12 * eps0
        assert abs(inf[1] - delta) < 1e-9
        assert inf[3] == tau
        assert _rel(MA[i].cpu().numpy(), ma) < 1e-8
        assert _rel(MB[i].cpu().numpy(), mb) < 1e-8


# ------------------------------------------------------- full update
@pytest.mark.parametrize("D,precision", [(3, 0), (4, 0), (6, 0), (4, 1), (4, 2), (6, 2)])
def test_batch_update_matches_oracle(D, precision):
    n = 3
    Ta, Tb, G = _items(700 + D, n, 2, D)
    ctx = _ctx(D, 2, precision=precision, max_batch=n, kmin=4, kmax=15 if precision == 0 else 8)
    Ta_o, Tb_o, info = ctx.batch_update_host(Ta, Tb, G)
    cfg = O.Config(D=D, r=2)
    for i in range(n):
        A2, B2, inf = O.bond_update(Ta[i], Tb[i], G[i], cfg)
        if precision == 0:
            assert _rel(Ta_o[i], A2) < 1e-9
            assert _rel(Tb_o[i], B2) < 1e-9
            assert abs(info[i, 1] - inf.delta) < 1e-8
        else:
            assert abs(info[i, 1] - inf.delta) <= 1e-2 * inf.delta
            pair = np.einsum("plurn,qrvwx->plunqvwx", Ta_o[i], Tb_o[i])
            ref = np.einsum("plurn,qrvwx->plunqvwx", A2, B2)
            assert _rel(pair, ref) < 1e-4


def test_batch_update_host_and_dev_agree_and_empty_batch():
    D, n = 3, 2
    Ta, Tb, G = _items(800, n, 2, D)
    ctx = _ctx(D, 2, max_batch=n)
    a1, b1, i1 = ctx.batch_update_host(Ta, Tb, G)
    ta, tb, gg = _dev(Ta), _dev(Tb), _dev(G)
    oa, ob = torch.empty_like(ta), torch.empty_like(tb)
    info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    ctx.batch_update_dev(n, ta, tb, gg, oa, ob, info)
    ctx.sync()
    assert np.array_equal(oa.cpu().numpy(), a1)
    assert np.array_equal(info.cpu().numpy(), i1)
    ctx.batch_update_dev(0, ta, tb, gg, oa, ob, info)     # empty batch is a no-op
    from paper_2107_06635_gb300.ntu import NTUError
    with pytest.raises(NTUError):
        ctx.batch_update_dev(n + 1, ta, tb, gg, oa, ob, info)


# --------------------------------------------------------- unit cell
def test_unit_cell_step_matches_oracle_d3():
    """One Trotter step of the 2-site cell, D=3, seed 1, exp(-i 0.01 ZZ),
    10 sweeps: R, g, delta per bond and the final state."""
    A, B = I.random_pair(1, 2, 3)
    G = I.zz_gate(0.01)
    cfg = O.Config(D=3, r=2, sweeps=10)
    ctx = _ctx(3, 2)
    ctx.set_state(A, B)
    Ao, Bo = A.copy(), B.copy()
    for b in range(4):
        RA, RB = ctx.apply_gate(b, G)
        g, diag = ctx.env_metric(b)
        res = ctx.als_truncate(b)
        Ao, Bo, info = O.update_bond(Ao, Bo, b, G, cfg, keep=True)
        assert _rel(RA @ RB.T, info.RA @ info.RB.T) < 1e-12
        assert _rel(g, info.g) < 1e-10
        assert abs(res["delta"] - info.delta) < 1e-8
        assert res["tau"] == info.tau
    A2, B2 = ctx.get_state()
    assert _rel(A2, Ao) < 1e-9 and _rel(B2, Bo) < 1e-9


def test_unit_cell_step_site_asymmetric_gates_d3():
    """The unit-cell calls with a different random two-site unitary on each
    bond (not symmetric under exchanging the sites, distinct operator-Schmidt
    values): exercises the gate-site swap of bonds 2 and 3 and the rotation
    of bonds 1 and 3 (Sec. II, Fig. 2) against the oracle, stage by stage."""
    A, B = I.random_pair(3, 2, 3)
    rng = np.random.default_rng(33)
    gates = [I.random_gate(rng) for _ in range(4)]
    for G in gates:
        assert np.linalg.norm(G - G.transpose(1, 0, 3, 2)) > 0.1
    cfg = O.Config(D=3, r=2, sweeps=10)
    ctx = _ctx(3, 2)
    ctx.set_state(A, B)
    Ao, Bo = A.copy(), B.copy()
    for b in range(4):
        RA, RB = ctx.apply_gate(b, gates[b])
        g, diag = ctx.env_metric(b)
        res = ctx.als_truncate(b)
        Ao, Bo, info = O.update_bond(Ao, Bo, b, gates[b], cfg, keep=True)
        assert _rel(RA @ RB.T, info.RA @ info.RB.T) < 1e-12, b
        assert _rel(g, info.g) < 1e-10, b
        assert abs(res["delta"] - info.delta) < 1e-8, b
        A2, B2 = ctx.get_state()
        assert _rel(A2, Ao) < 1e-9 and _rel(B2, Bo) < 1e-9, b


@pytest.mark.parametrize("precision", [0, 2])
def test_step_site_asymmetric_gates_matches_oracle(precision):
    """One Trotter step (ntu_step) with four different site-asymmetric bond
    gates and a random single-site unitary, D=4: per-bond delta and the final
    state against the oracle's step (FP64 context: state 1e-9, delta 1e-8;
    split-BF16 context: delta 1e-2 relative, the contracted A-B pair on
    every bond 1e-4)."""
    D = 4
    A, B = I.random_pair(4, 2, D)
    rng = np.random.default_rng(44)
    gates = [I.random_gate(rng) for _ in range(4)]
    u1 = _random_unitary(rng, 2)
    kmax = 15 if precision == 0 else 8
    cfg = O.Config(D=D, r=2, sweeps=10, tau_exponents=tuple(range(4, kmax + 1)))
    ctx = _ctx(D, 2, precision=precision, kmax=kmax)
    ctx.set_state(A, B)
    deltas = ctx.step(gates, u1)
    Ao, Bo, dref = O.ntu_step(A, B, gates, u1, cfg)
    A2, B2 = ctx.get_state()
    if precision == 0:
        assert np.max(np.abs(deltas - np.array(dref))) < 1e-8
        assert _rel(A2, Ao) < 1e-9 and _rel(B2, Bo) < 1e-9
    else:
        assert np.all(np.abs(deltas - np.array(dref)) <= 1e-2 * np.array(dref))
        for la, lb in ((3, 1), (2, 4), (1, 3), (4, 2)):
            pg = np.tensordot(A2, B2, axes=([la], [lb]))
            pr = np.tensordot(Ao, Bo, axes=([la], [lb]))
            assert _rel(pg, pr) < 1e-4


def _random_unitary(rng, n):
    m = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(m)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("precision", [0, 2])
def test_unit_cell_bond_legs_closed_form(precision):
    """Closed form, no oracle: from a D=1 product state zero-padded to D=2,
    the gate exp(-i t Z_A X_B) on bond b gives a state of bond rank 2, so the
    update is exact.  After each bond's update through the unit-cell calls,
    A' and B' carry the new bond only on the legs of bond b (A's leg b in
    the order r, u, l, dn; B's opposite leg) and contract to the exact
    two-site state with Z on A and X on B."""
    t = 0.3
    Z, X = I.pauli("Z"), I.pauli("X")
    G = I.two_site(np.cos(t) * np.eye(4) - 1j * np.sin(t) * np.kron(Z, X))
    psiA = np.array([0.6, 0.8], dtype=np.complex128)
    psiB = np.array([0.8, -0.6j], dtype=np.complex128)
    exact = (np.cos(t) * np.outer(psiA, psiB)
             - 1j * np.sin(t) * np.outer(Z @ psiA, X @ psiB)).reshape(-1)
    legs = {0: (3, 1), 1: (2, 4), 2: (1, 3), 3: (4, 2)}
    ctx = _ctx(2, 2, sweeps=4, precision=precision, kmax=15 if precision == 0 else 8)
    for b in range(4):
        ctx.set_state(I.product_state(psiA, 2), I.product_state(psiB, 2))
        ctx.apply_gate(b, G)
        ctx.env_metric(b)
        ctx.als_truncate(b)
        A2, B2 = ctx.get_state()
        la, lb = legs[b]
        for T, leg in ((A2, la), (B2, lb)):
            rest = np.moveaxis(T, leg, 1)[:, :, :, :, :].copy()
            rest[:, :, 0, 0, 0] = 0
            assert np.abs(rest).max() <= (1e-12 if precision == 0 else 1e-5) * np.abs(T).max(), \
                (b, leg)
        a = np.moveaxis(A2, la, -1)[:, 0, 0, 0, :]
        bb = np.moveaxis(B2, lb, -1)[:, 0, 0, 0, :]
        pair = (a @ bb.T).reshape(-1)
        ov = abs(np.vdot(pair, exact)) / (np.linalg.norm(pair) * np.linalg.norm(exact))
        assert abs(ov - 1) < (1e-13 if precision == 0 else 1e-8), (b, ov)   # ov = 1 - O(err^2)


def test_unit_cell_call_order_is_enforced():
    from paper_2107_06635_gb300.ntu import NTUError
    ctx = _ctx(2, 2)
    A, B = I.random_pair(2, 2, 2)
    ctx.set_state(A, B)
    with pytest.raises(NTUError) as e:
        ctx.env_metric(0)
    assert e.value.status == 7
    ctx.apply_gate(1, I.zz_gate(0.1))
    with pytest.raises(NTUError):
        ctx.env_metric(0)          # prepared bond was 1


def test_step_product_state_single_site_exact():
    """D=1, identity bond gates, field h: <sigma_z>(t) = cos(2 h t)."""
    h, dt = 0.7, 0.05
    ctx = _ctx(1, 1, sweeps=2)
    A = I.plus_z_state(1)
    ctx.set_state(A, A)
    for step in range(1, 11):
        deltas = ctx.step([I.identity_gate()] * 4, I.x_rotation(h * dt / 2))
        for site in (0, 1):
            z = ctx.measure(site, I.pauli("Z"))
            assert abs(z - np.cos(2 * h * step * dt)) < 1e-12
        assert np.all(deltas < 1e-14)


def test_step_classical_quench_exact_at_D2():
    ctx = _ctx(2, 2, sweeps=4)
    A = I.plus_x_state(2)
    ctx.set_state(A, A)
    gates2, _ = I.tfim_real_time_gates(0.0, 0.05)
    for _ in range(4):
        deltas = ctx.step(gates2, None)
        assert np.all(deltas <= 1e-12)


@pytest.mark.parametrize("D,steps", [(4, 5), (5, 3)])
def test_quench_observable_parity(D, steps):
    """TFIM quench h=2.5, dt=0.01 from |+x> zero-padded to D with a seeded
    1e-2 random admixture (which lifts the zero modes of the padded bonds):
    <sigma_x> after every step within 1e-6 of the oracle."""
    gates2, gate1 = I.tfim_real_time_gates(2.5, 0.01)
    cfg = O.Config(D=D, r=2, sweeps=10)
    A, B = I.quench_start(D)
    ctx = _ctx(D, 2)
    ctx.set_state(A, B)
    for _ in range(steps):
        ctx.step(gates2, gate1)
        A, B, _ = O.ntu_step(A, B, gates2, gate1, cfg)
        for site in (0, 1):
            x_gpu = ctx.measure(site, I.pauli("X"))
            x_ref = O.measure(A, B, site, I.pauli("X"), 1)
            assert abs(x_gpu - x_ref) < 1e-6


def test_quench_zero_padded_start_stays_finite_and_close():
    """The bare zero-padded start has exact zero modes: the oracle's own
    <sigma_x> moves by ~1e-5 under a 1e-14 perturbation of the start, so
    GPU and oracle can only agree to that level.  Checks finiteness, tiny
    truncation errors and agreement within 1e-4."""
    D = 4
    gates2, gate1 = I.tfim_real_time_gates(2.5, 0.01)
    cfg = O.Config(D=D, r=2, sweeps=10)
    A, B = I.quench_start(D, mix=0.0)
    ctx = _ctx(D, 2)
    ctx.set_state(A, B)
    for _ in range(3):
        deltas = ctx.step(gates2, gate1)
        assert np.all(np.isfinite(deltas)) and np.all(deltas < 1e-8)
        A, B, _ = O.ntu_step(A, B, gates2, gate1, cfg)
        x_gpu = ctx.measure(0, I.pauli("X"))
        assert abs(x_gpu - O.measure(A, B, 0, I.pauli("X"), 1)) < 1e-4


@pytest.mark.parametrize("D,precision,tol", [(4, 0, 1e-6), (4, 2, 1e-4), (5, 0, 1e-6)])
def test_purification_imaginary_time_parity(D, precision, tol):
    """Thermal state by purification (physical d=2 x ancilla 2, gates on the
    physical index): TFIM h=2.5, imaginary-time steps of dbeta=0.005 from the
    infinite-temperature purification zero-padded to D with a seeded 1e-2
    admixture (which lifts the zero modes of the padded bonds).  <sigma_x>
    and <sigma_z> after every step against the oracle: 1e-6 on the FP64
    context, 1e-4 on the split-BF16 tensor-core context."""
    rng = np.random.default_rng(77)
    A = I.purification_state(D) + 1e-2 * I.random_site_tensor(rng, 4, D)
    B = I.purification_state(D) + 1e-2 * I.random_site_tensor(rng, 4, D)
    A, B = A / np.linalg.norm(A), B / np.linalg.norm(B)
    gates2, gate1 = I.tfim_imag_time_gates(2.5, 0.005)
    cfg = O.Config(D=D, r=2, d_anc=2, sweeps=10,
                   tau_exponents=tuple(range(4, 16 if precision == 0 else 9)))
    ctx = _ctx(D, 2, d_anc=2, precision=precision, kmax=15 if precision == 0 else 8)
    ctx.set_state(A, B)
    for _ in range(3):
        ctx.step(gates2, gate1)
        A, B, _ = O.ntu_step(A, B, gates2, gate1, cfg)
        for site in (0, 1):
            for op in ("X", "Z"):
                v_gpu = ctx.measure(site, I.pauli(op))
                v_ref = O.measure(A, B, site, I.pauli(op), 2)
                assert abs(v_gpu - v_ref) < tol


def test_measure_matches_oracle():
    A, B = I.random_pair(9, 4, 3)
    ctx = _ctx(3, 2, d_anc=2)
    ctx.set_state(A, B)
    for site in (0, 1):
        for op in ("X", "Z"):
            v = ctx.measure(site, I.pauli(op))
            assert abs(v - O.measure(A, B, site, I.pauli(op), 2)) < 1e-12


# ------------------------------------------------------------- uneven batches
@pytest.mark.parametrize("D,precision", [(6, 0), (7, 0), (8, 0), (8, 2)])
def test_batch_update_r4_large_bond(D, precision):
    """r=4 gates at D=6, 7, 8: K = D r = 24, 28, 32 (32 is the largest bond
    the library takes), g of size K^2 = 576, 784, 1024 and reduced metrics of
    n_A = 144, 196, 256; the Heisenberg gate exp(-i 0.01 (XX+YY+ZZ)) has rank
    4.  From K = 24 on the SVDU start takes the preconditioned SVD."""
    n = 2
    rng = np.random.default_rng(900 + D)
    Ta = np.stack([I.random_site_tensor(rng, 2, D) for _ in range(n)])
    Tb = np.stack([I.random_site_tensor(rng, 2, D) for _ in range(n)])
    G = np.stack([I.heisenberg_gate(0.01)] * n)
    ctx = _ctx(D, 4, sweeps=8, precision=precision, max_batch=n, kmax=15 if precision == 0 else 8)
    Ta_o, Tb_o, info = ctx.batch_update_host(Ta, Tb, G)
    cfg = O.Config(D=D, r=4, sweeps=8, tau_exponents=tuple(range(4, 16 if precision == 0 else 9)))
    for i in range(n):
        A2, B2, inf = O.bond_update(Ta[i], Tb[i], G[i], cfg)
        if precision == 0:
            assert _rel(Ta_o[i], A2) < 1e-9
            assert _rel(Tb_o[i], B2) < 1e-9
            assert abs(info[i, 1] - inf.delta) < 1e-8
        else:
            assert abs(info[i, 1] - inf.delta) <= 1e-2 * inf.delta
            pair = np.einsum("plurn,qrvwx->plunqvwx", Ta_o[i], Tb_o[i])
            ref = np.einsum("plurn,qrvwx->plunqvwx", A2, B2)
            assert _rel(pair, ref) < 1e-4


@pytest.mark.parametrize("precision", [0, 2])
def test_uneven_batch_matches_oracle_and_modes_agree(precision):
    """The uneven workload (D uniform in 3..8, r in {2, 4}, complex64 draws,
    8 sweeps) in one call: every item against the oracle's bond update (FP64
    context: tensors 1e-9, delta 1e-8; split-BF16 context: delta 1e-2
    relative, the two-site state 1e-4); a kind with no items in the call is
    skipped.  Direct enqueue, CUDA-graph replay (twice, and after the counts
    change), the staged device-resident run in all three modes (grouped,
    graph, one launch sequence per item) give bit-identical results."""
    from paper_2107_06635_gb300 import ntu
    items = I.uneven_batch(41, 14)
    kinds = sorted({(it[0], it[1]) for it in items})
    unused = next((D, r) for D in range(3, 9) for r in (2, 4) if (D, r) not in kinds)
    kinds.append(unused)
    caps = [sum(1 for it in items if (it[0], it[1]) == k) or 1 for k in kinds]
    kmax = 15 if precision == 0 else 8
    ub = ntu.UnevenBatch(kinds, caps, sweeps=8, precision=precision, tau_kmax=kmax)
    try:
        oa, ob, info = ub.update(items, use_graph=False)
        for i, (D, r, ta, tb, g) in enumerate(items):
            cfg = O.Config(D=D, r=r, sweeps=8, tau_exponents=tuple(range(4, kmax + 1)))
            A2, B2, inf = O.bond_update(ta, tb, g, cfg)
            if precision == 0:
                assert _rel(oa[i], A2) < 1e-9, (i, D, r)
                assert _rel(ob[i], B2) < 1e-9, (i, D, r)
                assert abs(info[i, 1] - inf.delta) < 1e-8, (i, D, r)
            else:
                assert abs(info[i, 1] - inf.delta) <= 1e-2 * inf.delta, (i, D, r)
                pair = np.einsum("plurn,qrvwx->plunqvwx", oa[i], ob[i])
                ref = np.einsum("plurn,qrvwx->plunqvwx", A2, B2)
                assert _rel(pair, ref) < 1e-4, (i, D, r)

        def same(res):
            a, b, inf = res
            assert np.array_equal(inf, info)
            for i in range(len(items)):
                assert np.array_equal(a[i], oa[i]) and np.array_equal(b[i], ob[i])

        same(ub.update(items, use_graph=True))
        same(ub.update(items, use_graph=True))
        sub = items[:3]                       # other per-kind counts: captured again
        sa, sb, si = ub.update(sub, use_graph=True)
        for i in range(3):
            assert np.array_equal(sa[i], oa[i]) and np.array_equal(sb[i], ob[i])
        ub.stage(items)
        for mode in (ub.GROUPED, ub.GRAPH, ub.GRAPH, ub.PER_ITEM):
            ub.run(mode)
            ub.sync()
            assert ub.last_launch_count() > 0
            same(ub.fetch(items))
        with pytest.raises(ntu.NTUError):
            ub.fetch(sub)                     # counts differ from the staged items
        with pytest.raises(ntu.NTUError):
            ub.update(items + items, use_graph=False)      # beyond max_items
    finally:
        ub.close()


# ------------------------- full trajectories (TFIM quench, purification)
def _golden(name):
    import json
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", name)))


def _envelope(spread, w=3):
    """Largest value of a per-step spread within +-w steps."""
    s = np.asarray(spread)
    return np.array([s[max(0, i - w):i + w + 1].max() for i in range(s.size)])


@pytest.mark.parametrize("D,precision", [(4, 0), (5, 0), (4, 2), (5, 2)])
def test_quench_full_trajectory(D, precision):
    """TFIM quench h = 2.5, dt = 0.01 to t = 2 (200 steps, Sec. III):
    <sigma_x> of both sites after every step against the oracle's stored
    trajectory, bounded by the oracle's own spread when its inputs are
    perturbed at the level of the path's arithmetic (stored beside the
    trajectory by tests/golden/make_golden.py, largest value within +-3
    steps).  The early steps truncate singular values of weight ~1e-15, so
    the kept directions are chosen by rounding and any implementation that
    rounds differently moves <sigma_x> by up to ~2e-5 around steps 7-12.
    FP64 context: at most twice the spread of an ensemble with 1e-14
    perturbations of the start (observed at most 0.8 of it).  Split-BF16
    context: at most four times the spread of an ensemble whose environment
    operands carry the split representation's 2^-17 relative error and which
    uses the mixed tolerance grid 1e-4..1e-8 (observed at most 2.9 of it);
    1e-6 on the steps where that spread is below 1e-7."""
    gold = _golden(f"quench_d{D}.json")
    gates2, gate1 = I.tfim_real_time_gates(gold["h"], gold["dt"])
    ctx = _ctx(D, 2, precision=precision, kmax=15 if precision == 0 else 8)
    A, B = I.quench_start(D)
    ctx.set_state(A, B)
    err = []
    for s in range(len(gold["sx_A"])):
        ctx.step(gates2, gate1)
        err.append(max(abs(ctx.measure(0, I.pauli("X")).real - gold["sx_A"][s]),
                       abs(ctx.measure(1, I.pauli("X")).real - gold["sx_B"][s])))
    err = np.array(err)
    if precision == 0:
        bound = 2 * _envelope(gold["spread_fp64"]) + 1e-12
    else:
        bound = 4 * _envelope(gold["spread_split16"]) + 1e-12
        quiet = np.array(gold["spread_split16"]) < 1e-7
        assert quiet.any() and np.all(err[quiet] < 1e-6), err[quiet]
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, [(int(i), err[i], bound[i]) for i in bad[:5]]


def test_fp64_context_at_the_bench_configuration():
    """The FP64 GPU path (the denominator of the measured speedup) at the
    bench configuration D=8, d=2, r=2, exp(-i 0.01 ZZ), 10 sweeps, seed 5:
    the repaired metric g within 1e-10 (relative Frobenius) of the oracle's,
    delta within 1e-8 and A', B' within 1e-9."""
    from paper_2107_06635_gb300 import ntu
    D, n = 8, 2
    Ta, Tb, G = I.batch_items(5, n, 2, D, I.zz_gate(0.01))
    ctx = ntu.Context(D, 2, 1, 2, 10, ntu.NTU_FP64, 4, 15, n)
    m, K = 2 * D ** 3, D * 2
    ta, tb, gg = _dev(Ta), _dev(Tb), _dev(G)
    QA, RA, QB, RB = _empty((n, m, K)), _empty((n, K, K)), _empty((n, m, K)), _empty((n, K, K))
    g = _empty((n, K * K, K * K))
    diag = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.batch_gate_qr_dev(n, ta, tb, gg, QA, RA, QB, RB)
    ctx.batch_env_dev(n, ta, tb, QA, QB, g)
    ctx.batch_repair_dev(n, g, diag)
    ctx.sync()
    a, b, info = ctx.batch_update_host(Ta, Tb, G)
    cfg = O.Config(D=D, r=2, sweeps=10)
    for i in range(n):
        A2, B2, ref = O.bond_update(Ta[i], Tb[i], G[i], cfg, keep=True)
        assert _rel(g[i].cpu().numpy(), ref.g) < 1e-10
        assert abs(info[i, 1] - ref.delta) < 1e-8
        assert _rel(a[i], A2) < 1e-9 and _rel(b[i], B2) < 1e-9
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-4), (2, 1e-4)])
def test_purification_full_trajectory(precision, tol):
    """Purification with h = 2.5 to beta = 0.5 (100 imaginary-time steps of dbeta = 0.005),
    D = 4: <sigma_x>, <sigma_z> of site A after every step against the
    oracle's stored trajectory (observed 1.4e-5 on both paths; the start is
    a padded product state, conditioned as in the quench)."""
    gold = _golden("purification_d4.json")
    rng = np.random.default_rng(77)
    A = I.purification_state(4) + 1e-2 * I.random_site_tensor(rng, 4, 4)
    B = I.purification_state(4) + 1e-2 * I.random_site_tensor(rng, 4, 4)
    A, B = A / np.linalg.norm(A), B / np.linalg.norm(B)
    gates2, gate1 = I.tfim_imag_time_gates(gold["h"], gold["dbeta"])
    ctx = _ctx(4, 2, d_anc=2, precision=precision, kmax=15 if precision == 0 else 8)
    ctx.set_state(A, B)
    for s in range(len(gold["sx_A"])):
        ctx.step(gates2, gate1)
        assert abs(ctx.measure(0, I.pauli("X")).real - gold["sx_A"][s]) < tol, s
        assert abs(ctx.measure(0, I.pauli("Z")).real - gold["sz_A"][s]) < tol, s


@pytest.mark.parametrize("precision", [2, 1])
def test_split_als_identical_to_single_cta(precision):
    """A batch too small to fill the GPU runs each item's ALS on a cluster of
    CTAs that divide the reduced-metric build (a context for at most 3 items
    splits 4 ways; one for 240 items does not split).  The blocks are the
    same arithmetic either way, so with the same build of the reduced metric
    (lanes, or tensor cores) the bond updates agree bit for bit; the two
    builds agree to 1e-10, and all match the oracle within the mixed-path
    budget.  r=4 gives K=16, D=4."""
    n = 3
    rng = np.random.default_rng(910)
    Ta = np.stack([I.random_site_tensor(rng, 2, 4) for _ in range(n)])
    Tb = np.stack([I.random_site_tensor(rng, 2, 4) for _ in range(n)])
    G = np.stack([I.heisenberg_gate(0.01)] * n)
    small = _ctx(4, 4, precision=precision, max_batch=n, kmax=8)
    big = _ctx(4, 4, precision=precision, max_batch=240, kmax=8)
    assert small.get_tuning()[1] == 4 and big.get_tuning()[1] == 1
    res = {}
    for build in (1, 2):
        small.set_tuning(als_build=build)
        big.set_tuning(als_build=build)
        a1, b1, i1 = small.batch_update_host(Ta, Tb, G)
        a2, b2, i2 = big.batch_update_host(Ta, Tb, G)
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and np.array_equal(i1, i2)
        res[build] = (a1, b1, i1)
    (a1, b1, i1), (a3, b3, _) = res[1], res[2]
    assert _rel(a3, a1) < 1e-10 and _rel(b3, b1) < 1e-10
    cfg = O.Config(D=4, r=4, tau_exponents=tuple(range(4, 9)))
    for i in range(n):
        A2, B2, inf = O.bond_update(Ta[i], Tb[i], G[i], cfg)
        assert abs(i1[i, 1] - inf.delta) <= 1e-2 * inf.delta


def test_mixed_repair_double_fp32_certificate():
    """Split-BF16 context, D=4 with the rank-4 Heisenberg gate: the metric
    (entries at the scales 1 and theta^2 of the gate's Schmidt values) is not
    diagonally dominant, so the repair certifies it by the double-FP32
    Cholesky factorisation (counted under repair_cholesky) and writes g/tr;
    the bond update matches the oracle within the mixed-path budget."""
    n = 2
    rng = np.random.default_rng(920)
    Ta = np.stack([I.random_site_tensor(rng, 2, 4) for _ in range(n)])
    Tb = np.stack([I.random_site_tensor(rng, 2, 4) for _ in range(n)])
    G = np.stack([I.heisenberg_gate(0.01)] * n)
    ctx = _ctx(4, 4, precision=2, max_batch=n, kmax=8)
    ctx.solver_paths()
    a, b, info = ctx.batch_update_host(Ta, Tb, G)
    paths = ctx.solver_paths()
    assert paths["repair_cholesky"] == n and paths["repair_eigen"] == 0, paths
    cfg = O.Config(D=4, r=4, tau_exponents=tuple(range(4, 9)))
    for i in range(n):
        A2, B2, inf = O.bond_update(Ta[i], Tb[i], G[i], cfg)
        assert abs(info[i, 1] - inf.delta) <= 1e-2 * inf.delta
        pair = np.einsum("plurn,qrvwx->plunqvwx", a[i], b[i])
        ref = np.einsum("plurn,qrvwx->plunqvwx", A2, B2)
        assert _rel(pair, ref) < 1e-4


# ------------------------------------------- the bench workload, full size
@pytest.mark.parametrize("D", [8, 6])
def test_full_size_bench_batch_sampled_against_oracle(D):
    """The measured workload at its full size and in the launch shapes the
    measurement uses: 912 bond updates of D=8 (and the D=6 line), d=2, r=2
    from seed 5, gate
    exp(-i 0.01 ZZ), 10 sweeps, split-BF16 environment, tau grid 1e-4..1e-8,
    on a non-default stream.  Three items (first, middle, last: different
    CTAs of every persistent kernel and both ends of the batch) are checked
    against the oracle's bond update one by one; all 912 are checked for what
    holds at any size: unit-norm outputs (A16), delta = eps / eps0 with
    eps0 > 0 and 0 <= delta <= 1, tau on the grid."""
    from paper_2107_06635_gb300 import ntu
    B, r, S = 912, 2, 10
    Ta_h, Tb_h, G_h = I.batch_items(5, B, 2, D, I.zz_gate(0.01))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        Ta, Tb, G = _dev(Ta_h), _dev(Tb_h), _dev(G_h)
        Ta_o, Tb_o = torch.empty_like(Ta), torch.empty_like(Tb)
        info = torch.empty((B, 4), dtype=torch.float64, device="cuda")
        ctx = ntu.Context(D, 2, 1, r, S, ntu.NTU_MIXED_BF16X3, 4, 8, B,
                          stream=stream.cuda_stream)
        ctx.batch_update_dev(B, Ta, Tb, G, Ta_o, Tb_o, info)
        ctx.sync()
    A_o, B_o, inf = Ta_o.cpu().numpy(), Tb_o.cpu().numpy(), info.cpu().numpy()
    assert np.all(np.isfinite(A_o)) and np.all(np.isfinite(B_o)) and np.all(np.isfinite(inf))
    nA = np.linalg.norm(A_o.reshape(B, -1), axis=1)
    nB = np.linalg.norm(B_o.reshape(B, -1), axis=1)
    assert np.max(np.abs(nA - 1)) < 1e-12 and np.max(np.abs(nB - 1)) < 1e-12
    eps, delta, eps0, tau = inf[:, 0], inf[:, 1], inf[:, 2], inf[:, 3]
    assert np.all(eps0 > 0)
    assert np.all(delta >= 0) and np.all(delta <= 1)
    np.testing.assert_allclose(delta, eps / eps0, rtol=1e-12, atol=0)
    grid = np.array([10.0 ** -k for k in range(4, 9)])
    assert np.all(np.min(np.abs(tau[:, None] / grid[None, :] - 1), axis=1) < 1e-12)
    cfg = O.Config(D=D, r=r, sweeps=S, tau_exponents=tuple(range(4, 9)))
    for i in (0, B // 2, B - 1):
        A2, B2, ref = O.bond_update(Ta_h[i], Tb_h[i], G_h[i], cfg)
        assert abs(inf[i, 2] - ref.eps0) <= 1e-4 * ref.eps0
        assert abs(inf[i, 1] - ref.delta) <= 1e-2 * ref.delta
        pair = np.einsum("plurn,qrvwx->plunqvwx", A_o[i], B_o[i])
        pref = np.einsum("plurn,qrvwx->plunqvwx", A2, B2)
        assert _rel(pair, pref) < 1e-4


@pytest.mark.parametrize("D,r", [(4, 4), (3, 2)])
def test_mixed_als_scaled_metric(D, r):
    """A metric far outside [2^-60, 2^60] is split for the mixed ALS as
    g 2^-e with e from its largest entry (the per-item maximum and split
    kernels): every product of the build, the solves and the error is then
    scaled by exact powers of two, so g 2^70 and g 2^-70 give the same
    factors and delta as g, and eps scaled by 2^(+-70).  (4,4): the
    tensor-core build (K = 16); (3,2): the lane build with the swapped copy."""
    n, sweeps = 2, 6
    Ta, Tb, G = _items(700 + D, n, 2, D)
    cfg = O.Config(D=D, r=r, sweeps=sweeps, tau_exponents=tuple(range(4, 9)))
    gs, RAs, RBs = [], [], []
    for i in range(n):
        qa, ra, qb, rb = _oracle_stage(Ta[i], Tb[i], G[i], cfg)
        g, _ = O.hermitise_repair(O.metric_raw(Ta[i], Tb[i], qa, qb, 2, D))
        gs.append(g); RAs.append(ra); RBs.append(rb)
    ctx = _ctx(D, r, sweeps=sweeps, precision=2, max_batch=n, kmin=4, kmax=8)
    K = D * r
    outs = {}
    for p in (0, 70, -70):
        gsc = np.stack(gs) * 2.0 ** p
        MA, MB = _empty((n, K, D)), _empty((n, K, D))
        info = torch.empty((n, 4), dtype=torch.float64, device="cuda")
        ctx.batch_als_dev(n, _dev(gsc), _dev(np.stack(RAs)), _dev(np.stack(RBs)), MA, MB, info)
        ctx.sync()
        outs[p] = (MA.cpu().numpy(), MB.cpu().numpy(), info.cpu().numpy())
    MA0, MB0, i0 = outs[0]
    for p in (70, -70):
        MA, MB, inf = outs[p]
        assert _rel(MA, MA0) < 1e-12 and _rel(MB, MB0) < 1e-12, p
        assert np.allclose(inf[:, 1], i0[:, 1], rtol=1e-12, atol=0), p
        assert np.allclose(inf[:, 0], i0[:, 0] * 2.0 ** p, rtol=1e-12, atol=0), p
    ctx.close()
