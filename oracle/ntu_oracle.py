"""Plain FP64 CPU oracle of the neighbourhood tensor update (NTU) bond update.

Dziarmaga, "Time evolution of an infinite projected entangled pair state: a
neighborhood tensor update", arXiv:2107.06635.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or call this module.
The CUDA library never imports, links or calls it and shares no code with it;
it exists to prove the CUDA path right.

Every step is written as the plain definition or the paper's algorithm step,
with numpy's einsum / svd / eigh / qr as library primitives and no fusion or
reordering beyond what the definition states.  All arithmetic is complex128.

Index conventions (readings of points the paper leaves open; the figures of
the paper are not available, only their captions):

* site tensor ``T[p, l, u, r, dn]``; ``p = s_phys * d_anc + s_anc``;
* two-site gate ``G[sA', sB', sA, sB]``;
* bond 0 is the horizontal bond A.r -- B.l, with A ("left role") at (0,0) and
  B ("right role") at (1,0).  The eight-site neighbourhood (Fig. 3(b)) is
  A, B and the six nearest neighbours L=(-1,0), TL=(0,1), BL=(0,-1) of B type
  and R=(2,0), TR=(1,1), BR=(1,-1) of A type; the internal bonds are
  L.r-A.l, TL.dn-A.u, BL.u-A.dn, B.r-R.l, TR.dn-B.u, BR.u-B.dn and the two
  bonds parallel to the updated one, TL.r-TR.l and BL.r-BR.l (Sec. II).  The
  14 remaining neighbour bond legs are closed by pairing ket with bra
  (Fig. 4(b));
* reduced matrices: the gated left tensor is the (d_p D^3) x (D r) matrix with
  rows (p, l, u, dn) and columns (r_leg, k); the gated right tensor has rows
  (p, r, u, dn) and columns (l_leg, k).  Both row orders are "(p, e, u, dn)"
  with e the horizontal leg pointing away from the bond;
* metric ``g[(kA', kB'), (kA, kB)]``: rows are bra indices, columns ket
  indices, kA slow, so that eps = x^dag g x with x = vec(M_A M_B^T - R_A R_B^T)
  (Eq. 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TIE_REL = 1e-14          # tolerance-selection tie window, relative to eps0
PIVOT_REL = 1e-10        # phase pivot: first entry within this of the largest
GATE_DROP_REL = 1e-15    # gate-split singular values below this x sigma_1 -> 0


@dataclass
class Config:
    D: int
    d: int = 2
    d_anc: int = 1
    r: int = 2
    sweeps: int = 10
    tau_exponents: tuple = field(default_factory=lambda: tuple(range(4, 16)))

    @property
    def d_p(self) -> int:
        return self.d * self.d_anc

    @property
    def taus(self):
        """Candidate relative pseudo-inverse tolerances 1e-k, largest first
        (parsed from their decimal form, i.e. correctly rounded)."""
        return [float("1e-%d" % k) for k in sorted(self.tau_exponents)]


# ---------------------------------------------------------------- helpers
def _es(*operands):
    """numpy einsum; pairwise contractions go through BLAS (a library
    primitive), which changes only the summation order."""
    return np.einsum(*operands, optimize=True)


def _phase_pivot(u: np.ndarray) -> complex:
    """Unit phase that makes the first entry of u whose modulus is within
    PIVOT_REL of the largest modulus real and positive (1 for u = 0)."""
    a = np.abs(u)
    m = a.max() if a.size else 0.0
    if m == 0.0:
        return 1.0 + 0.0j
    i = int(np.nonzero(a >= (1.0 - PIVOT_REL) * m)[0][0])
    return np.conj(u[i]) / a[i]


def svd_canonical(X: np.ndarray):
    """X = U diag(s) Vh with s descending and each left singular vector's
    phase fixed by ``_phase_pivot`` (the right one compensates)."""
    U, s, Vh = np.linalg.svd(X)
    U = U.copy()
    Vh = Vh.copy()
    for k in range(s.size):
        ph = _phase_pivot(U[:, k])
        U[:, k] *= ph
        Vh[k, :] *= np.conj(ph)
    return U, s, Vh


def svd_truncate(X: np.ndarray, D: int):
    """Leading D singular triples of X, zero-padded when X has fewer."""
    U, s, Vh = svd_canonical(X)
    m, n = X.shape
    Ut = np.zeros((m, D), dtype=np.complex128)
    st = np.zeros(D)
    Vt = np.zeros((D, n), dtype=np.complex128)
    k = min(D, s.size)
    Ut[:, :k] = U[:, :k]
    st[:k] = s[:k]
    Vt[:k] = Vh[:k]
    return Ut, st, Vt


# ---------------------------------------------------- Fig. 2(a): gate split
def gate_split(G: np.ndarray, r: int):
    """Split the two-site gate into G_A[sA', sA, k] and G_B[sB', sB, k]
    contracted over k < r (Fig. 2(a)).

    X[(sA', sA), (sB', sB)] = G[sA', sB', sA, sB] = U S V^dag;
    G_A[:, k] = sqrt(s_k) u_k and G_B[:, k] = (u_k^dag X) / sqrt(s_k), so that
    sum_k G_A G_B reproduces X whenever its rank is <= r.  Components with
    s_k <= 1e-15 s_1 are kept as exact zeros so that shapes stay fixed."""
    d = G.shape[0]
    X = G.transpose(0, 2, 1, 3).reshape(d * d, d * d)
    U, s, _ = np.linalg.svd(X)
    GA = np.zeros((d * d, r), dtype=np.complex128)
    GB = np.zeros((d * d, r), dtype=np.complex128)
    for k in range(min(r, s.size)):
        if s[k] <= GATE_DROP_REL * s[0]:
            continue
        u = U[:, k] * _phase_pivot(U[:, k])
        GA[:, k] = np.sqrt(s[k]) * u
        GB[:, k] = (u.conj() @ X) / np.sqrt(s[k])
    return GA.reshape(d, d, r), GB.reshape(d, d, r)


# ------------------------------------------- Fig. 2(a,b): apply gate and QR
def gated_matrix(T: np.ndarray, GX: np.ndarray, d_anc: int, side: str) -> np.ndarray:
    """T contracted with its half of the gate on the physical index, as the
    (d_p D^3) x (D r) matrix whose columns are the gated bond (leg, k)."""
    d_p, D = T.shape[0], T.shape[1]
    d = d_p // d_anc
    r = GX.shape[2]
    T6 = T.reshape(d, d_anc, D, D, D, D)            # [s, c, l, u, w=r, n=dn]
    if side == "left":   # rows (t, c, l, u, n), columns (w, k)
        M = _es("tsk,scluwn->tclunwk", GX, T6)
    else:                # rows (t, c, w, u, n), columns (l, k)
        M = _es("tsk,scluwn->tcwunlk", GX, T6)
    return M.reshape(d_p * D ** 3, D * r)


def qr_positive(M: np.ndarray):
    """Thin QR with real non-negative diag(R) (Fig. 2(b)); unique when M has
    full column rank."""
    Q, R = np.linalg.qr(M)
    Q = Q.copy()
    R = R.copy()
    for j in range(R.shape[0]):
        a = abs(R[j, j])
        ph = R[j, j] / a if a > 0 else 1.0
        Q[:, j] *= ph
        R[j, :] *= np.conj(ph)
    return Q, R


# -------------------------------------- Fig. 4(a,b): edge double tensors
def edge_tensors(Ta: np.ndarray, Tb: np.ndarray) -> dict:
    """Neighbour double tensors with their external ket/bra legs paired.

    Left-side neighbours are of the right-role type Tb, right-side ones of the
    left-role type Ta.  Four-index tensors are stored [x, y, x', y'] with
    (x, y) ket and (x', y') bra; x is the horizontal leg that crosses between
    the two halves (TL.r, BL.r, TR.l, BR.l) and y the vertical leg that
    touches the bond site."""
    c = np.conj
    return {
        # L: keeps r (touches A.l)
        "L": _es("pluxn,pluyn->xy", Tb, c(Tb)),
        # TL: keeps r (-> TR.l) and dn (touches A.u)
        "TL": _es("pluhv,plujw->hvjw", Tb, c(Tb)),
        # BL: keeps r (-> BR.l) and u (touches A.dn)
        "BL": _es("plvhn,plwjn->hvjw", Tb, c(Tb)),
        # R: keeps l (touches B.r)
        "R": _es("pxurn,pyurn->xy", Ta, c(Ta)),
        # TR: keeps l (-> TL.r) and dn (touches B.u)
        "TR": _es("phurv,pjurw->hvjw", Ta, c(Ta)),
        # BR: keeps l (-> BL.r) and u (touches B.dn)
        "BR": _es("phvrn,pjwrn->hvjw", Ta, c(Ta)),
    }


# ------------------------------ Fig. 4(c,d): double isometry + half network
def half_environment(Q: np.ndarray, E_side, E_top, E_bot, d_p: int, D: int):
    """One half of diagram 4(d): the isometry Q (rows (p, e, u, dn)) and its
    conjugate, closed by the side edge tensor on e and the top / bottom edge
    tensors on u / dn.  Returns H[hb, hb', ht, ht', k, k'] with k ket and k'
    bra."""
    K = Q.shape[1]
    Q5 = Q.reshape(d_p, D, D, D, K)                         # [p, e, u, n, k]
    Y = _es("peunk,ef->pfunk", Q5, E_side)            # side edge on e
    T1 = _es("pfunk,pfvml->unkvml", Y, np.conj(Q5))   # double isometry
    T2 = _es("unkvml,hujv->hjnkml", T1, E_top)        # top edge on u, u'
    H = _es("hjnkml,anbm->abhjkl", T2, E_bot)         # bottom edge on n, n'
    return H


def join(HL: np.ndarray, HR: np.ndarray) -> np.ndarray:
    """Contract the two halves over the crossing bonds TL.r-TR.l and
    BL.r-BR.l (ket and bra) into g[(kA', kB'), (kA, kB)] (Fig. 4(d,e))."""
    K = HL.shape[-1]
    g4 = _es("abhikl,abhijm->lmkj", HL, HR)   # [kA', kB', kA, kB]
    return g4.reshape(K * K, K * K)


def metric_raw(Ta, Tb, QA, QB, d_p: int, D: int) -> np.ndarray:
    """Exact NTU metric of the eight-site neighbourhood, before any repair."""
    E = edge_tensors(Ta, Tb)
    HL = half_environment(QA, E["L"], E["TL"], E["BL"], d_p, D)
    HR = half_environment(QB, E["R"], E["TR"], E["BR"], d_p, D)
    return join(HL, HR)


def hermitise_repair(g: np.ndarray):
    """g <- (g + g^dag)/2, clip negative eigenvalues to zero, normalise to
    unit trace.  The paper states that the exact g is Hermitian and
    non-negative to machine precision (Sec. II); the repair only removes
    rounding (FP64) or contraction noise (mixed precision).
    Returns (g, (herm_err, lam_min / lam_max, log(trace)))."""
    nrm = np.linalg.norm(g)
    herm_err = float(np.linalg.norm(g - g.conj().T) / nrm) if nrm > 0 else 0.0
    gh = 0.5 * (g + g.conj().T)
    lam, W = np.linalg.eigh(gh)
    ratio = float(lam[0] / lam[-1]) if lam[-1] > 0 else 0.0
    gr = (W * np.maximum(lam, 0.0)) @ W.conj().T
    tr = float(np.real(np.trace(gr)))
    return gr / tr, (herm_err, ratio, float(np.log(tr)))


# ------------------------------------------- Fig. 2(c,d) and Fig. 5, Eqs 2-4
def svdu_init(X0: np.ndarray, D: int):
    """Local SVD truncation: R_A R_B^T = U S V^dag, keep D, absorb sqrt(S)
    on both sides: M_A = U sqrt(S), M_B = conj(V) sqrt(S) (Fig. 2(c,d))."""
    U, s, Vh = svd_truncate(X0, D)
    rs = np.sqrt(s)
    return U * rs, Vh.T * rs


def reduced_problem_A(g: np.ndarray, gx0: np.ndarray, MB: np.ndarray):
    """Reduced metric g_A and source J_A of Fig. 5(b,c):
    eps(M_A) = m^dag g_A m - m^dag J_A - J_A^dag m + eps0, m = vec(M_A)."""
    K, D = MB.shape
    g4 = g.reshape(K, K, K, K)           # [i', j', i, j]
    gA = _es("ya,xyzw,wb->xazb", np.conj(MB), g4, MB)
    JA = _es("ya,xy->xa", np.conj(MB), gx0.reshape(K, K))
    return gA.reshape(K * D, K * D), JA.reshape(K * D)


def reduced_problem_B(g: np.ndarray, gx0: np.ndarray, MA: np.ndarray):
    """Same as ``reduced_problem_A`` with the roles of the two sides swapped."""
    K, D = MA.shape
    g4 = g.reshape(K, K, K, K)
    gB = _es("xa,xyzw,zb->yawb", np.conj(MA), g4, MA)
    JB = _es("xa,xy->ya", np.conj(MA), gx0.reshape(K, K))
    return gB.reshape(K * D, K * D), JB.reshape(K * D)


def pinv_select(gA: np.ndarray, JA: np.ndarray, eps0: float, taus):
    """M = pinv_tau(g_A) J_A with the tolerance chosen to minimise eps (Eq. 4).

    With g_A = W diag(lam) W^dag and y = W^dag J_A, the candidate for a relative
    tolerance tau keeps lam_i > tau lam_max: v = sum_kept w_i y_i / lam_i.
    Inserting v in Eq. 3 gives eps(tau) = eps0 - sum_kept |y_i|^2 / lam_i.
    The chosen tau is the largest one whose eps is within 1e-14 eps0 of the
    smallest eps over the grid.  Returns (v, tau, eps(tau))."""
    lam, W = np.linalg.eigh(gA)
    lmax = lam[-1]
    if not lmax > 0:
        return np.zeros_like(JA), taus[0], eps0
    y = W.conj().T @ JA
    eps = []
    for tau in taus:
        keep = lam > tau * lmax
        eps.append(eps0 - float(np.sum(np.abs(y[keep]) ** 2 / lam[keep])))
    emin = min(eps)
    j = next(i for i, e in enumerate(eps) if e <= emin + TIE_REL * eps0)
    keep = lam > taus[j] * lmax
    v = W[:, keep] @ (y[keep] / lam[keep])
    return v, taus[j], eps[j]


def als_truncate(g: np.ndarray, RA: np.ndarray, RB: np.ndarray, D: int,
                 sweeps: int, taus):
    """NTU truncation of the bond from D r to D (Fig. 5, Eqs. 2-5).

    Starts from the SVDU product, then repeats (tilt, optimise M_A, tilt,
    optimise M_B) for a fixed number of sweeps, and finally balances the pair
    by absorbing sqrt(S) on both sides.  Returns
    (M_A, M_B, eps, delta = eps / eps0, eps0, last chosen tau)."""
    K = RA.shape[0]
    X0 = RA @ RB.T
    x0 = X0.reshape(-1)
    gx0 = g @ x0
    eps0 = float(np.real(np.vdot(x0, gx0)))
    MA, MB = svdu_init(X0, D)
    tau = None
    for _ in range(sweeps):
        U, s, Vh = svd_truncate(MA @ MB.T, D)     # tilt: M_A = U S, M_B^T = V^dag
        MA, MB = U * s, Vh.T
        gA, JA = reduced_problem_A(g, gx0, MB)
        v, tau, _ = pinv_select(gA, JA, eps0, taus)
        MA = v.reshape(K, D)
        U, s, Vh = svd_truncate(MA @ MB.T, D)     # tilt: M_A = U, M_B^T = S V^dag
        MA, MB = U, Vh.T * s
        gB, JB = reduced_problem_B(g, gx0, MA)
        v, tau, _ = pinv_select(gB, JB, eps0, taus)
        MB = v.reshape(K, D)
    U, s, Vh = svd_truncate(MA @ MB.T, D)         # balance (Fig. 5(d))
    rs = np.sqrt(s)
    MA, MB = U * rs, Vh.T * rs
    x = (MA @ MB.T).reshape(-1) - x0
    eps = float(np.real(np.vdot(x, g @ x)))
    delta = eps / eps0 if eps0 > 0 else 0.0
    return MA, MB, eps, delta, eps0, tau


# ---------------------------------------------------- Fig. 2(e): recompose
def recompose(Q: np.ndarray, M: np.ndarray, d_p: int, D: int, side: str) -> np.ndarray:
    """A' = Q_A M_A (B' = Q_B M_B) put back into [p, l, u, r, dn] order and
    normalised to unit Frobenius norm."""
    T5 = (Q @ M).reshape(d_p, D, D, D, M.shape[1])     # [p, e, u, n, a]
    if side == "left":      # e = l, a = r
        T = T5.transpose(0, 1, 2, 4, 3)
    else:                   # e = r, a = l
        T = T5.transpose(0, 4, 2, 1, 3)
    T = np.ascontiguousarray(T)
    return T / np.linalg.norm(T)


# ------------------------------------------------------ one bond update
@dataclass
class BondInfo:
    eps: float
    delta: float
    eps0: float
    tau: float
    diag: tuple
    g: np.ndarray = None
    RA: np.ndarray = None
    RB: np.ndarray = None
    QA: np.ndarray = None
    QB: np.ndarray = None
    MA: np.ndarray = None
    MB: np.ndarray = None


def bond_update(Ta: np.ndarray, Tb: np.ndarray, G: np.ndarray, cfg: Config,
                keep: bool = False):
    """One NTU update of the bond Ta.r -- Tb.l (bond-0 orientation):
    gate split, apply + QR, exact eight-site metric, Hermitise/repair,
    SVDU initial guess, ALS sweeps, balance and recompose."""
    D, d_p = cfg.D, cfg.d_p
    GA, GB = gate_split(G, cfg.r)
    QA, RA = qr_positive(gated_matrix(Ta, GA, cfg.d_anc, "left"))
    QB, RB = qr_positive(gated_matrix(Tb, GB, cfg.d_anc, "right"))
    g, diag = hermitise_repair(metric_raw(Ta, Tb, QA, QB, d_p, D))
    MA, MB, eps, delta, eps0, tau = als_truncate(g, RA, RB, D, cfg.sweeps, cfg.taus)
    Ta2 = recompose(QA, MA, d_p, D, "left")
    Tb2 = recompose(QB, MB, d_p, D, "right")
    info = BondInfo(eps, delta, eps0, tau, diag)
    if keep:
        info.g, info.RA, info.RB, info.QA, info.QB = g, RA, RB, QA, QB
        info.MA, info.MB = MA, MB
    return Ta2, Tb2, info


# ----------------------------------------- the four bonds of the unit cell
def rotate(T: np.ndarray) -> np.ndarray:
    """Rotate the lattice clockwise by 90 degrees: new (l, u, r, dn) =
    old (dn, l, u, r)."""
    return np.ascontiguousarray(T.transpose(0, 4, 1, 2, 3))


def unrotate(T: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(T.transpose(0, 2, 3, 4, 1))


def update_bond(A: np.ndarray, B: np.ndarray, bond: int, G: np.ndarray,
                cfg: Config, keep: bool = False):
    """Bond b of the checkerboard cell is A's leg b in the order (r, u, l, dn):
    0: A.r-B.l, 1: A.u-B.dn, 2: A.l-B.r, 3: A.dn-B.u.  Vertical bonds are
    rotated to horizontal ones; bonds 2 and 3 put B in the left role, with the
    gate's site order swapped to match."""
    if bond in (1, 3):
        A, B = rotate(A), rotate(B)
    if bond in (0, 1):
        Ta2, Tb2, info = bond_update(A, B, G, cfg, keep)
        A, B = Ta2, Tb2
    else:
        Gs = np.ascontiguousarray(G.transpose(1, 0, 3, 2))
        Ta2, Tb2, info = bond_update(B, A, Gs, cfg, keep)
        B, A = Ta2, Tb2
    if bond in (1, 3):
        A, B = unrotate(A), unrotate(B)
    return A, B, info


def apply_site_gate(T: np.ndarray, O: np.ndarray, d_anc: int) -> np.ndarray:
    """Single-site gate on the physical factor of p, then unit norm."""
    d_p, D = T.shape[0], T.shape[1]
    d = d_p // d_anc
    T6 = T.reshape(d, d_anc, D, D, D, D)
    T6 = _es("ts,sclurn->tclurn", O, T6)
    T = np.ascontiguousarray(T6.reshape(T.shape))
    return T / np.linalg.norm(T)


def ntu_step(A, B, gates2, gate1, cfg: Config):
    """One second-order Trotter step: half single-site gates, the four bond
    gates in the order 0, 1, 2, 3, half single-site gates.  Returns
    (A, B, [delta per bond])."""
    if gate1 is not None:
        A, B = apply_site_gate(A, gate1, cfg.d_anc), apply_site_gate(B, gate1, cfg.d_anc)
    deltas = []
    for b in range(4):
        A, B, info = update_bond(A, B, b, gates2[b], cfg)
        deltas.append(info.delta)
    if gate1 is not None:
        A, B = apply_site_gate(A, gate1, cfg.d_anc), apply_site_gate(B, gate1, cfg.d_anc)
    return A, B, deltas


def measure(A, B, site: int, O: np.ndarray, d_anc: int) -> complex:
    """Cluster estimator of <O> on site A (0) or B (1): the site with O on its
    physical factor, closed by the leaf edge tensors of its four neighbours,
    divided by the same network with the identity."""
    T, N = (A, B) if site == 0 else (B, A)
    c = np.conj
    d_p = T.shape[0]
    El = _es("pluxn,pluyn->xy", N, c(N))   # neighbour left of T keeps r
    Eu = _es("plurx,plury->xy", N, c(N))   # neighbour above T keeps dn
    Er = _es("pxurn,pyurn->xy", N, c(N))   # neighbour right of T keeps l
    Ed = _es("plxrn,plyrn->xy", N, c(N))   # neighbour below T keeps u
    Of = np.kron(O, np.eye(d_anc))
    net = "qabce,qp,plurd,la,ub,rc,de->"
    num = _es(net, c(T), Of, T, El, Eu, Er, Ed)
    den = _es(net, c(T), np.eye(d_p), T, El, Eu, Er, Ed)
    return complex(num / den)


# ------------------------------------------ simple update (SU), Sec. II
# The SU keeps a diagonal bond tensor lambda_b (D positive values) on each
# of the four inequivalent bonds; its metric is g_SU = 1_d (x) 1_d (x)
# prod_j lambda_j over the six outer bonds of the updated pair (Sec. II).
# Reading: the site tensors are held in the symmetric gauge, each leg
# carrying sqrt(lambda) of its bond, so a pair contracted over its bond
# carries lambda_b once.  With sqrt(lambda) more on each outer leg the pair
# carries the full lambda_j there, g_SU becomes the plain Frobenius norm, and
# its minimiser is the local SVD truncation (Fig. 2(c,d)) of the weighted
# reduced matrices.
SU_BONDS_A = (2, 1, 0, 3)     # bond carried by A's legs (l, u, r, dn)
SU_BONDS_B = (0, 3, 2, 1)     # bond carried by B's legs (l, u, r, dn)
LAMBDA_CUT = 1e-14            # lambda_i <= this x max lambda counts as zero


def su_weight(T: np.ndarray, lam: np.ndarray, bonds, skip: int, power: float) -> np.ndarray:
    """T with each leg j in (l, u, r, dn) multiplied by lam[bonds[j]] ** power,
    except the leg on bond `skip`.  Negative powers are pseudo-inverses:
    values at or below LAMBDA_CUT x max give weight 0."""
    T = T.copy()
    for j, b in enumerate(bonds):
        if b == skip:
            continue
        lv = np.asarray(lam[b], dtype=np.float64)
        w = np.zeros_like(lv)
        ok = lv > LAMBDA_CUT * lv.max() if power < 0 else np.ones(lv.size, bool)
        w[ok] = lv[ok] ** power
        shape = [1] * 5
        shape[j + 1] = lv.size
        T = T * w.reshape(shape)
    return T


def su_bond_update(Ta: np.ndarray, Tb: np.ndarray, G: np.ndarray, cfg: Config):
    """SU of the bond Ta.r -- Tb.l (bond-0 orientation) for tensors whose
    outer legs already carry the full lambda: gate split, apply + QR
    (Fig. 2(a,b)), truncated SVD of R_A R_B^T keeping D values with sqrt(S)
    on both sides (Fig. 2(c,d)), recompose.  Returns (A', B', the kept
    singular values s_1..s_D, delta = sum_{i>D} s_i^2 / sum_i s_i^2, the
    error of the truncation in the metric g_SU relative to that of no
    update)."""
    D = cfg.D
    GA, GB = gate_split(G, cfg.r)
    QA, RA = qr_positive(gated_matrix(Ta, GA, cfg.d_anc, "left"))
    QB, RB = qr_positive(gated_matrix(Tb, GB, cfg.d_anc, "right"))
    X0 = RA @ RB.T
    s_all = np.linalg.svd(X0, compute_uv=False)
    U, s, Vh = svd_truncate(X0, D)
    rs = np.sqrt(s)
    MA, MB = U * rs, Vh.T * rs
    tot = float(np.sum(s_all ** 2))
    delta = float(np.sum(s_all[D:] ** 2)) / tot if tot > 0 else 0.0
    return (recompose(QA, MA, cfg.d_p, D, "left"), recompose(QB, MB, cfg.d_p, D, "right"),
            s, delta)


def su_update_bond(A, B, lam, bond: int, G: np.ndarray, cfg: Config):
    """Simple update of bond `bond` of the checkerboard cell (Sec. II), with
    the cell's orientation rules of ``update_bond``.  The three outer legs of
    each site are weighted by sqrt(lambda) (full lambda on the outer bonds),
    the pair is updated by ``su_bond_update``, the outer weights are removed
    again (pseudo-inverse), each tensor is normalised, and lambda_bond
    becomes the kept singular values normalised to unit 2-norm.  Returns
    (A', B', lam', delta)."""
    Aw = su_weight(A, lam, SU_BONDS_A, bond, 0.5)
    Bw = su_weight(B, lam, SU_BONDS_B, bond, 0.5)
    if bond in (1, 3):
        Aw, Bw = rotate(Aw), rotate(Bw)
    if bond in (0, 1):
        A2, B2, s, delta = su_bond_update(Aw, Bw, G, cfg)
    else:
        B2, A2, s, delta = su_bond_update(Bw, Aw, np.ascontiguousarray(G.transpose(1, 0, 3, 2)),
                                          cfg)
    if bond in (1, 3):
        A2, B2 = unrotate(A2), unrotate(B2)
    A2 = su_weight(A2, lam, SU_BONDS_A, bond, -0.5)
    B2 = su_weight(B2, lam, SU_BONDS_B, bond, -0.5)
    lam2 = [np.array(l, dtype=np.float64, copy=True) for l in lam]
    lam2[bond] = s / np.linalg.norm(s)
    return A2 / np.linalg.norm(A2), B2 / np.linalg.norm(B2), lam2, delta


def su_step(A, B, lam, gates2, gate1, cfg: Config):
    """One second-order Trotter step of the simple update: half single-site
    gates, the four bonds in the order 0, 1, 2, 3, half single-site gates.
    Returns (A, B, lam, [delta per bond])."""
    if gate1 is not None:
        A, B = apply_site_gate(A, gate1, cfg.d_anc), apply_site_gate(B, gate1, cfg.d_anc)
    deltas = []
    for b in range(4):
        A, B, lam, d = su_update_bond(A, B, lam, b, gates2[b], cfg)
        deltas.append(d)
    if gate1 is not None:
        A, B = apply_site_gate(A, gate1, cfg.d_anc), apply_site_gate(B, gate1, cfg.d_anc)
    return A, B, lam, deltas
