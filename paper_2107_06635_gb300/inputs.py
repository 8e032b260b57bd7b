"""Seeded synthetic inputs for NTU bond updates.

This module only *generates* inputs: random iPEPS site tensors, the Trotter
gates of the 2D transverse-field Ising model written in closed form, and
zero-padded product states.  It holds none of the bond-update arithmetic, so
both the CUDA library and the CPU oracle can be fed from it without sharing
any of the method's code.

Layout of a site tensor: ``T[p, l, u, r, dn]`` (row-major, ``dn`` fastest),
complex128, with ``p = s_phys * d_anc + s_anc`` when an ancilla is present.
Layout of a two-site gate: ``G[sA', sB', sA, sB]`` (d x d x d x d).

Random numbers come from numpy's PCG64 generator (``numpy.random.default_rng``),
whose stream is fixed by its published definition and identical on x86_64 and
aarch64.
"""
from __future__ import annotations

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def pauli(name: str) -> np.ndarray:
    return {"I": _I2, "X": _X, "Y": _Y, "Z": _Z}[name].copy()


def two_site(op: np.ndarray) -> np.ndarray:
    """A 4x4 operator on (sA, sB) as the tensor G[sA', sB', sA, sB]."""
    return np.ascontiguousarray(op.reshape(2, 2, 2, 2))


def zz_gate(theta: float) -> np.ndarray:
    """exp(-i theta Z(x)Z) = cos(theta) 1 - i sin(theta) Z(x)Z, since (Z(x)Z)^2 = 1."""
    zz = np.kron(_Z, _Z)
    return two_site(np.cos(theta) * np.eye(4) - 1j * np.sin(theta) * zz)


def zz_gate_imag(a: float) -> np.ndarray:
    """exp(+a Z(x)Z) = cosh(a) 1 + sinh(a) Z(x)Z (real imaginary-time gate)."""
    zz = np.kron(_Z, _Z)
    return two_site(np.cosh(a) * np.eye(4) + np.sinh(a) * zz)


def heisenberg_gate(theta: float) -> np.ndarray:
    """exp(-i theta (XX+YY+ZZ)); XX+YY+ZZ = 2 SWAP - 1 and SWAP^2 = 1, so
    the gate is exp(i theta) (cos(2 theta) 1 - i sin(2 theta) SWAP).
    Its operator-Schmidt rank is 4."""
    swap = np.zeros((4, 4), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            swap[b * 2 + a, a * 2 + b] = 1.0
    m = np.exp(1j * theta) * (np.cos(2 * theta) * np.eye(4) - 1j * np.sin(2 * theta) * swap)
    return two_site(m)


def identity_gate(d: int = 2) -> np.ndarray:
    return two_site(np.eye(d * d, dtype=np.complex128)) if d == 2 else \
        np.ascontiguousarray(np.eye(d * d, dtype=np.complex128).reshape(d, d, d, d))


def random_gate(rng: np.random.Generator, d: int = 2) -> np.ndarray:
    """A random two-site unitary (QR of a complex Gaussian matrix); its
    operator-Schmidt spectrum is generically non-degenerate."""
    m = rng.standard_normal((d * d, d * d)) + 1j * rng.standard_normal((d * d, d * d))
    q, r = np.linalg.qr(m)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    return np.ascontiguousarray(q.reshape(d, d, d, d))


def x_rotation(phi: float) -> np.ndarray:
    """exp(+i phi X) = cos(phi) 1 + i sin(phi) X (single-site real-time gate)."""
    return np.cos(phi) * _I2 + 1j * np.sin(phi) * _X


def x_rotation_imag(a: float) -> np.ndarray:
    """exp(+a X) = cosh(a) 1 + sinh(a) X (single-site imaginary-time gate)."""
    return np.cosh(a) * _I2 + np.sinh(a) * _X


def tfim_real_time_gates(h: float, dt: float):
    """Second-order Trotter gates of U = exp(-i H dt) for
    H = -sum ZZ - h sum X: four bond gates exp(+i dt ZZ) and the single-site
    half step exp(+i h dt/2 X)."""
    g2 = zz_gate(-dt)
    return [g2.copy() for _ in range(4)], x_rotation(h * dt / 2)


def tfim_imag_time_gates(h: float, dbeta: float):
    """Second-order Trotter gates of exp(-dbeta H / 2) for the same H."""
    g2 = zz_gate_imag(dbeta / 2)
    return [g2.copy() for _ in range(4)], x_rotation_imag(h * dbeta / 4)


def random_site_tensor(rng: np.random.Generator, d_p: int, D: int,
                       dtype=np.complex128) -> np.ndarray:
    """iid N(0,1) real and imaginary parts, normalised to unit Frobenius norm."""
    shape = (d_p, D, D, D, D)
    t = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    t /= np.linalg.norm(t)
    return np.ascontiguousarray(t.astype(dtype))


def random_pair(seed: int, d_p: int, D: int, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    return random_site_tensor(rng, d_p, D, dtype), random_site_tensor(rng, d_p, D, dtype)


def integer_site_tensor(rng: np.random.Generator, d_p: int, D: int, lo: int = -3,
                        hi: int = 3) -> np.ndarray:
    """Small-integer complex tensor: every product and partial sum of the
    environment contraction stays an exact integer in FP64."""
    shape = (d_p, D, D, D, D)
    t = rng.integers(lo, hi + 1, shape) + 1j * rng.integers(lo, hi + 1, shape)
    return np.ascontiguousarray(t.astype(np.complex128))


def sparse_integer_array(rng: np.random.Generator, shape, density: float) -> np.ndarray:
    """Complex array with real and imaginary parts in {-1, 0, 1}, each entry
    kept with probability `density` (else 0)."""
    v = rng.integers(-1, 2, shape) + 1j * rng.integers(-1, 2, shape)
    keep = rng.random(shape) < density
    return np.ascontiguousarray((v * keep).astype(np.complex128))


def product_state(psi: np.ndarray, D: int, d_anc: int = 1) -> np.ndarray:
    """A D=1 product state zero-padded to bond dimension D:
    T[p, 0, 0, 0, 0] = psi[p], all other entries 0."""
    psi = np.asarray(psi, dtype=np.complex128).reshape(-1)
    t = np.zeros((psi.size, D, D, D, D), dtype=np.complex128)
    t[:, 0, 0, 0, 0] = psi
    return t


def plus_x_state(D: int) -> np.ndarray:
    return product_state(np.array([1, 1]) / np.sqrt(2), D)


def plus_z_state(D: int) -> np.ndarray:
    return product_state(np.array([1, 0]), D)


def quench_start(D: int, mix: float = 1e-2, seed: int = 123):
    """Initial (A, B) of the transverse-field quench: the polarised state
    |+x> zero-padded to bond dimension D plus a seeded random admixture of
    relative weight `mix`, which lifts the exact zero modes of the padded
    bonds (with mix=0 the pair is the bare padded product state)."""
    rng = np.random.default_rng(seed)
    A = plus_x_state(D)
    B = plus_x_state(D)
    if mix:
        A = A + mix * random_site_tensor(rng, 2, D)
        B = B + mix * random_site_tensor(rng, 2, D)
    return A / np.linalg.norm(A), B / np.linalg.norm(B)


def purification_state(D: int) -> np.ndarray:
    """Infinite-temperature purification: (|00> + |11>)/sqrt(2) on
    (physical, ancilla) at every site, p = s_phys * 2 + s_anc."""
    psi = np.zeros(4)
    psi[0] = psi[3] = 1 / np.sqrt(2)
    return product_state(psi, D, d_anc=2)


def batch_items(seed: int, n: int, d_p: int, D: int, gate: np.ndarray,
                dtype=np.complex128):
    """n independent bond-update items (Ta, Tb, G), stacked along axis 0."""
    rng = np.random.default_rng(seed)
    ta = np.empty((n, d_p, D, D, D, D), dtype=dtype)
    tb = np.empty_like(ta)
    for i in range(n):
        ta[i] = random_site_tensor(rng, d_p, D, dtype)
        tb[i] = random_site_tensor(rng, d_p, D, dtype)
    g = np.broadcast_to(gate, (n,) + gate.shape).copy()
    return ta, tb, g


def uneven_batch(seed: int, n: int, d_p: int = 2, theta: float = 0.01):
    """Uneven batch: D uniform in {3..8}, r uniform in {2, 4}; r=2 items
    carry exp(-i theta ZZ), r=4 items exp(-i theta (XX+YY+ZZ)).
    Site tensors are complex64 draws widened exactly to complex128."""
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(n):
        D = int(rng.integers(3, 9))
        r = int(rng.choice([2, 4]))
        ta = random_site_tensor(rng, d_p, D, np.complex64).astype(np.complex128)
        tb = random_site_tensor(rng, d_p, D, np.complex64).astype(np.complex128)
        g = zz_gate(theta) if r == 2 else heisenberg_gate(theta)
        items.append((D, r, ta, tb, g))
    return items


# ------------------------------------- real Hermitian iPEPO (thermal states)
def operator_basis():
    """The Hermitian operator basis of one spin-1/2 site, O^a for
    a = 0, 1, 2, 3: sigma_x, sigma_y, sigma_z, 1.  Tr(O^a O^b) = 2 delta_ab."""
    return [_X.copy(), _Y.copy(), _Z.copy(), _I2.copy()]


def superoperator_two_site(G: np.ndarray) -> np.ndarray:
    """The real tensor S[a', b', a, b] with
    G (O^a (x) O^b) G^dag = sum_{a'b'} S[a', b', a, b] O^a' (x) O^b',
    i.e. S = Tr((O^a' (x) O^b') G (O^a (x) O^b) G^dag) / 4 (orthogonality of
    the basis).  G is a 4 x 4 operator on (sA, sB); S is returned in the
    two-site gate layout [sA', sB', sA, sB] with d = 4."""
    Ob = operator_basis()
    S = np.zeros((4, 4, 4, 4))
    for a in range(4):
        for b in range(4):
            M = G @ np.kron(Ob[a], Ob[b]) @ G.conj().T
            for a2 in range(4):
                for b2 in range(4):
                    S[a2, b2, a, b] = np.real(np.trace(np.kron(Ob[a2], Ob[b2]) @ M)) / 4.0
    return S.astype(np.complex128)


def superoperator_one_site(U: np.ndarray) -> np.ndarray:
    """s[a', a] = Tr(O^a' U O^a U^dag) / 2: the action O -> U O U^dag on the
    coefficients of one site."""
    Ob = operator_basis()
    s = np.zeros((4, 4))
    for a in range(4):
        M = U @ Ob[a] @ U.conj().T
        for a2 in range(4):
            s[a2, a] = np.real(np.trace(Ob[a2] @ M)) / 2.0
    return s.astype(np.complex128)


def ipepo_thermal_gates(h: float, dbeta: float):
    """Second-order Trotter gates of rho(beta/2) -> e^{-dbeta H/4} rho e^{-dbeta H/4}
    for H = -sum ZZ - h sum X, acting on the coefficients of the real
    iPEPO: four bond gates, the superoperator of G = 1 + tanh(dbeta/4) Z(x)Z
    (proportional to e^{dbeta ZZ/4}), and the single-site half step, the
    superoperator of e^{h dbeta X/8}."""
    G = np.eye(4) + np.tanh(dbeta / 4) * np.kron(_Z, _Z)
    S2 = superoperator_two_site(G)
    s1 = superoperator_one_site(x_rotation_imag(h * dbeta / 8))
    return [S2.copy() for _ in range(4)], s1


def ipepo_identity(D: int) -> np.ndarray:
    """rho(0) = 1 at every site (coefficients (0, 0, 0, 1)), zero-padded to
    bond dimension D."""
    return product_state(np.array([0.0, 0.0, 0.0, 1.0]), D)


def ipepo_observable(O: np.ndarray) -> np.ndarray:
    """The 4 x 4 matrix M[a', a] = Tr(O^a' O O^a) / 2 that, put on one site of
    the coefficient network, turns its norm sum_a c_a^2 (= Tr(rho^2) / 2 per
    site) into Tr(rho O rho) / 2: with it the cluster estimator of a real
    iPEPO rho(beta/2) gives <O> = Tr(rho(beta) O) / Tr rho(beta), since
    rho(beta) = rho(beta/2)^2."""
    Ob = operator_basis()
    M = np.zeros((4, 4), dtype=np.complex128)
    for a2 in range(4):
        for a in range(4):
            M[a2, a] = np.trace(Ob[a2] @ O @ Ob[a]) / 2.0
    return M


def ipepo_start(D: int, mix: float = 1e-2, seed: int = 88):
    """Initial (A, B) of a thermal iPEPO run: rho(0) = 1 zero-padded to D plus
    a seeded real random admixture of relative weight `mix` (which lifts the
    exact zero modes of the padded bonds), each normalised; real."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        t = rng.standard_normal((4, D, D, D, D))
        t = ipepo_identity(D) + mix * t / np.linalg.norm(t)
        out.append(np.ascontiguousarray(t / np.linalg.norm(t)))
    return out[0], out[1]
