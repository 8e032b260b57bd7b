"""Thin ctypes binding of the NTU C ABI (include/ntu.h).

Argument marshalling only: every step of a bond update runs in the CUDA
library.  Host arrays are numpy complex128; device arrays are torch tensors
(complex128 or float64 views) or raw integer device pointers.  There is no
CPU fallback: if the library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

NTU_FP64, NTU_MIXED_FP32, NTU_MIXED_BF16X3 = 0, 1, 2
STATUS = {0: "NTU_OK", 1: "NTU_EINVAL", 2: "NTU_ENOMEM", 3: "NTU_ECUDA", 4: "NTU_ENUMERIC",
          5: "NTU_ETIMEOUT", 6: "NTU_EUNSUPPORTED", 7: "NTU_ESTATE"}


class NTUError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Tuning(ctypes.Structure):
    _fields_ = [("t12_pair", ctypes.c_int), ("als_ctas_per_sm", ctypes.c_int),
                ("als_split", ctypes.c_int), ("als_build", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Config(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("d_phys", ctypes.c_int), ("d_anc", ctypes.c_int),
                ("r", ctypes.c_int), ("als_sweeps", ctypes.c_int), ("precision", ctypes.c_int),
                ("tau_kmin", ctypes.c_int), ("tau_kmax", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("wait_budget", ctypes.c_int)]


_LIB = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)

# name -> argument types; every function returns int except the *_last_error ones
_SIGS = {
    "ntu_init": [ctypes.POINTER(Config), _P, ctypes.POINTER(_P)],
    "ntu_destroy": [_P],
    "ntu_last_error": [_P],
    "ntu_sync": [_P],
    "ntu_set_state": [_P, _P, _P],
    "ntu_get_state": [_P, _P, _P],
    "ntu_apply_gate": [_P, _I, _P, _P, _P],
    "ntu_env_metric": [_P, _I, _P, _P],
    "ntu_als_truncate": [_P, _I, _P, _P, _P],
    "ntu_step": [_P, _P, _P, _P],
    "ntu_measure": [_P, _I, _P, _P],
    "ntu_su_set_lambdas": [_P, _P],
    "ntu_su_get_lambdas": [_P, _P],
    "ntu_su_update": [_P, _I, _P, _P],
    "ntu_su_step": [_P, _P, _P, _P],
    "ntu_batch_update_dev": [_P, _I, _P, _P, _P, _P, _P, _P],
    "ntu_batch_update_host": [_P, _I, _P, _P, _P, _P, _P, _P],
    "ntu_batch_gate_qr_dev": [_P, _I, _P, _P, _P, _P, _P, _P, _P],
    "ntu_batch_env_dev": [_P, _I, _P, _P, _P, _P, _P],
    "ntu_batch_repair_dev": [_P, _I, _P, _P],
    "ntu_batch_als_dev": [_P, _I, _P, _P, _P, _P, _P, _P],
    "ntu_batch_recompose_dev": [_P, _I, _P, _P, _P, _P, _P, _P],
    "ntu_last_launch_count": [_P],
    "ntu_inject_wait_timeout": [_P, _I],
    "ntu_set_tuning": [_P, ctypes.POINTER(Tuning)],
    "ntu_get_tuning": [_P, ctypes.POINTER(Tuning), _P],
    "ntu_set_graphs": [_P, _I],
    "ntu_uneven_set_tuning": [_P, _I, ctypes.POINTER(Tuning)],
    "ntu_uneven_get_tuning": [_P, _I, ctypes.POINTER(Tuning), _P],
    "ntu_set_profiling": [_P, _I],
    "ntu_stage_times": [_P, _P],
    "ntu_solver_paths": [_P, _P],
    "ntu_gate_qr_noalloc": [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P],
    "ntu_uneven_init": [_I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, ctypes.POINTER(_P)],
    "ntu_uneven_update_host": [_P, _I, _P, _P, _P, _P, _P, _P, _P, _I],
    "ntu_uneven_stage": [_P, _I, _P, _P, _P, _P],
    "ntu_uneven_run": [_P, _I],
    "ntu_uneven_sync": [_P],
    "ntu_uneven_fetch": [_P, _I, _P, _P, _P, _P],
    "ntu_uneven_last_launch_count": [_P],
    "ntu_uneven_destroy": [_P],
    "ntu_uneven_last_error": [_P],
}


def header_symbols():
    """Function names declared in include/ntu.h."""
    path = os.path.join(os.path.dirname(_build.HERE), "include", "ntu.h")
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(ntu_\w+)\s*\(", text, re.M)))


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed) the CUDA library."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.LIB
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name.endswith("last_error") else ctypes.c_int
    _LIB = lib
    return lib


def _ptr(x) -> int:
    """Address of a numpy array, torch tensor or integer pointer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "host arrays must be C-contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "device tensors must be contiguous"
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


class Context:
    """One NTU context: a (D, d, r) configuration, its device work space and a
    two-site unit cell."""

    def __init__(self, D: int, d: int = 2, d_anc: int = 1, r: int = 2, sweeps: int = 10,
                 precision: int = NTU_FP64, tau_kmin: int = 4, tau_kmax: int = 15,
                 max_batch: int = 1, stream=None, wait_budget: int = 0):
        self.lib = load()
        self.cfg = Config(D, d, d_anc, r, sweeps, precision, tau_kmin, tau_kmax, max_batch,
                          wait_budget)
        self.D, self.d, self.d_anc, self.r = D, d, d_anc, r
        self.d_p = d * d_anc
        self.K = D * r
        self.max_batch = max_batch
        h = _P()
        st = self.lib.ntu_init(ctypes.byref(self.cfg), stream, ctypes.byref(h))
        if st != 0:
            raise NTUError(st, self.lib.ntu_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.ntu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _ck(self, st: int):
        if st != 0:
            raise NTUError(st, self.lib.ntu_last_error(self.h).decode())

    @property
    def site_shape(self):
        return (self.d_p, self.D, self.D, self.D, self.D)

    # ---- unit cell -------------------------------------------------------
    def set_state(self, A, B):
        A, B = _c128(A), _c128(B)
        assert A.shape == self.site_shape and B.shape == self.site_shape
        self._ck(self.lib.ntu_set_state(self.h, _ptr(A), _ptr(B)))

    def get_state(self):
        A = np.empty(self.site_shape, np.complex128)
        B = np.empty(self.site_shape, np.complex128)
        self._ck(self.lib.ntu_get_state(self.h, _ptr(A), _ptr(B)))
        return A, B

    def apply_gate(self, bond: int, gate):
        G = _c128(gate)
        RA = np.empty((self.K, self.K), np.complex128)
        RB = np.empty((self.K, self.K), np.complex128)
        self._ck(self.lib.ntu_apply_gate(self.h, bond, _ptr(G), _ptr(RA), _ptr(RB)))
        return RA, RB

    def env_metric(self, bond: int):
        n = self.K * self.K
        g = np.empty((n, n), np.complex128)
        diag = np.empty(3)
        self._ck(self.lib.ntu_env_metric(self.h, bond, _ptr(g), _ptr(diag)))
        return g, diag

    def als_truncate(self, bond: int):
        out = np.empty(3)
        v = [ctypes.c_double() for _ in range(3)]
        self._ck(self.lib.ntu_als_truncate(self.h, bond, *(ctypes.addressof(x) for x in v)))
        out[:] = [x.value for x in v]
        return {"eps": out[0], "delta": out[1], "tau": out[2]}

    def step(self, gates2, gate1_half=None):
        G = _c128(np.stack([_c128(g) for g in gates2]))
        g1 = None if gate1_half is None else _c128(gate1_half)
        deltas = np.empty(4)
        self._ck(self.lib.ntu_step(self.h, _ptr(G), _ptr(g1), _ptr(deltas)))
        return deltas

    # ---- simple update (Sec. II) ----------------------------------------
    def su_set_lambdas(self, lam):
        L = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(4, self.D))
        self._ck(self.lib.ntu_su_set_lambdas(self.h, _ptr(L)))

    def su_get_lambdas(self):
        L = np.empty((4, self.D))
        self._ck(self.lib.ntu_su_get_lambdas(self.h, _ptr(L)))
        return L

    def su_update(self, bond: int, gate) -> float:
        G = _c128(gate)
        d = ctypes.c_double()
        self._ck(self.lib.ntu_su_update(self.h, bond, _ptr(G), ctypes.addressof(d)))
        return d.value

    def su_step(self, gates2, gate1_half=None):
        G = _c128(np.stack([_c128(g) for g in gates2]))
        g1 = None if gate1_half is None else _c128(gate1_half)
        deltas = np.empty(4)
        self._ck(self.lib.ntu_su_step(self.h, _ptr(G), _ptr(g1), _ptr(deltas)))
        return deltas

    def measure(self, site: int, op) -> complex:
        O = _c128(op)
        v = np.empty(1, np.complex128)
        self._ck(self.lib.ntu_measure(self.h, site, _ptr(O), _ptr(v)))
        return complex(v[0])

    def sync(self):
        self._ck(self.lib.ntu_sync(self.h))

    # ---- batches ----------------------------------------------------------
    def batch_update_host(self, Ta, Tb, gates):
        Ta, Tb, G = _c128(Ta), _c128(Tb), _c128(gates)
        n = Ta.shape[0]
        Ta_out = np.empty_like(Ta)
        Tb_out = np.empty_like(Tb)
        info = np.empty((n, 4))
        self._ck(self.lib.ntu_batch_update_host(self.h, n, _ptr(Ta), _ptr(Tb), _ptr(G),
                                                _ptr(Ta_out), _ptr(Tb_out), _ptr(info)))
        return Ta_out, Tb_out, info

    def batch_update_dev(self, n, Ta, Tb, gates, Ta_out, Tb_out, info):
        self._ck(self.lib.ntu_batch_update_dev(self.h, n, _ptr(Ta), _ptr(Tb), _ptr(gates),
                                               _ptr(Ta_out), _ptr(Tb_out), _ptr(info)))

    def batch_gate_qr_dev(self, n, Ta, Tb, gates, QA, RA, QB, RB):
        self._ck(self.lib.ntu_batch_gate_qr_dev(self.h, n, _ptr(Ta), _ptr(Tb), _ptr(gates),
                                                _ptr(QA), _ptr(RA), _ptr(QB), _ptr(RB)))

    def batch_env_dev(self, n, Ta, Tb, QA, QB, g):
        self._ck(self.lib.ntu_batch_env_dev(self.h, n, _ptr(Ta), _ptr(Tb), _ptr(QA), _ptr(QB),
                                            _ptr(g)))

    def batch_repair_dev(self, n, g, diag):
        self._ck(self.lib.ntu_batch_repair_dev(self.h, n, _ptr(g), _ptr(diag)))

    def batch_als_dev(self, n, g, RA, RB, MA, MB, info):
        self._ck(self.lib.ntu_batch_als_dev(self.h, n, _ptr(g), _ptr(RA), _ptr(RB), _ptr(MA),
                                            _ptr(MB), _ptr(info)))

    def batch_recompose_dev(self, n, QA, QB, MA, MB, Ta_out, Tb_out):
        self._ck(self.lib.ntu_batch_recompose_dev(self.h, n, _ptr(QA), _ptr(QB), _ptr(MA),
                                                  _ptr(MB), _ptr(Ta_out), _ptr(Tb_out)))

    def set_tuning(self, t12_pair: int = -1, als_ctas_per_sm: int = 0, als_split: int = 0,
                   als_build: int = 0):
        t = Tuning(t12_pair, als_ctas_per_sm, als_split, als_build)
        self._ck(self.lib.ntu_set_tuning(self.h, ctypes.byref(t)))

    def get_tuning(self):
        t = Tuning()
        smax = ctypes.c_int()
        self._ck(self.lib.ntu_get_tuning(self.h, ctypes.byref(t), ctypes.addressof(smax)))
        return t.as_dict(), smax.value

    def set_graphs(self, on: bool = True):
        self._ck(self.lib.ntu_set_graphs(self.h, 1 if on else 0))

    def inject_wait_timeout(self, on: bool = True):
        self._ck(self.lib.ntu_inject_wait_timeout(self.h, 1 if on else 0))

    def last_launch_count(self) -> int:
        return self.lib.ntu_last_launch_count(self.h)

    def set_profiling(self, on: bool = True):
        self._ck(self.lib.ntu_set_profiling(self.h, 1 if on else 0))

    def stage_times(self):
        """Durations (ms) of the last update's stages: gate+QR, environment,
        repair, ALS, recompose."""
        ms = np.empty(5)
        self._ck(self.lib.ntu_stage_times(self.h, _ptr(ms)))
        return ms

    def solver_paths(self):
        """Counts since the last call: ALS solves certified by Gershgorin
        discs (CG solve), by shifted Cholesky (refinement solve), ALS eigen
        solves; metrics certified PD by Gershgorin discs, by Cholesky, and
        metrics eigen-repaired; QRs by double-FP32 CholeskyQR2 and by
        Householder."""
        c = np.zeros(8, dtype=np.int32)
        self._ck(self.lib.ntu_solver_paths(self.h, _ptr(c)))
        return {"als_gershgorin": int(c[0]), "als_cholesky": int(c[1]), "als_eigen": int(c[2]),
                "repair_gershgorin": int(c[3]), "repair_cholesky": int(c[4]),
                "repair_eigen": int(c[5]), "qr_cholesky2": int(c[6]),
                "qr_householder": int(c[7])}


class UnevenBatch:
    """Independent bond updates of different (D, r) in one call: one context
    and stream per kind, forked from and joined back into one stream;
    optionally replayed as one CUDA graph."""

    def __init__(self, kinds, max_items, d: int = 2, d_anc: int = 1, sweeps: int = 10,
                 precision: int = NTU_FP64, tau_kmin: int = 4, tau_kmax: int = 15, stream=None):
        self.lib = load()
        self.kinds = [tuple(k) for k in kinds]
        self.d, self.d_anc = d, d_anc
        self.precision = precision
        n = len(self.kinds)
        Ds = (ctypes.c_int * n)(*[k[0] for k in self.kinds])
        rs = (ctypes.c_int * n)(*[k[1] for k in self.kinds])
        caps = (ctypes.c_int * n)(*[int(m) for m in max_items])
        h = _P()
        st = self.lib.ntu_uneven_init(d, d_anc, sweeps, precision, tau_kmin, tau_kmax, n,
                                      ctypes.cast(Ds, _P), ctypes.cast(rs, _P),
                                      ctypes.cast(caps, _P), stream, ctypes.byref(h))
        if st != 0:
            raise NTUError(st, self.lib.ntu_uneven_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.ntu_uneven_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    GROUPED, GRAPH, PER_ITEM = 0, 1, 2

    def _ck(self, st):
        if st != 0:
            raise NTUError(st, self.lib.ntu_uneven_last_error(self.h).decode())

    def _pack(self, items):
        index = {k: i for i, k in enumerate(self.kinds)}
        kind = np.array([index[(it[0], it[1])] for it in items], dtype=np.int32)
        ta = np.ascontiguousarray(np.concatenate([np.asarray(it[2], np.complex128).ravel() for it in items]))
        tb = np.ascontiguousarray(np.concatenate([np.asarray(it[3], np.complex128).ravel() for it in items]))
        gg = np.ascontiguousarray(np.stack([np.asarray(it[4], np.complex128) for it in items]))
        return kind, ta, tb, gg

    @staticmethod
    def _unpack(items, oa, ob):
        outs_a, outs_b, o = [], [], 0
        for it in items:
            sz = np.asarray(it[2]).size
            outs_a.append(oa[o:o + sz].reshape(np.asarray(it[2]).shape))
            outs_b.append(ob[o:o + sz].reshape(np.asarray(it[3]).shape))
            o += sz
        return outs_a, outs_b

    def update(self, items, use_graph: bool = False):
        """items: list of (D, r, Ta, Tb, G) with complex128 arrays.  Returns
        (list of Ta', list of Tb', info n x 4)."""
        n = len(items)
        kind, ta, tb, gg = self._pack(items)
        oa, ob = np.empty_like(ta), np.empty_like(tb)
        info = np.empty((n, 4))
        self._ck(self.lib.ntu_uneven_update_host(self.h, n, _ptr(kind), _ptr(ta), _ptr(tb), _ptr(gg),
                                                 _ptr(oa), _ptr(ob), _ptr(info), 1 if use_graph else 0))
        return (*self._unpack(items, oa, ob), info)

    def stage(self, items):
        """Copy the items to the device; they stay there for run()."""
        kind, ta, tb, gg = self._pack(items)
        self._ck(self.lib.ntu_uneven_stage(self.h, len(items), _ptr(kind), _ptr(ta), _ptr(tb),
                                           _ptr(gg)))

    def run(self, mode: int = 0):
        """Enqueue the update of the staged items (GROUPED, GRAPH or
        PER_ITEM); asynchronous."""
        self._ck(self.lib.ntu_uneven_run(self.h, mode))

    def sync(self):
        self._ck(self.lib.ntu_uneven_sync(self.h))

    def fetch(self, items):
        """Results of the staged items (the same list that was staged)."""
        kind, ta, tb, _ = self._pack(items)
        oa, ob = np.empty_like(ta), np.empty_like(tb)
        info = np.empty((len(items), 4))
        self._ck(self.lib.ntu_uneven_fetch(self.h, len(items), _ptr(kind), _ptr(oa), _ptr(ob),
                                           _ptr(info)))
        return (*self._unpack(items, oa, ob), info)

    def last_launch_count(self) -> int:
        return self.lib.ntu_uneven_last_launch_count(self.h)

    def set_tuning(self, kind: int, t12_pair: int = -1, als_ctas_per_sm: int = 0,
                   als_split: int = 0, als_build: int = 0):
        t = Tuning(t12_pair, als_ctas_per_sm, als_split, als_build)
        self._ck(self.lib.ntu_uneven_set_tuning(self.h, kind, ctypes.byref(t)))

    def get_tuning(self, kind: int):
        t = Tuning()
        smax = ctypes.c_int()
        self._ck(self.lib.ntu_uneven_get_tuning(self.h, kind, ctypes.byref(t),
                                                ctypes.addressof(smax)))
        return t.as_dict(), smax.value

    def split_max(self, kind: int) -> int:
        return self.get_tuning(kind)[1]
