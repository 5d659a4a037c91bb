"""Plain CPU oracle of the Monte Carlo hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never links or calls
it, and the two share no code.

The arithmetic lives in ``qsg_oracle.c`` (int8 spins, one site at a time); this
module compiles it with gcc and wraps it with ctypes.  What each function
computes, with the section / equation of the paper it follows, is stated at the
top of the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            vp, i32, u32, u64, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
            L.orc_philox.argtypes = [vp, vp, vp]
            L.orc_create.restype = vp
            L.orc_create.argtypes = [i32] * 9
            L.orc_destroy.argtypes = [vp]
            L.orc_init.restype = i32
            L.orc_init.argtypes = [vp, u64, vp, i32, vp]
            L.orc_sweep.argtypes = [vp, i32]
            L.orc_energy.argtypes = [vp, vp]
            L.orc_swap.argtypes = [vp]
            L.orc_measure.argtypes = [vp]
            L.orc_read.argtypes = [vp] * 7
            L.orc_measure_one.argtypes = [vp, i32, i32, i32, vp, vp]
            L.orc_read_onetime.argtypes = [vp, vp, vp, vp]
            L.orc_read_pair_overlaps.argtypes = [vp, vp]
            L.orc_get_spins.argtypes = [vp, vp]
            L.orc_set_spins.argtypes = [vp, vp]
            L.orc_get_couplings.argtypes = [vp, vp]
            L.orc_get_tables.argtypes = [vp, vp, vp]
            L.orc_pt_threshold.restype = u64
            L.orc_pt_threshold.argtypes = [vp, i32, i32, i64]
            L.orc_get_accepts.argtypes = [vp, vp]
            L.orc_get_sweep.restype = u32
            L.orc_get_sweep.argtypes = [vp]
            L.orc_get_swaps.restype = u32
            L.orc_get_swaps.argtypes = [vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(counter, key):
    """Philox4x32-10 of a 4-word counter and a 2-word key -> 4 uint32."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


class OracleGroup:
    """One group of disorder samples of equal (L, L_tau) simulated by the oracle.

    Arrays returned use the layouts of the C file:
      spins      int8  [n_samples][R][K][L_tau][L][L]   (configuration at ladder j)
      couplings  int8  [n_samples][2][L][L]             ([0]: +x bond, [1]: +y bond)
      energies   int64 [n_samples][R][K]                (action E of Eq. Trotter-action)
      C, Q2      float64 [R][n_samples][K][L_tau/2+1]
      q2         float64 [n_samples][K]
    """

    def __init__(self, L, Ltau, n_samples, n_replicas, n_k, algo="metropolis", boundary="pbc", group_id=0,
                 first_sample=0):
        self.L, self.Ltau, self.n_samples, self.R, self.K = L, Ltau, n_samples, n_replicas, n_k
        self.algo = {"metropolis": 0, "heatbath": 1}[algo] if isinstance(algo, str) else int(algo)
        self.boundary = {"pbc": 0, "apbc": 1}[boundary] if isinstance(boundary, str) else int(boundary)
        self.group_id = group_id
        self.first_sample = first_sample
        self._h = lib().orc_create(L, Ltau, n_samples, n_replicas, n_k, self.algo, self.boundary, group_id,
                                   first_sample)
        if not self._h:
            raise ValueError("oracle: invalid shape")
        self.n_lag = Ltau // 2 + 1

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init(self, seed, ladder, couplings=None):
        lad = np.ascontiguousarray(ladder, dtype=np.float64)
        per_sample = 1 if lad.ndim == 2 else 0
        J = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.int8)
        rc = lib().orc_init(self._h, int(seed), _ptr(lad), per_sample, None if J is None else _ptr(J))
        if rc != 0:
            raise ValueError("oracle: invalid ladder")
        self._keep = (lad, J)

    def sweep(self, n=1):
        lib().orc_sweep(self._h, int(n))

    def energies(self):
        E = np.zeros((self.n_samples, self.R, self.K), dtype=np.int64)
        lib().orc_energy(self._h, _ptr(E))
        return E

    def swap(self):
        lib().orc_swap(self._h)

    def measure(self):
        lib().orc_measure(self._h)

    def measure_one(self, b, r, j):
        C = np.zeros(self.n_lag, dtype=np.int64)
        Q = np.zeros(self.n_lag, dtype=np.int64)
        lib().orc_measure_one(self._h, b, r, j, _ptr(C), _ptr(Q))
        return C, Q

    def read(self):
        shp = (self.R, self.n_samples, self.K, self.n_lag)
        C = np.zeros(shp); Q = np.zeros(shp); P = np.zeros((self.n_samples, self.K))
        Cr = np.zeros(shp, dtype=np.int64); Qr = np.zeros(shp, dtype=np.int64)
        Pr = np.zeros((self.n_samples, self.K), dtype=np.int64)
        lib().orc_read(self._h, _ptr(C), _ptr(Q), _ptr(P), _ptr(Cr), _ptr(Qr), _ptr(Pr))
        return dict(C=C, Q2=Q, q2=P, C_raw=Cr, Q2_raw=Qr, q2_raw=Pr)

    ONETIME_SAMPLE_FIELDS = ("q2", "q4", "chi2", "F2", "chi3", "F3", "chi_lin")
    ONETIME_K_FIELDS = ("chi2", "F2", "xi2", "chi3", "F3", "xi3", "B", "chi_lin")

    def read_onetime(self):
        """One-time observables: per (sample, k) and disorder-averaged per k,
        plus the raw integer sums (P4 as a Python int of 128 bits)."""
        H = self.L // 2
        ps = np.zeros((self.n_samples, self.K, 7))
        pk = np.zeros((self.K, 8))
        raw = np.zeros((self.n_samples, self.K, 4 + 2 * (H + 1)), dtype=np.int64)
        lib().orc_read_onetime(self._h, _ptr(ps), _ptr(pk), _ptr(raw))
        out = {f: ps[..., i] for i, f in enumerate(self.ONETIME_SAMPLE_FIELDS)}
        out["per_k"] = {f: pk[:, i] for i, f in enumerate(self.ONETIME_K_FIELDS)}
        out["raw"] = raw
        out["P4"] = [[int(raw[b, j, 1].astype(np.uint64)) + (int(raw[b, j, 2].astype(np.uint64)) << 64)
                      for j in range(self.K)] for b in range(self.n_samples)]
        return out

    def read_pair_overlaps(self):
        out = np.zeros((self.n_samples, self.K, self.R * (self.R - 1) // 2), dtype=np.int64)
        lib().orc_read_pair_overlaps(self._h, _ptr(out))
        return out

    def spins(self):
        S = np.zeros((self.n_samples, self.R, self.K, self.Ltau, self.L, self.L), dtype=np.int8)
        lib().orc_get_spins(self._h, _ptr(S))
        return S

    def set_spins(self, S):
        S = np.ascontiguousarray(S, dtype=np.int8)
        assert S.shape == (self.n_samples, self.R, self.K, self.Ltau, self.L, self.L)
        lib().orc_set_spins(self._h, _ptr(S))

    def couplings(self):
        J = np.zeros((self.n_samples, 2, self.L, self.L), dtype=np.int8)
        lib().orc_get_couplings(self._h, _ptr(J))
        return J

    def tables(self):
        Tm = np.zeros((self.n_samples, self.K, 3), dtype=np.uint32)
        Th = np.zeros((self.n_samples, self.K, 7), dtype=np.uint32)
        lib().orc_get_tables(self._h, _ptr(Tm), _ptr(Th))
        return Tm, Th

    def pt_threshold(self, b, i, n):
        return int(lib().orc_pt_threshold(self._h, b, i, int(n)))

    def accepts(self):
        A = np.zeros((self.n_samples, max(self.K - 1, 1)), dtype=np.int64)
        lib().orc_get_accepts(self._h, _ptr(A))
        return A

    @property
    def sweep_count(self):
        return int(lib().orc_get_sweep(self._h))

    @property
    def swap_count(self):
        return int(lib().orc_get_swaps(self._h))
