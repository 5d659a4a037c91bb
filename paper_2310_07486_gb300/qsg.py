"""Python binding of the C ABI in ``include/qsg.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the sm_103a kernels of
``libqsg.so``.  PyTorch provides the device workspace and the CUDA stream.
If the library cannot be loaded the binding raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libqsg.so")
_lib = None

METROPOLIS, HEATBATH = 0, 1
PBC, APBC = 0, 1
OPT_SWEEP_KERNEL, OPT_CHUNK, OPT_WAVEFRONT_VARIANT, OPT_CORR_KERNEL, OPT_PERSISTENT, OPT_GRAPH, OPT_ONETIME, OPT_TAIL = \
    1, 2, 3, 4, 5, 6, 7, 8
OPT_WAIT_LIMIT = 9
OPT_UNITS_PER_BLOCK = 10
CORR_TENSOR, CORR_INTEGER = 0, 1
SWEEP_AUTO, SWEEP_REFERENCE, SWEEP_WAVEFRONT = 0, 1, 2

STATUS = {0: "ok", -1: "invalid argument", -2: "invalid group shape", -3: "CUDA runtime error",
          -4: "bounded device wait gave up", -5: "call out of order", -6: "workspace missing or too small"}


class QSGError(RuntimeError):
    def __init__(self, status, what, detail=""):
        super().__init__("%s failed: %s%s" % (what, STATUS.get(status, status), (" (" + detail + ")") if detail else ""))
        self.status = status


class qsg_shape(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("Ltau", ctypes.c_int32), ("n_samples", ctypes.c_int32),
                ("n_replicas", ctypes.c_int32), ("n_k", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("boundary", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def load_library(path: str | None = None):
    """Load libqsg.so (building it first with nvcc if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, u32, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
    lib.qsg_workspace_bytes.restype = sz
    lib.qsg_workspace_bytes.argtypes = [vp, i32]
    lib.qsg_create.restype = i32
    lib.qsg_create.argtypes = [ctypes.POINTER(vp), vp, i32, vp, sz, vp]
    lib.qsg_destroy.restype = None
    lib.qsg_destroy.argtypes = [vp]
    lib.qsg_set_stream.restype = i32
    lib.qsg_set_stream.argtypes = [vp, vp]
    lib.qsg_init_samples.restype = i32
    lib.qsg_init_samples.argtypes = [vp, u64, vp]
    lib.qsg_set_couplings.restype = i32
    lib.qsg_set_couplings.argtypes = [vp, i32, vp]
    lib.qsg_sweep.restype = i32
    lib.qsg_sweep.argtypes = [vp, i32]
    lib.qsg_tempering_swap.restype = i32
    lib.qsg_tempering_swap.argtypes = [vp]
    lib.qsg_measure_correlators.restype = i32
    lib.qsg_measure_correlators.argtypes = [vp]
    lib.qsg_read_correlators.restype = i32
    lib.qsg_read_correlators.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.qsg_read_correlators_async.restype = i32
    lib.qsg_read_correlators_async.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.qsg_wait_correlators.restype = i32
    lib.qsg_wait_correlators.argtypes = [vp]
    lib.qsg_read_energies.restype = i32
    lib.qsg_read_onetime.argtypes = [vp, i32, vp, vp, vp]
    lib.qsg_read_onetime.restype = i32
    lib.qsg_read_energies.argtypes = [vp, i32, vp]
    lib.qsg_read_pair_overlaps.restype = i32
    lib.qsg_read_pair_overlaps.argtypes = [vp, i32, vp]
    lib.qsg_sample_features.restype = i32
    lib.qsg_sample_features.argtypes = [vp, i32, vp]
    lib.qsg_mlp_param_count.restype = i32
    lib.qsg_mlp_param_count.argtypes = []
    lib.qsg_mlp_workspace_bytes.restype = sz
    lib.qsg_mlp_workspace_bytes.argtypes = [ctypes.c_int64, i32]
    lib.qsg_mlp_create.restype = i32
    lib.qsg_mlp_create.argtypes = [ctypes.POINTER(vp), vp, sz, ctypes.c_int64, i32, vp]
    lib.qsg_mlp_destroy.restype = None
    lib.qsg_mlp_destroy.argtypes = [vp]
    for name in ("qsg_mlp_set_params", "qsg_mlp_get_params"):
        getattr(lib, name).restype = i32
        getattr(lib, name).argtypes = [vp, vp]
    lib.qsg_mlp_set_data.restype = i32
    lib.qsg_mlp_set_data.argtypes = [vp, vp, vp, ctypes.c_int64]
    lib.qsg_mlp_grad.restype = i32
    lib.qsg_mlp_grad.argtypes = [vp, vp, i32, vp, vp]
    lib.qsg_mlp_train.restype = i32
    lib.qsg_mlp_train.argtypes = [vp, vp, i32, i32, ctypes.c_float, vp]
    lib.qsg_mlp_predict.restype = i32
    lib.qsg_mlp_predict.argtypes = [vp, vp, ctypes.c_int64, i32, vp]
    lib.qsg_judge.restype = i32
    lib.qsg_judge.argtypes = [vp, vp, i32, i32, i32, i32, i32, ctypes.c_double, vp]
    lib.qsg_fit_correlators.restype = i32
    lib.qsg_fit_correlators.argtypes = [vp, vp, i32, ctypes.c_int64, i32, i32, vp]
    lib.qsg_tau_tilde.restype = None
    lib.qsg_tau_tilde.argtypes = [i32, vp]
    lib.qsg_read_accepts.restype = i32
    lib.qsg_read_accepts.argtypes = [vp, i32, vp]
    lib.qsg_get_spins.restype = i32
    lib.qsg_get_spins.argtypes = [vp, i32, vp]
    lib.qsg_set_spins.restype = i32
    lib.qsg_set_spins.argtypes = [vp, i32, vp]
    lib.qsg_get_spins_device.restype = i32
    lib.qsg_get_spins_device.argtypes = [vp, i32, vp]
    lib.qsg_set_spins_device.restype = i32
    lib.qsg_set_spins_device.argtypes = [vp, i32, vp]
    lib.qsg_get_counters.restype = i32
    lib.qsg_get_counters.argtypes = [vp, vp, vp, vp]
    lib.qsg_set_counters.restype = i32
    lib.qsg_set_counters.argtypes = [vp, u32, u32, ctypes.c_int64]
    lib.qsg_sweep_static_scratch.restype = i32
    lib.qsg_sweep_static_scratch.argtypes = [vp, vp, vp, vp, i32, vp, u64, u32, i32, vp]
    lib.qsg_set_option.restype = i32
    lib.qsg_set_option.argtypes = [vp, i32, ctypes.c_int64]
    lib.qsg_kernel_launches.restype = ctypes.c_uint64
    lib.qsg_kernel_launches.argtypes = []
    lib.qsg_strerror.restype = ctypes.c_char_p
    lib.qsg_strerror.argtypes = [i32]
    lib.qsg_last_cuda_error.restype = ctypes.c_char_p
    lib.qsg_last_cuda_error.argtypes = [vp]
    _lib = lib
    return lib


def exported_symbols():
    return ["qsg_workspace_bytes", "qsg_create", "qsg_destroy", "qsg_set_stream", "qsg_init_samples",
            "qsg_set_couplings", "qsg_sweep", "qsg_tempering_swap", "qsg_measure_correlators",
            "qsg_read_correlators", "qsg_read_correlators_async", "qsg_wait_correlators", "qsg_read_energies", "qsg_read_accepts", "qsg_get_spins", "qsg_set_spins",
            "qsg_get_spins_device", "qsg_set_spins_device",
            "qsg_get_counters", "qsg_set_counters", "qsg_set_option", "qsg_sweep_static_scratch", "qsg_kernel_launches", "qsg_strerror", "qsg_last_cuda_error"]


def qsg_sweep_static_scratch(spins, Jx, Jy, shape: "Shape", group_id, ladder, seed, first_sweep, n_sweeps,
                             stream=None):
    """Sweeps on caller-owned device buffers (torch tensors of 64-bit words)
    without any device allocation by the library.

    The C entry point cannot see the sizes of the buffers, so they are checked
    here: int64, contiguous, on the stream's device, spins of
    slots * L_tau * L * L words and couplings of words * L * L words each."""
    import torch
    lad = np.ascontiguousarray(np.asarray(ladder, dtype=np.float64).ravel())
    sh = shape.c()
    st = stream if stream is not None else torch.cuda.current_stream()
    want = {"spins": shape.slots * shape.Ltau * shape.L * shape.L, "Jx": shape.words * shape.L * shape.L,
            "Jy": shape.words * shape.L * shape.L}
    for name, t in (("spins", spins), ("Jx", Jx), ("Jy", Jy)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int64 and t.is_contiguous()):
            raise QSGError(-1, "qsg_sweep_static_scratch", "%s must be a contiguous int64 CUDA tensor" % name)
        if t.device != st.device:
            raise QSGError(-1, "qsg_sweep_static_scratch", "%s is not on the stream's device" % name)
        if t.numel() != want[name]:
            raise QSGError(-1, "qsg_sweep_static_scratch", "%s holds %d words, the shape needs %d"
                           % (name, t.numel(), want[name]))
    if lad.size != shape.n_k:
        raise QSGError(-1, "qsg_sweep_static_scratch", "ladder has %d values, n_k is %d" % (lad.size, shape.n_k))
    status = load_library().qsg_sweep_static_scratch(
        ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(Jx.data_ptr()), ctypes.c_void_p(Jy.data_ptr()),
        ctypes.byref(sh), int(group_id), _ptr(lad), int(seed) & ((1 << 64) - 1), int(first_sweep), int(n_sweeps),
        ctypes.c_void_p(st.cuda_stream))
    if status != 0:
        raise QSGError(status, "qsg_sweep_static_scratch")


def qsg_kernel_launches() -> int:
    return int(load_library().qsg_kernel_launches())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Shape:
    L: int
    Ltau: int
    n_samples: int
    n_replicas: int
    n_k: int
    algo: int = METROPOLIS
    boundary: int = PBC

    def c(self):
        return qsg_shape(self.L, self.Ltau, self.n_samples, self.n_replicas, self.n_k, self.algo, self.boundary, 0)

    @property
    def words(self):
        return (self.n_samples + 63) // 64

    @property
    def slots(self):
        return self.words * self.n_replicas * self.n_k

    @property
    def n_lag(self):
        return self.Ltau // 2 + 1


def _shape_array(shapes):
    arr = (qsg_shape * len(shapes))()
    for i, s in enumerate(shapes):
        arr[i] = s.c()
    return arr


def qsg_workspace_bytes(shapes) -> int:
    arr = _shape_array(shapes)
    return int(load_library().qsg_workspace_bytes(ctypes.cast(arr, ctypes.c_void_p), len(shapes)))


class Context:
    """A qsg_ctx over a torch-allocated device workspace.

    Methods map one-to-one onto the C entry points of the same name.
    """

    def __init__(self, shapes, device=None, stream=None):
        import torch
        self.lib = load_library()
        self.shapes = list(shapes)
        self._arr = _shape_array(self.shapes)
        nbytes = qsg_workspace_bytes(self.shapes)
        if nbytes == 0:
            raise QSGError(-2, "qsg_workspace_bytes")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        # torch's caching allocator returns blocks aligned to at least 512 bytes
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._pending_out = []  # host buffers of asynchronous reads not yet waited for
        h = ctypes.c_void_p()
        st = self._check(self.lib.qsg_create(ctypes.byref(h), ctypes.cast(self._arr, ctypes.c_void_p), len(self.shapes),
                                             ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                             ctypes.c_void_p(self.stream.cuda_stream)), "qsg_create", ctx=False)
        self.h = h

    def _check(self, status, what, ctx=True):
        if status != 0:
            detail = ""
            if ctx and status == -3:
                detail = self.lib.qsg_last_cuda_error(self.h).decode()
            raise QSGError(status, what, detail)
        return status

    def close(self):
        if getattr(self, "h", None):
            self.lib.qsg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- calls ----------------------------------------------------------
    def qsg_set_stream(self, stream):
        self.stream = stream
        self._check(self.lib.qsg_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "qsg_set_stream")

    def qsg_init_samples(self, seed, ladders):
        lad = np.ascontiguousarray(np.concatenate([np.asarray(l, dtype=np.float64).ravel() for l in ladders]))
        self._check(self.lib.qsg_init_samples(self.h, int(seed) & ((1 << 64) - 1), _ptr(lad)), "qsg_init_samples")

    def qsg_set_couplings(self, group, J):
        J = np.ascontiguousarray(J, dtype=np.int8)
        self._check(self.lib.qsg_set_couplings(self.h, group, _ptr(J)), "qsg_set_couplings")

    def qsg_sweep(self, n=1):
        self._check(self.lib.qsg_sweep(self.h, int(n)), "qsg_sweep")

    def qsg_tempering_swap(self):
        self._check(self.lib.qsg_tempering_swap(self.h), "qsg_tempering_swap")

    def qsg_measure_correlators(self):
        self._check(self.lib.qsg_measure_correlators(self.h), "qsg_measure_correlators")

    def correlator_buffers(self, group=0, pinned=False):
        """Host arrays C, Q2 [R][n_samples][K][L_tau/2+1] and q2 [n_samples][K]
        for qsg_read_correlators(out=...); page-locked (torch pin_memory) when
        pinned, so that the device copies run at DMA speed."""
        s = self.shapes[group]
        shp = (s.n_replicas, s.n_samples, s.n_k, s.n_lag)
        if pinned:
            import torch
            mk = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
        else:
            mk = lambda shape: np.empty(shape)
        return dict(C=mk(shp), Q2=mk(shp), q2=mk((s.n_samples, s.n_k)))

    def qsg_read_correlators(self, group=0, raw=False, out=None):
        """C, Q2 and q2 of one group; `out` (from correlator_buffers) receives
        them in place instead of new arrays."""
        s = self.shapes[group]
        shp = (s.n_replicas, s.n_samples, s.n_k, s.n_lag)
        if out is None:
            C = np.zeros(shp)
            Q = np.zeros(shp)
            P = np.zeros((s.n_samples, s.n_k))
        else:
            C, Q, P = out["C"], out["Q2"], out["q2"]
            for a, want in ((C, shp), (Q, shp), (P, (s.n_samples, s.n_k))):
                if a.shape != want or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("qsg_read_correlators: out arrays must be C-contiguous float64 of shape %s" % (want,))
        nc = int(np.prod(shp))
        R = np.zeros(2 * nc + s.n_samples * s.n_k, dtype=np.int64) if raw else None
        self._check(self.lib.qsg_read_correlators(self.h, group, _ptr(C), _ptr(Q), _ptr(P),
                                                  None if R is None else _ptr(R)), "qsg_read_correlators")
        out = dict(C=C, Q2=Q, q2=P)
        if raw:
            out.update(C_raw=R[:nc].reshape(shp), Q2_raw=R[nc:2 * nc].reshape(shp),
                       q2_raw=R[2 * nc:].reshape(s.n_samples, s.n_k))
        return out

    def qsg_read_correlators_async(self, out, stream, group=0):
        """Queues the finish of one group on the context's stream and the
        copies into `out` (from correlator_buffers, pinned for overlap) on
        `stream` (a torch.cuda.Stream or a raw cudaStream_t other than the
        context's); returns at once.  `out` holds the results after
        qsg_wait_correlators(); this object keeps it referenced until then."""
        s = self.shapes[group]
        shp = (s.n_replicas, s.n_samples, s.n_k, s.n_lag)
        C, Q, P = out["C"], out["Q2"], out["q2"]
        for a, want in ((C, shp), (Q, shp), (P, (s.n_samples, s.n_k))):
            if a.shape != want or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("qsg_read_correlators_async: out arrays must be C-contiguous float64 of shape %s"
                                 % (want,))
        raw_stream = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.qsg_read_correlators_async(self.h, group, _ptr(C), _ptr(Q), _ptr(P), None,
                                                        ctypes.c_void_p(int(raw_stream))),
                    "qsg_read_correlators_async")
        self._pending_out.append(out)

    def qsg_wait_correlators(self):
        """Waits for the copies of the last qsg_read_correlators_async;
        raises on the device flag as qsg_read_correlators does."""
        try:
            self._check(self.lib.qsg_wait_correlators(self.h), "qsg_wait_correlators")
        finally:
            self._pending_out = []

    ONETIME_SAMPLE_FIELDS = ("q2", "q4", "chi2", "F2", "chi3", "F3", "chi_lin")
    ONETIME_K_FIELDS = ("chi2", "F2", "xi2", "chi3", "F3", "xi3", "B", "chi_lin")

    def qsg_read_onetime(self, group=0):
        s = self.shapes[group]
        H = s.L // 2
        ps = np.zeros((s.n_samples, s.n_k, 7))
        pk = np.zeros((s.n_k, 8))
        raw = np.zeros((s.n_samples, s.n_k, 4 + 2 * (H + 1)), dtype=np.int64)
        self._check(self.lib.qsg_read_onetime(self.h, group, _ptr(ps), _ptr(pk), _ptr(raw)), "qsg_read_onetime")
        out = {f: ps[..., i] for i, f in enumerate(self.ONETIME_SAMPLE_FIELDS)}
        out["per_k"] = {f: pk[:, i] for i, f in enumerate(self.ONETIME_K_FIELDS)}
        out["raw"] = raw
        return out

    def qsg_read_pair_overlaps(self, group=0):
        s = self.shapes[group]
        out = np.zeros((s.n_samples, s.n_k, s.n_replicas * (s.n_replicas - 1) // 2), dtype=np.int64)
        self._check(self.lib.qsg_read_pair_overlaps(self.h, group, _ptr(out)), "qsg_read_pair_overlaps")
        return out

    def qsg_sample_features(self, group=0):
        s = self.shapes[group]
        out = np.zeros((s.n_samples, 64), dtype=np.float32)
        self._check(self.lib.qsg_sample_features(self.h, group, _ptr(out)), "qsg_sample_features")
        return out

    def qsg_read_energies(self, group=0):
        s = self.shapes[group]
        E = np.zeros((s.n_samples, s.n_replicas, s.n_k), dtype=np.int64)
        self._check(self.lib.qsg_read_energies(self.h, group, _ptr(E)), "qsg_read_energies")
        return E

    def qsg_read_accepts(self, group=0):
        s = self.shapes[group]
        A = np.zeros((s.n_samples, max(s.n_k - 1, 1)), dtype=np.int64)
        self._check(self.lib.qsg_read_accepts(self.h, group, _ptr(A)), "qsg_read_accepts")
        return A

    def qsg_get_spins(self, group=0):
        s = self.shapes[group]
        out = np.zeros((s.slots, s.Ltau, s.L, s.L), dtype=np.uint64)
        self._check(self.lib.qsg_get_spins(self.h, group, _ptr(out)), "qsg_get_spins")
        return out

    def qsg_set_spins(self, group, words):
        words = np.ascontiguousarray(words, dtype=np.uint64)
        self._check(self.lib.qsg_set_spins(self.h, group, _ptr(words)), "qsg_set_spins")

    def _check_device_words(self, group, t, what):
        import torch
        s = self.shapes[group]
        n = s.slots * s.Ltau * s.L * s.L
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int64 and t.is_contiguous()
                and t.numel() == n and t.device == self.device):
            raise QSGError(-1, what, "need a contiguous int64 tensor of %d words on %s" % (n, self.device))

    def qsg_get_spins_device(self, group, out):
        """Spin words into a device tensor (int64, the layout of qsg_get_spins),
        ordered on the context's stream, no host wait."""
        self._check_device_words(group, out, "qsg_get_spins_device")
        self._check(self.lib.qsg_get_spins_device(self.h, group, ctypes.c_void_p(out.data_ptr())),
                    "qsg_get_spins_device")

    def qsg_set_spins_device(self, group, words):
        """Spin words from a device tensor, ordered on the context's stream."""
        self._check_device_words(group, words, "qsg_set_spins_device")
        self._check(self.lib.qsg_set_spins_device(self.h, group, ctypes.c_void_p(words.data_ptr())),
                    "qsg_set_spins_device")

    def qsg_get_counters(self):
        a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
        self._check(self.lib.qsg_get_counters(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                    "qsg_get_counters")
        return a.value, b.value, c.value


    def qsg_set_option(self, option, value):
        self._check(self.lib.qsg_set_option(self.h, int(option), int(value)), "qsg_set_option")

    def qsg_set_counters(self, sweeps, swaps, n_meas=-1):
        self._check(self.lib.qsg_set_counters(self.h, int(sweeps), int(swaps), int(n_meas)), "qsg_set_counters")


class MLP:
    """A qsg_mlp over a torch-allocated device workspace; methods map onto
    the qsg_mlp_* entry points."""

    def __init__(self, n_data, max_batch, device=None, stream=None):
        import torch
        self.lib = load_library()
        nbytes = int(self.lib.qsg_mlp_workspace_bytes(int(n_data), int(max_batch)))
        if nbytes == 0:
            raise QSGError(-1, "qsg_mlp_workspace_bytes")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        st = self.lib.qsg_mlp_create(ctypes.byref(h), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                     int(n_data), int(max_batch), ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise QSGError(st, "qsg_mlp_create")
        self.h = h
        self.n_params = int(self.lib.qsg_mlp_param_count())

    def _check(self, st, what):
        if st != 0:
            raise QSGError(st, what)

    def close(self):
        if getattr(self, "h", None):
            self.lib.qsg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.n_params
        self._check(self.lib.qsg_mlp_set_params(self.h, _ptr(theta)), "qsg_mlp_set_params")

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        self._check(self.lib.qsg_mlp_get_params(self.h, _ptr(out)), "qsg_mlp_get_params")
        return out

    def set_data(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        self._keep = (X, T)
        self._check(self.lib.qsg_mlp_set_data(self.h, _ptr(X), _ptr(T), X.shape[0]), "qsg_mlp_set_data")

    def grad(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(self.lib.qsg_mlp_grad(self.h, _ptr(idx), idx.size, ctypes.byref(loss), _ptr(g)), "qsg_mlp_grad")
        return float(loss.value), g

    def train(self, idx, lr):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        steps, batch = idx.shape
        losses = np.zeros(steps, dtype=np.float32)
        self._check(self.lib.qsg_mlp_train(self.h, _ptr(idx), steps, batch, float(lr), _ptr(losses)),
                    "qsg_mlp_train")
        return losses

    def predict(self, X, bf16=True):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros((X.shape[0], 33), dtype=np.float32)
        self._check(self.lib.qsg_mlp_predict(self.h, _ptr(X), X.shape[0], 1 if bf16 else 0, _ptr(Y)),
                    "qsg_mlp_predict")
        return Y


def qsg_judge(E_bins, q_bins, n_last=3, n_sigma=2.0):
    """First passing bin per sample (-1 if none); E_bins [nb][ns][R][K],
    q_bins [nb][ns][K][pairs]."""
    E = np.ascontiguousarray(E_bins, dtype=np.float64)
    q = np.ascontiguousarray(q_bins, dtype=np.float64)
    nb, ns, R, K = E.shape
    assert q.shape == (nb, ns, K, R * (R - 1) // 2)
    out = np.zeros(ns, dtype=np.int32)
    st = load_library().qsg_judge(_ptr(E), _ptr(q), nb, ns, R, K, int(n_last), float(n_sigma), _ptr(out))
    if st != 0:
        raise QSGError(st, "qsg_judge")
    return out


class qsg_fit_result(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("C_ok", "C_tau_w", "C_tau_min", "Q_ok", "Q_tau_w", "Q_tau_min",
                                                "Q_n_exp", "plateau_ok")] + \
               [(n, ctypes.c_double) for n in ("eta", "eta_err", "C_amp", "C_chi2dof", "Q_pl", "Q_pl_err",
                                                 "plateau_chi2dof", "eta_e", "eta_e_err", "eta_2", "Q_chi2dof")]


def qsg_fit_correlators(C, Q2, Ltau, boundary=PBC):
    """Fits of every series of C, Q2 [R][n_series][L_tau/2+1] (the layout of
    qsg_read_correlators with the sample and k axes merged); list of dicts."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    Q2 = np.ascontiguousarray(Q2, dtype=np.float64)
    R, n = C.shape[0], int(np.prod(C.shape[1:-1]))
    out = (qsg_fit_result * max(n, 1))()
    st = load_library().qsg_fit_correlators(_ptr(C), _ptr(Q2), R, n, int(Ltau), int(boundary),
                                             ctypes.cast(out, ctypes.c_void_p))
    if st != 0:
        raise QSGError(st, "qsg_fit_correlators")
    return [{f: getattr(out[i], f) for f, _ in qsg_fit_result._fields_} for i in range(n)]


def qsg_tau_tilde(Ltau):
    out = np.zeros(Ltau // 2 + 1)
    load_library().qsg_tau_tilde(int(Ltau), _ptr(out))
    return out


# ---- host-side layout helpers (no method arithmetic) -----------------------
def unpack_spins(words: np.ndarray, shape: Shape) -> np.ndarray:
    """uint64 words [slots][Ltau][L][L] -> int8 spins [n_samples][R][K][Ltau][L][L]."""
    W, R, K = shape.words, shape.n_replicas, shape.n_k
    w = words.reshape(W, R, K, shape.Ltau, shape.L, shape.L)
    out = np.empty((shape.n_samples, R, K, shape.Ltau, shape.L, shape.L), dtype=np.int8)
    for b in range(shape.n_samples):
        bits = (w[b // 64] >> np.uint64(b % 64)) & np.uint64(1)
        out[b] = (1 - 2 * bits.astype(np.int8))
    return out


def pack_spins(spins: np.ndarray, shape: Shape) -> np.ndarray:
    """int8 spins [n_samples][R][K][Ltau][L][L] -> uint64 words (padding bits 0)."""
    W = shape.words
    words = np.zeros((W, shape.n_replicas, shape.n_k, shape.Ltau, shape.L, shape.L), dtype=np.uint64)
    for b in range(shape.n_samples):
        bit = (spins[b] < 0).astype(np.uint64) << np.uint64(b % 64)
        words[b // 64] |= bit
    return words.reshape(shape.slots, shape.Ltau, shape.L, shape.L)
