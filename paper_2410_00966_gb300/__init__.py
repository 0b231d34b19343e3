"""Python binding of the mmcq library (GB300 / sm_103a LLG + cavity-QED hot path).

Thin ctypes layer over the C ABI declared in include/mmcq.h: the module-level
``mmcq_*`` functions are the C entry points with their C names and argument
lists; ``Sim`` wraps a handle for convenience (numpy arrays are passed as host
pointers, CUDA torch tensors as device pointers).  Every step of the method
runs in the library's CUDA kernels; there is no Python or CPU fallback: when
the shared library is missing the import of the binding fails.

PyTorch, when present, provides device memory (through the allocator hook of
``mmcq_opts``) and the CUDA stream the library enqueues on.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmmcq.so")

MMCQ_OK = 0
MMCQ_ERR_ARG, MMCQ_ERR_UNSUPPORTED, MMCQ_ERR_CUDA, MMCQ_ERR_NUMERIC, MMCQ_ERR_TIMEOUT, MMCQ_ERR_STATE = -1, -2, -3, -4, -5, -6
MMCQ_HOST, MMCQ_DEVICE = 0, 1
MMCQ_RK4, MMCQ_DP45 = 0, 1
MMCQ_CAVITY_E, MMCQ_CAVITY_P = 0, 1
MMCQ_TERM_DEMAG, MMCQ_TERM_EXCHANGE, MMCQ_TERM_ANIS, MMCQ_TERM_ZEEMAN, MMCQ_TERM_CAVITY = 1, 2, 4, 8, 16
MMCQ_TERM_ALL = 31
MMCQ_POST_SLOTS = 4

_ERRNAMES = {-1: "MMCQ_ERR_ARG", -2: "MMCQ_ERR_UNSUPPORTED", -3: "MMCQ_ERR_CUDA", -4: "MMCQ_ERR_NUMERIC",
             -5: "MMCQ_ERR_TIMEOUT", -6: "MMCQ_ERR_STATE"}


class mmcq_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("batch", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class mmcq_opts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("mu0", ctypes.c_double), ("hbar", ctypes.c_double),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


class mmcq_cavity(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("t", "t_cav", "re_alpha", "im_alpha", "n_photon", "Gamma", "S", "C", "X", "dt")] + \
               [("accepted", ctypes.c_int64), ("rejected", ctypes.c_int64), ("err", ctypes.c_double)]


class mmcq_info(ctypes.Structure):
    _fields_ = [("px", ctypes.c_int), ("py", ctypes.c_int), ("pz", ctypes.c_int), ("tile", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("setup_ms", ctypes.c_double),
                ("launches_per_step", ctypes.c_int64)]


class mmcq_objective(ctypes.Structure):
    _fields_ = [("w", ctypes.c_double * 3), ("wn", ctypes.c_double), ("wavg", ctypes.c_double),
                ("window", ctypes.c_int64)]


class mmcq_tuning(ctypes.Structure):
    _fields_ = [("x_rows", ctypes.c_int), ("col_groups", ctypes.c_int * 4), ("z_split", ctypes.c_int),
                ("x_pipe", ctypes.c_int), ("y_split", ctypes.c_int * 2), ("eval_ms", ctypes.c_double),
                ("rule_ms", ctypes.c_double), ("candidates", ctypes.c_int)]


class mmcq_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


_H = ctypes.c_void_p
_FP = ctypes.c_void_p   # float* (host or device)
_DP = ctypes.POINTER(ctypes.c_double)

PROTOTYPES = {
    "mmcq_create": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(mmcq_grid), ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, _DP, ctypes.POINTER(mmcq_opts)]),
    "mmcq_destroy": (None, [_H]),
    "mmcq_last_error": (ctypes.c_char_p, [_H]),
    "mmcq_info_get": (ctypes.c_int, [_H, ctypes.POINTER(mmcq_info)]),
    "mmcq_set_ms_map": (ctypes.c_int, [_H, _FP, ctypes.c_int]),
    "mmcq_set_bias": (ctypes.c_int, [_H, ctypes.c_int, _DP]),
    "mmcq_set_m": (ctypes.c_int, [_H, ctypes.c_int, _FP, ctypes.c_int]),
    "mmcq_get_m": (ctypes.c_int, [_H, ctypes.c_int, _FP, ctypes.c_int]),
    "mmcq_set_cavity": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _FP,
                                       ctypes.c_int]),
    "mmcq_set_cavity_init": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "mmcq_set_cavity_mode": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _FP, ctypes.c_int]),
    "mmcq_set_cavity_init_mode": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "mmcq_get_cavity_mode": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(mmcq_cavity)]),
    "mmcq_reset_cavity": (ctypes.c_int, [_H, ctypes.c_int]),
    "mmcq_disable_cavity": (ctypes.c_int, [_H, ctypes.c_int]),
    "mmcq_set_integrator": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
    "mmcq_set_horizon": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double]),
    "mmcq_step": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_double]),
    "mmcq_sync": (ctypes.c_int, [_H]),
    "mmcq_get_cavity": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(mmcq_cavity)]),
    "mmcq_post_cavity": (ctypes.c_int, [_H]),
    "mmcq_take_cavity": (ctypes.c_int, [_H, ctypes.POINTER(mmcq_cavity)]),
    "mmcq_get_dt_history": (ctypes.c_int, [_H, ctypes.c_int, _DP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "mmcq_eval_field": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _FP, ctypes.c_int]),
    "mmcq_set_drive": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "mmcq_set_recording": (ctypes.c_int, [_H, ctypes.c_int]),
    "mmcq_get_mavg_history": (ctypes.c_int, [_H, ctypes.c_int, _DP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "mmcq_spectrum": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _DP, ctypes.c_int, _DP]),
    "mmcq_adjoint_rk4": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(mmcq_objective),
                                        ctypes.c_int64, _DP, _DP, ctypes.POINTER(ctypes.c_float)]),
    "mmcq_get_state": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "mmcq_group_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_H), ctypes.c_int,
                                         ctypes.c_int]),
    "mmcq_group_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double]),
    "mmcq_group_replays": (ctypes.c_int64, [ctypes.c_void_p]),
    "mmcq_group_destroy": (None, [ctypes.c_void_p]),
    "mmcq_group_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "mmcq_set_state": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int64]),
    "mmcq_profile": (ctypes.c_int, [_H, ctypes.c_int]),
    "mmcq_profile_read": (ctypes.c_int, [_H, ctypes.POINTER(mmcq_kernel_stat), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "mmcq_launch_count": (ctypes.c_int64, [_H]),
    "mmcq_autotune": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(mmcq_tuning)]),
    "mmcq_set_tuning": (ctypes.c_int, [_H, ctypes.POINTER(mmcq_tuning)]),
    "mmcq_get_tuning": (ctypes.c_int, [_H, ctypes.POINTER(mmcq_tuning)]),
    "mmcq_coupling_sum_noalloc": (ctypes.c_int, [_FP, _FP, _FP, ctypes.c_int64, ctypes.c_double, _DP,
                                                 ctypes.c_void_p]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmmcq.so and declare its prototypes; raises if it has not been built."""
    if not os.path.exists(path):
        raise ImportError(f"mmcq CUDA library not built ({path}); run paper_2410_00966_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def __getattr__(name):
    # module-level mmcq_* names are the C entry points
    if name in PROTOTYPES:
        return getattr(lib(), name)
    raise AttributeError(name)


class MMCQError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.blocks = {}
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.blocks[p] = t
        return p

    def _free(self, p, ctx):
        self.blocks.pop(p, None)


def _ptr(a, n_floats):
    """(pointer, where, keepalive) for a float32 array: numpy -> host, CUDA tensor -> device."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != n_floats:
                raise ValueError("expected a contiguous float32 tensor of %d values" % n_floats)
            return ctypes.c_void_p(a.data_ptr()), (MMCQ_DEVICE if a.is_cuda else MMCQ_HOST), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if arr.size != n_floats:
        raise ValueError("expected %d values, got %d" % (n_floats, arr.size))
    return ctypes.c_void_p(arr.ctypes.data), MMCQ_HOST, arr


class Sim:
    """A handle of `batch` instances on an nx*ny*nz grid (see include/mmcq.h)."""

    def __init__(self, nx, ny, nz, dx, dy, dz, Ms, Aex, alpha, Ku=0.0, axis=(1.0, 0.0, 0.0), batch=1,
                 gamma=0.0, mu0=0.0, hbar=0.0, device=0, use_torch=True):
        self._lib = lib()
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.batch = batch
        g = mmcq_grid(nx, ny, nz, dx, dy, dz, batch)
        o = mmcq_opts()
        o.gamma, o.mu0, o.hbar, o.device = gamma, mu0, hbar, device
        self._alloc = None
        self.stream = None
        if use_torch:
            try:
                import torch
                if torch.cuda.is_available():
                    dev = torch.device("cuda", device)
                    self._alloc = _TorchAllocator(dev)
                    o.alloc, o.free = self._alloc.c_alloc, self._alloc.c_free
                    self.stream = torch.cuda.current_stream(dev)
                    o.stream = ctypes.c_void_p(self.stream.cuda_stream)
            except ImportError:
                pass
        self._opts = o
        ax = (ctypes.c_double * 3)(*axis)
        h = _H()
        rc = self._lib.mmcq_create(ctypes.byref(h), ctypes.byref(g), Ms, Aex, alpha, Ku, ax, ctypes.byref(o))
        if rc != 0:
            raise MMCQError(rc, "mmcq_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mmcq_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _ck(self, rc):
        if rc != 0:
            raise MMCQError(rc, self._lib.mmcq_last_error(self._h).decode())
        return rc

    def info(self) -> dict:
        i = mmcq_info()
        self._ck(self._lib.mmcq_info_get(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in mmcq_info._fields_}

    def set_ms_map(self, ms):
        p, w, keep = _ptr(ms, self.n)
        self._ck(self._lib.mmcq_set_ms_map(self._h, p, w))

    def set_bias(self, B, inst=-1):
        self._ck(self._lib.mmcq_set_bias(self._h, inst, (ctypes.c_double * 3)(*B)))

    def set_m(self, m, inst=-1):
        p, w, keep = _ptr(m, 3 * self.n)
        self._ck(self._lib.mmcq_set_m(self._h, inst, p, w))

    def get_m(self, inst=0, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((self.n, 3), dtype=np.float32)
        p, w, keep = _ptr(out, 3 * self.n)
        self._ck(self._lib.mmcq_get_m(self._h, inst, p, w))
        return out

    def set_cavity(self, omega_c, kappa, g=0.0, profile=None, profile_is_brms=False, inst=-1):
        self.set_cavity_mode(0, omega_c, kappa, g, profile, profile_is_brms, inst)

    def set_cavity_mode(self, mode, omega_c, kappa, g=0.0, profile=None, profile_is_brms=False, inst=-1):
        keep = None
        p = None
        if profile is not None:
            keep = np.ascontiguousarray(np.asarray(profile, dtype=np.float32).reshape(-1))
            if keep.size != 3 * self.n:
                raise ValueError("profile must have N x 3 values")
            p = ctypes.c_void_p(keep.ctypes.data)
        self._ck(self._lib.mmcq_set_cavity_mode(self._h, inst, int(mode), omega_c, kappa, g, p,
                                                int(bool(profile_is_brms))))

    def set_cavity_init(self, x0, p0, inst=-1):
        self._ck(self._lib.mmcq_set_cavity_init(self._h, inst, x0, p0))

    def set_cavity_init_mode(self, mode, x0, p0, inst=-1):
        self._ck(self._lib.mmcq_set_cavity_init_mode(self._h, inst, int(mode), x0, p0))

    def reset_cavity(self, inst=-1):
        self._ck(self._lib.mmcq_reset_cavity(self._h, inst))

    def disable_cavity(self, inst=-1):
        self._ck(self._lib.mmcq_disable_cavity(self._h, inst))

    def set_integrator(self, kind=MMCQ_RK4, tol=1e-6, cavity_mode=MMCQ_CAVITY_E):
        self._ck(self._lib.mmcq_set_integrator(self._h, kind, tol, cavity_mode))

    def set_horizon(self, t_end, inst=-1):
        self._ck(self._lib.mmcq_set_horizon(self._h, inst, t_end))

    def step(self, n, dt=0.0):
        self._ck(self._lib.mmcq_step(self._h, int(n), float(dt)))

    def sync(self):
        self._ck(self._lib.mmcq_sync(self._h))

    def cavity(self, inst=0, mode=0):
        """Read-out of one instance (dict), or of all instances (list of dicts) for inst = -1."""
        n = self.batch if inst == -1 else 1
        c = (mmcq_cavity * n)()
        self._ck(self._lib.mmcq_get_cavity_mode(self._h, inst, int(mode), c))
        res = [{k: getattr(c[i], k) for k, _ in mmcq_cavity._fields_} for i in range(n)]
        return res if inst == -1 else res[0]

    def post_cavity(self):
        """Enqueue the read-out of every instance as of the work enqueued so far (no wait)."""
        self._ck(self._lib.mmcq_post_cavity(self._h))

    def take_cavity(self):
        """Wait for the oldest posted read-out; list of dicts, one per instance."""
        c = (mmcq_cavity * self.batch)()
        self._ck(self._lib.mmcq_take_cavity(self._h, c))
        return [{k: getattr(c[i], k) for k, _ in mmcq_cavity._fields_} for i in range(self.batch)]

    def dt_history(self, inst=0) -> np.ndarray:
        n = ctypes.c_int64()
        self._ck(self._lib.mmcq_get_dt_history(self._h, inst, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value)
        if n.value:
            self._ck(self._lib.mmcq_get_dt_history(self._h, inst, out.ctypes.data_as(_DP), n.value, ctypes.byref(n)))
        return out

    def profile(self, enable=True):
        self._ck(self._lib.mmcq_profile(self._h, int(bool(enable))))

    @staticmethod
    def _tuning_dict(t) -> dict:
        return {"x_rows": t.x_rows, "col_groups": list(t.col_groups), "z_split": t.z_split, "x_pipe": t.x_pipe,
                "y_split": list(t.y_split), "eval_ms": t.eval_ms, "rule_ms": t.rule_ms, "candidates": t.candidates}

    def autotune(self, reps=5) -> dict:
        """Time the launch-parameter candidates of this grid and keep the fastest (mmcq_autotune)."""
        t = mmcq_tuning()
        self._ck(self._lib.mmcq_autotune(self._h, int(reps), ctypes.byref(t)))
        return self._tuning_dict(t)

    def tuning(self) -> dict:
        t = mmcq_tuning()
        self._ck(self._lib.mmcq_get_tuning(self._h, ctypes.byref(t)))
        return self._tuning_dict(t)

    def set_tuning(self, plan=None):
        """Apply a plan (dict as returned by tuning()/autotune()); None restores the fixed rules."""
        if plan is None:
            self._ck(self._lib.mmcq_set_tuning(self._h, None))
            return
        t = mmcq_tuning()
        t.x_rows = int(plan["x_rows"])
        for k in range(4):
            t.col_groups[k] = int(plan["col_groups"][k])
        t.z_split = int(plan["z_split"])
        t.x_pipe = int(plan["x_pipe"])
        ys = plan.get("y_split", [-1, -1])
        for k in range(2):
            t.y_split[k] = int(ys[k])
        self._ck(self._lib.mmcq_set_tuning(self._h, ctypes.byref(t)))

    def profile_read(self) -> list:
        arr = (mmcq_kernel_stat * 16)()
        n = ctypes.c_int()
        self._ck(self._lib.mmcq_profile_read(self._h, arr, 16, ctypes.byref(n)))
        return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "total_ms": arr[i].total_ms,
                 "bytes": arr[i].bytes} for i in range(n.value)]

    def launch_count(self) -> int:
        return int(self._lib.mmcq_launch_count(self._h))

    def set_drive(self, amp, omega_cut, t0=0.0, inst=-1):
        """B_ext += amp * B_rms,i * sinc(omega_cut (t - t0)) (the paper's Appendix C excitation)."""
        self._ck(self._lib.mmcq_set_drive(self._h, inst, float(amp), float(omega_cut), float(t0)))

    def set_recording(self, every=1):
        """Record (t, <m>) after every `every`-th accepted step (0 stops)."""
        self._ck(self._lib.mmcq_set_recording(self._h, int(every)))

    def mavg_history(self, inst=0) -> np.ndarray:
        n = ctypes.c_int64()
        self._ck(self._lib.mmcq_get_mavg_history(self._h, inst, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 4))
        if n.value:
            self._ck(self._lib.mmcq_get_mavg_history(self._h, inst, out.ctypes.data_as(_DP), n.value,
                                                     ctypes.byref(n)))
        return out

    def spectrum(self, omega, comp=0, inst=0) -> np.ndarray:
        """Fourier transform (device) of the recorded <m_comp>(t) at angular frequencies omega."""
        w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        out = np.zeros(2 * w.size)
        self._ck(self._lib.mmcq_spectrum(self._h, inst, int(comp), w.ctypes.data_as(_DP), w.size,
                                         out.ctypes.data_as(_DP)))
        return out[0::2] + 1j * out[1::2]

    def adjoint_rk4(self, nsteps, dt, w=(0.0, 0.0, 0.0), wn=0.0, wavg=0.0, window=1, ckpt_every=1,
                    ms_grad=False):
        """J_b = w . <m>(T) + wn |alpha(T)|^2 + wavg <|alpha|^2>_(last `window` steps) after nsteps
        RK4 steps, and its gradient by the discrete adjoint (mmcq_adjoint_rk4):
        (J (B,), dJ/d(Bx, By, Bz, eta, omega_c, kappa) (B, 6), dJ/dMs (B, N) or None)."""
        obj = mmcq_objective((ctypes.c_double * 3)(*[float(v) for v in w]), float(wn), float(wavg), int(window))
        J = np.zeros(self.batch)
        g = np.zeros((self.batch, 6))
        gms = np.zeros((self.batch, self.n), dtype=np.float32) if ms_grad else None
        self._ck(self._lib.mmcq_adjoint_rk4(self._h, int(nsteps), float(dt), ctypes.byref(obj), int(ckpt_every),
                                            J.ctypes.data_as(_DP), g.ctypes.data_as(_DP),
                                            None if gms is None else gms.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return J, g, gms

    def get_state(self) -> bytes:
        """Snapshot of every instance (checkpoint), as bytes."""
        n = ctypes.c_int64()
        self._ck(self._lib.mmcq_get_state(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._ck(self._lib.mmcq_get_state(self._h, buf, n.value, ctypes.byref(n)))
        return buf.raw

    def set_state(self, snap: bytes):
        """Resume from a snapshot taken by get_state on an identically configured handle."""
        buf = ctypes.create_string_buffer(bytes(snap), len(snap))
        self._ck(self._lib.mmcq_set_state(self._h, buf, len(snap)))

    def eval_field(self, terms=MMCQ_TERM_ALL, inst=0, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((self.n, 3), dtype=np.float32)
        p, w, keep = _ptr(out, 3 * self.n)
        self._ck(self._lib.mmcq_eval_field(self._h, inst, terms, p, w))
        return out


class Group:
    """Several Sim handles (any mix of grids) stepped together as one CUDA graph
    (mmcq_group_*): ``step(n, dt)`` has the effect of ``sim.step(n, dt)`` on each."""

    def __init__(self, sims, chunk: int = 16):
        self._lib = lib()
        self.sims = list(sims)
        arr = (_H * len(self.sims))(*[s._h for s in self.sims])
        g = ctypes.c_void_p()
        rc = self._lib.mmcq_group_create(ctypes.byref(g), arr, len(self.sims), int(chunk))
        if rc:
            raise MMCQError(rc, "mmcq_group_create failed")
        self._g = g

    def step(self, n, dt=0.0):
        rc = self._lib.mmcq_group_step(self._g, int(n), float(dt))
        if rc:
            raise MMCQError(rc, self._lib.mmcq_group_last_error(self._g).decode())

    def replays(self) -> int:
        return int(self._lib.mmcq_group_replays(self._g))

    def close(self):
        if getattr(self, "_g", None):
            self._lib.mmcq_group_destroy(self._g)
            self._g = None

    def __del__(self):
        self.close()


def cavity_objective(sim, m0, params, nsteps, dt, w=(0.0, 0.0, 0.0), wn=0.0, wavg=0.0, window=1,
                     ckpt_every=1, profile=None, ms=None):
    """Differentiable objective (torch.autograd).  From the per-instance initial
    states m0 ((B, N, 3) array) and parameters params (torch (B, 6): B_ext x, y,
    z, coupling g, omega_c, kappa, all rad/s or T), and optionally the Ms map ms
    (torch (N,)): configure `sim` (coupling from g with the given profile shape),
    run nsteps RK4 steps and return J (torch (B,)) =
    w . <m>(T) + wn |alpha(T)|^2 + wavg <|alpha|^2>_(last window steps).
    The backward pass is the discrete adjoint on the device (Sim.adjoint_rk4)."""
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, p, msv):
            pc = p.detach().cpu().double().numpy()
            if msv is not None:
                sim.set_ms_map(msv.detach().cpu().float().numpy())
            for b in range(sim.batch):
                sim.set_m(np.asarray(m0[b], dtype=np.float32), inst=b)
                sim.set_bias(tuple(pc[b, :3]), inst=b)
                sim.set_cavity(pc[b, 4], pc[b, 5], pc[b, 3], profile=profile, inst=b)
            J, g, gms = sim.adjoint_rk4(nsteps, dt, w, wn, wavg, window, ckpt_every, ms_grad=msv is not None)
            gp = g.copy()
            # B_rms is proportional to g: dJ/dg = dJ/deta / g
            gsafe = np.where(pc[:, 3] != 0, pc[:, 3], 1.0)
            gp[:, 3] = np.where(pc[:, 3] != 0, g[:, 3] / gsafe, 0.0)
            ctx.save_for_backward(torch.from_numpy(gp).to(p.dtype),
                                  torch.from_numpy(gms).to(p.dtype) if gms is not None else torch.zeros(0))
            ctx.has_ms = msv is not None
            return torch.from_numpy(J).to(p.dtype)

        @staticmethod
        def backward(ctx, gout):
            gp, gms = ctx.saved_tensors
            gout = gout.detach().cpu().to(gp.dtype)
            dp = gout[:, None] * gp
            dms = (gout[:, None] * gms).sum(0) if ctx.has_ms else None
            return dp, dms

    return _Fn.apply(params, ms)
