"""FP64 CPU oracle for the LLG + cavity hot path of Mumax3-cQED (arXiv 2410.00966).

TEST INFRASTRUCTURE ONLY: tests, the package smoke check and the benchmark's
CPU-baseline / reference legs use it.  The product library never imports it,
and it imports nothing from the product package.

The numerics live in ``mmcq_oracle.cpp`` (plain loops, FP64); this module only
compiles it with g++ and marshals numpy arrays through ctypes.  Functions and
the paper passages they follow:

* ``newell`` / ``demag_tensor``: demag tensor (Sec. 2.1 field-term list; the
  paper does not give Mumax3's kernel, Newell et al. 1993 is used).
* ``Oracle.field`` / ``Oracle.rhs``: effective field and LLG torque, Eq. (llg),
  with the cavity field B_rms * Gamma, Eq. (bcav).
* ``Oracle.step``: RK4 / Dormand-Prince on (m, alpha) (E-mode, Sec. 2.2 and
  Appendix A) or on m with the S_n, C_n accumulators (P-mode, Sec. 3.1,
  Eq. Sdiscrete, Cdiscrete, gammadiscretefinal).
* ``Oracle.set_drive`` / ``Oracle.mavg_history`` / ``spectrum``: Appendix C
  excitation (amp * B_rms * sinc(omega_cut t) added to B_ext), the spatially
  averaged m, and its numerical Fourier transform.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mmcq_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAMMA_LL = 1.7595e11          # rad/(s T), the gyromagnetic ratio used throughout
MU0 = 4e-7 * np.pi            # T m / A
HBAR = 1.05457182e-34         # J s, the paper's HBAR default (Sec. 3.2)

DEMAG_NONE, DEMAG_DIRECT, DEMAG_FFT = 0, 1, 2
RK4, DP45 = 0, 1
CAV_E, CAV_P = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["g++", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c++17", "-o", tmp, _SRC]
            subprocess.check_call(cmd)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "or_newell": (None, [d, d, d, d, d, d, dp]),
        "or_newell_ld": (None, [d, d, d, d, d, d, dp]),
        "or_dipole": (None, [d, d, d, d, dp]),
        "or_demag_tensor": (None, [d, d, d, d, d, d, dp]),
        "or_r_switch": (d, []),
        "or_aharoni_dz": (d, [d, d, d]),
        "or_fft3d": (None, [dp, i, i, i, i]),
        "or_create": (p, [i, i, i, d, d, d, d, d, d, d, dp, d, d, d, i]),
        "or_destroy": (None, [p]),
        "or_ncells": (l, [p]),
        "or_pad_sizes": (None, [p, ctypes.POINTER(ctypes.c_int)]),
        "or_set_ms": (None, [p, dp]),
        "or_set_m": (None, [p, dp]),
        "or_get_m": (None, [p, dp]),
        "or_set_bias": (None, [p, dp]),
        "or_set_cavity": (None, [p, d, d, d, dp, i]),
        "or_get_brms": (None, [p, dp]),
        "or_set_cavity_init": (None, [p, d, d]),
        "or_reset_cavity": (None, [p]),
        "or_disable_cavity": (None, [p]),
        "or_set_integrator": (None, [p, i, d, i]),
        "or_step": (l, [p, l, d]),
        "or_replay": (None, [p, dp, l]),
        "or_last_error": (d, [p, d]),
        "or_dt_history": (l, [p, dp, l]),
        "or_get_cavity": (None, [p, dp]),
        "or_set_alpha": (None, [p, d, d]),
        "or_demag": (None, [p, dp, dp]),
        "or_exchange": (None, [p, dp, dp]),
        "or_anis": (None, [p, dp, dp]),
        "or_field": (None, [p, dp, d, dp]),
        "or_rhs": (None, [p, dp, d, d, d, dp, dp]),
        "or_cavity_X": (d, [p, dp]),
        "or_demag_at": (None, [p, dp, ctypes.POINTER(ctypes.c_long), l, dp]),
        "or_energy": (None, [p, dp]),
        "or_set_drive": (None, [p, d, d, d]),
        "or_set_cavity_mode": (None, [p, i, d, d, d, dp, i]),
        "or_set_cavity_init_mode": (None, [p, i, d, d]),
        "or_get_cavity_mode": (None, [p, i, dp]),
        "or_get_brms_mode": (None, [p, i, dp]),
        "or_set_alpha_mode": (None, [p, i, d, d]),
        "or_field_modes": (None, [p, dp, dp, dp]),
        "or_rhs_modes": (None, [p, dp, dp, d, dp, dp]),
        "or_cavity_X_mode": (d, [p, dp, i]),
        "or_max_modes": (i, []),
        "or_set_threads": (i, [i]),
        "or_adjoint_rk4": (d, [p, l, d, dp, d, d, l, dp, dp, dp]),
        "or_drive_factor": (d, [p, d]),
        "or_set_recording": (None, [p, i]),
        "or_mavg_history": (l, [p, dp, l]),
        "or_spectrum": (None, [dp, dp, l, dp, l, dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def newell(X, Y, Z, dx, dy, dz, long_double=False) -> np.ndarray:
    """Exact Newell tensor {Nxx,Nyy,Nzz,Nxy,Nxz,Nyz} between cells offset by (X,Y,Z)."""
    lib = _load()
    out = np.zeros(6)
    (lib.or_newell_ld if long_double else lib.or_newell)(X, Y, Z, dx, dy, dz, _dp(out))
    return out


def dipole(X, Y, Z, V) -> np.ndarray:
    lib = _load()
    out = np.zeros(6)
    lib.or_dipole(X, Y, Z, V, _dp(out))
    return out


def demag_tensor(X, Y, Z, dx, dy, dz) -> np.ndarray:
    """The demag tensor as defined by the method (Newell near, dipole far)."""
    lib = _load()
    out = np.zeros(6)
    lib.or_demag_tensor(X, Y, Z, dx, dy, dz, _dp(out))
    return out


def r_switch() -> float:
    return _load().or_r_switch()


def aharoni_dz(a, b, c) -> float:
    """Aharoni (1998) D_z of a prism with full edges (2a, 2b, 2c)."""
    return _load().or_aharoni_dz(a, b, c)


def fft3d(a: np.ndarray, sign: int) -> np.ndarray:
    """The oracle's own radix-2 3-D FFT of a complex [z][y][x] array (unnormalised)."""
    lib = _load()
    b = np.ascontiguousarray(a, dtype=np.complex128).copy()
    pz, py, px = b.shape
    lib.or_fft3d(b.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)), px, py, pz, sign)
    return b


class Oracle:
    """One simulation instance on an nx*ny*nz grid (arrays are [z][y][x] order, m is N x 3)."""

    def __init__(self, nx, ny, nz, dx, dy, dz, Ms, Aex, alpha, Ku=0.0, axis=(1.0, 0.0, 0.0),
                 gamma=GAMMA_LL, mu0=MU0, hbar=HBAR, demag=DEMAG_FFT):
        self._lib = _load()
        ax = _f64(axis, 3)
        self._h = self._lib.or_create(nx, ny, nz, dx, dy, dz, Ms, Aex, alpha, Ku, _dp(ax), gamma, mu0,
                                      hbar, demag)
        if not self._h:
            raise ValueError("bad grid")
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.hbar = hbar

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    def pad_sizes(self):
        out = (ctypes.c_int * 3)()
        self._lib.or_pad_sizes(self._h, out)
        return tuple(out)

    def set_ms(self, ms):
        self._lib.or_set_ms(self._h, _dp(_f64(ms, self.n)))

    def set_m(self, m):
        self._lib.or_set_m(self._h, _dp(_f64(m, 3 * self.n)))

    def get_m(self) -> np.ndarray:
        out = np.zeros((self.n, 3))
        self._lib.or_get_m(self._h, _dp(out))
        return out

    def set_bias(self, B):
        self._lib.or_set_bias(self._h, _dp(_f64(B, 3)))

    def set_cavity(self, omega_c, kappa, g=0.0, profile=None, profile_is_brms=False):
        prof = None if profile is None else _f64(profile, 3 * self.n)
        self._lib.or_set_cavity(self._h, omega_c, kappa, g, None if prof is None else _dp(prof),
                                int(bool(profile_is_brms)))

    def get_brms(self) -> np.ndarray:
        out = np.zeros((self.n, 3))
        self._lib.or_get_brms(self._h, _dp(out))
        return out

    def set_cavity_init(self, x0, p0):
        self._lib.or_set_cavity_init(self._h, x0, p0)

    def reset_cavity(self):
        self._lib.or_reset_cavity(self._h)

    def disable_cavity(self):
        self._lib.or_disable_cavity(self._h)

    def set_integrator(self, kind=RK4, tol=1e-6, cavity_mode=CAV_E):
        self._lib.or_set_integrator(self._h, kind, tol, cavity_mode)

    def step(self, n, dt):
        """RK4: n steps of dt.  DP45: n attempts (dt > 0 sets the trial step). Returns accepted count."""
        return self._lib.or_step(self._h, n, dt)

    def replay(self, dts):
        d = _f64(dts)
        self._lib.or_replay(self._h, _dp(d), d.size)

    def trial_error(self, dt):
        return self._lib.or_last_error(self._h, dt)

    def dt_history(self) -> np.ndarray:
        n = self._lib.or_dt_history(self._h, None, 0)
        out = np.zeros(n)
        if n:
            self._lib.or_dt_history(self._h, _dp(out), n)
        return out

    def cavity(self) -> dict:
        out = np.zeros(12)
        self._lib.or_get_cavity(self._h, _dp(out))
        keys = ["t", "t_cav", "re_alpha", "im_alpha", "n_photon", "Gamma", "S", "C", "X", "dt",
                "accepted", "rejected"]
        return dict(zip(keys, out.tolist()))

    def set_alpha(self, re, im):
        self._lib.or_set_alpha(self._h, re, im)

    def _eval(self, fn, m):
        mm = _f64(m, 3 * self.n)
        out = np.zeros((self.n, 3))
        fn(self._h, _dp(mm), _dp(out))
        return out

    def demag(self, m):
        return self._eval(self._lib.or_demag, m)

    def exchange(self, m):
        return self._eval(self._lib.or_exchange, m)

    def anis(self, m):
        return self._eval(self._lib.or_anis, m)

    def field(self, m, Gamma=0.0):
        mm = _f64(m, 3 * self.n)
        out = np.zeros((self.n, 3))
        self._lib.or_field(self._h, _dp(mm), Gamma, _dp(out))
        return out

    def rhs(self, m, alpha=0j, t_cav=0.0):
        mm = _f64(m, 3 * self.n)
        dm = np.zeros((self.n, 3))
        da = np.zeros(2)
        self._lib.or_rhs(self._h, _dp(mm), alpha.real, alpha.imag, t_cav, _dp(dm), _dp(da))
        return dm, complex(da[0], da[1])

    def cavity_X(self, m):
        return self._lib.or_cavity_X(self._h, _dp(_f64(m, 3 * self.n)))

    def demag_at(self, m, cells):
        mm = _f64(m, 3 * self.n)
        c = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
        out = np.zeros((c.size, 3))
        self._lib.or_demag_at(self._h, _dp(mm), c.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                              c.size, _dp(out))
        return out

    # ---- cavity modes (mode 0 is the single mode set by set_cavity) ----------
    def set_cavity_mode(self, k, omega_c, kappa, g=0.0, profile=None, profile_is_brms=False):
        prof = None if profile is None else _f64(profile, 3 * self.n)
        self._lib.or_set_cavity_mode(self._h, k, omega_c, kappa, g, None if prof is None else _dp(prof),
                                     int(bool(profile_is_brms)))

    def set_cavity_init_mode(self, k, x0, p0):
        self._lib.or_set_cavity_init_mode(self._h, k, x0, p0)

    def cavity_mode(self, k) -> dict:
        out = np.zeros(12)
        self._lib.or_get_cavity_mode(self._h, k, _dp(out))
        keys = ["t", "t_cav", "re_alpha", "im_alpha", "n_photon", "Gamma", "S", "C", "X", "dt",
                "accepted", "rejected"]
        return dict(zip(keys, out.tolist()))

    def get_brms_mode(self, k) -> np.ndarray:
        out = np.zeros((self.n, 3))
        self._lib.or_get_brms_mode(self._h, k, _dp(out))
        return out

    def set_alpha_mode(self, k, re, im):
        self._lib.or_set_alpha_mode(self._h, k, re, im)

    def field_modes(self, m, Gammas):
        mm = _f64(m, 3 * self.n)
        G = np.zeros(max_modes())
        G[:len(Gammas)] = Gammas
        out = np.zeros((self.n, 3))
        self._lib.or_field_modes(self._h, _dp(mm), _dp(G), _dp(out))
        return out

    def rhs_modes(self, m, alphas, t_cav=0.0):
        """dm/dt and d alpha_k/dt with every mode's amplitude given (list of complex)."""
        mm = _f64(m, 3 * self.n)
        K = max_modes()
        a = np.zeros(2 * K)
        for k, v in enumerate(alphas):
            a[2 * k], a[2 * k + 1] = v.real, v.imag
        dm = np.zeros((self.n, 3))
        da = np.zeros(2 * K)
        self._lib.or_rhs_modes(self._h, _dp(mm), _dp(a), t_cav, _dp(dm), _dp(da))
        return dm, da[0::2] + 1j * da[1::2]

    def cavity_X_mode(self, m, k):
        return self._lib.or_cavity_X_mode(self._h, _dp(_f64(m, 3 * self.n)), k)

    def adjoint_rk4(self, nsteps, dt, w=(0.0, 0.0, 0.0), wn=0.0, wavg=0.0, window=1):
        """J = w . <m>(T) + wn |alpha(T)|^2 + wavg * (mean |alpha_n|^2 over the last `window` steps)
        after nsteps RK4 steps (E-mode, mode 0) and its gradient by the discrete adjoint:
        (J, dJ/d(Bx, By, Bz, eta, omega_c, kappa), dJ/dm0 (n, 3), dJ/dMs (n,))."""
        wv = _f64(w, 3)
        g = np.zeros(6)
        gm = np.zeros((self.n, 3))
        gs = np.zeros(self.n)
        J = self._lib.or_adjoint_rk4(self._h, nsteps, dt, _dp(wv), wn, wavg, window, _dp(g), _dp(gm), _dp(gs))
        return J, g, gm, gs

    def set_drive(self, amp, omega_cut, t0=0.0):
        """Appendix C excitation: B_ext += amp * B_rms,i * sinc(omega_cut (t - t0)); amp = 0 turns it off."""
        self._lib.or_set_drive(self._h, amp, omega_cut, t0)

    def drive_factor(self, t) -> float:
        return self._lib.or_drive_factor(self._h, t)

    def set_recording(self, on=True):
        self._lib.or_set_recording(self._h, int(bool(on)))

    def mavg_history(self) -> np.ndarray:
        """(n, 4): t, <mx>, <my>, <mz> after each accepted step while recording."""
        n = self._lib.or_mavg_history(self._h, None, 0)
        out = np.zeros((n, 4))
        if n:
            self._lib.or_mavg_history(self._h, _dp(out), n)
        return out

    def energy(self) -> dict:
        out = np.zeros(7)
        self._lib.or_energy(self._h, _dp(out))
        return dict(zip(["zeeman", "demag", "exchange", "anis", "coupling", "photon", "total"],
                        out.tolist()))


def spectrum(t, y, omega) -> np.ndarray:
    """Trapezoid-weighted Fourier transform of samples y(t_n) at angular
    frequencies omega, after removing the time average (complex array)."""
    lib = _load()
    t = _f64(t)
    y = _f64(y)
    w = _f64(omega)
    out = np.zeros(2 * w.size)
    lib.or_spectrum(_dp(t), _dp(y), t.size, _dp(w), w.size, _dp(out))
    return out[0::2] + 1j * out[1::2]


def max_modes() -> int:
    """Cavity modes the oracle holds (mode 0 is the paper's single mode)."""
    return _load().or_max_modes()


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle (n < 1: all cores); returns the number in use."""
    return _load().or_set_threads(int(n))
