"""Pins of the oracle's fields, LLG integration and cavity coupling.

Each check ties the oracle to something other than itself: closed-form
solutions (macrospin precession, Kittel's formula, the Dicke-model equilibria
and polariton frequencies of Sec. 4, Eq. dickeeqmag / dickepolaritons),
exact discrete eigenvectors (exchange), conservation laws (energy at zero
damping and loss, |m| = 1) and convergence orders (RK4, Dormand-Prince,
E-mode vs the paper-literal P-mode).
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _prism_factors(oracle, Lx, Ly, Lz):
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return np.array([oracle.aharoni_dz(b, c, a), oracle.aharoni_dz(c, a, b), oracle.aharoni_dz(a, b, c)])


# ---------------------------------------------------------------------------
# local field terms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_exchange_discrete_spin_wave_eigenvalue(oracle_mod, axis):
    # cos(k (i + 1/2) d) with k = pi n / (N d) is an exact eigenvector of the
    # free-boundary (Neumann) 6-neighbour Laplacian, eigenvalue -2(1 - cos kd)/d^2
    N, d, A, Ms = 16, 3e-9, 1.3e-11, 8e5
    dims = [1, 1, 1]
    dims[axis] = N
    o = oracle_mod.Oracle(*dims, d, d, d, Ms, A, 0.0, demag=oracle_mod.DEMAG_NONE)
    for nmode in [0, 1, 5, 15]:
        k = math.pi * nmode / (N * d)
        u = np.cos(k * (np.arange(N) + 0.5) * d)
        m = np.zeros((N, 3))
        m[:, 2] = u
        B = o.exchange(m)
        lam = 2 * (1 - math.cos(k * d)) / d ** 2
        np.testing.assert_allclose(B[:, 2], -(2 * A / Ms) * lam * u, atol=1e-9 * (2 * A / Ms) / d ** 2)
        assert np.abs(B[:, :2]).max() == 0


def test_exchange_uniform_zero_and_empty_neighbours(oracle_mod):
    d, A, Ms = 2e-9, 1e-11, 5e5
    o = oracle_mod.Oracle(5, 4, 3, d, d, d, Ms, A, 0.0, demag=oracle_mod.DEMAG_NONE)
    m = np.tile([0.6, 0.0, 0.8], (60, 1))
    assert np.abs(o.exchange(m)).max() < 1e-20
    # a 5x1x1 chain with cell 2 empty splits into two free chains
    o = oracle_mod.Oracle(5, 1, 1, d, d, d, Ms, A, 0.0, demag=oracle_mod.DEMAG_NONE)
    o.set_ms([Ms, Ms, 0.0, Ms, Ms])
    m = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 0], [0, 0, 1], [1, 0, 0]], float)
    B = o.exchange(m)
    pre = 2 * A / Ms / d ** 2
    np.testing.assert_allclose(B[0], pre * (m[1] - m[0]))
    np.testing.assert_allclose(B[1], pre * (m[0] - m[1]))
    np.testing.assert_allclose(B[2], 0)
    np.testing.assert_allclose(B[3], pre * (m[4] - m[3]))


def test_anisotropy_field(oracle_mod):
    Ms, Ku = 8e5, 5e4
    o = oracle_mod.Oracle(2, 1, 1, 1e-9, 1e-9, 1e-9, Ms, 1e-11, 0.0, Ku=Ku, axis=(0, 0, 2.0),
                          demag=oracle_mod.DEMAG_NONE)
    m = np.array([[0.0, 0.6, 0.8], [1.0, 0.0, 0.0]])
    B = o.anis(m)
    np.testing.assert_allclose(B[0], [0, 0, 2 * Ku / Ms * 0.8])
    np.testing.assert_allclose(B[1], 0)


# ---------------------------------------------------------------------------
# macrospin LLG and integrators
# ---------------------------------------------------------------------------

def _macrospin(oracle_mod, alpha=0.1, B=0.1, theta0=1.0, kind=None, tol=1e-6):
    # one cubic cell: its self demag field is parallel to m and exerts no torque
    o = oracle_mod.Oracle(1, 1, 1, 5e-9, 5e-9, 5e-9, 8e5, 1e-11, alpha)
    o.set_bias([0, 0, B])
    o.set_m([math.sin(theta0), 0.0, math.cos(theta0)])
    if kind is not None:
        o.set_integrator(kind, tol)
    return o


def _macrospin_exact(oracle_mod, t, alpha=0.1, B=0.1, theta0=1.0):
    g = oracle_mod.GAMMA_LL / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(theta0 / 2) * math.exp(-alpha * g * B * t))
    ph = g * B * t
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def test_macrospin_closed_form_and_rk4_order(oracle_mod):
    T = 200e-12
    errs = []
    for nsteps in [200, 400, 800]:
        o = _macrospin(oracle_mod)
        o.step(nsteps, T / nsteps)
        m = o.get_m()[0]
        assert abs(np.linalg.norm(m) - 1) < 1e-14
        errs.append(np.abs(m - _macrospin_exact(oracle_mod, T)).max())
    assert errs[-1] < 1e-10
    for a, b in zip(errs, errs[1:]):
        assert 12 < a / b < 20   # fourth order


def test_dp45_adaptive_and_error_order(oracle_mod):
    o = _macrospin(oracle_mod, kind=oracle_mod.DP45, tol=1e-9)
    T = 200e-12
    o.step(1, 1e-13)
    while o.cavity()["t"] < T:
        o.step(1, 0)
    t = o.cavity()["t"]
    assert np.abs(o.get_m()[0] - _macrospin_exact(oracle_mod, t)).max() < 1e-7
    # the embedded error estimate is O(dt^5)
    o = _macrospin(oracle_mod, kind=oracle_mod.DP45)
    e1, e2 = o.trial_error(4e-12), o.trial_error(2e-12)
    assert 20 < e1 / e2 < 40
    # replaying the accepted sequence reproduces the run
    o1 = _macrospin(oracle_mod, kind=oracle_mod.DP45, tol=1e-8)
    o1.step(40, 1e-12)
    o2 = _macrospin(oracle_mod, kind=oracle_mod.DP45)
    o2.replay(o1.dt_history())
    np.testing.assert_array_equal(o1.get_m(), o2.get_m())


def test_kittel_single_prism_cell(oracle_mod):
    # a single non-cubic cell is exactly uniformly magnetised: it precesses at
    # Kittel's frequency with the prism demag factors (Aharoni)
    dx, dy, dz, Ms, B = 6e-9, 4e-9, 2e-9, 8e5, 0.05
    o = oracle_mod.Oracle(1, 1, 1, dx, dy, dz, Ms, 1e-11, 0.0)
    o.set_bias([B, 0, 0])
    o.set_m([math.cos(1e-4), math.sin(1e-4), 0.0])   # small: no amplitude shift
    D = _prism_factors(oracle_mod, dx, dy, dz)
    w = oracle_mod.GAMMA_LL * math.sqrt((B + (D[1] - D[0]) * oracle_mod.MU0 * Ms) *
                                        (B + (D[2] - D[0]) * oracle_mod.MU0 * Ms))
    period = 2 * math.pi / w
    dt = period / 200
    ys, ts = [], []
    for s in range(3000):
        o.step(1, dt)
        ys.append(o.get_m()[0, 1])
        ts.append((s + 1) * dt)
    ys = np.array(ys)
    cross = [ts[i] - ys[i] * dt / (ys[i + 1] - ys[i]) for i in range(len(ys) - 1)
             if ys[i] < 0 <= ys[i + 1]]
    measured = 2 * math.pi / np.mean(np.diff(cross))
    assert abs(measured / w - 1) < 1e-6


def _zero_crossing_frequency(ts, ys):
    cross = [ts[i] - ys[i] * (ts[i + 1] - ts[i]) / (ys[i + 1] - ys[i]) for i in range(len(ys) - 1)
             if ys[i] < 0 <= ys[i + 1]]
    return 2 * math.pi / np.mean(np.diff(cross))


def test_kittel_multicell_element_approaches_macrospin(oracle_mod):
    # several cells, so the FFT demag convolution, exchange and Zeeman all act:
    # an element below the exchange length (5.7 nm for Permalloy) stays close
    # to uniform and precesses near Kittel's frequency with the element's
    # prism factors; the deviation (non-uniform demag field) grows with size
    Ms, B = 8e5, 0.1
    dev = []
    for nx, ny, nz in [(6, 4, 2), (12, 8, 4)]:
        d = 2e-9
        o = oracle_mod.Oracle(nx, ny, nz, d, d, d, Ms, 1.3e-11, 0.0)
        th = 1e-3
        o.set_m(np.tile([math.cos(th), math.sin(th), 0.0], (nx * ny * nz, 1)))
        o.set_bias([B, 0, 0])
        D = _prism_factors(oracle_mod, nx * d, ny * d, nz * d)
        w = oracle_mod.GAMMA_LL * math.sqrt((B + (D[1] - D[0]) * oracle_mod.MU0 * Ms) *
                                            (B + (D[2] - D[0]) * oracle_mod.MU0 * Ms))
        dt = 2 * math.pi / w / 2000      # resolves the exchange modes of 2 nm cells
        o.set_recording(True)
        o.step(12000, dt)
        h = o.mavg_history()
        dev.append(_zero_crossing_frequency(h[:, 0], h[:, 2]) / w - 1)
    assert abs(dev[0]) < 5e-3
    assert abs(dev[1]) > abs(dev[0])


# ---------------------------------------------------------------------------
# cavity: Dicke-model benchmarks (Sec. 4) and the memory term
# ---------------------------------------------------------------------------

CELL = 4e-9
MS = 8e5


def _dicke(oracle_mod, wz, wc, lam, alpha=0.0, kappa=0.0, mode=None):
    """Single cubic cell mapped onto the Dicke model (Sec. 4):
    B_ext = (0, 0, omega_z / gamma), B_rms = (sqrt(2/S) lambda / gamma, 0, 0),
    S = Ms V / (hbar gamma) (Sec. 2.1, M_s = hbar gamma S / V_c)."""
    g = oracle_mod.GAMMA_LL
    S = MS * CELL ** 3 / (oracle_mod.HBAR * g)
    o = oracle_mod.Oracle(1, 1, 1, CELL, CELL, CELL, MS, 1e-11, alpha)
    o.set_bias([0, 0, wz / g])
    o.set_cavity(wc, kappa, profile=[math.sqrt(2 / S) * lam / g, 0, 0], profile_is_brms=True)
    if mode is not None:
        o.set_integrator(oracle_mod.RK4, 1e-6, mode)
    return o


def _jacobian_freqs(o, m_eq, a_eq, e1, e2):
    """Eigen-frequencies of the oracle's right-hand side linearised at (m_eq, a_eq),
    in tangent coordinates m = normalise(m_eq + u e1 + v e2) and alpha = a_eq + p + i q."""
    def f(y):
        m = m_eq + y[0] * e1 + y[1] * e2
        m = m / np.linalg.norm(m)
        dm, da = o.rhs(m.reshape(1, 3), a_eq + complex(y[2], y[3]))
        dm = dm[0]
        return np.array([dm @ e1, dm @ e2, da.real, da.imag])
    J = np.zeros((4, 4))
    for j in range(4):
        h = np.zeros(4)
        h[j] = 1e-7 if j < 2 else 1e-7 * max(1.0, abs(a_eq))
        J[:, j] = (f(h) - f(-h)) / (2 * h[j])
    ev = np.linalg.eigvals(J)
    return np.sort(np.abs(ev.imag))[::2], np.abs(ev.real).max()


def _normal_polaritons(wz, wc, lam):
    r = math.sqrt((wz ** 2 - wc ** 2) ** 2 + 16 * lam ** 2 * wz * wc)
    return math.sqrt((wz ** 2 + wc ** 2 - r) / 2), math.sqrt((wz ** 2 + wc ** 2 + r) / 2)


def _superradiant_polaritons(wz, wc, mu):
    # Eq. (dickepolaritons), superradiant branch, with the sign inside the root
    # read as minus (Emary & Brandes 2003); the printed plus makes Omega_-^2 < 0.
    a = wz ** 2 / mu ** 2
    r = math.sqrt((a - wc ** 2) ** 2 + 4 * wz ** 2 * wc ** 2)
    return math.sqrt((a + wc ** 2 - r) / 2), math.sqrt((a + wc ** 2 + r) / 2)


@pytest.mark.parametrize("ratio,wz_over_wc", [(0.0, 1.0), (0.3, 1.0), (0.6, 1.0), (0.8, 0.7), (0.5, 1.6)])
def test_dicke_normal_phase_polaritons(oracle_mod, ratio, wz_over_wc):
    wc = 2 * math.pi * 10e9
    wz = wz_over_wc * wc
    lam = ratio * math.sqrt(wc * wz) / 2
    o = _dicke(oracle_mod, wz, wc, lam)
    freqs, damp = _jacobian_freqs(o, np.array([0, 0, 1.0]), 0j, np.array([1.0, 0, 0]), np.array([0, 1.0, 0]))
    expect = sorted(_normal_polaritons(wz, wc, lam))
    np.testing.assert_allclose(freqs, expect, rtol=1e-6)
    assert damp < 1e-6 * wc


@pytest.mark.parametrize("ratio,wz_over_wc", [(1.4, 1.0), (2.0, 1.0), (1.3, 0.6)])
def test_dicke_superradiant_equilibrium_and_polaritons(oracle_mod, ratio, wz_over_wc):
    wc = 2 * math.pi * 10e9
    wz = wz_over_wc * wc
    lam_c = math.sqrt(wc * wz) / 2
    lam = ratio * lam_c
    mu = (lam_c / lam) ** 2
    mx = math.sqrt(1 - mu ** 2)
    o = _dicke(oracle_mod, wz, wc, lam)
    m_eq = np.array([mx, 0.0, mu])
    a_eq = complex(o.cavity_X(m_eq.reshape(1, 3)) / (oracle_mod.HBAR * wc), 0.0)
    # Eq. (dickeeqmag): the state is a fixed point of the oracle's dynamics
    dm, da = o.rhs(m_eq.reshape(1, 3), a_eq)
    assert np.abs(dm).max() < 1e-9 * wz and abs(da) < 1e-9 * wc * abs(a_eq)
    e1 = np.array([mu, 0.0, -mx])
    freqs, damp = _jacobian_freqs(o, m_eq, a_eq, e1, np.array([0, 1.0, 0]))
    np.testing.assert_allclose(freqs, sorted(_superradiant_polaritons(wz, wc, mu)), rtol=1e-5)


def test_dicke_golden_superradiant_relaxes_to_attractor(oracle_mod):
    gold = _read_golden("dicke_superradiant.txt")
    wc = 2 * math.pi * 10e9
    wz = gold["omega_ratio_z_over_c"] * wc
    lam = gold["lambda_over_lambda_c"] * math.sqrt(wc * wz) / 2
    kappa = 0.05 * wc
    # with cavity loss the fixed point follows from d(alpha)/dt = 0:
    # mu_kappa = omega_z (omega_c^2 + kappa^2) / (4 lambda^2 omega_c)
    mu_k = wz * (wc ** 2 + kappa ** 2) / (4 * lam ** 2 * wc)
    o = _dicke(oracle_mod, wz, wc, lam, alpha=0.05, kappa=kappa)
    o.set_m([0.05, 0.02, 1.0])
    dt = 2 * math.pi / wc / 80
    o.step(40000, dt)
    m = o.get_m()[0]
    assert abs(abs(m[0]) - math.sqrt(1 - mu_k ** 2)) < 1e-6
    assert abs(m[2] - mu_k) < 1e-6
    # the closed-cavity value of Eq. (dickeeqmag) is the kappa -> 0 limit
    mu = 1 / gold["lambda_over_lambda_c"] ** 2
    assert abs(math.sqrt(1 - mu ** 2) - 0.8600534) < 1e-6


def test_dicke_spectrum_peaks(oracle_mod):
    # time-domain check as in Sec. 4: the Fourier spectrum of m_x peaks at the
    # polariton frequencies (within one bin)
    wc = 2 * math.pi * 10e9
    wz = wc
    lam = 0.3 * math.sqrt(wc * wz) / 2
    o = _dicke(oracle_mod, wz, wc, lam)
    o.set_m([0.02, 0.0, 1.0])
    n, dt = 1 << 15, 2e-12
    xs = np.empty(n)
    for s in range(n):
        o.step(1, dt)
        xs[s] = o.get_m()[0, 0]
    spec = np.abs(np.fft.rfft((xs - xs.mean()) * np.hanning(n)))
    f = np.fft.rfftfreq(n, dt) * 2 * math.pi
    bin_w = f[1]
    peaks = [i for i in range(1, len(spec) - 1) if spec[i] > spec[i - 1] and spec[i] >= spec[i + 1]]
    top = sorted(sorted(peaks, key=lambda i: -spec[i])[:2])
    for i, w in zip(top, _normal_polaritons(wz, wc, lam)):
        assert abs(f[i] - w) <= bin_w


def test_coupling_g_conversion_gives_vacuum_rabi_splitting(oracle_mod):
    # set_cavity(g): B_rms = g sqrt(2 hbar / (gamma V_c sum Ms)); at resonance the
    # polaritons sit at omega sqrt(1 +- 2g/omega) (normal branch of Eq. dickepolaritons
    # with lambda = g), i.e. split by ~2g.
    w = 2 * math.pi * 8e9
    gc = 2 * math.pi * 50e6
    o = oracle_mod.Oracle(1, 1, 1, CELL, CELL, CELL, MS, 1e-11, 0.0)
    o.set_bias([0, 0, w / oracle_mod.GAMMA_LL])
    o.set_cavity(w, 0.0, g=gc)
    b = o.get_brms()[0]
    expect = gc * math.sqrt(2 * oracle_mod.HBAR / (oracle_mod.GAMMA_LL * MS * CELL ** 3))
    np.testing.assert_allclose(b, [0, expect, 0], rtol=1e-14)
    freqs, _ = _jacobian_freqs(o, np.array([0, 0, 1.0]), 0j, np.array([1.0, 0, 0]), np.array([0, 1.0, 0]))
    np.testing.assert_allclose(freqs, [w * math.sqrt(1 - 2 * gc / w), w * math.sqrt(1 + 2 * gc / w)], rtol=1e-6)
    assert abs((freqs[1] - freqs[0]) / (2 * gc) - 1) < 1e-4


def test_free_cavity_initial_condition_convention(oracle_mod):
    # no coupling: alpha(t) = alpha0 exp(-(kappa + i omega_c) t), alpha0 = (x0 - i p0)/2
    # (Sec. 3.2: x0 = 2 Re alpha0, p0 = -2 Im alpha0), and Eq. (gammadiscretefinal)
    # with S = C = 0 gives Gamma = exp(-kappa t)(x0 cos wt - p0 sin wt) = 2 Re alpha.
    wc, kappa, x0, p0 = 2 * math.pi * 5e9, 2 * math.pi * 0.1e9, 0.3, -0.2
    T = 0.37e-9
    for mode in (oracle_mod.CAV_E, oracle_mod.CAV_P):
        o = oracle_mod.Oracle(1, 1, 1, CELL, CELL, CELL, MS, 1e-11, 0.0)
        o.set_cavity_init(x0, p0)
        o.set_cavity(wc, kappa, profile=[0, 0, 0], profile_is_brms=True)
        o.set_integrator(oracle_mod.RK4, 1e-6, mode)
        o.step(2000, T / 2000)
        c = o.cavity()
        a = complex(x0, -p0) / 2 * np.exp(-complex(kappa, wc) * T)
        assert abs(complex(c["re_alpha"], c["im_alpha"]) - a) < 1e-9
        G = math.exp(-kappa * T) * (x0 * math.cos(wc * T) - p0 * math.sin(wc * T))
        assert abs(c["Gamma"] - G) < 1e-9


def _small_coupled(oracle_mod, mode, alpha=0.0, kappa=0.0):
    o = oracle_mod.Oracle(6, 5, 2, 3e-9, 3e-9, 3e-9, MS, 1.3e-11, alpha, Ku=2e4, axis=(0.3, 0.2, 1.0))
    rng = np.random.default_rng(7)
    m = np.array([1.0, 0.0, 0.0]) + 0.3 * rng.normal(size=(60, 3))
    o.set_m(m)
    o.set_bias([0.05, 0.01, 0.0])
    w = 2 * math.pi * 12e9
    o.set_cavity(w, kappa, g=2 * math.pi * 2e9)
    o.set_cavity_init(0.5, 0.2)
    o.set_integrator(oracle_mod.RK4, 1e-6, mode)
    return o


def _smooth_coupled(oracle_mod, demag, Aex, Ku, g, x0):
    o = oracle_mod.Oracle(6, 5, 2, 5e-9, 5e-9, 5e-9, MS, Aex, 0.0, Ku=Ku, axis=(0.3, 0.2, 1.0), demag=demag)
    idx = np.arange(60)
    x, y, z = idx % 6, (idx // 6) % 5, idx // 30
    o.set_m(np.stack([np.ones(60), 0.3 * np.sin(2 * np.pi * x / 6),
                      0.3 * np.cos(2 * np.pi * y / 5) + 0.1 * z], 1))
    o.set_bias([0.05, 0.01, 0.0])
    o.set_cavity_init(x0, 5.0)
    o.set_cavity(2 * math.pi * 12e9, 0.0, g=g)
    return o


def test_energy_conservation_zero_damping(oracle_mod):
    # alpha = 0 and kappa = 0: the total energy (Zeeman, demag, exchange,
    # anisotropy, cavity coupling -X 2Re(alpha), photon hbar omega_c |alpha|^2,
    # from Eq. startH) is conserved by the dynamics; the drift shrinks fast with dt
    drifts = []
    for nsteps in [200, 400]:
        o = _smooth_coupled(oracle_mod, oracle_mod.DEMAG_FFT, 1.3e-11, 2e4, 2 * math.pi * 2e9, 20.0)
        e0 = o.energy()
        o.step(nsteps, 20e-12 / nsteps)
        e1 = o.energy()
        drifts.append(abs(e1["total"] - e0["total"]) / abs(e0["total"]))
    assert drifts[1] < 1e-8
    assert drifts[0] / drifts[1] > 12


def test_energy_exchange_between_magnet_and_cavity(oracle_mod):
    # Zeeman + cavity only, Larmor frequency = omega_c: energy flows from the
    # precessing magnet into the photon mode (the photon energy grows many-fold)
    # while the total is conserved.  A wrong sign or factor in either coupling
    # direction (field on the spins, drive of alpha) breaks this balance.
    o = oracle_mod.Oracle(6, 5, 2, 5e-9, 5e-9, 5e-9, MS, 0.0, 0.0, demag=oracle_mod.DEMAG_NONE)
    o.set_m(np.tile([math.sin(0.5), 0.0, math.cos(0.5)], (60, 1)))
    w = 2 * math.pi * 12e9
    o.set_bias([0, 0, w / oracle_mod.GAMMA_LL])
    o.set_cavity_init(10.0, 0.0)
    o.set_cavity(w, 0.0, g=2 * math.pi * 2e9)
    e0 = o.energy()
    o.step(2500, 0.01e-12)
    e1 = o.energy()
    assert e1["photon"] > 50 * e0["photon"]
    moved = abs(e1["zeeman"] - e0["zeeman"])
    assert moved > 10 * e0["photon"]
    assert abs(e1["total"] - e0["total"]) < 1e-9 * moved


def test_damping_dissipates_energy(oracle_mod):
    o = _small_coupled(oracle_mod, oracle_mod.CAV_E, alpha=0.05, kappa=2 * math.pi * 0.5e9)
    e = [o.energy()["total"]]
    for _ in range(5):
        o.step(40, 1e-13)
        e.append(o.energy()["total"])
    assert all(b < a for a, b in zip(e, e[1:]))


def test_p_mode_converges_to_e_mode_first_order(oracle_mod):
    # the paper's rectangle-rule accumulators (P-mode) approximate the exact
    # memory integral (E-mode) with an O(dt) error
    T = 10e-12
    diffs = []
    for nsteps in [50, 100, 200]:
        res = []
        for mode in (oracle_mod.CAV_E, oracle_mod.CAV_P):
            o = _small_coupled(oracle_mod, mode, alpha=0.01, kappa=2 * math.pi * 0.2e9)
            o.step(nsteps, T / nsteps)
            c = o.cavity()
            res.append((o.get_m(), complex(c["re_alpha"], c["im_alpha"])))
        diffs.append((np.abs(res[0][0] - res[1][0]).max(), abs(res[0][1] - res[1][1])))
    for (dm1, da1), (dm2, da2) in zip(diffs, diffs[1:]):
        assert 1.7 < dm1 / dm2 < 2.3
        assert 1.7 < da1 / da2 < 2.3


def test_irms_worked_number():
    # Appendix C, Eq. (irms): i_rms = omega_0 sqrt(hbar pi / (4 Z_0)) = 11.3 nA
    g = _read_golden("irms_cpw.txt")
    hbar = _read_golden("materials.txt")["hbar"]
    i = 2 * math.pi * g["f0_hz"] * math.sqrt(hbar * math.pi / (4 * g["z0_ohm"]))
    assert abs(i / g["irms_a"] - 1) < g["rel_tol"]


def test_m_stays_unit_and_empty_cells_stay_zero(oracle_mod):
    o = oracle_mod.Oracle(4, 4, 1, 4e-9, 4e-9, 4e-9, MS, 1.3e-11, 0.02)
    ms = np.full(16, MS)
    ms[[0, 5, 10]] = 0
    o.set_ms(ms)
    rng = np.random.default_rng(1)
    o.set_m(rng.normal(size=(16, 3)))
    o.set_bias([0, 0.1, 0])
    o.step(50, 1e-13)
    m = o.get_m()
    r = np.linalg.norm(m, axis=1)
    np.testing.assert_allclose(r[ms > 0], 1, atol=1e-14)
    assert np.abs(m[ms == 0]).max() == 0
