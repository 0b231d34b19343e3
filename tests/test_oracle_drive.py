"""Pins of the oracle's excitation and spectrum (Appendix C of the paper: the
sample is driven by amp * B_rms * sinc(omega_cut t) added to B_ext, and the
broadband response is the numerical Fourier transform of the spatially
averaged magnetisation)."""
import math

import numpy as np

import oracle

GAMMA = oracle.GAMMA_LL


def test_spectrum_of_a_cosine_over_whole_periods_is_exact():
    # integral_0^T A cos(w0 t) e^{-i w0 t} dt = A T / 2 when T spans whole periods;
    # the trapezoid rule is exact for a trigonometric polynomial sampled over
    # whole periods, and the time average of the cosine is zero
    A, f0 = 0.3, 2.5e9
    w0 = 2 * math.pi * f0
    T = 40 / f0
    t = np.linspace(0.0, T, 4001)
    S = oracle.spectrum(t, A * np.cos(w0 * t), [w0])[0]
    assert abs(S - A * T / 2) <= 1e-10 * A * T
    # another whole-period harmonic is orthogonal
    S2 = oracle.spectrum(t, A * np.cos(w0 * t), [2 * w0])[0]
    assert abs(S2) <= 1e-10 * A * T


def test_spectrum_removes_the_mean_and_handles_uneven_steps():
    rng = np.random.default_rng(3)
    A, B, f0 = 0.2, 0.7, 1.0e9
    w0 = 2 * math.pi * f0
    T = 25 / f0
    t = np.sort(np.concatenate([[0.0, T], rng.uniform(0, T, 30000)]))
    y = A * np.cos(w0 * t) + B
    S = oracle.spectrum(t, y, [w0, 0.0])
    assert abs(S[0] - A * T / 2) <= 1e-4 * A * T       # trapezoid error O(h^2) on uneven samples
    assert abs(S[1]) <= 1e-12 * B * T                   # zero frequency sees only the removed mean
    # shifting every time by tau multiplies S by exp(-i w tau)
    tau = 3.3e-10
    S_shift = oracle.spectrum(t + tau, y, [w0])[0]
    assert abs(S_shift - S[0] * np.exp(-1j * w0 * tau)) <= 1e-9 * abs(S[0])


def test_drive_factor_is_amp_sinc():
    o = oracle.Oracle(1, 1, 1, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
    amp, wcut, t0 = 250.0, 2 * math.pi * 10e9, 1e-10
    o.set_drive(amp, wcut, t0)
    assert o.drive_factor(t0) == amp                     # sinc(0) = 1
    assert abs(o.drive_factor(t0 + math.pi / wcut)) <= 1e-13 * amp
    for t in (0.0, 3.7e-11, 2.2e-10):
        x = wcut * (t - t0)
        assert abs(o.drive_factor(t) - amp * math.sin(x) / x) <= 1e-15 * amp
    o.set_drive(0.0, wcut, t0)
    assert o.drive_factor(t0) == 0.0


def test_drive_adds_amp_sinc_brms_to_the_field_of_magnetised_cells():
    nx, ny, nz = 5, 4, 2
    o = oracle.Oracle(nx, ny, nz, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
    n = nx * ny * nz
    ms = np.full(n, 8e5)
    ms[7] = 0.0
    o.set_ms(ms)
    rng = np.random.default_rng(1)
    m = rng.normal(size=(n, 3))
    m /= np.linalg.norm(m, axis=1)[:, None]
    o.set_m(m)
    brms = rng.normal(size=(n, 3)) * 1e-6
    o.set_cavity(2 * math.pi * 5e9, 1e7, 0.0, profile=brms, profile_is_brms=True)
    o.disable_cavity()
    B0 = o.field(o.get_m())
    o.set_drive(300.0, 2 * math.pi * 8e9, -2e-11)
    f = o.drive_factor(0.0)
    B1 = o.field(o.get_m())
    expect = f * brms
    expect[7] = 0.0
    assert np.abs((B1 - B0) - expect).max() <= 1e-15 + 1e-12 * np.abs(expect).max()


def test_sinc_pulse_response_peaks_at_the_precession_frequency():
    # one cubic cell: the demag field is along m, so m precesses about B_ext at
    # gamma B / (1 + alpha^2); a sinc pulse with a cut-off above it rings the
    # mode and the transform of <m_x>(t) peaks there
    alpha, B = 0.01, 0.1
    o = oracle.Oracle(1, 1, 1, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, alpha)
    o.set_m(np.array([[0.0, 0.0, 1.0]]))
    o.set_bias((0.0, 0.0, B))
    o.set_cavity(1.0, 0.0, 0.0, profile=np.array([[1e-6, 0.0, 0.0]]), profile_is_brms=True)
    o.disable_cavity()
    o.set_drive(1000.0, 2 * math.pi * 20e9, 30e-12)       # 1 mT peak along x
    o.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
    o.set_recording(True)
    o.step(12000, 0.2e-12)
    h = o.mavg_history()
    assert h.shape == (12000, 4) and abs(h[-1, 0] - 12000 * 0.2e-12) < 1e-20
    wl = GAMMA * B / (1 + alpha * alpha)
    w = np.linspace(0.8 * wl, 1.2 * wl, 2001)
    S = np.abs(oracle.spectrum(h[:, 0], h[:, 1], w))
    assert abs(w[np.argmax(S)] - wl) <= 2e-3 * wl
