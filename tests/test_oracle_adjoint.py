"""Pins of the oracle's discrete adjoint of the RK4 path (gradients of
J = w . <m>(T) + wn |alpha(T)|^2 + wavg <|alpha|^2>_(last W steps) with
respect to the bias, the B_rms scale, omega_c, kappa, the initial
magnetisation and the per-cell Ms map): central finite differences of the
oracle's own forward map in FP64."""
import math

import numpy as np
import pytest

import oracle

NX, NY, NZ, D = 5, 4, 2, 4e-9
W = (0.3, -0.7, 0.2)
WN = 5.0
WAVG, WINDOW = 3.0, 12
STEPS, DT = 40, 2e-13


def _make(bias=(0.05, 0.01, 0.0), eta=1.0, wc=2 * math.pi * 7e9, kappa=2 * math.pi * 3e8, m0=None, ms=None):
    o = oracle.Oracle(NX, NY, NZ, D, D, D, 8e5, 1.3e-11, 0.02, Ku=2e4, axis=(0.6, 0.8, 0.0))
    n = o.n
    if ms is not None:
        o.set_ms(ms)
    rng = np.random.default_rng(11)
    if m0 is None:
        m0 = np.tile([1.0, 0.0, 0.0], (n, 1)) + 0.3 * rng.normal(size=(n, 3))
        m0 /= np.linalg.norm(m0, axis=1)[:, None]
        if ms is not None:
            m0[ms <= 0] = 0.0
    o.set_m(m0)
    o.set_bias(bias)
    prof = np.random.default_rng(12).normal(size=(n, 3)) * 2e-3
    o.set_cavity(wc, kappa, profile=eta * prof, profile_is_brms=True)
    o.set_cavity_init(0.8, -0.4)
    o.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
    return o, m0


def _J(**kw):
    o, _ = _make(**kw)
    J = o.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW)[0]
    return J


def _ms_map():
    ms = np.full(NX * NY * NZ, 8e5)
    ms[[3, 17, 30]] = 0.0
    ms[8] = 6e5
    return ms


@pytest.mark.parametrize("masked", [False, True], ids=["full", "masked"])
def test_parameter_gradients_match_finite_differences(masked):
    ms = _ms_map() if masked else None
    o, _ = _make(ms=ms)
    J, g, _, _ = o.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW)
    base = dict(bias=(0.05, 0.01, 0.0), eta=1.0, wc=2 * math.pi * 7e9, kappa=2 * math.pi * 3e8)
    checks = []
    for c in range(3):
        h = 1e-5
        bp = list(base["bias"]); bm = list(base["bias"])
        bp[c] += h; bm[c] -= h
        checks.append((g[c], (_J(**{**base, "bias": tuple(bp)}, ms=ms) - _J(**{**base, "bias": tuple(bm)}, ms=ms)) / (2 * h)))
    h = 1e-5
    checks.append((g[3], (_J(**{**base, "eta": 1 + h}, ms=ms) - _J(**{**base, "eta": 1 - h}, ms=ms)) / (2 * h)))
    h = 1e-6 * base["wc"]
    checks.append((g[4], (_J(**{**base, "wc": base["wc"] + h}, ms=ms) - _J(**{**base, "wc": base["wc"] - h}, ms=ms)) / (2 * h)))
    h = 1e-4 * base["kappa"]
    checks.append((g[5], (_J(**{**base, "kappa": base["kappa"] + h}, ms=ms) - _J(**{**base, "kappa": base["kappa"] - h}, ms=ms)) / (2 * h)))
    for k, (adj, fd) in enumerate(checks):
        assert abs(adj - fd) <= 1e-5 * abs(fd) + 1e-9 * abs(J), (k, adj, fd)
    assert abs(g[3]) > 0 and abs(g[4]) > 0


def test_initial_state_gradient_matches_finite_differences():
    o, m0 = _make()
    _, _, gm, _ = o.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW)
    # set_m normalises its input, so a perturbation of that input sees the
    # tangential part of dJ/dm0 (the derivative of m/|m| at |m| = 1 is the projector)
    gm = gm - np.sum(gm * m0, axis=1)[:, None] * m0
    rng = np.random.default_rng(5)
    for _ in range(6):
        i, c = int(rng.integers(NX * NY * NZ)), int(rng.integers(3))
        h = 1e-6
        mp, mm = m0.copy(), m0.copy()
        mp[i, c] += h
        mm[i, c] -= h
        fd = (_J(m0=mp) - _J(m0=mm)) / (2 * h)
        assert abs(gm[i, c] - fd) <= 1e-5 * abs(fd) + 1e-9, (i, c, gm[i, c], fd)


def test_ms_map_gradient_matches_finite_differences():
    ms = _ms_map()
    o, _ = _make(ms=ms)
    _, _, _, gs = o.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW)
    assert gs[3] == 0.0                                  # empty cells carry no gradient
    for i in (0, 8, 13, 29, 39):
        h = 1e-4 * ms[i]
        mp, mm = ms.copy(), ms.copy()
        mp[i] += h
        mm[i] -= h
        fd = (_J(ms=mp) - _J(ms=mm)) / (2 * h)
        assert abs(gs[i] - fd) <= 1e-4 * abs(fd) + 1e-12 * np.abs(gs).max(), (i, gs[i], fd)


def test_averaged_photon_term_alone():
    # with only the averaged term, J is the mean photon number over the window
    o, _ = _make()
    J, g, _, _ = o.adjoint_rk4(STEPS, DT, (0, 0, 0), 0.0, 1.0, WINDOW)
    p, _ = _make()
    ns = []
    for _ in range(STEPS):
        p.step(1, DT)
        ns.append(p.cavity()["n_photon"])
    assert abs(J - np.mean(ns[-WINDOW:])) <= 1e-12 * J
    assert abs(g[4]) > 0


def test_adjoint_leaves_the_forward_state():
    o, _ = _make()
    o.adjoint_rk4(STEPS, DT, W, WN)
    p, _ = _make()
    p.step(STEPS, DT)
    assert np.array_equal(o.get_m(), p.get_m())
