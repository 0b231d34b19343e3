"""Pins of the oracle's multimode cavity.  The paper keeps one mode and notes
that further modes follow the same equations, each with its own B_rms map
(Sec. 4, multimode remark): B_cav = sum_k B_rms,k Gamma_k, each mode driven by
its own X_k = V_c sum_i Ms_i m_i . B_rms,k,i."""
import math

import numpy as np
import pytest

import oracle

CELL, MS = 4e-9, 8e5


def _film(alpha=0.01):
    o = oracle.Oracle(6, 5, 2, CELL, CELL, CELL, MS, 1.3e-11, alpha)
    n = o.n
    rng = np.random.default_rng(7)
    m = np.tile([1.0, 0.0, 0.0], (n, 1)) + 0.1 * rng.normal(size=(n, 3))
    m /= np.linalg.norm(m, axis=1)[:, None]
    o.set_m(m)
    o.set_bias((0.05, 0.0, 0.0))
    return o, rng


@pytest.mark.parametrize("mode", [oracle.CAV_E, oracle.CAV_P], ids=["E", "P"])
def test_uncoupled_second_mode_changes_nothing(mode):
    runs = []
    for extra in (False, True):
        o, rng = _film()
        prof = rng.normal(size=(o.n, 3))
        o.set_cavity(2 * math.pi * 7e9, 2 * math.pi * 1e7, 2 * math.pi * 2e8, profile=prof)
        if extra:
            o.set_cavity_mode(1, 2 * math.pi * 9e9, 2 * math.pi * 3e7, 0.0, profile=prof)
        o.set_integrator(oracle.RK4, 0.0, mode)
        o.step(40, 1e-13)
        runs.append((o.get_m(), o.cavity()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1]["re_alpha"] == runs[1][1]["re_alpha"]


@pytest.mark.parametrize("mode", [oracle.CAV_E, oracle.CAV_P], ids=["E", "P"])
def test_two_identical_modes_equal_one_mode_with_sqrt2_coupling(mode):
    # alpha' = (alpha_0 + alpha_1)/sqrt2 with B' = sqrt2 B_rms obeys the single-mode
    # equations exactly; the antisymmetric combination is uncoupled and stays empty
    wc, kappa = 2 * math.pi * 7e9, 2 * math.pi * 2e7
    o2, rng = _film()
    prof = rng.normal(size=(o2.n, 3)) * 1e-6
    for k in (0, 1):
        o2.set_cavity_mode(k, wc, kappa, profile=prof, profile_is_brms=True)
    o2.set_integrator(oracle.RK4, 0.0, mode)
    o1, _ = _film()
    o1.set_cavity(wc, kappa, profile=math.sqrt(2) * prof, profile_is_brms=True)
    o1.set_integrator(oracle.RK4, 0.0, mode)
    for o in (o1, o2):
        o.step(300, 1e-13)
    assert np.abs(o1.get_m() - o2.get_m()).max() <= 1e-12
    a1 = complex(o1.cavity()["re_alpha"], o1.cavity()["im_alpha"])
    c0, c1 = o2.cavity_mode(0), o2.cavity_mode(1)
    a20, a21 = complex(c0["re_alpha"], c0["im_alpha"]), complex(c1["re_alpha"], c1["im_alpha"])
    assert abs(a20 - a21) <= 1e-12 * abs(a20)
    assert abs((a20 + a21) / math.sqrt(2) - a1) <= 1e-9 * abs(a1)


def _secular_roots(wz, modes):
    # (Omega^2 - wz^2) prod_k (Omega^2 - w_k^2) - sum_k 4 lam_k^2 wz w_k prod_{j != k} (Omega^2 - w_j^2) = 0,
    # the normal-phase polariton condition of Eq. (dickepolaritons) with one term per mode
    P = np.poly1d([1.0, -wz ** 2])
    for w, _ in modes:
        P = P * np.poly1d([1.0, -w ** 2])
    for k, (w, lam) in enumerate(modes):
        Q = np.poly1d([4 * lam ** 2 * wz * w])
        for j, (wj, _) in enumerate(modes):
            if j != k:
                Q = Q * np.poly1d([1.0, -wj ** 2])
        P = P - Q
    r = np.roots(P.coeffs)
    return np.sort(np.sqrt(r.real))


@pytest.mark.parametrize("lams", [(0.2, 0.1), (0.35, 0.3), (0.1, 0.45)])
def test_two_mode_polaritons_from_the_linearised_dynamics(lams):
    g = oracle.GAMMA_LL
    wz = 2 * math.pi * 10e9
    ws = [2 * math.pi * 9e9, 2 * math.pi * 11.5e9]
    S = MS * CELL ** 3 / (oracle.HBAR * g)
    o = oracle.Oracle(1, 1, 1, CELL, CELL, CELL, MS, 1e-11, 0.0)
    o.set_bias([0, 0, wz / g])
    modes = []
    for k, (w, r) in enumerate(zip(ws, lams)):
        lam = r * math.sqrt(w * wz) / 2
        modes.append((w, lam))
        o.set_cavity_mode(k, w, 0.0, profile=[math.sqrt(2 / S) * lam / g, 0, 0], profile_is_brms=True)
    m_eq = np.array([0, 0, 1.0])
    e1, e2 = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])

    def f(y):
        m = m_eq + y[0] * e1 + y[1] * e2
        m = m / np.linalg.norm(m)
        a = [complex(y[2], y[3]), complex(y[4], y[5])]
        dm, da = o.rhs_modes(m.reshape(1, 3), a)
        return np.array([dm[0] @ e1, dm[0] @ e2, da[0].real, da[0].imag, da[1].real, da[1].imag])
    J = np.zeros((6, 6))
    for j in range(6):
        h = np.zeros(6)
        h[j] = 1e-7
        J[:, j] = (f(h) - f(-h)) / (2e-7)
    ev = np.linalg.eigvals(J)
    freqs = np.sort(np.abs(ev.imag))[::2]
    np.testing.assert_allclose(freqs, _secular_roots(wz, modes), rtol=1e-6)
    assert np.abs(ev.real).max() < 1e-6 * wz


def test_multimode_energy_is_conserved_without_losses():
    # alpha_G = kappa_k = 0: the Hamiltonian with every mode's coupling and photon term is constant
    o, rng = _film(alpha=0.0)
    for k, f in enumerate((6.5e9, 8e9, 9.5e9)):
        o.set_cavity_mode(k, 2 * math.pi * f, 0.0, profile=rng.normal(size=(o.n, 3)) * 2e-3,
                          profile_is_brms=True)
    o.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
    e0 = o.energy()
    drift = []
    for dt in (2e-14, 1e-14):
        p, _ = _film(alpha=0.0)
        rng2 = np.random.default_rng(7)
        rng2.normal(size=(p.n, 3))
        for k, f in enumerate((6.5e9, 8e9, 9.5e9)):
            p.set_cavity_mode(k, 2 * math.pi * f, 0.0, profile=rng2.normal(size=(p.n, 3)) * 2e-3,
                              profile_is_brms=True)
        p.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
        p.step(int(round(2e-11 / dt)), dt)
        e = p.energy()
        drift.append(abs(e["total"] - e0["total"]))
        exch = max(abs(e["coupling"]), abs(e["photon"]))
    assert exch > 0
    assert drift[1] < drift[0] / 12 or drift[1] < 1e-12 * abs(e0["total"])
