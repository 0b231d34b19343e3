"""GPU trajectories vs the FP64 oracle on identical seeded inputs.

Bar: max |dm| <= 1e-5 per component over the stated horizon (the target the
method is held to), cavity amplitude within a stated relative tolerance.
Adaptive runs are compared by replaying the GPU's accepted step sequence in
the oracle (a flip of one accept/reject decision would otherwise change the
whole trajectory)."""
import math

import numpy as np
import pytest

from gpu_common import f32, make_pair, require_gpu

pytestmark = pytest.mark.gpu

TOL_M = 1e-5


def _setup(sim, o, m0, bias, cav=None, ms=None, profile=None, x0p0=None, inst=-1):
    if ms is not None:
        sim.set_ms_map(ms)
        o.set_ms(ms.astype(np.float64))
    sim.set_m(m0, inst=inst)
    o.set_m(m0.astype(np.float64))
    sim.set_bias(bias, inst=inst)
    o.set_bias(bias)
    if cav is not None:
        wc, kappa, g = cav
        if x0p0 is not None:
            sim.set_cavity_init(*x0p0, inst=inst)
            o.set_cavity_init(*x0p0)
        sim.set_cavity(wc, kappa, g, profile=profile, inst=inst)
        o.set_cavity(wc, kappa, g, profile=None if profile is None else profile.astype(np.float64))


def _alpha(c):
    return complex(c["re_alpha"], c["im_alpha"])


def test_film_32_rk4_full_horizon():
    """32x32x1 Permalloy film, cavity at the Kittel frequency, 5000 RK4 steps of 0.1 ps."""
    require_gpu()
    import synthetic
    w = synthetic.film_32()
    I = w.instances[0]
    sim, o = make_pair(I.nx, I.ny, I.nz, I.d, I.Ms, I.Aex, I.alpha)
    m0 = I.m0()
    _setup(sim, o, m0, I.bias, (I.omega_c, I.kappa, I.g))
    nsteps = int(round(w.horizon / w.dt))
    sim.step(nsteps, w.dt)
    o.step(nsteps, w.dt)
    dm = np.abs(sim.get_m().astype(np.float64) - o.get_m()).max()
    c, oc = sim.cavity(), o.cavity()
    print(f"film_32: max|dm| = {dm:.3e}, alpha gpu {_alpha(c)} oracle {_alpha(oc)}")
    assert dm <= TOL_M
    assert c["t"] == pytest.approx(oc["t"], rel=1e-12)
    assert abs(_alpha(c) - _alpha(oc)) <= 1e-3 * abs(_alpha(oc))
    assert c["X"] == pytest.approx(oc["X"], rel=1e-3, abs=1e-6 * abs(oc["X"]) + 1e-40)


@pytest.mark.parametrize("mode", [0, 1], ids=["E", "P"])
def test_3d_masked_profile_rk4(mode):
    """12x8x3 grid with an Ms mask, anisotropy, a Lorentzian coupling profile and
    a strong cavity; both cavity modes."""
    require_gpu()
    import synthetic
    nx, ny, nz, d = 12, 8, 3, 5e-9
    sim, o = make_pair(nx, ny, nz, d, 8e5, 1.3e-11, 0.02, Ku=3e4, axis=(1.0, 0.2, 0.0))
    sim.set_integrator(0, 1e-6, mode)
    o.set_integrator(0, 1e-6, mode)
    n = nx * ny * nz
    ms = synthetic.disk_ms(nx, ny, nz, d, d, 50e-9, 8e5)
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(7, mode), 0.3)
    prof = synthetic.lorentzian_profile(nx, ny, nz, d, 20e-9, direction=(0.0, 0.8, 0.6))
    _setup(sim, o, m0, (0.08, 0.01, 0.0), (2 * math.pi * 9e9, 2 * math.pi * 50e6, 2 * math.pi * 1.5e9),
           ms=ms, profile=prof, x0p0=(4.0, -2.0))
    sim.step(400, 5e-14)
    o.step(400, 5e-14)
    dm = np.abs(sim.get_m().astype(np.float64) - o.get_m()).max()
    c, oc = sim.cavity(), o.cavity()
    print(f"3d mode {mode}: max|dm| = {dm:.3e}, alpha {_alpha(c)} vs {_alpha(oc)}, S {c['S']} vs {oc['S']}")
    assert dm <= TOL_M
    assert abs(_alpha(c) - _alpha(oc)) <= 1e-4 * abs(_alpha(oc))
    assert c["Gamma"] == pytest.approx(oc["Gamma"], rel=1e-4, abs=1e-6)
    if mode == 1:
        assert c["S"] == pytest.approx(oc["S"], rel=1e-4)
        assert c["C"] == pytest.approx(oc["C"], rel=1e-4)


@pytest.mark.parametrize("mode", [0, 1], ids=["E", "P"])
def test_dp45_replay(mode):
    """Adaptive Dormand-Prince on 16x8x2: the oracle replays the GPU's accepted steps."""
    require_gpu()
    import synthetic
    nx, ny, nz, d = 16, 8, 2, 4e-9
    sim, o = make_pair(nx, ny, nz, d, 8e5, 1.3e-11, 0.01)
    sim.set_integrator(1, 1e-5, mode)
    o.set_integrator(1, 1e-5, mode)
    m0 = synthetic.tilted_m(nx * ny * nz, synthetic.derive_seed(8, mode), 0.4)
    _setup(sim, o, m0, (0.05, 0.0, 0.02), (2 * math.pi * 8e9, 2 * math.pi * 20e6, 2 * math.pi * 500e6))
    sim.step(80, 1e-13)
    c = sim.cavity()
    hist = sim.dt_history()
    assert len(hist) == c["accepted"] and c["accepted"] > 20
    assert c["t"] == pytest.approx(hist.sum(), rel=1e-12)
    o.replay(hist)
    dm = np.abs(sim.get_m().astype(np.float64) - o.get_m()).max()
    oc = o.cavity()
    print(f"dp45 mode {mode}: accepted {c['accepted']} rejected {c['rejected']} max|dm| = {dm:.3e}")
    assert dm <= TOL_M
    assert abs(_alpha(c) - _alpha(oc)) <= 1e-4 * abs(_alpha(oc))
    # the GPU's own error control: every accepted step met the tolerance in
    # the oracle's FP64 estimate too (within FP32 noise)
    assert oc["t"] == pytest.approx(c["t"], rel=1e-12)


def test_dp45_replay_fixed_shapes():
    """Adaptive Dormand-Prince on 256x40x16, a grid that takes the compile-time
    shapes of the x passes (rows of 256 cells), the y passes (P = 128) and the
    z pass (pz = 32): anisotropy, an Ms mask and a coupling profile, replayed by
    the oracle over the GPU's accepted steps."""
    require_gpu()
    import synthetic
    nx, ny, nz, d = 256, 40, 16, 5e-9
    sim, o = make_pair(nx, ny, nz, d, 1.4e5, 3.65e-12, 1e-3, Ku=1e3, axis=(1.0, 0.0, 0.0))
    sim.set_integrator(1, 1e-6, 0)
    o.set_integrator(1, 1e-6, 0)
    n = nx * ny * nz
    ms = synthetic.disk_ms(nx, ny, nz, d, d, 190e-9, 1.4e5)
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(11, 0), 0.2)
    prof = synthetic.lorentzian_profile(nx, ny, nz, d, 300e-9, direction=(0.0, 1.0, 0.0))
    _setup(sim, o, m0, (0.1, 0.0, 0.0), (2 * math.pi * 5e9, 2 * math.pi * 10e6, 2 * math.pi * 200e6),
           ms=ms, profile=prof)
    sim.step(30, 1e-13)
    c = sim.cavity()
    hist = sim.dt_history()
    assert len(hist) == c["accepted"] and c["accepted"] >= 10
    o.replay(hist)
    dm = np.abs(sim.get_m().astype(np.float64) - o.get_m()).max()
    oc = o.cavity()
    print(f"dp45 fixed shapes: accepted {c['accepted']} rejected {c['rejected']} max|dm| = {dm:.3e}")
    assert dm <= TOL_M
    assert abs(_alpha(c) - _alpha(oc)) <= 1e-4 * abs(_alpha(oc))


def test_dp45_horizon_lands_exactly():
    require_gpu()
    import synthetic
    sim, o = make_pair(8, 8, 1, 4e-9, 8e5, 1.3e-11, 0.01)
    sim.set_integrator(1, 1e-6, 0)
    sim.set_m(synthetic.tilted_m(64, 5, 0.3))
    sim.set_bias((0.05, 0, 0))
    T = 7.77e-12
    sim.set_horizon(T)
    sim.step(500, 1e-13)
    c = sim.cavity()
    assert c["t"] == pytest.approx(T, rel=1e-12)
    n_acc = c["accepted"]
    sim.step(5)
    assert sim.cavity()["accepted"] == n_acc


def test_batch_instances_are_independent():
    """Three instances in one handle (different bias, cavity, initial state)
    match three separate oracle runs."""
    require_gpu()
    import synthetic
    nx, ny, nz, d = 20, 12, 2, 4e-9
    import paper_2410_00966_gb300 as pkg
    import oracle
    sim = pkg.Sim(nx, ny, nz, d, d, d, 8e5, 1.3e-11, 0.01, batch=3)
    n = nx * ny * nz
    params = [((0.04, 0, 0), 2 * math.pi * 6e9, 2 * math.pi * 100e6),
              ((0.1, 0.02, 0), 2 * math.pi * 9e9, 2 * math.pi * 300e6),
              ((0.02, 0, 0.01), 2 * math.pi * 4e9, 2 * math.pi * 50e6)]
    m0s = [synthetic.tilted_m(n, synthetic.derive_seed(9, b), 0.2) for b in range(3)]
    for b, (bias, wc, g) in enumerate(params):
        sim.set_m(m0s[b], inst=b)
        sim.set_bias(bias, inst=b)
        sim.set_cavity(wc, 2 * math.pi * 10e6, g, inst=b)
    sim.step(300, 1e-13)
    for b, (bias, wc, g) in enumerate(params):
        o = oracle.Oracle(nx, ny, nz, d, d, d, 8e5, 1.3e-11, 0.01)
        o.set_m(m0s[b].astype(np.float64))
        o.set_bias(bias)
        o.set_cavity(wc, 2 * math.pi * 10e6, g)
        o.step(300, 1e-13)
        dm = np.abs(sim.get_m(inst=b).astype(np.float64) - o.get_m()).max()
        assert dm <= TOL_M, (b, dm)
        assert abs(_alpha(sim.cavity(b)) - _alpha(o.cavity())) <= 1e-4 * abs(_alpha(o.cavity()))


def test_dicke_single_cell_matches_oracle():
    """Single cell mapped onto the Dicke model (Sec. 4), lambda / lambda_c = 0.6."""
    require_gpu()
    import oracle
    cell, Ms = 4e-9, 8e5
    gam = oracle.GAMMA_LL
    S = Ms * cell ** 3 / (oracle.HBAR * gam)
    wc = wz = 2 * math.pi * 10e9
    lam = 0.6 * math.sqrt(wc * wz) / 2
    brms = np.array([[math.sqrt(2 / S) * lam / gam, 0.0, 0.0]], np.float32)
    sim, o = make_pair(1, 1, 1, cell, Ms, 1e-11, 0.0)
    m0 = np.array([[0.05, 0.0, 1.0]], np.float32)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    sim.set_bias((0, 0, wz / gam))
    o.set_bias((0, 0, wz / gam))
    sim.set_cavity(wc, 0.0, profile=brms, profile_is_brms=True)
    o.set_cavity(wc, 0.0, profile=brms.astype(np.float64), profile_is_brms=True)
    sim.step(3000, 1e-13)
    o.step(3000, 1e-13)
    dm = np.abs(sim.get_m().astype(np.float64) - o.get_m()).max()
    assert dm <= TOL_M
    assert abs(_alpha(sim.cavity()) - _alpha(o.cavity())) <= 1e-4 * abs(_alpha(o.cavity()))
