"""Multimode cavity on the GPU against the oracle: each enabled mode k adds
B_rms,k Gamma_k to the field and has its own amplitude (E-mode) or
accumulators (P-mode) driven by X_k (the paper keeps one mode and notes that
more follow the same equations, Sec. 4)."""
import math

import numpy as np
import pytest

from gpu_common import make_pair, require_gpu

pytestmark = pytest.mark.gpu

NX, NY, NZ, D = 16, 10, 3, 4e-9
MODES = [(6.0e9, 2e7, 3e8), (7.5e9, 5e7, 2e8), (9.0e9, 1e7, 1.5e8)]


def _pair(kind, mode):
    import oracle
    import synthetic
    n = NX * NY * NZ
    sim, o = make_pair(NX, NY, NZ, D, 8e5, 1.3e-11, 0.01)
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(70), 0.08)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    rng = np.random.default_rng(70)
    for h in (sim, o):
        h.set_bias((0.05, 0.0, 0.0))
    for k, (f, kap, g) in enumerate(MODES):
        prof = None if k == 0 else rng.normal(size=(n, 3)).astype(np.float32)
        sim.set_cavity_mode(k, 2 * math.pi * f, 2 * math.pi * kap, 2 * math.pi * g, profile=prof)
        o.set_cavity_mode(k, 2 * math.pi * f, 2 * math.pi * kap, 2 * math.pi * g,
                          profile=None if prof is None else prof.astype(np.float64))
    for k in range(len(MODES)):
        sim.set_cavity_init_mode(k, 0.3 * (k + 1), -0.1 * k)
        o.set_cavity_init_mode(k, 0.3 * (k + 1), -0.1 * k)
    sim.set_integrator(kind, 1e-6, mode)
    o.set_integrator(oracle.DP45 if kind == 1 else oracle.RK4, 1e-6, mode)
    return sim, o


def _alpha(c):
    return complex(c["re_alpha"], c["im_alpha"])


@pytest.mark.parametrize("mode", [0, 1], ids=["E", "P"])
def test_three_modes_rk4(mode):
    require_gpu()
    sim, o = _pair(0, mode)
    sim.step(200, 1e-13)
    o.step(200, 1e-13)
    dm = np.abs(sim.get_m().astype(np.float64) - o.get_m()).max()
    print(f"mode {mode}: max|dm| {dm:.3e}")
    assert dm <= 1e-5
    for k in range(len(MODES)):
        a, ao = _alpha(sim.cavity(0, k)), _alpha(o.cavity_mode(k))
        assert abs(a - ao) <= 1e-4 * abs(ao)
        assert abs(sim.cavity(0, k)["X"] - o.cavity_mode(k)["X"]) <= 1e-5 * abs(o.cavity_mode(k)["X"]) + 1e-40


@pytest.mark.parametrize("mode", [0, 1], ids=["E", "P"])
def test_three_modes_dp45_replay(mode):
    require_gpu()
    sim, o = _pair(1, mode)
    sim.step(30, 1e-13)
    o.replay(sim.dt_history())
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    for k in range(len(MODES)):
        a, ao = _alpha(sim.cavity(0, k)), _alpha(o.cavity_mode(k))
        assert abs(a - ao) <= 1e-4 * abs(ao)


def test_multimode_cavity_field_term():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    sim, o = _pair(0, 0)
    m = sim.get_m().astype(np.float64)
    B = sim.eval_field(pkg.MMCQ_TERM_CAVITY).astype(np.float64)
    G = [2 * o.cavity_mode(k)["re_alpha"] for k in range(len(MODES))]
    ref = o.field_modes(m, G) - o.field(m)        # field(m) carries no cavity term (Gamma = 0)
    assert np.abs(B - ref).max() <= 1e-6 * np.abs(ref).max()


def test_multimode_resume_is_bit_exact():
    require_gpu()
    a, _ = _pair(1, 0)
    a.step(8, 1e-13)
    snap = a.get_state()
    a.step(10)
    ref = (a.get_m(), [_alpha(a.cavity(0, k)) for k in range(len(MODES))])
    b, _ = _pair(1, 0)
    b.set_state(snap)
    b.step(10)
    assert np.array_equal(b.get_m(), ref[0])
    assert [_alpha(b.cavity(0, k)) for k in range(len(MODES))] == ref[1]
