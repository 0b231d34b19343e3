"""Edge cases of the GPU path against the oracle: adaptive steps with
rejections, a horizon that clips the last step, an instance with no magnetic
cells, and a ragged batch where one instance stops early."""
import math

import numpy as np
import pytest

from gpu_common import make_pair, require_gpu

pytestmark = pytest.mark.gpu


def _film_pair(nx=16, ny=12, nz=2, seed=90):
    import synthetic
    sim, o = make_pair(nx, ny, nz, 4e-9, 8e5, 1.3e-11, 0.01)
    m0 = synthetic.tilted_m(nx * ny * nz, synthetic.derive_seed(seed), 0.4)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    for h in (sim, o):
        h.set_bias((0.05, 0.02, 0.0))
        h.set_cavity(2 * math.pi * 8e9, 2 * math.pi * 1e7, 2 * math.pi * 2e8)
    return sim, o


def test_dp45_with_rejections_matches_oracle_replay():
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    sim, o = _film_pair()
    sim.set_integrator(pkg.MMCQ_DP45, 1e-7, pkg.MMCQ_CAVITY_E)
    o.set_integrator(oracle.DP45, 1e-7, oracle.CAV_E)
    sim.step(30, 2e-11)                          # far too long a first trial step
    c = sim.cavity()
    assert c["rejected"] > 0 and c["accepted"] > 5
    o.replay(sim.dt_history())
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    # the next trial step is the controller's rule applied to the last error
    # estimate (the rule itself is checked against the oracle's estimates in
    # test_gpu_controller.py)
    tol32 = float(np.float32(1e-7))
    f = 0.9 * (tol32 / c["err"]) ** 0.2 if c["err"] > 0 else 5.0
    last = sim.dt_history()[-1] if c["err"] <= tol32 else None
    assert c["dt"] > 0
    if last is not None:
        assert c["dt"] == pytest.approx(last * min(5.0, max(0.2, f)), rel=1e-12)
    sim.close()


def test_horizon_clips_the_last_step_and_stops():
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    sim, o = _film_pair()
    T = 3.7e-12
    sim.set_integrator(pkg.MMCQ_DP45, 1e-5, pkg.MMCQ_CAVITY_E)
    sim.set_horizon(T)
    sim.step(200, 1e-13)
    c = sim.cavity()
    hist = sim.dt_history()
    assert abs(c["t"] - T) <= 1e-9 * T and abs(hist.sum() - T) <= 1e-9 * T
    acc = c["accepted"]
    sim.step(10)                                  # nothing left to do
    assert sim.cavity()["accepted"] == acc
    o.set_integrator(oracle.DP45, 1e-5, oracle.CAV_E)
    o.replay(hist)
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    sim.close()


def test_instance_without_magnetic_cells_is_inert():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    sim = pkg.Sim(8, 8, 2, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
    sim.set_ms_map(np.zeros(128, np.float32))
    sim.set_cavity(2 * math.pi * 8e9, 1e7, 1e8)
    sim.set_bias((0.05, 0.0, 0.0))
    sim.step(20, 1e-13)
    sim.sync()
    assert not sim.get_m().any()
    c = sim.cavity()
    assert c["X"] == 0.0 and c["re_alpha"] == 0.0 and c["accepted"] == 20
    sim.close()


def test_ragged_batch_one_instance_stops_early():
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    n = 16 * 12 * 2
    sim = pkg.Sim(16, 12, 2, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01, batch=3)
    m0 = [synthetic.tilted_m(n, synthetic.derive_seed(91, b), 0.3) for b in range(3)]
    for b in range(3):
        sim.set_m(m0[b], inst=b)
        sim.set_bias((0.03 + 0.02 * b, 0.0, 0.0), inst=b)
    sim.set_integrator(pkg.MMCQ_DP45, 1e-6, pkg.MMCQ_CAVITY_E)
    sim.set_horizon(2e-12, inst=1)
    sim.step(60, 1e-13)
    cs = sim.cavity(-1)
    assert abs(cs[1]["t"] - 2e-12) <= 1e-21 and cs[0]["t"] > 2e-12 and cs[2]["t"] > 2e-12
    for b in range(3):
        o = oracle.Oracle(16, 12, 2, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
        o.set_m(m0[b].astype(np.float64))
        o.set_bias((0.03 + 0.02 * b, 0.0, 0.0))
        o.set_integrator(oracle.DP45, 1e-6, oracle.CAV_E)
        o.replay(sim.dt_history(b))
        assert np.abs(sim.get_m(b).astype(np.float64) - o.get_m()).max() <= 1e-5
    sim.close()


@pytest.mark.parametrize("shape", [(600, 3, 2), (4, 600, 2)], ids=["long-x", "long-y"])
def test_long_rows_dynamics(shape):
    # padded lengths 2048: the one-row x passes (L = 1024) and the split y passes
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    nx, ny, nz = shape
    sim, o = make_pair(nx, ny, nz, 4e-9, 8e5, 1.3e-11, 0.01)
    m0 = synthetic.tilted_m(nx * ny * nz, synthetic.derive_seed(92), 0.3)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    for h in (sim, o):
        h.set_bias((0.05, 0.02, 0.0))
        h.set_cavity(2 * math.pi * 8e9, 2 * math.pi * 1e7, 2 * math.pi * 2e8)
    sim.set_integrator(pkg.MMCQ_RK4, 0.0, pkg.MMCQ_CAVITY_E)
    o.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
    sim.step(20, 1e-13)
    o.step(20, 1e-13)
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    sim.close()
