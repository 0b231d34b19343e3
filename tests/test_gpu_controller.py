"""The adaptive integrator's own decisions on the GPU against the oracle.

The replay tests feed the GPU's accepted step lengths to the oracle, which
forces acceptance; they never look at the error estimate or at the step-size
controller.  These tests do, without replay:

* attempt by attempt, the GPU's error estimate max_i |m5_i - m4_i| (the value
  its controller used, read back through mmcq_cavity.err) against the
  oracle's FP64 estimate of an attempt of the same length from the same state
  (the GPU's own float32 m and its FP64 amplitude), the accept / reject
  decision against err <= tol, and the next trial step against
  dt * clamp(0.9 (tol / err)^(1/5), 0.2, 5) from both errors;
* the GPU and the oracle each running their own controller from the same
  start, through a sequence with rejections: the same accept / reject
  sequence and the same step lengths to the FP32 noise of the estimate.

Tolerance of the error estimate: err = |dt sum_j (b5_j - b4_j) k_j| is a
difference of stage torques; the FP32 rounding of each stage input (~6e-8 per
component) moves the torques by up to ~ |dk/dm| 6e-8, which with the exchange
stiffness of these grids (|dk/dm| ~ 1e12..1e13 1/s) and dt ~ 1e-12 s leaves
absolute noise of order 1e-9..1e-8 on errors of order tol = 1e-6, i.e. up to a
few per cent.  The test allows 5 %; a wrong weight b5_j - b4_j, a missing
stage or a wrong norm changes the estimate by far more.
"""
import math

import numpy as np
import pytest

from gpu_common import make_pair, require_gpu

pytestmark = pytest.mark.gpu

ERR_RTOL = 5e-2


def _controller(dt, err, tol):
    f = 0.9 * (tol / err) ** 0.2 if err > 0 else 5.0
    return dt * min(5.0, max(0.2, f))


def _case(name):
    import synthetic
    if name == "film":
        nx, ny, nz, d = 24, 20, 1, 4e-9
        sim, o = make_pair(nx, ny, nz, d, 8e5, 1.3e-11, 0.01)
        bias = (0.05, 0.0, 0.0)
        wc, g = 2 * math.pi * 6.4e9, 2 * math.pi * 200e6
    else:
        nx, ny, nz, d = 16, 8, 4, 5e-9
        sim, o = make_pair(nx, ny, nz, d, 1.4e5, 3.65e-12, 1e-3, Ku=1e3)
        bias = (0.1, 0.0, 0.0)
        wc, g = 2 * math.pi * 4.5e9, 2 * math.pi * 200e6
    n = nx * ny * nz
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(61, nz), 0.3)
    kappa = 2 * math.pi * 10e6
    for x in (sim, o):
        x.set_bias(bias)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    sim.set_cavity(wc, kappa, g)
    o.set_cavity(wc, kappa, g)
    return sim, o, m0


@pytest.mark.parametrize("name", ["film", "block"])
def test_dp45_error_estimate_and_controller_per_attempt(name):
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    tol = 1e-6
    tol32 = float(np.float32(tol))      # the tolerance as the device holds it
    sim, o, _ = _case(name)
    sim.set_integrator(pkg.MMCQ_DP45, tol, pkg.MMCQ_CAVITY_E)
    o.set_integrator(oracle.DP45, tol, oracle.CAV_E)
    dt0 = 1e-12                          # too long (omega dt ~ 1): the first attempts are rejected
    decisions = []
    worst = 0.0
    for k in range(16):
        m = sim.get_m().astype(np.float64)
        c = sim.cavity()
        dt = dt0 if k == 0 else c["dt"]
        o.set_m(m)
        o.set_alpha(c["re_alpha"], c["im_alpha"])
        err_o = o.trial_error(dt)
        sim.step(1, dt0 if k == 0 else 0.0)
        c1 = sim.cavity()
        acc = c1["accepted"] - c["accepted"]
        rej = c1["rejected"] - c["rejected"]
        assert acc + rej == 1
        err_g = c1["err"]
        rel = abs(err_g - err_o) / err_o
        worst = max(worst, rel)
        assert rel <= ERR_RTOL, (k, dt, err_g, err_o)
        # the decision: err <= tol, unless the two estimates straddle tol
        if abs(err_o - tol) > ERR_RTOL * tol:
            assert acc == int(err_o <= tol), (k, err_g, err_o)
        assert acc == int(err_g <= tol32)
        # the controller: exactly its formula on the device's own estimate,
        # and the oracle's formula to the noise of the estimate (1/5 power)
        assert c1["dt"] == pytest.approx(_controller(dt, err_g, tol32), rel=1e-12)
        assert c1["dt"] == pytest.approx(_controller(dt, err_o, tol), rel=ERR_RTOL / 4)
        if acc:
            assert c1["t"] == pytest.approx(c["t"] + dt, rel=1e-12)
        else:
            assert c1["t"] == c["t"]
            assert np.array_equal(sim.get_m(), m.astype(np.float32))
        decisions.append(acc)
    print(f"{name}: decisions {decisions}, worst relative error-estimate difference {worst:.2e}")
    assert 0 in decisions and 1 in decisions
    sim.close()


@pytest.mark.parametrize("name", ["film", "block"])
def test_dp45_free_running_controllers_agree(name):
    """Both sides run their own controllers from the same state and trial step."""
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    tol = 1e-6
    sim, o, _ = _case(name)
    sim.set_integrator(pkg.MMCQ_DP45, tol, pkg.MMCQ_CAVITY_E)
    o.set_integrator(oracle.DP45, tol, oracle.CAV_E)
    dt0 = 1e-12
    acc_g, acc_o, dts_g, dts_o = [], [], [], []
    for k in range(20):
        a = sim.cavity()["accepted"]
        sim.step(1, dt0 if k == 0 else 0.0)
        acc_g.append(sim.cavity()["accepted"] - a)
        dts_g.append(sim.cavity()["dt"])
        acc_o.append(o.step(1, dt0 if k == 0 else 0.0))
        dts_o.append(o.cavity()["dt"])
    print(f"{name}: GPU {acc_g}\n{name}: oracle {acc_o}")
    assert acc_g == acc_o
    np.testing.assert_allclose(dts_g, dts_o, rtol=ERR_RTOL)
    hist_g = sim.dt_history()
    hist_o = o.dt_history()
    assert len(hist_g) == len(hist_o) == sum(acc_o)
    np.testing.assert_allclose(hist_g, hist_o, rtol=ERR_RTOL)
    sim.close()
