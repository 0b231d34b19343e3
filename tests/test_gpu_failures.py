"""Failure detection without a GPU fault: the failures are made on the host.

* A non-finite direction handed to mmcq_set_m is stored as zero and reported
  as MMCQ_ERR_NUMERIC by the next synchronising call.
* A non-finite bias makes the torque non-finite: the stage kernel raises a
  device flag (no trap), the next synchronising call returns
  MMCQ_ERR_NUMERIC, and the handle stays usable once the input is fixed.
* An adaptive run with an unreachable tolerance shrinks its step until the
  controller flags a step-size underflow (MMCQ_ERR_NUMERIC) and stops the
  instance.
"""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_nonfinite_m_input_reported():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    sim = pkg.Sim(16, 8, 1, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
    bad = synthetic.tilted_m(128, 3, 0.2)
    bad[17, 1] = np.inf
    sim.set_m(bad)
    with pytest.raises(pkg.MMCQError) as e:
        sim.sync()
    assert e.value.code == pkg.MMCQ_ERR_NUMERIC
    m = sim.get_m()
    assert np.isfinite(m).all() and not m[17].any()
    sim.close()


def test_nan_field_reported_and_handle_recovers():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    sim = pkg.Sim(16, 8, 1, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
    m = synthetic.tilted_m(128, 3, 0.2)
    sim.set_m(m)
    sim.set_cavity(2 * np.pi * 5e9, 2 * np.pi * 1e7, 2 * np.pi * 5e7)
    sim.set_bias((float("nan"), 0.0, 0.0))
    sim.step(2, 1e-13)
    with pytest.raises(pkg.MMCQError) as e:
        sim.sync()
    assert e.value.code == pkg.MMCQ_ERR_NUMERIC
    sim.set_bias((0.05, 0.0, 0.0))
    sim.set_m(m)
    sim.reset_cavity()
    sim.step(2, 1e-13)
    sim.sync()
    assert np.isfinite(sim.get_m()).all()
    assert np.isfinite(sim.cavity()["re_alpha"])
    sim.close()


def test_step_size_underflow_is_flagged():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    sim = pkg.Sim(8, 8, 1, 4e-9, 4e-9, 4e-9, 8e5, 1.3e-11, 0.01)
    sim.set_m(synthetic.tilted_m(64, 4, 0.3))
    sim.set_bias((0.05, 0, 0))
    sim.set_integrator(pkg.MMCQ_DP45, 1e-30, pkg.MMCQ_CAVITY_E)
    sim.step(60, 1e-13)
    with pytest.raises(pkg.MMCQError) as e:
        sim.sync()
    assert e.value.code == pkg.MMCQ_ERR_NUMERIC
    c = sim.cavity()
    assert c["accepted"] == 0 and c["rejected"] >= 8
    sim.close()
