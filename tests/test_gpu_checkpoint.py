"""Checkpoint / resume through mmcq_get_state / mmcq_set_state.

The GPU path is deterministic (fixed-order FP64 reductions, no atomics in
the arithmetic), so a run resumed from a snapshot on a fresh handle must
continue bit-for-bit like the uninterrupted run, for both integrators and
both cavity modes, with the first-same-as-last stage and the adaptive step
carried over.  Malformed snapshots are rejected without touching the state."""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _make(pkg, synthetic, kind, mode, batch=3):
    sim = pkg.Sim(24, 12, 4, 5e-9, 5e-9, 5e-9, 1.4e5, 3.65e-12, 1e-3, Ku=1e3, axis=(1.0, 0.0, 0.0), batch=batch)
    n = 24 * 12 * 4
    for b in range(batch):
        sim.set_m(synthetic.tilted_m(n, synthetic.derive_seed(40, b), 0.05), inst=b)
        sim.set_bias((0.1, 0.0, 0.01 * b), inst=b)
        sim.set_cavity(2 * np.pi * (5e9 + 2e8 * b), 2 * np.pi * 1e7, 2 * np.pi * 5e8, inst=b)
    sim.set_integrator(kind, 1e-6, mode)
    return sim


@pytest.mark.parametrize("kind,mode", [(1, 0), (1, 1), (0, 0), (0, 1)], ids=["dp45-E", "dp45-P", "rk4-E", "rk4-P"])
def test_resume_is_bit_exact(kind, mode):
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    dt = 2e-13
    a = _make(pkg, synthetic, kind, mode)
    a.step(12, dt)
    snap = a.get_state()
    a.step(15, 0.0 if kind == 1 else dt)
    ref_m = [a.get_m(b) for b in range(3)]
    ref_c = a.cavity(-1)
    a.close()

    b_ = _make(pkg, synthetic, kind, mode)
    b_.set_bias((0.3, 0.0, 0.0))          # overwritten by the snapshot
    b_.set_state(snap)
    b_.step(15, 0.0 if kind == 1 else dt)
    for b in range(3):
        assert np.array_equal(b_.get_m(b), ref_m[b])
    got = b_.cavity(-1)
    for r, g in zip(ref_c, got):
        for key in ("t", "t_cav", "re_alpha", "im_alpha", "S", "C", "dt", "accepted", "rejected"):
            assert r[key] == g[key], key
    b_.close()


def test_bad_snapshots_rejected():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    import synthetic
    a = _make(pkg, synthetic, 1, 0)
    a.step(3, 1e-13)
    snap = a.get_state()
    m_before = a.get_m(0)
    for bad in (snap[:-1], b"x" * len(snap), snap[:40]):
        with pytest.raises(pkg.MMCQError) as e:
            a.set_state(bad)
        assert e.value.code == pkg.MMCQ_ERR_ARG
    other = _make(pkg, synthetic, 1, 0, batch=2)
    with pytest.raises(pkg.MMCQError):
        other.set_state(snap)
    assert np.array_equal(a.get_m(0), m_before)
    a.close()
    other.close()


def test_integrator_switch_keeps_accepted_state():
    """DP45 leaves the accepted state in either of its two buffers; switching
    to RK4 must continue from it (checked against the oracle doing the same)."""
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    from gpu_common import make_pair
    n = 16 * 8 * 2
    sim, o = make_pair(16, 8, 2, 4e-9, 8e5, 1.3e-11, 0.01)
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(41), 0.1)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    for h in (sim, o):
        h.set_bias((0.05, 0.0, 0.0))
        h.set_cavity(2 * np.pi * 8e9, 2 * np.pi * 1e7, 2 * np.pi * 2e8)
    sim.set_integrator(pkg.MMCQ_DP45, 1e-6, pkg.MMCQ_CAVITY_E)
    sim.step(3, 1e-13)
    for _ in range(4):
        if len(sim.dt_history()) % 2 == 1:
            break
        sim.step(1)
    hist = sim.dt_history()
    assert len(hist) % 2 == 1          # odd: accepted state in the second buffer
    o.set_integrator(oracle.DP45, 1e-6, oracle.CAV_E)
    o.replay(hist)
    sim.set_integrator(pkg.MMCQ_RK4, 0.0, pkg.MMCQ_CAVITY_E)
    o.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
    sim.step(20, 1e-13)
    o.step(20, 1e-13)
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    sim.close()
