"""GPU excitation and spectra (the paper's Appendix C: B_ext += amp B_rms
sinc(omega_cut t); the response is the Fourier transform of the spatially
averaged m) against the oracle on identical seeded inputs."""
import math

import numpy as np
import pytest

from gpu_common import make_pair, require_gpu

pytestmark = pytest.mark.gpu

NX, NY, NZ, D = 20, 12, 3, 4e-9


def _setup(kind, mode=0, every=1):
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    n = NX * NY * NZ
    sim, o = make_pair(NX, NY, NZ, D, 8e5, 1.3e-11, 0.02)
    ms = synthetic.disk_ms(NX, NY, NZ, D, D, 70e-9, 8e5)
    sim.set_ms_map(ms)
    o.set_ms(ms.astype(np.float64))
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(60), 0.05)
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    prof = synthetic.lorentzian_profile(NX, NY, NZ, D, 30e-9)
    for h in (sim, o):
        h.set_bias((0.04, 0.0, 0.0))
        h.set_cavity(2 * math.pi * 6e9, 2 * math.pi * 2e7, 2 * math.pi * 3e8,
                     profile=prof if h is sim else prof.astype(np.float64))
        h.set_drive(2e4, 2 * math.pi * 30e9, 15e-12)
    sim.set_integrator(kind, 1e-6, mode)
    o.set_integrator(oracle.DP45 if kind == 1 else oracle.RK4, 1e-6, mode)
    sim.set_recording(every)
    o.set_recording(True)
    return sim, o


def test_drive_field_matches_oracle():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    sim, o = _setup(0)
    sim.step(7, 1e-13)
    o.step(7, 1e-13)
    m = sim.get_m().astype(np.float64)
    assert o.drive_factor(7e-13) != 0.0
    Bz = sim.eval_field(pkg.MMCQ_TERM_ZEEMAN).astype(np.float64)
    # o.field(m) with Gamma = 0: bias + drive (+ demag, exchange, anisotropy removed here)
    ref = o.field(m) - o.demag(m) - o.exchange(m) - o.anis(m)
    mag = np.abs(m).sum(axis=1) > 0          # the GPU's field terms live on magnetised cells
    assert mag.sum() < mag.size
    assert np.abs(Bz[mag] - ref[mag]).max() <= 1e-6 * np.abs(ref[mag]).max()
    sim.close()


@pytest.mark.parametrize("mode", [0, 1], ids=["E", "P"])
def test_driven_rk4_trajectory_and_recorded_average(mode):
    require_gpu()
    sim, o = _setup(0, mode)
    sim.step(300, 1e-13)
    o.step(300, 1e-13)
    dm = np.abs(sim.get_m().astype(np.float64) - o.get_m()).max()
    hg, ho = sim.mavg_history(), o.mavg_history()
    print(f"mode {mode}: max|dm| {dm:.3e}, max|d<m>| {np.abs(hg[:, 1:] - ho[:, 1:]).max():.3e}")
    assert dm <= 1e-5
    assert hg.shape == ho.shape == (300, 4)
    assert np.allclose(hg[:, 0], ho[:, 0], rtol=1e-13, atol=0)
    assert np.abs(hg[:, 1:] - ho[:, 1:]).max() <= 1e-6
    sim.close()


def test_driven_dp45_replay_and_decimated_recording():
    require_gpu()
    sim, o = _setup(1, 0, every=3)
    sim.step(40, 1e-13)
    hist = sim.dt_history()
    o.replay(hist)
    assert np.abs(sim.get_m().astype(np.float64) - o.get_m()).max() <= 1e-5
    hg, ho = sim.mavg_history(), o.mavg_history()
    assert len(hg) == len(hist) // 3
    assert np.abs(hg[:, 1:] - ho[2::3][:len(hg), 1:]).max() <= 1e-6
    sim.close()


def test_spectrum_kernel_matches_oracle_transform():
    require_gpu()
    import oracle
    sim, o = _setup(0)
    sim.step(600, 1e-13)
    o.step(600, 1e-13)
    hg, ho = sim.mavg_history(), o.mavg_history()
    w = 2 * math.pi * np.linspace(0.5e9, 20e9, 257)
    for comp in range(3):
        Sg = sim.spectrum(w, comp)
        # the device transform of the device samples equals the oracle's transform of the same samples
        Sr = oracle.spectrum(hg[:, 0], hg[:, 1 + comp], w)
        assert np.abs(Sg - Sr).max() <= 1e-12 * np.abs(Sr).max() + 1e-30
        # and the physics: transform of the oracle's own trajectory
        So = oracle.spectrum(ho[:, 0], ho[:, 1 + comp], w)
        assert np.abs(Sg - So).max() <= 1e-4 * np.abs(So).max() + 1e-22
    sim.close()


def test_spectrum_without_recording_is_refused():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    sim = pkg.Sim(4, 4, 1, D, D, D, 8e5, 1.3e-11, 0.01)
    with pytest.raises(pkg.MMCQError) as e:
        sim.spectrum([1e10])
    assert e.value.code == pkg.MMCQ_ERR_STATE
    sim.close()
