"""Mode frequencies of GPU runs: the spectrum of the recorded spatial average
of m (Appendix C: the numerical Fourier transform of the averaged
magnetisation), taken on the device by mmcq_spectrum at the DFT bins
omega_k = 2 pi k / (n dt) of the run, must put each mode within one bin of
where the closed form or the oracle puts it.

* Dicke model (Sec. 4): one cubic cell mapped onto the Dicke Hamiltonian,
  omega_z = omega_c = 2 pi 10 GHz, lambda / lambda_c = 0.3 and 0.6, no loss:
  the two peaks of <m_x> are the normal-phase polaritons of Eq.
  dickepolaritons.
* Multi-cell Kittel mode: a 6x4x2 element of 2 nm cells (smaller than the
  exchange length, so close to uniform), bias 0.1 T along x, no damping: the
  <m_y> peak sits within one bin of Kittel's formula with the element's
  Aharoni prism factors (the oracle pins the frequency itself to 0.5 %).
* The 32x32x1 film of the small workload (4 nm Permalloy, bias 50 mT, a
  uniform 0.02 rad tilt): its main <m_y> peak on the GPU is the oracle's, bin
  for bin.  (That peak is near 3 GHz, not at the macrospin Kittel value of the
  whole film, 6.04 GHz: the internal field of a 128 nm square is far from
  uniform.)
"""
import math

import numpy as np
import pytest

from gpu_common import make_pair, require_gpu

pytestmark = pytest.mark.gpu


def _bins(n, dt, lo, hi):
    bw = 2 * math.pi / (n * dt)
    k = np.arange(max(1, int(lo / bw)), int(hi / bw) + 2)
    return k * bw, bw


def _peaks(S, count):
    a = np.abs(S)
    idx = [i for i in range(1, len(a) - 1) if a[i] > a[i - 1] and a[i] >= a[i + 1]]
    return sorted(sorted(idx, key=lambda i: -a[i])[:count])


@pytest.mark.parametrize("ratio", [0.3, 0.6])
def test_dicke_polaritons_from_gpu_spectrum(ratio):
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    cell, Ms = 4e-9, 8e5
    gam = oracle.GAMMA_LL
    S = Ms * cell ** 3 / (oracle.HBAR * gam)
    wc = wz = 2 * math.pi * 10e9
    lam = ratio * math.sqrt(wc * wz) / 2
    sim = pkg.Sim(1, 1, 1, cell, cell, cell, Ms, 1e-11, 0.0)
    sim.set_m(np.array([[0.02, 0.0, 1.0]], np.float32))
    sim.set_bias((0, 0, wz / gam))
    sim.set_cavity(wc, 0.0, profile=np.array([[math.sqrt(2 / S) * lam / gam, 0.0, 0.0]], np.float32),
                   profile_is_brms=True)
    n, dt = 1 << 15, 2e-12
    sim.set_recording(1)
    sim.step(n, dt)
    assert len(sim.mavg_history()) == n
    w, bw = _bins(n, dt, 0.4 * wc, 1.7 * wc)
    spec = sim.spectrum(w, comp=0)
    top = _peaks(spec, 2)
    r = math.sqrt(16 * lam ** 2 * wz * wc)
    expect = [math.sqrt((wz ** 2 + wc ** 2 - r) / 2), math.sqrt((wz ** 2 + wc ** 2 + r) / 2)]
    print(f"lambda/lambda_c = {ratio}: peaks {[w[i] / 2 / math.pi / 1e9 for i in top]} GHz, "
          f"Eq. dickepolaritons {[e / 2 / math.pi / 1e9 for e in expect]} GHz, bin {bw / 2 / math.pi / 1e6:.1f} MHz")
    for i, e in zip(top, expect):
        assert abs(w[i] - e) <= bw
    sim.close()


def _prism_factors(oracle, Lx, Ly, Lz):
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return oracle.aharoni_dz(b, c, a), oracle.aharoni_dz(c, a, b), oracle.aharoni_dz(a, b, c)


def test_multicell_kittel_mode_from_gpu_spectrum():
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    nx, ny, nz, d, Ms, B = 6, 4, 2, 2e-9, 8e5, 0.1
    D = _prism_factors(oracle, nx * d, ny * d, nz * d)
    wk = oracle.GAMMA_LL * math.sqrt((B + (D[1] - D[0]) * oracle.MU0 * Ms) * (B + (D[2] - D[0]) * oracle.MU0 * Ms))
    sim = pkg.Sim(nx, ny, nz, d, d, d, Ms, 1.3e-11, 0.0)
    th = 1e-3
    sim.set_m(np.tile(np.array([math.cos(th), math.sin(th), 0.0], np.float32), (nx * ny * nz, 1)))
    sim.set_bias((B, 0.0, 0.0))
    n, dt = 1 << 15, 2 * math.pi / wk / 2000
    sim.set_recording(1)
    sim.step(n, dt)
    w, bw = _bins(n, dt, 0.5 * wk, 1.5 * wk)
    spec = sim.spectrum(w, comp=1)
    k = int(np.argmax(np.abs(spec)))
    print(f"6x4x2 element: peak {w[k] / 2 / math.pi / 1e9:.4f} GHz, Kittel {wk / 2 / math.pi / 1e9:.4f} GHz, "
          f"bin {bw / 2 / math.pi / 1e6:.1f} MHz")
    assert abs(w[k] - wk) <= bw
    sim.close()


def test_film_mode_matches_oracle_bin_for_bin():
    require_gpu()
    import oracle
    nx, ny, nz, d = 32, 32, 1, 4e-9
    sim, o = make_pair(nx, ny, nz, d, 8e5, 1.3e-11, 0.01)
    th = 0.02
    m0 = np.tile(np.array([math.cos(th), math.sin(th), 0.0], np.float32), (nx * ny, 1))
    sim.set_m(m0)
    o.set_m(m0.astype(np.float64))
    sim.set_bias((0.05, 0.0, 0.0))
    o.set_bias((0.05, 0.0, 0.0))
    n, dt = 1 << 13, 2e-13
    sim.set_recording(1)
    o.set_recording(True)
    sim.step(n, dt)
    o.step(n, dt)
    w, bw = _bins(n, dt, 2 * math.pi * 0.5e9, 2 * math.pi * 20e9)
    hg, ho = sim.mavg_history(), o.mavg_history()
    np.testing.assert_allclose(hg[:, 0], ho[:, 0], rtol=1e-12)
    sg = sim.spectrum(w, comp=1)
    so = oracle.spectrum(ho[:, 0], ho[:, 2], w)
    kg, ko = int(np.argmax(np.abs(sg))), int(np.argmax(np.abs(so)))
    print(f"32x32x1 film: GPU peak {w[kg] / 2 / math.pi / 1e9:.3f} GHz, oracle {w[ko] / 2 / math.pi / 1e9:.3f} GHz, "
          f"bin {bw / 2 / math.pi / 1e6:.0f} MHz; spectra differ by "
          f"{np.abs(sg - so).max() / np.abs(so).max():.2e} of the peak")
    assert kg == ko
    assert np.abs(sg - so).max() <= 1e-3 * np.abs(so).max()
    sim.close()
