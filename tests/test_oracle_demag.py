"""Pins of the oracle's demag tensor and demag convolution.

Nothing here compares the oracle with itself: each check ties it to an
independent closed form (Aharoni's prism factors, the point dipole, Laplace's
equation), to an independent FFT (numpy's), or to a brute-force sum.
"""
import itertools
import math

import numpy as np
import pytest


def _prism_factors(oracle, Lx, Ly, Lz):
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return np.array([oracle.aharoni_dz(b, c, a), oracle.aharoni_dz(c, a, b), oracle.aharoni_dz(a, b, c)])


def test_aharoni_closed_form_sanity(oracle_mod):
    # cube: 1/3 each; any prism: the three factors sum to 1
    assert abs(oracle_mod.aharoni_dz(1, 1, 1) - 1 / 3) < 1e-14
    for L in [(1, 2, 3), (10, 10, 0.3), (0.2, 5, 1)]:
        assert abs(_prism_factors(oracle_mod, *L).sum() - 1) < 1e-12
    # thin-film limit: Dz -> 1 as the film gets thinner
    assert _prism_factors(oracle_mod, 1000, 1000, 1)[2] > 0.99


@pytest.mark.parametrize("cell", [(1, 1, 1), (1, 2, 3), (4, 4, 1), (2, 0.5, 0.7)])
def test_self_term_equals_aharoni(oracle_mod, cell):
    N = oracle_mod.newell(0, 0, 0, *cell)
    D = _prism_factors(oracle_mod, *cell)
    np.testing.assert_allclose(N[:3], D, rtol=0, atol=1e-13)
    np.testing.assert_allclose(N[3:], 0, atol=1e-14)
    assert abs(N[:3].sum() - 1) < 1e-13


def test_sample_average_equals_aharoni(oracle_mod):
    # (1/n) sum_i sum_j N(r_i - r_j) is the demag factor of the whole sample,
    # so the cell-pair tensor must reproduce Aharoni's prism factors.
    nx, ny, nz, d = 4, 3, 2, (1.0, 1.5, 0.7)
    acc = np.zeros(6)
    cells = list(itertools.product(range(nx), range(ny), range(nz)))
    for (i, j, k) in cells:
        for (a, b, c) in cells:
            acc += oracle_mod.demag_tensor((i - a) * d[0], (j - b) * d[1], (k - c) * d[2], *d)
    acc /= len(cells)
    D = _prism_factors(oracle_mod, nx * d[0], ny * d[1], nz * d[2])
    np.testing.assert_allclose(acc[:3], D, atol=1e-12)
    np.testing.assert_allclose(acc[3:], 0, atol=1e-13)


def test_long_chain_average_crosses_switch_radius(oracle_mod):
    # 64-cell chain: most pairs are beyond the switch radius (dipole form);
    # the average must still match the prism factor to the dipole form's accuracy.
    n = 64
    acc = np.zeros(6)
    for i in range(n):
        for j in range(n):
            acc += oracle_mod.demag_tensor(float(i - j), 0, 0, 1, 1, 1)
    acc /= n
    D = _prism_factors(oracle_mod, n, 1, 1)
    np.testing.assert_allclose(acc[:3], D, atol=2e-7)


def test_parity_and_permutation_symmetry(oracle_mod):
    X, Y, Z, d = 2.0, 3.0, 1.5, (1.0, 1.3, 0.6)
    N0 = oracle_mod.newell(X, Y, Z, *d)
    tol = 1e-11 * np.abs(N0).max()
    for sx, sy, sz in itertools.product([1, -1], repeat=3):
        N = oracle_mod.newell(sx * X, sy * Y, sz * Z, *d)
        np.testing.assert_allclose(N[:3], N0[:3], atol=tol)
        np.testing.assert_allclose(N[3], sx * sy * N0[3], atol=tol)   # xy odd in x, y
        np.testing.assert_allclose(N[4], sx * sz * N0[4], atol=tol)   # xz odd in x, z
        np.testing.assert_allclose(N[5], sy * sz * N0[5], atol=tol)   # yz odd in y, z
    assert abs(N0[3]) > 1e3 * tol and abs(N0[4]) > 1e3 * tol and abs(N0[5]) > 1e3 * tol
    # relabelling axes x<->y permutes the components
    Np = oracle_mod.newell(Y, X, Z, d[1], d[0], d[2])
    np.testing.assert_allclose([Np[1], Np[0], Np[2], Np[3], Np[5], Np[4]], N0, atol=tol)


def test_trace_vanishes_off_self(oracle_mod):
    # Laplace: outside the source the potential is harmonic, so the trace of the
    # cell-pair tensor is the overlap volume / V, which is 0 for distinct cells.
    for off in [(1, 0, 0), (0, 1, 0), (1, 1, 1), (3, -2, 1), (5, 5, 0)]:
        N = oracle_mod.newell(off[0] * 1.0, off[1] * 1.2, off[2] * 0.8, 1.0, 1.2, 0.8)
        assert abs(N[:3].sum()) < 1e-13 * max(1.0, np.abs(N).max())


def test_far_field_dipole_limit(oracle_mod):
    # relative deviation from the point dipole falls off like r^-4 for cubes
    errs = []
    for r in [4, 8, 16]:
        Nl = oracle_mod.newell(r, 0.5 * r, 0.25 * r, 1, 1, 1, long_double=True)
        Dp = oracle_mod.dipole(r, 0.5 * r, 0.25 * r, 1.0)
        errs.append(np.abs(Nl - Dp).max() / np.abs(Nl).max())
    assert errs[2] < 2e-5
    assert 10 < errs[0] / errs[1] < 25 and 10 < errs[1] / errs[2] < 25


def test_double_vs_long_double(oracle_mod):
    # cancellation in the 27-point stencil grows like r^5 (terms ~ r^3 log r,
    # result ~ r^-3) and stays below 1e-7 relative inside the switch radius
    for off in [(0, 0, 0), (1, 0, 0), (1, 2, 3), (4, 1, 0), (7, 3, 2), (12, 0, 5)]:
        a = oracle_mod.newell(*off, 1.0, 1.0, 1.0)
        b = oracle_mod.newell(*off, 1.0, 1.0, 1.0, long_double=True)
        r = max(1.0, math.sqrt(sum(v * v for v in off)))
        assert np.abs(a - b).max() <= 1e-13 * r ** 5 * np.abs(b).max()
    r = oracle_mod.r_switch()
    a = oracle_mod.newell(r, 0, 0, 1, 1, 1)
    b = oracle_mod.newell(r, 0, 0, 1, 1, 1, long_double=True)
    assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max()


def _numpy_fft_demag(oracle_mod, nx, ny, nz, d, ms, m, mu0):
    # independent convolution: numpy FFT on a padded grid of exactly 2n per axis
    px, py, pz = 2 * nx, 2 * ny, 2 * nz
    K = np.zeros((6, pz, py, px))
    for k in range(pz):
        for j in range(py):
            for i in range(px):
                X = i if i < nx else i - px
                Y = j if j < ny else j - py
                Z = k if k < nz else k - pz
                if abs(X) >= nx or abs(Y) >= ny or abs(Z) >= nz:
                    continue
                K[:, k, j, i] = oracle_mod.demag_tensor(X * d[0], Y * d[1], Z * d[2], *d)
    Kh = np.fft.fftn(K, axes=(1, 2, 3))
    M = np.zeros((3, pz, py, px))
    M[:, :nz, :ny, :nx] = (ms[:, None] * m).T.reshape(3, nz, ny, nx)
    Mh = np.fft.fftn(M, axes=(1, 2, 3))
    xx, yy, zz, xy, xz, yz = Kh
    H = np.stack([xx * Mh[0] + xy * Mh[1] + xz * Mh[2],
                  xy * Mh[0] + yy * Mh[1] + yz * Mh[2],
                  xz * Mh[0] + yz * Mh[1] + zz * Mh[2]])
    h = np.fft.ifftn(H, axes=(1, 2, 3)).real[:, :nz, :ny, :nx]
    return -mu0 * h.reshape(3, -1).T


@pytest.mark.parametrize("shape", [(5, 7, 3), (8, 1, 1), (1, 6, 1), (1, 1, 5), (6, 4, 1), (3, 3, 3)])
def test_direct_fft_numpy_agree(oracle_mod, shape):
    nx, ny, nz = shape
    d = (4e-9, 3e-9, 2.5e-9)
    rng = np.random.default_rng(sum(shape))
    n = nx * ny * nz
    m = rng.normal(size=(n, 3))
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    ms = 8e5 * (0.5 + rng.random(n))
    ms[rng.random(n) < 0.2] = 0.0
    od = oracle_mod.Oracle(nx, ny, nz, *d, 8e5, 1e-11, 0.01, demag=oracle_mod.DEMAG_DIRECT)
    of = oracle_mod.Oracle(nx, ny, nz, *d, 8e5, 1e-11, 0.01, demag=oracle_mod.DEMAG_FFT)
    od.set_ms(ms)
    of.set_ms(ms)
    mm = m * (ms > 0)[:, None]
    Bd, Bf = od.demag(mm), of.demag(mm)
    Bn = _numpy_fft_demag(oracle_mod, nx, ny, nz, d, ms, mm, oracle_mod.MU0)
    scale = np.abs(Bd).max()
    assert np.abs(Bd - Bf).max() <= 1e-12 * scale
    assert np.abs(Bd - Bn).max() <= 1e-12 * scale
    # sampled direct evaluation (used at full size) agrees too
    cells = np.arange(0, n, 3)
    np.testing.assert_allclose(od.demag_at(mm, cells), Bd[cells], atol=1e-12 * scale)


def test_uniform_sample_mean_field(oracle_mod):
    # uniformly magnetised prism: the cell-averaged demag field is -mu0 Ms D
    nx, ny, nz, d, Ms = 12, 8, 2, 2e-9, 8e5
    o = oracle_mod.Oracle(nx, ny, nz, d, d, d, Ms, 1e-11, 0.01)
    D = _prism_factors(oracle_mod, nx * d, ny * d, nz * d)
    for axis in range(3):
        m = np.zeros((nx * ny * nz, 3))
        m[:, axis] = 1.0
        B = o.demag(m).mean(0)
        assert abs(B[axis] + oracle_mod.MU0 * Ms * D[axis]) < 1e-11
        assert np.abs(np.delete(B, axis)).max() < 1e-11


def test_own_fft_matches_numpy(oracle_mod):
    rng = np.random.default_rng(3)
    a = rng.normal(size=(4, 8, 16)) + 1j * rng.normal(size=(4, 8, 16))
    np.testing.assert_allclose(oracle_mod.fft3d(a, -1), np.fft.fftn(a), atol=1e-12)
    np.testing.assert_allclose(oracle_mod.fft3d(a, +1), np.fft.ifftn(a) * a.size, atol=1e-12)
