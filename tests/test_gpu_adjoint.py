"""GPU discrete adjoint of the RK4 path against the oracle's adjoint (which
is pinned by finite differences): objective values and gradients with respect
to the bias, the B_rms scale, omega_c, kappa and the per-cell Ms map, per
instance of a batch, with the averaged photon-number term, with and without
checkpoint thinning; and the torch.autograd wrapper."""
import math

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

NX, NY, NZ, D = 12, 8, 3, 4e-9
W = (0.3, -0.7, 0.2)
WN = 5.0
WAVG, WINDOW = 3.0, 9
STEPS, DT = 30, 2e-13
BIASES = [(0.05, 0.01, 0.0), (0.08, -0.02, 0.01)]


def _instance_inputs(b, n):
    import synthetic
    m0 = synthetic.tilted_m(n, synthetic.derive_seed(80, b), 0.3)
    prof = np.random.default_rng(81).normal(size=(n, 3)).astype(np.float32) * 2e-3
    return m0, prof


@pytest.mark.parametrize("masked,ckpt", [(False, 1), (True, 7)], ids=["full-every-step", "masked-every-7"])
def test_adjoint_gradients_match_oracle(masked, ckpt):
    require_gpu()
    import oracle
    import paper_2410_00966_gb300 as pkg
    import synthetic
    n = NX * NY * NZ
    ms = synthetic.disk_ms(NX, NY, NZ, D, D, 40e-9, 8e5) if masked else np.full(n, 8e5, np.float32)
    sim = pkg.Sim(NX, NY, NZ, D, D, D, 8e5, 1.3e-11, 0.02, Ku=2e4, axis=(0.6, 0.8, 0.0), batch=len(BIASES))
    sim.set_ms_map(ms)
    wc, kap = 2 * math.pi * 7e9, 2 * math.pi * 3e8
    for b, bias in enumerate(BIASES):
        m0, prof = _instance_inputs(b, n)
        sim.set_m(m0, inst=b)
        sim.set_bias(bias, inst=b)
    sim.set_cavity(wc, kap, profile=prof, profile_is_brms=True)
    sim.set_cavity_init(0.8, -0.4)
    sim.set_integrator(pkg.MMCQ_DP45, 1e-6, pkg.MMCQ_CAVITY_E)     # restored after the adjoint
    J, g, gms = sim.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW, ckpt_every=ckpt, ms_grad=True)
    for b, bias in enumerate(BIASES):
        m0, prof = _instance_inputs(b, n)
        o = oracle.Oracle(NX, NY, NZ, D, D, D, 8e5, 1.3e-11, 0.02, Ku=2e4, axis=(0.6, 0.8, 0.0))
        o.set_ms(ms.astype(np.float64))
        o.set_m(m0.astype(np.float64))
        o.set_bias(bias)
        o.set_cavity(wc, kap, profile=prof.astype(np.float64), profile_is_brms=True)
        o.set_cavity_init(0.8, -0.4)
        o.set_integrator(oracle.RK4, 0.0, oracle.CAV_E)
        Jo, go, _, gso = o.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW)
        print(f"instance {b}: J {J[b]:.9e} vs {Jo:.9e}; grad {g[b]} vs {go}")
        assert abs(J[b] - Jo) <= 1e-5 * abs(Jo)
        assert np.abs(g[b, :3] - go[:3]).max() <= 2e-3 * np.abs(go[:3]).max()
        for k in (3, 4, 5):
            assert abs(g[b, k] - go[k]) <= 2e-3 * abs(go[k]), k
        assert np.abs(gms[b] - gso).max() <= 2e-3 * np.abs(gso).max()
        assert np.all(gms[b][ms <= 0] == 0)
        assert np.abs(sim.get_m(b).astype(np.float64) - o.get_m()).max() <= 1e-5
    assert sim.cavity()["accepted"] == STEPS
    sim.close()


def test_adjoint_refuses_unsupported_settings():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    sim = pkg.Sim(8, 8, 1, D, D, D, 8e5, 1.3e-11, 0.02)
    sim.set_cavity(1e10, 1e7, 1e8)
    sim.set_integrator(pkg.MMCQ_RK4, 0.0, pkg.MMCQ_CAVITY_P)
    with pytest.raises(pkg.MMCQError) as e:
        sim.adjoint_rk4(3, 1e-13, W, WN)
    assert e.value.code == pkg.MMCQ_ERR_UNSUPPORTED
    sim.set_integrator(pkg.MMCQ_RK4, 0.0, pkg.MMCQ_CAVITY_E)
    with pytest.raises(pkg.MMCQError) as e:
        sim.adjoint_rk4(0, 1e-13, W, WN)
    assert e.value.code == pkg.MMCQ_ERR_ARG
    sim.close()


def test_checkpoint_thinning_is_exact():
    require_gpu()
    import paper_2410_00966_gb300 as pkg
    out = []
    for ckpt in (1, 4, 30):
        sim = pkg.Sim(NX, NY, NZ, D, D, D, 8e5, 1.3e-11, 0.02, batch=1)
        m0, prof = _instance_inputs(0, NX * NY * NZ)
        sim.set_m(m0)
        sim.set_bias(BIASES[0])
        sim.set_cavity(2 * math.pi * 7e9, 2 * math.pi * 3e8, profile=prof, profile_is_brms=True)
        out.append(sim.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW, ckpt_every=ckpt, ms_grad=True))
        sim.close()
    for J, g, gms in out[1:]:
        assert np.array_equal(J, out[0][0]) and np.array_equal(g, out[0][1]) and np.array_equal(gms, out[0][2])


def test_autograd_wrapper_returns_the_adjoint_gradient():
    require_gpu()
    torch = pytest.importorskip("torch")
    import paper_2410_00966_gb300 as pkg
    n = NX * NY * NZ
    sim = pkg.Sim(NX, NY, NZ, D, D, D, 8e5, 1.3e-11, 0.02, batch=2)
    m0 = [_instance_inputs(b, n)[0] for b in range(2)]
    prof = _instance_inputs(0, n)[1]
    p = torch.tensor([[0.05, 0.01, 0.0, 2 * math.pi * 3e8, 2 * math.pi * 7e9, 2 * math.pi * 3e7],
                      [0.08, -0.02, 0.01, 2 * math.pi * 2e8, 2 * math.pi * 7.5e9, 2 * math.pi * 3e7]],
                     dtype=torch.float64, requires_grad=True)
    ms = torch.full((n,), 8e5, dtype=torch.float64, requires_grad=True)
    J = pkg.cavity_objective(sim, m0, p, STEPS, DT, W, WN, WAVG, WINDOW, profile=prof, ms=ms)
    (2.0 * J[0] + 3.0 * J[1]).backward()
    # the same numbers straight from the adjoint call
    for b in range(2):
        sim.set_m(m0[b], inst=b)
    sim.reset_cavity()
    _, g, gms = sim.adjoint_rk4(STEPS, DT, W, WN, WAVG, WINDOW, ms_grad=True)
    gd = g.copy()
    gd[:, 3] /= p.detach().numpy()[:, 3]
    np.testing.assert_allclose(p.grad.numpy(), np.array([2.0, 3.0])[:, None] * gd, rtol=1e-12)
    ref = 2.0 * gms[0].astype(np.float64) + 3.0 * gms[1].astype(np.float64)
    np.testing.assert_allclose(ms.grad.numpy(), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
    sim.close()
