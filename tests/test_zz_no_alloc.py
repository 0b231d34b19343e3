"""The allocation-free coupling sum (mmcq_coupling_sum_noalloc).

Some callers cannot allocate device memory: code that runs inside a host
framework whose memory pool owns the GPU, or a latency-bound loop that cannot
pay for cudaMalloc's device-wide synchronisation.  For them the library offers
one entry point whose scratch lives in a fixed static device array.  This test
calls it through the C ABI on device arrays and checks, on two calls in a row,
that it returns the same FP64 coupling sum X as the handle-based read-out
(mmcq_get_cavity), and that an oversized request is refused on the host.

The file name makes pytest collect it last, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import ctypes
import math

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_coupling_sum_matches_handle_readout():
    require_gpu()
    import torch

    import paper_2410_00966_gb300 as pkg
    import synthetic

    nx, ny, nz, d = 24, 20, 3, 4e-9
    n = nx * ny * nz
    sim = pkg.Sim(nx, ny, nz, d, d, d, 8e5, 1.3e-11, 0.01)
    ms = synthetic.disk_ms(nx, ny, nz, d, d, 80e-9, 8e5)
    sim.set_ms_map(ms)
    sim.set_m(synthetic.tilted_m(n, synthetic.derive_seed(77, 0), 0.6))
    # B_rms in tesla with a component along m (no cancellation in the sum)
    brms = (1e-6 * np.stack([np.linspace(0.5, 1.5, n), 0.3 * np.ones(n), np.zeros(n)], 1)).astype(np.float32)
    sim.set_cavity(2 * math.pi * 6e9, 2 * math.pi * 10e6, profile=brms, profile_is_brms=True)
    sim.step(20, 1e-13)
    x_ref = sim.cavity()["X"]

    dev = torch.device("cuda", 0)
    m_dev = torch.empty((n, 3), dtype=torch.float32, device=dev)
    sim.get_m(0, out=m_dev)
    ms_dev = torch.from_numpy(ms).to(dev)
    brms_dev = torch.from_numpy(brms).to(dev)
    torch.cuda.synchronize()
    lib = pkg.lib()
    vc = d ** 3
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    outs = []
    for _ in range(2):
        out = ctypes.c_double(0.0)
        rc = lib.mmcq_coupling_sum_noalloc(ctypes.c_void_p(m_dev.data_ptr()), ctypes.c_void_p(ms_dev.data_ptr()),
                                           ctypes.c_void_p(brms_dev.data_ptr()), n, vc, ctypes.byref(out), stream)
        assert rc == pkg.MMCQ_OK
        outs.append(out.value)
    assert x_ref != 0.0
    for x in outs:
        assert abs(x - x_ref) <= 1e-9 * abs(x_ref), (x, x_ref)
    assert outs[0] == outs[1]

    # beyond the static scratch: refused on the host with a clear code
    big = 4096 * 4096 + 1
    out = ctypes.c_double(0.0)
    rc = lib.mmcq_coupling_sum_noalloc(ctypes.c_void_p(m_dev.data_ptr()), ctypes.c_void_p(ms_dev.data_ptr()),
                                       ctypes.c_void_p(brms_dev.data_ptr()), big, vc, ctypes.byref(out), stream)
    assert rc == pkg.MMCQ_ERR_UNSUPPORTED
    sim.close()
