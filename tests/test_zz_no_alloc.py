"""The allocation-free residual entry point (dugks_residual_static).

Some callers of this library cannot call cudaMalloc: hosts whose own allocator already owns
the device memory, and loops that must not take cudaMalloc's implicit synchronisation.
dugks_residual_static gives them the FP64 residual and conservation totals with its partial
sums in a fixed device array. This test calls it through the C ABI and checks it against
dugks_residual (the handle's own reduction, which allocates its buffer at creation) on two
calls in a row, including a mesh above 4096 * 2048 cells where both reductions stride over
their cells with the capped number of blocks. It sits in a file of its own that pytest
collects last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1411_6121_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _call(lib, q, store, state, shape, rt, rho0, shift, uprev, have_prev, stream):
    dim = len(shape)
    nx, ny = shape[0], shape[1]
    nz = shape[2] if dim == 3 else 1
    out = np.zeros(dim + 2)
    sh = (C.c_double * 3)(*shift)
    rc = lib.dugks_residual_static(q, store, C.c_void_p(state.data_ptr()), nx, ny, nz, rt, rho0, sh, None,
                                   C.c_void_p(uprev.data_ptr()), have_prev, out.ctypes.data_as(C.POINTER(C.c_double)),
                                   C.c_void_p(stream))
    return rc, out


@pytest.mark.parametrize("q,shape,store", [(19, (40, 20, 12), 0), (9, (45, 38), 0), (19, (24, 16, 10), 1),
                                           (19, (256, 256, 130), 0)])
def test_static_residual_matches_handle(q, shape, store):
    import torch
    from paper_1411_6121_gb300 import dugks
    lib = dugks.load()
    dim = len(shape)
    g = (1e-5, 0.0, 0.0)
    dt = 0.5
    cfg = dict(shape=shape, q=q, nu=0.05, dt=dt, g=g, bcs=W.channel_bcs(dim), store=store)
    sim = dugks.Sim(**cfg)
    p, u = W.random_state_fields(shape, seed=3, u_amp=0.02, p_amp=1e-4)
    sim.init(p=p, u=u)
    ncell = int(np.prod(shape))
    nbytes = sim.state_bytes()
    state = torch.empty(nbytes // 2, dtype=torch.int16, device="cuda")
    uprev = torch.zeros(dim * ncell, dtype=torch.float64, device="cuda")
    shift = [gi * dt / 2 for gi in g]  # G(t) dt/2 with omega = 0
    stream = torch.cuda.current_stream().cuda_stream
    for call, steps in enumerate((5, 40)):
        sim.step(steps)
        ref = sim.residual()
        sim.get_state(out=state)
        torch.cuda.synchronize()
        rc, got = _call(lib, q, store, state, shape, 1.0 / 3.0, 1.0, shift, uprev, call, stream)
        assert rc == 0, lib.dugks_last_error(None)
        if call == 0:
            assert np.isinf(got[0]) and np.isinf(ref[0])
        else:
            assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert np.allclose(got[1:], ref[1:], rtol=1e-13, atol=1e-13 * abs(ref[1]))
    sim.close()


def test_static_residual_rejects_oversize():
    from paper_1411_6121_gb300 import dugks
    lib = dugks.load()
    out = np.zeros(5)
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    rc = lib.dugks_residual_static(19, 0, dummy, 257, 256, 256, 1.0 / 3.0, 1.0, None, None, dummy, 0,
                                   out.ctypes.data_as(C.POINTER(C.c_double)), None)
    assert rc == -1
    assert b"16777216" in lib.dugks_last_error(None)
