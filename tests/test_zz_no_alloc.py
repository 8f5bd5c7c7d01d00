"""The allocation-free least-squares entry point, ph_mgs_solve_static.

Some callers cannot allocate device memory: a process whose GPU memory is all
reserved by another allocator (a framework's caching allocator or a fixed
arena) would fail, or take the owner's memory, on one more cudaMalloc, and a
real-time loop cannot afford the device synchronisation an allocation
implies.  For them the solve runs in a static device array instead of a
context's buffers.  Checked through the C ABI:

* two calls in a row (the second finds what the first left in the shared
  array) give the solution of ph_mgs_solve with the same (grid) kernel bit
  for bit, and the oracle's textbook MGS within the parity bound of the MGS
  tests;
* device-resident inputs and outputs on a caller's non-default stream;
* a stream being captured into a graph is refused without disturbing the
  capture; sizes beyond the static array are refused.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from gpu_common import cabs_diff, complex_matrix, lead_complex, mgs_tol
from paper_1501_06625_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_ctx():
    from paper_1501_06625_gb300 import build, libph
    build.build()
    oracle.build()
    c = libph.Context(0)
    yield libph, c
    c.close()


@pytest.mark.parametrize("L,N,n", [(2, 64, 64), (2, 50, 33), (4, 40, 40), (1, 96, 80)])
def test_static_solve_matches_context_solve_and_oracle(lib_ctx, L, N, n):
    libph, ctx = lib_ctx
    libph.ph_mgs_set_variant(ctx.h, L, N, n, 0)        # the grid kernel, as the static form
    for call in range(2):
        J, rhs = synth.random_lsq(9100 + 17 * call + N + n + L, L, N, n)
        dx_ref = np.zeros((L, 2, n))
        rn_ref = libph.ph_mgs_solve(ctx.h, L, N, n, J, rhs, dx_ref)
        dx = np.full((L, 2, n), np.nan)
        rn = libph.ph_mgs_solve_static(0, None, L, N, n, J, rhs, dx)
        assert np.array_equal(dx, dx_ref), call
        assert rn == rn_ref
        st, dxo, rno = oracle.mgs_solve(J, rhs)
        assert st == oracle.OK
        err = cabs_diff(dx, dxo).max() / np.abs(lead_complex(dxo)).max()
        assert err <= mgs_tol(complex_matrix(J), lead_complex(rhs), L), (call, err)
        assert abs(rn - rno) <= 1e-12 * (1.0 + rno)


def test_static_solve_device_arrays_on_a_caller_stream(lib_ctx):
    import torch
    libph, ctx = lib_ctx
    L, N, n = 2, 70, 64
    J, rhs = synth.random_lsq(9300, L, N, n)
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        dJ = torch.tensor(J, device=dev)
        drhs = torch.tensor(rhs, device=dev)
        ddx = torch.full((L, 2, n), float("nan"), dtype=torch.float64, device=dev)
    s.synchronize()
    for _ in range(2):
        rn = libph.ph_mgs_solve_static(0, s, L, N, n, dJ, drhs, ddx)
    s.synchronize()
    st, dxo, rno = oracle.mgs_solve(J, rhs)
    dx = ddx.cpu().numpy()
    err = cabs_diff(dx, dxo).max() / np.abs(lead_complex(dxo)).max()
    assert err <= mgs_tol(complex_matrix(J), lead_complex(rhs), L), err
    assert abs(rn - rno) <= 1e-12 * (1.0 + rno)


def test_static_solve_refuses_a_capturing_stream(lib_ctx):
    import torch
    libph, _ = lib_ctx
    L, N, n = 2, 16, 16
    J, rhs = synth.random_lsq(9400, L, N, n)
    dev = torch.device("cuda", 0)
    dx = np.zeros((L, 2, n))
    libph.ph_mgs_solve_static(0, None, L, N, n, J, rhs, dx)    # set-up outside the capture
    y = torch.zeros(4, device=dev)
    s = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g, stream=s):
        y.add_(1.0)
        try:
            libph.ph_mgs_solve_static(0, s, L, N, n, J, rhs, dx)
        except libph.PhError as e:
            refused = e.status
    assert refused == libph.PH_EINVAL
    g.replay()                                          # the capture was left intact
    torch.cuda.synchronize()
    assert float(y.sum()) == 4.0


def test_static_solve_refuses_oversized(lib_ctx):
    libph, _ = lib_ctx
    n = 176                                             # QD fits up to 175
    with pytest.raises(libph.PhError) as ei:
        libph.ph_mgs_solve_static(0, None, 4, n, n, np.zeros((4, 2, n, n)), np.zeros((4, 2, n)),
                                  np.zeros((4, 2, n)))
    assert ei.value.status == libph.PH_EINVAL
