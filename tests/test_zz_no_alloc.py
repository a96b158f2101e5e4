"""The allocation-free Jacobian action, through the C ABI.

fe_jacobian_action_noalloc serves callers that cannot call cudaMalloc while they run: an
application whose device memory is all handed out by its own pool allocator (a cudaMalloc would
fail, or take memory the pool counts on), or a host loop with a latency budget that cannot absorb
the device-wide synchronisation an allocation may cause.  The call keeps its cross-tile partial
sums in one static device array instead of the context's own buffer.

Checks: against the oracle on directions no other call has used, with the context's own cross-tile
buffer first filled with NaN (a fix-up that read it instead of the static array would return NaN);
against fe_jacobian_action on the same directions, two calls in a row; the device's free memory
unchanged across calls after the first; oversized problems rejected.  This file is collected last
so that a failure here leaves every other test already run; it also passes on its own in a fresh
process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5, -32: 1e-5}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _call(lib, fn, ctx, v, y, precision, stream):
    """fe_jacobian_action (cached linearisation: u = NULL) or fe_jacobian_action_noalloc."""
    vp, yp = ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(y.data_ptr())
    if fn == "fe_jacobian_action":
        return lib.fe_jacobian_action(ctx, None, vp, yp, precision, stream)
    return getattr(lib, fn)(ctx, vp, yp, precision, stream)


@pytest.mark.parametrize("dim,n,k", [(3, 6, 3), (2, 16, 2), (3, 5, 2)])
def test_noalloc_against_oracle_and_regular_action(dim, n, k):
    import torch
    from paper_2506_00746_gb300 import Operator, abi
    lib = abi.library()
    V = I.lattice_vertices(dim, n, seed=0)
    u = I.smooth_field(dim, n, k, seed=1)
    op = Operator(dim, n, k, V, p=3.0)
    P = O.Problem(dim, n, k, V, p=3.0)
    op.linearize(torch.from_numpy(u).cuda())
    stream = abi.stream_handle()
    nan64 = torch.full((op.n_dofs,), float("nan"), dtype=torch.float64, device="cuda")
    for precision in (64, 32, -32):
        dtype = torch.float32 if precision == 32 else torch.float64
        # two calls in a row, each on a direction that no earlier call of this context has seen
        for call, seed in enumerate((100 + precision, 200 + precision)):
            # the regular action on an all-NaN direction leaves NaN partial sums in the context's
            # own cross-tile buffer
            ynan = torch.empty(op.n_dofs, dtype=dtype, device="cuda")
            assert _call(lib, "fe_jacobian_action", op.ctx, nan64.to(dtype), ynan, precision, stream) == 0
            v = torch.from_numpy(I.uniform_vector(op.n_dofs, seed=seed)).cuda().to(dtype)
            y = torch.full_like(v, float("nan"))
            st = _call(lib, "fe_jacobian_action_noalloc", op.ctx, v, y, precision, stream)
            assert st == 0, abi.fe_last_error(op.ctx)
            got = y.double().cpu().numpy()
            assert np.all(np.isfinite(got)), (precision, call)
            # the oracle on the same direction (rounded to FP32 where the action reads FP32)
            vref = v.double().cpu().numpy() if precision == 32 else v.cpu().numpy()
            if precision == -32:
                vref = vref.astype(np.float32).astype(np.float64)
            assert _rel(got, O.jv(P, u, vref)) <= TOL[precision], (precision, call)
            # and the existing entry point on the same direction
            y_reg = torch.empty_like(v)
            assert _call(lib, "fe_jacobian_action", op.ctx, v, y_reg, precision, stream) == 0
            assert _rel(got, y_reg.double().cpu().numpy()) <= TOL[precision], (precision, call)
    op.close()


def test_noalloc_calls_take_no_device_memory():
    """After the first call (which may load the library's static array), further calls leave the
    device's free memory as it was."""
    import torch
    from paper_2506_00746_gb300 import Operator, abi
    lib = abi.library()
    op = Operator(3, 6, 3, I.lattice_vertices(3, 6, seed=0), p=3.0)
    op.linearize(torch.from_numpy(I.smooth_field(3, 6, 3, seed=1)).cuda())
    stream = abi.stream_handle()
    v = torch.from_numpy(I.uniform_vector(op.n_dofs, seed=7)).cuda()
    ys = [torch.empty_like(v) for _ in range(3)]
    assert _call(lib, "fe_jacobian_action_noalloc", op.ctx, v, ys[0], 64, stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for y in ys[1:]:
        assert _call(lib, "fe_jacobian_action_noalloc", op.ctx, v, y, 64, stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(ys[1], ys[0]) and torch.equal(ys[2], ys[0])     # same inputs, same bits
    op.close()


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    import torch
    from paper_2506_00746_gb300 import Operator, abi
    lib = abi.library()
    op = Operator(3, 56, 3, I.lattice_vertices(3, 56, seed=0), p=3.0)   # ~2.7M cross-tile partial sums
    op.linearize(torch.from_numpy(I.smooth_field(3, 56, 3, seed=1)).cuda())
    v = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(v)
    st = _call(lib, "fe_jacobian_action_noalloc", op.ctx, v, y, 64, abi.stream_handle())
    assert st == 5                                                        # 8-byte words exceed 16 MiB
    assert "static array holds" in abi.fe_last_error(op.ctx)
    op.close()
