"""The allocation-free Jacobian action against the regular one, through the C ABI.

fe_jacobian_action_noalloc serves callers that cannot allocate device memory while they run
(for instance code inside a global-mode stream capture, where cudaMalloc is not allowed, or an
application whose GPU memory all belongs to its own pool allocator).  It keeps its cross-tile
partial sums in one static device array instead of the context's buffer.  This file is collected
last so that a failure here leaves every other test already run; it also passes on its own in a
fresh process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5, -32: 1e-5}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dim,n,k", [(3, 6, 3), (2, 16, 2), (3, 5, 2)])
def test_noalloc_matches_regular_action(dim, n, k):
    import torch
    from paper_2506_00746_gb300 import Operator, abi
    lib = abi.library()
    op = Operator(dim, n, k, I.lattice_vertices(dim, n, seed=0), p=3.0)
    op.linearize(torch.from_numpy(I.smooth_field(dim, n, k, seed=1)).cuda())
    v64 = torch.from_numpy(I.uniform_vector(op.n_dofs, seed=2)).cuda()
    stream = abi.stream_handle()
    for precision in (64, 32, -32):
        v = v64.float() if precision == 32 else v64
        y_ref = torch.empty_like(v)
        assert lib.fe_jacobian_action(op.ctx, None, ctypes.c_void_p(v.data_ptr()),
                                      ctypes.c_void_p(y_ref.data_ptr()), precision, stream) == 0
        ref = y_ref.double().cpu().numpy()
        for _ in range(2):                             # two calls in a row share the static scratch
            y = torch.full_like(v, float("nan"))
            st = lib.fe_jacobian_action_noalloc(op.ctx, ctypes.c_void_p(v.data_ptr()),
                                                ctypes.c_void_p(y.data_ptr()), precision, stream)
            assert st == 0, abi.fe_last_error(op.ctx)
            assert _rel(y.double().cpu().numpy(), ref) <= TOL[precision]
    op.close()


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    import torch
    from paper_2506_00746_gb300 import Operator, abi
    lib = abi.library()
    op = Operator(3, 56, 3, I.lattice_vertices(3, 56, seed=0), p=3.0)   # ~2.7M cross-tile partial sums
    op.linearize(torch.from_numpy(I.smooth_field(3, 56, 3, seed=1)).cuda())
    v = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(v)
    st = lib.fe_jacobian_action_noalloc(op.ctx, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(y.data_ptr()), 64,
                                        abi.stream_handle())
    assert st == 5                                                        # 8-byte words exceed 16 MiB
    assert "static array holds" in abi.fe_last_error(op.ctx)
    op.close()
