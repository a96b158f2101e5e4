"""Stream order of back-to-back Jacobian actions.

The FP32 tile kernel is launched programmatically: its first CTAs may be scheduled while the
fix-up of the previous action still runs, and wait for it before they read their input or write
the halo array.  Chained actions (each one's output the next one's input, the halo array reused
by every call) queued without any host synchronisation must therefore give, bit for bit, what
the same chain gives with the device synchronised between calls.  A torch kernel between two
actions (a scaling of the vector the next action reads) must be seen by that action as well.
"""
from __future__ import annotations

import pytest

from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _chain(op, x0, precision, steps, sync, stream, scale_between):
    import torch
    bufs = [x0.clone(), torch.empty_like(x0)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            src, dst = bufs[i % 2], bufs[(i + 1) % 2]
            op.jacobian_action(src, precision=precision, out=dst)
            if scale_between:
                dst.mul_(0.125)         # a torch kernel between two actions, on the same stream
            if sync:
                torch.cuda.synchronize()
    torch.cuda.synchronize()
    return bufs[steps % 2]


@pytest.mark.parametrize("precision", [32, -32])
@pytest.mark.parametrize("scale_between", [False, True])
@pytest.mark.parametrize("side_stream", [False, True])
def test_chained_actions_without_sync_match_synchronised(precision, scale_between, side_stream):
    import torch
    from paper_2506_00746_gb300 import Operator
    n, k = 40, 3                                   # 8,000 tiles: several waves of CTAs
    op = Operator(3, n, k, I.lattice_vertices(3, n, seed=0), p=3.0)
    op.linearize(torch.from_numpy(I.smooth_field(3, n, k, seed=1)).cuda())
    x0 = torch.from_numpy(I.uniform_vector(op.n_dofs, seed=2)).cuda()
    if precision == 32:
        x0 = x0.float()
    stream = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    ref = _chain(op, x0, precision, 6, True, stream, scale_between)
    for _ in range(3):
        got = _chain(op, x0, precision, 6, False, stream, scale_between)
        assert torch.equal(got, ref)
    assert torch.isfinite(ref).all() and ref.abs().max() > 0
    op.close()
