"""Batched instances in one persistent launch: the batched FP32 Jacobian action against the oracle
for both compiled tile edges of every order, bitwise against the single-instance operator where
both run the same tile variant, lock-step Newton checked by the oracle's residual per instance,
graph replay against plain launches, and the autotuner's cache."""
from __future__ import annotations

import json

import numpy as np
import pytest

import oracle as O
from paper_2506_00746_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (order, n, p): every order 1..4, ragged tiles for both tile edges, p in [2.5, 4]
SPEC = [(1, 5, 2.6), (2, 4, 3.3), (3, 3, 3.9), (4, 3, 2.9), (1, 7, 3.1), (2, 5, 3.7), (3, 5, 2.5), (4, 2, 3.5)]


def _instances():
    return [{"vertices": I.lattice_vertices(3, n, seed=100 + i), "n": n, "order": k, "p": p}
            for i, (k, n, p) in enumerate(SPEC)]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _states(inst):
    return [I.smooth_field(3, d["n"], d["order"], seed=200 + i) for i, d in enumerate(inst)]


# tile edges the batched launch is compiled for, per order 1..4: the larger and the smaller
BATCH_TILES = {1: (4, 2), 2: (2, 1), 3: (2, 1), 4: (2, 1)}


@pytest.mark.parametrize("policy", [1, 3])
@pytest.mark.parametrize("tiles", [[4, 2, 2, 2], [2, 1, 1, 1]])
def test_batch_jv_matches_oracle(tiles, policy):
    import torch
    from paper_2506_00746_gb300 import Batch
    inst = _instances()
    B = Batch(inst, tune=False, tiles=tiles, policy=policy)
    assert B.shape()["policy"] == policy
    assert B.tiles == [tiles[d["order"] - 1] for d in inst]
    us = _states(inst)
    B.linearize(B.concat(us))
    v32 = B.concat([I.uniform_vector(n, seed=300 + i) for i, n in enumerate(B.n_dofs)], torch.float32)
    y = B.jacobian_action(v32)
    y2 = B.jacobian_action(v32)
    assert torch.equal(y, y2)                       # deterministic
    for i, d in enumerate(inst):
        P = O.Problem(3, d["n"], d["order"], d["vertices"], p=d["p"])
        vi = B.split(v32)[i].double().cpu().numpy()
        assert _rel(B.split(y)[i].double().cpu().numpy(), O.jv(P, us[i], vi)) <= 1e-5
    B.close()


def test_batch_jv_bitwise_equals_single_instance():
    """Where the batched launch and an instance's own operator run the same tile variant (orders 1,
    3 and 4 at their largest tile edge), the results agree bit for bit; order 2 (tile edge 2 in the
    batch, 3 alone) agrees to FP32 rounding."""
    import torch
    from paper_2506_00746_gb300 import Batch, Operator
    inst = _instances()
    B = Batch(inst, tune=False, tiles=[4, 2, 2, 2])
    us = _states(inst)
    B.linearize(B.concat(us))
    vs = [I.uniform_vector(n, seed=300 + i) for i, n in enumerate(B.n_dofs)]
    y = B.jacobian_action(B.concat(vs, torch.float32))
    for i, d in enumerate(inst):
        op = Operator(3, d["n"], d["order"], d["vertices"], p=d["p"])
        op.linearize(torch.from_numpy(us[i]).cuda())
        yi = op.jacobian_action(torch.from_numpy(vs[i]).float().cuda(), precision=32)
        if d["order"] != 2:
            assert torch.equal(B.split(y)[i], yi)
        else:
            assert (torch.linalg.norm(B.split(y)[i].double() - yi.double()) <= 1e-6 * torch.linalg.norm(yi.double()))
        op.close()
    B.close()


def test_batch_policies_bitwise_equal():
    """The persistent launch (policies 0-2) and one launch per variant (policy 3) run the same tile
    code on the same tiles: identical results bit for bit, and the per-variant launches are
    counted."""
    import torch
    from paper_2506_00746_gb300 import Batch
    inst = _instances()
    us = _states(inst)
    ys = []
    for policy in (0, 2, 3):
        B = Batch(inst, tune=False, tiles=[4, 2, 2, 2], policy=policy)
        B.linearize(B.concat(us))
        v32 = B.concat([I.uniform_vector(n, seed=300 + i) for i, n in enumerate(B.n_dofs)], torch.float32)
        l0 = B.shape()["launches"]
        ys.append(B.jacobian_action(v32))
        nvar = len({(d["order"], t) for d, t in zip(inst, B.tiles)})
        assert B.shape()["launches"] - l0 == (nvar + 1 if policy == 3 else 2)
        B.close()
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])


@pytest.mark.parametrize("policy", [0, 3])
def test_batch_jv_captured_in_a_graph(policy):
    """The batched action captured in a CUDA graph (its launches on torch's capture stream) and
    replayed: bit for bit the direct call's result, on two different directions."""
    import torch
    from paper_2506_00746_gb300 import Batch
    inst = _instances()
    B = Batch(inst, tune=False, tiles=[4, 2, 2, 2], policy=policy)
    B.linearize(B.concat(_states(inst)))
    v = B.concat([I.uniform_vector(n, seed=300 + i) for i, n in enumerate(B.n_dofs)], torch.float32)
    y = torch.zeros_like(v)                            # the gaps between instances stay zero
    B.jacobian_action(v, out=y)                        # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.jacobian_action(v, out=y)
    for seed in (400, 500):
        w = B.concat([I.uniform_vector(n, seed=seed + i) for i, n in enumerate(B.n_dofs)], torch.float32)
        v.copy_(w)
        g.replay()
        torch.cuda.synchronize()
        ref = B.jacobian_action(w)
        for a, b in zip(B.split(y), B.split(ref)):
            assert torch.equal(a, b)
    B.close()


def test_batch_newton_matches_oracle():
    import torch
    from paper_2506_00746_gb300 import Batch
    inst = _instances()
    B = Batch(inst, tune=False)
    us = _states(inst)
    u = B.concat(us)
    reps, tot = B.newton_solve(u, rtol=1e-8)
    assert tot["status"] == "FE_OK"
    for i, d in enumerate(inst):
        assert reps[i]["status"] == "FE_OK" and reps[i]["rel"] <= 1e-8
        P = O.Problem(3, d["n"], d["order"], d["vertices"], p=d["p"])
        r0 = np.linalg.norm(O.residual(P, us[i]))
        ui = B.split(u)[i].cpu().numpy()
        assert np.linalg.norm(O.residual(P, ui)) <= 1e-8 * r0 * 1.01
    # graph replay and plain launches give bitwise the same iterates
    a, b, c = B.concat(us), B.concat(us), B.concat(us)
    ra, _ = B.newton_solve(a, use_graph=1)
    rb, _ = B.newton_solve(b, use_graph=0, cg_batch=3)
    rc, _ = B.newton_solve(c, use_graph=2, cg_batch=5)      # the whole CG as one graph launch
    assert torch.equal(a, b) and torch.equal(a, c)
    assert [r["cg_iters"] for r in ra] == [r["cg_iters"] for r in rb] == [r["cg_iters"] for r in rc]
    B.close()
    # one launch per variant: the same iterates
    B3 = Batch(inst, tune=False, policy=3)
    d = B3.concat(us)
    rd, _ = B3.newton_solve(d, use_graph=2)
    assert torch.equal(a, d) and [r["cg_iters"] for r in rd] == [r["cg_iters"] for r in ra]
    B3.close()


def test_batch_autotune_cache(tmp_path):
    from paper_2506_00746_gb300 import Batch
    inst = _instances()
    cache = tmp_path / "tune.json"
    B = Batch(inst, tune=True, tune_cache=str(cache))
    tiles, shape = B.tiles, B.shape()
    B.close()
    data = json.loads(cache.read_text())
    assert sum(k.endswith("|tile") for k in data) == 4          # one entry per order
    assert any(k.endswith("|grid") for k in data) and any(k.endswith("|policy") for k in data)
    for k, v in data.items():
        if k.endswith("|tile"):
            order = int(k.split("|order")[1].split("|")[0])
            assert v in BATCH_TILES[order]
    B2 = Batch(inst, tune=True, tune_cache=str(cache))           # read back, nothing re-timed
    assert B2.tiles == tiles
    s2 = B2.shape()
    assert s2["grid"] == shape["grid"] and s2["policy"] == shape["policy"]
    B2.close()


def test_batch_rejects_unsupported():
    from paper_2506_00746_gb300 import Batch, FeodError
    inst = _instances()[:2]
    inst[0] = dict(inst[0], order=5, vertices=I.lattice_vertices(3, 2, seed=1), n=2)
    with pytest.raises(FeodError):
        Batch(inst, tune=False)
