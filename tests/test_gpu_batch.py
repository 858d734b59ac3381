"""Batched ensembles (lbm_batch_*): one persistent launch per step over the tiles of
many contexts, replayed from a CUDA graph, must give exactly what stepping every
context alone gives, in 64-node tiles and in 32-node half tiles; tuning must leave
the state untouched."""

import numpy as np
import pytest

from oracle import lattices as OL
from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import check_close, deviation, gpu_sim, oracle_sim, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _members(count, seed, n_max=160):
    ps = [p for p in W.couette_ensemble(64, seed) if p["n"] <= n_max][:count]
    assert len(ps) == count
    return [W.ensemble_member(p) for p in ps]


def _make(ws, prec, stream=None):
    sims = []
    for k, w in enumerate(ws):
        s = gpu_sim(w, prec, scheme=(0, 1, 0, 1.0))
        rho, u = W.random_state(w["shape"], "D2Q9", 1.0, 0.005, seed=100 + k)
        s.init_equilibrium(rho, u)
        if stream is not None:
            s.set_stream(stream)
        sims.append(s)
    return sims


@pytest.mark.parametrize("prec", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("steps", [1, 2, 7])
@pytest.mark.parametrize("tile_w", [64, 32])
def test_batch_equals_individual_steps(prec, steps, tile_w):
    torch = require_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    ws = _members(6, seed=3)
    solo = _make(ws, prec, stream)
    grouped = _make(ws, prec, stream)
    batch = B.Batch(grouped)
    batch.set_stream(stream)
    batch.set_config(1, 0, 1, tile_w)
    assert batch.query()["tile_w"] == tile_w
    for s in solo:
        s.step(steps)
    batch.step(steps)
    for a, b, w in zip(solo, grouped, ws):
        fl = ~w["solid"]
        fa, fb = a.get_populations(), b.get_populations()
        assert np.array_equal(fa[:, fl], fb[:, fl])
        assert a.time() == b.time() == steps
    batch.close()


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("tile_w", [64, 32])
def test_batch_orders_and_graph_replay(order, split, tile_w):
    """Every tile order and tile width, with the members split into kernel classes
    (one launch per class: members whose rows start on 16-byte boundaries take the
    aligned-window sweep) or all through the general sweep; the graph is replayed."""
    torch = require_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    ws = _members(5, seed=4)
    aligned = [w["shape"][0] % 4 == 0 for w in ws]
    assert any(aligned) and not all(aligned)       # both classes present
    solo = _make(ws, "f32", stream)
    grouped = _make(ws, "f32", stream)
    batch = B.Batch(grouped)
    batch.set_stream(stream)
    batch.set_config(order, 3, split, tile_w)
    q = batch.query()
    assert q["launches_per_step"] == (2 if split else 1) and q["tile_w"] == tile_w
    for rep in range(3):            # the graph is captured once and replayed
        batch.step(10)
        for s in solo:
            s.step(10)
    for a, b, w in zip(solo, grouped, ws):
        fl = ~w["solid"]
        assert np.array_equal(a.get_populations()[:, fl], b.get_populations()[:, fl])
    batch.close()


def test_tune_leaves_state_unchanged():
    torch = require_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    ws = _members(4, seed=5)
    sims = _make(ws, "f32", stream)
    for s in sims:
        s.step(3)
    before = [s.get_populations() for s in sims]
    batch = B.Batch(sims)
    batch.set_stream(stream)
    order, blocks, split, tile_w = batch.tune(6)
    assert order in (0, 1, 2) and blocks in (0, 3, 4) and split in (0, 1) and tile_w in (32, 64)
    q = batch.query()
    assert q["order"] == order and q["blocks_per_sm"] == blocks and q["contexts"] == 4
    assert q["tile_w"] == tile_w
    for s, f0, w in zip(sims, before, ws):
        fl = ~w["solid"]
        assert s.time() == 3
        assert np.array_equal(s.get_populations()[:, fl], f0[:, fl])
    batch.close()


def test_batch_requires_same_parity_and_picks_up_changes():
    torch = require_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    ws = _members(3, seed=6)
    sims = _make(ws, "f64", stream)
    solo = _make(ws, "f64", stream)
    batch = B.Batch(sims)
    batch.set_stream(stream)
    sims[1].step(1)
    with pytest.raises(B.LbmError) as ei:
        batch.step(2)
    assert ei.value.code == -7
    sims[0].step(1)
    sims[2].step(1)
    for s in solo:
        s.step(1)
    # change a member's force between batch steps: the batch must see it
    sims[2].set_force((1e-6, -2e-6, 0.0))
    solo[2].set_force((1e-6, -2e-6, 0.0))
    batch.step(4)
    for s in solo:
        s.step(4)
    for a, b, w in zip(solo, sims, ws):
        fl = ~w["solid"]
        assert np.array_equal(a.get_populations()[:, fl], b.get_populations()[:, fl])
    batch.close()


@pytest.mark.parametrize("tile_w", [64, 32])
def test_batch_member_matches_oracle_and_d3q19_mix(tile_w):
    """A D3Q19 batch mixing the skew-periodic tilted pipe and a sphere box (different
    sizes, alignment and wrap) against the FP64 oracle."""
    require_gpu()
    w1 = W.tilted_pipe_3d(16)
    w2 = W.sphere_3d(13, 3.3, (6.2, 4.9, 4.4), s_nu=1.1, force=(1e-5, 2e-6, -3e-6))
    sims = []
    for w in (w1, w2):
        s = gpu_sim(w, "f64")
        rho, u = W.random_state(w["shape"], "D3Q19", 1.0, 0.005, seed=9)
        s.init_equilibrium(rho, u)
        sims.append((s, w, rho, u))
    batch = B.Batch([s for s, *_ in sims])
    batch.set_config(1, 0, 1, tile_w)
    batch.step(9)
    for s, w, rho, u in sims:
        o = oracle_sim(w)
        o.init_equilibrium(rho, u)
        o.step(9)
        fl = ~w["solid"]
        check_close(deviation(s.get_populations(), OL.D3Q19), deviation(o.f, OL.D3Q19), 1e-12, fl)
    batch.close()


@pytest.mark.parametrize("tile_w", [None, 32, 64])
def test_full_ensemble_batch_equals_one_launch_per_member(tile_w):
    """The benchmark's ensemble itself (96 Couette instances from seed 0, n in 48..768,
    FP32): after tuning (or in a fixed tile width) and an odd number of
    graph-replayed steps, every member of the batch holds exactly what stepping it
    alone gives."""
    torch = require_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    ws = [W.ensemble_member(p) for p in W.couette_ensemble(96, 0)]
    solo, grouped = [], []
    for w in ws:
        for lst in (solo, grouped):
            s = gpu_sim(w, "f32")
            s.init_equilibrium()
            s.set_stream(stream)
            lst.append(s)
    batch = B.Batch(grouped)
    batch.set_stream(stream)
    if tile_w is None:
        batch.tune(4)
    else:
        batch.set_config(1, 0, 1, tile_w)
    batch.step(7)
    for s in solo:
        s.step(7)
    for a, b, w in zip(solo, grouped, ws):
        fl = ~w["solid"]
        assert np.array_equal(a.get_populations()[:, fl], b.get_populations()[:, fl])
    batch.close()
