"""Data-parallel exchange over views, on two gloo ranks (CPU).

Each rank computes the oracle's gradient and Hutchinson diagonal on its own
view; after the exchange both ranks must hold what one process computes over
both views together (Sec. 4.1 normalisation by the total residual count m).
"""
import math
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _scene():
    from paper_2602_00395_gb300 import synth as S
    sc = S.make_scene(60, 1, seed=31, extent=0.6, log_scale_shift=math.log(3.0))
    cams = S.camera_ring(2, 32, 24, 0.6, seed=3, ring_factor=5.0)
    target = S.noise_target(2, 24, 32, seed=8)
    return sc, cams, target


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2602_00395_gb300.exchange import GradExchange
    sc, cams, target = _scene()
    P = O.params64(sc)
    r = O.backward(P, sc.sh_degree, [cams[rank]], target[rank:rank + 1].astype(np.float64), seed=5, t=1, nu=1)
    g = torch.from_numpy(r["grad"].copy())
    h = torch.from_numpy(r["hz"].copy())
    m_local = 3 * cams[rank].width * cams[rank].height
    m = GradExchange()(m_local, g, h)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), g.numpy())
    np.save(os.path.join(out_dir, f"h{rank}.npy"), h.numpy())
    np.save(os.path.join(out_dir, f"m{rank}.npy"), np.array([m]))
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_matches_single_process_over_all_views(tmp_path):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    import oracle as O
    sc, cams, target = _scene()
    ref = O.backward(O.params64(sc), sc.sh_degree, cams, target.astype(np.float64), seed=5, t=1, nu=1)
    for rank in range(2):
        g = np.load(tmp_path / f"g{rank}.npy")
        h = np.load(tmp_path / f"h{rank}.npy")
        assert float(np.load(tmp_path / f"m{rank}.npy")[0]) == 2 * 3 * 32 * 24
        np.testing.assert_allclose(g, ref["grad"], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h, ref["hz"], rtol=1e-12, atol=1e-15)


def test_exchange_is_identity_on_one_rank():
    from paper_2602_00395_gb300.exchange import GradExchange
    g = torch.randn(14, 32, dtype=torch.float64)
    g0 = g.clone()
    assert GradExchange()(123.0, g) == 123.0
    assert torch.equal(g, g0)


def _step_worker(rank, world, port, out_dir):
    """The engine's step on a rank, its kernels replaced by host stand-ins: the
    reverse pass leaves a rank-specific gradient and Hutchinson diagonal, and the
    update records what it sees."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2602_00395_gb300.engine import TRConfig, TRStep
    from paper_2602_00395_gb300.exchange import GradExchange
    e = object.__new__(TRStep)  # no device buffers: host tensors stand in for them
    e.nu, e.cfg, e.W, e.H, e.V = 1, TRConfig(l=1), 8 + 8 * rank, 4, 1 + rank
    e.grad = torch.zeros(3, 5, dtype=torch.float64)
    e.hz = torch.zeros(3, 5, dtype=torch.float64)
    e.loss_val = torch.zeros(1, dtype=torch.float64)
    calls = []
    e.project = lambda t, probes=True, stream=None: calls.append("project")
    e.bin_sort = lambda stream=None: calls.append("bin_sort")
    e.raster_fwd = lambda t, probes=True, stream=None: calls.append("raster_fwd")

    def bwd(t, probes=True, stream=None):
        calls.append("raster_bwd")
        e.grad.fill_(1.0 + rank)
        e.hz.fill_(10.0 * (1 + rank))
    e.raster_bwd = bwd
    seen = {}

    def update(t, eps, with_hz=True, eta_out=None, stream=None):
        calls.append("update")
        seen["g"], seen["h"] = e.grad.clone(), e.hz.clone()
    e.update = update
    e.step(1, 1e-6, exchange=GradExchange())
    np.save(os.path.join(out_dir, f"calls{rank}.npy"), np.array(calls))
    np.save(os.path.join(out_dir, f"sg{rank}.npy"), seen["g"].numpy())
    np.save(os.path.join(out_dir, f"sh{rank}.npy"), seen["h"].numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_engine_step_exchanges_between_reverse_pass_and_update(tmp_path):
    """TRStep.step with an exchange on two gloo ranks: the all-reduce comes after
    the reverse pass and before the update, and the update on every rank sees the
    sum of the ranks' buffers weighted by their residual counts m_r / m."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_step_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    m = [3 * 8 * 4 * 1, 3 * 16 * 4 * 2]  # 3 W H V of each rank
    w = [m[0] / sum(m), m[1] / sum(m)]
    for rank in range(2):
        assert list(np.load(tmp_path / f"calls{rank}.npy")) == ["project", "bin_sort", "raster_fwd", "raster_bwd",
                                                                "update"]
        np.testing.assert_allclose(np.load(tmp_path / f"sg{rank}.npy"), w[0] * 1.0 + w[1] * 2.0, rtol=1e-12)
        np.testing.assert_allclose(np.load(tmp_path / f"sh{rank}.npy"), w[0] * 10.0 + w[1] * 20.0, rtol=1e-12)
