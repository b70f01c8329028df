"""Multi-rank channel sharding on CPU (gloo, world size 2 and 3): every rank
correlates its own contiguous channel range, rank 0 gathers the blocks, and
the concatenation equals the single-process result bit for bit; for the
calibration, each rank's loss and gradient over its channels summed by one
all-reduce equal the single-process values (per-input gains and Jones
matrices; per-channel gains need no reduction of the gradient, only of the
loss).  The arithmetic on each rank is
the CPU oracle here; on GPUs it is the library, with the same partition
(bench.py --scaling strong)."""
import os
import socket

import numpy as np
import pytest

from paper_0902_0915_gb300.shard import all_ranges, channel_range


def test_ranges_partition_the_channels():
    for n in (0, 1, 7, 768, 3072):
        for w in (1, 2, 3, 8):
            rs = all_ranges(n, w)
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        channel_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = synth.spec_c0().with_(n_chan=11, n_time=200)
    c0, c1 = channel_range(spec.n_chan, rank, world)
    v = synth.fill_host(spec, chans=list(range(c0, c1)), threads=1)
    out = oracle.correlate(v, spec.sample_bits, spec.n_inputs, c1 - c0, spec.n_time, n_threads=1)
    blocks = [None] * world
    dist.all_gather_object(blocks, out)
    if rank == 0:
        q.put(np.concatenate(blocks, axis=0))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_equals_single(world):
    import torch.multiprocessing as mp

    import oracle
    import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec = synth.spec_c0().with_(n_chan=11, n_time=200)
    ref = oracle.correlate(synth.fill_host(spec), 4, spec.n_inputs, spec.n_chan, spec.n_time)
    np.testing.assert_array_equal(got, ref)


def _calib_worker(rank, world, port, q):
    """Each rank evaluates the calibration loss and gradient on its own
    channel range; one all-reduce (sum) of the 2N gradient components and the
    loss gives the full result (the design's only collective)."""
    import torch
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    V, M, g = _calib_problem()
    c0, c1 = channel_range(V.shape[0], rank, world)
    loss = oracle.calib_loss(V[c0:c1], M[c0:c1], g) if c1 > c0 else 0.0
    grad = oracle.calib_grad(V[c0:c1], M[c0:c1], g, n_threads=1) if c1 > c0 else np.zeros_like(g)
    t = torch.tensor(np.concatenate([[loss], grad.real, grad.imag]), dtype=torch.float64)
    dist.all_reduce(t)
    if rank == 0:
        q.put(t.numpy())
    dist.destroy_process_group()


def _calib_problem():
    rng = np.random.default_rng(9)
    N, C = 12, 7
    B = N * (N + 1) // 2
    V = rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))
    M = rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))
    g = rng.uniform(0.8, 1.2, N) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))
    return V, M, g


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_calibration_allreduce(world):
    import torch.multiprocessing as mp

    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_calib_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    V, M, g = _calib_problem()
    N = g.shape[0]
    ref_loss = oracle.calib_loss(V, M, g)
    ref_grad = oracle.calib_grad(V, M, g)
    assert got[0] == pytest.approx(ref_loss, rel=1e-12)
    np.testing.assert_allclose(got[1:1 + N] + 1j * got[1 + N:], ref_grad, rtol=1e-11, atol=1e-12)


def _variant_worker(rank, world, port, q):
    """Jones matrices: one all-reduce of the loss and the 8 n_tiles gradient
    components, as for per-input gains.  Per-channel gains: a rank's gradient
    rows are final for its channels (no reduction); only the loss is summed."""
    import torch
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    V, M, J, G = _variant_problem()
    c0, c1 = channel_range(V.shape[0], rank, world)
    lj = oracle.calib_jones_loss(V[c0:c1], M[c0:c1], J) if c1 > c0 else 0.0
    gj = oracle.calib_jones_grad(V[c0:c1], M[c0:c1], J) if c1 > c0 else np.zeros_like(J)
    t = torch.tensor(np.concatenate([[lj], gj.real.ravel(), gj.imag.ravel()]), dtype=torch.float64)
    dist.all_reduce(t)
    lc = oracle.calib_chan_loss(V[c0:c1], M[c0:c1], G[c0:c1]) if c1 > c0 else 0.0
    gc = (oracle.calib_chan_grad(V[c0:c1], M[c0:c1], G[c0:c1], n_threads=1) if c1 > c0
          else np.zeros((0, G.shape[1]), complex))
    tl = torch.tensor([lc], dtype=torch.float64)
    dist.all_reduce(tl)
    rows = [None] * world
    dist.all_gather_object(rows, gc)
    if rank == 0:
        q.put((t.numpy(), float(tl[0]), np.concatenate(rows, axis=0)))
    dist.destroy_process_group()


def _variant_problem():
    rng = np.random.default_rng(10)
    n_tiles, C = 5, 7
    N = 2 * n_tiles
    B = N * (N + 1) // 2
    V = rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))
    M = rng.standard_normal((C, B)) + 1j * rng.standard_normal((C, B))
    J = rng.standard_normal((n_tiles, 2, 2)) + 1j * rng.standard_normal((n_tiles, 2, 2))
    G = rng.uniform(0.8, 1.2, (C, N)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, N)))
    return V, M, J, G


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_calibration_variants(world):
    import torch.multiprocessing as mp

    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_variant_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    tj, lc, gc = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    V, M, J, G = _variant_problem()
    n8 = J.size
    assert tj[0] == pytest.approx(oracle.calib_jones_loss(V, M, J), rel=1e-12)
    np.testing.assert_allclose((tj[1:1 + n8] + 1j * tj[1 + n8:]).reshape(J.shape),
                               oracle.calib_jones_grad(V, M, J), rtol=1e-11, atol=1e-12)
    assert lc == pytest.approx(oracle.calib_chan_loss(V, M, G), rel=1e-12)
    np.testing.assert_allclose(gc, oracle.calib_chan_grad(V, M, G), rtol=1e-12, atol=1e-13)
