"""Multi-rank path on CPU (gloo, world size 2): waveforms shard across ranks with no
data-path exchange; together the ranks reproduce the single-process DBP (FP64 oracle)
exactly, the timing reduction takes the slowest rank, and the one exchange training
needs -- the sum over ranks of the parameter gradients -- reproduces the single-process
gradient of the whole batch."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_1507_00921_gb300 import dist as pdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist

    from oracle import dbp as odbp
    from oracle import fiber
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = synth.random_field(5, 3000, synth.dbm_to_w(2.0), seed=31)
    cfg = fiber.make_config(synth.link(10), synth.SAMPLE_RATE, 1, 4, 1024)
    start, count = pdist.shard(x.shape[0], world, rank)
    out = odbp.dbp(x[start:start + count], cfg)
    np.save(os.path.join(outdir, f"rank{rank}.npy"), out)
    t_max = pdist.max_over_ranks([1.0 + rank, 5.0 - rank])
    units = pdist.sum_over_ranks([count])
    np.save(os.path.join(outdir, f"red{rank}.npy"), np.array(t_max + units))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_partition():
    for n in [0, 1, 5, 128, 129]:
        for world in [1, 2, 3, 8]:
            parts = [pdist.shard(n, world, r) for r in range(world)]
            assert sum(c for _, c in parts) == n
            assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    assert pdist.throughput(10, 4, 5, 2.0) == 100.0
    with pytest.raises(ValueError):
        pdist.shard(4, 2, 2)


def test_two_gloo_ranks_reproduce_single_process(tmp_path):
    from oracle import dbp as odbp
    from oracle import fiber
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)])
    x = synth.random_field(5, 3000, synth.dbm_to_w(2.0), seed=31)
    ref = odbp.dbp(x, fiber.make_config(synth.link(10), synth.SAMPLE_RATE, 1, 4, 1024))
    assert np.array_equal(got, ref)
    for r in range(world):
        red = np.load(tmp_path / f"red{r}.npy")
        assert list(red) == [2.0, 5.0, 5.0]


def _grad_rank_main(rank, world, port, outdir):
    import torch.distributed as dist

    from oracle import adjoint
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, v, cfg = _grad_case()
    start, count = pdist.shard(x.shape[0], world, rank)
    gc = np.zeros_like(cfg.coeffs)
    gg = np.zeros(cfg.n_steps)
    gd = np.zeros(cfg.n_steps)
    for w in range(start, start + count):
        _, c_, g_, d_ = adjoint.dbp_vjp(x[w], cfg, v[w])
        gc += c_
        gg += g_
        gd += d_
    total = pdist.sum_over_ranks(list(gc.ravel()) + list(gg) + list(gd))
    np.save(os.path.join(outdir, f"grad{rank}.npy"), np.array(total))
    dist.barrier()
    dist.destroy_process_group()


def _grad_case():
    from oracle import fiber
    rng = np.random.default_rng(41)
    x = synth.random_field(5, 700, synth.dbm_to_w(3.0), seed=43)
    v = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
    c = np.array([[0.6, 0.2, 0.1], [0.5, 0.25, -0.1]])
    cfg = fiber.make_config(synth.link(2), synth.SAMPLE_RATE, 2, 2, 256, coeffs=c, overlap=96)
    cfg.gamma_eff = np.array([250.0, 300.0])
    return x, v, cfg


def test_two_gloo_ranks_sum_parameter_gradients(tmp_path):
    from oracle import adjoint
    world = 2
    mp.start_processes(_grad_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    x, v, cfg = _grad_case()
    gc = np.zeros_like(cfg.coeffs)
    gg = np.zeros(cfg.n_steps)
    gd = np.zeros(cfg.n_steps)
    for w in range(x.shape[0]):
        _, c_, g_, d_ = adjoint.dbp_vjp(x[w], cfg, v[w])
        gc += c_
        gg += g_
        gd += d_
    ref = np.array(list(gc.ravel()) + list(gg) + list(gd))
    for r in range(world):
        got = np.load(tmp_path / f"grad{r}.npy")
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
