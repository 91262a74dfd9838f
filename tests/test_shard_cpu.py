"""Source sharding across ranks (the multi-GPU path), on CPU: two gloo ranks
each trace a block of the sources with the oracle, sum their partial
intensities and path counts with the package's all-reduce, and must obtain
the oracle's result for all sources (Section 3: processes trace their own
beams and their results are gathered)."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_1912_03998_gb300 import shard, synth


def test_source_blocks_partition_the_sources():
    for n in (0, 1, 5, 16, 1000, 1001):
        for world in (1, 2, 3, 4, 7):
            blocks = [shard.source_block(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a, b), (c, d) in zip(blocks, blocks[1:]):
                assert b == c
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.source_block(5, 2, 2)


def _workload(directional=False):
    w = synth.tiny_city(seed=3, level=3, max_order=3, n_sources=5)
    if directional:
        # two patterns and an omnidirectional source: the shards must carry
        # each source's pattern with it
        w.directivity = synth.Directivity([synth.cardioid((1.0, 0.0, 0.0), 0.8),
                                           synth.cardioid((0.0, 1.0, 0.5), 0.5)],
                                          np.array([0, 1, -1, 0, 1], np.int32))
    return w


def _rank_main(rank, world, port, out_dir, directional=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload(directional)
        lo, hi = shard.source_block(len(w.src), rank, world)
        r = O.trace_workload(w.subset_sources(np.arange(lo, hi)))
        I = torch.from_numpy(np.ascontiguousarray(r["I"], np.float64))
        cnt = torch.from_numpy(np.ascontiguousarray(r["cnt"], np.int32))
        shard.allreduce_result(I, cnt, check_timeout_s=60.0)  # every rank arrives: the check passes
        np.save(os.path.join(out_dir, f"I{rank}.npy"), I.numpy())
        np.save(os.path.join(out_dir, f"c{rank}.npy"), cnt.numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world,directional", [(2, False), (3, False), (2, True)])
def test_gloo_ranks_sum_to_the_full_result(oracle_mod, tmp_path, world, directional):
    pytest.importorskip("torch")
    w = _workload(directional)
    full = oracle_mod.trace_workload(w)
    if directional:
        # the patterns matter: the omnidirectional result differs
        omni = oracle_mod.trace(oracle_mod.Scene(w.scene), w.src, w.power, w.level, w.mics, w.max_order)
        assert not np.allclose(omni["I"], full["I"])
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path), directional))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            p.join()
        assert p.exitcode == 0
    for r in range(world):
        I = np.load(tmp_path / f"I{r}.npy")
        c = np.load(tmp_path / f"c{r}.npy")
        assert (c == full["cnt"]).all()
        assert np.allclose(I, full["I"], rtol=1e-12, atol=0)


def test_microphone_blocks_partition_the_microphones():
    for n in (0, 7, 1024):
        for world in (1, 2, 3):
            blocks = [shard.mic_block(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(b == c for (a, b), (c, d) in zip(blocks, blocks[1:]))


def _mic_rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload(True)
        lo, hi = shard.mic_block(len(w.mics), rank, world)
        r = O.trace_workload(w.with_mics(w.mics[lo:hi]))
        I = shard.gather_blocks(torch.from_numpy(np.ascontiguousarray(r["I"], np.float64)), len(w.mics))
        cnt = shard.gather_blocks(torch.from_numpy(np.ascontiguousarray(r["cnt"], np.int32)), len(w.mics))
        np.save(os.path.join(out_dir, f"mI{rank}.npy"), I.numpy())
        np.save(os.path.join(out_dir, f"mc{rank}.npy"), cnt.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_microphone_blocks_gather_to_the_full_result(oracle_mod, tmp_path, world):
    # Section 3's microphone partitioning: every rank traces all sources
    # against its own block of microphones; the gathered blocks equal the
    # one-process result exactly (a microphone's result depends on no other)
    pytest.importorskip("torch")
    w = _workload(True)
    full = oracle_mod.trace_workload(w)
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_mic_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            p.join()
        assert p.exitcode == 0
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"mc{r}.npy"), full["cnt"])
        assert np.array_equal(np.load(tmp_path / f"mI{r}.npy"), full["I"])



def _failing_rank_main(rank, world, port, out_dir, bad_rank):
    # every rank traces its block; `bad_rank` fails before the exchange step
    # and leaves; the others must learn of it from the rank check, not hang
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime

    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    w = _workload()
    lo, hi = shard.source_block(len(w.src), rank, world)
    r = O.trace_workload(w.subset_sources(np.arange(lo, hi)))
    if rank == bad_rank:
        os._exit(7)  # a failed partial trace: the process leaves without the exchange
    I = torch.from_numpy(np.ascontiguousarray(r["I"], np.float64))
    cnt = torch.from_numpy(np.ascontiguousarray(r["cnt"], np.int32))
    try:
        shard.allreduce_result(I, cnt, check_timeout_s=5.0)
        outcome = "completed"
    except shard.ShardFailure as e:
        outcome = "detected: " + str(e).replace("\n", " ")[:300]
    with open(os.path.join(out_dir, f"outcome{rank}.txt"), "w") as f:
        f.write(outcome)
    os._exit(0)


def test_failed_rank_is_detected_before_the_exchange(tmp_path):
    pytest.importorskip("torch")
    world, bad = 3, 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, world, port, str(tmp_path), bad))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            p.join()
    assert procs[bad].exitcode == 7
    for r in range(world):
        if r == bad:
            continue
        assert procs[r].exitcode == 0
        outcome = (tmp_path / f"outcome{r}.txt").read_text()
        assert outcome.startswith("detected"), outcome
    # rank 0 runs the check and names the rank that left
    assert "2" in (tmp_path / "outcome0.txt").read_text()
