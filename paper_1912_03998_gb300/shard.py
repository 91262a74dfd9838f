"""Sharding one problem over several ranks (GPUs or contexts).

Sources: beams of different sources never interact (Section 2: every beam
carries its own source's energy; Section 3: processes trace their own beams
and their results are gathered), so the result for all sources is the sum of
the results for disjoint subsets of them.  Each rank traces one contiguous
block of the sources, the partial intensities and path counts are summed
over the ranks by one all-reduce, and every rank installs the sum with
bt_set_result and reads the levels through its own level kernel.

Microphones (Section 3, microphone partitioning: every process traces all
beams and measures them at its own microphones): a microphone's result does
not depend on the other microphones, so each rank traces every source
against one contiguous block of the microphones and the blocks' levels are
gathered in rank order.  This splits the scatter, which dominates when the
microphones fill a volume, at the price of tracing every beam on every rank.

Failure detection: before the exchange step, check_ranks (a monitored
barrier with a timeout on a gloo group) turns a rank that failed and left, or
hangs, into ShardFailure on the others instead of a collective that never
completes.
"""
from __future__ import annotations

import numpy as np

from . import btrace


def source_block(n_sources: int, rank: int, world: int) -> tuple[int, int]:
    """The block [lo, hi) of sources owned by `rank`: contiguous, sizes
    differing by at most one, blocks in rank order covering 0..n_sources."""
    if world < 1 or not 0 <= rank < world or n_sources < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n_sources, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


class ShardFailure(RuntimeError):
    """A rank did not reach the exchange step in time: it raised, exited or
    is stuck.  The message names the rank(s) where the backend can tell."""


def check_ranks(group=None, timeout_s: float = 30.0):
    """Failure detection before the exchange step: every rank of `group` (a
    gloo group; beside an NCCL group, one made with
    dist.new_group(backend="gloo")) must arrive within `timeout_s`.  A rank
    that failed its partial trace and left, or hangs, is then reported on the
    others as ShardFailure instead of a collective that never completes."""
    import datetime

    import torch.distributed as dist
    try:
        dist.monitored_barrier(group=group, timeout=datetime.timedelta(seconds=float(timeout_s)),
                               wait_all_ranks=True)
    except RuntimeError as e:
        raise ShardFailure(str(e)) from e


def allreduce_result(intensity, path_count, group=None, check_timeout_s=None, check_group=None):
    """Sum a float64 intensity tensor and an int32 path-count tensor over the
    ranks of `group`, in place (CPU tensors under gloo, CUDA tensors under
    NCCL).  With `check_timeout_s`, check_ranks runs first (on `check_group`,
    default `group`)."""
    import torch.distributed as dist
    if check_timeout_s is not None:
        check_ranks(check_group if check_group is not None else group, check_timeout_s)
    dist.all_reduce(intensity, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(path_count, op=dist.ReduceOp.SUM, group=group)
    return intensity, path_count


def trace_sharded(tracer, w, rank: int, world: int, group=None, **params):
    """Trace workload `w` with its sources split over `world` ranks; every
    rank gets the levels for all sources.  Returns dict(level, I, cnt) as
    numpy arrays and the scene id holding the summed result."""
    import torch
    import torch.distributed as dist
    lo, hi = source_block(len(w.src), rank, world)
    part = w.subset_sources(np.arange(lo, hi))
    g = tracer.run(part, **params)
    on_gpu = dist.get_backend(group) == "nccl"
    dev = torch.device("cuda", torch.cuda.current_device()) if on_gpu else torch.device("cpu")
    I = torch.from_numpy(g["I"]).to(dev)
    cnt = torch.from_numpy(g["cnt"]).to(dev)
    allreduce_result(I, cnt, group)
    sid = g["scene_id"]
    btrace.bt_set_result(tracer.ctx, sid, I, cnt)
    n, nb = I.shape
    level = np.empty((n, nb), np.float64)
    I_out = np.empty((n, nb), np.float64)
    cnt_out = np.empty(n, np.int32)
    btrace.bt_read_levels(tracer.ctx, sid, level, I_out, cnt_out)
    return dict(level=level, I=I_out, cnt=cnt_out, scene_id=sid)


def mic_block(n_mics: int, rank: int, world: int) -> tuple[int, int]:
    """The block [lo, hi) of microphones owned by `rank` (as source_block)."""
    return source_block(n_mics, rank, world)


def gather_blocks(part, n_total: int, group=None):
    """Concatenate per-rank blocks [lo, hi) of a result (rows of `part`, a
    CPU or CUDA tensor, shaped [hi - lo, ...]) into the full [n_total, ...]
    tensor on every rank, in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    full = torch.zeros((n_total,) + tuple(part.shape[1:]), dtype=part.dtype, device=part.device)
    rank = dist.get_rank(group)
    lo, hi = mic_block(n_total, rank, world)
    full[lo:hi] = part
    dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)
    return full


def trace_mic_sharded(tracer, w, rank: int, world: int, group=None, **params):
    """Trace workload `w` with its microphones split over `world` ranks (every
    rank traces all sources); every rank gets the levels, intensities and path
    counts of all microphones.  Returns dict(level, I, cnt) as numpy arrays."""
    import torch
    import torch.distributed as dist
    lo, hi = mic_block(len(w.mics), rank, world)
    g = tracer.run(w.with_mics(w.mics[lo:hi]), **params)
    btrace.bt_unload_scene(tracer.ctx, g["scene_id"])
    on_gpu = dist.get_backend(group) == "nccl"
    dev = torch.device("cuda", torch.cuda.current_device()) if on_gpu else torch.device("cpu")
    out = {}
    for k in ("level", "I", "cnt"):
        out[k] = gather_blocks(torch.from_numpy(np.ascontiguousarray(g[k])).to(dev), len(w.mics), group).cpu().numpy()
    return out

