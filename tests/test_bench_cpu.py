"""The bench's reference arm (the FP64 oracle on the host cores) keeps the
JSON line contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "tiny", "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "beam segments/s" and d["unit"] == "segments/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("tiny")


def _split_rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    from oracle import oracle as O
    from paper_1912_03998_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.tiny_city(seed=3, level=3, max_order=3, n_sources=5)

        def trace_block(lo, hi):  # the oracle stands in for a GPU's partial trace
            r = O.trace_workload(w.subset_sources(np.arange(lo, hi)))
            return torch.from_numpy(np.ascontiguousarray(r["I"])), torch.from_numpy(np.ascontiguousarray(r["cnt"]))

        I, cnt = bench.source_shard_result(trace_block, len(w.src), rank, world, shard.allreduce_result)
        np.save(os.path.join(out_dir, f"I{rank}.npy"), I.numpy())
        np.save(os.path.join(out_dir, f"c{rank}.npy"), cnt.numpy())
    finally:
        dist.destroy_process_group()


def test_bench_source_split_step_two_gloo_ranks(tmp_path, oracle_mod):
    """The bench's multi-GPU step (sources split over the ranks, one sum
    all-reduce), run by two gloo ranks on CPU with the oracle standing in for
    each rank's trace: every rank ends with the single-rank result."""
    import multiprocessing as mp
    import socket

    import numpy as np

    from paper_1912_03998_gb300 import synth
    from tests.parity import level_db
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    ps = [ctx.Process(target=_split_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(300)
        assert p.exitcode == 0
    w = synth.tiny_city(seed=3, level=3, max_order=3, n_sources=5)
    ref = oracle_mod.trace_workload(w)
    for r in range(2):
        I = np.load(tmp_path / f"I{r}.npy")
        cnt = np.load(tmp_path / f"c{r}.npy")
        assert (cnt == ref["cnt"]).all()
        assert np.allclose(I, ref["I"], rtol=1e-12, atol=0)
        L = level_db(I)
        both = np.isneginf(L) & np.isneginf(level_db(ref["I"]))
        assert np.where(both, 0.0, np.abs(L - level_db(ref["I"]))).max() < 1e-9
