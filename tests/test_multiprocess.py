"""Shots are independent units, so decoding shards on separate processes and
merging their counts must equal one run over all shots exactly.  Two gloo
ranks on the CPU each decode a contiguous range of the same seeded shots with
the double-precision oracle; the failure, iteration and near-tie counts they
sum with all_reduce equal a single-process run, shot for shot in the
concatenated outputs.  Also: the benchmark's replicas draw their shots from
seeds of their own (weak scaling), and the max-over-ranks timing reduction."""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2
B = 600


def _problem():
    from paper_2512_07057_gb300 import workloads as W
    prob = W.bb72_code_capacity(0.05)
    return prob, W.sample_shots(prob, B, "multiprocess_shards")


def _params(oracle):
    return oracle.Params(max_rounds=10, beam_width=8, initial_iters=50, iters_per_round=20, ms_scale=0.625)


def _counts(prob, shots, res):
    from paper_2512_07057_gb300 import workloads as W
    o = W.unpack_bits(res["obs"][:, :(prob.K + 31) // 32], prob.K)
    t = W.unpack_bits(shots.obs, prob.K)
    fail = (o != t).any(1) | (res["status"] == 4)
    near = (res["min_gap"] < 1e-4) | (res["ties"] > 0)
    return np.array([fail.sum(), res["iters"].astype(np.int64).sum(), near.sum(), (res["status"] == 2).sum()],
                    np.int64)


def _rank(rank, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    import oracle
    prob, shots = _problem()
    lo, hi = B * rank // WORLD, B * (rank + 1) // WORLD
    res = oracle.Graph(prob, "f64").decode_batch(shots.syndromes[lo:hi], _params(oracle), nthreads=1)
    from paper_2512_07057_gb300 import workloads as W
    sub = W.Shots(syndromes=shots.syndromes[lo:hi], obs=shots.obs[lo:hi], errors=None)
    c = torch.from_numpy(_counts(prob, sub, res))
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    # the benchmark's timing reduction: the slowest rank sets the step time
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), counts=c.numpy(), tmax=t.numpy(), lo=lo, hi=hi,
             corrections=res["corrections"], status=res["status"], iters=res["iters"])
    dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_merge_to_the_single_run(oracle_mod):
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(_free_port(), d), nprocs=WORLD, start_method="spawn", join=True)
        parts = [np.load(os.path.join(d, f"rank{r}.npz")) for r in range(WORLD)]
        prob, shots = _problem()
        single = oracle_mod.Graph(prob, "f64").decode_batch(shots.syndromes, _params(oracle_mod), nthreads=4)
        want = _counts(prob, shots, single)
        for p in parts:
            assert np.array_equal(p["counts"], want)
            assert float(p["tmax"][0]) == float(WORLD)
        assert [int(p["lo"]) for p in parts] == [0, B // 2] and int(parts[-1]["hi"]) == B
        for k in ("corrections", "status", "iters"):
            assert np.array_equal(np.concatenate([p[k] for p in parts]), single[k])
        assert want[3] > 0                                    # beam rounds ran on both shards


def test_benchmark_replicas_draw_their_own_shots():
    """Each rank of bench.py decodes shots from a seed of its own (weak
    scaling: per-GPU work fixed), reproducibly."""
    import bench
    a0 = bench.make_workload(0, 1000, (0.03,))[0][2].syndromes
    a1 = bench.make_workload(1, 1000, (0.03,))[0][2].syndromes
    assert np.array_equal(a0, bench.make_workload(0, 1000, (0.03,))[0][2].syndromes)
    assert not np.array_equal(a0, a1)
