"""The benchmark's multi-rank bookkeeping on the CPU: two gloo ranks stand in
for two GPUs running independent replicas.  The slowest rank's time sets the
step time, the job rate counts every rank's flops, a replica that did not
converge zeroes the line for all, and the oracle arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]                      # rank 1 is the slow one
        t = bench._reduce_over_ranks(ms, world, "cpu", "max")
        ok = bench._reduce_over_ranks([1.0, 0.0][rank], world, "cpu", "min")
        ok_all = bench._reduce_over_ranks(1.0, world, "cpu", "min")

        class A:                                        # the reference arm's arguments
            warmup, steps, gpus = 0, 0, world
        buf = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(buf):
                bench.run_reference(A, rank)
        out[rank] = (t, ok, ok_all, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    for rank in (0, 1):
        t, ok, ok_all, printed = out[rank]
        assert t == 150.0                      # max over ranks on every rank
        assert ok == 0.0 and ok_all == 1.0     # one failed replica fails the job
    assert out[1][3] == ""                     # rank 1 prints nothing in the oracle arm


def test_single_rank_is_identity():
    assert bench._reduce_over_ranks(3.5, 1, "cpu", "max") == 3.5
    assert bench._reduce_over_ranks(0.0, 1, "cpu", "min") == 0.0


@pytest.mark.parametrize("world", [1, 2, 8])
def test_job_rate_counts_every_replica(world):
    # weak scaling: each replica does F flops per step; the job's rate is
    # world * F over the slowest rank's step time
    F = 2.0 * 32768 ** 3 / 3.0 + 32768 ** 3 / 3.0
    r = bench._job_tflops(world, F, 400.0)
    assert r == pytest.approx(world * F / 0.4 / 1e12, rel=1e-15)


def test_step_stats():
    s = bench._step_stats([380.0, 381.0, 379.5, 382.0, 380.5])
    assert (s["median_ms"], s["min_ms"], s["max_ms"], s["steps"]) == (380.5, 379.5, 382.0, 5)
    # t(0.975, 4) * sd / sqrt(5), sd = 0.9618...
    assert s["ci95_mean_ms"] == pytest.approx(2.776 * 0.96176920308356 / 5 ** 0.5, rel=1e-9)
    assert bench._step_stats([1.0])["ci95_mean_ms"] is None


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_shards_of_the_batched_configuration(world):
    """The batched configuration shards over ranks by LPT on flops: every
    matrix on exactly one rank, loads within 0.1% of each other."""
    import numpy as np
    sizes = np.random.default_rng(7).integers(16, 513, 20000).tolist()
    kinds = [0 if i % 2 else 1 for i in range(len(sizes))]
    costs = [(2.0 if k == 0 else 1.0) * n ** 3 for n, k in zip(sizes, kinds)]
    shards = bench._lpt_shards(costs, world)
    assert len(shards) == world
    assert sorted(i for s in shards for i in s) == list(range(len(sizes)))
    loads = [sum(costs[i] for i in s) for s in shards]
    assert max(loads) / (sum(loads) / world) < 1.001
    assert bench._lpt_shards(costs, world) == shards          # deterministic


def test_lpt_shards_small_cases():
    assert bench._lpt_shards([5.0, 4.0, 3.0, 3.0, 3.0], 2) == [[0, 3], [1, 2, 4]]
    assert bench._lpt_shards([], 3) == [[], [], []]
    assert bench._lpt_shards([1.0], 2) == [[0], []]


def test_host_cpu_names(tmp_path):
    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nmodel name\t: Some CPU @ 2.70GHz\n\nprocessor\t: 1\nmodel name\t: Some CPU\n")
    assert bench._host_cpu(str(x86)).startswith("Some CPU @ 2.70GHz, ")
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n")
    assert bench._host_cpu(str(arm)).startswith("Arm implementer 0x41 part 0xd4f, ")
    assert "logical CPUs" in bench._host_cpu(str(tmp_path / "missing"))


def _line_keys(func_name):
    """Keys of the dict literal assigned to `line` inside bench.<func_name>."""
    import ast
    tree = ast.parse(open(bench.__file__).read())
    fn = next(n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name == func_name)
    for node in ast.walk(fn):
        if (isinstance(node, ast.Assign) and any(isinstance(t, ast.Name) and t.id == "line" for t in node.targets)
                and isinstance(node.value, ast.Dict)):
            return {k.value for k in node.value.keys if isinstance(k, ast.Constant)}
    raise AssertionError("no line = {...} in " + func_name)


def test_bench_line_carries_the_contract_keys():
    base = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}
    assert base | {"clocks", "gpu_launches", "roofline"} <= _line_keys("run_gpu")
    assert base | {"impl"} <= _line_keys("run_reference")


def test_forward_error_helper():
    import torch
    Xr = torch.tensor([[1.0, -4.0], [2.0, 1.0]], dtype=torch.float64)
    X = Xr + torch.tensor([[1e-12, 0.0], [0.0, 2e-12]], dtype=torch.float64)
    # column 0: 1e-12 / 2, column 1: 2e-12 / 4
    assert bench._fwd_err(X, Xr) == pytest.approx(5e-13, rel=1e-9)
