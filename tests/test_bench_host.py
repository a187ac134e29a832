"""Host-side logic of bench.py on CPU: the max-over-ranks / sum-of-units aggregation across two
gloo ranks, the clock-sample summary, the argument defaults and the reference arm's JSON line."""
import os
import socket

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    ms, units = bench.aggregate(10.0 + 5.0 * rank, 3.0 + rank, world)
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in out:
        assert ms == 15.0          # slowest rank
        assert units == 7.0        # sum over ranks


def test_single_rank_aggregate_is_identity():
    assert bench.aggregate(12.5, 4.0, 1) == (12.5, 4.0)


def test_clock_summary_parses_samples(tmp_path):
    c = bench.ClockSampler(0)
    c.proc = object()
    c.path = str(tmp_path / "clk.csv")
    with open(c.path, "w") as f:
        f.write("0, 1900, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1800, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 600, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s["sm_max_mhz"] == 2070
    assert s["sm_mhz"] == 1850           # median of the two loaded samples
    assert s["reasons"] == ["sw_power_cap"]


def test_default_arguments():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.impl == "gw" and a.workload == "plain"
    assert bench.WORKLOADS["plain"].n == 24


def test_workload_precision_and_error_target():
    """The 24^3 path runs FP16X3 with the library's default window; the 36^3 split configuration,
    stated with BF16 hi+lo operands and a 1e-4 target on P~, runs BF16X3 under that target; an
    explicit --precision wins."""
    a = bench.parse_args([])
    assert a.precision == "fp16x3" and bench.ERROR_TARGET.get(a.workload) is None
    s = bench.parse_args(["--workload", "split"])
    assert s.precision == "bf16x3" and bench.ERROR_TARGET["split"] == 1e-4
    assert bench.parse_args(["--workload", "split", "--precision", "fp16x3"]).precision == "fp16x3"


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle's C loop on the host cores and prints one
    JSON line with the contract's keys (no GPU needed)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "grid24_nv32_nc480"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
