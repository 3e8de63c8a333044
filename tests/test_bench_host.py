"""Host logic of bench.py without a GPU: byte accounting and the max/sum aggregation over ranks
(two gloo ranks on the CPU, the path bench.py takes under torchrun)."""
import multiprocessing as mp
import os
import socket

import pytest

import bench


def test_byte_model():
    """Each stored byte read once and each output written once; FP64-accurate work at FP64 bytes
    whatever carries it (the double-float copy is charged as the 6192-byte FP64 W per site)."""
    assert bench.APPLY32 == 3288 and bench.APPLY64 == 6576
    assert bench.W64_BYTES == 6192 and bench.W32_BYTES == 43 * 9 * 8 and bench.W16_BYTES == 1548
    assert bench.RESID64 == 6576 + 192
    assert bench.PRECOMPUTE["mixed"] == 576 + 6192 + 3096 and bench.PRECOMPUTE["f64"] == 576 + 6192
    assert bench.tc_apply_bytes(12) == 1548 + 12 * (96 + 96)
    info = dict(iters=10, fp64_applies=2, reliable_updates=1, restarts=0)
    V = 1000
    expect = V * (10 * (2 * 3288 + bench.ITER_VEC32) + 2 * bench.RESID64 + 2 * bench.RELIABLE32)
    assert bench.solve_bytes(V, info, "mixed") == expect
    assert bench.solve_bytes(V, dict(iters=0, fp64_applies=0, reliable_updates=0, restarts=0), "f64") == \
        V * bench.RESTART64


def test_host_cpu_record():
    nproc, model = bench.host_cpu()
    assert isinstance(nproc, int) and nproc >= 1 and isinstance(model, str) and model


def test_reduce_without_process_group():
    assert bench.reduce_max_sum(3.0, 7.0) == (3.0, 7.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = b.reduce_max_sum(10.0 + rank, 100.0 * (rank + 1))
        b.barrier()
        q.put((rank, t, u))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_max_time_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert out == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_reference_arm_line(capsys):
    """`bench.py --impl reference` times the oracle on the host and prints the contract's JSON line
    (W evaluated once, then one step on the full workload: about half a minute of CPU)."""
    import json
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GB/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["n_gpus"] == 1
    assert line["config"]["workload"] == bench.WORKLOAD and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["nproc"] >= 1 and line["cpu_baseline"]["cpu_model"]
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_charges_time_to_working_launches():
    """Launches of iterations enqueued after a halt return at once; the class's time is charged
    to the 2 x iterations launches that do the work (numbers of a 16^3x32 bench line)."""
    trace = {"apply_f32_dot": (1420, 152.0), "apply_f32_ts": (1420, 148.0), "apply_df64_resid": (60, 56.0)}
    infos = [{"iters": 60}] * 20
    r = bench.roofline(trace, infos, "apply_f32", bench.APPLY32 * 131072, 6790.0, "measured", None)
    assert r["launches"] == 2400 and r["launches_after_halt"] == 440
    assert abs(r["avg_launch_us"] - 300.0 / 2400 * 1e3) < 1e-9
    assert abs(r["achieved"] - bench.APPLY32 * 131072 / (125e-6) / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6790.0) < 1e-12 and r["bound"] == "hbm"
    empty = bench.roofline({}, [], "apply_f32", 1, 6790.0, "measured", None)
    assert empty["achieved"] is None and empty["frac"] is None
