"""Host logic of the multi-GPU (replicas) layout of bench.py, run as two
gloo ranks on the CPU: the step time is the maximum over ranks and the
value counts every rank's unknowns."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms_list, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate(ms_list[rank], 1000, world, "cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms_list = [2.0, 5.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ms_list, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 5.0
        assert value == pytest.approx(2 * 1000 / 5e-3)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.aggregate(4.0, 500, 1) == (4.0, 500 / 4e-3)


def _run_reference(env_extra):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, cwd=root, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    """The reference arm (the oracle on the host cores) prints one JSON line with
    the GPU arm's metric, unit and workload, the oracle as its CPU baseline and
    an end-to-end entry without device copies."""
    out = _run_reference({"RANK": "0"})
    assert len(out) == 1
    d = out[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == "unknowns solved/s to 1e-10 rel. residual" and d["unit"] == "unknowns/s"
    assert d["config"]["workload"] == "linear_mhs_129"
    # the configuration the GPU arm prints: the workload, the FP64 mode and the same run notes
    import bench
    pr, mags, cfg = bench.workload(0)
    assert d["config"] == dict(cfg, mode="fp64", **bench.RUN_NOTES)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    assert _run_reference({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_profiled_traffic_follows_the_measured_kernel_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu record only while
    the measured device function is unchanged: editing another function of the
    file keeps it, editing the function itself drops it (None)."""
    import json
    import shutil
    import bench
    assert bench.profiled_traffic("smooth64") is not None
    root = tmp_path
    (root / "profiles").mkdir()
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    src_rel = rec["kernels"]["smooth64"]["source"]
    (root / os.path.dirname(src_rel)).mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), root / "profiles" / "traffic.json")
    src = open(os.path.join(bench.ROOT, src_rel)).read()
    monkeypatch.setattr(bench, "ROOT", str(root))
    (root / src_rel).write_text(src + "\n// another function edited\n")
    assert bench.profiled_traffic("smooth64") == rec["kernels"]["smooth64"]["bytes_per_launch"]
    body = src.index("void colour_body(")
    edited = src[:body] + src[body:].replace("if (j > g.ny - 2) return;", "if (j >= g.ny - 1) return;", 1)
    assert edited != src
    (root / src_rel).write_text(edited)
    assert bench.profiled_traffic("smooth64") is None
    assert bench.profiled_traffic("no_such_kernel") is None
