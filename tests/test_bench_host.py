"""Host logic of bench.py for N > 1 ranks, on CPU with the gloo backend
(world size 2): max-over-ranks timing, whole-job throughput, and the reference
arm leaving every rank but 0 without work."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]
    m = bench.max_over_ranks(local_ms, world)
    bench.barrier(world)
    q.put((rank, m, bench.whole_job_mlups(1000, 10, world, m)))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, m, v in out:
        assert m == 20.0  # the slowest rank's time, on every rank
        assert v == pytest.approx(2 * 1000 * 10 / 20e-3 / 1e6)


def test_reference_arm_only_rank0_works(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        gpus, steps, warmup, workload = 2, 1, 0, "drop3d"

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_gpu_arm_helpers_resolve_and_count_bytes():
    """The helpers the GPU arm calls exist and give the per-launch byte counts
    the roofline line reports (240 B per node for FP32 D3Q27)."""
    from paper_2201_12404_gb300 import workloads as WL
    wl = WL.by_name("drop3d")
    assert bench.algorithmic_bytes_k2(wl, 4, 4) == 240 * wl.N
    assert bench.algorithmic_bytes_k2(wl, 8, 8) == 480 * wl.N
    t = bench.recorded_traffic("d3q27_fp32_collide_stream")
    assert t is None or 0.8 * 240 * wl.N < t < 1.5 * 240 * wl.N
    assert bench.recorded_traffic("no such kernel") is None

    class Args:
        precision = "fp32"
    metric, config = bench.metric_and_config(Args(), wl, 1)
    assert "D3Q27" in metric and config["nodes"] == wl.N


def test_pass1_bytes_count_the_padded_auxiliary_fields():
    """Pass 1 writes (rho, psi) at every padded node and j at the interior; pass 1b
    reads the pairs and writes q at every padded node (2 + 2 + 3 = 7 float32 words
    per padded node), reads j and writes F at the interior (with pass 1's j, 9 words
    per interior node), on top of the 27 population reads."""
    from paper_2201_12404_gb300 import workloads as WL
    wl = WL.by_name("drop3d")
    pn = 516 * 516 * 260  # (512 + 4, a multiple of 4) x (512 + 4) x (256 + 4)
    assert bench.algorithmic_bytes_k1(wl, 4, 4) == wl.N * 27 * 4 + pn * 7 * 4 + wl.N * 9 * 4


def test_oracle_crop_is_clipped_to_the_domain():
    """The oracle's sample is a crop of the benchmark domain, never larger than it:
    the 128x128 static drop is timed whole, the impacts on their fixed crops."""
    from paper_2201_12404_gb300 import workloads as WL
    assert bench.crop_of(WL.by_name("static2d")) == (1, 128, 128)
    assert bench.crop_of(WL.by_name("drop2d")) == bench.CPU_CROP_2D
    assert bench.crop_of(WL.by_name("drop3d")) == bench.CPU_CROP
    for name in ("static2d", "drop2d", "drop3d", "drop3d-small"):
        wl = WL.by_name(name)
        assert all(c <= n for c, n in zip(bench.crop_of(wl), (wl.nz, wl.ny, wl.nx)))



def _dict_keys(node):
    import ast
    return {k.value for k in node.keys if isinstance(k, ast.Constant)}


def _entry(d, key):
    return next(v for k, v in zip(d.keys, d.values) if getattr(k, "value", None) == key)


def test_json_lines_carry_the_contract_keys():
    """The benchmark's JSON lines (GPU arm and reference arm) are built from dict
    literals in bench.py: both carry the keys the benchmark contract names, and the
    nested roofline and e2e objects carry theirs."""
    import ast
    src = open(bench.__file__).read()
    tree = ast.parse(src)
    lines = {}
    for fn in (n for n in tree.body if isinstance(n, ast.FunctionDef) and n.name in ("run_ours", "run_reference")):
        for node in ast.walk(fn):
            if (isinstance(node, ast.Assign) and isinstance(node.value, ast.Dict)
                    and any(isinstance(t, ast.Name) and t.id == "line" for t in node.targets)):
                lines[fn.name] = node.value
    assert set(lines) == {"run_ours", "run_reference"}
    base = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "e2e"}
    assert base | {"roofline", "gpu_launches", "clocks"} <= _dict_keys(lines["run_ours"])
    assert base | {"impl", "cpu_baseline"} <= _dict_keys(lines["run_reference"])
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= _dict_keys(_entry(lines["run_ours"], "roofline"))
    for arm in lines.values():
        assert {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"} <= _dict_keys(_entry(arm, "e2e"))
    assert 'line["cpu_baseline"] = oracle_sample(wl)' in src
