"""Host logic of bench.py: percentiles, and the multi-process path (replicas with a barrier and a
max over ranks) on two gloo processes."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_percentiles():
    v = [5.0, 1.0, 3.0, 2.0, 4.0]
    assert bench.pct(v, 0.5) == 3.0
    assert bench.pct(v, 0.0) == 1.0 and bench.pct(v, 1.0) == 5.0
    assert abs(bench.pct(v, 0.99) - 4.96) < 1e-12



def test_cpu_baseline_all_cores_and_one_thread():
    import fegen
    import oracle
    prob = fegen.make(4, 4, mesh="jitter", lam=1.0)
    before = oracle.num_threads()
    H = oracle.Hierarchy.from_problem(prob, cheb_degree=3)
    x32 = H.solve(prob.b, rtol=1e-8, precision=1)[0]
    H.close()
    cpu, err = bench.cpu_baseline(prob, 3, 1e-8, {"mixed": x32, "zero": 0.0 * x32}, reps=2)
    assert cpu["kind"] == "oracle" and cpu["unit"] == "ms" and cpu["value"] > 0 and cpu["iters"] > 0
    assert cpu["cores"] == before and oracle.num_threads() == before
    assert cpu["plain"]["cores"] == 1 and cpu["plain"]["value"] > 0
    assert cpu["plain"]["bitwise_equal_to_all_cores"] is True
    # the distance of each given solution from the oracle's FP64 solve
    assert err["zero_vs_oracle_fp64"] == 1.0 and err["mixed_vs_oracle_fp64"] < 1e-8
    assert err["oracle_status"] == "ok" and err["oracle_relres"] <= 1e-8

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import bench
rank, ws, local, td = bench.dist()
v = bench.max_over_ranks(td, 10.0 + rank)
td.barrier()
print(f"rank {{rank}} of {{ws}} max {{v}}")
td.destroy_process_group()
"""


def test_two_rank_max_over_ranks_with_gloo():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    assert all("max 11.0" in o for o, _ in outs)


NCU_CSV = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","unnamed>::hyv_cheb_f32(int, const float *)","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","300.00"
"1","1","python","h","void unnamed>::csr_rows<16, double, 0>(long, const long *)","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","msecond","0.10"
"2","1","python","h","void (anonymous namespace)::hyv_cheb_f32(int, const float *)","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","nsecond","100000"
'''


def test_summarize_launches(tmp_path):
    """Launches and device time per kernel, whatever unit ncu prints and however it writes the
    anonymous namespace, and their shares."""
    path = tmp_path / "launches.csv"
    path.write_text(NCU_CSV)
    text = bench.summarize_launches(str(path), split="csr_rows")
    first = text.split("\n\n")[0]
    rows = {line.split()[-1]: line.split() for line in first.splitlines() if "%" in line}
    assert rows["hyv_cheb_f32"][:3] == ["2", "0.400", "80.00%"]
    assert rows["csr_rows<16,double,spmv>"][:3] == ["1", "0.100", "20.00%"]
    assert "segment 1 (from launch 1)" in text


def test_traffic_is_null_once_the_kernel_source_changes(monkeypatch):
    """roofline.traffic comes from the committed capture only while the kernel source is the one
    that was captured."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        import json
        rec = json.load(f)
    workload = next(iter(rec))
    mode = next(iter(rec[workload]))
    want = rec[workload][mode]["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec[workload][mode]["solve_kernels_sha"])
    assert bench.ncu_traffic(workload, mode) == want
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic(workload, mode) is None


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the CPU oracle on the host cores) prints one JSON line with
    the contract's keys, on the small workload."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "helmholtz_4cube_p4", "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and (d["steps"], d["warmup"]) == (3, 3)
    assert d["unit"] == "ms" and d["higher_is_better"] is False and d["value"] > 0
    assert d["config"]["workload"] == "helmholtz_4cube_p4" and d["config"]["dofs"] == 4913
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_once():
    """With two ranks (torchrun, gloo on the CPU) rank 0 alone runs the reference arm and prints
    its line; the other rank exits 0 without work."""
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
                        os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "helmholtz_4cube_p4",
                        "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert len([l for l in r.stdout.splitlines() if l.startswith("{")]) == 1
