"""Host-side logic of bench.py that needs no GPU: the replica plumbing used
when the benchmark runs as N processes (barrier and max-over-ranks timing on
a gloo process group, world size 2), and the reference arm (the CPU oracle)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    d = bench.Dist()
    d.barrier()
    slowest = d.max(1.0 + rank)  # rank 1 is the slow one
    d.barrier()
    q.put((rank, d.world, slowest))
    d.close()


def test_replicas_take_the_max_time_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.0), (1, 2, 2.0)]


def test_reference_arm_prints_one_json_line():
    """The oracle arm on a small mesh of the benchmark's generator; its config
    names the mesh it ran, and the OpenMP build reports the threads it used."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--ref-size", "64"], capture_output=True, text=True, check=True,
                       cwd=ROOT)
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["metric"] == "cell-updates/s" and j["value"] > 0
    assert j["higher_is_better"] is True and j["steps"] == 2 and j["warmup"] == 1
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert j["config"]["nx"] == 64 and j["config"]["workload"].endswith("64x64")
    assert j["e2e"]["h2d_bytes_per_step"] == 0


def test_kernel_source_hash_follows_code_not_comments(tmp_path):
    """The DRAM-traffic and FP64-flop counters under profiles/ are used only
    while this hash matches the one they were captured with: a comment or
    layout edit keeps it, any code edit changes it."""
    import shutil

    sys.path.insert(0, ROOT)
    import bench

    csrc = os.path.join("paper_1607_08710_gb300", "csrc")
    os.makedirs(tmp_path / csrc)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(ROOT, csrc, f), tmp_path / csrc / f)
    base = bench.kernel_source_hash(str(tmp_path))
    assert base == bench.kernel_source_hash()
    path = tmp_path / csrc / bench.KERNEL_SOURCES[0]
    text = path.read_text()
    path.write_text("// an added comment\n/* and a block\n   comment */\n" + text.replace("\n", "\n\n", 3))
    assert bench.kernel_source_hash(str(tmp_path)) == base
    path.write_text(text + "\nnamespace lf { inline int extra_code() { return 1; } }\n")
    assert bench.kernel_source_hash(str(tmp_path)) != base
