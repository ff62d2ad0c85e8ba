"""Host-side bookkeeping of bench.py on CPU: the algorithmic byte models and
the rule that ties an ncu DRAM-traffic figure to the code it was taken on.
No GPU involved."""
import json

import bench


def test_code_hash_ignores_comments_but_not_code():
    a = b"int x = 1;  // one\n\n// a comment line\nint y = 2;\n"
    b = b"int x = 1;\n// reworded comment\nint y = 2;   \n"
    c = b"int x = 1;\nint y = 3;\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)


def test_traffic_is_dropped_once_the_kernel_code_changes(tmp_path, monkeypatch):
    files = {"kcore.cu": b"__global__ void k() {}  // v1\n", "kcore_tail.cu": b"", "dsg_kernels.cuh": b"",
             "dsg_common.cuh": b""}
    sha = bench.kernel_source_sha("kcore", read=lambda f: files[f])
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(
        {"w": {"kcore": {"bytes": 123, "source_sha": sha, "capture": "test"}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda name, read=None: sha)
    assert bench.dram_traffic("w", "kcore") == 123
    assert bench.dram_traffic("w", "peel_rounds") is None
    assert bench.dram_traffic("other", "kcore") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda name, read=None: "0" * 16)
    assert bench.dram_traffic("w", "kcore") is None


def test_kcore_byte_model_follows_the_method():
    n, m = 10, 20
    st = {"rem_scanned": 30, "rem_written": 15, "atomics": 50}
    base = bench.kcore_bytes(n, m, st, sum_core=25)
    # the kernel's own atomics and list writes are schedule overhead, not method bytes
    assert bench.kcore_bytes(n, m, dict(st, atomics=51), 25) == base
    assert bench.kcore_bytes(n, m, dict(st, rem_written=16), 25) == base
    # each method decrement (2m - sum core) reads and writes 4 B; each scanned remaining vertex 8 B
    assert bench.kcore_bytes(n, m, st, 24) - base == 8
    assert bench.kcore_bytes(n, m, dict(st, rem_scanned=31), 25) - base == 8
    ov = bench.kcore_overhead_bytes(n, m, st, 25)
    assert ov["extra_atomics"] == 50 - (2 * m - 25)


def _serial_level_peel_decrements(n, rows):
    """Algorithm 2's first phase run by one thread: level k takes the vertices
    of degree k, and a drained vertex takes one from each neighbour whose
    degree is above k (a neighbour reaching k joins the level).  Returns the
    core numbers and the number of decrements."""
    deg = [len(r) for r in rows]
    done = [False] * n
    dec, visited, k = 0, 0, 0
    while visited < n:
        buf = [v for v in range(n) if not done[v] and deg[v] == k]
        for v in buf:
            done[v] = True
        i = 0
        while i < len(buf):
            v = buf[i]
            i += 1
            for u in rows[v]:
                if deg[u] > k:
                    deg[u] -= 1
                    dec += 1
                    if deg[u] == k:
                        done[u] = True
                        buf.append(u)
        visited += len(buf)
        k += 1
    return deg, dec


def test_method_decrements_are_degree_minus_core():
    import numpy as np
    import inputs
    for seed in range(6):
        raw = inputs.random_small(40, 0.05 + 0.04 * seed, seed)
        n = raw.n
        rows = [set() for _ in range(n)]
        for a, b in zip(raw.src.tolist(), raw.dst.tolist()):
            if a != b:
                rows[a].add(b)
                rows[b].add(a)
        rows = [sorted(r) for r in rows]
        m = sum(len(r) for r in rows) // 2
        core, dec = _serial_level_peel_decrements(n, rows)
        assert dec == bench.kcore_pkc_atomics(m, int(np.sum(core)))


def test_replica_launch_command_starts_n_ranks_on_localhost():
    cmd = bench.replica_launch_cmd(["--gpus", "4", "--steps", "2"], 4, 29501)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--master-addr=127.0.0.1" in cmd and "--master-port=29501" in cmd
    assert cmd[-4:] == ["--gpus", "4", "--steps", "2"]
    assert cmd[cmd.index("--master-port=29501") + 1].endswith("bench.py")


def test_replica_launch_runs_ranks_that_see_the_world(tmp_path):
    """The launcher command, pointed at a probe script instead of bench.py,
    starts two gloo ranks on CPU that agree on the world size."""
    import subprocess
    import sys
    probe = tmp_path / "probe.py"
    # each rank writes its own file: prints of two processes on one pipe can interleave
    probe.write_text("import os, sys, torch.distributed as d\n"
                     "d.init_process_group('gloo')\n"
                     "with open(os.path.join(sys.argv[-1], 'rank%d' % d.get_rank()), 'w') as f:\n"
                     "    f.write('rank %d of %d' % (d.get_rank(), d.get_world_size()))\n"
                     "d.destroy_process_group()\n")
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = bench.replica_launch_cmd([], 2, port)
    at = [i for i, c in enumerate(cmd) if c.endswith("bench.py")]
    assert len(at) == 1
    cmd[at[0]] = str(probe)
    cmd.append(str(tmp_path))
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=240)
    assert out.returncode == 0, out.stderr[-2000:]
    assert (tmp_path / "rank0").read_text() == "rank 0 of 2"
    assert (tmp_path / "rank1").read_text() == "rank 1 of 2"
