"""Host-side logic that needs no GPU: the seeded input recipes and the bench's
reference arm (its JSON line follows the bench contract)."""
import json
import math
import os
import subprocess
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ragged_instance_recipe():
    ns = synth.ragged_sizes(**synth.RAGGED_32)
    assert len(ns) == 32 and all(128 <= n <= 384 for n in ns)
    assert ns == synth.ragged_sizes(**synth.RAGGED_32)          # seeded
    inst = synth.ragged_instances(ns[:3], synth.RAGGED_32["seed"])
    for n, (f, m, d) in zip(ns[:3], inst):
        assert f == n / 8.0 and m.shape == (n, n) and d.shape == (1, 2)
        c = 1.0 / np.sqrt(1.0 - m)
        assert c.min() >= 0.8 - 1e-12 and c.max() <= 1.2 + 1e-12
        assert abs(np.linalg.norm(d) - 1.0) < 1e-14
        edge = max(np.abs(m[0]).max(), np.abs(m[-1]).max(), np.abs(m[:, 0]).max(), np.abs(m[:, -1]).max())
        assert edge <= 0.1 * np.abs(m).max()                        # c tapers to 1 towards the box boundary


def test_workload_recipes_are_seeded():
    for name in ("2d_n64", "2d_n256", "2d_n512_r64", "2d_n256_r16"):
        w = synth.WORKLOADS[name]
        m1, d1 = synth.make_workload(w)
        m2, d2 = synth.make_workload(w)
        assert np.array_equal(m1, m2) and np.array_equal(d1, d2)
        assert m1.shape == (w.n, w.n) and d1.shape == (w.n_rhs, 2)
        assert math.isclose(w.omega, 2 * math.pi * w.freq)


def test_bench_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host (the n = 64
    workload here, a few seconds; the default n = 512 workload takes minutes)."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "0",
                        "--workload", "2d_n64"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]
    assert line["steps"] == 2 and line["oracle_iters"] >= 1


def test_method_work_counts_match_the_stated_sizes():
    """The bench's algorithmic work model against the sizes stated for the
    workloads: n = 512 factorization about 3.1 GFLOP, 3D n = 64 factors about
    11.6 GB in FP32 per full read, the sweep reading them twice per slab solve."""
    sys.path.insert(0, ROOT)
    import bench

    class Fake:
        def __init__(self, n, dim, b, bs, L):
            self.n, self.dim, self.fft_len = n, dim, L
            self.n_tot = n + 2 + 2 * b
            self.n_slabs = -(-(n + 2) // bs)
            self.b, self.bs = b, bs

        def slab_info(self, i):
            n, b, bs, ns = self.n, self.b, self.bs, self.n_slabs
            if i == 0:
                return -b, b + bs, 0
            return i * bs, (n + 2 - i * bs) + b if i == ns - 1 else bs, b

    w2 = bench.method_work(Fake(512, 2, 12, 4, 1024), 4)
    # 128 slabs of width 16 and the last of width 26 (2 remainder + 12 PML + 12 auxiliary), n_y = 538
    exp = 538 * (8 / 3 + 8) * (128 * 16 ** 3 + 26 ** 3)
    assert abs(w2["factor"]["flops"] / exp - 1) < 1e-12 and abs(exp / 3.0e9 - 1) < 0.04
    assert abs(w2["matvec"]["flops"] / 210e6 - 1) < 0.01
    w3 = bench.method_work(Fake(64, 3, 8, 4, 128), 4)
    # sum over slabs of n_tot M^2 complex64 entries (16 x 984^2 + 1476^2) x 82 x 8 B = 11.6 GB
    fac = 82 * (16 * 984 ** 2 + 1476 ** 2) * 8
    assert abs(fac / 11.6e9 - 1) < 0.02
    assert w3["sweep"]["bytes"] == 2 * 82 * 8 * (2 * 16 * 984 ** 2 + 1476 ** 2)


def _max_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    got = bench.max_over_ranks([rank + 1.0, 10.0 - rank, 0.5 * rank], torch.device("cpu"), world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(got, f)


def test_max_over_ranks_with_two_gloo_ranks(tmp_path):
    """The multi-GPU bench path (independent replicas, max-over-ranks timing)
    on two CPU ranks: every rank gets the element-wise maximum."""
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_max_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            assert json.load(f) == [2.0, 10.0, 0.5]


def test_bench_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3, 1.5], None, 1) == [3.0, 1.5]


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
