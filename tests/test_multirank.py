"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

Observers are independent, so ranks shard the observer set and need no
collective on the data path: each rank owns an equally sized, distinct set,
the timing is reduced with a max over ranks, and rank 0 alone prints.  Here
the per-rank work is the CPU oracle (no GPU on this machine), which checks
that the shards together give exactly the unsharded result.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("ws", [2, 4])
def test_rank_observer_sets_are_distinct_and_equal(ws):
    import bench
    sets = [bench.rank_workload(r, ws).observers for r in range(ws)]
    base = bench.rank_workload(0, ws)
    for r in range(ws):
        w = bench.rank_workload(r, ws)
        assert w.observers.shape == base.observers.shape
        assert w.surface.n_panels == base.surface.n_panels and w.nt == base.nt
    allobs = np.concatenate(sets)
    d = np.linalg.norm(allobs[:, None, :] - allobs[None, :, :], axis=-1)
    np.fill_diagonal(d, np.inf)
    assert d.min() > 1e-6          # no observer is computed twice


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    from fwh_inputs import workload
    from oracle import Oracle
    wsz, rk, _ = bench.dist_setup()
    assert (wsz, rk) == (ws, rank)
    assert bench.max_over_ranks(float(rank + 1), ws) == float(ws)
    w = workload(1, scale=0.25)
    mine = np.arange(rank, w.observers.shape[0], ws)     # this rank's observer shard
    f = w.fields("float64").numpy()
    p, ts, nv = Oracle.from_workload(w).forward(f, w.observers[mine])
    # the test gathers the shards to compare them; the timed path never does
    gathered = [None] * ws
    dist.all_gather_object(gathered, (mine.tolist(), p.tolist(), nv.tolist()))
    bench.barrier(ws)
    if rank == 0:
        with open(os.path.join(out_dir, "shards.json"), "w") as fh:
            json.dump(gathered, fh)
    dist.destroy_process_group()


def test_gloo_two_ranks_shards_reassemble_the_unsharded_result(tmp_path):
    from fwh_inputs import workload
    from oracle import Oracle
    ws = 2
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn")
    shards = json.load(open(tmp_path / "shards.json"))
    w = workload(1, scale=0.25)
    p_all, _, nv_all = Oracle.from_workload(w).forward(w.fields("float64").numpy(),
                                                        w.observers)
    seen = []
    for idx, p, nv in shards:
        np.testing.assert_array_equal(np.asarray(p), p_all[idx])
        np.testing.assert_array_equal(np.asarray(nv), nv_all[idx])
        seen += idx
    assert sorted(seen) == list(range(w.observers.shape[0]))


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    # the reference arm carries the contract keys of the line it stands beside
    for k in ("metric", "unit", "higher_is_better", "steps", "warmup", "config"):
        assert k in d, k
    assert d["higher_is_better"] is True and d["unit"] == "evals/s"
    assert d["config"]["workload"] == "sphere-dipole-32768x2048x72"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]


# ---- panel sharding (Sec. III A Face partition, Sec. III B max/min all-reduce) ----

def test_face_partition_is_greedy_by_size():
    from paper_2312_16263_gb300.shard import partition_faces
    parts = partition_faces([5, 9, 3, 9, 1, 4], 2)
    # faces 1, 3 (9), 0 (5), 5 (4), 2 (3), 4 (1), each to the least-loaded rank
    assert parts == [[0, 1, 4], [2, 3, 5]]
    loads = [sum([5, 9, 3, 9, 1, 4][i] for i in p) for p in parts]
    assert loads == [15, 16]
    assert sorted(sum(partition_faces(list(range(1, 20)), 4), [])) == list(range(19))


class _OracleRankEngine:
    """CPU stand-in for one rank's FWH handle (the library needs a GPU): the
    same calls, answered by the FP64 oracle on the rank's faces."""

    def __init__(self, w, faces, mine):
        from oracle import Oracle
        self.w, self.faces, self.mine = w, faces, mine
        self.orc = Oracle.from_workload(w)        # full surface: its window is the global one
        self.set_extremes = None

    def observer_extremes(self):
        from paper_2312_16263_gb300.shard import rank_panels
        idx = rank_panels(self.faces, self.mine)
        y = self.w.surface.centroids[idx]
        d = (self.w.observers[:, None, :] - y[None, :, :]).reshape(-1, 3)
        R, _, _ = self.orc.convected_distance(d)
        R = R.reshape(self.w.observers.shape[0], -1)
        return R.max(axis=1), R.min(axis=1)

    def set_observer_extremes(self, mx, mn):
        self.set_extremes = (np.asarray(mx), np.asarray(mn))

    def forward(self, fields):
        import torch
        p = 0.0
        for f in self.mine:                       # the oracle sums one face range at a time
            pf, _, _ = self.orc.forward(fields, self.w.observers, p_range=self.faces[f])
            p = p + pf
        return torch.as_tensor(p)


def _panel_worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    from fwh_inputs import workload
    from paper_2312_16263_gb300.shard import (face_blocks, partition_faces, shard_setup,
                                              sharded_forward)
    bench.dist_setup()
    w = workload(1, scale=0.25)
    faces = face_blocks(w.surface.n_panels, 24)          # uneven last face
    parts = partition_faces([hi - lo for lo, hi in faces], ws)
    eng = _OracleRankEngine(w, faces, parts[rank])
    shard_setup(eng)
    p = sharded_forward(eng, w.fields("float64").numpy())
    mx, mn = eng.set_extremes
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"p": p.tolist(), "mx": mx.tolist(), "mn": mn.tolist(),
                   "parts": parts}, fh)
    dist.destroy_process_group()


def test_gloo_two_ranks_panel_shards_reassemble_the_unsharded_result(tmp_path):
    from fwh_inputs import workload
    from oracle import Oracle
    ws = 2
    mp.start_processes(_panel_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn")
    w = workload(1, scale=0.25)
    orc = Oracle.from_workload(w)
    p_all, ts_all, _ = orc.forward(w.fields("float64").numpy(), w.observers)
    d = (w.observers[:, None, :] - w.surface.centroids[None, :, :]).reshape(-1, 3)
    R = orc.convected_distance(d)[0].reshape(w.observers.shape[0], -1)
    outs = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    assert sorted(sum(outs[0]["parts"], [])) == list(range(len(sum(outs[0]["parts"], []))))
    for o in outs:   # every rank ends with the global extremes and the summed signal
        np.testing.assert_array_equal(np.asarray(o["mx"]), R.max(axis=1))
        np.testing.assert_array_equal(np.asarray(o["mn"]), R.min(axis=1))
        np.testing.assert_allclose(w.mach * np.asarray(o["mx"]), ts_all, rtol=1e-15)
        np.testing.assert_allclose(np.asarray(o["p"]), p_all, rtol=1e-12,
                                   atol=1e-13 * np.abs(p_all).max())
