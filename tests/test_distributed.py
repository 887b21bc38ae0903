"""Multi-rank host logic on CPU (gloo, world size 2): row shards summed by an
all-reduce equal the whole transform, and column shards merged by a coordinator give
the whole input's NMF anchors (the distributed remark of Section 4).  The per-rank
compute is the oracle's; what is tested is the sharding, the offsets, the collective
and the merge, and that a dead, absent or mismatched rank surfaces as an error."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1606_05732_gb300 import distributed as cgd
from paper_1606_05732_gb300 import synth

N, D, M, B, SEED = 3001, 23, 9, 257, 17


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X = synth.csr_bernoulli(N, D, 0.2, seed=5, values="uniform")
        # row shards: local transform with the global row offset, then a sum
        a, b = cgd.shard_range(N, world, rank)
        rp, ci, v = cgd.shard_csr_rows(X.row_ptr, X.col_idx, X.vals, a, b)
        Y = torch.from_numpy(oracle.apply_csr(SEED, b - a, D, M, B, rp, ci, v, row_offset=a))
        P = torch.from_numpy(oracle.plain_csr(SEED, b - a, D, M, rp, ci, v, row_offset=a))
        cgd.sum_outputs(Y)
        cgd.sum_outputs(P)
        # column shards: every row, some columns; local anchors, coordinator merge
        c0, c1 = cgd.shard_range(D, world, rank)
        rpc, cic, vc = cgd.shard_csr_cols(X.row_ptr, X.col_idx, X.vals, c0, c1)
        Zp = oracle.apply_csr(SEED, N, c1 - c0, M, B, rpc, cic, vc)
        recs = cgd.gather_anchor_records(cgd.local_anchor_records(Zp, c0))
        imax, imin = cgd.merge_anchor_records(recs)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), Y=Y.numpy(), P=P.numpy(), imax=imax, imin=imin)
    finally:
        dist.destroy_process_group()


def test_two_ranks_row_and_column_shards(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    X = synth.csr_bernoulli(N, D, 0.2, seed=5, values="uniform")
    Y = oracle.apply_csr(SEED, N, D, M, B, X.row_ptr, X.col_idx, X.vals)
    P = oracle.plain_csr(SEED, N, D, M, X.row_ptr, X.col_idx, X.vals)
    imax, imin = oracle.row_argmax_argmin(Y)
    for rank in range(world):
        r = np.load(tmp_path / f"rank{rank}.npz")
        np.testing.assert_allclose(r["Y"], Y, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r["P"], P, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(r["imax"], imax)
        np.testing.assert_array_equal(r["imin"], imin)


def test_shard_helpers():
    assert [cgd.shard_range(10, 3, r) for r in range(3)] == [(0, 4), (4, 7), (7, 10)]
    X = synth.csr_ragged(50, 9, seed=2)
    rp, ci, v = cgd.shard_csr_cols(X.row_ptr, X.col_idx, X.vals, 3, 7)
    dense = X.to_dense()[:, 3:7]
    got = synth.CSR(50, 4, rp, ci, v).to_dense()
    np.testing.assert_array_equal(got, dense)
    ties = [np.array([[5.0, 7.0, -1.0, 9.0]]), np.array([[5.0, 2.0, -1.0, 3.0]])]
    imax, imin = cgd.merge_anchor_records(ties)
    assert imax.tolist() == [2] and imin.tolist() == [3]


def _fault_worker(rank, world, port, out_dir, mode):
    """One rank of a two-rank group with a short timeout; rank 1 misbehaves per `mode`,
    rank 0 (and for "shape" both) records what the collective did."""
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=3))
    outcome = "ok"
    t0 = time.monotonic()
    if mode == "dead" and rank == 1:
        os._exit(0)  # dies before the collective, with nothing in flight
    if mode == "absent" and rank == 1:
        time.sleep(8.0)  # alive but never joins; leaves after the others gave up
        os._exit(0)
    try:
        Y = torch.ones(4, 3 if (mode != "shape" or rank == 0) else 2, dtype=torch.float64)
        cgd.sum_outputs(Y)
    except ValueError as e:
        outcome = "ValueError: " + str(e)
    except RuntimeError as e:
        outcome = "RuntimeError: " + str(e)[:200]
    with open(os.path.join(out_dir, f"fault{rank}.txt"), "w") as f:
        f.write(f"{time.monotonic() - t0:.2f}\n{outcome}\n")
    os._exit(0)


@pytest.mark.parametrize("mode", ["dead", "absent", "shape"])
def test_rank_faults_surface_as_errors(tmp_path, mode):
    """Failure detection of the combine step, on the host: a rank that dies before the
    all-reduce, a rank that never joins it, and ranks whose outputs differ in shape.  The
    others raise (connection closed, the process group's 3 s timeout, or the shape check
    on every rank) instead of hanging or returning a wrong sum."""
    import time
    t0 = time.monotonic()
    mp.start_processes(_fault_worker, args=(2, _free_port(), str(tmp_path), mode), nprocs=2,
                       start_method="spawn", join=True)
    assert time.monotonic() - t0 < 60
    lines = (tmp_path / "fault0.txt").read_text().split("\n")
    assert float(lines[0]) < 30
    if mode == "shape":
        for rank in range(2):
            out = (tmp_path / f"fault{rank}.txt").read_text()
            assert "ValueError: ranks hold outputs of different shapes" in out
    else:
        assert lines[1].startswith("RuntimeError"), lines[1]
        assert not (tmp_path / "fault1.txt").exists()
