"""The sharded library calls on the CUDA path (the distributed remark of Section 4), with
two gloo ranks that share the one GPU (their kernels never wait on each other; the
collectives run on the host): row shards through apply_csr_row_shard equal the oracle's
whole transform, and column shards through nmf_anchors_column_shard give the anchors of
the whole Z.  No scaling over GPUs is measured here."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1606_05732_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, D, M, B, SEED = 20011, 45, 24, 2048, 23


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_1606_05732_gb300 import distributed as cgd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cuda", 0)
        X = synth.csr_bernoulli(N, D, 0.05, seed=9, values="uniform")
        a, b = cgd.shard_range(N, world, rank)
        rp, ci, v = cgd.shard_csr_rows(X.row_ptr, X.col_idx, X.vals, a, b)
        Y = cgd.apply_csr_row_shard(torch.from_numpy(rp.astype(np.int32)).to(dev), torch.from_numpy(ci).to(dev),
                                    torch.from_numpy(v).to(dev), D, M, B, SEED, row_offset=a)
        c0, c1 = cgd.shard_range(D, world, rank)
        rpc, cic, vc = cgd.shard_csr_cols(X.row_ptr, X.col_idx, X.vals, c0, c1)
        imax, imin = cgd.nmf_anchors_column_shard(torch.from_numpy(rpc.astype(np.int32)).to(dev),
                                                  torch.from_numpy(cic.astype(np.int32)).to(dev),
                                                  torch.from_numpy(vc).to(dev), c1 - c0, M, B, SEED, col_offset=c0)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), Y=Y.cpu().numpy(), imax=imax, imin=imin)
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_one_gpu_row_and_column_shards(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    X = synth.csr_bernoulli(N, D, 0.05, seed=9, values="uniform")
    Yo = oracle.apply_csr(SEED, N, D, M, B, X.row_ptr, X.col_idx, X.vals)
    omax, omin = oracle.row_argmax_argmin(Yo)
    srt = np.sort(Yo, axis=1)
    scale = np.abs(Yo).max(axis=1)
    clear_max = (srt[:, -1] - srt[:, -2]) > 1e-4 * scale
    clear_min = (srt[:, 1] - srt[:, 0]) > 1e-4 * scale
    ys = []
    for rank in range(world):
        r = np.load(tmp_path / f"rank{rank}.npz")
        ys.append(r["Y"])
        assert np.linalg.norm(r["Y"] - Yo) <= 1e-5 * np.linalg.norm(Yo)
        np.testing.assert_array_equal(r["imax"][clear_max], omax[clear_max])
        np.testing.assert_array_equal(r["imin"][clear_min], omin[clear_min])
    np.testing.assert_array_equal(ys[0], ys[1])  # every rank holds the same sum
