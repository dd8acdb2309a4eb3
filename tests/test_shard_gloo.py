"""The multi-worker path on CPU: two gloo ranks each search their Sec. IV.A index range (with the
oracle standing in for the per-rank GPU search) and gather; the gathered result must equal the
single-process result.  A rank that leaves before the gather makes the other rank's collective
fail within a short timeout instead of hanging."""
import datetime
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_range(seqs, l, d, lo, hi):
    from oracle import oracle
    return oracle.search(seqs, l, d, lo=lo, hi=hi)[0]


def _worker(rank, world, port, l, d, seed, weights, out_dir, leave_early):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1403_1313_gb300 import fmgen
    from paper_1403_1313_gb300.shard import sharded_search
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=6))
    job = fmgen.fm_job(6, 90, l, d, seed)
    if leave_early and rank == 1:
        os._exit(0)  # leaves between steps: nothing of its own is in flight
    try:
        res = sharded_search(job.rows(), l, d, rank, world, weights=weights, search_fn=_oracle_range)
        np.save(os.path.join(out_dir, "rank%d.npy" % rank), res)
    except Exception as e:  # the collective noticed the missing peer
        with open(os.path.join(out_dir, "rank%d.err" % rank), "w") as f:
            f.write(type(e).__name__)
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


@pytest.mark.parametrize("weights", [None, [1.0, 3.0]])
def test_two_ranks_gather_equals_single(tmp_path, weights):
    from oracle import oracle
    from paper_1403_1313_gb300 import fmgen
    l, d, seed = 8, 2, 77
    mp.start_processes(_worker, args=(2, _free_port(), l, d, seed, weights, str(tmp_path), False),
                       nprocs=2, join=True, start_method="spawn")
    job = fmgen.fm_job(6, 90, l, d, seed)
    ref, _ = oracle.search(job.rows(), l, d)
    for r in range(2):
        got = np.load(tmp_path / ("rank%d.npy" % r))
        assert np.array_equal(got, ref)


def test_missing_rank_fails_fast(tmp_path):
    ctx = mp.start_processes(_worker, args=(2, _free_port(), 7, 2, 5, None, str(tmp_path), True),
                             nprocs=2, join=False, start_method="spawn")
    for p in ctx.processes:
        p.join(timeout=120)
    assert all(not p.is_alive() for p in ctx.processes)
    assert (tmp_path / "rank0.err").exists() or not (tmp_path / "rank0.npy").exists()


def _dyn_worker(rank, world, port, l, d, seed, chunk, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1403_1313_gb300 import fmgen
    from paper_1403_1313_gb300.shard import dynamic_sharded_search
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=30))
    store = dist.distributed_c10d._get_default_store()
    job = fmgen.fm_job(6, 90, l, d, seed)
    claimed = []

    def counting(seqs, l_, d_, lo, hi):
        claimed.append((lo, hi))
        return _oracle_range(seqs, l_, d_, lo, hi)

    res = dynamic_sharded_search(job.rows(), l, d, store, "motif-chunks-%d" % seed, chunk=chunk,
                                 search_fn=counting)
    np.save(os.path.join(out_dir, "dyn%d.npy" % rank), res)
    np.save(os.path.join(out_dir, "claims%d.npy" % rank), np.array(claimed, dtype=np.int64).reshape(-1, 2))
    dist.destroy_process_group()


@pytest.mark.parametrize("chunk", [1000, 4 ** 8 // 3, 4 ** 8])
def test_dynamic_chunks_gather_equals_single(tmp_path, chunk):
    from oracle import oracle
    from paper_1403_1313_gb300 import fmgen
    l, d, seed = 8, 2, 91
    mp.start_processes(_dyn_worker, args=(2, _free_port(), l, d, seed, chunk, str(tmp_path)),
                       nprocs=2, join=True, start_method="spawn")
    job = fmgen.fm_job(6, 90, l, d, seed)
    ref, _ = oracle.search(job.rows(), l, d)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / ("dyn%d.npy" % r)), ref)
    # Every chunk was claimed exactly once, by one rank or the other.
    claims = np.concatenate([np.load(tmp_path / ("claims%d.npy" % r)) for r in range(2)])
    claims = claims[np.argsort(claims[:, 0])]
    nchunks = (4 ** l + chunk - 1) // chunk
    assert len(claims) == nchunks
    assert claims[0, 0] == 0 and claims[-1, 1] == 4 ** l
    assert np.all(claims[1:, 0] == claims[:-1, 1])


def _dev_gather_worker(rank, world, port, l, d, seed, out_dir):
    """The bench's range-shard step with the oracle standing in for the rank's device search:
    shard.rank_range's split (whole tiles where there are enough), this rank's codes in a buffer
    longer than its count, and the variable-size tensor gather (counts, then codes padded to the
    largest count)."""
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_1403_1313_gb300 as m
    from paper_1403_1313_gb300 import fmgen
    from paper_1403_1313_gb300.shard import gather_codes_device
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=30))
    job = fmgen.fm_job(6, 90, l, d, seed)
    from paper_1403_1313_gb300.shard import rank_range
    lo, hi = rank_range(4 ** l, rank, world)
    codes = _oracle_range(job.rows(), l, d, lo, hi)
    buf = torch.full((codes.size + 5 + 3 * rank,), -1, dtype=torch.int64)  # room past the count
    buf[:codes.size] = torch.from_numpy(codes.astype(np.int64))
    cnt = torch.tensor([codes.size], dtype=torch.int64)
    got = gather_codes_device(buf, cnt)
    np.save(os.path.join(out_dir, "devgather%d.npy" % rank), got.numpy().astype(np.uint64))
    dist.destroy_process_group()


@pytest.mark.parametrize("l,d,seed", [(8, 2, 91), (7, 3, 12), (6, 0, 5), (9, 2, 33)])
def test_range_shard_tensor_gather_equals_single(tmp_path, l, d, seed):
    from oracle import oracle
    from paper_1403_1313_gb300 import fmgen
    mp.start_processes(_dev_gather_worker, args=(2, _free_port(), l, d, seed, str(tmp_path)),
                       nprocs=2, join=True, start_method="spawn")
    job = fmgen.fm_job(6, 90, l, d, seed)
    ref, _ = oracle.search(job.rows(), l, d)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / ("devgather%d.npy" % r)), ref)
