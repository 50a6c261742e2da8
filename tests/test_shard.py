"""Partitioning across ranks (paper_1811_09599_gb300.shard), world size 2 on
CPU with the gloo backend: the shards cover every unit once, the timing is
the max over ranks, and the slice partition's FP64 sum over ranks gives the
oracle's full path sum (Methods, "Cutting indexes")."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1811_09599_gb300.shard import bitstring_seed, max_over_ranks, shard, slice_sharded_amplitudes


def test_shard_covers_every_unit_once():
    for total in (0, 1, 5, 256, 1001):
        for world in (1, 2, 3, 8):
            got = [shard(total, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == total
            assert all(got[r][1] == got[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(10, 2, 2)
    assert bitstring_seed(1000, 0) != bitstring_seed(1000, 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import network as NW
        from qflex_inputs import grid_problem, random_bitstrings
        prob = grid_problem(3, 4, 16, 2, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2)
        bs = random_bitstrings(prob.n, 2, 7)
        tensors = NW.all_grid_tensors(prob.circuit)
        P = NW.n_slices(prob.circuit, prob.cut_edges)
        calls = []

        def compute(ids):
            calls.append(list(ids))
            out = np.zeros((len(bs), 1 << len(prob.open_tile)), dtype=np.complex128)
            for i, b in enumerate(bs):
                for s in ids:
                    out[i] += NW.slice_amplitudes(prob, b, s, tensors=tensors)
            return torch.from_numpy(out)

        total = slice_sharded_amplitudes(compute, P).numpy()
        t = max_over_ranks(1.0 + rank)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), total)
        # a list of ids: the paths of a rotation circuit that do not vanish
        rot = grid_problem(3, 4, 16, 2, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2, rotations=True)
        rt = NW.all_grid_tensors(rot.circuit)
        nz = NW.nonzero_slices(rot.circuit, rot.cut_edges)
        seen = []

        def compute_rot(ids):
            seen.extend(ids)
            out = np.zeros((len(bs), 1 << len(rot.open_tile)), dtype=np.complex128)
            for i, b in enumerate(bs):
                for s in ids:
                    out[i] += NW.slice_amplitudes(rot, b, s, tensors=rt)
            return torch.from_numpy(out)

        np.save(os.path.join(out_dir, f"rot{rank}.npy"), slice_sharded_amplitudes(compute_rot, nz).numpy())
        np.save(os.path.join(out_dir, f"rotids{rank}.npy"), np.array(seen, dtype=np.int64))
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {calls[0][0] if calls[0] else -1} {len(calls[0])} {P}\n")
    finally:
        dist.destroy_process_group()


def test_slice_partition_gloo_world2(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    from oracle import network as NW
    from qflex_inputs import grid_problem, random_bitstrings
    prob = grid_problem(3, 4, 16, 2, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2)
    bs = random_bitstrings(prob.n, 2, 7)
    ref = NW.amplitudes(prob, bs)
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)                      # every rank gets the same total
    assert np.max(np.abs(r0 - ref)) < 1e-15
    info = [open(tmp_path / f"r{r}.txt").read().split() for r in (0, 1)]
    P = int(info[0][3])
    assert float(info[0][0]) == float(info[1][0]) == 2.0          # max over ranks
    assert int(info[0][1]) == 0 and int(info[1][1]) == P // 2     # contiguous halves
    rot = grid_problem(3, 4, 16, 2, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2, rotations=True)
    nz = NW.nonzero_slices(rot.circuit, rot.cut_edges)
    assert len(nz) < NW.n_slices(rot.circuit, rot.cut_edges)
    ids = [list(np.load(tmp_path / f"rotids{r}.npy")) for r in (0, 1)]
    assert ids[0] + ids[1] == nz and abs(len(ids[0]) - len(ids[1])) <= 1
    got = np.load(tmp_path / "rot0.npy")
    assert np.array_equal(got, np.load(tmp_path / "rot1.npy"))
    assert np.max(np.abs(got - NW.amplitudes(rot, bs))) < 1e-15     # vanishing paths add nothing
    assert int(info[0][2]) + int(info[1][2]) == P
