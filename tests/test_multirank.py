"""Sharding over ranks with world_size-2 gloo ranks on CPU.

Two decompositions.  Target k-ranges: each rank computes V_x for its k-range
and its E_x share.  Blocks {k, q} (the one the benchmark runs): rank 0
broadcasts the orbitals, each rank computes the partial V_x c of the blocks the
library's assignment (xx_shard_blocks, host code) gives it, the partial V_x c
are all-reduced and the E_x shares summed in rank order.  On CPU the per-rank
compute is the FP64 oracle (the library's compute needs a GPU; the GPU test
test_gpu_shard checks that the library's shards add up); the host data path --
orbital broadcast, block assignment, V_x all-reduce, fixed-order E_x sum -- is
the one bench.py uses.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1111_0716_gb300 import shard


def test_k_ranges_tile_the_mesh():
    for nk in (1, 2, 7, 8, 64):
        for world in (1, 2, 3, 8):
            r = shard.k_ranges(nk, world)
            assert len(r) == world
            assert sum(n for _, n in r) == nk
            k = 0
            for k0, n in r:
                assert k0 == k
                k += n
            sizes = [n for _, n in r]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.k_ranges(4, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    from oracle import oracle
    from paper_1111_0716_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.make_workload("shard", synth.rhombohedral_lattice(7.0, 65.0), (16,) * 3,
                             synth.monkhorst_pack(2), 2.0, 3, 4, [1.0, 0.6, 0.2], 31)
    k0, kn = shard.k_ranges(wl.nk, world)[rank]
    sel = [(k, a) for k in range(k0, k0 + kn) for a in range(wl.n_tgt)]
    vx = oracle.apply(wl, sel=sel).reshape(kn, wl.n_tgt, -1)
    c = wl.c_tgt[k0:k0 + kn]
    w = wl.w_tgt[k0:k0 + kn]
    share = float(np.sum(w * np.einsum("kag,kag->ka", c.conj(), vx).real)) / wl.nk  # (s/2)=1
    total = shard.fixed_order_sum(share)
    if rank == 0:
        full = oracle.apply(wl)
        e_ref, _ = oracle.energy_from_vx(wl, full)
        with open(out_path, "w") as f:
            f.write("%.17g %.17g\n" % (total, e_ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_energy(tmp_path, oracle_mod):
    out = str(tmp_path / "res.txt")
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    total, ref = map(float, open(out).read().split())
    assert abs(total - ref) <= 1e-13 * abs(ref)


def test_block_assignment_covers_every_block_once():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_0716_gb300 import xx
    for nk, n_occ, n_tgt in ((1, 4, 6), (8, 160, 192), (8, 3, 4), (64, 18, 24)):
        nb = nk * (nk + 1) // 2
        for world in (1, 2, 3, 8):
            owner = xx.xx_shard_blocks(nk, n_occ, n_tgt, world)
            assert owner.shape == (nb,) and owner.min() >= 0 and owner.max() < world
            assert np.array_equal(owner, xx.xx_shard_blocks(nk, n_occ, n_tgt, world))
            # balance: no shard above the mean load plus one largest block
            rest = max(n_tgt - n_occ, 0) * n_occ
            cost = np.array([n_occ * (n_occ + 1) // 2 + rest if k == q else n_occ * n_occ + 2 * rest
                             for k in range(nk) for q in range(k, nk)])
            load = np.bincount(owner, weights=cost, minlength=world)
            assert load.max() <= cost.sum() / world + cost.max()
    with pytest.raises(xx.XXError):
        xx.xx_shard_blocks(0, 1, 1, 1)


def _block_worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    import __graft_entry__  # noqa: F401  (puts the repository on sys.path)
    from oracle import oracle
    from paper_1111_0716_gb300 import synth, xx
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = synth.make_workload("shard", synth.rhombohedral_lattice(7.0, 65.0), (16,) * 3,
                             synth.monkhorst_pack(2), 2.0, 3, 4, [1.0, 0.6, 0.2], 31)
    # orbital distribution: rank 0's coefficients reach every rank
    c = torch.from_numpy(wl.coeff.copy() if rank == 0 else np.zeros_like(wl.coeff))
    dist.broadcast(c, src=0)
    wl = wl.replace(coeff=c.numpy())
    owner = xx.xx_shard_blocks(wl.nk, wl.n_occ, wl.n_tgt, world)

    def blk(k, q):
        k, q = min(k, q), max(k, q)
        return k * wl.nk - k * (k - 1) // 2 + (q - k)
    # partial V_x c of this rank's blocks: for target k, the occupied bands of the
    # q-points whose block {k, q} this rank owns
    vx = np.zeros_like(wl.c_tgt)
    for k in range(wl.nk):
        w_mask = wl.w_occ.copy()
        for q in range(wl.nk):
            if owner[blk(k, q)] != rank:
                w_mask[q] = 0.0
        sel = [(k, a) for a in range(wl.n_tgt)]
        vx[k] = oracle.apply(wl, sel=sel, w_occ=w_mask).reshape(wl.n_tgt, -1)
    share, _ = oracle.energy_from_vx(wl, vx)
    total = shard.fixed_order_sum(share)
    vt = torch.from_numpy(vx)
    dist.all_reduce(vt)
    if rank == 0:
        full = oracle.apply(wl)
        e_ref, _ = oracle.energy_from_vx(wl, full)
        err_v = float(np.abs(vt.numpy() - full).max() / np.abs(full).max())
        with open(out_path, "w") as f:
            f.write("%.17g %.17g %.17g %d\n" % (total, e_ref, err_v, int(np.bincount(owner).size)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_block_shards_reproduce_the_operator(tmp_path, oracle_mod):
    import __graft_entry__
    __graft_entry__.build()
    out = str(tmp_path / "blocks.txt")
    world = 2
    mp.start_processes(_block_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    total, ref, err_v, used = open(out).read().split()
    assert abs(float(total) - float(ref)) <= 1e-13 * abs(float(ref))
    assert float(err_v) <= 1e-13
    assert int(used) == world


def _bench_collectives_worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(5)
    c_all = rng.standard_normal((2, 3, 7)) + 1j * rng.standard_normal((2, 3, 7))
    c = torch.from_numpy(c_all.copy() if rank == 0 else np.zeros_like(c_all))
    bench.distribute_orbitals(c)
    ok_c = bool(np.array_equal(c.numpy(), c_all))
    # a partial "V_x c" and E_x share per rank
    vx = torch.from_numpy((rank + 1) * c_all)
    ex = torch.tensor([-(rank + 1.5), 0.25 * rank], dtype=torch.float64)
    parts = [torch.empty(2, dtype=torch.float64) for _ in range(world)]
    bench.combine_shards(vx, ex, parts)
    want_vx = sum(r + 1 for r in range(world)) * c_all
    want_ex = [sum(-(r + 1.5) for r in range(world)), sum(0.25 * r for r in range(world))]
    ok = ok_c and np.allclose(vx.numpy(), want_vx, rtol=1e-15, atol=0) and \
        ex.tolist() == want_ex
    with open(out_path + ".%d" % rank, "w") as f:
        f.write("1" if ok else "0")
    dist.barrier()
    dist.destroy_process_group()


def test_bench_collectives_on_two_gloo_ranks(tmp_path):
    """bench.py's orbital broadcast and shard combination (the data path of its
    multi-GPU step) on CPU tensors."""
    out = str(tmp_path / "coll")
    world = 2
    mp.start_processes(_bench_collectives_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    for r in range(world):
        assert open(out + ".%d" % r).read() == "1"
