"""Sharding over target k-points with world_size-2 gloo ranks on CPU.

Each rank computes V_x for its k-range with the FP64 oracle (a stand-in for the
per-GPU library call, which needs a GPU) and its E_x share; the fixed-order
sum over ranks must equal the single-process E_x, and the k-ranges must tile
the mesh.
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
