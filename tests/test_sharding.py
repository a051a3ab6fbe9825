"""The frequency sharding used for N > 1 GPUs, exercised with two CPU ranks
over gloo: every (omega, direction) is solved by exactly one rank, and the
spectrum gathered from the ranks equals the single-process one (the solves
are independent, so no data-path collective is needed)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import oracle.tddft_oracle as O  # noqa: E402
from paper_1005_5340_gb300 import synth  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, w = synth.workload("tiny4")
    om = w["omega"][:10]
    groups = bench.omega_schedule(om.size, rank, world, per_step=3)
    mine = np.concatenate(groups)
    P, _ = O.polarizability_gmres(s, om[mine], w["eps"], w["restart"], 1e-12)
    buf = torch.zeros((om.size, 3, 3, 2), dtype=torch.float64)
    buf[torch.from_numpy(mine)] = torch.view_as_real(torch.from_numpy(P))
    owned = torch.zeros(om.size, dtype=torch.int64)
    owned[torch.from_numpy(mine)] = 1
    dist.all_reduce(buf)
    dist.all_reduce(owned)
    if rank == 0:
        out.put((torch.view_as_complex(buf).numpy(), owned.numpy()))
    dist.destroy_process_group()


def test_two_rank_frequency_sharding_matches_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    P, owned = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.all(owned == 1)
    s, w = synth.workload("tiny4")
    ref, _ = O.polarizability_gmres(s, w["omega"][:10], w["eps"], w["restart"], 1e-12)
    assert np.max(np.abs(P - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_schedule_partitions_every_grid():
    for n in (1, 7, 64, 256):
        for world in (1, 2, 3, 8):
            seen = np.concatenate([np.concatenate(bench.omega_schedule(n, r, world, 5) or [[]])
                                   for r in range(world)]).astype(int)
            assert sorted(seen.tolist()) == list(range(n))
