"""Host logic of the single-mesh multi-GPU partition (paper Section 2.4):
node ranges per rank, the elements each rank computes, its halo and the
per-step exchange lists.  Checked on the CPU: the plan's structure, and two
gloo ranks that each step their own sub-mesh (with the FP64 oracle standing
in for a rank's GPU) and exchange halo temperatures after every step must
reproduce the one-rank oracle run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1909_05098_gb300.partition import check_plan, plan_partition


def _internal_order(p):
    """The library's internal node order (host-only layout planning)."""
    from paper_1909_05098_gb300.build import build
    build()
    from paper_1909_05098_gb300 import fedfem as ff
    faces = p.conv_faces if len(p.conv_faces) else None
    d = ff.fedfem_plan_layout(p.elem_type, p.xyz, p.conn, dirichlet_nodes=p.dirichlet_nodes, faces=faces)
    return d["node_of"]


def _workloads():
    from synth.scenarios import cube_hex_td_convective, ellipsoid_tet_td
    return [cube_hex_td_convective(n=8), ellipsoid_tet_td(axes=(0.008, 0.006, 0.005))]


@pytest.mark.parametrize("n_ranks", [2, 3, 4])
def test_plan_is_consistent(n_ranks):
    for w in _workloads():
        p = w.problem
        free = np.ones(p.n_nodes, dtype=bool)
        free[p.dirichlet_nodes] = False
        plans = plan_partition(p.conn, p.n_nodes, free, n_ranks, _internal_order(p))
        check_plan(plans, p.conn, p.n_nodes, free)
        sizes = [len(pl.owned) for pl in plans]
        assert max(sizes) - min(sizes) <= 1                       # balanced node ranges
        # redundant (boundary) elements stay a fraction of the mesh on these small meshes
        assert sum(len(pl.elements) for pl in plans) < 2.0 * len(p.conn)


def _sub_problem(p, plan):
    """The rank's own problem: its elements, their nodes (increasing global id,
    so the oracle sums in the one-rank order), global Dirichlet nodes and the
    halo nodes held (the halo values are overwritten after every exchange),
    every film face of an owned node."""
    import copy
    from synth.problem import Problem
    loc = -np.ones(p.n_nodes, dtype=np.int64)
    loc[plan.nodes] = np.arange(len(plan.nodes))
    dir_global = np.asarray(p.dirichlet_nodes, dtype=np.int64)
    dir_T = dict(zip(dir_global.tolist(), np.asarray(p.dirichlet_T, dtype=np.float64).tolist()))
    T0 = p.T0_array()
    held = np.concatenate([dir_global[np.isin(dir_global, plan.nodes)], plan.halo])
    held_T = np.array([dir_T.get(int(g), T0[g]) for g in held])
    faces = np.asarray(p.conv_faces, dtype=np.int64)
    if len(faces):
        owned = np.zeros(p.n_nodes, dtype=bool)
        owned[plan.owned] = True
        faces = faces[owned[faces].any(axis=1)]
    q = copy.copy(p)
    q.xyz = p.xyz[plan.nodes]
    q.conn = loc[p.conn[plan.elements]].astype(np.int32)
    q.dirichlet_nodes = loc[held].astype(np.int32)
    q.dirichlet_T = held_T
    q.conv_faces = loc[faces].astype(np.int32) if len(faces) else np.zeros((0, 4), np.int32)
    q.T0 = T0[plan.nodes]
    return Problem(**{k: getattr(q, k) for k in Problem.__dataclass_fields__})


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_worker(rank, world, port, n_steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    from oracle import Oracle, critical_dt
    from synth.scenarios import cube_hex_td_convective
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = cube_hex_td_convective(n=8).problem
    dt = 0.5 * critical_dt(p)
    free = np.ones(p.n_nodes, dtype=bool)
    free[p.dirichlet_nodes] = False
    plan = plan_partition(p.conn, p.n_nodes, free, world, _internal_order(p))[rank]
    orc = Oracle(_sub_problem(p, plan))
    loc = -np.ones(p.n_nodes, dtype=np.int64)
    loc[plan.nodes] = np.arange(len(plan.nodes))
    T = orc.initial_field()
    for k in range(n_steps):
        T = orc.step(T, dt, k * dt)
        reqs, bufs = [], {}
        for peer, ids in sorted(plan.send.items()):
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(T[loc[ids]])), dst=peer))
        for peer, ids in sorted(plan.recv.items()):
            bufs[peer] = torch.empty(len(ids), dtype=torch.float64)
            reqs.append(dist.irecv(bufs[peer], src=peer))
        for r in reqs:
            r.wait()
        for peer, ids in plan.recv.items():
            T[loc[ids]] = bufs[peer].numpy()
    q.put((rank, plan.owned, T[loc[plan.owned]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_with_halo_exchange_equal_one_rank_bit_for_bit():
    from oracle import Oracle, critical_dt
    from synth.scenarios import cube_hex_td_convective
    n_steps = 40
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_worker, args=(r, 2, port, n_steps, q)) for r in range(2)]
    for pr in ps:
        pr.start()
    out = [q.get(timeout=300) for _ in ps]
    for pr in ps:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = cube_hex_td_convective(n=8).problem
    ref = Oracle(p).run(0.5 * critical_dt(p), n_steps)
    got = ref.copy()
    got[:] = np.nan
    free = np.ones(p.n_nodes, dtype=bool)
    free[p.dirichlet_nodes] = False
    got[~free] = ref[~free]
    for _, owned, vals in out:
        got[owned] = vals
    assert np.all(np.isfinite(got))
    assert ref.max() > 40.0
    assert np.array_equal(got, ref)
