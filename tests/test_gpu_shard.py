"""The sharded trace system on the GPU: two ranks (processes) on one GPU,
each with its own library context over its slab of a periodic mesh, exchanging
the shared faces over gloo on the host (no kernel of one rank waits for the
other).  After the exchange each rank's b-hat equals the whole mesh's on its
faces; the distributed GMRES and the local recovery give the whole mesh's
Newton increment."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from paper_2507_22195_gb300 import inputs as I  # noqa: E402
from paper_2507_22195_gb300 import shard as SH  # noqa: E402

pytestmark = pytest.mark.gpu
KW = dict(flux=1, Mach=0.3, prec=0)


def _case():
    mesh = I.periodic_mesh((4, 2, 1), 1, 2)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
    return mesh, st


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        mesh, st = _case()
        sh = SH.Shard(mesh, SH.partition(mesh, world), rank)
        sys_ = SH.ShardedSystem(sh, sh.local_state(st), dist, **KW)
        bh = sys_.condense()
        n = mesh.n_global_faces * 5 * mesh.n2
        x, it, res = sys_.solve(bh, rtol=1e-12, restart=n, max_iter=2 * n)
        dV = sys_.recover(x)
        torch.cuda.synchronize()
        out[rank] = (sh.elems, sh.gfaces, bh.cpu().numpy(), x.cpu().numpy(), dV.cpu().numpy(), it, res)
        sys_.close()
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_one_gpu_match_the_whole_mesh():
    from paper_2507_22195_gb300 import mehdg as M
    mesh, st = _case()
    ctx = M.Context(mesh, **KW)
    d = torch.device("cuda:0")
    ctx.set_state(torch.tensor(st.v, device=d), torch.tensor(st.vhat, device=d), None,
                  torch.tensor(st.vstar, device=d))
    bh = ctx.condense()
    n = bh.numel()
    x, it, res = ctx.solve_condensed(bh, rtol=1e-12, restart=n, max_iter=2 * n)
    dV = ctx.recover(x)
    torch.cuda.synchronize()
    bh, x, dV = bh.cpu().numpy(), x.cpu().numpy(), dV.cpu().numpy()
    ctx.close()
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_rank, args=(2, _port(), out), nprocs=2, join=True)
        out = dict(out)
    assert sorted(out) == [0, 1]
    for rank, (el, gf, bh_r, x_r, dV_r, it_r, res_r) in out.items():
        assert res_r <= 1e-12
        assert np.abs(bh_r - bh[gf]).max() <= 1e-12 * np.abs(bh).max()
        assert np.abs(x_r - x[gf]).max() <= 1e-9 * np.abs(x).max()
        assert np.abs(dV_r - dV[el]).max() <= 1e-9 * np.abs(dV).max()
