"""The sharded trace system on the host: two, three and four gloo ranks,
each condensing its own slab of a periodic mesh with the oracle; after the
shared-face exchange every rank's R_V-hat, b-hat and A-hat x equal the whole
mesh's on its faces, and the distributed dot product equals the global one (eq. s32c,
Algorithm 1: sums over the elements on both sides of every face)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

import oracle  # noqa: E402
from paper_2507_22195_gb300 import inputs as I  # noqa: E402
from paper_2507_22195_gb300 import shard as SH  # noqa: E402


def _case(viscous):
    mesh = I.periodic_mesh((4, 2, 1), 1, 2)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, viscous=viscous, M0=0.3)
    kw = dict(Mach=0.3, Re=100.0, viscous=1) if viscous else dict(Mach=0.3)
    return mesh, st, oracle.params(flux=1, **kw)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, viscous, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh, st, prm = _case(viscous)
        parts = SH.partition(mesh, world)
        sh = SH.Shard(mesh, parts, rank)
        ls = sh.local_state(st)
        bh, Ahats = oracle.condense_mesh(prm, sh.mesh, ls, want_Ahat=True)
        bh = sh.sum_shared(torch.tensor(bh), dist)
        x_glob = I.random_direction(st.vhat.shape, 91, 1.0)
        x = x_glob[sh.gfaces]
        y = oracle.assemble_Ahat(sh.mesh, Ahats) @ x.ravel()
        y = sh.sum_shared(torch.tensor(y.reshape(x.shape)), dist)
        d = sh.dot(torch.tensor(x), y, dist)
        _, _, rh = oracle.residual_mesh(prm, sh.mesh, ls)
        rh = sh.sum_shared(torch.tensor(rh), dist)
        out[rank] = (sh.gfaces, bh.numpy(), y.numpy(), d, {r: len(v) for r, v in sh.peers.items()}, rh.numpy())
    finally:
        dist.destroy_process_group()


def _run(world, viscous):
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_rank, args=(world, _free_port(), viscous, out), nprocs=world, join=True)
        return dict(out)


@pytest.mark.parametrize("world,viscous", [(2, False), (3, False), (4, False), (2, True)])
def test_sharded_condensation_matches_whole_mesh(world, viscous):
    mesh, st, prm = _case(viscous)
    bh_all, Ahats = oracle.condense_mesh(prm, mesh, st, want_Ahat=True)
    x = I.random_direction(st.vhat.shape, 91, 1.0)
    y_all = (oracle.assemble_Ahat(mesh, Ahats) @ x.ravel()).reshape(x.shape)
    _, _, rh_all = oracle.residual_mesh(prm, mesh, st)
    res = _run(world, viscous)
    assert sorted(res) == list(range(world))
    seen = np.zeros(mesh.n_global_faces, dtype=int)
    for rank, (gf, bh, y, d, peers, rh) in res.items():
        scale_b, scale_y, scale_r = np.abs(bh_all).max(), np.abs(y_all).max(), np.abs(rh_all).max()
        assert np.abs(bh - bh_all[gf]).max() <= 1e-12 * scale_b, rank
        assert np.abs(y - y_all[gf]).max() <= 1e-12 * scale_y, rank
        assert np.abs(rh - rh_all[gf]).max() <= 1e-12 * scale_r, rank
        assert d == pytest.approx(float(np.sum(x * y_all)), rel=1e-12)
        assert peers, "every slab of a periodic mesh borders another rank"
        seen[gf] += 1
    assert (seen >= 1).all()


def test_partition_covers_every_element_once():
    mesh = I.periodic_mesh((5, 2, 3), 1, 1)
    for world in (1, 2, 3, 5):
        parts = SH.partition(mesh, world)
        allk = np.sort(np.concatenate(parts))
        assert (allk == np.arange(mesh.nK)).all()
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 2 * 3      # one x-position of 2 x 3 elements at most
    with pytest.raises(ValueError):
        SH.partition(mesh, 6)


def test_single_rank_has_no_peers_and_sums_nothing():
    mesh = I.periodic_mesh((2, 1, 1), 1, 1)
    sh = SH.Shard(mesh, SH.partition(mesh, 1), 0)
    assert sh.peers == {} and sh.owned.all()
    t = torch.ones(mesh.n_global_faces, 5, mesh.n2)
    assert sh.sum_shared(t) is t and float(t.sum()) == t.numel()
