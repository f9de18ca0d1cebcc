"""The condensation replayed from one CUDA graph (mehdg_condense_graph)
against the direct calls: a uniform mesh (split BF16 and FP64), a changed
state in the same arrays, and a resident batch of uneven p, m (every group in
one graph); the factors left by a replay serve recover.  The Jacobian is
accumulated with atomics, so two condensations (direct or replayed) agree to
the refinement's accuracy, not bit for bit: 1e-9 relative to the largest
entry."""
import numpy as np
import pytest

from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.mark.parametrize("prec", [4, 0])
def test_graph_condense_equals_direct_uniform(prec):
    from paper_2507_22195_gb300 import mehdg as M
    mesh = I.periodic_mesh(2, 2, 2, 0.0, 10.0)
    st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
    d = torch.device("cuda:0")
    v, vh, vs = (torch.tensor(a, device=d) for a in (st.v, st.vhat, st.vstar))
    ctx = M.Context(mesh, flux=2, prec=prec, Mach=0.1)
    ctx.set_state(v, vh, None, vs)
    b_dir = ctx.condense().clone()
    s_dir, it_dir = ctx.status()
    bh = torch.empty_like(b_dir)
    for _ in range(3):
        M.mehdg_condense_graph(ctx.ctx, bh)
        torch.cuda.synchronize()
        assert torch.allclose(bh, b_dir, rtol=0, atol=TOL * float(b_dir.abs().max()))
    s_g, it_g = ctx.status()
    assert (s_g == 0).all() and (it_g == it_dir).all()
    # new values in the same arrays: the graph reads them
    v.add_(torch.tensor(I.random_direction(st.v.shape, 5, 1e-4), device=d))
    ctx.set_state(v, vh, None, vs)
    M.mehdg_condense_graph(ctx.ctx, bh)
    dvh = torch.tensor(I.random_direction(st.vhat.shape, 6, 1e-3), device=d)
    dV_g = ctx.recover(dvh)
    torch.cuda.synchronize()
    b_new = ctx.condense().clone()
    dV_dir = ctx.recover(dvh)
    torch.cuda.synchronize()
    assert torch.allclose(bh, b_new, rtol=0, atol=TOL * float(b_new.abs().max()))
    assert torch.allclose(dV_g, dV_dir, rtol=0, atol=TOL * float(dV_dir.abs().max()))
    ctx.close()


def test_graph_condense_resident_batch_and_streamed_refusal(monkeypatch):
    from paper_2507_22195_gb300 import mehdg as M
    mesh = I.uneven_batch(0, 22199, specs=[(1, 2), (2, 2), (3, 2), (2, 3), (1, 4), (2, 2), (3, 1)])
    st = I.make_uneven_state(mesh, 1e-2, 22200, 22201, 22202)
    d = torch.device("cuda:0")
    w = [torch.tensor(a, device=d) for a in (st.v, st.vhat)]
    ctx = M.BatchContext(mesh, prec=4, flux=1, Mach=0.1)
    ctx.set_state(w[0], w[1], None, torch.tensor(st.vstar, device=d))
    b_dir = ctx.condense().clone()
    bh = torch.empty_like(b_dir)
    M.mehdg_condense_graph(ctx.ctx, bh)
    M.mehdg_condense_graph(ctx.ctx, bh)
    dvh = torch.tensor(I.random_direction(st.vhat.shape, 7, 1e-3), device=d)
    dV_g = ctx.recover(dvh)
    torch.cuda.synchronize()
    assert torch.allclose(bh, b_dir, rtol=0, atol=TOL * float(b_dir.abs().max()))
    ctx.condense()
    dV_dir = ctx.recover(dvh)
    torch.cuda.synchronize()
    assert torch.allclose(dV_g, dV_dir, rtol=0, atol=TOL * float(dV_dir.abs().max()))
    ctx.close()
    per = max(g["bytes_per_element"] for g in M.BatchContext(mesh, prec=4, flux=1, Mach=0.1).report()["groups"])
    monkeypatch.setenv("MEHDG_BATCH_BUDGET_MB", str(1.05 * per / 1048576.0))
    ctx = M.BatchContext(mesh, prec=4, flux=1, Mach=0.1)
    ctx.set_state(w[0], w[1], None, torch.tensor(st.vstar, device=d))
    with pytest.raises(M.MehdgError, match="EINVAL"):
        M.mehdg_condense_graph(ctx.ctx, bh)
    ctx.close()
