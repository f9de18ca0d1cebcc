"""The adjoint condensed solve (transposed eqs. R2-R5, Euler) through the
C-ABI: the adjoint identity <A-hat^T x, z> = <x, A-hat z> against the forward
condensed operator, A-hat^T x against the oracle's assembled sum of A-hat^K,
and condense_adjoint -> GMRES on A-hat^T -> recover_adjoint against the
oracle's monolithic transposed Newton system solved by GEPP."""
import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(name):
    if name == "tgv_p1m1":
        mesh = I.periodic_mesh(2, 1, 1)
        st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
        return mesh, st, dict(Mach=0.3)
    mesh = I.periodic_mesh(2, 2, 1, 0.0, 10.0)
    st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
    return mesh, st, dict(Mach=0.1)


def _dev(a):
    return torch.tensor(a, device="cuda:0")


@pytest.mark.parametrize("name", ["tgv_p1m1", "vortex_p2m1"])
@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("flux", [1, 2])
def test_adjoint_condensed_solve_matches_oracle(name, prec, flux):
    from paper_2507_22195_gb300 import mehdg as M
    mesh, st, kw = _case(name)
    ctx = M.Context(mesh, flux=flux, prec=prec, **kw)
    ctx.set_state(_dev(st.v), _dev(st.vhat), None, _dev(st.vstar))
    ctx.condense()
    x = I.random_direction(st.vhat.shape, 83, 1.0)
    z = I.random_direction(st.vhat.shape, 84, 1.0)
    y_a = torch.empty_like(_dev(x))
    M.mehdg_apply_condensed_adjoint(ctx.ctx, _dev(x), y_a)
    Az = ctx.apply(_dev(z))
    torch.cuda.synchronize()
    lhs, rhs = float((y_a * _dev(z)).sum()), float((_dev(x) * Az).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    prm = oracle.params(flux=flux, **kw)
    bh, Ahats = oracle.condense_mesh(prm, mesh, st, want_Ahat=True)
    A = oracle.assemble_Ahat(mesh, Ahats)
    y_o = (A.T @ x.ravel()).reshape(x.shape)
    tol = 1e-10 if prec == 0 else 1e-8
    ya = y_a.cpu().numpy()
    assert np.linalg.norm(ya - y_o) <= tol * np.linalg.norm(y_o)
    # J^T lam = g by condensation, GMRES on A-hat^T and recovery
    gV = I.random_direction(st.v.shape, 85, 1.0)
    gH = I.random_direction(st.vhat.shape, 86, 1.0)
    b_a = torch.empty_like(_dev(gH))
    M.mehdg_condense_adjoint(ctx.ctx, _dev(gV), _dev(gH), b_a)
    lamH = torch.zeros_like(b_a)
    n = b_a.numel()
    it, res = M.mehdg_solve_condensed_adjoint(ctx.ctx, b_a, lamH, rtol=1e-13, restart=n, max_iter=2 * n)
    lamV = torch.empty_like(_dev(gV))
    M.mehdg_recover_adjoint(ctx.ctx, _dev(gV), lamH, lamV)
    torch.cuda.synchronize()
    stat, iters = ctx.status()
    assert (stat == 0).all(), (stat, iters)
    lv_o, lh_o = oracle.adjoint_solve(prm, mesh, st, gV, gH)
    e = (np.linalg.norm(lamV.cpu().numpy() - lv_o) / np.linalg.norm(lv_o),
         np.linalg.norm(lamH.cpu().numpy() - lh_o) / np.linalg.norm(lh_o))
    assert max(e) < (1e-9 if prec == 0 else 1e-8), (e, it, res)
    ctx.close()
