"""The nonlinear loop (Sec. 6.1): pseudo-transient Newton steps through the
C-ABI (condense, GMRES trace solve, recover, update) against the oracle's
monolithic Newton iterates on the same seeded state, step for step: the
residual norm before and after every step, the pseudo-time steps chosen from
them, and the final state."""
import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(viscous):
    if viscous:
        mesh = I.periodic_mesh((2, 1, 1), 2, 1)
        st = I.make_state(mesh, "tgv", 1e-2, 5, 6, viscous=True, M0=0.3)
        return mesh, st, dict(flux=1, Mach=0.3, Re=100.0, viscous=1)
    mesh = I.periodic_mesh(2, 2, 1, 0.0, 10.0)          # the 2^3 vortex, p = 2
    st = I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0)
    return mesh, st, dict(flux=1, Mach=0.1)


@pytest.mark.parametrize("viscous,prec", [(False, 0), (False, 4), (True, 0)])
def test_pseudo_time_newton_matches_oracle_iterates(viscous, prec):
    from paper_2507_22195_gb300 import mehdg as M
    mesh, st, kw = _case(viscous)
    nsteps, tau0 = (6, 1.0) if viscous else (8, 1.0)
    st_o, norms_o, taus_o = oracle.pseudo_time_newton(kw, mesh, st, nsteps, tau0, 1e8)
    dev = torch.device("cuda:0")
    v = torch.tensor(st.v, device=dev)
    vh = torch.tensor(st.vhat, device=dev)
    q = torch.tensor(st.q, device=dev) if viscous else None
    ctx = M.Context(mesh, prec=prec, **kw)
    ctx.set_state(v, vh, q, v.clone())
    n = st.vhat.size
    # on the inviscid vortex GMRES without a preconditioner stalls near 1e-11 once tau reaches 1e7
    # (the trace system tends to the steady one): its linear solves stop at 1e-10
    rn, taus, its = M.mehdg_pseudo_time_newton(ctx.ctx, v, vh, q, nsteps, tau0, 1e8,
                                               lin_rtol=1e-12 if viscous else 1e-10, restart=n, max_iter=4 * n)
    torch.cuda.synchronize()
    # the residual falls (a converging Newton loop) ...
    assert rn[-1] < 1e-3 * rn[0], rn
    # ... along the oracle's iterates: norms while above round-off, and the steps
    big = np.array(norms_o) > 1e-7 * norms_o[0]
    assert np.allclose(rn[big], np.array(norms_o)[big], rtol=1e-6), (rn, norms_o)
    assert np.allclose(taus, taus_o, rtol=1e-6), (taus, taus_o)
    tol = 1e-7
    for a, b in ((v, st_o.v), (vh, st_o.vhat)) + (((q, st_o.q),) if viscous else ()):
        a = a.cpu().numpy()
        assert np.abs(a - b).max() <= tol * np.abs(b).max(), np.abs(a - b).max() / np.abs(b).max()
    ctx.close()
