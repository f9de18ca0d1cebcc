"""DIRK(3,3) time steps (Sec. 5.3, eqs. C241, C242) through the C-ABI: the
stages' Newton iterations (condense, GMRES, recover) with the known stages
as an R_V source, against the oracle's DIRK step (monolithic Newton) on the
same seeded state."""
import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("viscous,prec", [(False, 0), (False, 4), (True, 0)])
def test_dirk_step_matches_oracle(viscous, prec):
    from paper_2507_22195_gb300 import mehdg as M
    mesh = I.periodic_mesh((2, 1, 1) if viscous else 2, 1 if not viscous else 2, 1)
    st = I.make_state(mesh, "tgv", 2e-2, 5, 6, viscous=viscous, M0=0.3)
    kw = dict(flux=1, Mach=0.3, Re=100.0, viscous=1) if viscous else dict(flux=1, Mach=0.3)
    dt = 0.2
    ref, stages, its_o = oracle.dirk_step(kw, mesh, st, dt)
    ref2, _, _ = oracle.dirk_step(kw, mesh, ref, dt)
    d = torch.device("cuda:0")
    v, vh = torch.tensor(st.v, device=d), torch.tensor(st.vhat, device=d)
    q = torch.tensor(st.q, device=d) if viscous else None
    ctx = M.Context(mesh, prec=prec, **kw)
    n = st.vhat.size
    for step, r in enumerate((ref, ref2)):
        its, rn = M.mehdg_dirk_step(ctx.ctx, v, vh, q, dt, newton_tol=1e-11, newton_max=12, lin_rtol=1e-13,
                                    restart=n, max_iter=4 * n)
        torch.cuda.synchronize()
        assert (rn <= 1e-11).all(), rn
        for a, b in ((v, r.v), (vh, r.vhat)) + (((q, r.q),) if viscous else ()):
            a = a.cpu().numpy()
            assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max(), (step, np.abs(a - b).max() / np.abs(b).max())
    ctx.close()
