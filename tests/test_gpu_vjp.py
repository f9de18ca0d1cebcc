"""VJP of the residual (eq. s32, Euler) through the C-ABI: against the oracle's
transposed complex-step Jacobian blocks, against central differences of the
GPU residual, and through torch.autograd."""
import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def M():
    from paper_2507_22195_gb300 import mehdg
    return mehdg


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else a
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(x):
    return torch.tensor(x, device="cuda:0")


def case(name):
    if name == "vortex_p2m1":
        mesh = I.periodic_mesh(2, 2, 1, 0.0, 10.0)
        return mesh, I.make_state(mesh, "vortex", 1e-3, 22195, 22196, period=10.0), 0.1
    if name == "tgv_p2m2":
        mesh = I.periodic_mesh((2, 1, 1), 2, 2)
        return mesh, I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3), 0.3
    raise ValueError(name)


def cotangents(mesh, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal((mesh.nK, 5, mesh.Nn)),
            g.standard_normal((mesh.n_global_faces, 5, mesh.n2)))


@pytest.mark.parametrize("name", ["vortex_p2m1", "tgv_p2m2"])
@pytest.mark.parametrize("flux", [0, 1, 2])
def test_residual_vjp_matches_oracle(name, flux):
    mesh, st, mach = case(name)
    ctx = M().Context(mesh, flux=flux, prec=M().MEHDG_FP64, Mach=mach)
    ctx.set_state(dev(st.v), dev(st.vhat), None, dev(st.vstar))
    lv, lh = cotangents(mesh, 31 + flux)
    gv, gh = ctx.residual_vjp(dev(lv), dev(lh))
    torch.cuda.synchronize()
    stat, _ = ctx.status()
    assert (stat == 0).all()
    gv_o, gh_o = oracle.residual_vjp_mesh(oracle.params(flux=flux, Mach=mach), mesh, st, lv, lh)
    assert rel(gv, gv_o) < 1e-11 and rel(gh, gh_o) < 1e-11, (rel(gv, gv_o), rel(gh, gh_o))
    ctx.close()


def test_residual_vjp_central_differences():
    """<lam, R(w + e d) - R(w - e d)> / 2e = <VJP(lam), d> on 20 seeded
    directions (ES flux: KEPES has a derivative that is unbounded where the two
    pressures meet, which central differences resolve only as e -> 0)"""
    mesh, st, mach = case("tgv_p2m2")
    ctx = M().Context(mesh, flux=1, prec=M().MEHDG_FP64, Mach=mach)
    lv, lh = cotangents(mesh, 7)
    ctx.set_state(dev(st.v), dev(st.vhat), None, dev(st.vstar))
    gv, gh = ctx.residual_vjp(dev(lv), dev(lh))
    gv, gh = gv.cpu().numpy(), gh.cpu().numpy()
    eps = 1e-6
    worst = 0.0
    for s in range(20):
        dv = I.random_direction(st.v.shape, 1000 + s, 1.0)
        dh = I.random_direction(st.vhat.shape, 2000 + s, 1.0)
        val = []
        for sgn in (1.0, -1.0):
            ctx.set_state(dev(st.v + sgn * eps * dv), dev(st.vhat + sgn * eps * dh), None, dev(st.vstar))
            RV, _, RH = ctx.residual()
            val.append(float((RV.cpu().numpy() * lv).sum() + (RH.cpu().numpy() * lh).sum()))
        fd = (val[0] - val[1]) / (2 * eps)
        ad = float((gv * dv).sum() + (gh * dh).sum())
        worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-12))
    assert worst < 1e-6, worst
    ctx.close()


def test_autograd_function_matches_vjp():
    mesh, st, mach = case("vortex_p2m1")
    ctx = M().Context(mesh, flux=1, prec=M().MEHDG_FP64, Mach=mach)
    Residual = M().residual_function()
    v = dev(st.v).requires_grad_(True)
    vh = dev(st.vhat).requires_grad_(True)
    RV, RH = Residual.apply(v, vh, ctx, dev(st.vstar))
    loss = (RV * RV).sum() + (RH * RH).sum()
    gv, gh = torch.autograd.grad(loss, (v, vh))
    ctx.set_state(dev(st.v), dev(st.vhat), None, dev(st.vstar))
    gv2, gh2 = ctx.residual_vjp(2.0 * RV.detach(), 2.0 * RH.detach())
    assert rel(gv, gv2.cpu().numpy()) < 1e-13 and rel(gh, gh2.cpu().numpy()) < 1e-13
    ctx.close()


def test_residual_vjp_rejects_viscous():
    mesh = I.periodic_mesh(2, 2, 1)
    st = I.make_state(mesh, "tgv", 1e-3, 1, 2, viscous=True, M0=0.1)
    ctx = M().Context(mesh, flux=1, prec=M().MEHDG_FP64, viscous=1, Mach=0.1)
    ctx.set_state(dev(st.v), dev(st.vhat), dev(st.q), dev(st.vstar))
    lv, lh = cotangents(mesh, 1)
    with pytest.raises(M().MehdgError):
        ctx.residual_vjp(dev(lv), dev(lh))
    ctx.close()
