"""Gradients through pseudo-time Newton steps (Sec. 6.1) with the adjoint
condensed solve, through the C-ABI:
  * a tiny periodic mesh: the cotangent of the initial state against the
    oracle's (monolithic transposed solves, complex-step Jacobians) and
    against central differences of the forward map on 20 seeded directions;
  * the adjoint workload (4^3 macro-elements of 2^3 micro-elements, p = 2,
    inviscid TGV at Mach 0.1, 5 steps of size 1): the gradient of the total
    kinetic energy after the steps with respect to the initial nodal velocity
    field, against central differences (step 1e-6) on seeded directions.
The kinetic energy and the map from nodal velocities to the initial entropy
variables are the user's objective and parametrisation, written here with
torch autograd; every Newton, condensation and adjoint step runs in the
library."""
import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
G = 1.4


def _dev(a):
    return torch.tensor(a, device="cuda:0")


def _forward(M, ctx, v0, vh0, nsteps, tau, n_trace, rtol):
    v, vh = v0.clone(), vh0.clone()
    M.mehdg_pseudo_time_newton(ctx.ctx, v, vh, None, nsteps, tau, tau, lin_rtol=rtol, restart=min(n_trace, 200),
                               max_iter=8000)
    return v, vh


@pytest.mark.parametrize("prec", [0, 4])
def test_newton_vjp_tiny_mesh_matches_oracle_and_differences(prec):
    from paper_2507_22195_gb300 import mehdg as M
    mesh = I.periodic_mesh(2, 1, 1)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
    kw = dict(flux=1, Mach=0.3)
    nsteps, tau = 5, 1.0
    gbv = I.random_direction(st.v.shape, 90, 1.0)
    gbh = I.random_direction(st.vhat.shape, 91, 1.0)
    ctx = M.Context(mesh, prec=prec, **kw)
    v, vh = _dev(st.v), _dev(st.vhat)
    g0v, g0h = torch.empty_like(v), torch.empty_like(vh)
    n = st.vhat.size
    M.mehdg_pseudo_time_newton_vjp(ctx.ctx, v, vh, nsteps, tau, _dev(gbv), _dev(gbh), g0v, g0h, lin_rtol=1e-13,
                                   restart=n, max_iter=2 * n)
    torch.cuda.synchronize()
    gv_o, gh_o, fin = oracle.newton_vjp(kw, mesh, st, nsteps, tau, gbv, gbh)
    assert np.abs(v.cpu().numpy() - fin.v).max() <= 1e-9 * np.abs(fin.v).max()
    g = np.concatenate([g0v.cpu().numpy().ravel(), g0h.cpu().numpy().ravel()])
    g_o = np.concatenate([gv_o.ravel(), gh_o.ravel()])
    assert np.linalg.norm(g - g_o) <= 1e-7 * np.linalg.norm(g_o), np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    if prec != 0:
        ctx.close()
        return
    # central differences of L(s0) = <gbar, s_5(s0)> on 20 seeded directions
    v0, vh0 = _dev(st.v), _dev(st.vhat)
    eps = 1e-6
    for i in range(20):
        dv = _dev(I.random_direction(st.v.shape, 200 + i, 1.0))
        dh = _dev(I.random_direction(st.vhat.shape, 300 + i, 1.0))
        L = []
        for sgn in (1.0, -1.0):
            a, b = _forward(M, ctx, v0 + sgn * eps * dv, vh0 + sgn * eps * dh, nsteps, tau, n, 1e-14)
            L.append(float((a * _dev(gbv)).sum() + (b * _dev(gbh)).sum()))
        fd = (L[0] - L[1]) / (2 * eps)
        ad = float((g0v * dv).sum() + (g0h * dh).sum())
        assert abs(fd - ad) <= 2e-5 * max(abs(ad), 1e-3 * float(torch.linalg.norm(g0v))), (i, fd, ad)
    ctx.close()


# ---------------------------------------------------------------- the adjoint workload
def _prim(v):
    """(rho, V, P) from entropy variables [K, 5, N] (inverse of eq. s222)"""
    beta = -v[:, 4]
    V = v[:, 1:4] / beta[:, None]
    s = G - (G - 1) * (v[:, 0] + beta * (V * V).sum(1) / 2)
    rho = (beta * torch.exp(s)) ** (1 / (1 - G))
    return rho, V, rho / beta


def _v_of(rho, V, P):
    """eq. s222 on [K, N] / [K, 3, N] arrays"""
    s = torch.log(P / rho ** G)
    beta = rho / P
    return torch.stack([(G - s) / (G - 1) - beta * (V * V).sum(1) / 2, beta * V[:, 0], beta * V[:, 1],
                        beta * V[:, 2], -beta], 1)


def test_kinetic_energy_gradient_adjoint_workload():
    from paper_2507_22195_gb300 import mehdg as M
    mesh = I.periodic_mesh(4, 2, 2)
    nK, Nn, n = mesh.nK, mesh.Nn, mesh.n
    nsteps, tau = 5, 1.0
    dev = torch.device("cuda:0")
    # TGV (Mach 0.1) at the nodes: density and pressure fixed, velocity U the variable
    rho0 = np.zeros((nK, Nn)); P0 = np.zeros((nK, Nn)); U0 = np.zeros((nK, 3, Nn))
    for K in range(nK):
        X, Y, Z = I.node_coords(mesh, K)
        r, V, P = I.tgv_prim(X, Y, Z, M0=0.1)
        rho0[K], P0[K], U0[K] = r, P, np.stack(V)
    fi = I.face_node_index(mesh)
    sides = [[] for _ in range(mesh.n_global_faces)]
    for K in range(nK):
        for f in range(6):
            sides[mesh.face_gid[K, f]].append((K, f))
    sK = torch.tensor([[s[0][0], s[1][0]] for s in sides], device=dev)
    sF = torch.tensor([[s[0][1], s[1][1]] for s in sides], device=dev)
    fidx = torch.tensor(fi, device=dev)
    rho_t, P_t = _dev(rho0), _dev(P0)

    def initial(U):
        """(v0, vhat0): eq. s222 at the nodes; a trace node takes the mean of
        the two adjacent elements' nodal values"""
        v0 = _v_of(rho_t, U, P_t)
        def face(x):       # x [K, c, N] -> [G, c, n^2]
            xa = torch.stack([x[sK[g, 0]][..., fidx[sF[g, 0]]] for g in range(len(sides))])
            xb = torch.stack([x[sK[g, 1]][..., fidx[sF[g, 1]]] for g in range(len(sides))])
            return 0.5 * (xa + xb)
        vh0 = _v_of(face(rho_t[:, None])[:, 0], face(U), face(P_t[:, None])[:, 0])
        return v0.contiguous(), vh0.contiguous()

    # nodal quadrature of the kinetic energy: tensor GLL weights of every micro-element, assembled
    w1 = np.zeros(n)
    wl = I.gll_weights(mesh.p)
    for e in range(mesh.m):
        w1[e * mesh.p:e * mesh.p + mesh.p + 1] += wl
    h = (mesh.boxes[0, 3] - mesh.boxes[0, 0]) / mesh.m / 2
    wq = _dev((np.einsum("k,j,i->kji", w1, w1, w1).ravel() * h ** 3))

    def ke(v):
        rho, V, _ = _prim(v)
        return (0.5 * rho * (V * V).sum(1) * wq).sum()

    ctx = M.Context(mesh, flux=1, prec=0, Mach=0.1)
    nt = mesh.n_global_faces * 5 * mesh.n2
    U = _dev(U0).requires_grad_(True)
    v0, vh0 = initial(U)
    v, vh = v0.detach().clone(), vh0.detach().clone()
    g0v, g0h = torch.empty_like(v), torch.empty_like(vh)
    # the final state (forward alone), the objective's cotangent there, then the VJP
    vtmp, vhtmp = _forward(M, ctx, v, vh, nsteps, tau, nt, 1e-12)
    vt = vtmp.clone().requires_grad_(True)
    E = ke(vt)
    gbar_v, = torch.autograd.grad(E, vt)
    M.mehdg_pseudo_time_newton_vjp(ctx.ctx, v, vh, nsteps, tau, gbar_v.contiguous(), None, g0v, g0h,
                                   lin_rtol=1e-12, restart=200, max_iter=8000)
    torch.cuda.synchronize()
    assert torch.allclose(v, vtmp, rtol=0, atol=1e-10)
    gU, = torch.autograd.grad((v0 * g0v).sum() + (vh0 * g0h).sum(), U)
    # central differences of KE(s_5(U)) on seeded directions
    eps = 1e-6
    for i in range(2):
        d = _dev(I.random_direction(U0.shape, 400 + i, 1.0))
        L = []
        for sgn in (1.0, -1.0):
            with torch.no_grad():
                a0, b0 = initial(U + sgn * eps * d)
            a, b = _forward(M, ctx, a0, b0, nsteps, tau, nt, 1e-12)
            L.append(float(ke(a)))
        fd = (L[0] - L[1]) / (2 * eps)
        ad = float((gU * d).sum())
        assert abs(fd - ad) <= 1e-4 * abs(ad), (i, fd, ad)
    ctx.close()
