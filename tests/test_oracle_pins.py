"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties a part of the oracle to something other than itself: a closed
form, an identity the paper proves, a library routine for a special case, a
number the paper prints, or a brute-force solve.  A plausible mistake in the
oracle (a dropped term, a sign, a transposed operand) fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2507_22195_gb300 import inputs as I

G = 1.4
HERE = os.path.dirname(os.path.abspath(__file__))


def rand_state(rng, M=0.3):
    """random physical entropy-variable state"""
    rho = rng.uniform(0.5, 2.0)
    P = rng.uniform(0.4, 2.0)
    V = rng.uniform(-M, M, 3)
    return I.entropy_vars(np.array(rho), [np.array(c) for c in V], np.array(P)).astype(float)


def normals():
    out = []
    for d in range(3):
        for s in (-1.0, 1.0):
            n = np.zeros(3); n[d] = s; out.append(n)
    return out


# ---------------------------------------------------------------- tables
@pytest.mark.parametrize("npt", [2, 3, 4, 5, 6])
def test_gauss_matches_library(npt):
    x, w = oracle.gauss(npt)
    xr, wr = np.polynomial.legendre.leggauss(npt)
    assert np.allclose(x, xr, atol=1e-15) and np.allclose(w, wr, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_are_lobatto_points(p):
    x = oracle.gll(p)
    assert x[0] == -1.0 and x[-1] == 1.0
    # interior nodes are the roots of P_p'
    dP = np.polynomial.legendre.Legendre.basis(p).deriv()
    assert np.allclose(dP(x[1:-1]), 0.0, atol=1e-14)


# ---------------------------------------------------------------- thermodynamics
def test_u_of_v_inverts_eq_s222():
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho, P = rng.uniform(0.3, 3), rng.uniform(0.3, 3)
        V = rng.uniform(-1, 1, 3)
        v = I.entropy_vars(np.array(rho), [np.array(c) for c in V], np.array(P)).astype(float)
        u = oracle.u_of_v(v)
        E = P / (G - 1) + 0.5 * rho * V @ V
        assert np.allclose(u, [rho, *(rho * V), E], rtol=1e-13)


def _H_of_u(u):
    """entropy function H = -rho s/(gamma-1), s = ln(P/rho^gamma) (eq. en)"""
    rho = u[0]
    P = (G - 1) * (u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / rho)
    s = np.log(P / rho ** G)
    return -rho * s / (G - 1)


def test_entropy_variables_are_dH_du():
    """v = dH/du (Sec. 2.2), derivative by complex step in the test"""
    rng = np.random.default_rng(2)
    for _ in range(10):
        v = rand_state(rng)
        u = oracle.u_of_v(v)
        g = np.zeros(5)
        for l in range(5):
            z = u.astype(complex); z[l] += 1e-30j
            g[l] = _H_of_u(z).imag / 1e-30
        assert np.allclose(g, v, rtol=1e-12, atol=1e-12)


def test_A0_closed_form_is_du_dv_and_spd():
    rng = np.random.default_rng(3)
    for _ in range(10):
        v = rand_state(rng)
        A, J = oracle.A0(v), oracle.dudv_cs(v)
        assert np.allclose(A, J, rtol=1e-13, atol=1e-14)
        assert np.allclose(A, A.T)
        assert np.linalg.eigvalsh(A).min() > 0


def test_entropy_potential_eq_poen():
    """Psi_n = F_n^T v - calF_n = rho V.n (eq. poen) with the entropy flux
    calF = H V = -rho s V/(gamma-1), the flux paired with H of eq. en (the
    printed calF = -rho s V lacks the 1/(gamma-1) of H)."""
    rng = np.random.default_rng(4)
    for _ in range(10):
        v = rand_state(rng)
        rho, V, P = oracle.prim_of_v(v)
        s = math.log(P / rho ** G)
        for n in normals():
            Fn = oracle.flux_phys(v, n)
            assert abs(Fn @ v - (-rho * s * V @ n / (G - 1)) - rho * V @ n) < 1e-13


def test_logmean():
    for a, b in [(1.0, 2.0), (0.3, 7.0), (1.0, 1.0 + 1e-3), (2.0, 2.0)]:
        ref = a if a == b else (b - a) / math.log(b / a)
        assert abs(oracle.logmean(a, b) - ref) <= 1e-15 * ref + (1e-12 if abs(a - b) < 1e-2 else 0)
    # continuity across the series/logarithm switch (u = 1e-4 <=> zeta ~ 1.0202)
    z = (1 + 1e-2) / (1 - 1e-2)
    lo, hi = oracle.logmean(1.0, z * (1 - 1e-12)), oracle.logmean(1.0, z * (1 + 1e-12))
    assert abs(hi - lo) < 1e-11


# ---------------------------------------------------------------- fluxes
@pytest.mark.parametrize("kind", [oracle.EC, oracle.ES, oracle.KEPES])
def test_flux_consistency(kind):
    """F-hat(a, a) = F(a).n"""
    rng = np.random.default_rng(5)
    for _ in range(5):
        v = rand_state(rng)
        for n in normals():
            assert np.allclose(oracle.flux_num(kind, v, v, n), oracle.flux_phys(v, n), rtol=1e-13, atol=1e-14)


def test_ec_symmetric_and_kep_structure():
    rng = np.random.default_rng(6)
    for _ in range(10):
        a, b = rand_state(rng), rand_state(rng)
        ra, Va, Pa = oracle.prim_of_v(a)
        rb, Vb, Pb = oracle.prim_of_v(b)
        for n in normals():
            F1, F2 = oracle.flux_num(oracle.EC, a, b, n), oracle.flux_num(oracle.EC, b, a, n)
            assert np.allclose(F1, F2, rtol=1e-14, atol=1e-15)
            Vbar = 0.5 * (Va + Vb)
            Pbar = 0.5 * (ra + rb) / (0.5 * (ra / Pa + rb / Pb))
            # momentum flux = Vbar * mass flux + Pbar n (eq. KEP)
            assert np.allclose(F1[1:4], Vbar * F1[0] + Pbar * n, rtol=1e-13, atol=1e-15)


def _psi_n(v, n):
    rho, V, P = oracle.prim_of_v(v)
    return rho * V @ n


def test_ec_condition_thm51():
    """[[v]].F-bar - [[Psi_n]] = 0 (Thm. 5.1, eq. EC_1)"""
    rng = np.random.default_rng(7)
    for _ in range(50):
        v, vh = rand_state(rng), rand_state(rng)
        for n in normals():
            F = oracle.flux_num(oracle.EC, vh, v, n)
            r = (vh - v) @ F - (_psi_n(vh, n) - _psi_n(v, n))
            assert abs(r) < 1e-13 * (1 + np.abs(vh - v).sum() * np.abs(F).sum())


def test_kepes_entropy_production_thm52():
    """[[v]].F-hat - [[Psi_n]] = -1/2 [[v]]^T R|L|T R^T [[v]] <= 0 (Thm. 5.2)"""
    rng = np.random.default_rng(8)
    for _ in range(50):
        v, vh = rand_state(rng), rand_state(rng)
        for n in normals():
            F = oracle.flux_num(oracle.KEPES, vh, v, n)
            R, L, T = oracle.kepes_parts(vh, v, n)
            dv = vh - v
            quad = dv @ R @ np.diag(L * T) @ R.T @ dv
            r = dv @ F - (_psi_n(vh, n) - _psi_n(v, n))
            assert quad >= 0
            assert abs(r + 0.5 * quad) < 1e-12 * (1 + quad + np.abs(dv).sum() * np.abs(F).sum())


def test_es_flux_small_jumps_dissipate():
    """ES flux (eq. Flux_En_Inv): entropy production <= 0 for near states"""
    rng = np.random.default_rng(9)
    for _ in range(50):
        v = rand_state(rng)
        vh = v + rng.uniform(-1e-3, 1e-3, 5)
        for n in normals():
            F = oracle.flux_num(oracle.ES, vh, v, n)
            r = (vh - v) @ F - (_psi_n(vh, n) - _psi_n(v, n))
            assert r <= 1e-15


def test_barth_scaling_at_equal_states():
    """R T R^T = A0 at equal states (eq. KEPES4)"""
    rng = np.random.default_rng(10)
    for _ in range(10):
        v = rand_state(rng)
        for n in normals():
            R, L, T = oracle.kepes_parts(v, v, n)
            assert np.allclose(R @ np.diag(T) @ R.T, oracle.A0(v), rtol=1e-12, atol=1e-13)


def _Fn_of_u(u, n, g=G):
    """normal inviscid flux (eq. C5) written in conservative variables"""
    rho, m, E = u[0], u[1:4], u[4]
    V = m / rho
    P = (g - 1.0) * (E - 0.5 * rho * V @ V)
    vn = V @ n
    return np.concatenate([[rho * vn], rho * V * vn + P * n, [(E + P) * vn]])


def _jac_fd(f, x, h=1e-6):
    """central-difference Jacobian, columns d f / d x_j"""
    cols = []
    for j in range(len(x)):
        e = np.zeros(len(x)); e[j] = h * max(1.0, abs(x[j]))
        cols.append((f(x + e) - f(x - e)) / (2 * e[j]))
    return np.stack(cols, axis=1)


def _An_eig(v, n):
    """A_n = d(F.n)/du at the state v, from the conservative-variable flux
    above, and its eigenvalues/eigenvectors sorted by eigenvalue (numpy)"""
    u = oracle.u_of_v(v)
    An = _jac_fd(lambda uu: _Fn_of_u(uu, n), u, 1e-7)
    w, X = np.linalg.eig(An)
    o = np.argsort(w.real)
    return An, w.real[o], X.real[:, o]


def _general_normals():
    rng = np.random.default_rng(21)
    out = normals()
    for _ in range(3):
        n = rng.normal(size=3); out.append(n / np.linalg.norm(n))
    return out


def test_kepes_eigenvectors_order_and_equal_state_dissipation():
    """KEPES at equal states (eqs. KEPES3-KEPES5): the columns of R-bar are
    right eigenvectors of the normal flux Jacobian A_n = d(F.n)/du with the
    eigenvalues v_n - c, v_n, v_n, v_n, v_n + c in that order (A_n from the
    conservative flux, its eigenvalues from a numerical eigendecomposition),
    and |Lambda-bar| (theta = 0) holds the reading's |v_n| + c, |v_n|, |v_n|,
    |v_n|, |v_n| + c, with c the spectral gap of A_n; the flux's dissipation
    F_KEPES - F_EC at a small pressure-preserving jump equals
    -1/2 R |Lambda| T R^T [[v]] with these parts."""
    rng = np.random.default_rng(22)
    for _ in range(8):
        v = rand_state(rng)
        rho, V, P = oracle.prim_of_v(v)
        for n in _general_normals():
            An, w, X = _An_eig(v, n)
            vn = V @ n
            c = 0.5 * (w[4] - w[0])                 # spectral gap of A_n
            assert np.allclose(w, [vn - c, vn, vn, vn, vn + c], atol=1e-8)
            assert abs(c - math.sqrt(G * P / rho)) < 1e-8
            R, L, T = oracle.kepes_parts(v, v, n)
            lam = np.array([vn - c, vn, vn, vn, vn + c])
            assert np.allclose(An @ R, R @ np.diag(lam), atol=1e-7 * np.abs(R).max())
            assert np.allclose(L, [abs(vn) + c, abs(vn), abs(vn), abs(vn), abs(vn) + c], rtol=1e-12)
            # a jump of density and velocity at equal pressure: theta = 0
            rho2, V2 = rho * (1 + 1e-3), V + 1e-3 * rng.uniform(-1, 1, 3)
            vh = I.entropy_vars(np.array(rho2), [np.array(x) for x in V2], np.array(P)).astype(float)
            R2, L2, T2 = oracle.kepes_parts(vh, v, n)
            diss = oracle.flux_num(oracle.KEPES, vh, v, n) - oracle.flux_num(oracle.EC, vh, v, n)
            dv = vh - v
            assert np.allclose(diss, -0.5 * R2 @ np.diag(L2 * T2) @ R2.T @ dv, rtol=1e-9,
                               atol=1e-12 * np.abs(diss).max())


def test_kepes_hybrid_theta_from_pressure_ratio():
    """|Lambda-bar| = (1 - theta)|lambda| + theta lambda_max with theta =
    sqrt(|(P - P-hat)/(P + P-hat)|): under the reading |lambda_1| = |lambda_5|
    = lambda_max = |v_n-bar| + c-bar, entries 1 and 5 stay lambda_max and the
    middle ones equal |v_n-bar| + theta c-bar, so theta is recovered from the
    parts and compared with the pressures; c-bar = sqrt(gamma P-bar / rho^ln)
    with P-bar = rho-bar / beta-bar (eq. EC); a large pressure ratio drives
    theta towards 1 (LF dissipation everywhere)."""
    rng = np.random.default_rng(23)
    for ratio in (1.0 + 1e-6, 1.3, 4.0, 1e4):
        for _ in range(4):
            rho, P = rng.uniform(0.5, 2.0), rng.uniform(0.4, 2.0)
            V, Vh = rng.uniform(-0.3, 0.3, 3), rng.uniform(-0.3, 0.3, 3)
            rhoh, Ph = rho * rng.uniform(0.8, 1.2), P * ratio
            v = I.entropy_vars(np.array(rho), [np.array(x) for x in V], np.array(P)).astype(float)
            vh = I.entropy_vars(np.array(rhoh), [np.array(x) for x in Vh], np.array(Ph)).astype(float)
            for n in _general_normals():
                R, L, T = oracle.kepes_parts(vh, v, n)
                vnb = abs(0.5 * (V + Vh) @ n)
                Pb = 0.5 * (rho + rhoh) / (0.5 * (rho / P + rhoh / Ph))
                cb = math.sqrt(G * Pb / oracle.logmean(rho, rhoh))
                theta = math.sqrt(abs((P - Ph) / (P + Ph)))
                assert abs(L[0] - (vnb + cb)) < 1e-12 and abs(L[4] - (vnb + cb)) < 1e-12
                assert np.allclose(L[1:4], vnb + theta * cb, rtol=1e-12)
                if ratio > 1e3:
                    assert np.all(L[1:4] > 0.97 * L[0])


def test_es_sigma_is_the_spectral_radius_at_vhat():
    """ES flux (eq. Flux_En_Inv): at equal states d F/dv - d F/dv-hat =
    sigma A0 (the averages of F cancel), and at any pair of states
    F - 1/2 (F(v-hat) + F(v)).n = -1/2 sigma(v-hat) A0(v-hat) [[v]], where
    sigma(v-hat) = lambda_max = the spectral radius of A_n(v-hat) from a
    numerical eigendecomposition (not a formula for the wave speed)."""
    rng = np.random.default_rng(24)
    for _ in range(6):
        v = rand_state(rng)
        vh = v + rng.uniform(-2e-2, 2e-2, 5)
        for n in _general_normals():
            _, w, _ = _An_eig(v, n)
            sig = np.abs(w).max()
            Jv = _jac_fd(lambda x: oracle.flux_num(oracle.ES, v, x, n), v, 1e-6)
            Jh = _jac_fd(lambda x: oracle.flux_num(oracle.ES, x, v, n), v, 1e-6)
            A0 = oracle.A0(v)
            assert np.allclose(Jv - Jh, sig * A0, rtol=1e-6, atol=1e-7 * np.abs(A0).max())
            _, wh, _ = _An_eig(vh, n)
            sigh = np.abs(wh).max()
            diss = oracle.flux_num(oracle.ES, vh, v, n) - 0.5 * (oracle.flux_phys(vh, n) + oracle.flux_phys(v, n))
            assert np.allclose(diss, -0.5 * sigh * oracle.A0(vh) @ (vh - v), rtol=1e-7,
                               atol=1e-9 * np.abs(diss).max())


# ---------------------------------------------------------------- viscous
def test_viscous_flux_dissipates_entropy_and_is_linear_in_q():
    """sum_j q_j . G_j = -q^T K q <= 0 (eq. entropy evolution diffuse) and
    G(v, a q1 + b q2) = a G(v,q1) + b G(v,q2)"""
    prm = oracle.params(viscous=1, Re=100.0, Mach=0.3)
    rng = np.random.default_rng(11)
    for _ in range(20):
        v = rand_state(rng)
        q1, q2 = rng.normal(size=15), rng.normal(size=15)
        G1, G2 = oracle.visc_flux(prm, v, q1), oracle.visc_flux(prm, v, q2)
        assert np.sum(q1.reshape(5, 3) * G1) <= 1e-15
        G12 = oracle.visc_flux(prm, v, 0.3 * q1 - 1.7 * q2)
        assert np.allclose(G12, 0.3 * G1 - 1.7 * G2, rtol=1e-12, atol=1e-14)


def test_viscous_flux_vanishes_for_rigid_rotation():
    """tau = 0 and grad T = 0 for a rigid rotation V = w x r at constant state"""
    prm = oracle.params(viscous=1, Re=100.0, Mach=0.3)
    w = np.array([0.3, -0.2, 0.5])
    rho, P = 1.2, 0.9
    V = np.array([0.1, 0.2, -0.1])
    gradV = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])   # dV_i/dx_j
    beta = rho / P
    v = I.entropy_vars(np.array(rho), [np.array(c) for c in V], np.array(P)).astype(float)
    # grad v at constant rho, P: dv1 = -beta V.gradV, dv_{2..4} = beta gradV, dv5 = 0
    q = np.zeros((5, 3))
    q[0] = -beta * V @ gradV
    q[1:4] = beta * gradV
    assert np.abs(oracle.visc_flux(prm, v, q.ravel())).max() < 1e-15


VPRM = dict(viscous=1, Re=1600.0, Mach=0.1, Pr=0.71)


def _q_const_rho_P(V, gradV, rho, P):
    """grad v at constant rho and P (eq. s222): dv1 = -beta V.grad V,
    dv_{2..4} = beta grad V, dv5 = 0, as [5][3] with q[k][d] = dv_k/dx_d"""
    beta = rho / P
    q = np.zeros((5, 3))
    q[0] = -beta * V @ gradV
    q[1:4] = beta * gradV
    return q


def test_viscous_shear_stress_couette():
    """Couette shear V = (a y, 0, 0) at uniform rho, P: tau_xy = tau_yx =
    (Mach/Re) a (eq. C6 with mu/Re_c = Mach/Re), every other stress 0, no
    heat flux; G = -[0, tau, tau V - phi] (eq. C5), so G_{x,y} = G_{y,x} =
    -(Mach/Re) a and the energy row -(tau V)_y = -(Mach/Re) a^2 y"""
    prm = oracle.params(**VPRM)
    mu = VPRM["Mach"] / VPRM["Re"]
    rho, P, a, y = 1.1, 0.8, 0.37, 0.6
    V = np.array([a * y, 0.0, 0.0])
    gradV = np.zeros((3, 3)); gradV[0, 1] = a
    v = I.entropy_vars(np.array(rho), [np.array(c) for c in V], np.array(P)).astype(float)
    Gv = oracle.visc_flux(prm, v, _q_const_rho_P(V, gradV, rho, P).ravel())
    exp = np.zeros((5, 3))
    exp[1, 1] = -mu * a          # momentum x, flux in y
    exp[2, 0] = -mu * a          # momentum y, flux in x
    exp[4, 1] = -mu * a * a * y  # energy, flux in y
    assert np.allclose(Gv, exp, rtol=1e-12, atol=1e-18)


def test_viscous_bulk_coefficient_uniaxial_stretch():
    """V = (b x, 0, 0): div V = b, so tau_xx = mu (2 + lambda) b and
    tau_yy = tau_zz = mu lambda b; lambda = -2/3 (Stokes) gives 4/3 mu b and
    -2/3 mu b (any other bulk coefficient fails)"""
    prm = oracle.params(**VPRM)
    mu = VPRM["Mach"] / VPRM["Re"]
    rho, P, b, x = 0.9, 1.3, 0.21, -0.4
    V = np.array([b * x, 0.0, 0.0])
    gradV = np.zeros((3, 3)); gradV[0, 0] = b
    v = I.entropy_vars(np.array(rho), [np.array(c) for c in V], np.array(P)).astype(float)
    Gv = oracle.visc_flux(prm, v, _q_const_rho_P(V, gradV, rho, P).ravel())
    tau = np.diag([4.0 / 3.0 * mu * b, -2.0 / 3.0 * mu * b, -2.0 / 3.0 * mu * b])
    exp = np.zeros((5, 3))
    exp[1:4] = -tau
    exp[4] = -(tau @ V)
    assert np.allclose(Gv, exp, rtol=1e-12, atol=1e-18)


def test_viscous_heat_flux_linear_temperature():
    """At rest with uniform P and T = T0 + c x (gamma P = rho T): tau = 0 and
    G_energy = phi = -kappa dT/dx e_x with kappa = (Mach/Re) / ((gamma-1) Pr)
    (the reading of eq. C6: mu c_p / Pr, c_p = 1/(gamma-1)); grad v by
    fourth-order differences of eq. s222 along x"""
    prm = oracle.params(**VPRM)
    kap = VPRM["Mach"] / VPRM["Re"] / ((G - 1.0) * VPRM["Pr"])
    P, T0, c, x0 = 0.75, 1.05, 0.3, 0.2

    def vx(x):
        T = T0 + c * x
        rho = G * P / T
        return I.entropy_vars(np.array(rho), [np.array(0.0)] * 3, np.array(P)).astype(float)

    h = 1e-3
    dvdx = (8 * (vx(x0 + h) - vx(x0 - h)) - (vx(x0 + 2 * h) - vx(x0 - 2 * h))) / (12 * h)
    q = np.zeros((5, 3)); q[:, 0] = dvdx
    Gv = oracle.visc_flux(prm, vx(x0), q.ravel())
    exp = np.zeros((5, 3)); exp[4, 0] = -kap * c
    assert np.allclose(Gv, exp, rtol=1e-9, atol=1e-15)


def test_viscous_face_penalty_sigma_vis():
    """eq. Flux_En_Vis: with q = 0 the viscous face flux adds exactly
    -1/2 sigma^vis [[v]], sigma^vis = (1/Re) diag(0, 1, 1, 1,
    1/((gamma-1) M^2 Pr)), component by component, to the inviscid flux"""
    rng = np.random.default_rng(25)
    pv, pi = oracle.params(flux=oracle.ES, **VPRM), oracle.params(flux=oracle.ES, Mach=VPRM["Mach"])
    Re, M, Pr = VPRM["Re"], VPRM["Mach"], VPRM["Pr"]
    sv = np.array([0.0, 1.0, 1.0, 1.0, 1.0 / ((G - 1.0) * M * M * Pr)]) / Re
    for _ in range(10):
        v, vh = rand_state(rng), rand_state(rng)
        for n in normals():
            d = oracle.face_flux(pv, vh, v, np.zeros(15), n) - oracle.face_flux(pi, vh, v, None, n)
            assert np.allclose(d, -0.5 * sv * (vh - v), rtol=1e-10, atol=1e-16)


# ---------------------------------------------------------------- residual
@pytest.mark.parametrize("flux", [oracle.EC, oracle.ES, oracle.KEPES])
@pytest.mark.parametrize("vis", [0, 1])
def test_free_stream_preservation(flux, vis):
    """P1: constant state, v-hat = v, q = 0  =>  R = 0"""
    mesh = I.periodic_mesh(2, 2, 2)
    st = I.make_state(mesh, "const", 0.0, 1, 2, viscous=bool(vis))
    if vis:
        st.q[:] = 0
    prm = oracle.params(flux=flux, viscous=vis)
    RV, RQ, RH = oracle.residual_mesh(prm, mesh, st)
    assert np.abs(RV).max() < 1e-13 and np.abs(RH).max() < 1e-13
    if vis:
        assert np.abs(RQ).max() < 1e-13


@pytest.mark.parametrize("flux", [oracle.EC, oracle.KEPES, oracle.ES])
def test_discrete_entropy_identity_prop41(flux):
    """P5: periodic Euler, time term off:
    v^T R_V - vhat^T R_Vhat = -D_Q - sum <[[v]].F-hat - [[Psi_n]]>_Q ;
    the last sum vanishes for EC (Thm. 5.1) and is <= 0 for KEPES/ES."""
    mesh = I.periodic_mesh(2, 2, 2)
    st = I.make_state(mesh, "tgv", 1e-2, 3, 4, M0=0.3)
    prm = oracle.params(flux=flux, viscous=0, time_term=0)
    RV, _, RH = oracle.residual_mesh(prm, mesh, st)
    lhs = np.sum(st.v * RV) - np.sum(st.vhat * RH)
    D = sum(oracle.entropy_defect_K(prm, 2, 2, mesh.boxes[K], st.v[K]) for K in range(mesh.nK))
    if flux == oracle.EC:
        assert abs(lhs + D) < 1e-12 * (abs(lhs) + abs(D) + np.abs(RV).sum() * 1e-3)
    else:
        assert lhs + D > 0


def _box_moments(fun, box, npts=12):
    """-int_K F_{k,j}(u) dV (moment with x_j) and the face integrals
    int_dK F.n dS, int_dK x_j F.n dS, by a tensor Gauss rule of the test's own"""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    lo, hi = np.array(box[:3]), np.array(box[3:])
    X = [lo[d] + (hi[d] - lo[d]) * (xg + 1) / 2 for d in range(3)]
    W = [(hi[d] - lo[d]) / 2 * wg for d in range(3)]
    vol = np.zeros((5, 3))
    Z, Y, Xx = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    WW = (W[2][:, None, None] * W[1][None, :, None] * W[0][None, None, :])
    F = fun(Xx, Y, Z)                        # [5][3][...]
    for j in range(3):
        vol[:, j] = -np.sum(F[:, j] * WW, axis=(1, 2, 3))
    face0 = np.zeros(5)
    face1 = np.zeros((5, 3))
    for d in range(3):
        t1, t2 = [(1, 2), (0, 2), (0, 1)][d]
        B2, B1 = np.meshgrid(X[t2], X[t1], indexing="ij")
        Wf = W[t2][:, None] * W[t1][None, :]
        for side, sgn in ((0, -1.0), (1, 1.0)):
            pts = [None] * 3
            pts[t1], pts[t2] = B1, B2
            pts[d] = np.full_like(B1, hi[d] if side else lo[d])
            Ff = fun(*pts)[:, d] * sgn
            face0 += np.sum(Ff * Wf, axis=(1, 2))
            for j in range(3):
                face1[:, j] += np.sum(Ff * pts[j] * Wf, axis=(1, 2))
    return vol, face0, face1


def test_exact_vortex_truncation_converges():
    """P6: with the exact vortex (eq. S601) on the nodes and traces of one
    macro-element and no time term, the moments sum_a R_V[a] and
    sum_a x_a R_V[a] (the C0 basis reproduces 1 and x) approach the exact
    integrals int_dK F.n and -int_K F_j + int_dK x_j F.n as h -> 0."""
    p = 3
    box = [3.5, 3.5, 3.5, 6.5, 6.5, 6.5]

    def Fexact(x, y, z):
        rho, V, P = I.vortex_prim(x, y, z)
        E = P / (G - 1) + 0.5 * rho * (V[0] ** 2 + V[1] ** 2 + V[2] ** 2)
        F = np.zeros((5, 3) + np.shape(x))
        for j in range(3):
            F[0, j] = rho * V[j]
            for i in range(3):
                F[1 + i, j] = rho * V[i] * V[j] + (P if i == j else 0)
            F[4, j] = V[j] * (E + P)
        return F

    vol, f0, f1 = _box_moments(Fexact, box, npts=20)
    errs = []
    for m in (1, 2, 4):
        mesh = I.Mesh(p, m, np.array([box]), np.arange(6).reshape(1, 6), 6)
        st = I.make_state(mesh, "vortex", 0.0, 1, 2)
        prm = oracle.params(flux=oracle.KEPES, time_term=0)
        RV, _, _ = oracle.residual_mesh(prm, mesh, st)
        X, Y, Z = I.node_coords(mesh, 0)
        m0 = RV[0].sum(axis=1)
        m1 = np.stack([RV[0] @ X, RV[0] @ Y, RV[0] @ Z], axis=1)
        errs.append((np.abs(m0 - f0).max() / np.abs(f0).max(),
                     np.abs(m1 - (vol + f1)).max() / np.abs(vol + f1).max()))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert errs[-1].max() < 1e-5, errs
    assert rates.min() >= p, (errs, rates)


def test_rq_linear_and_mass_block():
    """P10: R_Q is linear in (q, v, vhat); A_qq = I_15 (x) M with M SPD,
    1^T M 1 = |K|; A_qv 1 = boundary term (int d_d phi_a = oint n_d phi_a)."""
    p, m = 2, 1
    mesh = I.periodic_mesh(1, p, m, 0.0, 1.3)
    st = I.make_state(mesh, "tgv", 1e-2, 3, 4, viscous=True, M0=0.3)
    prm = oracle.params(viscous=1, Re=100.0, Mach=0.3)
    vh = oracle.gather_trace(mesh, st.vhat, 0)
    B = oracle.jacobian_K(prm, p, m, mesh.boxes[0], st.v[0], st.vstar[0], vh, st.q[0])
    Nn = mesh.Nn
    Aqq = B["Aqq"]
    M = Aqq[:Nn, :Nn]
    assert np.allclose(Aqq, np.kron(np.eye(15), M))
    assert np.allclose(M, M.T) and np.linalg.eigvalsh(M).min() > 0
    assert abs(M.sum() - 1.3 ** 3) < 1e-13
    _, RQ0, _ = oracle.residual_K(prm, p, m, mesh.boxes[0], st.v[0], st.vstar[0], vh, st.q[0])
    lin = Aqq @ st.q[0].ravel() + B["Aqv"] @ st.v[0].ravel() + B["Aqh"] @ vh.ravel()
    assert np.allclose(RQ0, lin, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("flux", [oracle.EC, oracle.ES])
@pytest.mark.parametrize("vis", [0, 1])
def test_jacobian_matches_central_differences(flux, vis):
    """P8: complex-step Jacobian blocks vs central differences (step 1e-6)"""
    p, m = 2, 1
    mesh = I.periodic_mesh(2, p, m)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, viscous=bool(vis), M0=0.3)
    prm = oracle.params(flux=flux, viscous=vis, Re=100.0, Mach=0.3)
    K = 3
    vh = oracle.gather_trace(mesh, st.vhat, K)
    q = None if st.q is None else st.q[K]
    B = oracle.jacobian_K(prm, p, m, mesh.boxes[K], st.v[K], st.vstar[K], vh, q)
    rng = np.random.default_rng(0)
    dv, dh = rng.uniform(-1, 1, st.v[K].shape), rng.uniform(-1, 1, vh.shape)
    dq = None if q is None else rng.uniform(-1, 1, q.shape)
    eps = 1e-6

    def R(s):
        return oracle.residual_K(prm, p, m, mesh.boxes[K], st.v[K] + s * dv, st.vstar[K], vh + s * dh,
                                 None if q is None else q + s * dq)
    Rp, Rm = R(eps), R(-eps)
    jV = B["Avv"] @ dv.ravel() + B["Avh"] @ dh.ravel() + (B["Avq"] @ dq.ravel() if vis else 0)
    jH = B["Ahv"] @ dv.ravel() + B["Ahh"] @ dh.ravel() + (B["Ahq"] @ dq.ravel() if vis else 0)
    for fd, j in (((Rp[0] - Rm[0]) / (2 * eps), jV), ((Rp[2] - Rm[2]) / (2 * eps), jH)):
        assert np.linalg.norm(fd - j) / np.linalg.norm(j) < 5e-9


@pytest.mark.parametrize("mp", [(1, 1), (1, 2), (2, 1)])
@pytest.mark.parametrize("vis", [0, 1])
def test_condensation_matches_monolithic_brute_force(mp, vis):
    """P7: condense (R3, R5) -> dense global solve -> recover (R2, R6) equals
    the monolithic GEPP solve of the full Newton system on 2^3 elements"""
    m, p = mp
    mesh = I.periodic_mesh(2, p, m)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, viscous=bool(vis), M0=0.3)
    prm = oracle.params(flux=oracle.ES if vis else oracle.KEPES, viscous=vis, Re=100.0, Mach=0.3)
    dQ, dV, dH = oracle.brute_force(prm, mesh, st)
    bh, Ahats = oracle.condense_mesh(prm, mesh, st, want_Ahat=True)
    A = oracle.assemble_Ahat(mesh, Ahats)
    x = oracle.solve(A, bh.ravel()).reshape(dH.shape)
    dV2, dQ2 = oracle.recover_mesh(prm, mesh, st, x)
    e = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert e(x, dH) < 1e-10 and e(dV2, dV) < 1e-10
    if vis:
        assert e(dQ2, dQ) < 1e-10


def test_brute_force_on_self_periodic_mesh():
    """P7 on a 2x1x1 periodic mesh, where an element's y-/y+ and z-/z+
    faces are the same global face (both sides summed, eq. s32c)"""
    mesh = I.periodic_mesh((2, 1, 1), 1, 1)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
    prm = oracle.params(flux=oracle.KEPES, Mach=0.3)
    dQ, dV, dH = oracle.brute_force(prm, mesh, st)
    bh, Ahats = oracle.condense_mesh(prm, mesh, st, want_Ahat=True)
    x = oracle.solve(oracle.assemble_Ahat(mesh, Ahats), bh.ravel()).reshape(dH.shape)
    dV2, _ = oracle.recover_mesh(prm, mesh, st, x)
    e = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert e(x, dH) < 1e-10 and e(dV2, dV) < 1e-10


def test_getrf_matches_library_solve():
    rng = np.random.default_rng(12)
    A = rng.normal(size=(60, 60)); b = rng.normal(size=60)
    x = oracle.solve(A, b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-11)
    LU, piv, info = oracle.getrf(A)
    assert piv[0] == int(np.argmax(np.abs(A[:, 0])))


def test_dof_tables():
    """P9: counting reproduces Tables Inv_TGV_DOF / TGV_DOF"""
    rows = json.load(open(os.path.join(HERE, "golden", "dof_tables.json")))["rows"]
    for r in rows:
        for m in (1, 2):
            loc, glo = oracle.dof_counts_tet(r["p"], m, r["N_ele"])
            assert loc == r[f"m{m}_local"] and glo == r[f"m{m}_global"], (r, m, loc, glo)


def test_oracle_residual_vjp_against_central_differences():
    """the oracle's VJP (transposed complex-step blocks, assembled over the
    mesh) against central differences of the oracle residual.  ES flux: the
    KEPES flux's theta = sqrt(|(P - Phat)/(P + Phat)|) has an unbounded
    derivative as P -> Phat, so central differences of it converge only as
    the step goes to zero."""
    import numpy as np
    from paper_2507_22195_gb300 import inputs as I
    mesh = I.periodic_mesh((2, 1, 1), 1, 1)
    st = I.make_state(mesh, "tgv", 1e-2, 5, 6, M0=0.3)
    prm = oracle.params(flux=1, Mach=0.3)
    g = np.random.default_rng(3)
    lv = g.standard_normal((mesh.nK, 5, mesh.Nn))
    lh = g.standard_normal((mesh.n_global_faces, 5, mesh.n2))
    gv, gh = oracle.residual_vjp_mesh(prm, mesh, st, lv, lh)
    dv = g.standard_normal(st.v.shape)
    dh = g.standard_normal(st.vhat.shape)
    eps = 1e-6
    vals = []
    for sgn in (1.0, -1.0):
        s2 = I.State(v=st.v + sgn * eps * dv, vhat=st.vhat + sgn * eps * dh, q=None, vstar=st.vstar)
        rv, _, rh = oracle.residual_mesh(prm, mesh, s2)
        vals.append((rv * lv).sum() + (rh * lh).sum())
    fd = (vals[0] - vals[1]) / (2 * eps)
    ad = (gv * dv).sum() + (gh * dh).sum()
    assert abs(fd - ad) < 1e-7 * abs(ad), (fd, ad)


def test_dirk33_table_and_third_order_in_time():
    """DIRK(3,3) (Sec. 5.3): the table satisfies the order conditions up to
    order 3 (b.1 = 1, b.c = 1/2, b.c^2 = 1/3, b.A c = 1/6, c = A 1) and is
    stiffly accurate; on a perturbed TGV the oracle's steps show third order in
    time: with errors against the finest of dt, dt/2, dt/4, the ratio
    |u_dt - u_dt/4| / |u_dt/2 - u_dt/4| is 2^p + 1 = 9 for order p = 3
    asymptotically (5 for p = 2)."""
    A, b, c = oracle.dirk33()
    assert abs(b.sum() - 1) < 1e-14 and abs(b @ c - 0.5) < 1e-14
    assert abs(b @ c ** 2 - 1 / 3) < 1e-14 and abs(b @ A @ c - 1 / 6) < 1e-14
    assert np.allclose(A.sum(1), c, atol=1e-14) and np.allclose(A[-1], b, atol=1e-15)
    mesh = I.periodic_mesh(2, 1, 1)
    st0 = I.make_state(mesh, "tgv", 2e-2, 5, 6, M0=0.3)
    kw = dict(flux=1, Mach=0.3)
    T, res = 0.4, {}
    for n in (2, 4, 8):
        st = st0
        for _ in range(n):
            st, _, its = oracle.dirk_step(kw, mesh, st, T / n)
            assert max(its) < 12
        res[n] = st.v
    ratio = np.linalg.norm(res[2] - res[8]) / np.linalg.norm(res[4] - res[8])
    assert 7.0 < ratio < 10.0, ratio
