"""FP64 CPU oracle for the macro-element HDG Newton step (arXiv 2507.22195).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg; never by the product path.  The C source
``mehdg_oracle.c`` is compiled here with gcc into ``liborc.so`` (no shared
code with the CUDA library).

Mesh-level helpers below gather traces from the global trace vector, call the
per-macro-element C routines and sum the two sides of every global face
(eq. s32c; Algorithm 1, assembly of b-hat), then offer a monolithic
brute-force Newton solve for tiny meshes to pin the condensation
(eqs. R1-R6).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mehdg_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

EC, ES, KEPES = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("Re", C.c_double), ("Pr", C.c_double),
                ("Mach", C.c_double), ("dt", C.c_double), ("viscous", C.c_int),
                ("flux", C.c_int), ("time_term", C.c_int)]


def params(gamma=1.4, Re=1600.0, Pr=0.71, Mach=0.1, dt=1.0, viscous=0, flux=KEPES, time_term=1):
    return Params(gamma, Re, Pr, Mach, dt, int(viscous), int(flux), int(time_term))


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_long)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_gauss.argtypes = [C.c_int, _dp, _dp]
            L.orc_gll.argtypes = [C.c_int, _dp]
            L.orc_u_of_v.argtypes = [C.c_double, _dp, _dp]
            L.orc_prim_of_v.argtypes = [C.c_double, _dp, _dp, _dp, _dp]
            L.orc_A0.argtypes = [C.c_double, _dp, _dp]
            L.orc_dudv_cs.argtypes = [C.c_double, _dp, _dp]
            L.orc_flux_phys.argtypes = [C.c_double, _dp, _dp, _dp]
            L.orc_flux_num.argtypes = [C.c_int, C.c_double, _dp, _dp, _dp, _dp]
            L.orc_face_flux.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp]
            L.orc_visc_flux.argtypes = [C.POINTER(Params), _dp, _dp, _dp]
            L.orc_kepes_parts.argtypes = [C.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_logmean.argtypes = [C.c_double, C.c_double]
            L.orc_logmean.restype = C.c_double
            L.orc_residual.argtypes = [C.POINTER(Params), C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp,
                                       _dp, _dp, _dp]
            L.orc_entropy_defect.argtypes = [C.POINTER(Params), C.c_int, C.c_int, _dp, _dp]
            L.orc_entropy_defect.restype = C.c_double
            L.orc_jacobian.argtypes = [C.POINTER(Params), C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp] + [_dp] * 9
            L.orc_getrf.argtypes = [C.c_int, _dp, _ip]
            L.orc_getrs.argtypes = [C.c_int, _dp, _ip, C.c_int, _dp]
            L.orc_condense_blocks.argtypes = [C.c_int, C.c_long, C.c_long, C.c_long] + [_dp] * 12 + \
                [_dp, _dp, _dp, _dp, _dp]
            L.orc_matvec.argtypes = [C.c_long, C.c_long, _dp, _dp, _dp]
            L.orc_dof_counts_tet.argtypes = [C.c_int, C.c_int, C.c_long, _lp, _lp]
            L.orc_dof_counts_hex.argtypes = [C.c_int, C.c_int, C.c_long, C.c_int, _lp, _lp]
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, (a.dtype, a.flags)
    return a.ctypes.data_as(_dp)


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- tables
def gauss(n):
    x, w = np.zeros(n), np.zeros(n)
    assert lib().orc_gauss(n, _p(x), _p(w)) == 0
    return x, w


def gll(p):
    x = np.zeros(p + 1)
    assert lib().orc_gll(p, _p(x)) == 0
    return x


# ---------------------------------------------------------------- point-wise
def u_of_v(v, gamma=1.4):
    v = _f(v); u = np.zeros(5); lib().orc_u_of_v(gamma, _p(v), _p(u)); return u


def prim_of_v(v, gamma=1.4):
    v = _f(v); r, P = C.c_double(), C.c_double(); V = np.zeros(3)
    lib().orc_prim_of_v(gamma, _p(v), C.byref(r), _p(V), C.byref(P))
    return r.value, V, P.value


def A0(v, gamma=1.4):
    v = _f(v); A = np.zeros(25); lib().orc_A0(gamma, _p(v), _p(A)); return A.reshape(5, 5)


def dudv_cs(v, gamma=1.4):
    v = _f(v); A = np.zeros(25); lib().orc_dudv_cs(gamma, _p(v), _p(A)); return A.reshape(5, 5)


def flux_phys(v, n, gamma=1.4):
    v, n = _f(v), _f(n); F = np.zeros(5); lib().orc_flux_phys(gamma, _p(v), _p(n), _p(F)); return F


def flux_num(kind, vh, v, n, gamma=1.4):
    vh, v, n = _f(vh), _f(v), _f(n); F = np.zeros(5)
    lib().orc_flux_num(kind, gamma, _p(vh), _p(v), _p(n), _p(F)); return F


def face_flux(prm, vh, v, q, n):
    vh, v, n = _f(vh), _f(v), _f(n); q = None if q is None else _f(q); F = np.zeros(5)
    lib().orc_face_flux(C.byref(prm), _p(vh), _p(v), _p(q), _p(n), _p(F)); return F


def visc_flux(prm, v, q):
    v, q = _f(v), _f(q); G = np.zeros(15)
    lib().orc_visc_flux(C.byref(prm), _p(v), _p(q), _p(G)); return G.reshape(5, 3)


def kepes_parts(vh, v, n, gamma=1.4):
    vh, v, n = _f(vh), _f(v), _f(n)
    R, L, T = np.zeros(25), np.zeros(5), np.zeros(5)
    lib().orc_kepes_parts(gamma, _p(vh), _p(v), _p(n), _p(R), _p(L), _p(T))
    return R.reshape(5, 5), L, T


def logmean(a, b):
    return lib().orc_logmean(float(a), float(b))


# ---------------------------------------------------------------- one element
def sizes(p, m):
    n = m * p + 1
    Nn = n ** 3
    return n, Nn, 5 * Nn, 15 * Nn, 30 * n * n


def residual_K(prm, p, m, box, v, vs, vh_loc, q=None):
    n, Nn, Nv, Nq, Nt = sizes(p, m)
    RV, RQ, RH = np.zeros(Nv), np.zeros(Nq), np.zeros(Nt)
    rc = lib().orc_residual(C.byref(prm), p, m, _p(_f(box)), _p(_f(v)), _p(_f(vs)),
                            _p(_f(vh_loc)), _p(None if q is None else _f(q)), _p(RV), _p(RQ), _p(RH))
    assert rc == 0
    return RV, (RQ if q is not None else None), RH


def entropy_defect_K(prm, p, m, box, v):
    return lib().orc_entropy_defect(C.byref(prm), p, m, _p(_f(box)), _p(_f(v)))


def jacobian_K(prm, p, m, box, v, vs, vh_loc, q=None):
    n, Nn, Nv, Nq, Nt = sizes(p, m)
    vis = q is not None
    B = dict(Avv=np.zeros((Nv, Nv)), Avh=np.zeros((Nv, Nt)), Ahv=np.zeros((Nt, Nv)),
             Ahh=np.zeros((Nt, Nt)))
    if vis:
        B.update(Avq=np.zeros((Nv, Nq)), Ahq=np.zeros((Nt, Nq)), Aqq=np.zeros((Nq, Nq)),
                 Aqv=np.zeros((Nq, Nv)), Aqh=np.zeros((Nq, Nt)))
    g = lambda k: _p(B[k]) if k in B else None
    rc = lib().orc_jacobian(C.byref(prm), p, m, _p(_f(box)), _p(_f(v)), _p(_f(vs)), _p(_f(vh_loc)),
                            _p(None if q is None else _f(q)),
                            g("Avv"), g("Avh"), g("Ahv"), g("Ahh"), g("Avq"), g("Ahq"),
                            g("Aqq"), g("Aqv"), g("Aqh"))
    assert rc == 0
    return B


def getrf(A):
    A = _f(A).copy(); N = A.shape[0]; piv = np.zeros(N, dtype=np.int32)
    info = lib().orc_getrf(N, _p(A), piv.ctypes.data_as(_ip))
    return A, piv, info


def getrs(LU, piv, B):
    B = _f(B).copy(); N = LU.shape[0]
    nrhs = 1 if B.ndim == 1 else B.shape[1]
    lib().orc_getrs(N, _p(LU), piv.ctypes.data_as(_ip), nrhs, _p(B))
    return B


def solve(A, b):
    LU, piv, info = getrf(A)
    assert info == 0, "singular"
    return getrs(LU, piv, b)


def condense_K(viscous, R, B, want_Ahat=False, dvh=None):
    """eqs. R2-R6 for one element from its residuals R=(RV,RQ,RH) and blocks B."""
    RV, RQ, RH = R
    Nv, Nt = B["Avv"].shape[0], B["Avh"].shape[1]
    Nq = B["Aqq"].shape[0] if viscous else 0
    bhat = np.zeros(Nt)
    Ahat = np.zeros((Nt, Nt)) if want_Ahat else None
    dV = np.zeros(Nv) if dvh is not None else None
    dQ = np.zeros(Nq) if (dvh is not None and viscous) else None
    g = lambda k: _p(B[k]) if (k in B) else None
    rc = lib().orc_condense_blocks(int(viscous), Nv, Nq, Nt, _p(_f(RV)),
                                   _p(None if RQ is None else _f(RQ)), _p(_f(RH)),
                                   g("Avv"), g("Avh"), g("Ahv"), g("Ahh"), g("Avq"), g("Ahq"),
                                   g("Aqq"), g("Aqv"), g("Aqh"),
                                   _p(bhat), _p(Ahat), _p(None if dvh is None else _f(dvh)),
                                   _p(dV), _p(dQ))
    assert rc == 0, rc
    return bhat, Ahat, dV, dQ


def dof_counts_tet(p, m, n_tet):
    a, b = C.c_long(), C.c_long()
    lib().orc_dof_counts_tet(p, m, n_tet, C.byref(a), C.byref(b))
    return a.value, b.value


def dof_counts_hex(p, m, n_macro, viscous):
    a, b = C.c_long(), C.c_long()
    lib().orc_dof_counts_hex(p, m, n_macro, int(viscous), C.byref(a), C.byref(b))
    return a.value, b.value


# ---------------------------------------------------------------- mesh level
def gather_trace(mesh, vhat_global, K):
    """local trace [6][5][n2] of element K from the global trace vector"""
    return np.ascontiguousarray(vhat_global[mesh.face_gid[K]])


def scatter_trace(mesh, local, K, out):
    for f in range(6):
        out[mesh.face_gid[K, f]] += local[f]


def residual_mesh(prm, mesh, st, Ks=None):
    """R_V [K,5,Nn], R_Q [K,5,3,Nn] or None, R_Vhat global [G,5,n2] (sum of both sides)."""
    p, m, Nn, n2 = mesh.p, mesh.m, mesh.Nn, mesh.n2
    Ks = range(mesh.nK) if Ks is None else Ks
    RV = np.zeros((mesh.nK, 5, Nn))
    RQ = np.zeros((mesh.nK, 5, 3, Nn)) if st.q is not None else None
    RH = np.zeros((mesh.n_global_faces, 5, n2))
    for K in Ks:
        vh = gather_trace(mesh, st.vhat, K)
        rv, rq, rh = residual_K(prm, p, m, mesh.boxes[K], st.v[K], st.vstar[K], vh,
                                None if st.q is None else st.q[K])
        RV[K] = rv.reshape(5, Nn)
        if RQ is not None:
            RQ[K] = rq.reshape(5, 3, Nn)
        scatter_trace(mesh, rh.reshape(6, 5, n2), K, RH)
    return RV, RQ, RH


def residual_vjp_mesh(prm, mesh, st, lam_V, lam_H):
    """VJP of the residual of eq. s32 (Euler), by definition: the transposed
    complex-step Jacobian blocks of every element applied to the cotangents,
    g_v[K] = Avv^T lam_V[K] + Ahv^T lam_H(K), g_vhat = sum_K scatter(Avh^T
    lam_V[K] + Ahh^T lam_H(K)), with lam_H(K) the element's six faces of the
    global cotangent lam_H [G,5,n2]."""
    p, m, Nn, n2 = mesh.p, mesh.m, mesh.Nn, mesh.n2
    gv = np.zeros((mesh.nK, 5, Nn))
    gh = np.zeros((mesh.n_global_faces, 5, n2))
    for K in range(mesh.nK):
        vh = gather_trace(mesh, st.vhat, K)
        B = jacobian_K(prm, p, m, mesh.boxes[K], st.v[K], st.vstar[K], vh, None)
        lv = lam_V[K].ravel()
        lh = gather_trace(mesh, lam_H, K).ravel()
        gv[K] = (B["Avv"].T @ lv + B["Ahv"].T @ lh).reshape(5, Nn)
        scatter_trace(mesh, (B["Avh"].T @ lv + B["Ahh"].T @ lh).reshape(6, 5, n2), K, gh)
    return gv, gh


def element_system(prm, mesh, st, K):
    p, m = mesh.p, mesh.m
    vh = gather_trace(mesh, st.vhat, K)
    q = None if st.q is None else st.q[K]
    R = residual_K(prm, p, m, mesh.boxes[K], st.v[K], st.vstar[K], vh, q)
    B = jacobian_K(prm, p, m, mesh.boxes[K], st.v[K], st.vstar[K], vh, q)
    return R, B


def condense_mesh(prm, mesh, st, want_Ahat=False):
    """b-hat global (sum over elements, Algorithm 1 local contributions) and,
    optionally, the list of local A-hat^K."""
    n2 = mesh.n2
    bh = np.zeros((mesh.n_global_faces, 5, n2))
    Ahats = []
    for K in range(mesh.nK):
        R, B = element_system(prm, mesh, st, K)
        b, A, _, _ = condense_K(prm.viscous, R, B, want_Ahat)
        scatter_trace(mesh, b.reshape(6, 5, n2), K, bh)
        Ahats.append(A)
    return bh, Ahats


def assemble_Ahat(mesh, Ahats):
    G = mesh.n_global_faces * 5 * mesh.n2
    A = np.zeros((G, G))
    idx = lambda K: (mesh.face_gid[K][:, None] * 5 * mesh.n2 + np.arange(5 * mesh.n2)[None, :]).ravel()
    for K, AK in enumerate(Ahats):
        ii = idx(K)
        # a face may appear twice in one element (periodic with itself): add, never overwrite
        np.add.at(A, (ii[:, None], ii[None, :]), AK)
    return A


def recover_mesh(prm, mesh, st, dvh_global):
    """eqs. R2, R6 for every element: dV [K,5,Nn], dQ [K,5,3,Nn] or None."""
    Nn = mesh.Nn
    dV = np.zeros((mesh.nK, 5, Nn))
    dQ = np.zeros((mesh.nK, 5, 3, Nn)) if prm.viscous else None
    for K in range(mesh.nK):
        R, B = element_system(prm, mesh, st, K)
        dvh = np.ascontiguousarray(dvh_global[mesh.face_gid[K]]).ravel()
        _, _, v_, q_ = condense_K(prm.viscous, R, B, False, dvh)
        dV[K] = v_.reshape(5, Nn)
        if dQ is not None:
            dQ[K] = q_.reshape(5, 3, Nn)
    return dV, dQ


def monolithic_system(prm, mesh, st):
    """The monolithic Newton system of eq. R1 over (Q, V, V-hat global) for all
    elements: J and R, unknowns ordered Q (viscous) of every element, V of
    every element, then the global traces."""
    return _assemble(prm, mesh, st)


def adjoint_solve(prm, mesh, st, gV, gVh):
    """J^T (lam_V, lam_Vhat) = (g_V, g_Vhat) for the monolithic Euler system
    (the transposed Newton system, solved by the oracle's GEPP; tiny meshes)."""
    J, _ = _assemble(prm, mesh, st)
    g = np.concatenate([np.asarray(gV).ravel(), np.asarray(gVh).ravel()])
    lam = solve(np.ascontiguousarray(J.T), g)
    nv = mesh.nK * 5 * mesh.Nn
    return lam[:nv].reshape(mesh.nK, 5, mesh.Nn), lam[nv:].reshape(mesh.n_global_faces, 5, mesh.n2)


def brute_force(prm, mesh, st, src_V=None):
    """Monolithic Newton increment: assemble J over (Q, V, V-hat global) for all
    elements and solve J d = -R with the oracle's GEPP (tiny meshes only).
    src_V [K,5,Nn] (optional) is a constant added to R_V."""
    J, R = _assemble(prm, mesh, st)
    if src_V is not None:
        nq = mesh.nK * 15 * mesh.Nn if prm.viscous else 0
        R = R.copy()
        R[nq:nq + src_V.size] += np.asarray(src_V).ravel()
    nK, Nn, n2 = mesh.nK, mesh.Nn, mesh.n2
    Nv, Nq = 5 * Nn, 15 * Nn
    vis = bool(prm.viscous)
    nq_tot = nK * Nq if vis else 0
    offH = nq_tot + nK * Nv
    d = solve(J, -R)
    dQ = d[:nq_tot].reshape(nK, 5, 3, Nn) if vis else None
    dV = d[nq_tot:offH].reshape(nK, 5, Nn)
    dH = d[offH:].reshape(mesh.n_global_faces, 5, n2)
    return dQ, dV, dH


def _assemble(prm, mesh, st):
    nK, Nn, n2 = mesh.nK, mesh.Nn, mesh.n2
    Nv, Nq, Ntg = 5 * Nn, 15 * Nn, mesh.n_global_faces * 5 * n2
    vis = bool(prm.viscous)
    nq_tot = nK * Nq if vis else 0
    N = nq_tot + nK * Nv + Ntg
    J = np.zeros((N, N))
    R = np.zeros(N)
    offQ = lambda K: K * Nq
    offV = lambda K: nq_tot + K * Nv
    offH = nq_tot + nK * Nv
    for K in range(nK):
        (RV, RQ, RH), B = element_system(prm, mesh, st, K)
        iv = offV(K) + np.arange(Nv)
        ih = (offH + mesh.face_gid[K][:, None] * 5 * n2 + np.arange(5 * n2)[None, :]).ravel()
        # np.add.at: trace indices repeat when an element is periodic with itself
        add = lambda r, c, X: np.add.at(J, (r[:, None], c[None, :]), X)
        np.add.at(R, iv, RV)
        np.add.at(R, ih, RH)
        add(iv, iv, B["Avv"]); add(iv, ih, B["Avh"]); add(ih, iv, B["Ahv"]); add(ih, ih, B["Ahh"])
        if vis:
            iq = offQ(K) + np.arange(Nq)
            np.add.at(R, iq, RQ)
            add(iq, iq, B["Aqq"]); add(iq, iv, B["Aqv"]); add(iq, ih, B["Aqh"])
            add(iv, iq, B["Avq"]); add(ih, iq, B["Ahq"])
    return J, R


# ---------------------------------------------------------------- element samples in parallel
def _condense_one(args):
    """worker: b-hat^K and, for a trace increment, dV^K (eq. R2) and dQ^K
    (eq. R6) of one element, from its own data only; also the seconds taken"""
    import time
    fields, p, m, box, v, vs, vh_loc, q, dvh_loc = args
    prm = Params(*fields)
    t = time.time()
    R = residual_K(prm, p, m, box, v, vs, vh_loc, q)
    B = jacobian_K(prm, p, m, box, v, vs, vh_loc, q)
    bh, _, dV, dQ = condense_K(prm.viscous, R, B, False, dvh_loc)
    return bh, dV, dQ, time.time() - t


def condense_elements(prm, mesh, st, Ks, dvh_global=None, procs=1):
    """For each element K in Ks: (b-hat^K [6,5,n2], dV^K [5,Nn] or None,
    dQ^K or None, seconds).  Elements are independent (Algorithm 1, local
    parts), so a sample of a large mesh is condensed without the others;
    procs > 1 runs them in a spawned process pool."""
    fields = tuple(getattr(prm, f) for f, _ in Params._fields_)
    jobs = []
    for K in Ks:
        vh = gather_trace(mesh, st.vhat, K)
        dvh = None if dvh_global is None else gather_trace(mesh, dvh_global, K).ravel()
        q = None if st.q is None else np.ascontiguousarray(st.q[K])
        jobs.append((fields, mesh.p, mesh.m, mesh.boxes[K].copy(), np.ascontiguousarray(st.v[K]),
                     np.ascontiguousarray(st.vstar[K]), vh, q, dvh))
    if procs <= 1:
        out = [_condense_one(j) for j in jobs]
    else:
        import multiprocessing as mp
        build()
        with mp.get_context("spawn").Pool(procs) as pool:
            out = pool.map(_condense_one, jobs)
    Nn, n2 = mesh.Nn, mesh.n2
    res = []
    for bh, dV, dQ, t in out:
        res.append((bh.reshape(6, 5, n2), None if dV is None else dV.reshape(5, Nn),
                    None if dQ is None else dQ.reshape(5, 3, Nn), t))
    return res


def residual_norm(prm, mesh, st):
    """2-norm of the whole residual (R_Q, R_V, R_V-hat) of eq. s32 at the state"""
    RV, RQ, RH = residual_mesh(prm, mesh, st)
    s = float(np.sum(RV * RV) + np.sum(RH * RH))
    if RQ is not None:
        s += float(np.sum(RQ * RQ))
    return float(np.sqrt(s))


def pseudo_time_newton(prm_kw, mesh, st, nsteps, tau_init=1.0, tau_max=1e8):
    """Inexact Newton with pseudo-transient continuation (Sec. 6.1, eqs.
    C31221-C31223), each linear system solved exactly by the monolithic GEPP
    of brute_force: at step k the stage term is (u(v) - u(v_k)) / tau_k
    (v* = v_k), the increment solves J dV = -R (eq. C312) and the state is
    updated (eq. C31223); tau_0 = tau_init and tau_{k+1} = min(tau_max,
    tau_k ||R_k|| / ||R_{k+1}||) (residual-based growth), ||R|| the residual
    at the iterate with v* = v (the steady residual).  Returns (final state,
    norms [nsteps+1], taus [nsteps]).  Tiny meshes only."""
    from paper_2507_22195_gb300.inputs import State
    s = State(v=st.v.copy(), vhat=st.vhat.copy(), q=None if st.q is None else st.q.copy(), vstar=st.v.copy())
    norms = [residual_norm(params(dt=tau_init, **prm_kw), mesh, s)]
    taus = []
    tau = tau_init
    for _ in range(nsteps):
        taus.append(tau)
        prm = params(dt=tau, **prm_kw)
        s.vstar = s.v.copy()
        dQ, dV, dH = brute_force(prm, mesh, s)
        s.v = s.v + dV
        s.vhat = s.vhat + dH
        if s.q is not None:
            s.q = s.q + dQ
        s.vstar = s.v.copy()
        r = residual_norm(prm, mesh, s)
        tau = min(tau_max, tau * norms[-1] / r) if r > 0 else tau_max
        norms.append(r)
    return s, norms, taus


def condense_uneven(prm, mesh, st, Ks, dvh=None, procs=1):
    """condense_elements for a batch of uneven p, m (inputs.UnevenMesh with
    flattened arrays): each element K of Ks as its own one-element problem
    (Algorithm 1, local parts), with its traces gathered from the flattened
    trace vectors.  Returns, per element, (b-hat^K [6,5,n2], dV^K [5,Nn] or
    None, dQ^K or None, seconds)."""
    from paper_2507_22195_gb300.inputs import State
    voff, toff = mesh.voff, mesh.toff
    out = []
    # one element per call of condense_elements, batched into one pool
    jobs = []
    for K in Ks:
        em = mesh.element_mesh(K)
        n2, Nn = em.n2, em.Nn
        vK = st.v[voff[K]:voff[K + 1]].reshape(1, 5, Nn)
        vsK = st.vstar[voff[K]:voff[K + 1]].reshape(1, 5, Nn)
        qK = None if st.q is None else st.q[3 * voff[K]:3 * voff[K + 1]].reshape(1, 5, 3, Nn)
        vh = np.stack([st.vhat[toff[g]:toff[g + 1]].reshape(5, n2) for g in mesh.face_gid[K]])
        dh = None if dvh is None else np.stack([dvh[toff[g]:toff[g + 1]].reshape(5, n2) for g in mesh.face_gid[K]])
        jobs.append((em, State(v=vK, vhat=vh, q=qK, vstar=vsK), dh))
    if procs <= 1:
        for em, s, dh in jobs:
            out.append(condense_elements(prm, em, s, [0], dh)[0])
        return out
    import multiprocessing as mp
    build()
    fields = tuple(getattr(prm, f) for f, _ in Params._fields_)
    args = []
    for em, s, dh in jobs:
        args.append((fields, em.p, em.m, em.boxes[0].copy(), np.ascontiguousarray(s.v[0]),
                     np.ascontiguousarray(s.vstar[0]), np.ascontiguousarray(s.vhat),
                     None if s.q is None else np.ascontiguousarray(s.q[0]),
                     None if dh is None else np.ascontiguousarray(dh).ravel()))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_condense_one, args)
    for (em, _, _), (bh, dV, dQ, t) in zip(jobs, res):
        out.append((bh.reshape(6, 5, em.n2), None if dV is None else dV.reshape(5, em.Nn),
                    None if dQ is None else dQ.reshape(5, 3, em.Nn), t))
    return out


def newton_vjp(prm_kw, mesh, st, nsteps, tau, gbar_v, gbar_vh, fd_step=1e-7):
    """Cotangent of the initial state (v0, vhat0) for the cotangent (gbar_v,
    gbar_vh) of the state after nsteps Newton steps with the stage term at
    v* = v_k and a fixed step tau (Sec. 6.1, eqs. C312, C31223; Euler):
    reverse recursion gbar_k = gbar_{k+1} - J_steady(s_k)^T lam - (d/de
    J(s_k + e d_k)^T lam)|0 with lam = J(s_k)^-T gbar_{k+1}, every J the
    monolithic complex-step Jacobian (J_steady without the stage term), the
    transposed solves by GEPP, the last term by central differences with
    h = fd_step max|s_k| / max|d_k|.  Returns (g_v0, g_vh0, final State).
    Tiny meshes only."""
    from paper_2507_22195_gb300.inputs import State
    prm = params(dt=tau, **prm_kw)
    prm_s = params(dt=tau, time_term=0, **prm_kw)
    v, vh = st.v.copy(), st.vhat.copy()
    traj = []
    for _ in range(nsteps):
        s = State(v=v, vhat=vh, q=None, vstar=v.copy())
        _, dV, dH = brute_force(prm, mesh, s)
        traj.append((v.copy(), vh.copy(), dV, dH))
        v, vh = v + dV, vh + dH
    g = np.concatenate([np.asarray(gbar_v).ravel(), np.asarray(gbar_vh).ravel()])
    for v0, vh0, dV, dH in reversed(traj):
        sk = State(v=v0, vhat=vh0, q=None, vstar=v0.copy())
        J, _ = _assemble(prm, mesh, sk)
        lam = solve(np.ascontiguousarray(J.T), g)
        Js, _ = _assemble(prm_s, mesh, sk)
        a = Js.T @ lam
        dm = max(np.abs(dV).max(), np.abs(dH).max())
        smax = max(np.abs(v0).max(), np.abs(vh0).max())
        h = fd_step * smax / dm
        Jp, _ = _assemble(prm, mesh, State(v=v0 + h * dV, vhat=vh0 + h * dH, q=None, vstar=v0.copy()))
        Jm, _ = _assemble(prm, mesh, State(v=v0 - h * dV, vhat=vh0 - h * dH, q=None, vstar=v0.copy()))
        g = g - a - (Jp.T @ lam - Jm.T @ lam) / (2 * h)
    nv = mesh.nK * 5 * mesh.Nn
    return (g[:nv].reshape(st.v.shape), g[nv:].reshape(st.vhat.shape),
            State(v=v, vhat=vh, q=None, vstar=v.copy()))



# ---------------------------------------------------------------- DIRK stages (Sec. 5.3)
def dirk33():
    """Butcher table (A, b, c) of the three-stage, third-order, L-stable,
    stiffly accurate DIRK method of Alexander (the DIRK(3,3) of Sec. 7):
    alpha is the root of x^3 - 3 x^2 + 3/2 x - 1/6 in (1/6, 1/2)."""
    # bisection for the root (no tabulated digits)
    lo, hi = 1.0 / 6.0, 0.5
    f = lambda x: x ** 3 - 3 * x ** 2 + 1.5 * x - 1.0 / 6.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(lo) * f(mid) <= 0:
            hi = mid
        else:
            lo = mid
    a = 0.5 * (lo + hi)
    t2 = (1 + a) / 2
    b1 = -(6 * a * a - 16 * a + 1) / 4
    b2 = (6 * a * a - 20 * a + 5) / 4
    A = np.array([[a, 0, 0], [t2 - a, a, 0], [b1, b2, a]])
    return A, np.array([b1, b2, a]), np.array([a, t2, 1.0])


def stage_difference(prm_kw, mesh, st, va, vb):
    """(u(va_h) - u(vb_h), w) over the volume quadrature, [K,5,Nn]: the
    stage term of eq. C242 at dt = 1, as the difference of two residuals whose
    other terms are identical (v = va, v* = vb against v* = va)."""
    from paper_2507_22195_gb300.inputs import State
    prm = params(dt=1.0, time_term=1, **prm_kw)
    r1, _, _ = residual_mesh(prm, mesh, State(v=va, vhat=st.vhat, q=st.q, vstar=vb))
    r0, _, _ = residual_mesh(prm, mesh, State(v=va, vhat=st.vhat, q=st.q, vstar=va))
    return r1 - r0


def dirk_step(prm_kw, mesh, st, dt, table=None, newton_tol=1e-11, newton_max=12):
    """One step of a stiffly accurate DIRK method (eqs. C241, C242) from the
    state st (v^n, vhat^n, q^n): stage i solves, by monolithic Newton,
      (d_ii / dt)(u(v) - u(v^n)) + sum_{j<i} (d_ij / dt)(u(v^{n,j}) - u(v^n))
        + spatial terms = 0       (tested against w; D = A^-1)
    i.e. the residual with the stage term at v* = v^n and step dt / d_ii plus
    the known stages as a source; u^{n+1} = u^{n,s} (e = b^T D = e_s for a
    stiffly accurate table).  Returns (state after the step, [stage states],
    [Newton iterations per stage])."""
    from paper_2507_22195_gb300.inputs import State
    A, b, c = dirk33() if table is None else table
    D = np.linalg.inv(A)
    s = A.shape[0]
    vn = st.v.copy()
    cur = State(v=st.v.copy(), vhat=st.vhat.copy(), q=None if st.q is None else st.q.copy(), vstar=vn)
    stages, its = [], []
    for i in range(s):
        src = np.zeros_like(vn)
        for j in range(i):
            src += D[i, j] / dt * stage_difference(prm_kw, mesh, cur, stages[j].v, vn)
        prm = params(dt=dt / D[i, i], **prm_kw)
        k = 0
        for k in range(newton_max):
            cur.vstar = vn
            RV, RQ, RH = residual_mesh(prm, mesh, cur)
            rn = np.sqrt(np.sum((RV + src) ** 2) + np.sum(RH ** 2) + (0 if RQ is None else np.sum(RQ ** 2)))
            if rn < newton_tol:
                break
            dQ, dV, dH = brute_force(prm, mesh, cur, src_V=src)
            cur.v = cur.v + dV
            cur.vhat = cur.vhat + dH
            if cur.q is not None:
                cur.q = cur.q + dQ
        its.append(k)
        stages.append(State(v=cur.v.copy(), vhat=cur.vhat.copy(), q=None if cur.q is None else cur.q.copy(),
                            vstar=vn))
    out = State(v=cur.v.copy(), vhat=cur.vhat.copy(), q=None if cur.q is None else cur.q.copy(), vstar=cur.v.copy())
    return out, stages, its
