"""Thin Python binding of the C-ABI in include/mehdg.h (argument marshalling
only; every step of the Newton step runs in libmehdg.so's CUDA kernels).

The functions keep the C names.  Device arrays are torch CUDA tensors (FP64,
contiguous); mesh arrays are numpy arrays.  ``stream`` defaults to the
current torch stream.  Loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmehdg.so")

MEHDG_FLUX_EC, MEHDG_FLUX_ES, MEHDG_FLUX_KEPES = 0, 1, 2
MEHDG_FP64, MEHDG_MIXED_TF32, MEHDG_MIXED_BF16, MEHDG_MIXED_TF32X3, MEHDG_MIXED_BF16X3 = 0, 1, 2, 3, 4
ERRORS = {0: "MEHDG_OK", -1: "MEHDG_EINVAL", -2: "MEHDG_ENONPHYS", -3: "MEHDG_ESINGULAR",
          -4: "MEHDG_ENOCONV", -5: "MEHDG_ECUDA", -6: "MEHDG_ENOMEM", -7: "MEHDG_ESTATE",
          -8: "MEHDG_ETIMEOUT"}
PHASES = ["residual", "jacobian", "lu_panels", "lu_trailing_update", "solve", "tangent", "lu_pack_outer"]

EXPORTED = ["mehdg_default_params", "mehdg_create", "mehdg_set_mesh", "mehdg_set_state",
            "mehdg_residual", "mehdg_condense", "mehdg_apply_condensed", "mehdg_recover",
            "mehdg_status", "mehdg_last_error", "mehdg_destroy", "mehdg_profile_enable",
            "mehdg_profile_read", "mehdg_launch_count", "mehdg_test_trailing_update",
            "mehdg_test_trailing_work_bytes", "mehdg_residual_static", "mehdg_solve_condensed",
            "mehdg_residual_vjp", "mehdg_status_device", "mehdg_set_dt", "mehdg_pseudo_time_newton",
            "mehdg_batch_layout", "mehdg_batch_autotune", "mehdg_batch_report", "mehdg_condense_adjoint",
            "mehdg_apply_condensed_adjoint", "mehdg_solve_condensed_adjoint", "mehdg_recover_adjoint",
            "mehdg_pseudo_time_newton_vjp", "mehdg_set_source", "mehdg_dirk_step", "mehdg_condense_graph"]


class mehdg_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("Re", C.c_double), ("Pr", C.c_double), ("Mach", C.c_double),
                ("dt", C.c_double), ("viscous", C.c_int), ("flux", C.c_int), ("prec", C.c_int),
                ("refine_tol", C.c_double), ("refine_max_iter", C.c_int), ("time_term", C.c_int)]


class MehdgError(RuntimeError):
    pass


_lib = None
_vp = C.c_void_p


def load(path: str | None = None):
    """Load libmehdg.so (built by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise MehdgError(f"{p} is missing: build it with paper_2507_22195_gb300.build.build()")
    L = C.CDLL(p)
    L.mehdg_default_params.argtypes = [C.POINTER(mehdg_params)]
    L.mehdg_default_params.restype = None
    L.mehdg_create.argtypes = [C.POINTER(_vp), C.POINTER(mehdg_params)]
    L.mehdg_set_mesh.argtypes = [_vp, C.c_int64, _vp, _vp, _vp, _vp, C.c_int64]
    L.mehdg_set_state.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.mehdg_residual.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.mehdg_condense.argtypes = [_vp, _vp, _vp, _vp]
    L.mehdg_apply_condensed.argtypes = [_vp, _vp, _vp, _vp]
    L.mehdg_recover.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.mehdg_status.argtypes = [_vp, _vp, _vp]
    L.mehdg_status_device.argtypes = [_vp, _vp, _vp, _vp]
    L.mehdg_set_dt.argtypes = [_vp, C.c_double]
    L.mehdg_batch_layout.argtypes = [_vp, _vp, _vp]
    L.mehdg_condense_adjoint.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.mehdg_apply_condensed_adjoint.argtypes = [_vp, _vp, _vp, _vp]
    L.mehdg_solve_condensed_adjoint.argtypes = [_vp, _vp, _vp, C.c_double, C.c_int, C.c_int, _vp, _vp, _vp]
    L.mehdg_recover_adjoint.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.mehdg_set_source.argtypes = [_vp, _vp]
    L.mehdg_condense_graph.argtypes = [_vp, _vp, _vp]
    L.mehdg_dirk_step.argtypes = [_vp, _vp, _vp, _vp, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                                  _vp, _vp, _vp]
    L.mehdg_pseudo_time_newton_vjp.argtypes = [_vp, _vp, _vp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                               _vp, _vp, _vp, _vp, C.c_double, _vp]
    L.mehdg_batch_autotune.argtypes = [_vp, C.c_int64, _vp]
    L.mehdg_batch_report.argtypes = [_vp, _vp, C.c_size_t]
    L.mehdg_pseudo_time_newton.argtypes = [_vp, _vp, _vp, _vp, C.c_int, C.c_double, C.c_double, C.c_double,
                                           C.c_int, C.c_int, _vp, _vp, _vp, _vp]
    L.mehdg_solve_condensed.argtypes = [_vp, _vp, _vp, C.c_double, C.c_int, C.c_int, _vp, _vp, _vp]
    L.mehdg_residual_vjp.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.mehdg_last_error.argtypes = [_vp]
    L.mehdg_last_error.restype = C.c_char_p
    L.mehdg_destroy.argtypes = [_vp]
    L.mehdg_destroy.restype = None
    L.mehdg_profile_enable.argtypes = [_vp, C.c_int]
    L.mehdg_profile_read.argtypes = [_vp, _vp, _vp, _vp, C.c_int]
    L.mehdg_launch_count.argtypes = []
    L.mehdg_launch_count.restype = C.c_int64
    L.mehdg_test_trailing_update.argtypes = [C.c_int64, C.c_int64, _vp, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_int, C.c_int, C.c_int, _vp, _vp]
    L.mehdg_test_trailing_work_bytes.argtypes = [C.c_int64, C.c_int64]
    L.mehdg_test_trailing_work_bytes.restype = C.c_size_t
    L.mehdg_residual_static.argtypes = [C.POINTER(mehdg_params), C.c_int64, C.c_int, C.c_int, _vp, _vp,
                                        C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        import torch
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), (t.device, t.dtype)
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(ctx, rc, what):
    if rc != 0:
        msg = load().mehdg_last_error(ctx).decode() if ctx else ""
        raise MehdgError(f"{what}: {ERRORS.get(rc, rc)}: {msg}")


def mehdg_default_params(**overrides) -> mehdg_params:
    p = mehdg_params()
    load().mehdg_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def mehdg_create(params: mehdg_params):
    h = _vp()
    _check(None, load().mehdg_create(C.byref(h), C.byref(params)), "mehdg_create")
    return h.value


def mehdg_set_mesh(ctx, p, m, box, face_gid, n_global_faces):
    p = np.ascontiguousarray(p, dtype=np.int32)
    m = np.ascontiguousarray(m, dtype=np.int32)
    box = np.ascontiguousarray(box, dtype=np.float64)
    gid = np.ascontiguousarray(face_gid, dtype=np.int64)
    _check(ctx, load().mehdg_set_mesh(ctx, len(p), p.ctypes.data, m.ctypes.data, box.ctypes.data,
                                      gid.ctypes.data, int(n_global_faces)), "mehdg_set_mesh")


def mehdg_set_state(ctx, v, vhat, q, vstar, stream=None):
    _check(ctx, load().mehdg_set_state(ctx, _ptr(v), _ptr(vhat), _ptr(q), _ptr(vstar), _stream(stream)),
           "mehdg_set_state")


def mehdg_residual(ctx, R_V, R_Q, R_Vhat, stream=None):
    _check(ctx, load().mehdg_residual(ctx, _ptr(R_V), _ptr(R_Q), _ptr(R_Vhat), _stream(stream)),
           "mehdg_residual")


def mehdg_solve_condensed(ctx, bhat, dVhat, rtol=1e-10, restart=30, max_iter=500, stream=None, check=True):
    """GMRES on sum A-hat dVhat = bhat; dVhat (device) holds the initial guess
    and receives the iterate.  Returns (products used, relative residual)."""
    it = C.c_int(0)
    res = C.c_double(0.0)
    rc = load().mehdg_solve_condensed(ctx, _ptr(bhat), _ptr(dVhat), float(rtol), int(restart), int(max_iter),
                                      C.byref(it), C.byref(res), _stream(stream))
    if check:
        _check(ctx, rc, "mehdg_solve_condensed")
    return it.value, res.value


def mehdg_residual_vjp(ctx, lam_V, lam_Vhat, g_v, g_vhat, stream=None):
    _check(ctx, load().mehdg_residual_vjp(ctx, _ptr(lam_V), _ptr(lam_Vhat), _ptr(g_v), _ptr(g_vhat),
                                          _stream(stream)), "mehdg_residual_vjp")


def mehdg_condense(ctx, bhat, Ahat_local=None, stream=None):
    _check(ctx, load().mehdg_condense(ctx, _ptr(bhat), _ptr(Ahat_local), _stream(stream)), "mehdg_condense")


def mehdg_condense_graph(ctx, bhat, stream=None):
    _check(ctx, load().mehdg_condense_graph(ctx, _ptr(bhat), _stream(stream)), "mehdg_condense_graph")


def mehdg_apply_condensed(ctx, x, y, stream=None):
    _check(ctx, load().mehdg_apply_condensed(ctx, _ptr(x), _ptr(y), _stream(stream)), "mehdg_apply_condensed")


def mehdg_recover(ctx, dVhat, dV, dQ=None, stream=None):
    _check(ctx, load().mehdg_recover(ctx, _ptr(dVhat), _ptr(dV), _ptr(dQ), _stream(stream)), "mehdg_recover")


def mehdg_status(ctx, nK):
    st = np.zeros(nK, dtype=np.int32)
    it = np.zeros(nK, dtype=np.int32)
    _check(ctx, load().mehdg_status(ctx, st.ctypes.data, it.ctypes.data), "mehdg_status")
    return st, it


def mehdg_status_device(ctx, status, iters=None, stream=None):
    """status, iters: int32 CUDA tensors [nK], filled asynchronously on the stream"""
    import torch
    for t in (status, iters):
        assert t is None or (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous())
    _check(ctx, load().mehdg_status_device(ctx, status.data_ptr(), None if iters is None else iters.data_ptr(),
                                           _stream(stream)), "mehdg_status_device")


def mehdg_set_dt(ctx, dt):
    _check(ctx, load().mehdg_set_dt(ctx, float(dt)), "mehdg_set_dt")


def mehdg_pseudo_time_newton(ctx, v, vhat, q, nsteps, tau_init=1.0, tau_max=1e8, lin_rtol=1e-10, restart=30,
                             max_iter=500, stream=None):
    """Pseudo-transient Newton steps on the device state (updated in place).
    Returns (residual norms [nsteps+1], taus [nsteps], GMRES products [nsteps])."""
    rn = np.zeros(nsteps + 1)
    ta = np.zeros(max(nsteps, 1))
    li = np.zeros(max(nsteps, 1), dtype=np.int32)
    _check(ctx, load().mehdg_pseudo_time_newton(ctx, _ptr(v), _ptr(vhat), _ptr(q), int(nsteps), float(tau_init),
                                                float(tau_max), float(lin_rtol), int(restart), int(max_iter),
                                                rn.ctypes.data, ta.ctypes.data, li.ctypes.data, _stream(stream)),
           "mehdg_pseudo_time_newton")
    return rn, ta[:nsteps], li[:nsteps]


def mehdg_condense_adjoint(ctx, g_V, g_Vhat, bhat_a, stream=None):
    _check(ctx, load().mehdg_condense_adjoint(ctx, _ptr(g_V), _ptr(g_Vhat), _ptr(bhat_a), _stream(stream)),
           "mehdg_condense_adjoint")


def mehdg_apply_condensed_adjoint(ctx, x, y, stream=None):
    _check(ctx, load().mehdg_apply_condensed_adjoint(ctx, _ptr(x), _ptr(y), _stream(stream)),
           "mehdg_apply_condensed_adjoint")


def mehdg_solve_condensed_adjoint(ctx, bhat_a, x, rtol=1e-10, restart=30, max_iter=500, stream=None, check=True):
    it = C.c_int(0)
    res = C.c_double(0.0)
    rc = load().mehdg_solve_condensed_adjoint(ctx, _ptr(bhat_a), _ptr(x), float(rtol), int(restart), int(max_iter),
                                              C.byref(it), C.byref(res), _stream(stream))
    if check:
        _check(ctx, rc, "mehdg_solve_condensed_adjoint")
    return it.value, res.value


def mehdg_recover_adjoint(ctx, g_V, lam_Vhat, lam_V, stream=None):
    _check(ctx, load().mehdg_recover_adjoint(ctx, _ptr(g_V), _ptr(lam_Vhat), _ptr(lam_V), _stream(stream)),
           "mehdg_recover_adjoint")


def mehdg_pseudo_time_newton_vjp(ctx, v, vhat, nsteps, tau, gbar_v, gbar_vhat, g_v0, g_vhat0, lin_rtol=1e-12,
                                 restart=30, max_iter=1000, fd_step=1e-7, stream=None):
    _check(ctx, load().mehdg_pseudo_time_newton_vjp(ctx, _ptr(v), _ptr(vhat), int(nsteps), float(tau), float(lin_rtol),
                                                    int(restart), int(max_iter), _ptr(gbar_v), _ptr(gbar_vhat),
                                                    _ptr(g_v0), _ptr(g_vhat0), float(fd_step), _stream(stream)),
           "mehdg_pseudo_time_newton_vjp")


def mehdg_set_source(ctx, src):
    _check(ctx, load().mehdg_set_source(ctx, _ptr(src)), "mehdg_set_source")


def mehdg_dirk_step(ctx, v, vhat, q, dt, newton_tol=1e-11, newton_max=12, lin_rtol=1e-12, restart=30, max_iter=2000,
                    stream=None):
    """One DIRK(3,3) step on the device state (in place); returns (Newton
    steps per stage, final residual norm per stage)."""
    its = np.zeros(3, dtype=np.int32)
    rn = np.zeros(3)
    _check(ctx, load().mehdg_dirk_step(ctx, _ptr(v), _ptr(vhat), _ptr(q), float(dt), float(newton_tol),
                                       int(newton_max), float(lin_rtol), int(restart), int(max_iter),
                                       its.ctypes.data, rn.ctypes.data, _stream(stream)), "mehdg_dirk_step")
    return its, rn


def mehdg_batch_layout(ctx, nK, G):
    """host offsets (voff [nK+1], toff [G+1]) of a batch context's arrays"""
    voff = np.zeros(nK + 1, dtype=np.int64)
    toff = np.zeros(G + 1, dtype=np.int64)
    _check(ctx, load().mehdg_batch_layout(ctx, voff.ctypes.data, toff.ctypes.data), "mehdg_batch_layout")
    return voff, toff


def mehdg_batch_autotune(ctx, trial_max=16, stream=None):
    _check(ctx, load().mehdg_batch_autotune(ctx, int(trial_max), _stream(stream)), "mehdg_batch_autotune")


def mehdg_batch_report(ctx) -> dict:
    import json
    n = load().mehdg_batch_report(ctx, None, 0)
    if n < 0:
        _check(ctx, n, "mehdg_batch_report")
    buf = C.create_string_buffer(n + 1)
    load().mehdg_batch_report(ctx, buf, n + 1)
    return json.loads(buf.value.decode())


def mehdg_last_error(ctx) -> str:
    return load().mehdg_last_error(ctx).decode()


def mehdg_destroy(ctx):
    load().mehdg_destroy(ctx)


def mehdg_profile_enable(ctx, enable=True):
    _check(ctx, load().mehdg_profile_enable(ctx, int(enable)), "mehdg_profile_enable")


def mehdg_profile_read(ctx):
    n = len(PHASES)
    ms, cnt, fl = np.zeros(n), np.zeros(n, dtype=np.int64), np.zeros(n)
    _check(ctx, load().mehdg_profile_read(ctx, ms.ctypes.data, cnt.ctypes.data, fl.ctypes.data, n),
           "mehdg_profile_read")
    return {PHASES[i]: dict(ms=float(ms[i]), launches=int(cnt[i]), flops=float(fl[i])) for i in range(n)}


def mehdg_test_trailing_update(S, r0, c0, k0, M, N, Kd, prec, work=None, stream=None):
    """S: torch float32 CUDA tensor [nK][ld][ld] holding column-major matrices
    (element [K][j][i] is row i, column j)."""
    import torch
    assert S.is_cuda and S.dtype == torch.float32 and S.is_contiguous()
    nK, ld = S.shape[0], S.shape[1]
    if work is None:
        nb = load().mehdg_test_trailing_work_bytes(nK, ld)
        work = torch.empty(nb, dtype=torch.uint8, device=S.device)
    _check(None, load().mehdg_test_trailing_update(nK, ld, S.data_ptr(), r0, c0, k0, M, N, Kd, prec,
                                                   work.data_ptr(), _stream(stream)),
           "mehdg_test_trailing_update")


def mehdg_residual_static(params, p, m, box, face_gid, n_global_faces, v, vhat, q, vstar, R_V, R_Q, R_Vhat,
                          stream=None):
    """Allocation-free residual: every array is a caller-owned CUDA tensor
    (box float64 [nK,6], face_gid int64 [nK,6], the rest float64)."""
    import torch
    assert box.is_cuda and box.dtype == torch.float64 and face_gid.is_cuda and face_gid.dtype == torch.int64
    nK = box.shape[0]
    rc = load().mehdg_residual_static(C.byref(params), nK, p, m, box.data_ptr(), face_gid.data_ptr(),
                                      int(n_global_faces), _ptr(v), _ptr(vhat), _ptr(q), _ptr(vstar), _ptr(R_V),
                                      _ptr(R_Q), _ptr(R_Vhat), _stream(stream))
    _check(None, rc, "mehdg_residual_static")


def mehdg_launch_count() -> int:
    return int(load().mehdg_launch_count())


class Context:
    """Owner of one library context over a mesh (see inputs.Mesh)."""

    def __init__(self, mesh, **params):
        self.mesh = mesh
        self.params = mehdg_default_params(**params)
        self.ctx = mehdg_create(self.params)
        nK = mesh.nK
        mehdg_set_mesh(self.ctx, np.full(nK, mesh.p), np.full(nK, mesh.m), mesh.boxes, mesh.face_gid,
                       mesh.n_global_faces)
        self._state = None

    def close(self):
        if self.ctx:
            mehdg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, v, vhat, q=None, vstar=None):
        self._state = (v, vhat, q, vstar)      # keep the tensors alive
        mehdg_set_state(self.ctx, v, vhat, q, vstar)

    def residual(self):
        import torch
        m = self.mesh
        dev = self._state[0].device
        RV = torch.empty((m.nK, 5, m.Nn), dtype=torch.float64, device=dev)
        RQ = torch.empty((m.nK, 5, 3, m.Nn), dtype=torch.float64, device=dev) if self.params.viscous else None
        RH = torch.empty((m.n_global_faces, 5, m.n2), dtype=torch.float64, device=dev)
        mehdg_residual(self.ctx, RV, RQ, RH)
        return RV, RQ, RH

    def condense(self, bhat=None):
        import torch
        m = self.mesh
        if bhat is None:
            bhat = torch.empty((m.n_global_faces, 5, m.n2), dtype=torch.float64, device=self._state[0].device)
        mehdg_condense(self.ctx, bhat)
        return bhat

    def apply(self, x):
        import torch
        y = torch.empty_like(x)
        mehdg_apply_condensed(self.ctx, x, y)
        return y

    def solve_condensed(self, bhat, x0=None, rtol=1e-10, restart=30, max_iter=500):
        """global trace solve (GMRES); returns (dVhat, products, relative residual)"""
        import torch
        x = torch.zeros_like(bhat) if x0 is None else x0.clone()
        it, res = mehdg_solve_condensed(self.ctx, bhat, x, rtol, restart, max_iter)
        return x, it, res

    def residual_vjp(self, lam_V, lam_Vhat=None):
        """(g_v, g_vhat): the residual's VJP at the current state (Euler)"""
        import torch
        m = self.mesh
        gv = torch.empty((m.nK, 5, m.Nn), dtype=torch.float64, device=lam_V.device)
        gh = torch.empty((m.n_global_faces, 5, m.n2), dtype=torch.float64, device=lam_V.device)
        mehdg_residual_vjp(self.ctx, lam_V, lam_Vhat, gv, gh)
        return gv, gh

    def recover(self, dvh, with_dQ=False, out=None):
        import torch
        m = self.mesh
        dV = torch.empty((m.nK, 5, m.Nn), dtype=torch.float64, device=dvh.device) if out is None else out
        dQ = torch.empty((m.nK, 5, 3, m.Nn), dtype=torch.float64, device=dvh.device) if self.params.viscous else None
        mehdg_recover(self.ctx, dvh, dV, dQ)
        return (dV, dQ) if with_dQ else dV

    def status(self):
        return mehdg_status(self.ctx, self.mesh.nK)


class BatchContext:
    """Owner of one library context over macro-elements of uneven p and m
    (inputs.UnevenMesh); arrays are flattened with mesh.voff / mesh.toff."""

    def __init__(self, mesh, **params):
        self.mesh = mesh
        self.params = mehdg_default_params(**params)
        self.ctx = mehdg_create(self.params)
        mehdg_set_mesh(self.ctx, mesh.p, mesh.m, mesh.boxes, mesh.face_gid, mesh.n_global_faces)
        self.voff, self.toff = mehdg_batch_layout(self.ctx, mesh.nK, mesh.n_global_faces)
        assert (self.voff == mesh.voff).all() and (self.toff == mesh.toff).all()
        self._state = None

    close = Context.close
    __del__ = Context.__del__
    status = Context.status

    def set_state(self, v, vhat, q=None, vstar=None):
        self._state = (v, vhat, q, vstar)
        mehdg_set_state(self.ctx, v, vhat, q, vstar)

    def _t(self, n):
        import torch
        return torch.empty(n, dtype=torch.float64, device=self._state[0].device)

    def residual(self):
        RV, RH = self._t(self.voff[-1]), self._t(self.toff[-1])
        RQ = self._t(3 * self.voff[-1]) if self.params.viscous else None
        mehdg_residual(self.ctx, RV, RQ, RH)
        return RV, RQ, RH

    def condense(self, bhat=None):
        bhat = self._t(self.toff[-1]) if bhat is None else bhat
        mehdg_condense(self.ctx, bhat)
        return bhat

    def apply(self, x):
        import torch
        y = torch.empty_like(x)
        mehdg_apply_condensed(self.ctx, x, y)
        return y

    def recover(self, dvh, with_dQ=False):
        dV = self._t(self.voff[-1])
        dQ = self._t(3 * self.voff[-1]) if self.params.viscous else None
        mehdg_recover(self.ctx, dvh, dV, dQ)
        return (dV, dQ) if with_dQ else dV

    def autotune(self, trial_max=16):
        mehdg_batch_autotune(self.ctx, trial_max)

    def report(self):
        return mehdg_batch_report(self.ctx)


def residual_function():
    """torch.autograd.Function: (R_V, R_Vhat) = residual(v, vhat) of an Euler
    Context at a fixed v*, with the backward pass through mehdg_residual_vjp."""
    import torch

    class Residual(torch.autograd.Function):
        @staticmethod
        def forward(fctx, v, vhat, context, vstar):
            context.set_state(v.detach().contiguous(), vhat.detach().contiguous(), None, vstar)
            RV, _, RH = context.residual()
            fctx.context = context
            fctx.save_for_backward(v, vhat, vstar)
            return RV, RH

        @staticmethod
        def backward(fctx, gRV, gRH):
            v, vhat, vstar = fctx.saved_tensors
            context = fctx.context
            context.set_state(v.detach().contiguous(), vhat.detach().contiguous(), None, vstar)
            gv, gh = context.residual_vjp(gRV.contiguous(), None if gRH is None else gRH.contiguous())
            return gv, gh, None, None

    return Residual
