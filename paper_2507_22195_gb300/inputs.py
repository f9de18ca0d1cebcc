"""Seeded synthetic inputs for the macro-element Newton step.

This module only builds inputs: meshes of axis-aligned macro-elements, nodal
entropy variables of closed-form flow fields, and seeded perturbations.  It is
shared by the tests, the benchmark and the oracle checks, and it holds none of
the hot path's arithmetic (no residual, flux, Jacobian or solve).

Fields (restated from the paper):
  * isentropic vortex, eq. S601, with the free stream (1,1,0), rho=P=1 at
    infinity, vortex strength eps, centre (5,5,5), axis z; the perturbation
    amplitude is eps/(2 pi) and M_inf^2 = 1/gamma so that P_inf = 1;
  * Taylor-Green vortex, eq. TGV0, acoustic scaling: rho0 = 1, P0 = 1/gamma,
    V0 = M0, isothermal rho = gamma P, on [0, 2 pi]^3 (a periodic shift of
    the paper's [-pi, pi]^3).
Entropy variables are eq. s222: v = [(gamma-s)/(gamma-1) - beta|V|^2/2,
beta V, -beta], beta = rho/P, s = ln(P/rho^gamma).

Layouts follow the C-ABI: v [K][5][Nn] with node i + n (j + n k); q
[K][5][3][Nn]; global trace [faces][5][n^2], face node c = i_t1 + n i_t2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4

# Gauss-Lobatto-Legendre nodes on [-1, 1] (closed forms, p <= 4), used only
# to place nodal samples of the input fields.
_GLL = {
    1: [-1.0, 1.0],
    2: [-1.0, 0.0, 1.0],
    3: [-1.0, -1.0 / math.sqrt(5.0), 1.0 / math.sqrt(5.0), 1.0],
    4: [-1.0, -math.sqrt(3.0 / 7.0), 0.0, math.sqrt(3.0 / 7.0), 1.0],
}


@dataclasses.dataclass
class Mesh:
    p: int
    m: int
    boxes: np.ndarray          # [K, 6] float64: x0 y0 z0 x1 y1 z1
    face_gid: np.ndarray       # [K, 6] int64 global face of each local face
    n_global_faces: int

    @property
    def nK(self) -> int:
        return self.boxes.shape[0]

    @property
    def n(self) -> int:
        return self.m * self.p + 1

    @property
    def Nn(self) -> int:
        return self.n ** 3

    @property
    def n2(self) -> int:
        return self.n ** 2


def periodic_mesh(nk: int | tuple, p: int, m: int, lo=0.0, hi=2 * math.pi) -> Mesh:
    """Structured periodic mesh of nk^3 (or nx*ny*nz) macro-elements on [lo,hi]^3."""
    if isinstance(nk, int):
        nk = (nk, nk, nk)
    nx, ny, nz = nk
    nK = nx * ny * nz
    L = hi - lo
    boxes = np.zeros((nK, 6))
    gid = np.zeros((nK, 6), dtype=np.int64)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                K = ix + nx * (iy + ny * iz)
                boxes[K] = [lo + L * ix / nx, lo + L * iy / ny, lo + L * iz / nz,
                            lo + L * (ix + 1) / nx, lo + L * (iy + 1) / ny, lo + L * (iz + 1) / nz]
                gid[K, 0] = ix + nx * (iy + ny * iz)
                gid[K, 1] = (ix + 1) % nx + nx * (iy + ny * iz)
                gid[K, 2] = nK + ix + nx * (iy + ny * iz)
                gid[K, 3] = nK + ix + nx * ((iy + 1) % ny + ny * iz)
                gid[K, 4] = 2 * nK + ix + nx * (iy + ny * iz)
                gid[K, 5] = 2 * nK + ix + nx * (iy + ny * ((iz + 1) % nz))
    return Mesh(p, m, boxes, gid, 3 * nK)


def sub_mesh(mesh: Mesh, Ks) -> Mesh:
    """The elements Ks of a mesh; faces shared inside the subset stay shared,
    the others become unshared faces (global face ids renumbered)."""
    Ks = np.asarray(Ks)
    gid = mesh.face_gid[Ks]
    uniq, inv = np.unique(gid, return_inverse=True)
    return Mesh(mesh.p, mesh.m, mesh.boxes[Ks].copy(), inv.reshape(gid.shape).astype(np.int64), len(uniq))


def block_elements(nk: int, b: int):
    """element ids of the b^3 corner block of an nk^3 structured mesh"""
    return [ix + nk * (iy + nk * iz) for iz in range(b) for iy in range(b) for ix in range(b)]


def independent_mesh(nK: int, p: int, m: int, size=1.0, seed=0) -> Mesh:
    """nK macro-elements with unshared faces (each face its own global face)."""
    boxes = np.zeros((nK, 6))
    for K in range(nK):
        boxes[K] = [0, 0, 0, size, size, size]
    gid = np.arange(6 * nK, dtype=np.int64).reshape(nK, 6)
    return Mesh(p, m, boxes, gid, 6 * nK)


def unshared(mesh: Mesh, Ks=None) -> Mesh:
    """The elements Ks of a mesh (default: all) with every face unshared:
    element K's local face f becomes global face 6 K' + f (K' = position in
    Ks).  The elements keep their boxes, so the input fields vary from
    element to element."""
    Ks = np.arange(mesh.nK) if Ks is None else np.asarray(Ks)
    nK = len(Ks)
    gid = np.arange(6 * nK, dtype=np.int64).reshape(nK, 6)
    return Mesh(mesh.p, mesh.m, mesh.boxes[Ks].copy(), gid, 6 * nK)


def node_coords_1d(lo: float, hi: float, p: int, m: int) -> np.ndarray:
    xi = np.array(_GLL[p])
    h = (hi - lo) / m
    n = m * p + 1
    x = np.zeros(n)
    for i in range(n):
        e = min(i // p, m - 1)
        l = i - e * p
        x[i] = lo + h * (e + (xi[l] + 1.0) / 2.0)
    return x


def node_coords(mesh: Mesh, K: int):
    b = mesh.boxes[K]
    xs = [node_coords_1d(b[d], b[3 + d], mesh.p, mesh.m) for d in range(3)]
    # node A = i + n (j + n k)  ->  arrays indexed [k, j, i]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def face_coords(mesh: Mesh, K: int, f: int):
    """Coordinates of the n^2 trace nodes of local face f of K (c = i_t1 + n i_t2)."""
    b = mesh.boxes[K]
    d = f // 2
    t1, t2 = [(1, 2), (0, 2), (0, 1)][d]
    x1 = node_coords_1d(b[t1], b[3 + t1], mesh.p, mesh.m)
    x2 = node_coords_1d(b[t2], b[3 + t2], mesh.p, mesh.m)
    C2, C1 = np.meshgrid(x2, x1, indexing="ij")
    pts = np.zeros((3, mesh.n2))
    pts[t1] = C1.ravel()
    pts[t2] = C2.ravel()
    pts[d] = b[3 + d] if f % 2 else b[d]
    return pts


# ---------------------------------------------------------------- fields
def entropy_vars(rho, V, P, gamma=GAMMA):
    """eq. s222 (inputs only)."""
    s = np.log(P / rho ** gamma)
    beta = rho / P
    V2 = V[0] ** 2 + V[1] ** 2 + V[2] ** 2
    return np.stack([(gamma - s) / (gamma - 1) - beta * V2 / 2,
                     beta * V[0], beta * V[1], beta * V[2], -beta])


def vortex_prim(x, y, z, t=0.0, eps=5.0, center=(5.0, 5.0, 5.0), vinf=(1.0, 1.0, 0.0),
                gamma=GAMMA, period=None):
    """Translating isentropic vortex (eq. S601 with M_inf^2 = 1/gamma)."""
    dx = x - center[0] - vinf[0] * t
    dy = y - center[1] - vinf[1] * t
    if period is not None:
        dx = (dx + period / 2) % period - period / 2
        dy = (dy + period / 2) % period - period / 2
    r2 = dx * dx + dy * dy
    Tt = 1.0 - eps ** 2 * (gamma - 1.0) / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = Tt ** (1.0 / (gamma - 1.0))
    amp = eps / (2.0 * math.pi) * np.exp((1.0 - r2) / 2.0)
    V = [vinf[0] - amp * dy, vinf[1] + amp * dx, vinf[2] + 0.0 * x]
    P = rho ** gamma
    return rho, V, P


def tgv_prim(x, y, z, M0=0.1, gamma=GAMMA):
    """Taylor-Green vortex initial field (eq. TGV0), acoustic scaling."""
    V0 = M0
    P0 = 1.0 / gamma
    V = [V0 * np.sin(x) * np.cos(y) * np.cos(z),
         -V0 * np.cos(x) * np.sin(y) * np.cos(z),
         0.0 * x]
    P = P0 + V0 ** 2 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = gamma * P          # isothermal: P/rho = P0/rho0
    return rho, V, P


def _field_v(kind, x, y, z, **kw):
    if kind == "vortex":
        rho, V, P = vortex_prim(x, y, z, **kw)
    elif kind == "tgv":
        rho, V, P = tgv_prim(x, y, z, **kw)
    elif kind == "const":
        rho = np.full_like(x, kw.get("rho", 1.0))
        V = [np.full_like(x, c) for c in kw.get("V", (0.3, -0.2, 0.1))]
        P = np.full_like(x, kw.get("P", 1.0))
    else:
        raise ValueError(kind)
    return entropy_vars(rho, V, P)


def _grad_v(kind, x, y, z, hfd=1e-5, **kw):
    """grad v of the closed-form field by 4th-order central differences, [5][3][N]."""
    g = np.zeros((5, 3) + x.shape)
    for d in range(3):
        def sh(s):
            xx = [x, y, z]
            xx = [c + (s * hfd if i == d else 0.0) for i, c in enumerate(xx)]
            return _field_v(kind, *xx, **kw)
        g[:, d] = (8 * (sh(1) - sh(-1)) - (sh(2) - sh(-2))) / (12 * hfd)
    return g


@dataclasses.dataclass
class State:
    v: np.ndarray          # [K,5,Nn]
    vhat: np.ndarray       # [G,5,n2]
    q: np.ndarray | None   # [K,5,3,Nn]
    vstar: np.ndarray      # [K,5,Nn]


def make_state(mesh: Mesh, kind: str, amp: float, seed_v: int, seed_vh: int,
               viscous: bool = False, **kw) -> State:
    """Nodal entropy variables of the field plus U(-amp, amp) perturbations
    (independent streams for v and v-hat); v* = unperturbed-plus-perturbed v;
    q = nodal samples of the analytic grad v of the unperturbed field."""
    nK, Nn, n2 = mesh.nK, mesh.Nn, mesh.n2
    v = np.zeros((nK, 5, Nn))
    q = np.zeros((nK, 5, 3, Nn)) if viscous else None
    for K in range(nK):
        X, Y, Z = node_coords(mesh, K)
        v[K] = _field_v(kind, X, Y, Z, **kw)
        if viscous:
            q[K] = _grad_v(kind, X, Y, Z, **kw)
    vh = np.zeros((mesh.n_global_faces, 5, n2))
    seen = np.zeros(mesh.n_global_faces, dtype=bool)
    for K in range(nK):
        for f in range(6):
            g = mesh.face_gid[K, f]
            if seen[g]:
                continue
            seen[g] = True
            pts = face_coords(mesh, K, f)
            vh[g] = _field_v(kind, pts[0], pts[1], pts[2], **kw)
    rv = np.random.Generator(np.random.PCG64(seed_v))
    rh = np.random.Generator(np.random.PCG64(seed_vh))
    v = v + rv.uniform(-amp, amp, size=v.shape)
    vh = vh + rh.uniform(-amp, amp, size=vh.shape)
    return State(v=np.ascontiguousarray(v), vhat=np.ascontiguousarray(vh), q=q,
                 vstar=np.ascontiguousarray(v.copy()))


def random_direction(shape, seed: int, amp: float = 1.0) -> np.ndarray:
    r = np.random.Generator(np.random.PCG64(seed))
    return r.uniform(-amp, amp, size=shape)
