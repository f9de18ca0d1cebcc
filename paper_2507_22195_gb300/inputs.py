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


# ---------------------------------------------------------------- uneven batches
@dataclasses.dataclass
class UnevenMesh:
    """Macro-elements of per-element degree p[K] and micro-element count
    m[K].  Arrays are flattened: element K's [5][Nn(K)] block of v starts at
    voff[K] (q: [5][3][Nn(K)] at 3 voff[K]), face g's [5][n_g^2] block of a
    trace vector at toff[g]."""
    p: np.ndarray
    m: np.ndarray
    boxes: np.ndarray
    face_gid: np.ndarray
    n_global_faces: int

    @property
    def nK(self) -> int:
        return len(self.p)

    def n(self, K) -> int:
        return int(self.m[K] * self.p[K] + 1)

    @property
    def voff(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([5 * self.n(K) ** 3 for K in range(self.nK)])]).astype(np.int64)

    @property
    def toff(self) -> np.ndarray:
        fn = np.zeros(self.n_global_faces, dtype=np.int64)
        for K in range(self.nK):
            fn[self.face_gid[K]] = self.n(K)
        return np.concatenate([[0], np.cumsum(5 * fn * fn)]).astype(np.int64)

    def element_mesh(self, K) -> Mesh:
        """element K alone, as a one-element mesh with unshared faces"""
        return Mesh(int(self.p[K]), int(self.m[K]), self.boxes[K:K + 1].copy(),
                    np.arange(6, dtype=np.int64).reshape(1, 6), 6)


def uneven_batch(nK: int, seed: int, p_choices=(1, 2, 3, 4), m_choices=(2, 3, 4), cells=8,
                 L=2 * math.pi, specs=None) -> UnevenMesh:
    """nK independent macro-elements (unshared faces), p and m drawn from the
    choices with the seed (or given as specs = [(p, m), ...]); each element is
    a cell of a cells^3 grid of [0, L]^3 at a seeded position, so the fields
    vary from element to element."""
    r = np.random.Generator(np.random.PCG64(seed))
    if specs is not None:
        nK = len(specs)
        p = np.array([s[0] for s in specs], dtype=np.int32)
        m = np.array([s[1] for s in specs], dtype=np.int32)
    else:
        p = r.choice(np.asarray(p_choices), size=nK).astype(np.int32)
        m = r.choice(np.asarray(m_choices), size=nK).astype(np.int32)
    pos = r.integers(0, cells, size=(nK, 3))
    h = L / cells
    boxes = np.concatenate([pos * h, (pos + 1) * h], axis=1).astype(np.float64)
    gid = np.arange(6 * nK, dtype=np.int64).reshape(nK, 6)
    return UnevenMesh(p, m, boxes, gid, 6 * nK)


def make_uneven_state(mesh: UnevenMesh, amp: float, seed_v: int, seed_vh: int, seed_M: int,
                      M0_range=(0.1, 0.3), viscous: bool = False) -> State:
    """TGV-like field per element with its own Mach number M0 ~ U(M0_range)
    (seed_M), plus U(-amp, amp) on v and, independently, on v-hat; v* = v; q
    = nodal samples of the analytic grad v of the unperturbed field.  Arrays
    are flattened with mesh.voff / mesh.toff."""
    voff, toff = mesh.voff, mesh.toff
    rM = np.random.Generator(np.random.PCG64(seed_M))
    M0 = rM.uniform(M0_range[0], M0_range[1], size=mesh.nK)
    v = np.zeros(voff[-1])
    q = np.zeros(3 * voff[-1]) if viscous else None
    vh = np.zeros(toff[-1])
    for K in range(mesh.nK):
        em = mesh.element_mesh(K)
        X, Y, Z = node_coords(em, 0)
        v[voff[K]:voff[K + 1]] = _field_v("tgv", X, Y, Z, M0=M0[K]).ravel()
        if viscous:
            q[3 * voff[K]:3 * voff[K + 1]] = _grad_v("tgv", X, Y, Z, M0=M0[K]).ravel()
        for f in range(6):
            g = mesh.face_gid[K, f]
            pts = face_coords(em, 0, f)
            vh[toff[g]:toff[g + 1]] = _field_v("tgv", pts[0], pts[1], pts[2], M0=M0[K]).ravel()
    rv = np.random.Generator(np.random.PCG64(seed_v))
    rh = np.random.Generator(np.random.PCG64(seed_vh))
    v = v + rv.uniform(-amp, amp, size=v.shape)
    vh = vh + rh.uniform(-amp, amp, size=vh.shape)
    return State(v=v, vhat=vh, q=q, vstar=v.copy())


def face_node_index(mesh: Mesh) -> np.ndarray:
    """[6][n^2] element node A = i + n (j + n k) of every trace node c = i_t1 +
    n i_t2 of local face f (x-, x+, y-, y+, z-, z+; (t1, t2) the two other
    axes in increasing order)."""
    n = mesh.n
    out = np.zeros((6, n * n), dtype=np.int64)
    for f in range(6):
        d, side = f // 2, f % 2
        t1, t2 = [(1, 2), (0, 2), (0, 1)][d]
        for b in range(n):
            for a in range(n):
                ijk = [0, 0, 0]
                ijk[d] = n - 1 if side else 0
                ijk[t1], ijk[t2] = a, b
                out[f, a + n * b] = ijk[0] + n * (ijk[1] + n * ijk[2])
    return out


def gll_weights(p: int) -> np.ndarray:
    """Gauss-Lobatto-Legendre weights on [-1, 1] (closed forms, p <= 4)."""
    return np.array({1: [1.0, 1.0], 2: [1 / 3, 4 / 3, 1 / 3], 3: [1 / 6, 5 / 6, 5 / 6, 1 / 6],
                     4: [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]}[p])
