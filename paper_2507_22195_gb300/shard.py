"""Sharding of one mesh over several ranks (one GPU each) for the global trace
system of Algorithm 1.

Every rank condenses its own macro-elements with its own context. The trace
residual R_V-hat, the condensed right-hand side b-hat (eq. R5b) and the
condensed product A-hat x (the four stages of Sec. 6.3) are sums over the
elements on both sides of every face (eq. s32c). A rank therefore holds the
whole sum on the faces inside its part, but only its own side on the faces it
shares with another rank. This module makes the parts and the plan of those
shared faces, then completes the sums with one point-to-point exchange per
neighbouring rank. It also reduces dot products over the trace unknowns,
counting every face once.

Trace vectors are torch tensors [faces][5][n^2] in the rank's local face
numbering (that of `inputs.sub_mesh`), on any device. The exchange uses
torch.distributed point-to-point operations posted together as one batch
(batch_isend_irecv), so that no rank's send waits behind its own receive;
it moves 5 n^2 values per shared face and does no arithmetic of the method
beyond the sums.  It is tested with gloo ranks on the host; the NCCL path
between GPUs has not been run (every run available here has one GPU).
"""
from __future__ import annotations

import numpy as np

from . import inputs as I


def partition(mesh: I.Mesh, world: int) -> list[np.ndarray]:
    """Contiguous slabs of elements, cut along the axis with the most distinct
    element positions: sizes differ by at most one element position.
    Returns the element ids of every rank, ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    centre = 0.5 * (mesh.boxes[:, :3] + mesh.boxes[:, 3:])
    levels = [np.unique(np.round(centre[:, a], 12)) for a in range(3)]
    axis = int(np.argmax([len(lv) for lv in levels]))
    lv = levels[axis]
    if len(lv) < world:
        raise ValueError(f"{len(lv)} element positions along the longest axis for {world} ranks")
    pos = np.searchsorted(lv, np.round(centre[:, axis], 12))
    cuts = np.linspace(0, len(lv), world + 1).round().astype(int)
    return [np.flatnonzero((pos >= cuts[r]) & (pos < cuts[r + 1])) for r in range(world)]


class Shard:
    """One rank's part of a mesh and the plan of its shared faces.

    elems    element ids of this rank (ascending), the local element order
    mesh     the local mesh (`inputs.sub_mesh`): local face j is global face gfaces[j]
    gfaces   global face id of every local face (ascending)
    peers    {rank: local face indices shared with that rank, ordered by global id}
    owned    [local faces] bool: this rank is the lowest rank touching the face
    """

    def __init__(self, mesh: I.Mesh, parts: list[np.ndarray], rank: int):
        self.rank, self.world = rank, len(parts)
        self.elems = np.asarray(parts[rank])
        self.mesh = I.sub_mesh(mesh, self.elems)
        self.gfaces = np.unique(mesh.face_gid[self.elems])
        touch: dict[int, set] = {}
        for r, el in enumerate(parts):
            for g in np.unique(mesh.face_gid[np.asarray(el)]):
                touch.setdefault(int(g), set()).add(r)
        self.peers: dict[int, np.ndarray] = {}
        owned = np.ones(len(self.gfaces), dtype=bool)
        for j, g in enumerate(self.gfaces):
            rs = touch[int(g)]
            if min(rs) != rank:
                owned[j] = False
            for r in rs:
                if r != rank:
                    self.peers.setdefault(r, []).append(j)
        # local faces are in ascending global order, so every peer list already
        # follows the global ids: both ranks send and receive in the same order
        self.peers = {r: np.asarray(v, dtype=np.int64) for r, v in sorted(self.peers.items())}
        self.owned = owned

    def local_state(self, st: I.State) -> I.State:
        """This rank's elements and faces of a global state (host arrays)."""
        return I.State(v=st.v[self.elems].copy(), vhat=st.vhat[self.gfaces].copy(),
                       q=None if st.q is None else st.q[self.elems].copy(),
                       vstar=st.vstar[self.elems].copy())

    def sum_shared(self, t, dist=None):
        """t [local faces][5][n^2]: add the other ranks' sides on the shared
        faces, in place; returns t.  No-op on a single rank.  With the gloo
        backend a device tensor is exchanged through host copies."""
        if dist is None or not self.peers:
            return t
        import torch
        if t.is_cuda and dist.get_backend() == "gloo":
            h = t.cpu()
            self.sum_shared(h, dist)
            t.copy_(h)
            return t
        sends, recvs, ops = [], [], []
        for r, idx in self.peers.items():
            ii = torch.as_tensor(idx, device=t.device)
            buf = t.index_select(0, ii).contiguous()
            got = torch.empty_like(buf)
            sends.append(buf)
            recvs.append((ii, got))
            ops.append(dist.P2POp(dist.isend, buf, r))
            ops.append(dist.P2POp(dist.irecv, got, r))
        for q in dist.batch_isend_irecv(ops):
            q.wait()
        for ii, got in recvs:
            t.index_add_(0, ii, got)
        return t

    def dot(self, a, b, dist=None) -> float:
        """Dot product over the global trace unknowns, every face counted once
        (by the lowest rank that touches it)."""
        import torch
        own = torch.as_tensor(self.owned, device=a.device)
        s = (a[own].to(torch.float64) * b[own].to(torch.float64)).sum().reshape(1)
        if dist is not None and self.world > 1:
            dist.all_reduce(s, op=dist.ReduceOp.SUM)
        return float(s.item())


class ShardedSystem:
    """One rank's part of the condensed trace system on its own GPU context:
    the rank condenses its elements (Algorithm 1, local parts), completes the
    face sums of b-hat and A-hat x with its neighbours (sum_shared), and takes
    part in a GMRES over the distributed trace vector whose dot products count
    every face once (dot).  Recovery is local (every element's faces are on
    its rank).  The vector arithmetic of the Krylov iteration on the rank's
    trace vector is torch on the device; the Hessenberg least-squares problem
    is host arithmetic, identical on every rank."""

    def __init__(self, shard, state, dist=None, device="cuda", **params):
        import torch
        from . import mehdg as M
        self.sh, self.dist = shard, dist
        self.ctx = M.Context(shard.mesh, **params)
        d = torch.device(device)
        self._st = [None if a is None else torch.tensor(a, device=d) for a in (state.v, state.vhat, state.q,
                                                                              state.vstar)]
        self.ctx.set_state(*self._st)

    def condense(self):
        return self.sh.sum_shared(self.ctx.condense(), self.dist)

    def apply(self, x):
        return self.sh.sum_shared(self.ctx.apply(x.contiguous()), self.dist)

    def recover(self, dvh):
        return self.ctx.recover(dvh.contiguous())

    def dot(self, a, b):
        return self.sh.dot(a, b, self.dist)

    def solve(self, b, rtol=1e-10, restart=30, max_iter=500):
        """restarted GMRES on sum_K A-hat^K x = b (classical Gram-Schmidt applied
        twice); returns (x, products, relative residual)"""
        import math
        import torch
        x = torch.zeros_like(b)
        bn = math.sqrt(max(self.dot(b, b), 1e-300))
        r = b - self.apply(x)
        beta = math.sqrt(self.dot(r, r))
        it, res = 0, beta / bn
        while res > rtol and it < max_iter:
            V = [r / beta]
            H = [[0.0] * restart for _ in range(restart + 1)]
            cs, sn, g = [0.0] * restart, [0.0] * restart, [0.0] * (restart + 1)
            g[0] = beta
            j = 0
            while j < restart and it < max_iter:
                w = self.apply(V[j])
                it += 1
                for _ in range(2):
                    h = [self.dot(V[i], w) for i in range(j + 1)]
                    for i in range(j + 1):
                        w = w - h[i] * V[i]
                        H[i][j] += h[i]
                hn = math.sqrt(max(self.dot(w, w), 0.0))
                H[j + 1][j] = hn
                V.append(w / hn if hn > 0 else w)
                for i in range(j):
                    a_, b_ = H[i][j], H[i + 1][j]
                    H[i][j], H[i + 1][j] = cs[i] * a_ + sn[i] * b_, -sn[i] * a_ + cs[i] * b_
                rr = math.hypot(H[j][j], H[j + 1][j])
                cs[j], sn[j] = (H[j][j] / rr, H[j + 1][j] / rr) if rr > 0 else (1.0, 0.0)
                H[j][j], H[j + 1][j] = rr, 0.0
                g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
                j += 1
                res = abs(g[j]) / bn
                if res <= rtol or hn == 0:
                    break
            y = [0.0] * j
            for i in range(j - 1, -1, -1):
                y[i] = (g[i] - sum(H[i][k] * y[k] for k in range(i + 1, j))) / H[i][i] if H[i][i] else 0.0
            for i in range(j):
                x = x + y[i] * V[i]
            r = b - self.apply(x)
            beta = math.sqrt(self.dot(r, r))
            res = beta / bn
            if beta == 0:
                break
        return x, it, res

    def close(self):
        self.ctx.close()
