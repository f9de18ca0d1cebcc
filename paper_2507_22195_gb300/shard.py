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
        faces, in place; returns t.  No-op on a single rank."""
        if dist is None or not self.peers:
            return t
        import torch
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
