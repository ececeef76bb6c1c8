"""Partitioned meshes: halo bookkeeping and the exchanges between the phases
of an evaluation (paper Sec. 2.1: space-filling-curve subdomains, one per
rank and GPU, with the face data of the subdomain boundaries exchanged).

The library evaluates a partitioned context in three phases (``dg.h``):
phase 1 packs the state traces of the halo faces, phase 2 runs the lifting
and packs the viscous-flux traces, phase 4 evaluates the face fluxes and the
volume kernel.  Its adjoint runs in four phases around three exchanges
(state traces; the cotangents of the viscous-flux traces; the cotangents of
the state traces).  Between them every rank sends each peer the rows of the
faces they share; both ranks list those faces in the same order, so the
exchange is a block copy per peer.

Two transports:
  * ``exchange`` -- torch.distributed point-to-point messages (NCCL for device
    tensors, gloo for host tensors), one rank per process;
  * ``LocalRanks`` -- several ranks' contexts in one process (one GPU), the
    exchange done by device copies; no kernel waits on another.
"""
import numpy as np

from . import dg


def peer_blocks(halo):
    """{peer: (first, last + 1)} rows of a halo list (grouped by peer)."""
    out = {}
    for h, peer in enumerate(np.asarray(halo)[:, 0] if len(halo) else []):
        a, b = out.get(int(peer), (h, h))
        out[int(peer)] = (min(a, h), h + 1)
    return out


def local_coordinates(X, l2g):
    """Node coordinates [3][K_local][n^3] of a rank's elements."""
    return np.ascontiguousarray(np.asarray(X)[:, l2g, :])


def local_state(U, l2g):
    return np.ascontiguousarray(np.asarray(U)[:, l2g, :])


def exchange(send, recv, halo, group=None):
    """Send every peer its rows of ``send`` and receive its rows into ``recv``
    (torch.distributed isend / irecv)."""
    import torch.distributed as dist
    reqs = []
    for peer, (a, b) in sorted(peer_blocks(halo).items()):
        reqs.append(dist.irecv(recv[a:b], src=peer, group=group))
        reqs.append(dist.isend(send[a:b].contiguous(), dst=peer, group=group))
    for r in reqs:
        r.wait()


class LocalRanks:
    """The contexts of all ranks of a partition in one process.

    ops[r] is rank r's dg.Operator on its local mesh; stage() and
    time_derivative() run the three phases on every rank with the halo
    exchanges between them as device copies."""

    def __init__(self, N, X, nbr, phys, nranks, part=None, nbr_face=None, orient=None, **opts):
        self.N = N
        self.part = dg.partition_sfc(N, X, nranks) if part is None else np.asarray(part, dtype=np.int32)
        self.nranks = nranks
        self.l2g, self.halo, self.ops = [], [], []
        for r in range(nranks):
            l2g, nbl, nfl, orl, halo = dg.partition_local(nbr, self.part, r, nbr_face, orient)
            self.l2g.append(l2g)
            self.halo.append(halo)
            self.ops.append(dg.Operator(N, local_coordinates(X, l2g), nbl, phys, nbr_face=nfl, orient=orl, **opts))
        self.buf = [op.halo_buffers() for op in self.ops]
        # the slave side of each halo face takes the master's normals
        geo = [op.halo_geometry() for op in self.ops]
        for r in range(nranks):
            if len(self.halo[r]) == 0:
                continue
            g = geo[r].copy()
            for q, (a, b) in peer_blocks(self.halo[r]).items():
                qa, qb = peer_blocks(self.halo[q])[r]
                g[a:b] = geo[q][qa:qb]
            self.ops[r].set_halo_geometry(g)

    def _move(self, key_send, key_recv):
        for r in range(self.nranks):
            for q, (a, b) in peer_blocks(self.halo[r]).items():
                qa, qb = peer_blocks(self.halo[q])[r]
                self.buf[r][key_recv][a:b].copy_(self.buf[q][key_send][qa:qb])

    def set_state(self, U):
        import torch
        for r, op in enumerate(self.ops):
            Ul = U[:, torch.as_tensor(self.l2g[r], device=U.device, dtype=torch.long), :].contiguous()
            op.set_state(Ul)

    def get_state(self, U):
        import torch
        for r, op in enumerate(self.ops):
            Ul = torch.empty((5, len(self.l2g[r]), U.shape[2]), dtype=U.dtype, device=U.device)
            op.get_state(Ul)
            U[:, torch.as_tensor(self.l2g[r], device=U.device, dtype=torch.long), :] = Ul

    def stage(self, s, t, dt):
        for op in self.ops:
            op.stage_phase(1, s, t, dt)
        self._move("send_U", "recv_U")
        for op in self.ops:
            op.stage_phase(2, s, t, dt)
        self._move("send_G", "recv_G")
        for op in self.ops:
            op.stage_phase(4, s, t, dt)

    def steps(self, t, dt, nsteps):
        for it in range(nsteps):
            for s in range(5):
                self.stage(s, t, dt)

    def time_derivative(self, Ut, U):
        """Ut, U: device tensors [5][K][n^3] of the whole mesh."""
        import torch
        loc = []
        for r, op in enumerate(self.ops):
            idx = torch.as_tensor(self.l2g[r], device=U.device, dtype=torch.long)
            loc.append((idx, U[:, idx, :].contiguous(), torch.empty((5, len(idx), U.shape[2]), dtype=U.dtype,
                                                                    device=U.device)))
        for phase, move in ((1, ("send_U", "recv_U")), (2, ("send_G", "recv_G")), (4, None)):
            for (idx, Ul, Utl), op in zip(loc, self.ops):
                op.time_derivative_phase(phase, Utl, Ul)
            if move:
                self._move(*move)
        for idx, Ul, Utl in loc:
            Ut[:, idx, :] = Utl

    def vjp(self, lam, gU, U, gtheta=None):
        """gU <- (dUt/dU)^T lam over the whole mesh (device tensors [5][K][n^3]),
        gtheta (device tensor of 2) <- (dUt/d(kappa, B))^T lam summed over the
        ranks: the four adjoint phases with the three exchanges between them
        (state traces; cotangents of the viscous-flux traces; cotangents of the
        state traces)."""
        import torch
        loc = []
        for r, op in enumerate(self.ops):
            idx = torch.as_tensor(self.l2g[r], device=U.device, dtype=torch.long)
            loc.append((idx, U[:, idx, :].contiguous(), lam[:, idx, :].contiguous(),
                        torch.empty((5, len(idx), U.shape[2]), dtype=U.dtype, device=U.device),
                        torch.zeros(2, dtype=U.dtype, device=U.device)))
        for phase, move in ((1, ("send_U", "recv_U")), (2, ("send_G", "recv_G")), (3, ("send_U", "recv_U")),
                            (4, None)):
            for (idx, Ul, laml, gl, th), op in zip(loc, self.ops):
                op.vjp_phase(phase, laml, gl, Ul, th)
            if move:
                self._move(*move)
        for idx, Ul, laml, gl, th in loc:
            gU[:, idx, :] = gl
        if gtheta is not None:
            gtheta.copy_(sum(th for *_, th in loc))
        return gU

    def check_status(self):
        for op in self.ops:
            op.check_status()

    def close(self):
        for op in self.ops:
            op.close()
