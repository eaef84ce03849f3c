"""Block decomposition of a periodic Cartesian element grid with ghost-layer halos.

The grid of ne[0] x ne[1] x ne[2] elements is cut into parts[0] x parts[1] x parts[2]
blocks, one per sub-domain (rank). A sub-domain's context is an ordinary context over its
owned block extended by `depth` ghost layers on both sides of every split axis (an axis
that is not split keeps its periodic wrap inside the box and needs no ghosts). The residual
of an owned element reads only elements within its stencil (Secs. 2.1-2.3 of the paper):

  compact: one layer of ghost elements, filled by one exchange of the state per residual
           (max |d| <= 1 and |d|_1 <= 2: the normal interface gradient uses only the
           own-face correction, Eqs. v:s:l / v:s:r);
  BR1:     either two ghost layers and one state exchange, or one ghost layer and two
           exchanges per residual: the state, then the ghosts' own interface gradients on the
           faces they share with owned elements (the BR1 normal gradient of a neighbour uses
           both of its corrections, Eq. v:e, so the ghost's value needs its far neighbour).

Exchanges run axis by axis (x, then y, then z); along axis a a rank sends its first and last
`depth` owned layers, taken over the full extended range of the axes already exchanged and
the owned range of the later ones, so that edge and corner ghosts arrive with the second and
third axis. Element indices are local to the extended box, x fastest.

Everything here is host logic (plans, neighbours, message order). The data moves through
the library's pack / unpack kernels (sd_pack_elements, sd_unpack_elements,
sd_pack_face_gradients, sd_unpack_face_gradients); `LocalDecomposition` runs every
sub-domain of a grid in one process on one GPU (device-to-device copies between the
sub-domains' halo buffers), `exchange_state_dist` / `exchange_grad_dist` move the same
buffers between processes with torch.distributed point-to-point messages.
"""
import ctypes
import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Message:
    """One halo message of an exchange: `send` (local element indices packed, in order) goes
    to `peer`, whose matching message (same axis, opposite side) lands in its `recv`
    indices; `faces` (face-gradient exchange only) are the face indices of each element."""
    axis: int
    side: int                  # 0: towards the -axis neighbour, 1: towards the +axis neighbour
    peer: int
    send: np.ndarray
    recv: np.ndarray
    send_faces: np.ndarray = None
    recv_faces: np.ndarray = None


class Partition:
    """Block partition of the periodic grid `ne` into `parts` blocks with `depth` ghost
    layers on each side of every split axis."""

    def __init__(self, ne, parts, depth=1):
        self.ne = tuple(int(x) for x in ne)
        self.parts = tuple(int(x) for x in parts)
        self.depth = int(depth)
        if len(self.ne) != 3 or len(self.parts) != 3:
            raise ValueError("ne and parts need three entries")
        if self.depth < 1:
            raise ValueError("depth must be >= 1")
        for d in range(3):
            if self.parts[d] < 1 or self.parts[d] > self.ne[d]:
                raise ValueError("parts[%d] must be in 1..ne[%d]" % (d, d))
            if self.parts[d] > 1 and self.ne[d] // self.parts[d] < self.depth:
                raise ValueError("axis %d: blocks of %d elements cannot feed %d ghost layers"
                                 % (d, self.ne[d] // self.parts[d], self.depth))
        self.size = self.parts[0] * self.parts[1] * self.parts[2]

    # ------------------------------------------------------------------ ranks and blocks
    def coords(self, rank):
        px, py, _ = self.parts
        return (rank % px, (rank // px) % py, rank // (px * py))

    def rank(self, c):
        px, py, pz = self.parts
        return (c[0] % px) + px * ((c[1] % py) + py * (c[2] % pz))

    def halo(self, d):
        return self.depth if self.parts[d] > 1 else 0

    def owned(self, rank):
        """Global element range [lo, hi) of the rank's block along each axis."""
        c = self.coords(rank)
        lo = tuple(c[d] * self.ne[d] // self.parts[d] for d in range(3))
        hi = tuple((c[d] + 1) * self.ne[d] // self.parts[d] for d in range(3))
        return lo, hi

    def local_shape(self, rank):
        """Elements of the extended box along each axis."""
        lo, hi = self.owned(rank)
        return tuple(hi[d] - lo[d] + 2 * self.halo(d) for d in range(3))

    def owned_local(self, rank):
        """The owned block inside the extended box, [lo, hi) per axis."""
        lo, hi = self.owned(rank)
        return (tuple(self.halo(d) for d in range(3)),
                tuple(self.halo(d) + hi[d] - lo[d] for d in range(3)))

    def neighbour(self, rank, axis, side):
        c = list(self.coords(rank))
        c[axis] += 1 if side else -1
        return self.rank(c)

    def box_origin(self, rank):
        """Global element coordinates of the extended box's first element (may be negative:
        the box wraps periodically)."""
        lo, _ = self.owned(rank)
        return tuple(lo[d] - self.halo(d) for d in range(3))

    # ------------------------------------------------------------------ index lists
    def _indices(self, rank, ranges):
        ex, ey, _ = self.local_shape(rank)
        xs, ys, zs = (np.arange(a, b) for a, b in ranges)
        z, y, x = np.meshgrid(zs, ys, xs, indexing="ij")
        return (x + ex * (y + ey * z)).reshape(-1).astype(np.int32)

    def state_plan(self, rank):
        """Messages of one state exchange, axis by axis (split axes only)."""
        shp = self.local_shape(rank)
        (olo, ohi) = self.owned_local(rank)
        out = []
        for a in range(3):
            h = self.halo(a)
            if h == 0:
                continue
            for side in (0, 1):
                ranges_s, ranges_r = [], []
                for b in range(3):
                    if b == a:
                        if side == 0:
                            ranges_s.append((olo[a], olo[a] + h))          # first owned layers
                            ranges_r.append((0, h))                        # - ghosts
                        else:
                            ranges_s.append((ohi[a] - h, ohi[a]))          # last owned layers
                            ranges_r.append((ohi[a], ohi[a] + h))          # + ghosts
                    elif b < a:
                        ranges_s.append((0, shp[b]))
                        ranges_r.append((0, shp[b]))
                    else:
                        ranges_s.append((olo[b], ohi[b]))
                        ranges_r.append((olo[b], ohi[b]))
                out.append(Message(a, side, self.neighbour(rank, a, side),
                                   self._indices(rank, ranges_s), self._indices(rank, ranges_r)))
        return out

    def grad_plan(self, rank):
        """Messages of the BR1 face-gradient exchange (one ghost layer): along a split axis a,
        the rank's first owned layer sends its -a faces (face 2a) to the -a neighbour, whose
        + ghosts take them on face 2a; its last layer sends its +a faces (2a + 1) to the +a
        neighbour, whose - ghosts take them on face 2a + 1. Only the owned range of the other
        axes: the ghosts that share a face with an owned element."""
        (olo, ohi) = self.owned_local(rank)
        out = []
        for a in range(3):
            if self.halo(a) == 0:
                continue
            for side in (0, 1):
                rs, rr = [], []
                for b in range(3):
                    if b == a:
                        if side == 0:
                            rs.append((olo[a], olo[a] + 1))
                            rr.append((olo[a] - 1, olo[a]))
                        else:
                            rs.append((ohi[a] - 1, ohi[a]))
                            rr.append((ohi[a], ohi[a] + 1))
                    else:
                        rs.append((olo[b], ohi[b]))
                        rr.append((olo[b], ohi[b]))
                send = self._indices(rank, rs)
                recv = self._indices(rank, rr)
                # the message sent towards side s carries faces 2a + s; the one received from
                # side s (sent by that neighbour towards 1 - s) lands on faces 2a + (1 - s)
                sf = np.full(send.shape, 2 * a + side, dtype=np.int32)
                rf = np.full(recv.shape, 2 * a + (1 - side), dtype=np.int32)
                out.append(Message(a, side, self.neighbour(rank, a, side), send, recv, sf, rf))
        return out

    # ------------------------------------------------------------------ layouts
    def extend(self, rank, U):
        """The rank's extended box cut from a global state U[v][ez][ey][ex][pts...] (host,
        numpy), ghosts taken by periodic wrap: the reference the exchanges must reproduce."""
        o = self.box_origin(rank)
        shp = self.local_shape(rank)
        idx = [np.arange(o[d], o[d] + shp[d]) % self.ne[d] for d in range(3)]
        return U[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]

    def scatter(self, U):
        """Extended boxes of every rank from a global state (host)."""
        return [np.ascontiguousarray(self.extend(r, U)) for r in range(self.size)]

    def gather_owned(self, parts_list, like):
        """Global array assembled from the ranks' owned blocks (host)."""
        out = np.empty_like(like)
        for r, A in enumerate(parts_list):
            lo, hi = self.owned(r)
            (llo, lhi) = self.owned_local(r)
            out[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = \
                A[:, llo[2]:lhi[2], llo[1]:lhi[1], llo[0]:lhi[0]]
        return out


def depth_for(scheme, grad_exchange):
    """Ghost layers the residual needs: compact 1; BR1 1 with the face-gradient exchange,
    else 2."""
    if scheme == "compact":
        return 1
    return 1 if grad_exchange else 2


def run_plan(plan, pack, unpack, deliver):
    """Run the messages of one exchange axis by axis: pack every message of the axis, deliver
    them (deliver(messages, buffers) -> received buffers in the same order), unpack. Axes
    run in order because edge and corner ghosts travel with a later axis."""
    for a in range(3):
        msgs = [m for m in plan if m.axis == a]
        if not msgs:
            continue
        bufs = [pack(m) for m in msgs]
        got = deliver(msgs, bufs)
        for m, b in zip(msgs, got):
            unpack(m, b)


def dist_deliver(dist, rank):
    """A deliver function over torch.distributed point-to-point messages: the message sent
    towards side s of axis a is received by the peer as its message from side 1 - s (tag
    2a + s)."""
    import torch

    def deliver(msgs, bufs):
        reqs, got = [], []
        for m, b in zip(msgs, bufs):
            got.append(torch.empty_like(b))
        for m, b in zip(msgs, bufs):
            reqs.append(dist.isend(b, m.peer, tag=2 * m.axis + m.side))
        for m, g in zip(msgs, got):
            # the buffer that lands in our side-s ghosts was sent towards 1 - s by the peer
            reqs.append(dist.irecv(g, m.peer, tag=2 * m.axis + (1 - m.side)))
        for r in reqs:
            r.wait()
        return got

    return deliver


# ---------------------------------------------------------------------- one GPU, all ranks
class LocalDecomposition:
    """Every sub-domain of one grid in this process, on the current GPU: one context per
    sub-domain over its extended box, halo messages delivered by device-to-device copies.
    residual(), rk_step() and diagnostics() match the single-domain calls on the owned
    elements."""

    def __init__(self, ne, parts, lo, hi, p, scheme, physics, precision="f32", grad_exchange=None):
        import torch
        from . import SD
        self.scheme = scheme
        if grad_exchange is None:
            grad_exchange = False
        if grad_exchange and scheme != "br1":
            raise ValueError("the face-gradient exchange belongs to the BR1 scheme")
        self.grad_exchange = grad_exchange
        self.part = Partition(ne, parts, depth_for(scheme, grad_exchange))
        self.p, self.n = p, p + 1
        h = [(hi[d] - lo[d]) / ne[d] for d in range(3)]
        self.subs = []
        for r in range(self.part.size):
            shp = self.part.local_shape(r)
            o = self.part.box_origin(r)
            blo = tuple(lo[d] + o[d] * h[d] for d in range(3))
            bhi = tuple(blo[d] + shp[d] * h[d] for d in range(3))
            ctx = SD(3, shp, blo, bhi, p, scheme, physics, precision)
            ctx.set_owned_box(*self.part.owned_local(r))
            plan = self.part.state_plan(r)
            gplan = self.part.grad_plan(r) if grad_exchange else []
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
            self.subs.append(dict(ctx=ctx, plan=plan, gplan=gplan,
                                  dplan={id(m): (dev(m.send), dev(m.recv)) for m in plan},
                                  dgplan={id(m): (dev(m.send), dev(m.recv), dev(m.send_faces),
                                                  dev(m.recv_faces)) for m in gplan}))
        self.dtype = self.subs[0]["ctx"].dtype
        self.nvar = self.subs[0]["ctx"].nvar

    def close(self):
        for s in self.subs:
            s["ctx"].close()

    # ------------------------------------------------------------------ layouts
    def scatter(self, U, dtype=None):
        """Device extended boxes of every sub-domain from a global host state (in the
        residual precision unless dtype is given: torch.float64 for Runge-Kutta states)."""
        import torch
        dt = self.dtype if dtype is None else dtype
        return [torch.from_numpy(A).to("cuda", dt) for A in self.part.scatter(np.asarray(U))]

    def gather(self, parts_list, like):
        return self.part.gather_owned([A.double().cpu().numpy() for A in parts_list], like)

    # ------------------------------------------------------------------ exchanges
    def _exchange(self, arrays, grad):
        """All sub-domains' halos, axis by axis; arrays: the extended state of each
        sub-domain (state exchange) or None (face-gradient exchange of the contexts)."""
        from . import pack_elements, unpack_elements, pack_face_gradients, unpack_face_gradients
        for a in range(3):
            outbox = {}
            for r, s in enumerate(self.subs):
                for m in (s["gplan"] if grad else s["plan"]):
                    if m.axis != a:
                        continue
                    if grad:
                        se, _, sf, _ = s["dgplan"][id(m)]
                        outbox[(m.peer, a, 1 - m.side)] = pack_face_gradients(s["ctx"], se, sf)
                    else:
                        se, _ = s["dplan"][id(m)]
                        outbox[(m.peer, a, 1 - m.side)] = pack_elements(s["ctx"], arrays[r], se)
            for r, s in enumerate(self.subs):
                for m in (s["gplan"] if grad else s["plan"]):
                    if m.axis != a:
                        continue
                    buf = outbox[(r, a, m.side)]
                    if grad:
                        _, re_, _, rf = s["dgplan"][id(m)]
                        unpack_face_gradients(s["ctx"], buf, re_, rf)
                    else:
                        _, re_ = s["dplan"][id(m)]
                        unpack_elements(s["ctx"], buf, re_, arrays[r])

    def exchange_state(self, arrays):
        self._exchange(arrays, grad=False)

    # ------------------------------------------------------------------ method
    def residual(self, Us, Rs):
        """R = dU/dt on every sub-domain (owned elements exact); Us, Rs: extended boxes."""
        from . import residual_begin, residual_end
        self.exchange_state(Us)
        if self.grad_exchange:
            for s, U in zip(self.subs, Us):
                residual_begin(s["ctx"], U)
            self._exchange(None, grad=True)
            for s, U, R in zip(self.subs, Us, Rs):
                residual_end(s["ctx"], U, R)
        else:
            for s, U, R in zip(self.subs, Us, Rs):
                s["ctx"].residual(U, R)

    def rk_step(self, U64s, t, dt, rk="ssprk54"):
        """One Runge-Kutta step of every sub-domain's FP64 state (extended boxes), the halos
        of every stage input exchanged before its residual (one state exchange per stage)."""
        if self.grad_exchange:
            raise ValueError("stage-by-stage stepping uses the one-exchange layouts (BR1: depth 2)")
        from . import rk_prepare, rk_stage
        ins = [rk_prepare(s["ctx"], U) for s, U in zip(self.subs, U64s)]
        nst = 4 if rk == "rk4" else 5
        for k in range(nst):
            self.exchange_state(ins)
            ins = [rk_stage(s["ctx"], U, k, dt, rk) for s, U in zip(self.subs, U64s)]

    def diagnostics(self, U64s, t=0.0):
        """FP64 diagnostics over the owned elements of every sub-domain, summed in FP64 (the
        host-side counterpart of an FP64 all-reduce). The FP64 states' ghosts are refreshed
        first: the gradient at an owned element's points uses its neighbours' traces."""
        self.exchange_state(U64s)
        keys = ("ke", "ke_rho", "enstrophy", "mass", "energy", "l2sq", "volume")
        tot = {k: 0.0 for k in keys}
        mom = [0.0, 0.0, 0.0]
        nonfinite = 0
        for s, U in zip(self.subs, U64s):
            d = s["ctx"].diagnostics(U, t, raise_nonfinite=False)
            for k in keys:
                tot[k] += d[k]
            for i in range(3):
                mom[i] += d["mom"][i]
            nonfinite |= d["nonfinite"]
        tot["mom"] = mom
        tot["nonfinite"] = nonfinite
        tot["t"] = t
        return tot


def allreduce_diagnostics(d, dist, device="cpu"):
    """Sum one rank's owned-box diagnostics over all ranks in FP64 (torch.distributed)."""
    import torch
    keys = ("ke", "ke_rho", "enstrophy", "mass", "energy", "l2sq", "volume")
    v = torch.tensor([d[k] for k in keys] + list(d["mom"]) + [float(d["nonfinite"])],
                     dtype=torch.float64, device=device)
    dist.all_reduce(v)
    out = {k: float(v[i]) for i, k in enumerate(keys)}
    out["mom"] = [float(v[len(keys) + i]) for i in range(3)]
    out["nonfinite"] = int(v[-1] > 0)
    out["t"] = d.get("t", 0.0)
    return out


del ctypes, math
