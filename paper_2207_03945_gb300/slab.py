"""One flock square decomposed over several ranks (devices): the square's
cell rows are split into R contiguous bands, one per rank; each rank owns
the agents whose cell row lies in its band.

A step (Section 4.1: every agent acts, then every agent observes the new
positions) on rank b:
  1. the own agents take their actions;
  2. with their new positions, every own agent goes to each band whose
     region (band rows plus H halo rows on each side, modulo the rows of the
     square) holds its row: to the band that holds the row itself as an own
     agent (a migrant, if that is another band), to the others as a ghost.
     An agent that left but lies in this band's own halo stays here as a
     ghost.  One exchange with each of the two neighbouring bands;
  3. the own agents observe their own and the ghost agents.
Every neighbour within the view radius of an own agent lies in the stencil
rows, hence in the band's region, so the own agents' observations, rewards
and collisions equal those on the undivided square, bit for bit: positions
keep their coordinates on the square (ghosts are never shifted), and the
minimum-image offsets are formed from them exactly as on the square.

The compute of a band is a backend: the CUDA slab environment of the
library (CudaBand) on a device, or any object with the same two methods.
The exchange is torch.distributed point-to-point messages (DistExchange;
gloo on the host, NCCL between devices) or, for several bands emulated in
one process, an in-memory router (LocalExchange).  Agents keep global ids,
so results can be put back in the square's agent order.
"""
from __future__ import annotations

import numpy as np


def bands(nc: int, world: int, halo: int):
    """[(r_lo, r_hi)] per rank: rank b owns rows [floor(b nc / R),
    floor((b + 1) nc / R)).  Each band needs at least `halo` rows (and R > 1
    needs a region, band plus two halos, within the nc rows)."""
    out = [(b * nc // world, (b + 1) * nc // world) for b in range(world)]
    if world > 1 and any(hi - lo < max(halo, 1) for lo, hi in out):
        raise ValueError("%d bands of %d rows: a band is thinner than the halo (%d rows)"
                         % (world, nc, halo))
    if world > 1 and min(hi - lo for lo, hi in out) + 2 * halo > nc:
        raise ValueError("a band's region would cover the square more than once")
    return out


def cell_rows(y, inv_cell_width: float, nc: int):
    """Cell row of each y (float32): trunc(y * (nc / L)) clamped to [0, nc),
    the library's binning (one float32 multiply, truncation)."""
    import torch
    if isinstance(y, torch.Tensor):
        r = (y * torch.tensor(inv_cell_width, dtype=torch.float32, device=y.device)).to(torch.int64)
        return r.clamp(0, nc - 1)
    r = (np.asarray(y, dtype=np.float32) * np.float32(inv_cell_width)).astype(np.int64)
    return np.clip(r, 0, nc - 1)


def in_rows(rows, lo: int, hi: int, nc: int):
    """rows within [lo, hi) taken modulo nc (lo may be negative, hi > nc)."""
    return ((rows - lo) % nc) < (hi - lo)


class DistExchange:
    """Exchange through torch.distributed point-to-point messages: to each
    peer the count, then ids (int64) and states (float32 n x 4) of its own
    agents and its ghosts.  `device`: where the message tensors live (the
    host for gloo, the GPU for NCCL)."""

    def __init__(self, group=None, device="cpu"):
        import torch
        self.group = group
        self.device = torch.device(device)

    def __call__(self, outgoing):
        """outgoing: {peer: (ids_own, st_own, ids_ghost, st_ghost)}; returns
        the same structure received from each peer."""
        import torch
        import torch.distributed as dist
        peers = sorted(outgoing)
        counts_out = {p: torch.tensor([outgoing[p][0].numel(), outgoing[p][2].numel()],
                                      dtype=torch.int64, device=self.device) for p in peers}
        counts_in = {p: torch.empty(2, dtype=torch.int64, device=self.device) for p in peers}
        ops = []
        for p in peers:
            ops.append(dist.P2POp(dist.isend, counts_out[p], p, self.group))
            ops.append(dist.P2POp(dist.irecv, counts_in[p], p, self.group))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        recv = {}
        ops = []
        for p in peers:
            ni, ng = (int(x) for x in counts_in[p].tolist())
            n_out = outgoing[p][0].numel() + outgoing[p][2].numel()
            ids = torch.empty(ni + ng, dtype=torch.int64, device=self.device)
            st = torch.empty((ni + ng, 4), dtype=torch.float32, device=self.device)
            recv[p] = (ni, ids, st)
            o_ids = torch.cat([outgoing[p][0], outgoing[p][2]]).to(self.device)
            o_st = torch.cat([outgoing[p][1], outgoing[p][3]]).to(self.device)
            if n_out:
                ops.append(dist.P2POp(dist.isend, o_ids.contiguous(), p, self.group))
                ops.append(dist.P2POp(dist.isend, o_st.contiguous(), p, self.group))
            if ni + ng:
                ops.append(dist.P2POp(dist.irecv, ids, p, self.group))
                ops.append(dist.P2POp(dist.irecv, st, p, self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        return {p: (ids[:ni], st[:ni], ids[ni:], st[ni:]) for p, (ni, ids, st) in recv.items()}


class LocalExchange:
    """Routes the messages of several bands emulated in one process."""

    def __init__(self):
        self.mail = {}

    def post(self, src, outgoing):
        for dst, msg in outgoing.items():
            self.mail.setdefault(dst, {})[src] = msg

    def take(self, dst):
        return self.mail.pop(dst, {})


class SlabBand:
    """The bookkeeping of rank b's band: its own agents (global ids and
    states), the ghosts of the current step, and the selection of what goes
    to each neighbouring band.  `backend` computes on the band's device:
    apply(state, actions) moves the own agents in place; observe(own, ghosts)
    returns (obs, reward, coll) of the own agents.  Tensors live on
    `device`."""

    def __init__(self, nc: int, halo: int, inv_cell_width: float, rank: int, world: int,
                 backend, device="cpu"):
        import torch
        self.nc, self.halo, self.invw = int(nc), int(halo), float(inv_cell_width)
        self.rank, self.world = int(rank), int(world)
        self.all_bands = bands(self.nc, self.world, self.halo)
        self.lo, self.hi = self.all_bands[self.rank]
        self.peers = sorted({(self.rank - 1) % self.world, (self.rank + 1) % self.world} -
                            {self.rank})
        self.backend = backend
        self.device = torch.device(device)
        self.ids = torch.empty(0, dtype=torch.int64, device=self.device)
        self.st = torch.empty((0, 4), dtype=torch.float32, device=self.device)
        self.ghost_ids = self.ids
        self.ghost_st = self.st

    def region(self, b):
        lo, hi = self.all_bands[b]
        return lo - self.halo, hi + self.halo

    def load(self, ids, state):
        """Keeps the agents of the square (global ids, states) whose row lies
        in this band."""
        import torch
        ids = torch.as_tensor(ids, dtype=torch.int64).to(self.device)
        st = torch.as_tensor(state, dtype=torch.float32).to(self.device)
        rows = cell_rows(st[:, 1], self.invw, self.nc)
        keep = in_rows(rows, self.lo, self.hi, self.nc)
        self.ids, self.st = ids[keep].contiguous(), st[keep].contiguous()

    def apply(self, actions_by_id):
        """The own agents act: actions_by_id[id] is agent id's action (a
        tensor indexed by global id, on this band's device)."""
        if self.ids.numel():
            act = actions_by_id[self.ids].to(dtype=self.backend.action_dtype).contiguous()
            self.backend.apply(self.st, act)

    def outgoing(self):
        """After the move: keeps the own agents still in the band and the
        ones that left into its halo (as ghosts), and returns, per
        neighbouring band, (ids, states) of the agents it now owns and of
        its ghosts."""
        rows = cell_rows(self.st[:, 1], self.invw, self.nc)
        mine = in_rows(rows, self.lo, self.hi, self.nc)
        lo, hi = self.region(self.rank)
        near = in_rows(rows, lo, hi, self.nc) & ~mine
        out = {}
        for p in self.peers:
            plo, phi = self.all_bands[p]
            own_p = in_rows(rows, plo, phi, self.nc)
            rlo, rhi = self.region(p)
            ghost_p = in_rows(rows, rlo, rhi, self.nc) & ~own_p
            out[p] = (self.ids[own_p], self.st[own_p], self.ids[ghost_p], self.st[ghost_p])
        self.ghost_ids, self.ghost_st = self.ids[near], self.st[near]
        self.ids, self.st = self.ids[mine].contiguous(), self.st[mine].contiguous()
        return out

    def incoming(self, received):
        """Adds what the neighbouring bands sent: their agents now in this
        band (own) and their agents in this band's halo (ghosts)."""
        import torch
        own_ids, own_st = [self.ids], [self.st]
        g_ids, g_st = [self.ghost_ids], [self.ghost_st]
        for p in sorted(received):
            i_own, s_own, i_gh, s_gh = received[p]
            own_ids.append(i_own.to(self.device))
            own_st.append(s_own.to(self.device))
            g_ids.append(i_gh.to(self.device))
            g_st.append(s_gh.to(self.device))
        self.ids = torch.cat(own_ids).contiguous()
        self.st = torch.cat(own_st).contiguous()
        self.ghost_ids = torch.cat(g_ids).contiguous()
        self.ghost_st = torch.cat(g_st).contiguous()

    def observe(self):
        """(ids, obs, reward, coll) of the own agents."""
        obs, rew, coll = self.backend.observe(self.st, self.ghost_st)
        return self.ids, obs, rew, coll


class CudaBand:
    """Band compute on a device: the library's slab environment of the
    band's rows plus the halos, grown when a step brings more agents than it
    holds."""
    action_dtype = None

    def __init__(self, params: dict, nc: int, halo: int, lo: int, hi: int, device="cuda",
                 n_max: int = 1024, tuning: dict | None = None):
        import torch
        self.params, self.tuning = dict(params), tuning
        self.row0 = (lo - halo) % nc
        self.nrows = hi - lo + 2 * halo
        self.device = torch.device(device)
        self.action_dtype = torch.int32
        self.slab = None
        self._make(max(int(n_max), 1))

    def _make(self, n_max):
        from . import FlockSlab
        if self.slab is not None:
            self.slab.close()
        self.n_max = n_max
        self.slab = FlockSlab(self.params, n_max, self.row0, self.nrows, device=self.device,
                              tuning=self.tuning)

    def apply(self, state, actions):
        if state.shape[0] > self.n_max:
            self._make(2 * int(state.shape[0]))
        self.slab.apply(state, actions)

    def observe(self, own, ghosts):
        import torch
        st = torch.cat([own, ghosts]).contiguous()
        if st.shape[0] > self.n_max:
            self._make(2 * int(st.shape[0]))
        n = int(own.shape[0])
        obs = torch.empty((n, self.slab.obs_dim), dtype=torch.float32, device=self.device)
        rew = torch.empty(n, dtype=torch.float32, device=self.device)
        coll = torch.empty(n, dtype=torch.int32, device=self.device)
        self.slab.observe(st, n, obs, rew, coll)
        return obs, rew, coll

    def error(self) -> int:
        return self.slab.error()

    def close(self):
        if self.slab is not None:
            self.slab.close()
            self.slab = None


def geometry(params: dict, stencil: int = 1):
    """(cells per side, halo rows, float32 inverse cell width) of the square
    under the library's cell list."""
    from . import flock_derive
    d = flock_derive(params, {"stencil": stencil})
    return int(d["cells_per_side"]), int(d["stencil"]), float(d["inv_cell_width"])


def step_local(bands_, exchange: LocalExchange, actions_by_id=None):
    """One step of several bands emulated in one process (actions_by_id
    None: observe the current positions).  Returns per band (ids, obs,
    reward, coll) of its own agents."""
    if actions_by_id is not None:
        for b in bands_:
            b.apply(actions_by_id)
    for b in bands_:
        exchange.post(b.rank, b.outgoing())
    for b in bands_:
        b.incoming(exchange.take(b.rank))
    return [b.observe() for b in bands_]


def step_dist(band: SlabBand, exchange: DistExchange, actions_by_id=None):
    """One step of this rank's band, exchanging with the neighbouring
    ranks."""
    if actions_by_id is not None:
        band.apply(actions_by_id)
    band.incoming(exchange(band.outgoing()))
    return band.observe()
