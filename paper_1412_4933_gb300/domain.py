"""Domain decomposition of one grid into column strips.

One W x H scenario is split into strips of columns; each strip advances with
``sim_step_strip`` (the automaton's step, Sec. IV.b-d, on the strip's own
columns plus a halo of ``HALO`` columns on each side) and, before every step,
its halo columns are refreshed from the neighbouring strips' interiors:
occupancy, ids and both pheromone planes of those cells, and the per-agent
entries (arrival step, tour length) of the agents standing on them.  A cell's
state after one step depends on cells at most three columns away, so with
three halo columns every strip's interior advances bit for bit as the whole
grid would (the halo's own results are overwritten by the next exchange).

Two transports move the halos:

* ``LocalExchange`` -- every strip in this process (on one device or several):
  slices of the strips' tensors are copied directly;
* ``DistExchange`` -- one strip per rank: each rank sends its two boundary
  slabs (fixed-size tensors) to its neighbours and receives theirs, with
  ``torch.distributed`` point-to-point calls (NCCL between GPUs, gloo on CPU).

The exchange is communication only; every step of the automaton runs in the
library's kernels.  The paper runs one grid on one GPU; it does not address
splitting a grid over several devices.
"""
from __future__ import annotations

import numpy as np

HALO = 3  # columns a cell's next state can depend on, each side


def partition(W: int, n: int) -> list[tuple[int, int]]:
    """Interior column ranges [a, b) of n strips covering 0..W-1, as even as
    possible; every strip at least HALO columns wide (a halo then comes from
    one neighbour)."""
    if n < 1 or W < n * HALO:
        raise ValueError(f"cannot split {W} columns into {n} strips of >= {HALO} columns")
    base, extra = divmod(W, n)
    out, a = [], 0
    for r in range(n):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def extended(W: int, a: int, b: int) -> tuple[int, int]:
    """Local columns [ea, eb) of the strip with interior [a, b): the interior
    and up to HALO columns on each side (clipped at the grid's edges)."""
    return max(0, a - HALO), min(W, b + HALO)


class StripLayout:
    """Column bookkeeping of one strip: interior [a, b) (global), local
    columns [ea, eb) (global), interior_lo/hi as local indices."""

    def __init__(self, W: int, a: int, b: int):
        self.W, self.a, self.b = W, a, b
        self.ea, self.eb = extended(W, a, b)
        self.width = self.eb - self.ea
        self.lo, self.hi = a - self.ea, b - self.ea

    def local(self, g0: int, g1: int) -> slice:
        """Local column slice of global columns [g0, g1)."""
        return slice(g0 - self.ea, g1 - self.ea)

    def left_halo(self) -> tuple[int, int]:
        return self.ea, self.a

    def right_halo(self) -> tuple[int, int]:
        return self.b, self.eb


class StripState:
    """The tensors of one strip (any torch device): occupancy and pheromone
    planes by step parity, ids, per-agent arrays, the proposal scratch plane
    and the interior's counters."""

    def __init__(self, torch, layout: StripLayout, H: int, n_agents: int, aco: bool, device):
        w = layout.width
        self.layout = layout
        self.occ = [torch.zeros((H, w), dtype=torch.uint8, device=device) for _ in range(2)]
        self.ids = torch.zeros((H, w), dtype=torch.int32, device=device)
        self.tau = ([[torch.zeros((H, w), dtype=torch.float32, device=device) for _ in range(2)]
                     for _ in range(2)] if aco else None)
        self.arrival = torch.zeros(n_agents + 1, dtype=torch.int32, device=device)
        self.tour = torch.zeros(n_agents + 1, dtype=torch.float32, device=device)
        self.scratch = torch.zeros((H, w), dtype=torch.uint8, device=device)
        self.counters = torch.zeros(4, dtype=torch.int64, device=device)

    def planes(self, par: int):
        """The state planes of parity `par`, in a fixed order."""
        out = [self.occ[par], self.ids]
        if self.tau is not None:
            out += [self.tau[0][par], self.tau[1][par]]
        return out


def slab(st: StripState, par: int, g0: int, g1: int):
    """The cells of global columns [g0, g1) of a strip, packed: its state
    planes and, per cell, the arrival step and tour length of the agent on
    it (0 on empty cells)."""
    cols = st.layout.local(g0, g1)
    planes = [p[:, cols].contiguous() for p in st.planes(par)]
    occupied = planes[0] != 0
    ids = planes[1].long() * occupied  # (stale ids at empty cells are not looked up)
    arrival = st.arrival[ids] * occupied
    tour = st.tour[ids] * occupied
    return planes + [arrival, tour]


def apply_slab(st: StripState, par: int, g0: int, g1: int, packed) -> None:
    """Writes a slab received for global columns [g0, g1) into the strip:
    the planes, and the per-agent entries of the agents on those cells."""
    cols = st.layout.local(g0, g1)
    planes = st.planes(par)
    for dst, src in zip(planes, packed[:len(planes)]):
        dst[:, cols] = src
    arrival, tour = packed[len(planes)], packed[len(planes) + 1]
    occupied = packed[0] != 0
    ids = packed[1].long()[occupied]
    st.arrival[ids] = arrival[occupied]
    st.tour[ids] = tour[occupied]


class LocalExchange:
    """Halo exchange between strips held by this process: between strips on
    the same GPU one ``sim_strip_halo`` kernel per halo (the library's copy of
    the planes and of the halo agents' entries, no host synchronisation),
    otherwise the packed slabs through torch."""

    def __init__(self, strips):
        self.strips = strips

    @staticmethod
    def _copy(src: StripState, dst: StripState, par: int, g0: int, g1: int) -> None:
        if not (src.ids.is_cuda and src.ids.device == dst.ids.device):
            apply_slab(dst, par, g0, g1, [t.to(dst.ids.device) for t in slab(src, par, g0, g1)])
            return
        import torch
        from . import pedsim as P

        def bufs(st):
            tau = (st.tau[0][par], st.tau[1][par]) if st.tau is not None else (None, None)
            return (st.occ[par], st.ids) + tau + (st.arrival, st.tour)

        rc = P.strip_halo(dst.occ[par].shape[0], g1 - g0, dst.arrival.numel() - 1,
                          bufs(src), src.layout.width, src.layout.local(g0, g1).start,
                          bufs(dst), dst.layout.width, dst.layout.local(g0, g1).start,
                          stream=torch.cuda.current_stream(dst.ids.device))
        if rc != P.OK:
            raise P.PedsimError(rc, "sim_strip_halo failed")

    def exchange(self, par: int) -> None:
        for r, st in enumerate(self.strips):
            lay = st.layout
            if r > 0 and lay.ea < lay.a:
                g0, g1 = lay.left_halo()
                self._copy(self.strips[r - 1], st, par, g0, g1)
            if r + 1 < len(self.strips) and lay.b < lay.eb:
                g0, g1 = lay.right_halo()
                self._copy(self.strips[r + 1], st, par, g0, g1)


class DistExchange:
    """Halo exchange with one strip per rank (torch.distributed point to
    point): each rank sends the HALO boundary columns of its interior to each
    neighbour and receives the neighbour's into its halo."""

    def __init__(self, dist, strip: StripState, rank: int, world: int, layouts):
        self.dist, self.strip, self.rank, self.world = dist, strip, rank, world
        self.layouts = layouts

    def exchange(self, par: int) -> None:
        dist, st, r = self.dist, self.strip, self.rank
        lay = st.layout
        reqs, inbox = [], []
        if r > 0:
            # my left halo is my left neighbour's right boundary, and vice versa
            g0, g1 = lay.left_halo()
            for t in slab(st, par, lay.a, min(lay.a + HALO, lay.b)):
                reqs.append(dist.isend(t, r - 1))
            bufs = [t.new_empty(t.shape) for t in slab(st, par, g0, g1)]
            inbox.append((g0, g1, bufs))
            reqs += [dist.irecv(b, r - 1) for b in bufs]
        if r + 1 < self.world:
            g0, g1 = lay.right_halo()
            for t in slab(st, par, max(lay.b - HALO, lay.a), lay.b):
                reqs.append(dist.isend(t, r + 1))
            bufs = [t.new_empty(t.shape) for t in slab(st, par, g0, g1)]
            inbox.append((g0, g1, bufs))
            reqs += [dist.irecv(b, r + 1) for b in bufs]
        for q in reqs:
            q.wait()
        for g0, g1, bufs in inbox:
            apply_slab(st, par, g0, g1, bufs)


class StripDomain:
    """A W x H scenario advanced as `n_strips` column strips, all in this
    process (`devices`: one torch device per strip, default all on cuda:0).
    State in and out as the dicts of ``pedsim.Sim.read_grid`` /
    ``read_agents``."""

    def __init__(self, W: int, H: int, params, seed: int, n_strips: int, devices=None):
        import torch
        from . import pedsim as P
        self.torch, self.P = torch, P
        self.W, self.H, self.params, self.seed = W, H, params, seed
        self.n_agents = 2 * params.n_per_side
        self.aco = params.model == P.ACO
        if P.validate(W, H, params) != P.OK:
            raise ValueError("invalid scenario")
        devices = devices or ["cuda:0"] * n_strips
        self.layouts = [StripLayout(W, a, b) for a, b in partition(W, n_strips)]
        self.strips = [StripState(torch, lay, H, self.n_agents, self.aco, dev)
                       for lay, dev in zip(self.layouts, devices)]
        self.exchanger = LocalExchange(self.strips)
        self.step_index = 0
        self.par = 0

    def load(self, step: int, grid: dict, agents: dict) -> None:
        """Sets the state at step `step` from a whole-grid state."""
        torch = self.torch
        occ = np.ascontiguousarray(grid["occ"], np.uint8)
        ids = np.ascontiguousarray(grid["ids"], np.uint32).view(np.int32)
        self.step_index, self.par = step, 0
        for st in self.strips:
            dev = st.ids.device
            cols = slice(st.layout.ea, st.layout.eb)
            st.occ[0].copy_(torch.from_numpy(occ[:, cols].copy()).to(dev))
            st.ids.copy_(torch.from_numpy(ids[:, cols].copy()).to(dev))
            if self.aco:
                for g, name in ((0, "tauA"), (1, "tauB")):
                    t = np.ascontiguousarray(grid[name], np.float32)[:, cols].copy()
                    st.tau[g][0].copy_(torch.from_numpy(t).to(dev))
            st.arrival.copy_(torch.from_numpy(
                np.ascontiguousarray(agents["arrival"], np.uint32).view(np.int32)).to(dev))
            st.tour.copy_(torch.from_numpy(np.ascontiguousarray(agents["tour"], np.float32)).to(dev))
            st.counters.zero_()

    def step(self, n: int = 1) -> None:
        P = self.P
        for _ in range(n):
            self.exchanger.exchange(self.par)
            for st in self.strips:
                lay = st.layout
                nxt = self.par ^ 1
                tau = st.tau
                with self.torch.cuda.device(st.ids.device):
                    rc = P.step_strip(
                        lay.width, self.H, lay.ea, self.W, lay.lo, lay.hi, self.params, self.seed,
                        self.step_index, st.occ[self.par], st.occ[nxt], st.ids,
                        tau[0][self.par] if tau else None, tau[1][self.par] if tau else None,
                        tau[0][nxt] if tau else None, tau[1][nxt] if tau else None,
                        st.arrival, st.tour, st.scratch, st.counters,
                        stream=self.torch.cuda.current_stream(st.ids.device))
                if rc != P.OK:
                    raise P.PedsimError(rc, "sim_step_strip failed")
            self.par ^= 1
            self.step_index += 1

    def read_grid(self) -> dict:
        """The whole grid assembled from the strips' interiors (ids 0 at
        empty cells)."""
        occ = np.zeros((self.H, self.W), np.uint8)
        ids = np.zeros((self.H, self.W), np.uint32)
        tau = [np.zeros((self.H, self.W), np.float32) for _ in range(2)]
        for st in self.strips:
            lay = st.layout
            cols = slice(lay.lo, lay.hi)
            occ[:, lay.a:lay.b] = st.occ[self.par][:, cols].cpu().numpy()
            ids[:, lay.a:lay.b] = st.ids[:, cols].cpu().numpy().view(np.uint32)
            if self.aco:
                for g in range(2):
                    tau[g][:, lay.a:lay.b] = st.tau[g][self.par][:, cols].cpu().numpy()
        ids[occ == 0] = 0
        out = {"occ": occ, "ids": ids}
        if self.aco:
            out["tauA"], out["tauB"] = tau
        return out

    def read_agents(self) -> dict:
        """Per-agent arrays: each agent's entries from the strip it stands in."""
        arrival = np.zeros(self.n_agents + 1, np.uint32)
        tour = np.zeros(self.n_agents + 1, np.float32)
        for st in self.strips:
            lay = st.layout
            cols = slice(lay.lo, lay.hi)
            occ = st.occ[self.par][:, cols].cpu().numpy()
            ids = st.ids[:, cols].cpu().numpy().view(np.uint32)[occ != 0]
            arrival[ids] = st.arrival.cpu().numpy().view(np.uint32)[ids]
            tour[ids] = st.tour.cpu().numpy()[ids]
        return {"arrival": arrival, "tour": tour}

    def counters(self) -> dict:
        """moved, conflicts, crossed[A], crossed[B] since load(), summed over
        the strips (each counts the events of its interior)."""
        tot = sum(st.counters.cpu().numpy() for st in self.strips)
        return {"moved": int(tot[0]), "conflicts": int(tot[1]),
                "crossed": [int(tot[2]), int(tot[3])]}


class RankStrip:
    """One strip per rank of a torch.distributed group (``torchrun``, one
    process per GPU): rank r owns the r-th strip of ``partition(W, world)``,
    refreshes its halo from its neighbours with ``DistExchange`` (NCCL on
    GPUs) and steps it with ``sim_step_strip``.  Loading takes the whole-grid
    state every rank can build itself (e.g. the library's deterministic
    placement of the same seed)."""

    def __init__(self, dist, W: int, H: int, params, seed: int, device):
        import torch
        from . import pedsim as P
        self.torch, self.P = torch, P
        self.W, self.H, self.params, self.seed = W, H, params, seed
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.layouts = [StripLayout(W, a, b) for a, b in partition(W, self.world)]
        self.strip = StripState(torch, self.layouts[self.rank], H, 2 * params.n_per_side,
                                params.model == P.ACO, device)
        self.exchanger = DistExchange(dist, self.strip, self.rank, self.world, self.layouts)
        self.step_index, self.par = 0, 0

    def load(self, step: int, grid: dict, agents: dict) -> None:
        torch, st = self.torch, self.strip
        dev = st.ids.device
        cols = slice(st.layout.ea, st.layout.eb)
        st.occ[0].copy_(torch.from_numpy(np.ascontiguousarray(grid["occ"], np.uint8)[:, cols].copy()).to(dev))
        st.ids.copy_(torch.from_numpy(
            np.ascontiguousarray(grid["ids"], np.uint32).view(np.int32)[:, cols].copy()).to(dev))
        if st.tau is not None:
            for g, name in ((0, "tauA"), (1, "tauB")):
                st.tau[g][0].copy_(torch.from_numpy(
                    np.ascontiguousarray(grid[name], np.float32)[:, cols].copy()).to(dev))
        st.arrival.copy_(torch.from_numpy(
            np.ascontiguousarray(agents["arrival"], np.uint32).view(np.int32)).to(dev))
        st.tour.copy_(torch.from_numpy(np.ascontiguousarray(agents["tour"], np.float32)).to(dev))
        st.counters.zero_()
        self.step_index, self.par = step, 0

    def step(self, n: int = 1) -> None:
        P, st = self.P, self.strip
        lay, tau = st.layout, st.tau
        for _ in range(n):
            self.exchanger.exchange(self.par)
            nxt = self.par ^ 1
            rc = P.step_strip(lay.width, self.H, lay.ea, self.W, lay.lo, lay.hi, self.params,
                              self.seed, self.step_index, st.occ[self.par], st.occ[nxt], st.ids,
                              tau[0][self.par] if tau else None, tau[1][self.par] if tau else None,
                              tau[0][nxt] if tau else None, tau[1][nxt] if tau else None,
                              st.arrival, st.tour, st.scratch, st.counters,
                              stream=self.torch.cuda.current_stream(st.ids.device))
            if rc != P.OK:
                raise P.PedsimError(rc, "sim_step_strip failed")
            self.par = nxt
            self.step_index += 1

    def interior(self) -> dict:
        """This rank's interior columns [a, b) of the current state."""
        st, lay = self.strip, self.strip.layout
        cols = slice(lay.lo, lay.hi)
        out = {"columns": (lay.a, lay.b), "occ": st.occ[self.par][:, cols].cpu().numpy(),
               "ids": st.ids[:, cols].cpu().numpy().view(np.uint32)}
        if st.tau is not None:
            out["tauA"] = st.tau[0][self.par][:, cols].cpu().numpy()
            out["tauB"] = st.tau[1][self.par][:, cols].cpu().numpy()
        return out
