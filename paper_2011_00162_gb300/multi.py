"""Host-side logic for runs on several ranks (one process per GPU).

The OD2P iteration of one reconstruction runs on one GPU.  Several GPUs run
independent work: replicas of one workload, or disjoint shares of a batch of
independent reconstructions.  Neither needs a data-path collective; the only
collective is the max-over-ranks of the timed interval.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(costs: list[float], rank: int, world: int) -> list[int]:
    """Indices of the items rank `rank` owns: greedy longest-processing-time
    assignment of the costs to `world` ranks (ties to the lowest rank), so every
    item has exactly one owner and the loads are balanced."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def max_over_ranks(value: float, device: torch.device | None = None) -> float:
    """Largest `value` over all ranks (identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- subdomain sharding
# One reconstruction over several ranks (section 3.1: the subdomain problems are
# coupled only through their overlaps).  Each rank owns a contiguous block of
# subdomains -- their frames (f, Gamma), u_d, Lambda_{d,e} and, blind, W_d and
# Delta_d -- and keeps halo copies of the rest.  Between iterations the owner of
# e sends every rank that owns a neighbour d of e the strip of u_e on the overlap
# of Omega_e and Omega_d and the multiplier Lambda_{e,d}, which is all the owner
# of d reads of e when it forms v_{d,e} (eq. updateV-multi); blind, it sends its
# W_e and Delta_e to every rank, since the w-update (eq. blind_w) sums all of
# them.  Owned values are then computed exactly as in the undivided iteration.

def partition_subdomains(frame_sub, n_sub: int, world: int) -> list[int]:
    """owner[d] for d < n_sub: `world` contiguous blocks of subdomains (in d
    order) of about J / world frames each -- rank r's block starts at the first
    subdomain whose frames' midpoint passes r J / world -- with every rank
    owning at least one subdomain when n_sub >= world."""
    if world < 1:
        raise ValueError("need world >= 1")
    counts = [0] * n_sub
    for d in frame_sub:
        counts[int(d)] += 1
    total = sum(counts)
    mid, acc = [], 0
    for c in counts:
        mid.append(acc + 0.5 * c)
        acc += c
    starts = [0]
    for r in range(1, world):
        t = r * total / world
        cand = next((d for d in range(n_sub) if mid[d] >= t), n_sub)
        cand = max(cand, starts[-1] + 1)
        cand = min(cand, max(n_sub - (world - r), starts[-1] + 1), n_sub)
        starts.append(cand)
    starts.append(n_sub)
    owner = [0] * n_sub
    for r in range(world):
        for d in range(starts[r], starts[r + 1]):
            owner[d] = r
    return owner


class HaloSchedule:
    """The strips one rank sends to and receives from each peer, in a fixed
    order both sides derive from the decomposition: for every ordered pair
    (e, d) in pair order with owner[e] = sender and owner[d] = receiver, the
    strip of u_e on the pair's rectangle (Omega_e n Omega_d, in e's coordinates;
    with periodic boundaries Omega_d moved by the pair's shift), row-major,
    followed by Lambda_{e,d}; then,
    blind, W_e and Delta_e (m x m each) of every e the sender owns, e
    ascending.  Arrays are the concatenated layouts of the state (u by
    subdomain rectangles, Lambda by pair rectangles, W_d and Delta_d by d)."""

    def __init__(self, rect, pairs, pair_rect, owner, rank: int, m: int, blind: bool):
        rect = [tuple(int(x) for x in r) for r in rect]
        pairs = [tuple(int(x) for x in p) for p in pairs]
        pair_rect = [tuple(int(x) for x in r) for r in pair_rect]
        self.rank, self.owner, self.m, self.blind = rank, list(owner), m, blind
        self.world = max(self.owner) + 1
        self.u_off = [0]
        for r0, c0, r1, c1 in rect:
            self.u_off.append(self.u_off[-1] + (r1 - r0) * (c1 - c0))
        self.lam_off = [0]
        for r0, c0, r1, c1 in pair_rect:
            self.lam_off.append(self.lam_off[-1] + (r1 - r0) * (c1 - c0))
        self.rect, self.pairs, self.pair_rect = rect, pairs, pair_rect
        self.send = {q: self._segments(rank, q) for q in range(self.world) if q != rank}
        self.recv = {q: self._segments(q, rank) for q in range(self.world) if q != rank}

    def _segments(self, sender: int, receiver: int):
        """[(array, offset, pitch, rows, cols)] in message order."""
        seg = []
        for k, (e, d) in enumerate(self.pairs):
            if self.owner[e] != sender or self.owner[d] != receiver:
                continue
            R = self.rect[e]
            r0, c0, r1, c1 = self.pair_rect[k]
            pitch = R[3] - R[1]
            seg.append(("u", self.u_off[e] + (r0 - R[0]) * pitch + (c0 - R[1]), pitch, r1 - r0, c1 - c0))
            seg.append(("lam", self.lam_off[k], c1 - c0, r1 - r0, c1 - c0))
        if self.blind:
            mm = self.m * self.m
            for e in range(len(self.rect)):
                if self.owner[e] == sender:
                    seg.append(("W", e * mm, self.m, self.m, self.m))
                    seg.append(("Delta", e * mm, self.m, self.m, self.m))
        return seg

    @staticmethod
    def size(segs) -> int:
        return sum(rows * cols for _, _, _, rows, cols in segs)

    def pack(self, peer: int, arrays: dict):
        """The message for `peer` from this rank's arrays {"u", "lam", "W", "Delta"} (flat)."""
        segs = self.send[peer]
        ref = arrays["u"]
        out = ref.new_empty(self.size(segs)) if hasattr(ref, "new_empty") else \
            __import__("numpy").empty(self.size(segs), ref.dtype)
        k = 0
        for name, off, pitch, rows, cols in segs:
            a = arrays[name]
            for r in range(rows):
                out[k:k + cols] = a[off + r * pitch:off + r * pitch + cols]
                k += cols
        return out

    def unpack(self, peer: int, msg, arrays: dict) -> None:
        """Write the message from `peer` into this rank's halo copies (in place)."""
        k = 0
        for name, off, pitch, rows, cols in self.recv[peer]:
            a = arrays[name]
            for r in range(rows):
                a[off + r * pitch:off + r * pitch + cols] = msg[k:k + cols]
                k += cols


def exchange_halos(sched: HaloSchedule, arrays: dict, group=None) -> None:
    """One halo exchange over torch.distributed (any backend that has isend /
    irecv): every rank packs its strips for each peer, the messages cross, and
    each rank unpacks what it received.  `arrays` holds complex torch tensors
    on the process group's device."""
    ops, inbox = [], {}
    for q, segs in sched.recv.items():
        n = HaloSchedule.size(segs)
        if n:
            buf = torch.empty(n, dtype=arrays["u"].dtype, device=arrays["u"].device)
            inbox[q] = buf
            ops.append(dist.P2POp(dist.irecv, torch.view_as_real(buf), q, group))
    for q, segs in sched.send.items():
        if HaloSchedule.size(segs):
            ops.append(dist.P2POp(dist.isend, torch.view_as_real(sched.pack(q, arrays)), q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for q, buf in inbox.items():
        sched.unpack(q, buf, arrays)


def exchange_shard_halos(plan, group=None) -> None:
    """One halo exchange of a library shard plan (api.ptycho_plan_shard) over
    torch.distributed: the library packs each peer's message on the device, the
    messages cross by isend / irecv (NCCL between GPUs), and the library
    unpacks what arrived.  Call it before every od2p_iterate(plan, 1)."""
    from . import api
    world = max(plan.owner) + 1
    ops, inbox = [], {}
    for q in range(world):
        if q == plan.rank:
            continue
        n_send, n_recv = api.od2p_halo_size(plan, q)
        if n_recv:
            buf = torch.empty(n_recv, dtype=torch.complex64, device=plan.device)
            inbox[q] = buf
            ops.append(dist.P2POp(dist.irecv, torch.view_as_real(buf), q, group))
        if n_send:
            ops.append(dist.P2POp(dist.isend, torch.view_as_real(api.od2p_halo_pack(plan, q)), q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for q, buf in inbox.items():
        api.od2p_halo_unpack(plan, q, buf)


def exchange_local(shards) -> None:
    """The halo exchange among shard plans held by one process (shards[r] is
    rank r's): every message is packed first, then every message unpacked."""
    from . import api
    msgs = {}
    for a, pa in enumerate(shards):
        for b in range(len(shards)):
            if a != b and api.od2p_halo_size(pa, b)[0]:
                msgs[(a, b)] = api.od2p_halo_pack(pa, b)
    for (a, b), msg in msgs.items():
        api.od2p_halo_unpack(shards[b], a, msg)
