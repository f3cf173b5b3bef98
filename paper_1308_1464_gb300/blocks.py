"""A grid decomposed into blocks, one block per rank, stepped block by block.

The update of a cell reads cells up to two away, its diagonal neighbours
included through the transverse terms (LeVeque 2002, §21.8), so a block
needs, before every step, two ghost layers from the blocks beside it; the
global boundary keeps its boundary kinds, and a periodic direction split
over several blocks wraps from the last block to the first.  The step size
of the whole grid follows from the largest wave speed over all blocks (the
variable time-step rule of the paper's "dynamic time stepping", §1.2,
Table 1), one max-reduction per step.

The ghost fill runs in two phases, x then y, so that the corner ghosts of a
block come out as in the single-grid fill: phase x exchanges the two columns
next to each shared x side (interior rows) and fills the physical x sides;
phase y then exchanges the two rows next to each shared y side across the
full padded width, x ghost columns included, and fills the physical y sides.

This module is marshalling and message passing only.  Packing, unpacking,
ghost fills and steps are done by a block's ``ops`` (``DeviceBlockOps``: the
library's kernels through the C ABI); messages go through a transport
(``DistTransport``: torch.distributed point-to-point, one rank per block) or,
for every block held by one process, through ``exchange_local``.
"""
from __future__ import annotations

import contextlib
import copy
from dataclasses import dataclass

from . import BC_GIVEN, BC_PERIODIC, Context, McError, MC_EINVAL

XLO, XHI, YLO, YHI = 0, 1, 2, 3


def lpt_shards(weights, nparts: int):
    """Independent units (patches, interfaces) shared among nparts ranks by
    greedy longest processing time: units in decreasing weight, each to the
    currently lightest part (ties go to the lower part index).  Each shard
    lists its units in increasing index order.  The heaviest part is at most
    4/3 - 1/(3 nparts) times the best possible (Graham's bound)."""
    import heapq
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    order = sorted(range(len(weights)), key=lambda k: (-weights[k], k))
    heap = [(0, part) for part in range(nparts)]
    shards = [[] for _ in range(nparts)]
    for k in order:
        load, part = heapq.heappop(heap)
        shards[part].append(k)
        heapq.heappush(heap, (load + weights[k], part))
    return [sorted(s) for s in shards]


def split(n: int, parts: int):
    """Sizes and offsets of `parts` near-equal pieces of n cells (the first
    n % parts pieces one cell larger)."""
    base, extra = divmod(n, parts)
    sizes = [base + (1 if k < extra else 0) for k in range(parts)]
    offsets = [sum(sizes[:k]) for k in range(parts)]
    return sizes, offsets


@dataclass(frozen=True)
class Extent:
    i0: int
    j0: int
    mx: int
    my: int


class Decomposition:
    """px x py blocks of a global problem; rank r is block (r % px, r // px)."""

    def __init__(self, problem, px: int, py: int):
        if px < 1 or py < 1:
            raise ValueError("px and py must be positive")
        if problem.mx < 2 * px or problem.my < 2 * py:
            raise ValueError(f"{problem.mx} x {problem.my} cells cannot give {px} x {py} blocks "
                             "of at least 2 x 2 cells")
        self.problem = problem
        self.px, self.py = px, py
        self.nx, self.ox = split(problem.mx, px)
        self.ny, self.oy = split(problem.my, py)

    @property
    def nblocks(self) -> int:
        return self.px * self.py

    def coords(self, rank: int):
        return rank % self.px, rank // self.px

    def rank_of(self, bx: int, by: int) -> int:
        return by * self.px + bx

    def extent(self, rank: int) -> Extent:
        bx, by = self.coords(rank)
        return Extent(self.ox[bx], self.oy[by], self.nx[bx], self.ny[by])

    def neighbour(self, rank: int, side: int):
        """Rank whose interior provides the ghosts on `side`, or None where
        the side keeps the global boundary kind (a periodic direction of a
        single block wraps onto itself through its own boundary kind)."""
        bx, by = self.coords(rank)
        n = self.px if side < 2 else self.py
        b = bx if side < 2 else by
        b += -1 if side % 2 == 0 else 1
        if 0 <= b < n:
            pass
        elif self.problem.bc[side] == BC_PERIODIC and n > 1:
            b %= n
        else:
            return None
        return self.rank_of(b, by) if side < 2 else self.rank_of(bx, b)

    def local_problem(self, rank: int):
        """The block's problem: its own size, MC_BC_GIVEN on shared sides."""
        e = self.extent(rank)
        p = copy.copy(self.problem)
        p.mx, p.my = e.mx, e.my
        for side in range(4):
            if self.neighbour(rank, side) is not None:
                p.bc[side] = BC_GIVEN
        return p

    def messages(self, rank: int, direction: int):
        """The halo messages of one phase (direction 0: x, 1: y).

        sends: (side, dst) -- the strip next to `side` of this block, for the
        ghosts on the opposite side of dst; recvs: (side, src) -- the ghosts
        on `side`.  A message's tag is the receiving side.  Sends are listed
        in decreasing side order and receives in increasing order: with two
        blocks in a periodic direction both sides of a block face the same
        peer, and transports without tags match the messages of a pair in
        posting order, which these orders keep consistent."""
        sides = (2 * direction, 2 * direction + 1)
        sends = [(s, self.neighbour(rank, s)) for s in reversed(sides)
                 if self.neighbour(rank, s) is not None]
        recvs = [(s, self.neighbour(rank, s)) for s in sides if self.neighbour(rank, s) is not None]
        return sends, recvs


class Block:
    """One rank's block: its problem, its ops, and the halo buffers."""

    def __init__(self, decomp: Decomposition, rank: int, ops):
        self.decomp = decomp
        self.rank = rank
        self.ops = ops
        self.problem = decomp.local_problem(rank)
        self._send = {s: ops.alloc(ops.halo_elems(s)) for s in range(4)
                      if decomp.neighbour(rank, s) is not None}
        self._recv = {s: ops.alloc(ops.halo_elems(s)) for s in range(4)
                      if decomp.neighbour(rank, s) is not None}

    def outgoing(self, q, direction: int):
        """Pack the strips of one phase: [(dst, tag, buffer)]."""
        sends, _ = self.decomp.messages(self.rank, direction)
        out = []
        for side, dst in sends:
            buf = self._send[side]
            self.ops.pack(q, side, buf)
            out.append((dst, side ^ 1, buf))
        return out

    def incoming(self, direction: int):
        """Receive buffers of one phase: [(src, tag, buffer)]."""
        _, recvs = self.decomp.messages(self.rank, direction)
        return [(src, side, self._recv[side]) for side, src in recvs]

    def finish(self, q, direction: int) -> None:
        """Unpack the received strips of one phase, then fill the physical
        sides of that direction."""
        _, recvs = self.decomp.messages(self.rank, direction)
        for side, _ in recvs:
            self.ops.unpack(self._recv[side], side, q)
        self.ops.fill_dir(q, direction)


def exchange(block: Block, q, transport) -> None:
    """The two-phase ghost fill of one rank's block."""
    for direction in (0, 1):
        out = block.outgoing(q, direction)
        inc = block.incoming(direction)
        transport.exchange(out, inc)
        block.finish(q, direction)


def exchange_local(blocks, qs) -> None:
    """The two-phase ghost fill of every block, all held by this process."""
    for direction in (0, 1):
        mail = {}
        for b, q in zip(blocks, qs):
            for dst, tag, buf in b.outgoing(q, direction):
                mail[(b.rank, dst, tag)] = buf
        for b, q in zip(blocks, qs):
            for src, tag, buf in b.incoming(direction):
                b.ops.copy(mail.pop((src, b.rank, tag)), buf)
            b.finish(q, direction)
        if mail:
            raise RuntimeError(f"unmatched halo messages: {sorted(mail)}")


def _on_stream(blocks):
    """Torch's current stream set to the blocks' stream for device blocks (a
    transport's collectives and tensor copies then queue behind their
    kernels); nothing for host blocks."""
    s = getattr(blocks[0].ops, "torch_stream", None) if blocks else None
    if s is None:
        return contextlib.nullcontext()
    import torch
    return torch.cuda.stream(s)


class Stepper:
    """Steps of a decomposed grid with one global time step.

    `blocks` are the blocks this process holds (one per rank with a
    transport, or all of them with ``transport=None``); states are passed as
    lists in the same order."""

    def __init__(self, blocks, transport=None):
        self.blocks = list(blocks)
        self.transport = transport
        if transport is not None and len(self.blocks) != 1:
            raise ValueError("a transport serves one block per rank")

    def fill(self, qs) -> None:
        if self.transport is None:
            exchange_local(self.blocks, qs)
        else:
            exchange(self.blocks[0], qs[0], self.transport)

    def _max(self, values) -> float:
        v = max(values)
        return v if self.transport is None else self.transport.max(v)

    def max_cell_speed(self, qs) -> float:
        return self._max([b.ops.max_speed(q) for b, q in zip(self.blocks, qs)])

    def step(self, qs_in, qs_out, dt: float) -> float:
        """One step of every block with dt; returns the global smax of the
        step's waves (Courant number = dt * smax)."""
        with _on_stream(self.blocks):
            self.fill(qs_in)
            return self._max([b.ops.step(qi, qo, dt) for b, qi, qo in zip(self.blocks, qs_in, qs_out)])

    def advance(self, qa, qb, nsteps: int, cfl_desired: float, cfl_max: float, t: float = 0.0,
                dt: float | None = None):
        """nsteps accepted steps with the variable time-step rule: an attempt
        whose Courant number exceeds cfl_max is retaken with
        dt = cfl_desired / smax; an accepted one proposes that dt for the
        next.  Returns (t, dt, result_in_b, nrejected)."""
        if dt is None:
            dt = cfl_desired / self.max_cell_speed(qa)
        cur, nxt = qa, qb
        in_b, nacc, nrej = False, 0, 0
        while nacc < nsteps:
            if nacc + nrej > 100 * nsteps + 100:
                raise McError(MC_EINVAL, "too many rejected steps")
            smax = self.step(cur, nxt, dt)
            if smax > 0 and dt * smax > cfl_max:
                nrej += 1
            else:
                t += dt
                nacc += 1
                cur, nxt = nxt, cur
                in_b = not in_b
            if smax > 0:
                dt = cfl_desired / smax
        return t, dt, in_b, nrej


class DistTransport:
    """Halo messages and the speed maximum over torch.distributed (one rank
    per block).  With the gloo backend device buffers are staged through
    host memory; NCCL sends device buffers directly."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.backend = dist.get_backend(group)

    def _stage(self, t):
        return t.cpu() if (self.backend == "gloo" and t.is_cuda) else t

    def exchange(self, sends, recvs) -> None:
        import torch
        dist = self.dist
        if not sends and not recvs:
            return
        staged = [(src, tag, buf, self._stage(torch.empty_like(buf)) if buf.is_cuda and
                   self.backend == "gloo" else buf) for src, tag, buf in recvs]
        ops = [dist.P2POp(dist.isend, self._stage(buf), dst, self.group, tag)
               for dst, tag, buf in sends]
        ops += [dist.P2POp(dist.irecv, host, src, self.group, tag) for src, tag, _, host in staged]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        for _, _, buf, host in staged:
            if host is not buf:
                buf.copy_(host)

    def max(self, value: float) -> float:
        import torch
        dist = self.dist
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def max_tensor(self, t) -> None:
        """In-place max-reduction of a one-element tensor over the ranks
        (NCCL: on the device, no host read; gloo: through host memory)."""
        dist = self.dist
        if self.backend == "gloo" and t.is_cuda:
            h = t.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.MAX, group=self.group)
            t.copy_(h)
        else:
            dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)


class DeviceBlockOps:
    """A block's packing, unpacking, ghost fills and steps: the library's
    kernels through the C ABI.  States are device addresses; halo buffers
    are torch tensors on the context's device."""

    def __init__(self, ctx: Context, stream: int = 0):
        import torch
        self.ctx = ctx
        self.stream = stream
        self.dtype = torch.float64 if ctx.layout.elem_bytes == 8 else torch.float32
        # the same stream as torch sees it: tensor copies, reductions and
        # collectives issued for this block queue behind its kernels there
        self.torch_stream = (torch.cuda.default_stream() if stream == 0
                             else torch.cuda.ExternalStream(stream))

    def halo_elems(self, side: int) -> int:
        return self.ctx.halo_elems(side)

    def alloc(self, n: int):
        import torch
        return torch.empty(int(n), dtype=self.dtype, device="cuda")

    def copy(self, src, dst) -> None:
        # on torch's current stream: the steppers make it this block's
        # stream (or, while an attempt is captured, the capturing stream)
        dst.copy_(src)

    def pack(self, q: int, side: int, buf) -> None:
        self.ctx.halo_pack(q, side, buf.data_ptr(), self.stream)

    def unpack(self, buf, side: int, q: int) -> None:
        self.ctx.halo_unpack(buf.data_ptr(), side, q, self.stream)

    def fill_dir(self, q: int, direction: int) -> None:
        self.ctx.bc_fill_dir(q, direction, self.stream)

    def step(self, q_in: int, q_out: int, dt: float) -> float:
        return self.ctx.step(q_in, q_out, dt, True, self.stream)

    def max_speed(self, q: int) -> float:
        return self.ctx.max_cell_speed(q, self.stream)


class DeviceStepper:
    """Steps of a decomposed grid with the time-step state on the device
    (mc_block_*): per attempt the two-phase halo exchange of the current
    buffer, the fused step with the device dt, a max-reduction of the speed
    maximum over the blocks, and the accept/reject rule on each block's
    device; the host reads nothing back until the attempts are enqueued.
    With a transport (one block per rank) the strips and the maximum travel
    through it: NCCL moves device buffers and reduces the device scalar in
    place; gloo stages them through host memory.  Without one, every block is
    held by this process and the exchange and reduction are device copies;
    an attempt is then captured once into a CUDA graph (graph=True) and
    replayed, since every launch of it reads the device state alone.

    Blocks must use DeviceBlockOps, all on one stream; states are passed as
    lists of the two buffers of each block (qa, qb), the current one chosen
    on the device."""

    def __init__(self, blocks, transport=None, graph: bool = True):
        import torch
        self.blocks = list(blocks)
        self.transport = transport
        if transport is not None and len(self.blocks) != 1:
            raise ValueError("a transport serves one block per rank")
        if len({b.ops.stream for b in self.blocks}) != 1:
            raise ValueError("the blocks' operations must share one stream")
        # the speed maximum of each block's attempt: int64 bits of a
        # non-negative double (ordered like the doubles)
        self.smax = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in self.blocks]
        self.graph = graph and transport is None
        self._graphs = {}

    def _ctx(self, b):
        return b.ops.ctx

    def _exchange(self, qas, qbs, stream) -> None:
        for direction in (0, 1):
            mail = {}
            outs = []
            for b, qa, qb in zip(self.blocks, qas, qbs):
                sends, _ = b.decomp.messages(b.rank, direction)
                out = []
                for side, dst in sends:
                    buf = b._send[side]
                    self._ctx(b).block_pack(qa, qb, side, buf.data_ptr(), stream)
                    out.append((dst, side ^ 1, buf))
                    mail[(b.rank, dst, side ^ 1)] = buf
                outs.append(out)
            if self.transport is None:
                for b in self.blocks:
                    for src, tag, buf in b.incoming(direction):
                        b.ops.copy(mail.pop((src, b.rank, tag)), buf)
                if mail:
                    raise RuntimeError(f"unmatched halo messages: {sorted(mail)}")
            else:
                b = self.blocks[0]
                self.transport.exchange(outs[0], b.incoming(direction))
            for b, qa, qb in zip(self.blocks, qas, qbs):
                _, recvs = b.decomp.messages(b.rank, direction)
                for side, _src in recvs:
                    self._ctx(b).block_unpack(b._recv[side].data_ptr(), side, qa, qb, stream)
                self._ctx(b).block_fill_dir(qa, qb, direction, stream)

    def _reduce_max(self) -> None:
        if self.transport is None:
            if len(self.smax) > 1:
                m = self.smax[0]
                for s in self.smax[1:]:
                    m = m.maximum(s)
                for s in self.smax:
                    s.copy_(m)
        else:
            self.transport.max_tensor(self.smax[0])

    def _attempt(self, qas, qbs, cfl_desired: float, cfl_max: float, stream) -> None:
        self._exchange(qas, qbs, stream)
        for b, qa, qb, sm in zip(self.blocks, qas, qbs, self.smax):
            self._ctx(b).block_sweep(qa, qb, sm.data_ptr(), stream)
        self._reduce_max()
        for b, sm in zip(self.blocks, self.smax):
            self._ctx(b).block_dt_rule(sm.data_ptr(), cfl_desired, cfl_max, stream)

    def _attempt_graph(self, qas, qbs, cfl_desired: float, cfl_max: float):
        """The captured attempt for these buffers and CFL numbers, captured
        after an eager attempt has encoded the buffers' tensor maps; the
        attempt with the two buffers' roles exchanged is captured with it
        (capturing runs nothing), so a later call that starts from the other
        buffer finds its graph ready."""
        import torch
        key = (tuple(qas), tuple(qbs), float(cfl_desired), float(cfl_max))
        if key not in self._graphs:
            for a, b in ((qas, qbs), (qbs, qas)):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self._attempt(a, b, cfl_desired, cfl_max, torch.cuda.current_stream().cuda_stream)
                self._graphs[(tuple(a), tuple(b), float(cfl_desired), float(cfl_max))] = g
        return self._graphs[key]

    def max_cell_speed(self, qas) -> float:
        v = max(b.ops.max_speed(q) for b, q in zip(self.blocks, qas))
        return v if self.transport is None else self.transport.max(v)

    def advance(self, qas, qbs, nsteps: int, cfl_desired: float, cfl_max: float, t: float = 0.0,
                dt: float | None = None):
        """nsteps accepted steps from the states in qas; returns (t, dt,
        result_in_b, nrejected), the same on every rank.  The reductions,
        copies, collectives and graph replays go to the blocks' stream."""
        import torch
        with torch.cuda.stream(self.blocks[0].ops.torch_stream):
            return self._advance(qas, qbs, nsteps, cfl_desired, cfl_max, t, dt)

    def _advance(self, qas, qbs, nsteps, cfl_desired, cfl_max, t, dt):
        if dt is None:
            dt = cfl_desired / self.max_cell_speed(qas)
        stream = self.blocks[0].ops.stream
        for b in self.blocks:
            self._ctx(b).block_begin(t, dt, b.ops.stream)
        attempts, total = nsteps, 0
        res = None
        while True:
            if attempts > 0:
                self._attempt(qas, qbs, cfl_desired, cfl_max, stream)
                if attempts > 1:
                    if self.graph:
                        g = self._attempt_graph(qas, qbs, cfl_desired, cfl_max)
                        for _ in range(attempts - 1):
                            g.replay()
                    else:
                        for _ in range(attempts - 1):
                            self._attempt(qas, qbs, cfl_desired, cfl_max, stream)
            total += attempts
            res = [self._ctx(b).block_end(b.ops.stream) for b in self.blocks]
            nacc = res[0][3]
            if nacc >= nsteps:
                break
            if total > 100 * nsteps + 100:
                raise McError(MC_EINVAL, "too many rejected steps")
            attempts = nsteps - nacc
        t, dt, cur, nacc, nrej = res[0]
        return t, dt, bool(cur), nrej
