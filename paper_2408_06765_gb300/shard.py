"""Target-sharded RSI chain: the stages of one chain split over several
processes, one GPU each.

Within a stage every target's value is a sum over the source points of its
own (Eq. incident_field for the piston, Eq. rayleigh_sommerfeld for an
interface), independent of every other target.  So the targets of each stage
are split among the ranks, and the only data a rank needs from the others is
the source density of the next stage:

  * every rank regenerates every QMC point set from (seed, set_id): no point
    data is exchanged;
  * interface stage s: rank r computes the field on its contiguous share of
    the interface's point slots, applies the transmission coefficient
    (Eq. transmission_coefficient) on that share, and ONE all-gather of the
    complex amplitudes, in slot order, gives every rank the whole source
    density of the next stage;
  * the image: rank r computes its contiguous block of image rows; a last
    gather assembles the image.

The host logic here is device-neutral.  A rank's steps are a generator that
yields at each gather, so the same steps run

  * as one process per rank (`run_rank`), the gather being a collective
    (torch.distributed all-gather: NCCL on GPUs, gloo on CPUs), or
  * as all ranks in one process, one after another (`run_emulated`), the
    gather being a concatenation -- no rank ever waits for another.

The stage sums come from a backend object.  `LibrsiBackend` runs every step
in librsi's kernels (rsi_make_qmc_points, rsi_points_slice,
rsi_propagate_stage(_multi), rsi_interface_transmit, rsi_field_image); tests
can pass other backends with the same methods.  1-4 workloads that differ only
in frequency run together, each stage evaluating all frequencies on the shared
points (Sec. 4: a broadband field is a superposition of single frequencies).
"""
from __future__ import annotations

import math


def share(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of n items for `rank` of `world`: the first
    n % world ranks take one item more than the others."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if n < 0:
        raise ValueError("negative item count")
    q, r = divmod(int(n), int(world))
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shares(n: int, world: int) -> list[int]:
    """Item counts of every rank's share, in rank order."""
    return [hi - lo for lo, hi in (share(n, world, r) for r in range(world))]


def _wavenumber(freq: float, c: float) -> float:
    return 2.0 * math.pi * float(freq) / float(c)


def _check_family(cfgs: list) -> None:
    if not 1 <= len(cfgs) <= 4:
        raise ValueError("a sharded chain takes 1-4 workloads")
    strip = lambda c: {k: v for k, v in c.items() if k not in ("freq", "name")}
    if any(strip(c) != strip(cfgs[0]) for c in cfgs[1:]):
        raise ValueError("the workloads of a sharded chain may differ only in frequency")


def rank_steps(cfgs: list, rank: int, world: int, be):
    """The steps of `rank`: a generator that yields (local amplitudes
    [nf, share], total count) at each gather and expects the gathered
    [nf, total] amplitudes back; it returns ((row0, row1), image rows
    [nf, row1 - row0, nx] or None for an empty share)."""
    _check_family(cfgs)
    cfg = cfgs[0]
    seed = int(cfg.get("seed", 0))
    v0 = float(cfg.get("v0", 1.0))
    media = cfg["media"]
    C = math.sin(float(cfg["piston"].get("tilt", 0.0))) / float(media[0]["c"])
    mode = cfg.get("tmode", "global")
    freqs = [float(c["freq"]) for c in cfgs]
    nf = len(freqs)
    pc = cfg["piston"]
    src = be.points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]))
    sigma = None        # source density of the next stage (None: the piston)
    src_curved = False  # the sources carry their own normals

    def stage(ks, tgt):
        if sigma is None:
            return be.piston(ks, v0, src, tgt)
        return be.rsi(ks, src_curved, src, sigma, tgt)

    for s, it in enumerate(cfg["interfaces"]):
        n = int(it["n"])
        pts = be.points(it, seed, int(it["set_id"]), n)
        lo, hi = share(n, world, rank)
        if hi > lo:
            tgt = be.slice(pts, lo, hi)
            phi = stage([_wavenumber(f, media[s]["c"]) for f in freqs], tgt)
            local = be.transmit(tgt, phi, media[s], media[s + 1], C, mode)
        else:
            local = be.empty(nf)
        sigma = yield local, n
        src, src_curved = pts, it["kind"] != "rect"
    g = cfg["grid"]
    nx, nz = int(g["nx"]), int(g["nz"])
    r0, r1 = share(nz, world, rank)
    if r1 == r0:
        return (r0, r1), None
    tgt = be.slice(be.grid(g), r0 * nx, r1 * nx)
    k_last = [_wavenumber(f, media[len(cfg["interfaces"])]["c"]) for f in freqs]
    phi = stage(k_last, tgt)
    return (r0, r1), be.image(phi, k_last, v0, nx, r1 - r0)


def run_rank(cfgs: list, rank: int, world: int, be, allgather):
    """This process's rank of a sharded chain.  allgather(local [nf, share],
    total) must return the [nf, total] concatenation of every rank's share in
    rank order.  Returns ((row0, row1), image rows or None)."""
    steps = rank_steps(cfgs, rank, world, be)
    try:
        local, total = next(steps)
        while True:
            local, total = steps.send(allgather(local, total))
    except StopIteration as done:
        return done.value


def run_emulated(cfgs: list, world: int, be) -> list:
    """Every rank of a sharded chain in this process, one after another (the
    gathers are concatenations).  Returns each rank's ((row0, row1), rows)."""
    gens = [rank_steps(cfgs, r, world, be) for r in range(world)]
    msgs = [next(g) for g in gens]
    while True:
        total = msgs[0][1]
        full = be.concat([m[0] for m in msgs], total)
        out, done = [], []
        for g in gens:
            try:
                out.append(g.send(full))
            except StopIteration as stop:
                done.append(stop.value)
        if done:
            if out:
                raise RuntimeError("ranks of a sharded chain finished at different stages")
            return done
        msgs = out


def assemble(results: list, be):
    """The image [nf, nz, nx] from every rank's ((row0, row1), rows)."""
    parts = [rows for (_, rows) in sorted(results, key=lambda t: t[0][0]) if rows is not None]
    return be.cat_rows(parts)


def row_counts(cfgs: list, world: int) -> list[int]:
    """Image values (rows x nx) of every rank's block of rows, in rank order."""
    nx, nz = int(cfgs[0]["grid"]["nx"]), int(cfgs[0]["grid"]["nz"])
    return [c * nx for c in shares(nz, world)]


def torch_allgather(world: int):
    """allgather for run_rank over torch.distributed: complex amplitudes as
    real pairs, every share padded to the largest one (all_gather needs equal
    sizes), trimmed and concatenated in rank order.  The shares are those of
    `shares(total, world)` unless `counts` gives them (the image rows)."""
    import torch
    import torch.distributed as dist

    def gather(local, total: int, counts: list | None = None):
        counts = counts or shares(total, world)
        if sum(counts) != total or local.shape[1] != counts[dist.get_rank()]:
            raise ValueError("the local share does not match the partition")
        width = max(counts)
        nf = local.shape[0]
        buf = torch.zeros((nf, width, 2), dtype=torch.float64, device=local.device)
        if local.shape[1]:
            buf[:, :local.shape[1]] = torch.view_as_real(local)
        got = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(got, buf)
        full = torch.cat([g[:, :c] for g, c in zip(got, counts)], dim=1)
        return torch.view_as_complex(full.contiguous())

    return gather


class LibrsiBackend:
    """Stage steps in librsi's kernels (device tensors, complex128 fields)."""

    def __init__(self, precision: str = "fp32c", device="cuda", stream=None):
        from . import rsi
        self.lib = rsi  # the binding (the method `rsi` below is the RSI stage)
        self.prec = precision
        self.device = device
        self.stream = stream
        self.ws = rsi.Workspace(device)

    def points(self, surf, seed, set_id, n):
        return self.lib.make_qmc_points(surf, seed, set_id, n, device=self.device, stream=self.stream)

    def grid(self, g):
        return self.lib.grid_points(g, device=self.device, stream=self.stream)

    def slice(self, pts, lo, hi):
        return self.lib.points_slice(pts, lo, hi - lo, stream=self.stream)

    def _stage(self, st, ks, src, sigma, tgt):
        r = self.lib
        if len(ks) == 1 or self.prec != "fp32c":
            out = []
            for f, k in enumerate(ks):
                st.k = float(k)
                out.append(r.propagate_stage(st, src, None if sigma is None else sigma[f].contiguous(), tgt,
                                             workspace=self.ws, stream=self.stream))
            import torch
            return torch.stack(out)
        return r.propagate_stage_multi(st, ks, src, sigma, tgt, workspace=self.ws, stream=self.stream)

    def piston(self, ks, v0, src, tgt):
        st = self.lib.stage_struct(self.lib.STAGE_PISTON, self.prec, ks[0], v0)
        return self._stage(st, ks, src, None, tgt)

    def rsi(self, ks, curved, src, sigma, tgt):
        r = self.lib
        st = r.stage_struct(r.STAGE_RSI, self.prec, ks[0], 1.0, r.NORMALS_POINTS if curved else r.NORMALS_Z)
        return self._stage(st, ks, src, sigma, tgt)

    def transmit(self, pts, phi, m_in, m_out, C, mode):
        import torch
        out = torch.empty_like(phi)
        for f in range(phi.shape[0]):
            self.lib.interface_transmit(pts, phi[f], m_in, m_out, C, mode, out=out[f], stream=self.stream)
        return out

    def image(self, phi, ks, v0, nx, rows):
        import torch
        g = {"x0": 0.0, "x1": 1.0, "z0": 0.0, "z1": 1.0, "nx": nx, "nz": rows}  # only nx, nz are used
        return torch.stack([self.lib.field_image(g, phi[f], k, v0, stream=self.stream) for f, k in enumerate(ks)])

    def empty(self, nf):
        import torch
        return torch.empty((nf, 0), dtype=torch.complex128, device=self.device)

    def concat(self, parts, total):
        import torch
        full = torch.cat(parts, dim=1)
        assert full.shape[1] == total
        return full

    def cat_rows(self, parts):
        import torch
        return torch.cat(parts, dim=1)
