"""The target-sharded chain (paper_2408_06765_gb300/shard.py) on the CPU.

A stage's targets are independent sums (Eq. incident_field, Eq.
rayleigh_sommerfeld), so splitting them among ranks, all-gathering the
transmitted amplitudes after each interface and concatenating the image rows
must reproduce the one-rank chain.  The per-rank stage sums here are the FP64
oracle's (the sharding logic takes them as a parameter; the product path
passes librsi's kernels), so the sharded result equals the oracle's own
one-rank chain to rounding -- in fact exactly, since every target's sum is the
same arithmetic in the same source order on either side."""
import copy
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2408_06765_gb300 import shard
from paper_2408_06765_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleBackend:
    """Stage steps of the FP64 oracle on numpy arrays (index order)."""

    def points(self, surf, seed, set_id, n):
        return oracle.make_points(surf, seed, set_id, n)

    def grid(self, g):
        return oracle.grid_points(g)

    def slice(self, pts, lo, hi):
        return {k: np.asarray(v)[lo:hi] for k, v in pts.items()}

    def piston(self, ks, v0, src, tgt):
        return np.stack([oracle.piston_field(src, tgt, k, v0) for k in ks])

    def rsi(self, ks, curved, src, sigma, tgt):
        return np.stack([oracle.rsi_field(src, sigma[f], tgt, k) for f, k in enumerate(ks)])

    def transmit(self, pts, phi, m_in, m_out, C, mode):
        return np.stack([oracle.transmit(pts, phi[f], m_in, m_out, C, mode)[0] for f in range(phi.shape[0])])

    def image(self, phi, ks, v0, nx, rows):
        return np.stack([(k / v0) * phi[f].reshape(rows, nx) for f, k in enumerate(ks)])

    def empty(self, nf):
        return np.zeros((nf, 0), np.complex128)

    def concat(self, parts, total):
        full = np.concatenate(parts, axis=1)
        assert full.shape[1] == total
        return full

    def cat_rows(self, parts):
        return np.concatenate(parts, axis=1)


def small_multilayer():
    cfg = W.c3_multilayer(curved=True, n_per_surface=301)
    cfg["grid"] = dict(cfg["grid"], nx=23, nz=13)
    return cfg


def ragged_family():
    return [W.small_ragged("fp64", freq=f, n_piston=257, n_iface=641, nx=17, nz=11) for f in (2.5e6, 4e6, 7.5e6)]


def one_rank(cfgs):
    return np.stack([oracle.field_image(c) for c in cfgs])


def test_shares_cover_every_item_once():
    for n in (0, 1, 5, 7, 64, 1000):
        for world in (1, 2, 3, 8):
            spans = [shard.share(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            counts = shard.shares(n, world)
            assert sum(counts) == n and max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        shard.share(10, 2, 2)


@pytest.mark.parametrize("world", [1, 2, 3, 16])
def test_emulated_ranks_reproduce_the_one_rank_chain(world):
    # 16 ranks for 13 image rows: some ranks hold no rows at all
    cfg = small_multilayer()
    be = OracleBackend()
    img = shard.assemble(shard.run_emulated([cfg], world, be), be)
    want = one_rank([cfg])
    assert img.shape == want.shape
    assert np.max(np.abs(img - want)) <= 1e-12 * np.max(np.abs(want))


def test_frequencies_share_the_sharded_points():
    cfgs = ragged_family()
    be = OracleBackend()
    img = shard.assemble(shard.run_emulated(cfgs, 3, be), be)
    want = one_rank(cfgs)
    assert np.max(np.abs(img - want)) <= 1e-12 * np.max(np.abs(want))


def test_workloads_must_share_their_geometry():
    cfgs = ragged_family()
    cfgs[1] = copy.deepcopy(cfgs[1])
    cfgs[1]["piston"]["n"] += 1
    with pytest.raises(ValueError):
        list(shard.rank_steps(cfgs, 0, 1, OracleBackend()))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, which, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from test_shard import OracleBackend, ragged_family, small_multilayer
    from paper_2408_06765_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfgs = [small_multilayer()] if which == "multilayer" else ragged_family()
    gather = sh.torch_allgather(world)
    # the oracle backend works on numpy arrays; the collective on CPU tensors
    to_np = lambda local, total, counts=None: gather(torch.from_numpy(local), total, counts).numpy()
    rows, img = sh.run_rank(cfgs, rank, world, OracleBackend(), to_np)
    nf, nx = len(cfgs), int(cfgs[0]["grid"]["nx"])
    local = np.zeros((nf, 0), np.complex128) if img is None else img.reshape(nf, -1)
    counts = sh.row_counts(cfgs, world)
    full = to_np(local, sum(counts), counts)
    out.put((rank, rows, full))
    dist.destroy_process_group()


@pytest.mark.parametrize("which", ["multilayer", "frequencies"])
def test_two_gloo_ranks_reproduce_the_one_rank_chain(which):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, which, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = []
    while len(res) < len(procs):
        try:
            res.append(q.get(timeout=5))
        except Exception:
            assert all(p.is_alive() or p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res.sort(key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfgs = [small_multilayer()] if which == "multilayer" else ragged_family()
    want = one_rank(cfgs)
    nz = int(cfgs[0]["grid"]["nz"])
    assert [r[1] for r in res] == [shard.share(nz, 2, 0), shard.share(nz, 2, 1)]
    for _, _, full in res:  # every rank holds the whole image after the last gather
        img = full.reshape(want.shape)
        assert np.max(np.abs(img - want)) <= 1e-12 * np.max(np.abs(want))


def test_librsi_backend_offers_every_step():
    """The product backend has every step the rank logic calls (constructing
    it allocates nothing, so this runs without a GPU)."""
    be = shard.LibrsiBackend("fp32c", device="cuda")
    for name in ("points", "grid", "slice", "piston", "rsi", "transmit", "image", "empty", "concat", "cat_rows"):
        assert callable(getattr(be, name)), name
    assert callable(getattr(OracleBackend(), "rsi"))
