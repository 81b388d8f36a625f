"""Work across GPUs: placement of independent lattices and requests, and one
lattice split into y-slabs with one slab per rank.

Independent lattices (batches, served requests) share nothing, so they are
placed whole: ``partition_by_bytes`` spreads them over the ranks by their
device bytes (largest first onto the least-loaded rank), each rank steps its
share with the single-GPU library, and ``gather_by_index`` brings the
results back to rank 0 in the original order.  No data crosses ranks while
they step.

One large periodic lattice is split into slabs of whole rows (section 2.1,
Eq. blbs: row y couples only to rows y - 1 and y + 1).  ``SlabRank`` holds
this rank's slab (``lbm_slab_create``) and, between steps, packs the rows
that cross its two boundaries, exchanges them with the neighbouring ranks
through torch.distributed point-to-point operations (NCCL between GPUs), and
unpacks what it received (``lbm_slab_pack`` / ``lbm_slab_unpack``).  The
exchange logic (``slab_rows``, ``neighbours``, ``exchange``) is plain
torch.distributed and works on CPU tensors with the gloo backend as well.
"""
import numpy as np

ESIZE = {0: 8, 1: 4, 2: 2, 3: 2, 4: 8}  # bytes per stored population, by storage type


def lattice_bytes(nx, ny, dtype):
    """Device bytes of one lattice's two population buffers (row padding not
    counted): the quantity placement balances."""
    return 2 * 9 * int(nx) * int(ny) * ESIZE[int(dtype)]


def partition_by_bytes(sizes, parts):
    """Indices of `sizes` split into `parts` lists with nearly equal sums:
    items in decreasing size (ties by index) each go to the part with the
    smallest sum so far (ties by part number).  Deterministic; every index
    appears once; the largest part exceeds the mean by at most the largest
    item."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * parts
    out = [[] for _ in range(parts)]
    for i in order:
        p = min(range(parts), key=lambda q: (load[q], q))
        out[p].append(i)
        load[p] += sizes[i]
    for lst in out:
        lst.sort()
    return out


def gather_by_index(local, world, rank, dst=0):
    """local: {index: result} of this rank.  Returns, on rank dst, the list of
    all ranks' results ordered by index (None elsewhere)."""
    import torch.distributed as dist

    if world == 1:
        return [local[k] for k in sorted(local)]
    objs = [None] * world if rank == dst else None
    dist.gather_object(local, objs, dst=dst)
    if rank != dst:
        return None
    merged = {}
    for d in objs:
        for k, v in d.items():
            if k in merged:
                raise RuntimeError("index %d placed on two ranks" % k)
            merged[k] = v
    return [merged[k] for k in sorted(merged)]


# --------------------------------------------------------------- slabs
def slab_rows(ny, world):
    """(first row, rows) of every rank's slab: rank k owns rows
    [floor(k ny / world), floor((k + 1) ny / world)), as lbm_slabs_create."""
    if world < 1 or ny < world:
        raise ValueError("need 1 <= world <= ny")
    return [(k * ny // world, (k + 1) * ny // world - k * ny // world) for k in range(world)]


def neighbours(rank, world):
    """(rank below, rank above) on the periodic ring of slabs."""
    return (rank - 1) % world, (rank + 1) % world


def exchange(to_below, to_above, from_below, from_above, rank, world):
    """Send to_below to the rank below and to_above to the rank above;
    receive into from_below what the rank below sent upwards and into
    from_above what the rank above sent downwards.  Sends are posted upward
    part first and receives lower part first on every rank, so that with two
    ranks (where both neighbours are the same rank, and NCCL matches messages
    between a pair of ranks in order) each part still lands in its place."""
    if world == 1:
        from_below.copy_(to_above)
        from_above.copy_(to_below)
        return
    import torch.distributed as dist

    below, above = neighbours(rank, world)
    ops = [dist.P2POp(dist.isend, to_above, above, tag=1),
           dist.P2POp(dist.isend, to_below, below, tag=2),
           dist.P2POp(dist.irecv, from_below, below, tag=1),
           dist.P2POp(dist.irecv, from_above, above, tag=2)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


class SlabRank:
    """This rank's slab of one nx x ny periodic lattice (one GPU per rank).

    Stepping runs one library step, then the forward halo exchange; an
    initialisation is followed by the reverse exchange (see lbm_slab_pack).
    The halo buffers are CUDA tensors on this rank's device; the pack is
    waited for before the transport starts and the transport before the
    unpack (host synchronisation on both sides, whatever streams the
    transport uses).  With a process group whose backend moves host tensors
    only (gloo), the outgoing parts are staged through host memory."""

    def __init__(self, L, nx, ny, S, rank, world, rho0=1.0, u0=(0.0, 0.0), dtype=None):
        import torch

        self.L, self.nx, self.ny = L, nx, ny
        self.rank, self.world = rank, world
        self.y0, self.rows = slab_rows(ny, world)[rank]
        dtype = L.LBM_F32DEV if dtype is None else dtype
        self.h = L.lbm_slab_create(nx, ny, self.y0, self.rows, S, rho0, u0, dtype)
        nb = L.lbm_slab_halo_bytes(self.h)
        dev = torch.cuda.current_device()
        self.buf = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(4)]
        self.host = None
        if world > 1:
            import torch.distributed as dist

            if dist.get_backend() != "nccl":
                self.host = [torch.empty(nb, dtype=torch.uint8) for _ in range(4)]

    def _exchange(self, reverse):
        import torch

        tb, ta, fb, fa = self.buf
        self.L.lbm_slab_pack(self.h, reverse, tb, ta)
        self.L.lbm_sync(self.h)
        if self.host is None:
            exchange(tb, ta, fb, fa, self.rank, self.world)
        else:
            htb, hta, hfb, hfa = self.host
            htb.copy_(tb)
            hta.copy_(ta)
            exchange(htb, hta, hfb, hfa, self.rank, self.world)
            fb.copy_(hfb)
            fa.copy_(hfa)
        torch.cuda.synchronize()
        self.L.lbm_slab_unpack(self.h, reverse, fb, fa)

    def init_field(self, rho, ux, uy):
        """rho, ux, uy: whole-lattice (ny, nx) host arrays (each rank reads
        its own rows)."""
        r = slice(self.y0, self.y0 + self.rows)
        self.L.lbm_init_field(self.h, *(np.ascontiguousarray(a[r]) for a in (rho, ux, uy)))
        self._exchange(True)

    def step(self, n):
        for _ in range(int(n)):
            self.L.lbm_step(self.h, 1)
            self._exchange(False)

    def moments(self):
        """(rho, ux, uy) of this rank's rows."""
        return self.L.lbm_moments(self.h)

    def drift(self):
        return self.L.lbm_drift(self.h)

    def close(self):
        self.L.lbm_sync(self.h)
        self.L.lbm_destroy(self.h)
