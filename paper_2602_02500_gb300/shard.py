"""One Muon step's matrix list shared out over the ranks of a job.

Every matrix is orthogonalized on its own (Algorithm 1 works per matrix), so
the list shards as independent units: each rank runs the library on its share
and the results are then exchanged, so that every rank ends with the whole
list's updates (a replicated optimizer).  The share is chosen by greedy
longest-processing-time on the nominal FLOPs of Algorithm 1, 4h^2 w +
2(L - 1)h^3 for an h x w matrix (h <= w): a list's matrices have a few
distinct shapes of different cost (on the synthetic 1B list a 2048 x 5632
matrix costs 1.23 times a 2048 x 2048 one), so equal counts per rank would
not balance.

The exchange is one all-gather over the process group (NCCL for CUDA
tensors, gloo on CPU): each rank packs its share's results into one flat
buffer, every rank receives every rank's buffer, and unpacks the matrices it
did not compute.  The layout of the buffers follows from the list's shapes
and the partition, which every rank knows, so nothing else crosses ranks.
Only host-side logic lives here: the compute is the caller's call into the
library.
"""


def ifnso_cost(rows, cols, L):
    """Nominal FLOPs of Algorithm 1 on an rows x cols matrix (oriented so that h <= w)."""
    h, w = min(rows, cols), max(rows, cols)
    return 4 * h * h * w + 2 * (L - 1) * h ** 3


def lpt_partition(costs, world):
    """Greedy LPT: matrices by decreasing cost, each to the rank with the least
    load so far (ties: the lower rank; equal costs keep list order).  Returns
    one ascending index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def owner_table(parts):
    """owner[i] = the rank whose share holds matrix i."""
    n = sum(len(p) for p in parts)
    owner = [-1] * n
    for r, p in enumerate(parts):
        for i in p:
            owner[i] = r
    if min(owner, default=0) < 0:
        raise ValueError("the shares do not cover the list")
    return owner


def pack_layout(parts, numels):
    """Flat exchange layout: rank r's buffer holds the matrices of parts[r]
    back to back in ascending index order, and every buffer is padded to the
    largest share's length.  Returns (that length in elements,
    {matrix: (rank, element offset)})."""
    offs = {}
    seg = 0
    for r, p in enumerate(parts):
        o = 0
        for i in p:
            offs[i] = (r, o)
            o += numels[i]
        seg = max(seg, o)
    if len(offs) != len(numels):
        raise ValueError("the shares do not cover the list")
    return seg, offs


def sharded_orthogonalize(run_local, outs, parts, rank, dist=None, group=None):
    """Run this rank's share, then exchange the results.

    run_local(indices) writes outs[i] for every i of this rank's share (one
    library call over those matrices).  Afterwards every rank holds all of
    outs (tensors of one dtype on one device): one all-gather of the ranks'
    packed results.  dist is torch.distributed (None or a world of one: no
    exchange)."""
    run_local(parts[rank])
    if dist is None or len(parts) == 1:
        return outs
    import torch

    world = len(parts)
    seg, offs = pack_layout(parts, [o.numel() for o in outs])
    ref = outs[0]
    send = torch.zeros(seg, dtype=ref.dtype, device=ref.device)
    for i in parts[rank]:
        _, o = offs[i]
        send[o:o + outs[i].numel()].copy_(outs[i].reshape(-1))
    recv = torch.empty(world * seg, dtype=ref.dtype, device=ref.device)
    dist.all_gather_into_tensor(recv, send, group=group)
    for i, (r, o) in offs.items():
        if r != rank:
            base = r * seg + o
            outs[i].copy_(recv[base:base + outs[i].numel()].view(outs[i].shape))
    return outs
