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

The exchange is one broadcast per matrix from the rank that owns it, on the
process group's device (NCCL for CUDA tensors, gloo on CPU); nothing else
crosses ranks.  Only host-side logic lives here: the compute is the caller's
call into the library.
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


def sharded_orthogonalize(run_local, outs, parts, rank, dist=None, group=None):
    """Run this rank's share, then exchange the results.

    run_local(indices) writes outs[i] for every i of this rank's share (one
    library call over those matrices).  Afterwards every rank holds all of
    outs: each matrix is broadcast from its owner.  dist is
    torch.distributed (None or a world of one: no exchange)."""
    run_local(parts[rank])
    if dist is None or len(parts) == 1:
        return outs
    owner = owner_table(parts)
    for i, r in enumerate(owner):
        dist.broadcast(outs[i], src=r, group=group)
    return outs
