"""Host-side multi-rank logic: sample-range sharding and exact merging of sums.

MLMC samples are independent, so N ranks (one GPU each) simulate disjoint
sample ranges of the same work items and only their per-item sums are
combined.  Integer sums (approximate-only estimators) merge exactly; real sums
merge by FP64 addition in rank order.  The merge is a host operation after the
timed region (no collective on the data path).
"""


def shard_weak(items, rank):
    """Weak scaling: every rank simulates its own N samples of every item,
    rank r taking samples [first + r N, first + (r+1) N)."""
    out = []
    for it in items:
        d = dict(it)
        d["first_sample"] = int(it.get("first_sample", 0)) + rank * int(it["N"])
        out.append(d)
    return out


def shard_strong(items, rank, world):
    """Strong scaling: the N samples of every item are split into `world`
    contiguous, disjoint ranges (the first N mod world ranks take one more)."""
    out = []
    for it in items:
        N = int(it["N"])
        base, extra = divmod(N, world)
        n = base + (1 if rank < extra else 0)
        start = int(it.get("first_sample", 0)) + rank * base + min(rank, extra)
        d = dict(it)
        d["first_sample"] = start
        d["N"] = n
        out.append(d)
    return out


def merge_sums(per_rank):
    """Merge per-rank lists of sums dicts (same items, same order) into one list."""
    world = len(per_rank)
    n_items = len(per_rank[0])
    merged = []
    for i in range(n_items):
        parts = [per_rank[r][i] for r in range(world)]
        m = dict(parts[0])
        m["n"] = sum(int(p["n"]) for p in parts)
        m["saturations"] = sum(int(p["saturations"]) for p in parts)
        if all(p.get("exact_int") for p in parts):
            m["isum"] = sum(int(p["isum"]) for p in parts)
            m["isum2"] = sum(int(p["isum2"]) for p in parts)
        s, s2 = 0.0, 0.0
        for p in parts:
            s += p["sum"]
            s2 += p["sum2"]
        m["sum"], m["sum2"] = s, s2
        merged.append(m)
    return merged


def allgather_merge(local_sums, group=None):
    """Gather every rank's sums (torch.distributed, any backend) and merge them."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gathered = [None] * world
    dist.all_gather_object(gathered, local_sums, group=group)
    return merge_sums(gathered)
