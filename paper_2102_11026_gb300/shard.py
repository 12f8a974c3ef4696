"""Partition of independent systems across ranks (one process per GPU).

The strings of a substructured model are independent Newton systems (Sec. 6, the
puffer ball's 320 strings), so a multi-GPU run gives each rank a subset of them and
needs no collective on the data path.  The work of one Newton evaluation of a string
is proportional to its weight count P times the stacked forward column count
C_f = 4r + 4 (the perturbation columns of Sec. 4.2-4.3), so strings are assigned by
that cost with longest-processing-time-first list scheduling: the most expensive
string first, always to the least-loaded rank.  Every rank computes the same
partition from the same shapes, without communication.
"""


def string_cost(widths):
    """Cost estimate of one Newton evaluation of a decoder with layer widths
    ``widths`` (latent r = widths[0]): P * (4r + 4)."""
    P = sum(int(a) * int(b) for a, b in zip(widths[:-1], widths[1:]))
    return P * (4 * int(widths[0]) + 4)


def shard_by_cost(costs, world):
    """Split the indices 0..len(costs)-1 over ``world`` ranks.

    Longest processing time first: indices in order of decreasing cost (ties by index)
    go one by one to the rank with the least load so far (ties by rank).  Returns one
    ascending index list per rank; their union is every index exactly once, and the
    largest load is at most total/world + (1 - 1/world) * max(costs) (list scheduling)."""
    world = int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        w = min(range(world), key=lambda k: (load[k], k))
        parts[w].append(i)
        load[w] += costs[i]
    return [sorted(p) for p in parts]
