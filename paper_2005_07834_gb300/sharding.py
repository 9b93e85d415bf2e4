"""Partition of independent sites over ranks (one process per GPU).

Sites are independent once the orbitals are known (each processor group of
the paper works on its own site, Sec. VI.D), so a multi-GPU run shards the
sites with no collective on the data path: every rank loads the same
orbitals and builds chi0 and W of its own sites.  Sites go to ranks by
longest-processing-time first on the algorithmic cost of a site build,
8 N^2 K nf (chi0) + 14/3 N^3 (Dyson).
"""
import heapq


def site_cost(npts, K, nfreq):
    return 8.0 * npts * npts * K * nfreq + 14.0 / 3.0 * float(npts) ** 3


def lpt_partition(costs, nranks):
    """Lists of site indices per rank; each site goes to the least loaded rank, largest first."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    heap = [(0.0, r) for r in range(nranks)]
    parts = [[] for _ in range(nranks)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def shard_sites(sites, K, nfreq, rank, nranks):
    """Indices of the sites that `rank` builds."""
    costs = [site_cost(s.npts, K, nfreq) for s in sites]
    return lpt_partition(costs, nranks)[rank]
