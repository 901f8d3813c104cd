"""Test-only: oracle references of the full-size workloads, computed in
worker processes (spawn start method) so that several single-threaded oracle
runs proceed side by side on the host cores.  Each worker regenerates its
seeded graph itself (graphgen is deterministic), so no large array crosses a
process boundary; the oracle inside each worker stays plain and
single-threaded."""
import concurrent.futures as cf
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

C = 0.85
_cache = {}


def _rmat(scale, ef):
    key = ("rmat", scale, ef)
    if key not in _cache:
        import graphgen
        import oracle
        rp, col = graphgen.rmat(scale, ef, seed=1)
        _cache[key] = (rp, col, oracle.build_M(rp, col))
    return _cache[key]


def rwr_column(scale, ef, s, tol):
    """The oracle's RWR fixed point (Eq. 9, restart 1 - C) from node s."""
    import oracle
    rp, col, M = _rmat(scale, ef)
    r, _, _ = oracle.rwr(rp, col, int(s), C, tol=tol, M=M)
    return r


def batch_graph(g, n):
    """Graph g of the 512-graph batch (Chung-Lu, exponent 2.3, degree 12)."""
    import graphgen
    n = int(n)
    return graphgen.chung_lu(n, 12 * n, 2.3, max(2.0, n / 4), seed=1000 + g)


def batch_pagerank(g, n, tol):
    import oracle
    rp, col = batch_graph(g, n)
    p, _, _ = oracle.pagerank(rp, col, C, tol=tol)
    return p


def pool_map(fn, args, workers):
    """[fn(*a) for a in args] in `workers` spawned processes (in order)."""
    workers = max(1, min(workers, len(args), os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(workers, mp_context=ctx) as ex:
        futs = [ex.submit(fn, *a) for a in args]
        return [f.result() for f in futs]
