"""Work-queue plan of a batch of independent problems (msdd_batch_plan,
host only): items ordered by decreasing Neumann-band cost n (b + 1), and the
makespan of greedy list scheduling in that order, checked against the
oracle's decomposition and an independent list-scheduling loop."""
import ctypes
import heapq

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import fem
from oracle.decomposition import Decomposition


@pytest.fixture(scope="module")
def msdd():
    import __graft_entry__ as ge
    ge.build()
    from paper_2106_06404_gb300 import msdd
    return msdd


def _expected(problems, nworkers):
    items = []
    for p, (n, parts, overlap, faces) in enumerate(problems):
        dec = Decomposition(fem.Mesh(n, faces), parts, overlap, 2, (1,) * len(n))
        for i, s in enumerate(dec.fine):
            w = [hi - lo + 1 for lo, hi in s.neumann_box]
            b = w[0] * w[1] + w[0] + 1 if len(n) == 3 else w[0] + 1
            items.append((float(np.prod(w)) * (b + 1), p, i))
    items.sort(key=lambda t: -t[0])          # stable: ties keep (problem, subdomain) order
    heap = [(0.0, w) for w in range(nworkers)]
    mk = 0.0
    for c, _, _ in items:
        load, w = heapq.heappop(heap)
        load += c
        mk = max(mk, load)
        heapq.heappush(heap, (load, w))
    total = sum(c for c, _, _ in items)
    return items, mk, max(total / nworkers, max(c for c, _, _ in items))


def test_plan_of_the_batch_recipe(msdd):
    batch = si.batch256(seed=0, count=64)
    problems = [(w.n, w.parts, w.overlap, w.dirichlet_faces) for w in batch]
    items, cost, mk, lb = msdd.batch_plan(problems, 304)
    want, mk_ref, lb_ref = _expected(problems, 304)
    assert items.shape == (sum(w.parts[0] * w.parts[1] for w in batch), 2)
    assert [tuple(r) for r in items] == [(p, i) for _, p, i in want]
    assert np.array_equal(cost, [c for c, _, _ in want])
    assert np.all(np.diff(cost) <= 0)
    assert mk == mk_ref and lb == lb_ref
    assert lb <= mk <= lb + cost.max()                     # list scheduling bound (Graham)


def test_plan_3d_and_small_worker_counts(msdd):
    problems = [((12, 10, 8), (3, 2, 2), 1, 0b1), ((20, 9), (3, 2), 2, 0b1010)]
    for nw in (1, 2, 5):
        items, cost, mk, lb = msdd.batch_plan(problems, nw)
        want, mk_ref, lb_ref = _expected(problems, nw)
        assert [tuple(r) for r in items] == [(p, i) for _, p, i in want]
        assert mk == mk_ref and lb == lb_ref
    assert msdd.batch_plan(problems, 1)[2] == pytest.approx(cost.sum())   # one worker: everything


def test_plan_rejects_invalid_arguments(msdd):
    lib = msdd.load()
    m = (msdd.Mesh * 1)(msdd.make_mesh((8, 8), 0))      # no Dirichlet face
    d = (msdd.Decomp * 1)(msdd._decomp((2, 2), 1))
    cnt = ctypes.c_longlong(-1)
    assert lib.msdd_batch_plan(1, m, d, 4, None, None, 0, ctypes.byref(cnt), None, None) == -1
    m = (msdd.Mesh * 1)(msdd.make_mesh((8, 8), 1))
    assert lib.msdd_batch_plan(1, m, d, 0, None, None, 0, ctypes.byref(cnt), None, None) == -1
    assert lib.msdd_batch_plan(1, m, d, 4, None, None, 0, ctypes.byref(cnt), None, None) == 0 and cnt.value == 4
    buf = (ctypes.c_int * 2)()
    assert lib.msdd_batch_plan(1, m, d, 4, buf, None, 1, ctypes.byref(cnt), None, None) == -1
    assert b"smaller" in lib.msdd_last_error()
