"""GPU tests of the serving engine (hx_server_*): continuous admission of
solve requests on several worker slots, device-memory admission, the
admission order (first come first served, or smallest first with a bound on
the wait), resident models across frequencies, cancellation, and results
independent of the mix.

Every wavefield is also checked against its own equation: the oracle's
assembled matrix (Eq. 3 rows, Eqs. 4-8, GA weights) applied on the CPU must
leave a relative residual below the solve tolerance (1e-10, mixed mode
refines in FP64).  "Same alone and in the mix" is checked to 1e-6 relative
L2, the accuracy bound the solver is held to; in practice the two agree to
the refinement tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operator as O
from oracle import solve as S
from oracle import weights as W
from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth


@pytest.fixture(scope="module")
def otable():
    return W.fit_table()


def _requests(n, seed):
    """Seeded small solve requests: grids 22..34 per side, 4..6-node PML,
    f for G between 6 and 10, 1..3 sources per request, models shared by id."""
    rng = np.random.default_rng(seed)
    models = {}
    reqs = []
    for k in range(n):
        mid = int(rng.integers(0, 3))
        if mid not in models:
            shape = tuple(int(s) for s in rng.integers(22, 35, 3))
            v = synth.random_velocity(shape, 500 + mid, 1500.0, 3000.0)
            models[mid] = v
        v = models[mid]
        nz, ny, nx = v.shape
        h = 25.0
        f = float(1500.0 / (h * rng.uniform(6.0, 10.0)))
        npml = int(rng.integers(4, 7))
        nrhs = int(rng.integers(1, 4))
        src = [(int(rng.integers(npml + 1, nx - npml - 1)), int(rng.integers(npml + 1, ny - npml - 1)),
                int(rng.integers(npml + 1, nz - npml - 1)), r, 1.0) for r in range(nrhs)]
        g = B.make_grid(v.shape, h, f, (npml,) * 6, float(v.max()))
        reqs.append(dict(model_id=mid, v=v, grid=g, src=src, nrhs=nrhs, f=f, h=h, npml=npml))
    return reqs


def _run(srv, reqs, concurrent):
    outs = [np.zeros((r["nrhs"],) + r["v"].shape, dtype=np.complex128) for r in reqs]
    res = [None] * len(reqs)
    if concurrent:
        tickets = [srv.submit(r["grid"], r["v"], r["src"], r["nrhs"], o, model_id=r["model_id"])
                   for r, o in zip(reqs, outs)]
        for i, t in enumerate(tickets):
            res[i] = srv.wait(t, timeout=120.0)
    else:
        for i, (r, o) in enumerate(zip(reqs, outs)):
            res[i] = srv.wait(srv.submit(r["grid"], r["v"], r["src"], r["nrhs"], o, model_id=r["model_id"]),
                              timeout=120.0)
    return outs, res


def _residual(otable, r, p):
    nodes, T = otable
    prof = O.profiles_for(r["v"].shape, r["h"], (r["npml"],) * 6, float(r["v"].max()), 1e-3)
    A = O.assemble_csr(r["v"], r["h"], r["f"], prof, T, nodes)
    s = S.point_sources(r["v"].shape, r["h"], [q[:3] for q in r["src"]])
    worst = 0.0
    for k in range(r["nrhs"]):
        rhs = s[k].reshape(-1)
        worst = max(worst, np.linalg.norm(rhs - A @ p[k].reshape(-1)) / np.linalg.norm(rhs))
    return worst


def test_results_are_the_same_alone_and_in_the_mix(otable):
    reqs = _requests(8, 11)
    alone_srv = B.Server(otable[1], slots=1)
    alone, res_a = _run(alone_srv, reqs, concurrent=False)
    alone_srv.close()
    srv = B.Server(otable[1], slots=3)
    fillers = _requests(6, 12)
    mix = reqs[:4] + fillers[:3] + reqs[4:] + fillers[3:]
    outs, res = _run(srv, mix, concurrent=True)
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res_a + res)
    assert st["completed"] == len(mix) and st["failed"] == 0
    assert st["max_concurrent"] >= 2                      # requests overlapped on the GPU
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    got = outs[:4] + outs[7:11]
    for a, b in zip(alone, got):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    for r, p in zip(reqs[:3], alone[:3]):
        assert _residual(otable, r, p) <= 1e-9


def test_memory_budget_serialises_admission(otable):
    reqs = _requests(4, 21)
    # room for one request (and its model) at a time
    est = max(r["grid"].nx * r["grid"].ny * r["grid"].nz * (r["nrhs"] * 116.0 + 5.0) for r in reqs)
    srv = B.Server(otable[1], slots=3, mem_budget=est + 64 * 2 ** 20 + 1.5 * est)
    outs, res = _run(srv, reqs, concurrent=True)
    st = srv.stats()
    assert all(r["status"] == 0 for r in res)
    assert st["max_concurrent"] == 1
    # a request larger than the whole budget is refused at submission
    big = reqs[0]
    with pytest.raises(B.HxError) as e:
        srv.submit(B.make_grid((200, 200, 200), 25.0, 5.0, (10,) * 6, 3000.0), np.zeros((200, 200, 200), np.float32),
                   big["src"], 1, np.zeros((1, 1, 1, 1), np.complex128))
    assert e.value.code == -2
    srv.close()


def test_resident_model_served_at_several_frequencies(otable):
    v = synth.random_velocity((26, 28, 30), 77, 1500.0, 3000.0)
    srv = B.Server(otable[1], slots=2)
    outs = []
    for f in (5.0, 6.0, 7.5):
        g = B.make_grid(v.shape, 25.0, f, (5,) * 6, float(v.max()))
        o = np.zeros((1,) + v.shape, np.complex128)
        r = srv.wait(srv.submit(g, v, [(15, 14, 13, 0, 1.0)], 1, o, model_id=9), timeout=120.0)
        assert r["status"] == 0
        outs.append((f, o))
    srv.close()
    for f, o in outs:
        rq = dict(v=v, h=25.0, f=f, npml=5, nrhs=1, src=[(15, 14, 13, 0, 1.0)])
        assert _residual(otable, rq, o) <= 1e-9


def test_bad_requests_are_refused(otable):
    srv = B.Server(otable[1], slots=1)
    v = np.full((10, 10, 10), 1500.0, np.float32)
    o = np.zeros((1, 10, 10, 10), np.complex128)
    g = B.make_grid(v.shape, 25.0, 5.0, (2,) * 6, 1500.0)
    with pytest.raises(B.HxError):
        srv.submit(g, v, [(20, 1, 1, 0, 1.0)], 1, o)          # source outside the grid
    with pytest.raises(B.HxError):
        srv.submit(g, v, [(5, 5, 5, 1, 1.0)], 1, o)           # rhs index out of range
    r = srv.wait(srv.submit(g, v, [(5, 5, 5, 0, 1.0)], 1, o), timeout=60.0)
    assert r["status"] == 0
    srv.close()


def test_cancel_queued_and_running_requests(otable):
    # hx_server_cancel: a queued request completes at once as cancelled; a
    # running one stops at its next convergence check (best iterate written);
    # the request served after them matches its solo result
    import time
    reqs = _requests(3, 31)
    outs = [np.zeros((r["nrhs"],) + r["v"].shape, dtype=np.complex128) for r in reqs]
    srv = B.Server(otable[1], slots=1)
    long_r = reqs[0]
    t_long = srv.submit(long_r["grid"], long_r["v"], long_r["src"], long_r["nrhs"], outs[0],
                        model_id=long_r["model_id"], tol=1e-30, max_outer=100000, time_limit_s=30.0)
    t_q = srv.submit(reqs[1]["grid"], reqs[1]["v"], reqs[1]["src"], reqs[1]["nrhs"], outs[1],
                     model_id=reqs[1]["model_id"])
    t_ok = srv.submit(reqs[2]["grid"], reqs[2]["v"], reqs[2]["src"], reqs[2]["nrhs"], outs[2],
                      model_id=reqs[2]["model_id"])
    t0 = time.time()
    while srv.stats()["max_concurrent"] < 1:        # wait until the long request has started
        assert time.time() - t0 < 60.0
        time.sleep(0.05)
    time.sleep(0.5)
    srv.cancel(t_q)
    srv.cancel(t_long)
    r_long = srv.wait(t_long, timeout=60.0)
    r_q = srv.wait(t_q, timeout=60.0)
    r_ok = srv.wait(t_ok, timeout=120.0)
    st = srv.stats()
    with pytest.raises(B.HxError) as e:             # already collected
        srv.cancel(t_ok)
    assert e.value.code == -1
    srv.close()
    assert r_long["status"] == -8 and r_long["worker"] == 0 and r_long["run_ms"] < 30000.0
    assert np.isfinite(outs[0]).all() and np.abs(outs[0]).max() > 0     # best iterate written
    assert r_q["status"] == -8 and r_q["worker"] == -1
    assert not outs[1].any()                                            # never ran
    assert r_ok["status"] == 0
    assert st["cancelled"] == 2 and st["failed"] == 2 and st["completed"] == 1
    solo_srv = B.Server(otable[1], slots=1)
    solo, res = _run(solo_srv, reqs[2:], concurrent=False)
    solo_srv.close()
    assert res[0]["status"] == 0
    assert np.linalg.norm(solo[0] - outs[2]) <= 1e-6 * np.linalg.norm(solo[0])


def _one(shape, nrhs, seed):
    v = synth.random_velocity(shape, seed, 1500.0, 3000.0)
    nz, ny, nx = shape
    h, npml = 25.0, 4
    f = 1500.0 / (h * 8.0)
    src = [(nx // 2, ny // 2, nz // 2 - r, r, 1.0) for r in range(nrhs)]
    g = B.make_grid(shape, h, f, (npml,) * 6, float(v.max()))
    return dict(model_id=seed, v=v, grid=g, src=src, nrhs=nrhs, f=f, h=h, npml=npml)


@pytest.mark.parametrize("order,max_wait,first", [("smallest", 0.0, "small"), ("fifo", 0.0, "big"),
                                                  ("smallest", 0.3, "big")])
def test_admission_order(otable, order, max_wait, first):
    # One slot, busy with a request that runs for 2 s; a large and then a small
    # request queue behind it.  Smallest-first admits the small one first;
    # first-come-first-served, or smallest-first once the large request has
    # waited past the bound, admits the large one first.  Both still solve.
    import time
    blocker, big, small = _one((30, 28, 26), 1, 61), _one((34, 34, 34), 3, 62), _one((22, 22, 22), 1, 63)
    srv = B.Server(otable[1], slots=1, order=order, max_wait_s=max_wait)
    outs = {k: np.zeros((r["nrhs"],) + r["v"].shape, dtype=np.complex128)
            for k, r in (("blocker", blocker), ("big", big), ("small", small))}
    t_b = srv.submit(blocker["grid"], blocker["v"], blocker["src"], 1, outs["blocker"], model_id=61,
                     tol=1e-30, max_outer=100000, time_limit_s=2.0)
    t0 = time.time()
    while srv.stats()["max_concurrent"] < 1:        # the blocker has started
        assert time.time() - t0 < 60.0
        time.sleep(0.02)
    sub, tick = {}, {}
    for k, r in (("big", big), ("small", small)):
        sub[k] = time.perf_counter()
        tick[k] = srv.submit(r["grid"], r["v"], r["src"], r["nrhs"], outs[k], model_id=r["model_id"])
        time.sleep(0.4)
    rb = srv.wait(t_b, timeout=60.0)
    res = {k: srv.wait(tick[k], timeout=120.0) for k in tick}
    srv.close()
    assert rb["status"] == -3                       # stopped by its time limit
    start = {k: sub[k] + res[k]["queue_ms"] / 1e3 for k in res}
    assert min(start, key=start.get) == first, (start, res)
    for k, r in (("big", big), ("small", small)):
        assert res[k]["status"] == 0
        assert _residual(otable, r, outs[k]) <= 1e-9


def test_server_config_errors(otable):
    with pytest.raises(B.HxError) as e:
        B.Server(otable[1], slots=1, order="largest")
    assert e.value.code == -1
    with pytest.raises(B.HxError) as e:
        B.Server(otable[1], slots=1, order="smallest", max_wait_s=-1.0)
    assert e.value.code == -1
