"""Serving form on the GPU: continuous batching gives every request exactly
the map it gets alone (and from rs_shoot_map), every served map agrees with
the FP64 oracle's map of the same request within the flip bar, admission
respects the device-memory budget, and failures are handled on the host."""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


def req_jobs(n=6, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        npix = int(rng.choice([32, 64, 128]))
        nl = int(rng.choice([1, 40, 300, 1500]))
        kstar = float(rng.uniform(0.2, 0.6))
        out.append(W.MapJob(name=f"r{k}", kappa_star=kstar, kappa_s=float(rng.uniform(0, 0.2)),
                            gamma=float(rng.uniform(0, 0.4)), n_lens=nl,
                            lens_radius=float(np.sqrt(nl / kstar)),
                            mass_model=int(rng.integers(0, 2)), seed=int(rng.integers(1, 2**40)),
                            n1=int(rng.integers(150, 600)), n2=int(rng.integers(150, 600)),
                            half1=float(rng.uniform(4, 8)), half2=float(rng.uniform(4, 8)),
                            width=float(rng.uniform(3, 7)), npix=npix))
    return out


def reference(rs, job, prec=1, shape=12):
    lens = rs.make_lenses(job)
    c, st = rs.shoot_map(job, lens, precision=prec, shape=shape)
    return c, st, rs.magnification(job, c)


# rays in another pixel than the oracle's, per precision form: the flip bar
# 1e-5 for double-single, the compensated form's documented 2e-4 (its FP32
# per-term rounding floor at fine pixels), one ray for the refined form (its
# rays near an edge are decided in FP64)
SERVE_FLIPS = {1: 2e-4, 2: 1e-5}


# whole served maps go to the oracle up to this many ray-lens interactions
# (about a second on the host); larger ones are bit-identical to
# rs_shoot_map's map, which the sampled full-size parity tests pin
ORACLE_MAX_WORK = 2e9


def check_oracle(rs, job, counts, stats, prec):
    """A served map against the oracle's map of the same request (its own lens
    draw): exact conservation on both sides, and the rays in another pixel
    within the bar of their precision form."""
    if job.n1 * job.n2 * max(1, rs.job_lens_count(job)) > ORACLE_MAX_WORK:
        return
    co, so = oracle.shoot(job, oracle.make_lenses(job))
    n = job.n1 * job.n2
    assert so["n_in"] + so["n_out"] + so["n_singular"] == n
    assert stats[0] + stats[1] + stats[2] == n
    diff = int(np.abs(counts.cpu().numpy().astype(np.int64) - co).sum())
    moved = (diff + 1) // 2                 # a ray between pixels counts twice
    bar = 1 if prec == 3 else max(2, int(SERVE_FLIPS[prec] * n))
    assert moved <= bar, (job.name, prec, moved, n)
    assert abs(int(stats[0]) - so["n_in"]) <= diff


def check_same(rs, srv, ticket, job, prec=1, shape=12):
    res = srv.wait(ticket, timeout_s=120)
    assert res.state == rs.REQ_DONE, (job.name, res.state, res.error)
    mu, counts = rs.Server.map_tensors(res, job.npix)
    c, st, m = reference(rs, job, prec, shape)
    assert torch.equal(counts, c), job.name
    assert list(res.stats) == st.cpu().tolist(), job.name
    assert torch.equal(mu, m), job.name
    assert res.t_submit <= res.t_admit <= res.t_done
    check_oracle(rs, job, counts, list(res.stats), prec)
    return res


@pytest.mark.parametrize("threaded", [False, True])
def test_each_request_alone_equals_in_the_mix(rs, threaded):
    jobs = req_jobs()
    # alone: one request per server, whole map in one slice
    alone = {}
    for j in jobs[:3]:
        srv = rs.Server(hbm_budget=1 << 30, slice_ms=0, threaded=threaded)
        t = srv.submit(j)
        res = srv.wait(t, 120)
        alone[j.name] = rs.Server.map_tensors(res, j.npix)[1].clone()
        srv.close()
    # in the mix: all requests, small slices so every map spans many launches
    srv = rs.Server(hbm_budget=1 << 30, slice_ms=0.001, threaded=threaded)
    tickets = [srv.submit(j) for j in jobs]
    for t, j in zip(tickets, jobs):
        res = check_same(rs, srv, t, j)
        if j.name in alone:
            assert torch.equal(rs.Server.map_tensors(res, j.npix)[1], alone[j.name])
    cnt = srv.counters()
    assert cnt["completed"] == len(jobs) and cnt["failed"] == 0
    assert cnt["slices"] > len(jobs)            # maps were split over slices
    srv.close()


def test_budget_limits_resident_requests(rs):
    jobs = [W.PARITY.with_(name=f"b{k}", n1=400, n2=400, npix=256, n_lens=50, seed=50 + k)
            for k in range(6)]
    per = 256 * 256 * 8 + 3 * 50 * 8 + 1024
    budget = 2 * per + 4096                     # room for two requests at a time
    srv = rs.Server(hbm_budget=budget, slice_ms=0.05, threaded=True, max_active=8)
    tickets = [srv.submit(j) for j in jobs]
    for t, j in zip(tickets, jobs):
        check_same(rs, srv, t, j)
        srv.release(t)                          # frees room for the queue
    cnt = srv.counters()
    assert cnt["peak_bytes"] <= budget and cnt["completed"] == 6
    srv.close()


def test_rejections_and_timeouts(rs):
    srv = rs.Server(hbm_budget=1 << 20, threaded=False, max_queue=2)
    big = W.PARITY.with_(npix=1024)             # 8 MB of maps > 1 MB budget
    with pytest.raises(rs.RSError) as e:
        srv.submit(big)
    assert e.value.code == -6
    small = W.PARITY.with_(n1=64, n2=64, npix=16)
    srv.submit(small)
    srv.submit(small)
    with pytest.raises(rs.RSError) as e:        # queue full
        srv.submit(small)
    assert e.value.code == -5
    srv.drain(60)
    srv.close()
    # a wait that cannot finish in time returns RS_ETIMEOUT, server still usable
    srv = rs.Server(hbm_budget=4 << 30, threaded=True, slice_ms=5)
    t = srv.submit(W.GERLUMPH)                  # about a second of GPU work
    with pytest.raises(rs.RSError) as e:
        srv.wait(t, timeout_s=0.01)
    assert e.value.code == -4
    res = srv.wait(t, timeout_s=120)
    assert res.state == rs.REQ_DONE
    srv.close()


def test_injected_allocation_failures(rs):
    jobs = req_jobs(n=3, seed=11)
    # nothing running when the allocation fails: the request fails cleanly
    srv = rs.Server(hbm_budget=1 << 30, threaded=False, inject_alloc_failures=1)
    t = srv.submit(jobs[0])
    res = srv.wait(t, 30)
    assert res.state == rs.REQ_FAILED and res.error == -2
    # the next one goes through
    t2 = srv.submit(jobs[1])
    check_same(rs, srv, t2, jobs[1])
    srv.close()
    # a failure while others run: the request waits and is retried
    srv = rs.Server(hbm_budget=1 << 30, threaded=False)
    big = W.GERLUMPH                            # about a second of GPU work
    ta = srv.submit(big)
    srv.step()                                  # admits it and starts its first slice
    srv.inject_alloc_failures(1)
    tb = srv.submit(jobs[2])                    # first admission attempt fails
    check_same(rs, srv, tb, jobs[2])
    check_same(rs, srv, ta, big)
    srv.close()


def test_cancel(rs):
    srv = rs.Server(hbm_budget=1 << 30, threaded=False, slice_ms=1)
    jobs = req_jobs(n=3, seed=21)
    tk = [srv.submit(j) for j in jobs]
    srv.cancel(tk[1])                           # still queued: never runs
    srv.drain(60)
    assert srv.poll(tk[1]).state == rs.REQ_CANCELLED
    for t, j in ((tk[0], jobs[0]), (tk[2], jobs[2])):
        check_same(rs, srv, t, j)
    # cancel a running request: its memory comes back
    t = srv.submit(W.GERLUMPH)
    srv.step()
    srv.cancel(t)
    srv.drain(60)
    assert srv.poll(t).state == rs.REQ_CANCELLED
    assert srv.counters()["cancelled"] == 2
    srv.close()


def test_poisson_stream_threaded(rs):
    """Requests arriving over time while others run are admitted and finish;
    latencies are measured from the GPU events."""
    jobs = req_jobs(n=12, seed=99)
    rng = np.random.default_rng(5)
    gaps = rng.exponential(0.01, size=len(jobs))
    srv = rs.Server(hbm_budget=1 << 30, slice_ms=2, threaded=True)
    tickets = []
    for j, g in zip(jobs, gaps):
        time.sleep(g)
        tickets.append(srv.submit(j))
    lat = []
    for t, j in zip(tickets, jobs):
        res = check_same(rs, srv, t, j)
        lat.append(res.t_done - res.t_submit)
    assert max(lat) < 60 and min(lat) > 0
    srv.close()


@pytest.mark.parametrize("shape", [12, 28], ids=["default", "shape28"])
def test_refined_requests_equal_single_maps(rs, shape):
    """The refined form served: every request's map is the single-map refined
    map of the same shape (rays near pixel edges listed across slices, the
    second pass run when the request's last tiles are done), alone and in
    the mix -- for the default shape and for a tuning candidate (4 lens
    groups per loop body)."""
    jobs = req_jobs(n=6, seed=7)
    srv = rs.Server(hbm_budget=1 << 30, slice_ms=0.001, precision=3, shape=shape)
    tickets = [srv.submit(j) for j in jobs]
    for t, j in zip(tickets, jobs):
        res = check_same(rs, srv, t, j, prec=3, shape=shape)
        assert res.stats[3] > 0 or j.n1 * j.n2 < 1000
    cnt = srv.counters()
    assert cnt["completed"] == len(jobs) and cnt["failed"] == 0
    assert cnt["slices"] > len(jobs)
    srv.close()


@pytest.mark.parametrize("prec", [2, 3], ids=["double-single", "refined"])
def test_mixed_masses_in_one_slice(rs, prec):
    """A unit-mass and a Salpeter request in one slice: where the unit-mass
    and the general kernel round differently (the double-single sum, the
    refined form's second pass) the server runs one launch per mass model,
    so both maps equal their single-map maps."""
    base = req_jobs(n=2, seed=7)
    jobs = [base[0].with_(mass_model=rs.MASS_UNIT), base[1].with_(mass_model=rs.MASS_SALPETER)]
    srv = rs.Server(hbm_budget=1 << 30, slice_ms=0, precision=prec, threaded=False)
    tickets = [srv.submit(j) for j in jobs]
    for t, j in zip(tickets, jobs):
        check_same(rs, srv, t, j, prec=prec)
    cnt = srv.counters()
    assert cnt["completed"] == 2 and cnt["slices"] == 1
    srv.close()


def test_double_single_requests_equal_single_maps(rs):
    """The double-single form served across many slices of mixed requests."""
    jobs = req_jobs(n=6, seed=9)
    srv = rs.Server(hbm_budget=1 << 30, slice_ms=0.001, precision=2)
    tickets = [srv.submit(j) for j in jobs]
    for t, j in zip(tickets, jobs):
        check_same(rs, srv, t, j, prec=2)
    cnt = srv.counters()
    assert cnt["completed"] == len(jobs) and cnt["failed"] == 0
    srv.close()
