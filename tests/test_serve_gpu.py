"""Serving loop (pdilqr_serve_*): continuous batching with warm starts kept on
the device, checked against the FP64 oracle and against itself.

The oracle side emulates the real-time iteration: tick 0 starts from
x_k = xhat_0, u_k = uref_k, lam = 0; every later tick starts from the
previous solution shifted by one step (x_k <- x_{k+1}, u_k <- u_{k+1},
lam_k <- lam_{k+1}, last entries repeated) and runs one SQP iteration.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_07823_b300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


def problem(client, N=30, nrob=1):
    return synth.srbd_problem(N, seed=1000 + client, nrob=nrob)


def tick_state(pr, t):
    """Measured state of tick t: the problem's xhat_0 drifting slowly."""
    g = np.random.default_rng(77 + t)
    return (pr["x0hat"] + 0.01 * t + g.normal(0, 0.002, pr["x0hat"].shape)).astype(np.float32)


def submit(srv, client, pr, t, nrob=1, reset=False):
    N = pr["N"]
    return srv.submit(client, nrob, N, tick_state(pr, t), pr["xref"], pr["uref"], pr["contact"],
                      reset=reset)


def oracle_ticks(prm, pr, ticks):
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    N = pr["N"]
    x = np.tile(r32(tick_state(pr, 0)), (N + 1, 1))
    u = r32(pr["uref"]).copy()
    lam = np.zeros_like(x)
    outs = []
    for t in range(ticks):
        if t > 0:
            idx = np.minimum(np.arange(N + 1) + 1, N)
            x, lam = x[idx], lam[idx]
            iu = np.minimum(np.arange(N + 1) + 1, N - 1)
            u = u[iu]
            u[N] = 0.0
        x, u, lam, info = oracle.srbd_sqp(prm, r32(tick_state(pr, t)), x, u, lam, r32(pr["xref"]),
                                          r32(pr["uref"]), pr["contact"], max_iters=1)
        outs.append((x.copy(), u.copy(), lam.copy(), info))
    return outs


def make_server(params=None, **kw):
    from paper_2506_07823_b300 import pdilqr
    args = dict(hbm_budget_bytes=64 << 20, max_batch=64, max_inflight=2, max_N=60, sqp_iters=1,
                warps=8)
    args.update(kw)
    return pdilqr.Server(params if params is not None else synth.srbd_params(), **args)


def test_rti_ticks_match_oracle():
    prm = synth.srbd_params()
    pr = problem(3)
    srv = make_server()
    ref = oracle_ticks(prm, pr, 3)
    for t in range(3):
        tk = submit(srv, 3, pr, t)
        res = srv.poll(tk, n=12, N=pr["N"])
        assert res["status"] == 0 and res["iters"] == 1
        x, u, _, info = ref[t]
        assert rel(res["x"], x) <= REL_TOL, (t, rel(res["x"], x))
        assert rel(res["u"][:-1], u[:-1]) <= REL_TOL, (t, rel(res["u"][:-1], u[:-1]))
        np.testing.assert_allclose(res["u0"], res["u"][0])
        assert res["latency_us"] > 0
    srv.close()


def run_client_alone(client, ticks):
    srv = make_server()
    pr = problem(client)
    outs = []
    for t in range(ticks):
        outs.append(srv.poll(submit(srv, client, pr, t), n=12, N=pr["N"]))
    srv.close()
    return outs


def test_alone_equals_in_the_mix():
    """A client's results do not depend on the requests batched with it."""
    alone = run_client_alone(5, 3)
    srv = make_server(max_batch=32)
    others = list(range(100, 163))
    probs = {c: problem(c, N=[20, 30, 45, 60][c % 4]) for c in others}
    probs[5] = problem(5)
    for t in range(3):
        tickets = {}
        for c in others[: 30 + 10 * t]:
            tickets[c] = submit(srv, c, probs[c], t)
        tickets[5] = submit(srv, 5, probs[5], t)
        for c in others[30 + 10 * t:]:
            tickets[c] = submit(srv, c, probs[c], t)
        got = {c: srv.poll(tk, n=12, N=probs[c]["N"]) for c, tk in tickets.items()}
        assert np.array_equal(got[5]["x"], alone[t]["x"])
        assert np.array_equal(got[5]["u"], alone[t]["u"])
        assert all(r["status"] == 0 or r["status"] == 8 for r in got.values())
    st = srv.stats()
    assert st["completed"] == st["submitted"] and st["mean_batch"] > 1.0
    srv.close()


def test_admission_refused_then_released():
    from paper_2506_07823_b300 import pdilqr
    srv = make_server(hbm_budget_bytes=64 << 10)
    pr = problem(0)
    admitted = []
    with pytest.raises(pdilqr.PdilqrError) as e:
        for c in range(64):
            srv.poll(submit(srv, c, pr, 0))
            admitted.append(c)
    assert e.value.code == pdilqr.E_ADMISSION
    assert 1 <= len(admitted) < 64
    srv.release(admitted[0])
    srv.poll(submit(srv, 999, pr, 0))       # fits again
    assert srv.stats()["refused"] == 1
    srv.close()


def test_admission_by_free_device_memory():
    """The first client of a size class is admitted only if the device's free
    memory holds the class's batch workspace plus the reserve: with a reserve
    larger than any device the client is refused before anything is
    allocated; with the default reserve the same client is admitted."""
    from paper_2506_07823_b300 import pdilqr
    prm = synth.srbd_params()
    srv = pdilqr.Server(prm, hbm_budget_bytes=64 << 20, max_N=50, hbm_reserve_bytes=1 << 60)
    pr = problem(3)
    with pytest.raises(pdilqr.PdilqrError) as e:
        submit(srv, 3, pr, 0)
    assert e.value.code == pdilqr.E_ADMISSION
    assert srv.stats()["refused"] == 1
    srv.close()
    srv = pdilqr.Server(prm, hbm_budget_bytes=64 << 20, max_N=50)   # default reserve
    srv.poll(submit(srv, 3, pr, 0))
    assert srv.stats()["refused"] == 0
    srv.close()


def test_snapshot_restore_resumes():
    pr = problem(9)
    srv = make_server()
    for t in range(2):
        srv.poll(submit(srv, 9, pr, t))
    x, u, lam = srv.snapshot(9, 12, pr["N"])
    cont = srv.poll(submit(srv, 9, pr, 2), n=12, N=pr["N"])
    srv.close()
    srv2 = make_server()
    srv2.poll(submit(srv2, 42, pr, 0))      # admits the client
    srv2.restore(42, x, u, lam)
    resumed = srv2.poll(submit(srv2, 42, pr, 2), n=12, N=pr["N"])
    assert np.array_equal(resumed["x"], cont["x"]) and np.array_equal(resumed["u"], cont["u"])
    srv2.close()


def test_poisoned_request_does_not_affect_others():
    alone = run_client_alone(5, 1)
    srv = make_server()
    bad = problem(77)
    x0 = tick_state(bad, 0)
    x0[4] = np.nan
    t_bad = srv.submit(77, 1, bad["N"], x0, bad["xref"], bad["uref"], bad["contact"])
    t_ok = submit(srv, 5, problem(5), 0)
    r_bad = srv.poll(t_bad)
    r_ok = srv.poll(t_ok, n=12, N=30)
    assert r_bad["status"] != 0
    assert np.array_equal(r_ok["x"], alone[0]["x"])
    srv.close()


def test_two_size_classes_and_timeouts():
    from paper_2506_07823_b300 import pdilqr
    prm2 = synth.srbd_params(2)
    srv = make_server(prm2)      # formation constants are server-wide
    pr1, pr2 = problem(1), problem(2, N=25, nrob=2)
    t1 = submit(srv, 1, pr1, 0)
    t2 = srv.submit(2, 2, 25, pr2["x0hat"].astype(np.float32), pr2["xref"], pr2["uref"], pr2["contact"])
    r2 = srv.poll(t2, n=24, N=25)
    r1 = srv.poll(t1)
    assert r1["status"] == 0 and r2["status"] in (0, 8)
    # the two-robot result matches the oracle's first SQP iteration
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    x, u, lam, info = oracle.srbd_sqp(prm2, r32(pr2["x0hat"]), np.tile(r32(pr2["x0hat"]), (26, 1)),
                                      r32(pr2["uref"]), np.zeros((26, 24)), r32(pr2["xref"]),
                                      r32(pr2["uref"]), pr2["contact"], max_iters=1)
    assert rel(r2["x"], x) <= REL_TOL
    with pytest.raises(pdilqr.PdilqrError) as e:
        srv.poll(123456)
    assert e.value.code == pdilqr.E_INVALID_ARG
    # a client that never polls does not block shutdown
    submit(srv, 1, pr1, 1)
    srv.close()


def test_large_classes_match_oracle():
    """Clients of four and sixteen robots (n = 48 and 192), each class with its
    own formation constants, next to single-robot clients."""
    cls = {r: synth.srbd_params(r) for r in (1, 4, 16)}
    srv = make_server(cls[1], class_params=cls, max_N=30)
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    cases = {40: (4, 12), 41: (16, 6), 42: (1, 30)}
    probs = {c: synth.srbd_problem(N, seed=2000 + c, nrob=r) for c, (r, N) in cases.items()}
    tickets = {c: srv.submit(c, r, N, probs[c]["x0hat"].astype(np.float32), probs[c]["xref"],
                             probs[c]["uref"], probs[c]["contact"]) for c, (r, N) in cases.items()}
    for c, (r, N) in cases.items():
        res = srv.poll(tickets[c], n=12 * r, N=N, timeout_us=60_000_000)
        assert res["status"] in (0, 8), (c, res["status"])
        pr = probs[c]
        x, u, lam, info = oracle.srbd_sqp(cls[r], r32(pr["x0hat"]),
                                          np.tile(r32(pr["x0hat"]), (N + 1, 1)), r32(pr["uref"]),
                                          np.zeros((N + 1, 12 * r)), r32(pr["xref"]), r32(pr["uref"]),
                                          pr["contact"], max_iters=1)
        assert rel(res["x"], x) <= REL_TOL, (c, rel(res["x"], x))
        assert rel(res["u"][:-1], u[:-1]) <= REL_TOL, (c, rel(res["u"][:-1], u[:-1]))
    from paper_2506_07823_b300 import pdilqr
    with pytest.raises(pdilqr.PdilqrError) as e:
        srv.submit(50, 3, 10, np.zeros(36, np.float32), np.zeros((11, 36), np.float32),
                   np.zeros((11, 36), np.float32), np.zeros((11, 12), np.uint8))
    assert e.value.code == pdilqr.E_INVALID_ARG
    srv.close()


def test_large_cta_budget_splits_batches():
    """With a budget of two large-class instances in flight, six four-robot
    requests that arrive together run as batches of at most two, each result
    still the oracle's; a negative budget is an invalid argument."""
    from paper_2506_07823_b300 import pdilqr
    prm4 = synth.srbd_params(4)
    srv = make_server(prm4, class_params={4: prm4}, max_N=12, max_inflight=4, large_cta_budget=2)
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    N = 8
    probs = {c: synth.srbd_problem(N, seed=3000 + c, nrob=4) for c in range(60, 66)}
    tickets = {c: srv.submit(c, 4, N, p["x0hat"].astype(np.float32), p["xref"], p["uref"],
                             p["contact"]) for c, p in probs.items()}
    for c, tk in tickets.items():
        res = srv.poll(tk, n=48, N=N, timeout_us=60_000_000)
        assert res["status"] in (0, 8), (c, res["status"])
        p = probs[c]
        x, u, lam, info = oracle.srbd_sqp(prm4, r32(p["x0hat"]), np.tile(r32(p["x0hat"]), (N + 1, 1)),
                                          r32(p["uref"]), np.zeros((N + 1, 48)), r32(p["xref"]),
                                          r32(p["uref"]), p["contact"], max_iters=1)
        assert rel(res["x"], x) <= REL_TOL, (c, rel(res["x"], x))
    st = srv.stats()
    assert st["completed"] == 6 and st["batches"] >= 3, st
    srv.close()
    with pytest.raises(pdilqr.PdilqrError) as e:
        make_server(large_cta_budget=-1)
    assert e.value.code == pdilqr.E_INVALID_ARG


def test_split_classes_match_oracle():
    """With split_min_robots=4 the four- and eight-robot classes run the split
    scan (16 CTAs per instance, one split batch in flight, at most two
    instances per split batch): five four-robot requests of ragged horizons
    and two eight-robot requests that arrive together, next to one-robot
    clients, each result the oracle's one real-time iteration; a robot count
    that is no size class is an invalid split_min_robots."""
    from paper_2506_07823_b300 import pdilqr
    cls = {r: synth.srbd_params(r) for r in (1, 4, 8)}
    srv = make_server(cls[1], class_params=cls, max_N=40, max_inflight=4, split_min_robots=4,
                      split_max_batch=2, hbm_budget_bytes=256 << 20)
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    cases = {70: (4, 13), 71: (4, 40), 72: (4, 22), 73: (4, 31), 74: (4, 17), 75: (8, 20),
             76: (8, 35), 77: (1, 30), 78: (1, 9)}
    probs = {c: synth.srbd_problem(N, seed=4000 + c, nrob=r) for c, (r, N) in cases.items()}
    tickets = {c: srv.submit(c, r, N, probs[c]["x0hat"].astype(np.float32), probs[c]["xref"],
                             probs[c]["uref"], probs[c]["contact"]) for c, (r, N) in cases.items()}
    for c, (r, N) in cases.items():
        res = srv.poll(tickets[c], n=12 * r, N=N, timeout_us=60_000_000)
        assert res["status"] in (0, 8), (c, res["status"])
        pr = probs[c]
        x, u, lam, info = oracle.srbd_sqp(cls[r], r32(pr["x0hat"]),
                                          np.tile(r32(pr["x0hat"]), (N + 1, 1)), r32(pr["uref"]),
                                          np.zeros((N + 1, 12 * r)), r32(pr["xref"]), r32(pr["uref"]),
                                          pr["contact"], max_iters=1)
        assert rel(res["x"], x) <= REL_TOL, (c, rel(res["x"], x))
        assert rel(res["u"][:-1], u[:-1]) <= REL_TOL, (c, rel(res["u"][:-1], u[:-1]))
    st = srv.stats()
    # five four-robot requests in batches of at most two, two eight-robot ones
    assert st["completed"] == len(cases) and st["batches"] >= 5, st
    srv.close()
    with pytest.raises(pdilqr.PdilqrError) as e:
        make_server(split_min_robots=3)
    assert e.value.code == pdilqr.E_INVALID_ARG
    # 16 CTAs per instance: a batch cap whose CTAs cannot all be resident
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with pytest.raises(pdilqr.PdilqrError) as e:
        make_server(split_min_robots=16, split_max_batch=sms // 16 + 1)
    assert e.value.code == pdilqr.E_INVALID_ARG
