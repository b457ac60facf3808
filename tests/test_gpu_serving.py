"""The serving layer (continuous batching of decomposition requests): results match the
oracle's stopped driver (Sec. 4.1 termination by the change of the relative error), are the
same alone and in any mix of other requests and whatever the arrival times, equal the
batched driver at the same sweep count, and admission respects the HBM budget."""

import time

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_paper(core_dev):
    return np.ascontiguousarray(np.transpose(core_dev.cpu().numpy(), (1, 0, 2)))


def make_request(dims, ranks, seed, J, xdt, noise=1e-2):
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=seed, rel_noise=noise, dtype=xdt)
    init_np = [c.numpy() for c in inputs.random_cores(dims, ranks, seed + 1000)]
    init_dev = [torch.from_numpy(np.ascontiguousarray(c.transpose(1, 0, 2))).to(DEV)
                for c in init_np]
    return dict(X=X.to(DEV), Xh=X, ranks=ranks, J=J, seed=seed + 7, init_np=init_np,
                init_dev=init_dev)


def submit(srv, rq, **kw):
    cores = [c.clone() for c in rq["init_dev"]]
    t = srv.submit(rq["X"], rq["ranks"], rq["J"], rq["seed"], cores, init_given=True, **kw)
    return t, cores


def drain(srv, tickets, limit=100000):
    for _ in range(limit):
        if all(srv.poll(t)["done"] for t in tickets):
            return
        srv.tick()
    raise AssertionError("requests did not finish")


# Mixed-precision server used by the alone-vs-mix tests: the launch geometry is fixed by
# these limits, so every request sees the same kernels whatever else is in flight.
MIX_CFG = dict(max_slots=16, max_modes=5, max_dim=96, max_rank=6, max_samples=360,
               max_sweeps=8, fit_tol=1e-4, X_dtype=T.TR_F32, prec=T.TR_PREC_MIXED,
               hbm_budget_bytes=1 << 30, arena_bytes=256 << 20)

TARGET = ((14, 10, 12, 9), (3, 4, 2, 3), 120)
OTHERS = [((30, 25, 20), (3, 4, 2), 160), ((40, 6, 33), (4, 3, 5), 200),
          ((21, 17), (3, 5), 150), ((8, 9, 7, 6, 5), (2, 3, 2, 2, 3), 90),
          ((64, 48, 20), (6, 5, 6), 360), ((12, 11, 10), (3, 3, 3), 90),
          ((50, 3, 40), (5, 4, 2), 200), ((9, 8, 10, 11), (4, 2, 3, 2), 120)]


def test_served_fp64_matches_oracle_stopped_driver():
    """FP64 server against the oracle's Alg. 2 with the fit-change stop, on the same initial
    cores and Philox stream: same number of sweeps where the stop decision is not within
    rounding of the tolerance, per-sweep fits and final cores to 1e-8."""
    srv = T.Server(max_slots=8, max_modes=4, max_dim=64, max_rank=5, max_samples=400,
                   max_sweeps=12, fit_tol=1e-3, X_dtype=T.TR_F64, prec=T.TR_PREC_FP64,
                   hbm_budget_bytes=1 << 30, arena_bytes=256 << 20)
    shapes = [((20, 24, 28), (3, 2, 4), 160), ((12, 9, 10, 11), (2, 3, 2, 3), 150),
              ((40, 6, 33), (4, 3, 5), 250)]
    reqs = [make_request(d, r, 61 + i, J, torch.float64) for i, (d, r, J) in enumerate(shapes)]
    subs = [submit(srv, rq) for rq in reqs]
    drain(srv, [t for t, _ in subs])
    for rq, (t, cores) in zip(reqs, subs):
        res = srv.poll(t)
        ref, fits, conv = orc.tr_als_sampled_until(rq["Xh"].numpy(), rq["init_np"], rq["J"],
                                                   rq["seed"], fit_tol=1e-3, max_sweeps=12,
                                                   solver="normal")
        margins = [abs(abs(fits[s] - fits[s - 1]) - 1e-3) for s in range(1, len(fits))]
        if min(margins, default=1.0) > 1e-7:
            assert res["sweeps"] == len(fits)
            assert res["status"] == (T.TR_OK if conv else T.TR_ERR_NOT_CONVERGED)
        n = min(res["sweeps"], len(fits))
        np.testing.assert_allclose(res["fit_history"][:n], fits[:n], rtol=0, atol=1e-8)
        if res["sweeps"] == len(fits):
            for k in range(len(ref)):
                assert rel(to_paper(cores[k]), ref[k]) < 1e-8
    srv.close()


def test_served_result_is_the_same_alone_and_in_a_mix():
    """A request's cores, sweep count and fit history are bit-identical when it runs alone
    and when it is admitted in the middle of a stream of other requests of other shapes
    (mode counts 2-5, wide modes), arriving before, with and after it."""
    alone_srv = T.Server(**MIX_CFG)
    tgt = make_request(*TARGET[:2], 81, TARGET[2], torch.float32)
    t0, cores_alone = submit(alone_srv, tgt)
    drain(alone_srv, [t0])
    res_alone = alone_srv.poll(t0)
    alone_srv.close()
    assert res_alone["sweeps"] >= 2

    srv = T.Server(**MIX_CFG)
    others = [make_request(d, r, 90 + i, J, torch.float32) for i, (d, r, J) in enumerate(OTHERS)]
    tickets = [submit(srv, rq)[0] for rq in others[:4]]
    for _ in range(3):
        srv.tick()
    tgt2 = make_request(*TARGET[:2], 81, TARGET[2], torch.float32)
    t1, cores_mix = submit(srv, tgt2)
    tickets += [submit(srv, rq)[0] for rq in others[4:6]]
    for _ in range(5):
        srv.tick()
    tickets += [submit(srv, rq)[0] for rq in others[6:]]
    drain(srv, tickets + [t1])
    res_mix = srv.poll(t1)
    assert res_mix["sweeps"] == res_alone["sweeps"]
    assert res_mix["status"] == res_alone["status"]
    assert res_mix["fit_history"] == res_alone["fit_history"]
    for a, b in zip(cores_alone, cores_mix):
        assert torch.equal(a, b)
    assert srv.stats()["peak_active"] >= 5
    srv.close()


def test_served_result_is_the_same_under_the_worker_thread():
    """Requests submitted from a Python thread at random times to the native worker give
    the same results as under manual ticks."""
    rng = np.random.default_rng(5)
    srv = T.Server(**MIX_CFG)
    reqs = [make_request(d, r, 120 + i, J, torch.float32) for i, (d, r, J) in enumerate(OTHERS)]
    manual = [submit(srv, rq) for rq in reqs]
    drain(srv, [t for t, _ in manual])
    want = [(srv.poll(t), cores) for t, cores in manual]
    srv.close()

    srv = T.Server(**MIX_CFG)
    srv.start()
    subs = []
    for rq in reqs:
        subs.append(submit(srv, rq))
        time.sleep(float(rng.uniform(0, 0.01)))
    got = [(srv.wait(t, timeout_ms=120000), cores) for t, cores in subs]
    srv.stop()
    for (ra, ca), (rb, cb) in zip(want, got):
        assert ra["sweeps"] == rb["sweeps"] and ra["fit_history"] == rb["fit_history"]
        for a, b in zip(ca, cb):
            assert torch.equal(a, b)
        assert rb["t_submit_ns"] <= rb["t_admit_ns"] <= rb["t_done_ns"]
    srv.close()


def test_served_equals_batched_driver_at_the_same_sweep_count():
    """With the stop disabled (tolerance 0) a request runs its sweep cap and its cores equal
    those of the batched driver with that many sweeps."""
    ctx = T.Context(0)
    srv = T.Server(**{**MIX_CFG, "fit_tol": 0.0, "max_sweeps": 3})
    shapes = [TARGET, OTHERS[1], OTHERS[3]]
    reqs = [make_request(d, r, 140 + i, J, torch.float32) for i, (d, r, J) in enumerate(shapes)]
    subs = [submit(srv, rq) for rq in reqs]
    drain(srv, [t for t, _ in subs])
    for rq, (t, cores) in zip(reqs, subs):
        res = srv.poll(t)
        assert res["sweeps"] == 3 and res["status"] == T.TR_ERR_NOT_CONVERGED
        prob = dict(X=rq["X"], ranks=rq["ranks"], J=rq["J"], seed=rq["seed"],
                    cores=[c.clone() for c in rq["init_dev"]], init=True)
        T.tr_als_sampled_batched(ctx, [prob], 3, T.TR_PREC_MIXED)
        for a, b in zip(cores, prob["cores"]):
            assert torch.equal(a, b)
        # the served fit is the relative fit of the returned cores
        e = T.tr_rel_error(ctx, rq["X"], rq["ranks"], cores)
        assert abs((1.0 - e) - res["fit"]) < 1e-6
    srv.close()
    ctx.close()


def test_stop_rule_extremes():
    """Tolerance above any change: every request stops after exactly two sweeps (TR_OK);
    tolerance 0: every request runs its cap (TR_ERR_NOT_CONVERGED)."""
    for tol, cap, want_sweeps, want_status in ((1.0, 6, 2, T.TR_OK),
                                               (0.0, 3, 3, T.TR_ERR_NOT_CONVERGED)):
        srv = T.Server(**{**MIX_CFG, "fit_tol": tol, "max_sweeps": cap})
        reqs = [make_request(d, r, 160 + i, J, torch.float32)
                for i, (d, r, J) in enumerate(OTHERS[:4])]
        subs = [submit(srv, rq) for rq in reqs]
        drain(srv, [t for t, _ in subs])
        for t, _ in subs:
            res = srv.poll(t)
            assert res["sweeps"] == want_sweeps and res["status"] == want_status
            assert len(res["fit_history"]) == want_sweeps
        srv.close()


def test_admission_respects_the_hbm_budget():
    """With a budget that holds two requests at a time, at most two are ever admitted, the
    charged bytes never exceed the budget, and all requests finish; a request larger than
    the budget and one outside the server's limits are refused at submission."""
    reqs = [make_request((30, 25, 20), (3, 4, 2), 180 + i, 160, torch.float32)
            for i in range(6)]
    probe = T.Server(**MIX_CFG)
    t, _ = submit(probe, reqs[0])
    probe.tick()
    one = probe.stats()["charged_bytes"]
    probe.close()
    budget = 2 * one + one // 2
    srv = T.Server(**{**MIX_CFG, "hbm_budget_bytes": budget, "arena_bytes": budget})
    subs = [submit(srv, rq) for rq in reqs]
    drain(srv, [t for t, _ in subs])
    st = srv.stats()
    assert st["peak_active"] == 2
    assert st["peak_charged_bytes"] <= budget
    assert st["completed"] == 6 and st["charged_bytes"] == 0
    big = make_request((90, 80, 70), (6, 6, 6), 190, 360, torch.float32)
    with pytest.raises(T.TrError) as e:
        submit(srv, big)
    assert e.value.status == T.TR_ERR_BUDGET
    bad = make_request((10, 10, 10, 10, 10, 10), (2,) * 6, 191, 40, torch.float32)
    with pytest.raises(T.TrError) as e:
        submit(srv, bad)
    assert e.value.status == T.TR_ERR_INVALID_ARG
    srv.close()


def test_serving_stream_of_uneven_requests():
    """A small stream shaped like the serving workload (N in {3, 4, 5}, uneven sizes and
    ranks 4-16, J = 10 max L) runs to completion under the worker with every request
    stopped by the fit rule or its cap and a finite fit."""
    shapes = inputs.serving_requests(12, seed=3, emin=1e4, emax=3e5)
    srv = T.Server(max_slots=16, max_modes=5, max_dim=1024, max_rank=16, max_samples=2560,
                   max_sweeps=10, fit_tol=1e-4, hbm_budget_bytes=4 << 30,
                   arena_bytes=2 << 30)
    srv.start()
    subs = []
    for i, sh in enumerate(shapes):
        X, _ = inputs.tr_plus_noise(sh["dims"], sh["ranks"], seed=200 + i, rel_noise=1e-2,
                                    device=DEV)
        cores = T.empty_cores(sh["dims"], sh["ranks"])
        subs.append(srv.submit(X, sh["ranks"], sh["J"], 300 + i, cores))
    for t in subs:
        res = srv.wait(t, timeout_ms=300000)
        assert res["done"] and res["status"] in (T.TR_OK, T.TR_ERR_NOT_CONVERGED)
        assert np.isfinite(res["fit"]) and 2 <= res["sweeps"] <= 10
    srv.stop()
    srv.close()
