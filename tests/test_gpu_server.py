"""The continuous-batching server: results against the oracle, bitwise equality of every
result alone and in a mix of concurrently running requests, device-memory admission and
the plan cache."""
import numpy as np
import pytest

import oracle as O
from paper_2605_20491_b300 import synth as S
from gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch  # noqa: F401
    from paper_2605_20491_b300 import tschrod
    return tschrod


def build(T, spec, prec):
    """Device buffers and submit arguments of one request descriptor."""
    import torch
    n, L = spec["n"], spec["L"]
    f = S.harmonic(n, L, spec["omega"])
    N = int(np.prod(n))
    kw = dict(n=n, L=L, f=f, sigma=spec["sigma"], tau=spec["tau"], prec=prec)
    if spec["kind"] == "exp":
        psi = S.complex_normal(spec["rhs_seed"], N)
        kw.update(kind=T.TS_REQ_EXP, inp=dev(psi), out=torch.zeros(2 * N, dtype=torch.float64, device="cuda"),
                  dtype=T.TS_C128)
        host_in = psi
    else:
        b = S.normal(spec["rhs_seed"], N)
        kw.update(inp=dev(b), out=torch.zeros(N, dtype=torch.float64, device="cuda"), dtype=T.TS_R64)
        host_in = b
        if spec["kind"] == "pcg":
            V2 = S.v2_cos_bumps(n, L, seed=1) + 5.0
            kw.update(kind=T.TS_REQ_PCG, V2=dev(V2), tol=1e-11, maxit=100)
            spec = dict(spec, V2=V2)
        else:
            kw.update(kind=T.TS_REQ_INVERSE)
    return kw, host_in, f


def oracle_answer(spec, host_in, f):
    Po = O.plan(spec["n"], spec["L"], f)
    if spec["kind"] == "exp":
        return O.apply_exp(Po, spec["tau"], host_in)
    if spec["kind"] == "inverse":
        return O.apply_inverse(Po, spec["sigma"], host_in)
    x, _, _ = O.pcg(Po, host_in, sigma=spec["sigma"], V2=spec["V2"], tol=1e-12)
    return x


def test_server_alone_equals_mix_and_oracle(T):
    specs = S.serving_requests(14, seed=4, sizes=(16, 24, 32, 48))
    precs = [T.TS_FP64 if i % 3 == 0 else T.TS_BF16X3 for i in range(len(specs))]
    server = T.Server(max_inflight=6)
    alone = []
    for spec, prec in zip(specs, precs):
        kw, host_in, f = build(T, spec, prec)
        st, lat, it = server.wait(server.submit(**kw))
        assert st == T.TS_OK, T.ts_last_error()
        alone.append(host(kw["out"]))
        if spec["kind"] == "pcg":
            spec["V2"] = S.v2_cos_bumps(spec["n"], spec["L"], seed=1) + 5.0
        want = oracle_answer(spec, host_in, f)
        tol = {"pcg": 1e-9}.get(spec["kind"], 1e-12 if prec == T.TS_FP64 else 5e-5)
        assert rel(alone[-1], want) < tol, (spec, prec, rel(alone[-1], want))
    # the same requests, all in flight together
    kws = [build(T, spec, prec)[0] for spec, prec in zip(specs, precs)]
    tickets = [server.submit(**kw) for kw in kws]
    for t in tickets:
        st, _, _ = server.wait(t)
        assert st == T.TS_OK
    for a, kw in zip(alone, kws):
        assert np.array_equal(a, host(kw["out"]))
    stats = server.stats()
    assert stats["completed"] == 2 * len(specs)
    assert stats["plan_hits"] >= len(specs)  # the mix reuses the plans of the first pass
    assert stats["batches"] >= 1 and stats["p99_ms"] >= stats["p50_ms"] > 0
    server.close()


def test_server_memory_admission(T):
    """A budget that holds one request at a time still completes every request, never holds
    more scratch than the budget, and refuses a request that can never fit."""
    specs = S.serving_requests(6, seed=7, sizes=(32,), mix=(0.0, 1.0, 0.0))
    budget = 3 << 20  # two 32^3 FP64 inverses (2 x 256 KiB + 1 MiB margin each) at a time
    server = T.Server(memory_budget_bytes=budget, max_inflight=6)
    kws = [build(T, s, T.TS_FP64)[0] for s in specs]
    tickets = [server.submit(**kw) for kw in kws]
    for t in tickets:
        assert server.wait(t)[0] == T.TS_OK
    assert server.stats()["peak_scratch_bytes"] <= budget
    big = S.serving_requests(1, seed=8, sizes=(128,), mix=(0.0, 1.0, 0.0))[0]
    kw = build(T, big, T.TS_FP64)[0]
    st, _, _ = server.wait(server.submit(**kw))
    assert st == T.TS_ERR_NO_MEMORY
    server.close()


def test_server_planner_threads_and_admission_order(T):
    """Results do not depend on how many planner threads build the plans, nor on the order
    in which built requests are admitted: one planner (requests admitted in submission
    order) and eight (plans finishing out of order, later requests admitted first) give
    the same bits as each request served alone."""
    specs = S.serving_requests(16, seed=11, sizes=(16, 32, 48), mix=(0.25, 0.5, 0.25))
    precs = [T.TS_FP64 if i % 4 == 0 else T.TS_BF16X3 for i in range(len(specs))]
    ref_server = T.Server(max_inflight=1, planner_threads=1)
    alone = []
    for spec, prec in zip(specs, precs):
        kw = build(T, spec, prec)[0]
        assert ref_server.wait(ref_server.submit(**kw))[0] == T.TS_OK
        alone.append(host(kw["out"]))
    ref_server.close()
    for threads in (1, 8):
        server = T.Server(max_inflight=8, planner_threads=threads)
        kws = [build(T, spec, prec)[0] for spec, prec in zip(specs, precs)]
        tickets = [server.submit(**kw) for kw in kws]
        for t in tickets:
            assert server.wait(t)[0] == T.TS_OK, T.ts_last_error()
        for a, kw in zip(alone, kws):
            assert np.array_equal(a, host(kw["out"]))
        assert server.stats()["completed"] == len(specs)
        server.close()
