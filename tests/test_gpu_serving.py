"""Serving runtime on the GPU: results alone vs in a concurrent mix, admission, bounded waits."""
import numpy as np
import pytest

from synthetic import make_problem

pytestmark = pytest.mark.gpu


def _requests():
    """A mix of uneven dense (SRHT) and CSR (CountSketch) problems."""
    out = []
    for i, (name, kw) in enumerate([("c2_small", dict(n=3000, d=96, m=192)),
                                    ("c2_small", dict(n=2000, d=64, m=128, T=17)),
                                    ("c3_small", dict(n=4000, d=150, m=300, s=1)),
                                    ("c2_small", dict(n=5000, d=120, m=240, T=33)),
                                    ("c3_small", dict(n=3500, d=90, m=180, s=1, T=25)),
                                    ("c1_small", dict())]):
        out.append(make_problem(name, seed=i, **kw))
    return out


def _req(ihs, prob, compute):
    kw = dict(sketch=prob.sketch, m=prob.m, s=prob.s, seed=prob.sketch_seed, lambda_min=prob.lambda_min,
              lambda_max=prob.lambda_max, eps=1e-6, auto_rho=True, jmax=32, compute=compute)
    if prob.layout == "csr":
        return ihs.make_request(B=prob.B, lambdas=prob.lambdas, dtype=prob.storage,
                                csr=(prob.row_ptr, prob.col_idx, prob.val), shape=(prob.n, prob.d), **kw)
    return ihs.make_request(prob.A, prob.B, prob.lambdas, dtype=prob.storage, **kw)


def _alone(ihs, ctx, prob, compute):
    if prob.layout == "csr":
        p = ihs.Problem(ctx, B=prob.B, dtype=prob.storage, csr=(prob.row_ptr, prob.col_idx, prob.val),
                        shape=(prob.n, prob.d))
    else:
        p = ihs.Problem(ctx, prob.A, prob.B, dtype=prob.storage)
    p.sketch(prob.sketch, prob.m, prob.s, prob.sketch_seed)
    p.build_basis(prob.lambda_min, prob.lambda_max, k=None, k_default=0, eps=1e-6, auto_rho=True, jmax=32,
                  compute=compute)
    X = p.eval_path(prob.lambdas)
    p.close()
    return X


@pytest.mark.parametrize("compute", ["f64", "f32x2"])
def test_each_result_same_alone_and_in_the_mix(lib, compute):
    from paper_2210_12212_gb300 import ihsbin as ihs
    ctx = ihs.Context(0)
    probs = _requests()
    alone = [_alone(ihs, ctx, p, compute) for p in probs]
    srv = ihs.Server(ctx, slots=3)
    sub = []
    for p in probs:
        req, keep, out = _req(ihs, p, compute)
        sub.append((srv.submit(req, keep), out))
    for (t, out), ref in zip(sub, alone):
        st, times = srv.wait(t)
        assert st == ihs.OK
        err = np.max(np.linalg.norm((out - ref).reshape(len(out), -1), axis=1)
                     / np.linalg.norm(ref.reshape(len(ref), -1), axis=1))
        assert err <= (1e-12 if compute == "f64" else 1e-9), err
    srv.close()


def test_admission_under_a_small_budget(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    ctx = ihs.Context(0)
    probs = _requests()[:3]
    reqs = [_req(ihs, p, "f32x2") for p in probs]
    fp = [ihs.request_footprint(r[0]) for r in reqs]
    budget = max(fp) + min(fp) // 2          # at most one request in flight at a time
    srv = ihs.Server(ctx, slots=3, hbm_budget_bytes=budget)
    tickets = [srv.submit(r, k) for r, k, _ in reqs]
    times = []
    for t in tickets:
        st, t4 = srv.wait(t)
        assert st == ihs.OK
        times.append(t4)
    # with room for one request, the others waited in the queue
    assert sum(t4[0] > 0.0 for t4 in times) >= 1
    big, keep, _ = _req(ihs, make_problem("c2_small", seed=9, n=8000, d=256, m=512), "f32x2")
    with pytest.raises(ihs.IhsbinError) as ei:
        srv.submit(big, keep)
    assert ei.value.status == ihs.ERR_ADMISSION
    srv.close()


def test_wait_is_bounded(lib):
    from paper_2210_12212_gb300 import ihsbin as ihs
    ctx = ihs.Context(0)
    prob = make_problem("c2_small", seed=4, n=6000, d=200, m=400)
    srv = ihs.Server(ctx, slots=1)
    req, keep, out = _req(ihs, prob, "f64")
    t = srv.submit(req, keep)
    try:
        srv.wait(t, timeout_us=0)            # polled immediately: still running
        polled_done = True
    except ihs.IhsbinError as e:
        assert e.status == ihs.ERR_TIMEOUT
        polled_done = False
    if not polled_done:
        st, _ = srv.wait(t)
        assert st == ihs.OK
    srv.close()
