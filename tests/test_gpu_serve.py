"""GPU parity of the serving loop through the C ABI: requests that arrive
while others run, admission by a device-memory budget, continuous batching.

A request served in a mix of others (its passes then share the batched
tensor-core launch with them, split over clusters differently) must give the
result it gives when served alone within 1e-6 relative, and the oracle's
within 1e-6.
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel
from oracle import cca as OC
from oracle import lda as OL
from synth import cca_latent_problem, lda_problem

pytestmark = pytest.mark.gpu

SCALE = [1.0, 0.8, 0.6, 0.45, 0.33, 0.25, 0.18, 0.13, 0.1, 0.07, 0.05, 0.035]
OPT = dict(max_iter=3000, gtol=0.0, rtol=1e-7, check_every=8, refine=2)


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2106_12060_gb300 as m
    torch.cuda.set_device(0)
    return m


def _cca_req(n, dx, dy, k, dt, seed):
    P = cca_latent_problem(n, dx, dy, latent=12, dtype=dt, seed=seed, latent_scale=SCALE, colscale=(1.0, 1e-2))
    return dict(kind="cca", P=P, n=n, dx=dx, dy=dy, k=k, dt=dt, lam=1e-3)


def _submit(gb, srv, r, host=False):
    import torch
    if r["kind"] == "cca":
        X, Y = to_dev(r["P"]["X"], r["dt"]), to_dev(r["P"]["Y"], r["dt"])
        if host:
            X, Y = X.cpu().pin_memory(), Y.cpu().pin_memory()
        return srv.submit_cca(X, Y, r["k"], r["lam"], r["lam"], gb.default_options(**OPT))
    X = to_dev(r["P"]["X"], "f32")
    y = torch.from_numpy(r["P"]["y"]).cuda()
    return srv.submit_lda(X, y, r["l"], r["k"], r["lam"], gb.default_options(**OPT))


def _drain(srv, ids):
    """Steps the server until every id has finished; returns the largest
    number of requests seen running at once and queued at once."""
    most_run = most_queue = 0
    for _ in range(100000):
        q, r = srv.step()
        most_run, most_queue = max(most_run, r), max(most_queue, q)
        if all(srv.state(i) >= 2 for i in ids):
            return most_run, most_queue
    raise AssertionError("server did not finish")


def _oracle(r):
    if r["kind"] == "cca":
        return OC.cca_qr(r["P"]["X64"], r["P"]["Y64"], r["lam"], r["lam"], r["k"])[0]
    return OL.lda_geneig(r["P"]["X64"], r["P"]["y"], r["l"], r["lam"], r["k"])[0]


def test_alone_vs_mix(gb):
    """The target request (BF16 CCA, n = 12000) served alone and then inside
    a stream of six others that arrive while it runs (BF16 and FP32 CCA, an
    FDA request, a request with 2k = 30, one passed from pinned host memory),
    under a budget that holds only some at a time."""
    import torch
    target = _cca_req(12000, 160, 96, 6, "bf16", seed=101)
    others = [_cca_req(9000, 200, 120, 5, "bf16", 102), _cca_req(6001, 96, 80, 4, "f32", 103),
              _cca_req(15000, 256, 128, 10, "bf16", 104), _cca_req(4000, 64, 48, 15, "bf16", 105),
              _cca_req(7000, 120, 64, 3, "bf16", 106)]
    PL = lda_problem(8000, 60, 6, dtype="f32", seed=107)
    others.append(dict(kind="lda", P=PL, n=8000, d=60, l=6, k=5, lam=1e-2))
    # alone
    srv = gb.Server()
    tid = _submit(gb, srv, target)
    _drain(srv, [tid])
    alone = np64(srv.result(tid)[0])
    srv.close()
    # in the mix: a budget of about three such requests' memory, arrivals
    # spread over the first steps
    srv0 = gb.Server()
    probe = _submit(gb, srv0, target)
    _drain(srv0, [probe])
    held = srv0.result(probe)[4]["device_bytes"]
    srv0.close()
    assert held > 0
    srv = gb.Server(gb.default_server_options(hbm_budget=3 * held, tick_iters=4))
    ids = [_submit(gb, srv, others[0]), _submit(gb, srv, others[1])]
    srv.step()
    ids.append(_submit(gb, srv, target))
    srv.step()
    for j, r in enumerate(others[2:]):
        ids.append(_submit(gb, srv, r, host=(j == 1)))
    most_run, most_queue = _drain(srv, ids)
    res = {i: srv.result(i) for i in ids}
    srv.close()
    mixed = np64(res[ids[2]][0])
    assert rel(mixed, alone) < 1e-6, (mixed, alone)
    ref = _oracle(target)
    assert rel(mixed, ref) < 1e-6 and rel(alone, ref) < 1e-6, (mixed, alone, ref)
    allreq = others[:2] + [target] + others[2:]
    for i, r in zip(ids, allreq):
        vals, U, V, info, times = res[i]
        assert info["status"] == gb.OK, (r["kind"], info)
        assert rel(np64(vals), _oracle(r)) < 1e-6, (r.get("dx"), np64(vals), _oracle(r))
        assert times["submit_s"] <= times["admit_s"] <= times["finish_s"], times
    assert most_run >= 2, most_run


def test_budget_admission_and_oversize(gb):
    """With a budget that holds one request at a time, requests run one after
    another (never two at once) and all finish; a request larger than the
    whole budget fails with GBCCA_ERR_OOM without stopping the others."""
    from synth.batch_mix import latent_views_device
    small = [_cca_req(3000, 48, 40, 3, "bf16", 200 + i) for i in range(3)]
    srv0 = gb.Server()
    probe = _submit(gb, srv0, small[0])
    _drain(srv0, [probe])
    held = srv0.result(probe)[4]["device_bytes"]
    srv0.close()
    srv = gb.Server(gb.default_server_options(hbm_budget=int(1.5 * held), tick_iters=8))
    ids = [_submit(gb, srv, r) for r in small]
    # 2e6 x 128 BF16 values: 512 MB of data alone, far above 1.5 x a small request
    Xb, Yb = latent_views_device(2_000_000, 64, 64, seed=210)
    assert Xb.numel() * 2 * 2 > 1.5 * held
    bid = srv.submit_cca(Xb, Yb, 2, 1e-3, 1e-3, gb.default_options(**OPT))
    most_run, most_queue = _drain(srv, ids + [bid])
    assert most_run == 1 and most_queue >= 2, (most_run, most_queue)
    for i, r in zip(ids, small):
        vals = np64(srv.result(i)[0])
        assert rel(vals, _oracle(r)) < 1e-6
    with pytest.raises(gb.GbccaError) as e:
        srv.result(bid)
    assert e.value.code == gb.ERR_OOM
    srv.close()
