"""Serving loop: continuous batching gives each request the same ciphertexts
it gets alone, and those ciphertexts are the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
T = 65537

MODELS = None


def models():
    from paper_2401_16732_gb300.serve import ModelSpec
    return {
        "a": ModelSpec("a", 4096, 2, ((16, 16, 16, 16, 3, 1, 1), (16, 8, 16, 16, 1, 2, 0)), weight_seed=5),
        "b": ModelSpec("b", 2048, 3, ((3, 4, 20, 20, 7, 2, 3), (4, 6, 10, 10, 3, 1, 1)), weight_seed=6),
    }


@pytest.mark.parametrize("kernel", ["per_layer", "queue"])
def test_each_result_is_the_same_alone_and_in_the_mix(oracle, kernel):
    from paper_2401_16732_gb300 import flashgpu, serve
    kid = flashgpu.FL_STACK_QUEUE if kernel == "queue" else flashgpu.FL_STACK_PER_LAYER
    reqs = [serve.Request(rid=i, model="ab"[i % 2], B=1 + i % 3, arrival=0.001 * i, seed=4) for i in range(7)]
    keep = {(q.rid, li) for q in reqs for li in range(2)}
    mix = serve.Server(models(), keep_outputs=keep, stack_kernel=kid)
    finished, _ = mix.run(reqs, realtime=False)
    assert len(finished) == len(reqs) and mix.rounds >= 2
    for q in finished:
        alone_req = serve.Request(rid=q.rid, model=q.model, B=q.B, arrival=0.0, seed=4)
        alone = serve.Server(models(), keep_outputs={(q.rid, 0), (q.rid, 1)})
        alone.run([alone_req], realtime=False)
        for li in range(2):
            assert torch.equal(q.outputs[li], alone_req.outputs[li]), (q.rid, li)
    # oracle on a sampled subset: every layer of requests 0 and 1, both images of request 1
    for q in finished[:2]:
        r = mix.res[q.model]
        for li in range(2):
            ct, m = serve.layer_inputs(q, r, li, torch.device("cuda"))
            ct = ct.cpu().numpy().view(np.uint32)
            m = m.cpu().numpy().view(np.uint32)
            geo = oracle.geometry(r.spec.N, *r.spec.layers[li])
            got = q.outputs[li].cpu().numpy().view(np.uint32)
            for b in range(q.B):
                want = oracle.mask(oracle.conv_alg1(ct[b], r.w[li], geo, r.ctx.primes), m[b], r.ctx.primes)
                assert (got[b] == want).all(), (q.rid, li, b)


def test_admission_respects_the_memory_budget():
    from paper_2401_16732_gb300 import serve
    srv = serve.Server(models())
    need = max(srv.res["a"].peak_bytes(3), srv.res["b"].peak_bytes(3))
    srv.mem_budget = 2 * need  # at most two requests of this size at once
    reqs = [serve.Request(rid=i, model="ab"[i % 2], B=3, arrival=0.0, seed=4) for i in range(6)]
    finished, _ = srv.run(reqs, realtime=False)
    assert len(finished) == 6
    assert srv.peak_reserved <= srv.mem_budget
    assert 2 <= srv.peak_active < 6  # requests overlap, but the budget holds the rest back
    st = serve.latency_stats(finished)
    assert st["p50_ms"] <= st["p99_ms"]


def test_oversized_request_is_rejected_not_admitted():
    """A request whose peak live set exceeds the whole budget is refused at
    admission (host-side fault: an admission request larger than memory);
    the others are served."""
    from paper_2401_16732_gb300 import serve
    srv = serve.Server(models())
    srv.mem_budget = srv.res["a"].peak_bytes(2) + srv.res["b"].peak_bytes(2)
    big = serve.Request(rid=99, model="a", B=64, arrival=0.0, seed=4)
    reqs = [serve.Request(rid=i, model="ab"[i % 2], B=1, arrival=0.0, seed=4) for i in range(4)] + [big]
    finished, _ = srv.run(reqs, realtime=False)
    assert sorted(q.rid for q in finished) == [0, 1, 2, 3]
    assert srv.rejected == [big] and "above the budget" in big.error
    assert big.done is None and big.admitted is None


def test_cancel_mid_queue_releases_the_request():
    """Cancelling between rounds withdraws a pending and an active request
    (host-side fault: a client that goes away); the rest finish, with the
    same outputs as without the cancellation."""
    from paper_2401_16732_gb300 import serve
    reqs = [serve.Request(rid=i, model="a", B=1, arrival=0.0, seed=4) for i in range(5)]
    keep = {(q.rid, li) for q in reqs for li in range(2)}
    srv = serve.Server(models(), keep_outputs=keep)
    srv.mem_budget = 2 * srv.res["a"].peak_bytes(1)  # two at a time: the rest wait in the queue

    def on_round(server, finished):
        if server.rounds == 1:
            server.cancel(0)   # active, one layer done
            server.cancel(4)   # still pending
    finished, _ = srv.run(reqs, realtime=False, on_round=on_round)
    assert sorted(q.rid for q in finished) == [1, 2, 3]
    assert sorted(q.rid for q in srv.cancelled) == [0, 4]
    assert all(q.error == "cancelled" and q.done is None for q in srv.cancelled)
    ref = serve.Server(models(), keep_outputs={(2, 0), (2, 1)})
    alone = serve.Request(rid=2, model="a", B=1, arrival=0.0, seed=4)
    ref.run([alone], realtime=False)
    q2 = next(q for q in finished if q.rid == 2)
    assert torch.equal(q2.outputs[1], alone.outputs[1])


def test_device_wait_bound_reports_timeout():
    """Failure detection on the GPU without a fault: a wait on a barrier that
    nothing completes gives up after its bound, the call reports
    FL_ERR_TIMEOUT with the probe's bit, and the context keeps working."""
    from paper_2401_16732_gb300 import flashgpu, synth
    rc, word = flashgpu.selftest_wait_timeout()
    assert rc == flashgpu.FL_ERR_TIMEOUT and word == 4
    assert "gave up" in flashgpu.fl_last_error()
    c = flashgpu.Context(2048, 1)
    x = torch.from_numpy(synth.raw_ciphertexts(3, c.primes, (2, 1, 2048)).view(np.int32)).cuda()
    y = x.clone()
    c.ntt_forward(y)
    c.ntt_inverse(y)
    assert torch.equal(x, y)
