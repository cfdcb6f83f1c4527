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


def test_each_result_is_the_same_alone_and_in_the_mix(oracle):
    from paper_2401_16732_gb300 import serve
    reqs = [serve.Request(rid=i, model="ab"[i % 2], B=1 + i % 3, arrival=0.001 * i, seed=4) for i in range(7)]
    keep = {(q.rid, li) for q in reqs for li in range(2)}
    mix = serve.Server(models(), keep_outputs=keep)
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
