"""The serving loop: continuous batching with admission by memory budget.
Every result must equal the oracle and the same request run alone, whatever
it was batched with."""
import numpy as np
import pytest
import torch

import paper_1412_8266_gb300 as srng
from oracle import oracle as O
from paper_1412_8266_gb300 import workload as W

pytestmark = pytest.mark.gpu
N_STREAMS = 1000


@pytest.fixture(scope="module")
def mrg_set():
    h = srng.srng_create_from_state([12345] * 6, N_STREAMS, srng.SRNG_SPACING_SUBSTREAM)
    yield h
    srng.srng_destroy(h)


def _read(srv, t, n, np_dtype):
    host = np.empty(n, dtype=np_dtype)
    srng.srng_server_read(srv, t, host, True)
    return host


def _oracle_f32(stream, pos, n):
    st = O.mrg_stream_starts([12345] * 6, 76, stream, 1)[0]
    if pos:
        st = O.mrg_jump(st, pos)
    v, _ = O.mrg_generate(st, n, O.OUT_F32)
    return v


def _alone(set_h, stream, pos, n, out_type, dtype):
    out = torch.empty(n, dtype=dtype, device="cuda")
    srng.srng_batch_run([set_h], [srng.Instance(set_index=0, stream=stream, offset=pos, length=n, out_offset=0)],
                        srng.SRNG_BATCH_WRITE, out_type, out)
    return out.cpu().numpy()


@pytest.mark.parametrize("extra", [{}, dict(chunk=96), dict(chunk=1024)])
def test_mixed_requests_equal_oracle_and_alone(mrg_set, extra):
    """Default per-step chunks and fixed ones give the same outputs."""
    rng = np.random.default_rng(2)
    srv = srng.srng_server_create(mrg_set, dict(budget_bytes=64 << 20, max_step_draws=1 << 18, max_inflight=4, **extra))
    try:
        reqs = []
        pos = {}
        for i in range(300):
            s = int(rng.integers(0, 40))  # few streams: many repeats on one stream
            n = int(np.exp(rng.uniform(0, np.log(400_000))))
            t = srng.srng_server_submit(srv, s, n, srng.SRNG_OUT_F32)
            reqs.append((t, s, pos.get(s, 0), n))
            pos[s] = pos.get(s, 0) + n
        for t, s, p, n in reqs:
            srng.srng_server_wait(srv, t, 60000)
        checked = 0
        for t, s, p, n in reqs:
            got = _read(srv, t, n, np.float32)
            alone = _alone(mrg_set, s, p, n, srng.SRNG_OUT_F32, torch.float32)
            assert np.array_equal(got.view(np.uint32), alone.view(np.uint32)), (t, s, p, n)
            if n <= 50_000 and checked < 60:
                assert np.array_equal(got.view(np.uint32), _oracle_f32(s, p, n).view(np.uint32)), (t, s, p, n)
                checked += 1
            srng.srng_server_release(srv, t)
        st = srng.srng_server_get_stats(srv)
        assert st.completed == 300 and st.steps > 1 and st.p99_us >= st.p50_us > 0
        assert st.peak_pool_bytes <= 64 << 20
        srng.srng_server_reset_stats(srv)  # counters restart; the pool holds nothing after the releases
        st = srng.srng_server_get_stats(srv)
        assert st.submitted == st.completed == st.steps == st.kernels == st.draws_completed == 0
        assert st.p50_us == st.p99_us == 0 and st.peak_pool_bytes == 0
    finally:
        srng.srng_server_destroy(srv)


def test_same_result_alone_and_in_the_mix(mrg_set):
    """A request run alone on a fresh server (explicit position) equals the
    same request run among many others."""
    rng = np.random.default_rng(7)
    srv = srng.srng_server_create(mrg_set, dict(budget_bytes=512 << 20))
    try:
        mix = []
        pos = {}
        for i in range(120):
            s = int(rng.integers(0, N_STREAMS))
            n = int(rng.integers(1, 3_000_000))
            t = srng.srng_server_submit(srv, s, n, srng.SRNG_OUT_F32)
            mix.append((t, s, pos.get(s, 0), n))
            pos[s] = pos.get(s, 0) + n
        outs = {}
        for t, s, p, n in mix:
            srng.srng_server_wait(srv, t, 60000)
            outs[t] = _read(srv, t, n, np.float32)
            srng.srng_server_release(srv, t)
    finally:
        srng.srng_server_destroy(srv)
    srv = srng.srng_server_create(mrg_set, dict(budget_bytes=64 << 20, max_inflight=1))
    try:
        for t, s, p, n in mix[::7]:
            t2 = srng.srng_server_submit_at(srv, s, p, n, srng.SRNG_OUT_F32)
            srng.srng_server_wait(srv, t2, 60000)
            alone = _read(srv, t2, n, np.float32)
            srng.srng_server_release(srv, t2)
            assert np.array_equal(alone.view(np.uint32), outs[t].view(np.uint32)), (s, p, n)
    finally:
        srng.srng_server_destroy(srv)


@pytest.mark.parametrize("out_type,np_dtype,tdtype", [(srng.SRNG_OUT_U32, np.uint32, torch.int32),
                                                      (srng.SRNG_OUT_F64, np.float64, torch.float64)])
def test_philox_server_and_types(out_type, np_dtype, tdtype):
    h = srng.srng_create(srng.SRNG_PHILOX4X32_10, 0xC0FFEE, 64)
    srv = srng.srng_server_create(h, dict(budget_bytes=32 << 20, max_step_draws=100_000))
    try:
        rng = np.random.default_rng(3)
        reqs = []
        pos = {}
        for i in range(50):
            s = int(rng.integers(0, 8))
            n = int(rng.integers(1, 300_000))
            reqs.append((srng.srng_server_submit(srv, s, n, out_type), s, pos.get(s, 0), n))
            pos[s] = pos.get(s, 0) + n
        for t, s, p, n in reqs:
            srng.srng_server_wait(srv, t, 60000)
            got = _read(srv, t, n, np_dtype)
            ref = O.philox_generate((0xC0FFEE, 0), s, p, n, out_type)
            assert np.array_equal(got.view(np.uint8), ref.view(np.uint8)), (s, p, n)
            srng.srng_server_release(srv, t)
    finally:
        srng.srng_server_destroy(srv)
        srng.srng_destroy(h)


def test_budget_admission_and_bounded_waits(mrg_set):
    """Host-side failure handling: a request larger than the whole budget is
    rejected; a request that cannot be admitted while memory is held times out
    on a bounded wait and completes once the memory is released."""
    srv = srng.srng_server_create(mrg_set, dict(budget_bytes=1 << 20))
    try:
        with pytest.raises(srng.SrngError) as e:
            srng.srng_server_submit(srv, 0, (1 << 18) + 1, srng.SRNG_OUT_F32)
        assert e.value.name == "SRNG_ERR_BUDGET"
        a = srng.srng_server_submit(srv, 0, 1 << 18, srng.SRNG_OUT_F32)  # the whole pool
        srng.srng_server_wait(srv, a, 60000)
        b = srng.srng_server_submit(srv, 1, 1000, srng.SRNG_OUT_F32)
        with pytest.raises(srng.SrngError) as e:
            srng.srng_server_wait(srv, b, 50)
        assert e.value.name == "SRNG_ERR_TIMEOUT"
        done, _ = srng.srng_server_poll(srv, b)
        assert not done
        with pytest.raises(srng.SrngError) as e:
            srng.srng_server_release(srv, b)
        assert e.value.name == "SRNG_ERR_ARG"
        srng.srng_server_release(srv, a)
        srng.srng_server_wait(srv, b, 60000)
        got = _read(srv, b, 1000, np.float32)
        assert np.array_equal(got.view(np.uint32), _oracle_f32(1, 0, 1000).view(np.uint32))
        srng.srng_server_release(srv, b)
        with pytest.raises(srng.SrngError) as e:
            srng.srng_server_release(srv, b)
        assert e.value.name == "SRNG_ERR_CLOSED"
        st = srng.srng_server_get_stats(srv)
        assert st.rejected == 1 and st.completed == 2
    finally:
        srng.srng_server_destroy(srv)


def test_replay_of_the_serving_trace():
    """A short slice (20 ms of arrivals) of the serving workload replayed by the
    native client: every request completes and latencies are reported."""
    trace = W.serving_trace(0.02)
    h = srng.srng_create_from_state([12345] * 6, W.SERVING["n_streams"], srng.SRNG_SPACING_SUBSTREAM)
    srv = srng.srng_server_create(h, dict(budget_bytes=W.SERVING["budget"]))
    try:
        st = srng.srng_server_replay(srv, [(r.arrival_s, r.stream, r.n) for r in trace], srng.SRNG_OUT_F32, 1.0)
        assert st.completed == len(trace) and st.submitted == len(trace)
        assert st.draws_completed == sum(r.n for r in trace)
        assert st.p99_us >= st.p50_us > 0
    finally:
        srng.srng_server_destroy(srv)
        srng.srng_destroy(h)


def _oracle_points(s, p, n, offsets):
    """Draws p + k (k in offsets) of substream s as FP32, each reached by the
    oracle's own jump-ahead from the substream's start (point evaluation)."""
    st0 = O.mrg_stream_starts([12345] * 6, 76, s, 1)[0]
    out = np.empty(len(offsets), dtype=np.float32)
    for i, k in enumerate(offsets):
        v, _ = O.mrg_generate(O.mrg_jump(st0, p + int(k)), 1, O.OUT_F32)
        out[i] = v[0]
    return out


def _oracle_full(s, p, n, threads=0):
    """The whole request from the oracle: the range is cut into pieces whose
    start states the oracle reaches by jump-ahead, then stepped (on all host
    threads)."""
    st0 = O.mrg_stream_starts([12345] * 6, 76, s, 1)[0]
    piece = 1 << 20
    k = (n + piece - 1) // piece
    starts = np.stack([O.mrg_jump(st0, p + j * piece) for j in range(k)])
    vals, _ = O.mrg_bulk(starts, piece, O.OUT_F32, threads)
    return vals.ravel()[:n]


def test_serving_workload_slice_equals_oracle():
    """A seeded slice of the serving workload at its own sizes: Poisson
    arrivals of FP32 requests with n log-uniform in [1e3, 1e8] over the 10^6
    MRG32k3a substreams of the all-12345 state, a 16 GB budget, submitted in
    arrival order with up to 48 requests outstanding (continuous batching:
    requests join steps while others run).  Requests of at most 10^6 draws are
    compared with the oracle in full; larger ones at 256 seeded positions plus
    their first and last 4096 draws by oracle jump-ahead, and three of them
    (seeded) in full.  Zero tolerance: FP32 values are exact functions of
    integers."""
    trace = W.serving_trace(0.02)  # 20 ms of arrivals at 20,000 requests/s
    h = srng.srng_create_from_state([12345] * 6, W.SERVING["n_streams"], srng.SRNG_SPACING_SUBSTREAM)
    srv = srng.srng_server_create(h, dict(budget_bytes=W.SERVING["budget"]))
    rng = np.random.default_rng(14128266)
    large = [i for i, r in enumerate(trace) if r.n > 1_000_000]
    full_large = set(rng.choice(large, min(3, len(large)), replace=False).tolist()) if large else set()
    pos = {}
    pending = []
    counts = dict(requests=0, full=0, sampled=0, draws=0, draws_checked=0)

    def check(t, i, s, p, n):
        srng.srng_server_wait(srv, t, 120000)
        got = _read(srv, t, n, np.float32)
        srng.srng_server_release(srv, t)
        if n <= 1_000_000 or i in full_large:
            ref = _oracle_full(s, p, n) if n > 1_000_000 else _oracle_f32(s, p, n)
            assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (i, s, p, n)
            counts["full"] += 1
            counts["draws_checked"] += n
        else:
            ks = np.unique(np.concatenate([rng.integers(0, n, 256), [0, n - 1]]))
            assert np.array_equal(got[ks].view(np.uint32), _oracle_points(s, p, n, ks).view(np.uint32)), (i, s, p, n)
            head = _oracle_f32(s, p, 4096)
            tail = _oracle_f32(s, p + n - 4096, 4096)
            assert np.array_equal(got[:4096].view(np.uint32), head.view(np.uint32)), (i, s, p, n)
            assert np.array_equal(got[-4096:].view(np.uint32), tail.view(np.uint32)), (i, s, p, n)
            counts["sampled"] += 1
            counts["draws_checked"] += len(ks) + 8192
        counts["requests"] += 1
        counts["draws"] += n

    try:
        for i, r in enumerate(trace):
            t = srng.srng_server_submit(srv, r.stream, r.n, srng.SRNG_OUT_F32)
            p = pos.get(r.stream, 0)
            pos[r.stream] = p + r.n
            pending.append((t, i, r.stream, p, r.n))
            if len(pending) > 48:
                check(*pending.pop(0))
        while pending:
            check(*pending.pop(0))
        st = srng.srng_server_get_stats(srv)
        assert st.completed == len(trace) and st.peak_pool_bytes <= W.SERVING["budget"]
    finally:
        srng.srng_server_destroy(srv)
        srng.srng_destroy(h)
    assert counts["requests"] == len(trace) and counts["full"] > 100 and counts["sampled"] > 50
    print(f"serving slice: {counts['requests']} requests, {counts['draws']} draws; {counts['full']} compared in "
          f"full, {counts['sampled']} at sampled points; {counts['draws_checked']} draws checked against the oracle")
