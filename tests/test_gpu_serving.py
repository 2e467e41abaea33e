"""Serving behaviour through the C ABI: results are the same alone and in a mix, problems
that do not fit the device-memory budget wait and run when earlier ones retire, and the
error paths return their codes."""
import time

import numpy as np
import pytest

from oracle import tilt_oracle as O
from paper_1205_5351_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1205_5351_gb300 import build, tilt
    build.build()
    return tilt


def _stream(count, first=0):
    times, patches = synth.served_stream(count, first=first)
    return [p for p in patches if max(p.m, p.n) <= 96]   # keep the test short


def test_result_is_the_same_alone_and_in_the_mix(T):
    patches = _stream(140)[:8]
    assert len(patches) == 8
    prm = T.default_params(max_outer=3)
    with T.Context(0) as ctx:
        alone = []
        for p in patches:
            t = ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, prm)
            alone.append(ctx.wait(t, 300000))
        # the same problems again, submitted one at a time while the others run, in
        # reverse order, interleaved with extra problems of other sizes
        extra = _stream(100, first=1000)[:8]
        tickets = []
        for p, q in zip(reversed(patches), extra):
            tickets.append(("mix", ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, prm)))
            tickets.append(("extra", ctx.submit(q.img, q.m, q.n, q.tau0, q.ttype, prm)))
        mixed = [ctx.wait(t, 300000) for kind, t in tickets if kind == "mix"][::-1]
    for a, b in zip(alone, mixed):
        # one CTA owns one problem and reduces in a fixed order: bit-identical
        np.testing.assert_array_equal(a["tau"], b["tau"])
        assert a["inner_iters"] == b["inner_iters"] and a["rank"] == b["rank"]


def test_admission_waits_for_memory_and_matches_oracle(T):
    patches = [p for p in synth.mixed_affine_batch(60, first=500) if max(p.m, p.n) <= 90][:5]
    assert len(patches) == 5
    prm = T.default_params(max_outer=2)
    # a budget that holds about two of these problems at a time
    one = max(p.m * p.n * 4 * 15 + p.img.nbytes for p in patches)
    with T.Context(0, hbm_budget_bytes=int(2.5 * one)) as ctx:
        tickets = [ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, prm) for p in patches]
        res = [ctx.wait(t, 300000) for t in tickets]
    for p, r in zip(patches, res):
        ref = O.tilt(p.img.astype(np.float64), p.tau0, p.ttype, p.m, p.n, O.Params(max_outer=2))
        assert O.tau_error(r["tau"], ref.tau) <= 1e-3


def test_error_codes(T):
    p = _stream(40)[0]
    with T.Context(0, hbm_budget_bytes=1 << 20) as ctx:
        with pytest.raises(T.TiltError) as e:
            ctx.submit(np.zeros((600, 600), np.float32), 500, 500, [1, 0, 300, 0, 1, 300], 6)
        assert e.value.code == T.TILT_E_NOMEM
        with pytest.raises(T.TiltError) as e:
            ctx.submit(p.img, 1, p.n, p.tau0, p.ttype)
        assert e.value.code == T.TILT_E_INVAL
        with pytest.raises(T.TiltError) as e:
            ctx.poll(987654)
        assert e.value.code == T.TILT_E_NOTFOUND
        bad = T.default_params(rho0=0.5)
        with pytest.raises(T.TiltError) as e:
            ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype, bad)
        assert e.value.code == T.TILT_E_INVAL


def test_destroy_cancels_running_and_queued_work(T):
    # 200 x 200 projective windows take seconds each; destroying the context right after
    # submitting a grouped launch and more work to the persistent workers must not wait for
    # them: running solves stop after their current inner iteration, queued ones unsolved
    patches = synth.projective_batch(24, first=900)
    ctx = T.Context(0)
    ctx.submit_batch([(p.img, p.m, p.n, p.tau0, p.ttype) for p in patches[:16]], None)
    for p in patches[16:]:
        ctx.submit(p.img, p.m, p.n, p.tau0, p.ttype)
    time.sleep(0.5)
    t0 = time.perf_counter()
    ctx.close()
    assert time.perf_counter() - t0 < 10.0
    # a new context on the same device works afterwards
    q = _stream(40)[0]
    with T.Context(0) as ctx2:
        r = ctx2.wait(ctx2.submit(q.img, q.m, q.n, q.tau0, q.ttype, T.default_params(max_outer=1)), 300000)
    assert r["status"] in (0, 1, 2)
