"""Runtime features through the C ABI on the GPU: autotuner, graph-replayed
run to steady state, CUDA stream hand-off and the torch allocator hook."""
import numpy as np
import pytest

from paper_1711_03254_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_03254_gb300 import build
    build.build()
    from paper_1711_03254_gb300 import lbm as mod
    return mod


def _sim(lbm, n=24, precision="fp64", **kw):
    t, r1, r2, u = W.droplet(n, n, n, n / 4)
    t[:, 0, :] = W.SOLID
    r1[t == W.SOLID] = 0
    r2[t == W.SOLID] = 0
    s = lbm.Sim(n, n, n, [dict(tau=(0.8, 1.2), G=-1.8, rho_s=0.1, g=(1e-5, 0, 0))], precision=precision, **kw)
    s.set_geometry(t[None])
    s.set_fields(r1[None], r2[None], u[None])
    return s


def test_autotune_keeps_state_and_results(lbm, tmp_path):
    """Tuning leaves the state untouched: the next updates match a run that
    never tuned, and a second tune hits the cache file."""
    a = _sim(lbm)
    b = _sim(lbm, kernel="two_pass")
    a.step(3)
    b.step(3)
    cache = str(tmp_path / "tune.jsonl")
    k, t, z = lbm.lbm_autotune(a.ctx, 2, cache)
    assert k in (1, 2, 3, 4, 5, 6)
    a.step(10)
    b.step(10)
    for x, y in zip(a.get_fields(), b.get_fields()):
        assert np.allclose(x, y, rtol=0, atol=1e-13)
    c = _sim(lbm)
    assert lbm.lbm_autotune(c.ctx, 2, cache) == (k, t, z)
    assert len(open(cache).read().strip().splitlines()) == 1


@pytest.mark.parametrize("check_every", [50, 25])
def test_run_to_steady_matches_plain_steps(lbm, check_every):
    """The graph-replayed loop stops once the residual is below tol and leaves
    the same state as plain updates of the same count."""
    a = _sim(lbm, precision="fp32")
    done, res = lbm.lbm_run_to_steady(a.ctx, check_every, 1e-4, 4000, 1)
    assert done % check_every == 0 and 0 < done <= 4000
    assert res[0] <= 1e-4 or done == 4000
    b = _sim(lbm, precision="fp32")
    for _ in range(done // check_every):
        b.step(check_every)
        b.reduce()
    for x, y in zip(a.get_fields(), b.get_fields()):
        assert np.array_equal(x, y)


def test_stream_and_torch_allocator(lbm):
    import torch
    lbm.use_torch_allocator()
    try:
        s = torch.cuda.Stream()
        a = _sim(lbm, precision="fp32")
        lbm.lbm_set_stream(a.ctx, s.cuda_stream)
        a.step(20)
        ref = _sim(lbm, precision="fp32")
        ref.step(20)
        for x, y in zip(a.get_fields(), ref.get_fields()):
            assert np.array_equal(x, y)
        a.close()
        ref.close()
    finally:
        lbm.lbm_set_allocator()


def test_launch_counts(lbm):
    a = _sim(lbm, precision="fp32", kernel="fused")
    l0 = a.launches
    a.step(7)
    assert a.launches - l0 == 7
    b = _sim(lbm, precision="fp32", kernel="cluster")
    l0 = b.launches
    b.step(7)
    assert b.launches - l0 == 1


def test_per_kernel_timing(lbm):
    """Event timing brackets every launch of lbm_step: counts per part, times
    positive and no larger than the wall time of the steps, results unchanged."""
    import torch
    for kernel, parts in (("two_pass", {"psi": 6, "collide": 6}), ("fused", {"fused": 6}),
                          ("cluster", {"cluster": 1}), ("compact", {"psi": 6, "collide": 6})):
        a = _sim(lbm, precision="fp32", kernel=kernel)
        b = _sim(lbm, precision="fp32", kernel=kernel)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lbm.lbm_timing_begin(a.ctx, 64)
        e0.record()
        a.step(6)
        e1.record()
        t = lbm.lbm_timing_end(a.ctx)
        torch.cuda.synchronize()
        assert {k: v[1] for k, v in t.items()} == parts, kernel
        total = e0.elapsed_time(e1)
        assert all(v[0] > 0 for v in t.values())
        assert sum(v[0] for v in t.values()) <= total * 1.01 + 0.01
        b.step(6)
        np.testing.assert_array_equal(a.get_f(), b.get_f())
        a.close()
        b.close()


def test_timing_capacity_and_state_errors(lbm):
    a = _sim(lbm, precision="fp32", kernel="two_pass")
    lbm.lbm_timing_begin(a.ctx, 4)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_timing_begin(a.ctx, 4)
    assert e.value.status == 6
    a.step(5)  # 10 launches: only the first 4 are timed
    t = lbm.lbm_timing_end(a.ctx)
    assert t["psi"][1] == 2 and t["collide"][1] == 2
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_timing_end(a.ctx)
    assert e.value.status == 6
    a.close()


def test_allocator_hook_failure_is_oom(lbm):
    """An allocator hook that returns NULL makes lbm_create fail with
    LBM_ERR_OOM and leave nothing allocated; a hook that fails only on a later
    request (the scratch of lbm_set_geometry) gives LBM_ERR_OOM there, and the
    context stays usable once the hook allows allocations again."""
    import torch
    live = {}

    def alloc_ok(n, s):
        p = int(torch.cuda.caching_allocator_alloc(int(n), torch.cuda.current_device(), s))
        live[p] = n
        return p

    def release(p, s):
        live.pop(int(p), None)
        torch.cuda.caching_allocator_delete(int(p))

    try:
        lbm.lbm_set_allocator(lambda n, s: 0, release)
        with pytest.raises(lbm.LbmError) as e:
            lbm.Sim(8, 8, 8, [dict(tau=(1.0, 1.0), G=-2.0)], precision="fp32")
        assert e.value.status == 3

        budget = {"left": None}

        def alloc_limited(n, s):
            if budget["left"] is not None:
                if budget["left"] <= 0:
                    return 0
                budget["left"] -= 1
            return alloc_ok(n, s)

        lbm.lbm_set_allocator(alloc_limited, release)
        t, r1, r2, u = W.droplet(8, 8, 8, 2.0)
        s = lbm.Sim(8, 8, 8, [dict(tau=(1.0, 1.0), G=-2.0)], precision="fp32")
        budget["left"] = 0
        with pytest.raises(lbm.LbmError) as e:
            s.set_geometry(t[None])
        assert e.value.status == 3
        budget["left"] = None
        s.set_geometry(t[None])
        s.set_fields(r1[None], r2[None], u[None])
        s.step(3)
        assert np.isfinite(s.reduce()).all()
        s.close()
        assert not live
    finally:
        lbm.lbm_set_allocator()


def test_run_to_steady_reports_timeout(lbm):
    """A tolerance the run cannot reach within max_steps returns
    LBM_ERR_TIMEOUT from the C ABI with the update count and residual filled;
    the Python binding hands them back without raising."""
    import ctypes
    a = _sim(lbm, precision="fp32")
    done = ctypes.c_int(-1)
    res = np.full(1, -1.0)
    rc = lbm.library().lbm_run_to_steady(a.ctx, 10, 0.0, 30, ctypes.byref(done),
                                         res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == 5 and done.value == 30 and res[0] > 0
    done2, res2 = lbm.lbm_run_to_steady(a.ctx, 10, 0.0, 20, 1)
    assert done2 == 20 and res2[0] > 0
    a.close()
