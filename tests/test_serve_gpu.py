"""Continuous-batching serving loop: correctness alone vs in the mix, batching, admission."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
sp = pytest.importorskip("paper_2503_05408_gb300")

pytestmark = pytest.mark.gpu
F64_TOL = 1e-12
GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.lib()


@pytest.fixture(scope="module")
def factors():
    fs = [W.batch_factor(f) for f in range(9)]
    plans = [sp.Plan(A) for A in fs]
    pools = []
    for i, A in enumerate(fs):
        xs, b = W.manufactured_rhs(A, 16, seed=500 + i)
        pools.append((b, torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T))   # column-major (n, 16)
    return fs, plans, pools


def _submit(srv, fids, pools, f, r):
    b = pools[f][1][:, :r] if r > 1 else pools[f][1][:, 0].contiguous()
    x = torch.full_like(b, float("nan")) if r == 1 else torch.full((r, b.shape[0]), float("nan"),
                                                                       dtype=torch.float64, device="cuda").T
    return srv.submit(fids[f], b, x), x


@pytest.mark.parametrize("precision", ["f32_refine", "f64"])
def test_same_result_alone_and_in_the_mix(factors, precision):
    fs, plans, pools = factors
    srv = sp.Server(8 * GB, precision=precision)
    fids = [srv.register(p) for p in plans]
    f0, r0 = 2, 5
    rid, x_alone = _submit(srv, fids, pools, f0, r0)
    srv.wait(rid)
    rng = np.random.default_rng(3)
    jobs = []
    for k in range(60):                      # the same request buried among 60 others
        f = int(rng.integers(0, len(fs)))
        jobs.append(_submit(srv, fids, pools, f, int(rng.integers(1, 17))) + (f,))
        if k == 30:
            rid_mix, x_mix = _submit(srv, fids, pools, f0, r0)
    srv.drain()
    assert srv.wait(rid_mix)["status"] == 0
    assert torch.equal(x_alone, x_mix)       # computed by one block alone: bit-identical
    xo = oracle.solve(fs[f0], pools[f0][0][:, :r0])
    assert oracle.rel_error(x_mix.cpu().numpy(), xo) <= F64_TOL
    for rid, x, f in jobs:
        rep = srv.wait(rid)
        assert rep["status"] == 0
        r = x.shape[1] if x.dim() == 2 else 1
        assert oracle.rel_error(x.cpu().numpy().reshape(fs[f].n, -1),
                                oracle.solve(fs[f], pools[f][0][:, :r])) <= F64_TOL
    st = srv.stats()
    assert st["completed"] == 62 and st["launches"] < 62 and st["mean_batch"] > 1.0
    srv.close()


def test_admission_waits_for_memory_and_rejects_impossible(factors):
    fs, plans, pools = factors
    need = sum(p.stats()["device_bytes"] for p in plans)
    big = max(A.n for A in fs)
    # workspace for ~3 large requests only: the rest must wait for memory to free up
    srv = sp.Server(need + 3 * 2 * 4 * big * 16 + (1 << 20), precision="f32_refine")
    fids = [srv.register(p) for p in plans]
    jobs = [_submit(srv, fids, pools, f % len(fs), 16) + (f % len(fs),) for f in range(30)]
    srv.drain()
    for rid, x, f in jobs:
        assert srv.wait(rid)["status"] == 0
        assert oracle.rel_error(x.cpu().numpy(), oracle.solve(fs[f], pools[f][0])) <= F64_TOL
    assert srv.stats()["peak_workspace_bytes"] <= srv.stats()["arena_bytes"]
    srv.close()
    tiny = sp.Server(need + 4096, precision="f32_refine")
    fids = [tiny.register(p) for p in plans]
    with pytest.raises(sp.SptrsvError) as e:
        _submit(tiny, fids, pools, 0, 16)
    assert e.value.status == sp.ERR_BUDGET
    assert tiny.stats()["rejected"] == 1
    tiny.close()


def test_serial_f64_baseline_mode(factors):
    fs, plans, pools = factors
    srv = sp.Server(8 * GB, mode="serial", precision="f64")
    fids = [srv.register(p) for p in plans]
    jobs = [_submit(srv, fids, pools, f, 3) + (f,) for f in range(len(fs))]
    srv.drain()
    for rid, x, f in jobs:
        assert srv.wait(rid)["status"] == 0
        assert oracle.rel_error(x.cpu().numpy(), oracle.solve(fs[f], pools[f][0][:, :3])) <= F64_TOL
    st = srv.stats()
    assert st["completed"] == len(fs) and st["launches"] == 0
    srv.close()


def test_register_after_submit_and_unknown_ids(factors):
    fs, plans, pools = factors
    srv = sp.Server(8 * GB)
    fid = srv.register(plans[0])
    rid, x = _submit(srv, [fid], pools, 0, 1)
    srv.wait(rid)
    with pytest.raises(sp.SptrsvError):
        srv.register(plans[1])
    with pytest.raises(sp.SptrsvError):
        srv.poll(123456789)
    srv.close()


def _host_pair(b_np, r, pinned, ld_pad=0):
    """Column-major CPU tensors for b (first r columns) and x (NaN), optional padded ld."""
    n = b_np.shape[0]
    ld = n + ld_pad
    bb = torch.zeros((r, ld), dtype=torch.float64)
    bb[:, :n] = torch.from_numpy(np.ascontiguousarray(b_np[:, :r].T))
    xx = torch.full((r, ld), float("nan"), dtype=torch.float64)
    if pinned:
        bb, xx = bb.pin_memory(), xx.pin_memory()
    b, x = bb.T[:n], xx.T[:n]
    if r == 1 and ld_pad == 0:
        b, x = bb[0], xx[0]
    return b, x


@pytest.mark.parametrize("mode,precision", [("continuous", "f32_refine"), ("continuous", "f64"), ("serial", "f64")])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_requests_match_the_oracle(factors, mode, precision, pinned):
    # b and x in host memory: staged through the server's HBM budget, x copied back before
    # the request completes; mixed with device-buffer requests of the same factors
    fs, plans, pools = factors
    srv = sp.Server(8 * GB, mode=mode, precision=precision)
    fids = [srv.register(p) for p in plans]
    rng = np.random.default_rng(11)
    host_jobs, dev_jobs = [], []
    for k in range(40):
        f, r = int(rng.integers(0, len(fs))), int(rng.integers(1, 17))
        if k % 2 == 0:
            b, x = _host_pair(pools[f][0], r, pinned, ld_pad=3 if k % 4 == 0 else 0)
            host_jobs.append((srv.submit_host(fids[f], b, x), b, x, f, r))
        else:
            dev_jobs.append(_submit(srv, fids, pools, f, r) + (f,))
    srv.drain()
    for rid, b, x, f, r in host_jobs:
        rep = srv.wait(rid)
        assert rep["status"] == 0
        xo = oracle.solve(fs[f], pools[f][0][:, :r])
        assert oracle.rel_error(x.numpy().reshape(fs[f].n, -1) if x.dim() == 1 else x.numpy(), xo) <= F64_TOL
        assert np.array_equal(b.numpy().reshape(fs[f].n, -1), pools[f][0][:, :r])        # b untouched
    for rid, x, f in dev_jobs:
        assert srv.wait(rid)["status"] == 0
        r = x.shape[1] if x.dim() == 2 else 1
        assert oracle.rel_error(x.cpu().numpy().reshape(fs[f].n, -1),
                                oracle.solve(fs[f], pools[f][0][:, :r])) <= F64_TOL
    st = srv.stats()
    assert st["completed"] == 40 and st["peak_workspace_bytes"] <= st["arena_bytes"]
    srv.close()


def test_host_buffer_request_same_as_device_request(factors):
    # the host form runs the same kernel on the same values: identical bits
    fs, plans, pools = factors
    srv = sp.Server(8 * GB, precision="f32_refine")
    fids = [srv.register(p) for p in plans]
    rid, x_dev = _submit(srv, fids, pools, 4, 7)
    srv.wait(rid)
    b, x = _host_pair(pools[4][0], 7, True)
    srv.wait(srv.submit_host(fids[4], b, x))
    assert np.array_equal(x.numpy(), x_dev.cpu().numpy())
    with pytest.raises(TypeError):
        srv.submit_host(fids[4], pools[4][1][:, :2], pools[4][1][:, :2])     # device tensors: wrong form
    srv.close()


def test_host_buffer_budget_counts_the_staging(factors):
    fs, plans, pools = factors
    need = sum(p.stats()["device_bytes"] for p in plans)
    A = fs[0]
    # room for the device-buffer request's workspace, not for workspace + staging of b and x
    ws = 2 * ((A.n * 16 * 4 + 255) // 256 * 256) + (A.n * 16 * 4 + 64 + 255) // 256 * 256 + 256
    srv = sp.Server(need + ws + 1024, precision="f32_refine")
    fids = [srv.register(p) for p in plans]
    rid, x = _submit(srv, fids, pools, 0, 16)
    assert srv.wait(rid)["status"] == 0
    b, xh = _host_pair(pools[0][0], 16, False)
    with pytest.raises(sp.SptrsvError) as e:
        srv.submit_host(fids[0], b, xh)
    assert e.value.status == sp.ERR_BUDGET
    srv.close()
