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
