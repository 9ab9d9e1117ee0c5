"""Serving on the GPU: the served results are the same alone and in the mix,
and match the oracle.

* Requests of mixed shapes and dtypes run concurrently on the server's
  streams give bitwise the potentials of one-at-a-time solves, with the
  FP64 class served in FP64 and as float pairs (df64), as the benchmark
  serves it.
* Plans created on four threads at once (shared and distinct spectra) solve
  bitwise like plans created one at a time.
* The whole 10 000-request serving mix (cubic N log-uniform in [32, 384],
  70 % FP32 / 30 % FP64 class as df64), served cold (plans and spectra built
  on the server's four background threads while it serves, two express
  slots on high-priority streams, as the benchmark serves it): every request with
  N <= 64 against the full-grid FP64 oracle, and a seeded 1 % sample of the
  rest at sampled cells against the direct sum.
"""
import numpy as np
import pytest

import oracle
from paper_1106_0557_gb300 import native, serving, sources

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12, "df64": 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _alone_equals_mix(reqs, slots, budget):
    from paper_1106_0557_gb300 import Plan
    be = serving.TorchBackend(slots=slots, express_slots=2)
    be.prepare(reqs)
    srv = serving.Server(be, budget_bytes=budget, slots=slots, keep_outputs=True, async_plans=True,
                         plan_workers=4, express_slots=2)
    srv.run(reqs)
    torch.cuda.synchronize()
    assert all(r.status == serving.OK for r in reqs)
    for r in reqs:
        src = be.source(r.n, r.dtype)
        with Plan((r.n,) * 3, (1.0 / r.n,) * 3, r.dtype) as p:
            alone = p.solve(src)
        torch.cuda.synchronize()
        assert torch.equal(alone, r.out), r.id
    srv.close()
    return be


@pytest.mark.parametrize("fp64_class", ["f64", "df64"])
def test_alone_equals_mix(fp64_class):
    g = np.random.default_rng(0)
    reqs = [serving.Request(i, int(g.integers(12, 72)), "f32" if g.uniform() < 0.7 else fp64_class, i, 0.0)
            for i in range(48)]
    be = _alone_equals_mix(reqs, slots=6, budget=8e9)
    for r in reqs[:4]:
        s64 = be.source(r.n, r.dtype).double().cpu().numpy()
        ref = oracle.solve(s64, (1.0 / r.n,) * 3)
        assert oracle.max_rel_error(r.out.double().cpu().numpy(), ref) <= TOL[r.dtype]


def _serving_mix(count, fp64_class="df64"):
    spec = sources.serving_requests(count=count, seed=0)
    return [serving.Request(r["id"], r["n"], fp64_class if r["dtype"] == "f64" else r["dtype"], r["seed"], 0.0)
            for r in spec]


def test_mix_subset_alone_equals_mix_df64():
    """The first 200 requests of the benchmark's serving mix, as served
    (FP64 class as df64): each bitwise equal to its solve alone."""
    _alone_equals_mix(_serving_mix(10000)[:200], slots=8, budget=120e9)


def test_served_mix_matches_oracle():
    reqs = _serving_mix(10000)
    g = np.random.default_rng(7)
    big = [r.id for r in reqs if r.n > 64]
    sample = set(int(i) for i in g.choice(big, size=len(reqs) // 100, replace=False))
    kept = {}      # request id -> potential on the host
    cells = {}     # request id -> sampled flat cell indices

    def on_finish(r):
        if r.n <= 64:
            kept[r.id] = r.out.double().cpu().numpy()
        elif r.id in sample:
            c = np.concatenate([g.integers(0, r.n ** 3, 6), [0, r.n ** 3 - 1]])
            cells[r.id] = c
            kept[r.id] = r.out.double().reshape(-1)[torch.from_numpy(c).to(r.out.device)].cpu().numpy()

    be = serving.TorchBackend(slots=8, express_slots=2)
    be.prepare(reqs)
    native.ipf_greens_cache_trim(0)
    srv = serving.Server(be, budget_bytes=120e9, slots=8, on_finish=on_finish, async_plans=True, plan_workers=4,
                         express_slots=2)
    srv.run(reqs)
    torch.cuda.synchronize()
    srv.close()
    assert all(r.status == serving.OK for r in reqs)
    n_small = sum(1 for r in reqs if r.n <= 64)
    assert len(kept) == n_small + len(sample) and n_small > 2000
    # every request with N <= 64: the full-grid oracle of its (N, dtype) source
    refs = {}
    for r in reqs:
        if r.n > 64:
            continue
        key = (r.n, r.dtype)
        if key not in refs:
            refs[key] = oracle.solve(be.source(r.n, r.dtype).double().cpu().numpy(), (1.0 / r.n,) * 3)
        assert oracle.max_rel_error(kept[r.id], refs[key]) <= TOL[r.dtype], (r.id, r.n, r.dtype)
    # the 1 % sample of the larger requests: direct sums at sampled cells
    for r in reqs:
        if r.id not in sample:
            continue
        s64 = be.source(r.n, r.dtype).double().cpu().numpy()
        ref = oracle.direct_points(s64, (1.0 / r.n,) * 3, cells[r.id])
        scale = np.abs(ref).max()
        assert np.abs(kept[r.id] - ref).max() / scale <= TOL[r.dtype], (r.id, r.n, r.dtype)


def test_plans_created_concurrently_solve_like_plans_created_alone():
    """Four threads create plans at once (several share a doubled mesh and
    so a cached spectrum, built by one of them while the others wait); each
    plan's solve is bitwise that of a plan created alone afterwards."""
    import concurrent.futures as cf
    from paper_1106_0557_gb300 import Plan
    shapes = [(40, "f32"), (48, "f32"), (40, "df64"), (70, "f32"), (100, "df64"), (36, "f32"), (64, "f64"),
              (90, "f32")]
    native.ipf_greens_cache_trim(0)
    be = serving.TorchBackend(slots=1)

    def make(shape):
        n, dtype = shape
        return be.create_plan(n, dtype)[0]

    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        plans = list(ex.map(make, shapes))
    torch.cuda.synchronize()
    for (n, dtype), p in zip(shapes, plans):
        src = be.source(n, dtype)
        out = torch.empty_like(src)
        native.ipf_solve(p, src.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        with Plan((n,) * 3, (1.0 / n,) * 3, dtype) as q:
            alone = q.solve(src)
        torch.cuda.synchronize()
        assert torch.equal(out, alone), (n, dtype)
        native.ipf_plan_destroy(p)
