"""The served results are the same alone and in the mix: requests of mixed
shapes and dtypes run concurrently on the server's streams give bitwise the
potentials of one-at-a-time solves (and match the oracle)."""
import numpy as np
import pytest

import oracle
from paper_1106_0557_gb300 import serving

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_alone_equals_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_0557_gb300 import Plan
    g = np.random.default_rng(0)
    reqs = [serving.Request(i, int(g.integers(12, 72)), "f32" if g.uniform() < 0.7 else "f64", i, 0.0)
            for i in range(48)]
    be = serving.TorchBackend(slots=6)
    be.prepare(reqs)
    srv = serving.Server(be, budget_bytes=8e9, slots=6, keep_outputs=True)
    srv.run(reqs)
    torch.cuda.synchronize()
    assert all(r.status == serving.OK for r in reqs)
    for r in reqs:
        src = be.source(r.n, r.dtype)
        with Plan((r.n,) * 3, (1.0 / r.n,) * 3, r.dtype) as p:
            alone = p.solve(src)
        torch.cuda.synchronize()
        assert torch.equal(alone, r.out), r.id
    for r in reqs[:4]:
        s64 = be.source(r.n, r.dtype).double().cpu().numpy()
        ref = oracle.solve(s64, (1.0 / r.n,) * 3)
        tol = 1e-5 if r.dtype == "f32" else 1e-12
        assert oracle.max_rel_error(r.out.double().cpu().numpy(), ref) <= tol
    srv.close()
