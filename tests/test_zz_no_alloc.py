"""ipf_solve_noalloc: the allocation-free solve, for callers that cannot
allocate device memory (a pooled allocator owns the device, a stream is being
captured, or a time-step loop must avoid the synchronisation an allocation
implies).  Its potentials must match the plan-based ipf_solve within the
tolerances of the parity tests, on consecutive calls that share the library's
static scratch array.  Kept in a file that is collected last."""
import numpy as np
import pytest

from paper_1106_0557_gb300 import native

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12}
TDT = {"f32": torch.float32, "f64": torch.float64}


def _src(N, seed, dtype):
    g = np.random.default_rng(seed)
    s = g.uniform(0.0, 1.0, (N[2], N[1], N[0]))
    s[g.uniform(size=s.shape) > 0.5] = 0.0
    return torch.from_numpy(s).to("cuda", TDT[dtype])


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_plan_solve_on_consecutive_calls(dtype, oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_0557_gb300 import Plan
    stream = torch.cuda.current_stream().cuda_stream
    # (16, 300, 16): 768-point y lines, which FP32 runs in the streamed y form
    # (tensor maps over the static array); the others take the tile form
    cases = [((40, 33, 24), (1.0, 1.0, 1.0), 1), ((32, 20, 17), (0.5, 0.25, 1.0), 2),
             ((40, 33, 24), (1.0, 1.0, 1.0), 3), ((16, 300, 16), (1.0, 0.5, 1.0), 4)]
    for N, h, seed in cases:
        src = _src(N, seed, dtype)
        got = torch.empty_like(src)
        native.ipf_solve_noalloc(N, h, dtype, src.data_ptr(), got.data_ptr(), stream)
        with Plan(N, h, dtype) as p:
            ref = p.solve(src)
        torch.cuda.synchronize()
        native.ipf_noalloc_check(stream)  # no bounded device wait gave up
        assert _rel(got, ref) <= TOL[dtype], (N, h, dtype)
        # and against the FP64 oracle on the same (dtype-rounded) source
        want = oracle_mod.solve(src.double().cpu().numpy(), h)
        err = oracle_mod.max_rel_error(got.double().cpu().numpy(), want)
        assert err <= TOL[dtype], (N, h, dtype, err)


def test_noalloc_rejects_oversize_and_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    src = torch.zeros(16, device="cuda")
    with pytest.raises(native.IsofftError) as ei:
        native.ipf_solve_noalloc((256, 256, 256), (1.0, 1.0, 1.0), "f32", src.data_ptr(), src.data_ptr())
    assert ei.value.status == native.IPF_BUDGET_EXCEEDED
    with pytest.raises(native.IsofftError) as ei:
        native.ipf_solve_noalloc((8, 8, 0), (1.0, 1.0, 1.0), "f64", src.data_ptr(), src.data_ptr())
    assert ei.value.status == native.IPF_INVALID_ARG
