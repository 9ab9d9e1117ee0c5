"""The library's test hooks, on the GPU.  None of them faults, traps or hangs
a device; each makes a failure or a hazard visible on the host.

* IPF_FLAG_TEST_CANARY fills the whole workspace with NaN bytes before every
  solve.  The potential must stay finite and bitwise equal to that of a plan
  without the hook: no pass reads a workspace element that no earlier pass
  of the same solve wrote (the z padding, the rows y >= Ny of the forward y
  pass, the columns past Kx are all supplied as zeros, never read).  Two
  solves of a plan are bitwise equal as well (determinism).
* ISOFFT_TEST_FAIL_ALLOC makes one buffer's device allocation fail as if the
  device were out of memory: the call returns IPF_OUT_OF_MEMORY, frees what
  it had allocated, leaves no spectrum in the cache, and the next plan works.
* ISOFFT_NVTX=1 wraps each pass's launches in an NVTX range; the potential
  is unchanged.
"""
import numpy as np
import pytest

import oracle
from paper_1106_0557_gb300 import native

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64, "df64": np.float64}
TOL = {"f32": 1e-5, "f64": 1e-12, "df64": 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    native.lib()


def rand_src(N, seed):
    g = np.random.default_rng(seed)
    s = g.uniform(0.0, 1.0, (N[2], N[1], N[0]))
    s[g.uniform(size=s.shape) > 0.6] = 0.0
    return s


def device_solves(N, h, dtype, flags, src, count=2):
    from paper_1106_0557_gb300 import Plan
    d = torch.from_numpy(src.astype(NP[dtype])).cuda()
    with Plan(N, h, dtype, flags=flags) as p:
        outs = [p.solve(d).clone() for _ in range(count)]
        host = p.solve_host(src.astype(NP[dtype]))
        p.check()
    torch.cuda.synchronize()
    return outs, host


CANARY_SHAPES = [
    ((37, 20, 13), (1.0, 0.5, 2.0)),     # ragged on every axis
    ((64, 64, 64), (1.0, 1.0, 1.0)),
    ((100, 60, 130), (0.5, 0.25, 1.0)),  # Mz = 384
    ((9, 1100, 8), (1.0, 2.0, 1.0)),     # My = 2304
    ((60, 30, 1100), (1.0, 1.0, 1.0)),   # Mz = 2304: paired z tiles
]


@pytest.mark.parametrize("dtype", ["f32", "df64"])
@pytest.mark.parametrize("form", [0, native.IPF_FLAG_Y_TILES, native.IPF_FLAG_Y_STREAM])
@pytest.mark.parametrize("N,h", CANARY_SHAPES)
def test_canary_workspace_reads_only_what_the_solve_wrote(N, h, form, dtype):
    src = rand_src(N, sum(N))
    plain, host_plain = device_solves(N, h, dtype, form, src)
    canary, host_canary = device_solves(N, h, dtype, form | native.IPF_FLAG_TEST_CANARY, src)
    assert torch.isfinite(canary[0]).all() and torch.isfinite(canary[1]).all()
    assert torch.equal(canary[0], plain[0]) and torch.equal(canary[1], plain[0])
    assert torch.equal(plain[1], plain[0])  # determinism
    assert np.isfinite(host_canary).all()
    assert np.array_equal(host_canary, host_plain)
    assert np.array_equal(host_plain, plain[0].cpu().numpy())


@pytest.mark.parametrize("i,kind", list(enumerate(["workspace", "tables", "spectrum"])))
def test_forced_allocation_failure_frees_everything(i, kind, monkeypatch):
    """The failing plan leaves device memory and the spectrum cache as they
    were; a plan made afterwards solves correctly."""
    from paper_1106_0557_gb300 import Plan
    N = (40, 36, 30)
    # width ratios no other test uses (one set per case), so that the
    # spectrum is not cached yet and the plan has to allocate it
    h = (1.0, 1.7, 1.3 + 0.01 * i)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    cache0 = native.ipf_greens_cache_bytes()
    monkeypatch.setenv("ISOFFT_TEST_FAIL_ALLOC", kind)
    with pytest.raises(native.IsofftError) as ei:
        Plan(N, h, "f32")
    assert ei.value.status == native.IPF_OUT_OF_MEMORY
    monkeypatch.delenv("ISOFFT_TEST_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert native.ipf_greens_cache_bytes() == cache0
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 8 << 20
    src = rand_src(N, 5)
    with Plan(N, h, "f32") as p:
        phi = p.solve(torch.from_numpy(src.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
        p.check()
    ref = oracle.solve(src.astype(np.float32).astype(np.float64), h)
    assert oracle.max_rel_error(phi, ref) <= TOL["f32"]


def test_forced_staging_failure_then_host_solves_work(monkeypatch):
    from paper_1106_0557_gb300 import Plan
    N, h = (33, 20, 17), (1.0, 1.0, 1.0)
    src = rand_src(N, 6).astype(np.float32)
    with Plan(N, h, "f32") as p:
        want = p.solve(torch.from_numpy(src).cuda()).cpu().numpy()
        monkeypatch.setenv("ISOFFT_TEST_FAIL_ALLOC", "staging")
        with pytest.raises(native.IsofftError) as ei:
            p.solve_host(src)
        assert ei.value.status == native.IPF_OUT_OF_MEMORY
        monkeypatch.delenv("ISOFFT_TEST_FAIL_ALLOC")
        assert np.array_equal(p.solve_host(src), want)


def test_nvtx_ranges_leave_the_potential_unchanged(monkeypatch):
    N, h = (48, 40, 33), (1.0, 1.0, 1.0)
    src = rand_src(N, 7)
    plain, _ = device_solves(N, h, "f32", 0, src, count=1)
    monkeypatch.setenv("ISOFFT_NVTX", "1")
    traced, _ = device_solves(N, h, "f32", 0, src, count=1)
    assert torch.equal(traced[0], plain[0])


@pytest.mark.parametrize("dtype", ["f32", "df64"])
def test_spectrum_directory_lets_a_restart_skip_the_build(dtype, tmp_path, monkeypatch, capfd):
    """With ISOFFT_SPECTRUM_DIR set, the first plan builds the spectrum and
    writes it; once the in-memory cache is trimmed, the next plan reads the
    file (no build) and solves bitwise the same; a corrupted file is
    ignored, rebuilt and replaced."""
    from paper_1106_0557_gb300 import Plan
    N = (30, 26, 22)
    h = (1.0, 1.3, 0.9) if dtype == "f32" else (1.0, 1.3, 0.8)  # width ratios no other test uses
    monkeypatch.setenv("ISOFFT_SPECTRUM_DIR", str(tmp_path))
    monkeypatch.delenv("ISOFFT_VERBOSITY", raising=False)
    d = torch.from_numpy(rand_src(N, 11).astype(NP[dtype])).cuda()

    def restart():
        with Plan(N, h, dtype, verbosity=native.IPF_CONSOLE_INFO_1) as p:
            out = p.solve(d).cpu().numpy()
            p.check()
        native.ipf_greens_cache_trim(0)  # the next plan finds no spectrum in memory
        return out, capfd.readouterr().err

    first, log = restart()
    assert "building Green's spectrum" in log
    files = list(tmp_path.glob("isofft_spectrum_*.bin"))
    assert len(files) == 1
    second, log = restart()
    assert "loaded Green's spectrum" in log and "building Green's spectrum" not in log
    assert np.array_equal(second, first)
    raw = bytearray(files[0].read_bytes())
    raw[-5] ^= 0xFF
    files[0].write_bytes(bytes(raw))
    third, log = restart()
    assert "building Green's spectrum" in log
    assert np.array_equal(third, first)
    fourth, log = restart()
    assert "loaded Green's spectrum" in log
    assert np.array_equal(fourth, first)
