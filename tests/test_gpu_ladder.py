"""The paper's convergence ladders (Secs. 4.1 and 4.2) on one GPU, up to the
largest mesh the paper ran, 1152^3 cells (doubled mesh 2304^3).

* Parity at 1152^3: a unit source at a corner returns the Green's function
  (Eq. 6, Eq. 9 at the origin) at every one of the 1.5e9 cells, read from
  the oracle slab by slab; and the uniform sphere at sampled cells against
  the definition (route 1, a direct sum over all source cells).
* Physics: the L1 error (Eq. 11) against the closed forms (Eq. 10 for the
  sphere, Eqs. 14-19 for the spheroid) over the paper's resolutions
  48^3 ... 1152^3.  The paper reports convergence better than first order
  for the sphere and between first and second order for the spheroid;
  the tests fit the order over the ladder and require it above 1.

Sources are made on the device (sources.rasterize_torch, the seeded input
generator); every expected value comes from the oracle on the CPU.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_1106_0557_gb300 import native, sources

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    native.lib()


def solve_on_device(w, dtype="f32"):
    from paper_1106_0557_gb300 import Plan
    tdt = torch.float32 if dtype == "f32" else torch.float64
    src = sources.rasterize_torch(w.bodies, w.N, w.h, w.lo, dtype=tdt)
    with Plan(w.N, w.h, dtype) as p:
        phi = p.solve(src, src)  # in place, as the paper overwrites its source
        p.check()
    torch.cuda.synchronize()
    return phi


def slab_reduce(phi, fn, slab=32, workers=16):
    """Apply fn(k0, phi_slab_fp64) to z slabs of a device array on host
    threads (numpy releases the GIL in its ufuncs); returns the list of
    results in slab order."""
    nz = phi.shape[0]
    starts = list(range(0, nz, slab))
    out = []
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for b in range(0, len(starts), workers):  # at most `workers` slabs on the host at once
            futs = [ex.submit(fn, k0, phi[k0:k0 + slab].cpu().numpy().astype(np.float64))
                    for k0 in starts[b:b + workers]]
            out += [f.result() for f in futs]
    return out


def l1_against_closed_form(w, phi):
    """Eq. 11 over all cells, the closed form evaluated per slab."""
    x, y, z = w.coords()

    def part(k0, ph):
        ex = analytic.bodies_potential(w.bodies, x, y, z[k0:k0 + ph.shape[0]])
        return float(np.abs(ph - ex).sum()), float(np.abs(ex).sum())

    parts = slab_reduce(phi, part)
    return sum(p[0] for p in parts) / sum(p[1] for p in parts)


def fitted_order(ns, errs):
    """Least-squares slope of log(error) against log(h), h ~ 1/n."""
    return float(-np.polyfit(np.log(np.asarray(ns, float)), np.log(np.asarray(errs, float)), 1)[0])


def ladder(make, ns):
    errs = []
    for n in ns:
        w = make(n)
        phi = solve_on_device(w)
        errs.append(l1_against_closed_form(w, phi))
        del phi
        torch.cuda.empty_cache()
    return errs


def test_impulse_response_1152_is_green_function():
    """A unit source at the corner (0, 0, 0) of 1152^3 cells (doubled mesh
    2304^3, FP32): every cell of the potential equals the Green's function
    at its offset (normwise 1e-5), read from the oracle slab by slab."""
    from paper_1106_0557_gb300 import Plan
    n, h = 1152, (1.0, 1.0, 1.0)
    src = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    src[0, 0, 0] = 1.0
    with Plan((n, n, n), h, "f32") as p:
        assert p.padded_shape == (2304, 2304, 2304)
        phi = p.solve(src, src)
        p.check()
    torch.cuda.synchronize()

    def part(k0, ph):
        want = oracle.green_block((0, 0, k0), (n, n, ph.shape[0]), h)
        return float(np.max(np.abs(ph - want))), float(np.max(np.abs(want)))

    parts = slab_reduce(phi, part, slab=16)
    err = max(p[0] for p in parts) / max(p[1] for p in parts)
    print("impulse 1152^3 FP32 normwise error %.3e" % err)
    assert err <= 1e-5


def test_paper_sphere_ladder_to_1152():
    """Sec. 4.1: the uniform unit sphere in [-1.2, 1.2]^3 over the paper's
    resolutions.  At 1152^3 sampled cells match the definition (route 1);
    over the ladder the L1 error falls faster than first order."""
    ns = sources.PAPER_LADDER
    errs = ladder(sources.paper_sphere, ns)
    order = fitted_order(ns, errs)
    print("sphere ladder", ns, ["%.3e" % e for e in errs], "fitted order %.2f" % order)
    assert order > 1.0, (errs, order)
    assert errs[-1] < errs[0] / (ns[-1] / ns[0]), errs

    # parity at full size against the definition, at sampled cells
    w = sources.paper_sphere(1152)
    phi = solve_on_device(w)
    src = sources.rasterize_torch(w.bodies, w.N, w.h, w.lo, dtype=torch.float32).cpu().numpy()
    g = np.random.default_rng(17)
    cells = np.concatenate([g.integers(0, src.size, 6), [0, src.size - 1, src.size // 2 + w.N[0] // 2]])
    ref = oracle.direct_points(src, w.h, cells)
    got = phi.flatten()[torch.from_numpy(cells).cuda()].double().cpu().numpy()
    scale = float(phi.abs().max())
    assert np.max(np.abs(got - ref)) / scale <= 1e-5


def test_paper_spheroid_ladder_to_1152():
    """Sec. 4.2: the uniform spheroid (e = 0.9, a = 0.5) in [-1, 1]^3 over
    the paper's resolutions: the L1 error falls faster than first order."""
    ns = sources.PAPER_LADDER
    errs = ladder(sources.paper_spheroid, ns)
    order = fitted_order(ns, errs)
    print("spheroid ladder", ns, ["%.3e" % e for e in errs], "fitted order %.2f" % order)
    assert order > 1.0, (errs, order)
    assert errs[-1] < errs[0] / (ns[-1] / ns[0]), errs
