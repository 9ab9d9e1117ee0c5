"""Seeded synthetic source distributions shaped like the paper's test problems.

This module is shared by the tests, the benchmark and the smoke check; it
holds none of the solver's arithmetic -- only the drawing of bodies and their
point sampling on the mesh.  Every workload is reproducible from its seed
(numpy ``Generator(PCG64(seed))``).

Conventions (the paper leaves them open):
* mesh points are cell centres, x_i = lo + (i + 1/2) h, arrays are C order
  [z][y][x];
* Newton's constant is 1 and the source is S = 4 pi rho (Sec. 4.1);
* a homogeneous body is sampled by its indicator at the cell centres;
  overlapping bodies add.

Bodies are dicts so the oracle's closed forms can evaluate the same list:
``{"kind": "sphere", "center", "radius", "rho"}``,
``{"kind": "spheroid", "center", "a", "b", "rho"}`` (oblate, axis z),
``{"kind": "gaussian", "center", "sigma", "amp"}``.
"""
import math

import numpy as np

FOUR_PI = 4.0 * math.pi


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def cell_centers(N, h, lo=(0.0, 0.0, 0.0)):
    """Open-mesh coordinates (z, y, x broadcastable) of the cell centres."""
    Nx, Ny, Nz = N
    x = lo[0] + (np.arange(Nx) + 0.5) * h[0]
    y = lo[1] + (np.arange(Ny) + 0.5) * h[1]
    z = lo[2] + (np.arange(Nz) + 0.5) * h[2]
    return x[None, None, :], y[None, :, None], z[:, None, None]


def rasterize(bodies, N, h, lo=(0.0, 0.0, 0.0), dtype=np.float64):
    """Point-sample S = 4 pi rho of the bodies at the cell centres."""
    x, y, z = cell_centers(N, h, lo)
    S = np.zeros((N[2], N[1], N[0]), dtype=np.float64)
    for bd in bodies:
        c = bd["center"]
        if bd["kind"] == "sphere":
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            S += np.where(r2 <= bd["radius"] ** 2, FOUR_PI * bd["rho"], 0.0)
        elif bd["kind"] == "spheroid":
            q = ((x - c[0]) ** 2 + (y - c[1]) ** 2) / bd["a"] ** 2 + (z - c[2]) ** 2 / bd["b"] ** 2
            S += np.where(q <= 1.0, FOUR_PI * bd["rho"], 0.0)
        elif bd["kind"] == "gaussian":
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            S += FOUR_PI * bd["amp"] * np.exp(-r2 / (2.0 * bd["sigma"] ** 2))
        else:
            raise ValueError(bd["kind"])
    return S.astype(dtype, copy=False)


def rasterize_torch(bodies, N, h, lo=(0.0, 0.0, 0.0), device="cuda", dtype=None):
    """The same point sampling as `rasterize`, evaluated with torch on a
    device (for large sources made in bulk, e.g. a serving source bank)."""
    import torch
    dtype = dtype or torch.float64
    Nx, Ny, Nz = N
    x = (lo[0] + (torch.arange(Nx, device=device, dtype=torch.float64) + 0.5) * h[0]).view(1, 1, Nx)
    y = (lo[1] + (torch.arange(Ny, device=device, dtype=torch.float64) + 0.5) * h[1]).view(1, Ny, 1)
    z = (lo[2] + (torch.arange(Nz, device=device, dtype=torch.float64) + 0.5) * h[2]).view(Nz, 1, 1)
    S = torch.zeros((Nz, Ny, Nx), dtype=torch.float64, device=device)
    for bd in bodies:
        c = bd["center"]
        if bd["kind"] == "sphere":
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            S += (r2 <= bd["radius"] ** 2).to(torch.float64) * (FOUR_PI * bd["rho"])
        elif bd["kind"] == "spheroid":
            q = ((x - c[0]) ** 2 + (y - c[1]) ** 2) / bd["a"] ** 2 + (z - c[2]) ** 2 / bd["b"] ** 2
            S += (q <= 1.0).to(torch.float64) * (FOUR_PI * bd["rho"])
        elif bd["kind"] == "gaussian":
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            S += FOUR_PI * bd["amp"] * torch.exp(-r2 / (2.0 * bd["sigma"] ** 2))
        else:
            raise ValueError(bd["kind"])
    return S.to(dtype)


class Workload:
    """A seeded problem: mesh shape N = (Nx, Ny, Nz), cell widths h, the box
    origin and the bodies that make the source."""

    def __init__(self, name, N, h, bodies, lo=(0.0, 0.0, 0.0), dtype="f64"):
        self.name = name
        self.N = tuple(int(n) for n in N)
        self.h = tuple(float(v) for v in h)
        self.lo = tuple(float(v) for v in lo)
        self.bodies = bodies
        self.dtype = dtype

    def source(self, dtype=np.float64):
        return rasterize(self.bodies, self.N, self.h, self.lo, dtype)

    def coords(self):
        return cell_centers(self.N, self.h, self.lo)

    def __repr__(self):
        return "Workload(%s, N=%s, h=%s, %d bodies)" % (self.name, self.N, self.h, len(self.bodies))


def single_sphere(n=32, radius=0.25, rho=1.0):
    """Unit box [0,1]^3, n^3 cells, one homogeneous sphere at the centre:
    a scaled copy of the Sec. 4.1 test."""
    h = 1.0 / n
    return Workload("sphere-%d" % n, (n, n, n), (h, h, h),
                    [{"kind": "sphere", "center": (0.5, 0.5, 0.5), "radius": radius, "rho": rho}])


def multi_sphere_bodies(g, extent=(1.0, 1.0, 1.0), n_spheres=8, gaussian=True):
    """8 spheres with centres U[0.3,0.7] (fraction of the box), radii
    U[0.02,0.1] x the smallest box extent, densities U[0.5,2], plus one
    Gaussian blob of sigma 0.05 x the smallest extent, centre in the same
    range."""
    L = min(extent)
    bodies = []
    for _ in range(n_spheres):
        c = tuple(float(v) * e for v, e in zip(g.uniform(0.3, 0.7, 3), extent))
        bodies.append({"kind": "sphere", "center": c,
                       "radius": float(g.uniform(0.02, 0.1)) * L,
                       "rho": float(g.uniform(0.5, 2.0))})
    if gaussian:
        c = tuple(float(v) * e for v, e in zip(g.uniform(0.3, 0.7, 3), extent))
        bodies.append({"kind": "gaussian", "center": c, "sigma": 0.05 * L, "amp": 1.0})
    return bodies


def multi_sphere(n=256, seed=0):
    """n^3 cells in the unit box with multi_sphere_bodies: the 256^3 solve
    (doubled mesh 512^3) the throughput figures are quoted on."""
    h = 1.0 / n
    return Workload("multisphere-%d-s%d" % (n, seed), (n, n, n), (h, h, h),
                    multi_sphere_bodies(rng(seed)))


def oblate_spheroids(n=512, seed=0, count=4):
    """n x n x n cells with anisotropic widths h = (1, 1, 2)/n over the box
    [0,1]^2 x [0,2]: seed-drawn uniform oblate spheroids (axis z,
    b/a ~ U[0.3,1], a ~ U[0.05,0.15], centres U[0.3,0.7]^2 x U[0.6,1.4],
    rho ~ U[0.5,2]) on a zero background, the Sec. 4.2 test problem
    generalised."""
    g = rng(seed)
    bodies = []
    for _ in range(count):
        a = float(g.uniform(0.05, 0.15))
        ratio = float(g.uniform(0.3, 1.0))
        c = (float(g.uniform(0.3, 0.7)), float(g.uniform(0.3, 0.7)), float(g.uniform(0.6, 1.4)))
        bodies.append({"kind": "spheroid", "center": c, "a": a, "b": a * ratio,
                       "rho": float(g.uniform(0.5, 2.0))})
    h = (1.0 / n, 1.0 / n, 2.0 / n)
    return Workload("spheroids-%d-s%d" % (n, seed), (n, n, n), h, bodies)


def binary_spheroid(n=384, e=0.28, a=0.5, rho=1.0):
    """The binary-spheroid test of Sec. 4.3: a box x in [-2, 2], y, z in
    [-1, 1] of 2n x n x n cells (isotropic h = 2/n), and two uniform oblate
    spheroids (symmetry axis z, eccentricity e, semi-major axis a) centred at
    (+-1, 0, 0).  n = 384 is the paper's 768 x 384 x 384 resolution; e = 0.28
    is the value of its figure caption."""
    h = 2.0 / n
    b = a * math.sqrt(1.0 - e * e)
    bodies = [{"kind": "spheroid", "center": (cx, 0.0, 0.0), "a": a, "b": b, "rho": rho} for cx in (-1.0, 1.0)]
    return Workload("binary-spheroid-%d" % n, (2 * n, n, n), (h, h, h), bodies, lo=(-2.0, -1.0, -1.0))


# The mesh resolutions of the convergence figures of Secs. 4.1 and 4.2.
PAPER_LADDER = (48, 144, 288, 384, 576, 768, 1152)


def paper_sphere(n, R=1.0, rho=1.0):
    """The Sec. 4.1 test: a uniform sphere of radius 1 centred at the origin
    of the box [-1.2, 1.2]^3, n^3 cells."""
    h = 2.4 / n
    return Workload("paper-sphere-%d" % n, (n, n, n), (h, h, h),
                    [{"kind": "sphere", "center": (0.0, 0.0, 0.0), "radius": R, "rho": rho}],
                    lo=(-1.2, -1.2, -1.2))


def paper_spheroid(n, e=0.9, a=0.5, rho=1.0):
    """The Sec. 4.2 test: a uniform oblate spheroid (axis z, eccentricity
    0.9, semi-major axis 0.5) centred at the origin of a box of size two in
    every dimension, [-1, 1]^3, n^3 cells."""
    h = 2.0 / n
    b = a * math.sqrt(1.0 - e * e)
    return Workload("paper-spheroid-%d" % n, (n, n, n), (h, h, h),
                    [{"kind": "spheroid", "center": (0.0, 0.0, 0.0), "a": a, "b": b, "rho": rho}],
                    lo=(-1.0, -1.0, -1.0))


BATCH_SIZES = (32, 48, 64, 96, 128)


def ragged_batch(count=64, h=1.0 / 128):
    """`count` independent grids; grid g draws each of Nx, Ny, Nz from
    {32, 48, 64, 96, 128} with seed g, isotropic cell width h, and sources
    drawn as in multi_sphere inside its own box."""
    out = []
    for gi in range(count):
        g = rng(gi)
        N = tuple(int(v) for v in g.choice(BATCH_SIZES, 3))
        extent = tuple(n * h for n in N)
        bodies = multi_sphere_bodies(g, extent)
        out.append(Workload("batch-%d" % gi, N, (h, h, h), bodies))
    return out


def serving_requests(count=10000, seed=0, n_lo=32, n_hi=384, fp32_share=0.7):
    """A stream of solve requests: cubic N = round(exp U[ln n_lo, ln n_hi]),
    h = 1/N, dtype 'f32' with probability fp32_share else 'f64', sources as
    in multi_sphere with a per-request seed.  Returns dicts with the shape,
    dtype and the seed that rebuilds the workload lazily."""
    g = rng(seed)
    logn = g.uniform(math.log(n_lo), math.log(n_hi), count)
    kinds = g.uniform(0.0, 1.0, count)
    reqs = []
    for i in range(count):
        n = int(round(math.exp(logn[i])))
        reqs.append({"id": i, "n": n, "dtype": "f32" if kinds[i] < fp32_share else "f64",
                     "seed": seed * 1000003 + i})
    return reqs


def request_workload(req):
    n = req["n"]
    h = 1.0 / n
    return Workload("req-%d" % req["id"], (n, n, n), (h, h, h),
                    multi_sphere_bodies(rng(req["seed"])), dtype=req["dtype"])
