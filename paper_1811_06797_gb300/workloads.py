"""Seeded synthetic workloads: geometries, discretisations, targets.

This module only builds input data (knot vectors, NURBS control nets, the
desired-state description, seeded random draws).  It holds none of the
method's arithmetic (no basis evaluation, no quadrature, no assembly), so
both the CUDA path and the CPU oracle take their inputs from here.

Geometries (Sec. 2, eq. geometryMapping and the NURBS curve definition):
  * unit cube       -- trilinear identity map, weight rank 1;
  * quarter annulus -- exact quadratic NURBS quarter circle (weights 1,
                       sqrt(2)/2, 1) swept between radii 1 and 2, extruded
                       linearly in z in [0, 1] (Sec. 6 "quarter annulus");
  * twisted annulus -- the same map composed with a rotation of angle
                       twist * z about the z-axis;
  * random volume   -- cubic B-spline map with 8 control points per
                       direction at the Greville abscissae of an open
                       uniform knot vector, each perturbed by seeded
                       Gaussian noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# kinds understood by both sides
GEO_NURBS = 0          # plain (rational) tensor-product map
GEO_NURBS_TWIST = 1    # map followed by rotation R(twist * z) about e_z

TARGET_ZERO = 0        # yhat = 0
TARGET_SINPROD = 1     # yhat = prod_k sin(pi x_k)
TARGET_GAUSS = 2       # yhat = exp(-|x - c|^2 / width)


def open_uniform_knots(degree: int, nelem: int) -> np.ndarray:
    """Open knot vector on [0, 1] with degree+1 fold end knots and nelem spans."""
    inner = np.linspace(0.0, 1.0, nelem + 1)
    return np.concatenate([np.zeros(degree), inner, np.ones(degree)])


@dataclass
class Geometry:
    kind: int
    degree: tuple
    knots: tuple               # three 1-D float64 arrays
    ctrl: np.ndarray           # (n1, n2, n3, 3) control points
    weights: np.ndarray        # (n1, n2, n3) NURBS weights (all 1 for B-splines)
    twist: float = 0.0         # radians per unit z (kind GEO_NURBS_TWIST)
    volume: float | None = None  # exact domain volume when known

    def homogeneous(self) -> np.ndarray:
        """Control net as (w x, w y, w z, w), shape (n1, n2, n3, 4), C order."""
        hw = np.empty(self.ctrl.shape[:3] + (4,), dtype=np.float64)
        hw[..., :3] = self.ctrl * self.weights[..., None]
        hw[..., 3] = self.weights
        return np.ascontiguousarray(hw)


@dataclass
class Space:
    degree: tuple
    knots: tuple               # three open knot vectors of the trial/test space
    nquad: int                 # Gauss points per element and direction

    @property
    def nbasis(self):
        return tuple(len(k) - p - 1 for k, p in zip(self.knots, self.degree))

    @property
    def ninterior(self):
        return tuple(n - 2 for n in self.nbasis)


@dataclass
class Target:
    kind: int
    center: tuple = (0.0, 0.0, 0.0)
    width: float = 1.0

    def params(self) -> np.ndarray:
        return np.array([*self.center, self.width], dtype=np.float64)


@dataclass
class Workload:
    name: str
    geometry: Geometry
    space: Space
    target: Target
    beta: float
    tol: float
    extra: dict = field(default_factory=dict)


def uniform_space(degree: int, nelem: int, nquad: int | None = None) -> Space:
    k = open_uniform_knots(degree, nelem)
    return Space(degree=(degree,) * 3, knots=(k, k.copy(), k.copy()),
                 nquad=degree + 1 if nquad is None else nquad)


def unit_cube() -> Geometry:
    k = np.array([0.0, 0.0, 1.0, 1.0])
    c = np.zeros((2, 2, 2, 3))
    for i in range(2):
        for j in range(2):
            for m in range(2):
                c[i, j, m] = (i, j, m)
    return Geometry(GEO_NURBS, (1, 1, 1), (k, k.copy(), k.copy()), c,
                    np.ones((2, 2, 2)), 0.0, 1.0)


def affine_box(a: np.ndarray, shift=(0.0, 0.0, 0.0)) -> Geometry:
    """Trilinear map x = a @ xhat + shift (a parallelepiped)."""
    g = unit_cube()
    c = np.einsum("ij,abcj->abci", np.asarray(a, float), g.ctrl) + np.asarray(shift)
    return Geometry(GEO_NURBS, g.degree, g.knots, c, g.weights, 0.0,
                    abs(float(np.linalg.det(a))))


def quarter_annulus(r_in: float = 1.0, r_out: float = 2.0, height: float = 1.0,
                    twist: float = 0.0) -> Geometry:
    """Direction 1 angular (quadratic NURBS), 2 radial (linear), 3 axial (linear)."""
    ks = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    kl = np.array([0.0, 0.0, 1.0, 1.0])
    c = np.zeros((3, 2, 2, 3))
    w = np.zeros((3, 2, 2))
    s2 = math.sqrt(2.0) / 2.0
    for j, r in enumerate((r_in, r_out)):
        for m, z in enumerate((0.0, height)):
            c[0, j, m] = (r, 0.0, z)
            c[1, j, m] = (r, r, z)
            c[2, j, m] = (0.0, r, z)
            w[:, j, m] = (1.0, s2, 1.0)
    vol = 0.25 * math.pi * (r_out ** 2 - r_in ** 2) * height
    kind = GEO_NURBS_TWIST if twist != 0.0 else GEO_NURBS
    return Geometry(kind, (2, 1, 1), (ks, kl, kl.copy()), c, w, twist, vol)


def greville(knots: np.ndarray, degree: int) -> np.ndarray:
    n = len(knots) - degree - 1
    return np.array([knots[i + 1:i + degree + 1].mean() for i in range(n)])


def random_volume(seed: int = 1811, degree: int = 3, nctrl: int = 8,
                  sigma_frac: float = 0.05) -> Geometry:
    """Cubic B-spline volume, control points at Greville abscissae + N(0, sigma)."""
    nel = nctrl - degree
    k = open_uniform_knots(degree, nel)
    g = greville(k, degree)
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1)
    rng = np.random.default_rng(seed)
    c = c + rng.normal(0.0, sigma_frac / nel, size=c.shape)
    return Geometry(GEO_NURBS, (degree,) * 3, (k, k.copy(), k.copy()), c,
                    np.ones(c.shape[:3]), 0.0, None)


ANNULUS_CENTROID = (28.0 / (9.0 * math.pi), 28.0 / (9.0 * math.pi), 0.5)


def config(idx: int) -> Workload:
    """The five synthetic workloads, by index 1..5."""
    if idx == 1:
        return Workload("unit_cube_p2_e16", unit_cube(), uniform_space(2, 16),
                        Target(TARGET_SINPROD), beta=1e-6, tol=1e-12)
    if idx == 2:
        return Workload("quarter_annulus_p3_e64", quarter_annulus(), uniform_space(3, 64),
                        Target(TARGET_GAUSS, ANNULUS_CENTROID, 0.1), beta=1e-4, tol=1e-6)
    if idx == 3:
        return Workload("twisted_annulus_p3_e256", quarter_annulus(twist=math.pi / 4),
                        uniform_space(3, 256), Target(TARGET_GAUSS, ANNULUS_CENTROID, 0.1),
                        beta=1e-4, tol=1e-8, extra={"betas": (1e-2, 1e-4, 1e-6)})
    if idx == 4:
        return Workload("twisted_annulus_p3_e128_grad", quarter_annulus(twist=math.pi / 4),
                        uniform_space(3, 128), Target(TARGET_GAUSS, ANNULUS_CENTROID, 0.1),
                        beta=1e-4, tol=1e-8, extra={"batch": 8, "seeds": tuple(range(8))})
    if idx == 5:
        return Workload("random_volume_p2_e512", random_volume(), uniform_space(2, 512),
                        Target(TARGET_SINPROD), beta=1e-6, tol=1e-8)
    raise ValueError(idx)


def small(geometry: Geometry, degree: int, nelem: int, target: Target | None = None,
          beta: float = 1e-2, tol: float = 1e-10, nquad: int | None = None) -> Workload:
    """A small parity case on any geometry."""
    return Workload(f"small_p{degree}_e{nelem}", geometry, uniform_space(degree, nelem, nquad),
                    target or Target(TARGET_SINPROD), beta, tol)


def random_controls(n_interior: tuple, seeds) -> np.ndarray:
    """Seeded N(0,1) control coefficient tensors, shape (len(seeds), n1, n2, n3)."""
    out = [np.random.default_rng(s).standard_normal(n_interior) for s in seeds]
    return np.stack(out)


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)
