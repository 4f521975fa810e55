"""Seeded synthetic workloads shared by the CUDA path's tests/bench and by the CPU oracle.

This module holds input generation only: solid masks of the paper's geometries (a circular
cylinder, Sec. IV.A; a sphere, Sec. IV.C; flat plates, Sec. IV.B), the initial density field
(a tanh droplet profile plus seeded noise) and the named workload configurations.  It holds
none of the method's arithmetic: no equation of state, no coexistence densities, no collision.
Coexistence densities are parameters here; callers obtain them from their own solver.

Array layout everywhere: C order with x fastest, i.e. numpy shape (ny, nx) in 2D and
(nz, ny, nx) in 3D.  A node's linear index is x + nx*(y + ny*z).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

NOISE_SEED = 1234          # density-noise seed of the parity configurations
BATCH_SEED = 20190812      # parameter draws of the batched workload
ADJOINT_TARGET_SEED = 7    # smooth random wettability target of the adjoint workload


def _grid(shape):
    """Integer node coordinates (x, y[, z]) for an array of numpy shape `shape` (x fastest)."""
    idx = np.indices(shape, dtype=np.float64)
    return idx[::-1]  # (x, y) or (x, y, z)


def _min_image(d, n):
    """Periodic minimum-image displacement along an axis of length n."""
    return d - n * np.round(d / n)


def ball_mask(shape, center, radius):
    """Solid mask of a disc (2D) or ball (3D): node solid iff |x - c|^2 <= R^2 (integer nodes).

    The cylinder of Sec. IV.A and the sphere of Sec. IV.C are staircase-discretised this way.
    Periodic images are not considered (the bodies of the paper's tests stay inside the box).
    """
    coords = _grid(shape)
    r2 = sum((c - float(cc)) ** 2 for c, cc in zip(coords, center))
    return (r2 <= float(radius) ** 2).astype(np.uint8)


def plates_mask(shape, axis_from_last=1):
    """Two solid plates: the first and last layer along y (2D) are solid (Sec. IV.B channel)."""
    m = np.zeros(shape, dtype=np.uint8)
    if len(shape) == 2:
        m[0, :] = 1
        m[-1, :] = 1
    else:
        m[:, 0, :] = 1
        m[:, -1, :] = 1
    return m


def flat_wall_mask(shape, thickness):
    """A solid slab occupying y < thickness (2D) / y < thickness (3D); periodic elsewhere."""
    m = np.zeros(shape, dtype=np.uint8)
    if len(shape) == 2:
        m[:thickness, :] = 1
    else:
        m[:, :thickness, :] = 1
    return m


def tanh_drop_density(shape, center, radius, rho_l, rho_g, width=2.0, periodic=True):
    """Initial density of a liquid drop in gas: a tanh profile of the given width.

    rho(x) = (rho_l + rho_g)/2 + (rho_l - rho_g)/2 * tanh(2 (r - |x - c|) / W),
    with |x - c| the periodic minimum-image distance when `periodic`.
    """
    coords = _grid(shape)
    d2 = np.zeros(shape)
    for c, cc, n in zip(coords, center, shape[::-1]):
        d = c - float(cc)
        if periodic:
            d = _min_image(d, n)
        d2 += d * d
    dist = np.sqrt(d2)
    return 0.5 * (rho_l + rho_g) + 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (radius - dist) / width)


def slab_density(shape, lo, hi, rho_l, rho_g, width=2.0):
    """Liquid slab lo < y < hi in gas (flat interfaces normal to y), tanh edges."""
    y = _grid(shape)[1]
    return rho_g + (rho_l - rho_g) * 0.5 * (np.tanh(2.0 * (y - lo) / width) - np.tanh(2.0 * (y - hi) / width))


def density_noise(shape, amplitude=1e-6, seed=NOISE_SEED):
    """Seeded uniform noise amplitude*U(-1, 1) (numpy PCG64), generated once and passed to both sides."""
    rng = np.random.default_rng(seed)
    return amplitude * rng.uniform(-1.0, 1.0, size=shape)


# ----------------------------------------------------------------------------------------------
# Named workloads.  Geometry follows Sec. IV.A (cylinder) and Sec. IV.C (sphere); sizes, EOS and
# wall parameters are the benchmark configurations of this project.
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    lattice: str                  # "D2Q9" or "D3Q19"
    shape: tuple                  # numpy shape (ny, nx) / (nz, ny, nx)
    body_center: tuple            # (x, y[, z]) of the cylinder/sphere
    body_radius: float
    drop_center: tuple
    drop_radius: float
    eos: str                      # "CS" or "PR"
    t_over_tc: float
    kappa: float                  # unified IVD parameter: kappa>=0 -> phi=1+kappa, kappa<0 -> drho=-kappa
    steps: int
    noise: float = 1e-6
    width: float = 2.0

    @property
    def nodes(self) -> int:
        return int(np.prod(self.shape))

    def mask(self) -> np.ndarray:
        return ball_mask(self.shape, self.body_center, self.body_radius)

    def rho0(self, rho_l: float, rho_g: float, seed: int = NOISE_SEED) -> np.ndarray:
        """Initial density: tanh drop plus noise at fluid nodes; solid nodes hold rho_g (unused)."""
        rho = tanh_drop_density(self.shape, self.drop_center, self.drop_radius, rho_l, rho_g, self.width)
        if self.noise > 0:
            rho = rho + density_noise(self.shape, self.noise, seed)
        m = self.mask()
        rho = np.where(m != 0, rho_g, rho)
        return np.ascontiguousarray(rho, dtype=np.float64)


def c1_parity_cylinder() -> Workload:
    """100x100 periodic, cylinder R=20 at (50,50), tangent drop r=25 at (50,95), C-S 0.7Tc, phi=1.2."""
    return Workload("c1_d2q9_fp64_100x100", "D2Q9", (100, 100), (50.0, 50.0), 20.0,
                    (50.0, 95.0), 25.0, "CS", 0.7, 0.2, 1000)


def c2_cylinder_sweep_kappas(rho_l: float, rho_g: float, points: int = 24) -> list:
    """Wall-parameter sweep of the 600x400 cylinder workload from hydrophilic to hydrophobic, in the
    unified kappa form: half of the points have phi evenly spaced from 1.5 down to 1.0 (kappa =
    phi - 1, Eq. 16's first branch, theta below about 90 degrees), the other half drho evenly
    spaced up to 0.25 (rho_l - rho_g) (kappa = -drho, the second branch, theta above it)."""
    d = rho_l - rho_g
    h = points // 2
    phi = [0.5 - 0.5 * i / (h - 1) for i in range(h)]                       # kappa = phi - 1
    drho = [0.25 * d * (i + 1) / (points - h) for i in range(points - h)]   # kappa = -drho
    return phi + [-x for x in drho]


def c2_cylinder_600x400(kappa: float = 0.15) -> Workload:
    """600x400, cylinder R=60 at (300,150), drop r=70 at (300,280) (tangent-ish), C-S 0.6Tc."""
    return Workload("c2_d2q9_600x400", "D2Q9", (400, 600), (300.0, 150.0), 60.0,
                    (300.0, 280.0), 70.0, "CS", 0.6, kappa, 20000)


def c3_sphere_256() -> Workload:
    """256^3 D3Q19, sphere R=40 at (128,128,100), drop r=45 at (128,128,185), C-S 0.7Tc."""
    return Workload("c3_d3q19_256cube", "D3Q19", (256, 256, 256), (128.0, 128.0, 100.0), 40.0,
                    (128.0, 128.0, 185.0), 45.0, "CS", 0.7, 0.2, 5000)


def sphere_fig14(kappa: float, steps: int = 30000) -> Workload:
    """The Sec. IV.C sphere as the paper sets it up (Fig. 14): 200 x 200 x 280 D3Q19, sphere R = 50 at
    (100, 100, 100), drop r = 45 at (100, 100, 180), Peng-Robinson at 0.86 Tc (the Sec. IV.A EOS and
    densities), wall parameter kappa (0.2: phi = 1.2; 0: phi = 1; -0.55: drho = 0.55)."""
    return Workload("fig14_sphere_200x200x280", "D3Q19", (280, 200, 200), (100.0, 100.0, 100.0), 50.0,
                    (100.0, 100.0, 180.0), 45.0, "PR", 0.86, kappa, steps)


def sphere_drop_64(steps: int = 1000, kappa: float = 0.2) -> Workload:
    """64^3 D3Q19 drop on a sphere, for runs the oracle can finish: the 256^3 workload's sphere scaled
    by 1/4 (R = 10, at (32, 32, 20)) with a tangent drop r = 16 at (32, 32, 46), C-S 0.7 Tc, wall
    parameter kappa (0.2 as in the full workload).  The drop is larger than the scaled 11.25: at that
    radius the Laplace pressure raises the equilibrium vapour density enough that the whole drop
    evaporates into the box within 1000 steps (Kelvin effect), leaving no interface to fit."""
    return Workload("d3q19_sphere_drop_64cube", "D3Q19", (64, 64, 64), (32.0, 32.0, 20.0), 10.0,
                    (32.0, 32.0, 46.0), 16.0, "CS", 0.7, kappa, steps)


def c4_batch(n_instances: int = 96, seed: int = BATCH_SEED) -> list:
    """Batched 2D instances: square N ~ U{128..512}, cylinder radius U(0.15,0.25) N at the centre,
    drop radius U(1.1,1.4) x cylinder radius placed tangent above it, kappa per instance.

    kappa is drawn uniformly in [-0.6, 0.6]; negative values are drho in units of the EOS's
    (rho_l - rho_g) and are converted by the caller (`kappa_abs`)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        n = int(rng.integers(128, 513))
        rc = float(rng.uniform(0.15, 0.25)) * n
        rd = float(rng.uniform(1.1, 1.4)) * rc
        kap = float(rng.uniform(-0.6, 0.6))
        c = (n / 2.0, n / 2.0)
        d = (n / 2.0, n / 2.0 + rc + rd)   # centre distance R + r: tangent, drop above (+y)
        out.append(Workload(f"c4_inst{i}_{n}", "D2Q9", (n, n), c, rc, d, rd, "CS", 0.7, kap, 4000))
    return out


def c5_adjoint_256() -> Workload:
    """256x256, cylinder R=40, per-wall-node wettability; 2000 steps, checkpoint every 100."""
    return Workload("c5_adjoint_256", "D2Q9", (256, 256), (128.0, 100.0), 40.0,
                    (128.0, 100.0 + 40.0 + 45.0), 45.0, "CS", 0.7, 0.1, 2000)


def smooth_polar_field(angles: np.ndarray, modes: int = 4, amplitude: float = 0.2,
                       seed: int = ADJOINT_TARGET_SEED) -> np.ndarray:
    """A seeded smooth random function of the polar angle: sum of `modes` Fourier modes."""
    rng = np.random.default_rng(seed)
    a = rng.normal(size=modes)
    b = rng.normal(size=modes)
    v = np.zeros_like(angles, dtype=np.float64)
    for k in range(1, modes + 1):
        v += a[k - 1] * np.cos(k * angles) + b[k - 1] * np.sin(k * angles)
    v *= amplitude / max(1e-12, np.max(np.abs(v)))
    return v


def impact_300x400() -> Workload:
    """Droplet impact on a cylinder (Sec. IV.B): 300x400, cylinder R=70 at (150,180), drop r=50 at
    (150,310) moving down at U0 = 0.06 (Re = U0 2r / nu = 600, so nu = 0.01), PR EOS at 0.86 Tc;
    10000 steps in the paper.  The wall parameter is the caller's (the paper tunes each scheme to
    theta ~ 60 deg: phi ~ 1.135 for IVD, rho_w ~ 3.45 for VD)."""
    return Workload("impact_300x400", "D2Q9", (400, 300), (150.0, 180.0), 70.0, (150.0, 310.0), 50.0,
                    "PR", 0.86, 0.135, 10000)


def drop_velocity(rho0: np.ndarray, rho_l: float, rho_g: float, velocity) -> np.ndarray:
    """Initial velocity carried by the liquid: u = velocity x (rho0 - rho_g)/(rho_l - rho_g), clipped
    to [0, 1], so the drop moves and the gas starts at rest with a smooth transition across the
    tanh interface.  Shape (d,) + rho0.shape."""
    frac = np.clip((rho0 - rho_g) / (rho_l - rho_g), 0.0, 1.0)
    return np.stack([v * frac for v in velocity])
