"""Seeded synthetic inputs: initial phase fields, velocity fields and named workloads.

This module holds no step arithmetic of the method.  It only builds initial conditions and
parameter sets, in FP64 numpy, so that the CUDA path and the CPU oracle read identical bytes.

Phase convention: phi = 1 is the heavy (liquid) phase, phi = 0 the light (gas) phase; the
interface sits at phi = 1/2.  Initial profiles use the equilibrium interface of the
conservative Allen-Cahn equation (Section "Allen-Cahn equation for interface tracking"), read
as phi = 1/2 + 1/2 tanh(2 d / W) with d the signed Euclidean distance to the interface (the
printed profile uses an L1 distance without the factor 2; with the factor 2 the profile is the
exact zero of the chemical potential with beta = 12 sigma/W, kappa = 3 sigma W/2 and of the
sharpening flux with kappa_AC = 4 D/W).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def _axes(nx, ny, nz):
    """Node coordinates as broadcastable axes of shapes (1, 1, nx), (1, ny, 1), (nz, 1, 1): the
    same values as _grid without three full-size arrays (a 512^3 box would need 3 GB for them).
    Callers must combine all three so that the result has the full (nz, ny, nx) shape."""
    return (np.arange(nx, dtype=np.float64)[None, None, :], np.arange(ny, dtype=np.float64)[None, :, None],
            np.arange(nz, dtype=np.float64)[:, None, None])


def _min_image(d, n, periodic):
    if not periodic:
        return d
    return d - n * np.round(d / n)


def sphere_phi(nx, ny, nz, center, radius, width, inside=1.0, periodic=(True, True, True)):
    """tanh sphere: phi -> inside at the centre, 1 - inside far away."""
    x, y, z = _axes(nx, ny, nz)
    dx = _min_image(x - center[0], nx, periodic[0])
    dy = _min_image(y - center[1], ny, periodic[1])
    dz = _min_image(z - center[2], nz, periodic[2])
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    prof = 0.5 + 0.5 * np.tanh(2.0 * (radius - r) / width)
    return prof if inside == 1.0 else 1.0 - prof


def cylinder_phi(nx, ny, nz, center, radius, width, inside=1.0):
    """tanh cylinder along z (a 2D droplet when nz is small)."""
    x, y, _ = _grid(nx, ny, nz)
    dx = _min_image(x - center[0], nx, True)
    dy = _min_image(y - center[1], ny, True)
    r = np.sqrt(dx * dx + dy * dy)
    prof = 0.5 + 0.5 * np.tanh(2.0 * (radius - r) / width)
    return prof if inside == 1.0 else 1.0 - prof


def slab_phi(nx, ny, nz, z_lo, z_hi, width):
    """Heavy slab between two planar interfaces normal to z (at z_lo and z_hi)."""
    _, _, z = _grid(nx, ny, nz)
    return 0.5 + 0.5 * np.tanh(2.0 * np.minimum(z - z_lo, z_hi - z) / width)


def layer_phi(nx, ny, nz, z_if, width, heavy_below=True):
    """One planar interface normal to z at z_if."""
    _, _, z = _grid(nx, ny, nz)
    s = (z_if - z) if heavy_below else (z - z_if)
    return 0.5 + 0.5 * np.tanh(2.0 * s / width)


def fourier_velocity(nx, ny, nz, modes=8, amplitude=0.01, seed=1234):
    """Smooth random periodic velocity: `modes` random Fourier modes with wave numbers 1..2 per
    axis, random phases and directions, scaled so that max |u| = amplitude.  FP64."""
    rng = np.random.default_rng(seed)
    x, y, z = _axes(nx, ny, nz)
    u = np.zeros((3, nz, ny, nx))
    for _ in range(modes):
        k = rng.integers(-2, 3, size=3)
        if not k.any():
            k[0] = 1
        kv = 2.0 * math.pi * k / np.array([nx, ny, nz], dtype=np.float64)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        amp = rng.normal(size=3)
        arg = kv[0] * x + kv[1] * y + kv[2] * z + ph
        s = np.sin(arg)
        for a in range(3):
            u[a] += amp[a] * s
    m = np.sqrt((u ** 2).sum(axis=0)).max()
    return u * (amplitude / m)


def wall_damp(u, nz):
    """Multiply a velocity field by sin(pi (z+1/2)/nz) so it vanishes at z walls."""
    z = np.arange(nz, dtype=np.float64)
    d = np.sin(math.pi * (z + 0.5) / nz)
    return u * d[None, :, None, None]


@dataclasses.dataclass
class Workload:
    """A named physical configuration (lattice units)."""
    name: str
    nx: int
    ny: int
    nz: int
    wall_z: int
    rho_l: float
    rho_g: float
    mu_l: float
    mu_g: float
    sigma: float
    width: float
    mobility: float
    gravity: tuple
    rho_ref: float
    body: tuple
    kind: str                  # "droplet" or "bubble"
    center: tuple
    radius: float
    noise: float = 0.0         # amplitude of the seeded Fourier velocity
    seed: int = 1234
    balanced_p0: bool = True   # start from pstar0() (Laplace + hydrostatic) instead of p* = 0

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def phi0(self):
        if self.kind == "droplet":
            return sphere_phi(self.nx, self.ny, self.nz, self.center, self.radius, self.width,
                              inside=1.0, periodic=(True, True, not self.wall_z))
        if self.kind == "bubble":
            return sphere_phi(self.nx, self.ny, self.nz, self.center, self.radius, self.width,
                              inside=0.0, periodic=(True, True, not self.wall_z))
        raise ValueError(self.kind)

    def u0(self):
        if self.noise == 0.0:
            return np.zeros((3, self.nz, self.ny, self.nx))
        u = fourier_velocity(self.nx, self.ny, self.nz, amplitude=self.noise, seed=self.seed)
        return wall_damp(u, self.nz) if self.wall_z else u

    def inside(self):
        """Indicator of the dispersed phase: phi for a droplet, 1 - phi for a bubble."""
        phi = self.phi0()
        return phi if self.kind == "droplet" else 1.0 - phi

    def pressure0(self):
        """Initial pressure p0 of the undeformed dispersed sphere in mechanical balance: the
        Laplace jump 2 sigma / R inside it, plus the hydrostatic head of the body force
        (rho - rho_ref) g in each phase, taken about the sphere's centre."""
        chi = self.inside()
        x, y, z = _axes(self.nx, self.ny, self.nz)
        per = (True, True, not self.wall_z)
        r = [_min_image(c - c0, n, pp) for c, c0, n, pp in
             zip((x, y, z), self.center, (self.nx, self.ny, self.nz), per)]
        head = sum(self.gravity[a] * r[a] for a in range(3))
        rho_in, rho_out = (self.rho_l, self.rho_g) if self.kind == "droplet" else (self.rho_g, self.rho_l)
        return (2.0 * self.sigma / self.radius) * chi + ((rho_in - self.rho_ref) * chi
                                                         + (rho_out - self.rho_ref) * (1.0 - chi)) * head

    def pstar0(self):
        """Initial non-dimensional pressure p*0 = p0 / (rho cs^2), with rho interpolated in phi."""
        phi = self.phi0()
        rho = self.rho_l * phi + (1.0 - phi) * self.rho_g
        return 3.0 * self.pressure0() / rho

    def pstar_init(self):
        """p*0 handed to the initialisation: pstar0() or None (p* = 0)."""
        return self.pstar0() if self.balanced_p0 else None

    def params(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, wall_z=self.wall_z, rho_l=self.rho_l,
                    rho_g=self.rho_g, mu_l=self.mu_l, mu_g=self.mu_g, sigma=self.sigma,
                    width=self.width, mobility=self.mobility, gravity=tuple(self.gravity),
                    rho_ref=self.rho_ref, body=tuple(self.body))


def static_droplet(L=48, radius=None, noise=0.0, seed=1234, sigma=0.01):
    """Static droplet: periodic L^3, sphere R (default L/4) centred, W = 4, density ratio 10,
    viscosity ratio 10 (nu_L = nu_G = 0.1, tau = 0.8), sigma = 0.01, D = 0.1, fluid at rest."""
    R = L / 4.0 if radius is None else radius
    c = (L - 1) / 2.0
    return Workload(name=f"static_droplet_{L}^3", nx=L, ny=L, nz=L, wall_z=0,
                    rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=sigma, width=4.0,
                    mobility=0.1, gravity=(0.0, 0.0, 0.0), rho_ref=1.0, body=(0.0, 0.0, 0.0),
                    kind="droplet", center=(c, c, c), radius=R, noise=noise, seed=seed)


def rising_bubble_params(Eo=10.0, Mo=1e-4, R=16.0, sqrt_gR=0.04, rho_l=1.0, rho_ratio=1000.0,
                         mu_ratio=100.0):
    """Gravity, surface tension and viscosities for a rising bubble from Eo and Mo.

    Eo = rho_L g R^2 / sigma and Ga = sqrt(g R) R / nu_L (Section "Rising bubble"); the Morton
    number is read as Mo = Eo^3 / Ga^4 = g mu_L^4 / (rho_L sigma^3).  The velocity scale
    sqrt(g R) is chosen, which fixes g."""
    g = sqrt_gR ** 2 / R
    sigma = g * rho_l * R * R / Eo
    Ga = (Eo ** 3 / Mo) ** 0.25
    nu_l = sqrt_gR * R / Ga
    mu_l = rho_l * nu_l
    return dict(g=g, sigma=sigma, Ga=Ga, nu_l=nu_l, mu_l=mu_l, mu_g=mu_l / mu_ratio,
                rho_g=rho_l / rho_ratio)


def rising_bubble(nx=128, ny=128, nz=256, R=16.0, zc=40.0, Eo=10.0, Mo=1e-4, rho_ratio=1000.0,
                  mu_ratio=100.0, width=4.0, mobility=0.25, sqrt_gR=0.02):
    """Rising bubble: walls on z, periodic x, y; gas bubble of radius R at (nx/2, ny/2, zc);
    density ratio 1000, viscosity ratio 100; gravity from Eo and Mo; buoyancy acts on the
    light phase only (rho_ref = rho_L).

    The velocity scale sqrt(gR) and the mobility D are not fixed by Eo, Mo and the ratios.  At
    W = 4 and density ratio 1000 the coupled step stays bounded over 20k steps for
    sqrt(gR) <= 0.025 with D in [0.2, 0.3], and diverges for sqrt(gR) >= 0.03 or D = 0.1; the
    defaults sqrt(gR) = 0.02, D = 0.25 sit inside that range (tau_L = 0.517, tau_G = 0.671)."""
    p = rising_bubble_params(Eo=Eo, Mo=Mo, R=R, sqrt_gR=sqrt_gR, rho_ratio=rho_ratio, mu_ratio=mu_ratio)
    return Workload(name=f"rising_bubble_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, wall_z=1,
                    rho_l=1.0, rho_g=p["rho_g"], mu_l=p["mu_l"], mu_g=p["mu_g"], sigma=p["sigma"],
                    width=width, mobility=mobility, gravity=(0.0, 0.0, -p["g"]), rho_ref=1.0,
                    body=(0.0, 0.0, 0.0), kind="bubble", center=(nx / 2.0, ny / 2.0, zc),
                    radius=R)


def droplet_ensemble(n=256, seed=2501, L_min=32, L_max=96, v_max=0.02):
    """Ensemble of independent static-droplet boxes with seeded, uneven sizes and properties.

    Box b: periodic cube of side L ~ U{L_min .. L_max}; droplet radius R ~ U[6, L/4] at the centre;
    sigma ~ U[0.001, 0.02]; density ratio rho_L/rho_G log-uniform in [10, 1000] (rho_L = 1); equal
    kinematic viscosity nu = 0.1 in both phases (tau = 0.8; the dynamic viscosity ratio equals the
    density ratio); W = 4, D = 0.1; a seeded Fourier velocity field of amplitude ~ U[0, v_max].
    Every draw comes from numpy default_rng(seed), in box order.  L_min >= 24 (R >= 6 needs
    L/4 >= 6)."""
    if L_min < 24 or L_max < L_min:
        raise ValueError("droplet_ensemble needs 24 <= L_min <= L_max")
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        L = int(rng.integers(L_min, L_max + 1))
        R = float(rng.uniform(6.0, L / 4.0))
        sigma = float(rng.uniform(0.001, 0.02))
        ratio = float(np.exp(rng.uniform(np.log(10.0), np.log(1000.0))))
        amp = float(rng.uniform(0.0, v_max))
        rho_g = 1.0 / ratio
        c = (L - 1) / 2.0
        out.append(Workload(name=f"ensemble_droplet_{b}_{L}^3", nx=L, ny=L, nz=L, wall_z=0,
                            rho_l=1.0, rho_g=rho_g, mu_l=0.1, mu_g=0.1 * rho_g, sigma=sigma, width=4.0,
                            mobility=0.1, gravity=(0.0, 0.0, 0.0), rho_ref=1.0, body=(0.0, 0.0, 0.0),
                            kind="droplet", center=(c, c, c), radius=R, noise=amp, seed=seed * 1000 + b))
    return out


@dataclasses.dataclass
class Collision:
    """Head-on binary droplet collision in a periodic cube: two drops of radius R on the z axis,
    their surfaces a gap apart, approaching each other at relative speed `speed` (each drop moves
    at speed/2 towards the other), with an optional lateral offset b of the drop centres along x
    and a seeded Fourier velocity noise.  Density ratio rho_L/rho_G, equal kinematic viscosity nu in
    both phases, surface tension sigma, interface width W, mobility D."""
    L: int = 128
    R: float = 20.0
    speed: float = 0.05
    ratio: float = 100.0
    gap: float = 12.0
    offset: float = 0.0
    nu: float = 0.04
    sigma: float = 0.005
    width: float = 4.0
    mobility: float = 0.1
    noise: float = 0.0
    seed: int = 0
    name: str = "collision"
    profile_width: float = None   # width of the initial tanh profiles (default: width)

    @property
    def nx(self):
        return self.L

    ny = nx
    nz = nx

    @property
    def n(self):
        return self.L ** 3

    def _centres(self):
        c = (self.L - 1) / 2.0
        d = 2.0 * self.R + self.gap
        return ((c + self.offset / 2, c, c - d / 2), (c - self.offset / 2, c, c + d / 2))

    def _drops(self):
        c1, c2 = self._centres()
        w = self.width if self.profile_width is None else self.profile_width
        return (sphere_phi(self.L, self.L, self.L, c1, self.R, w),
                sphere_phi(self.L, self.L, self.L, c2, self.R, w))

    def fields(self):
        """(phi0, u0, p*0) in one pass: phi = the two drop profiles (capped at 1), u = +-speed/2
        along z inside each drop plus the noise, p* = 3 p / rho(phi) with the Laplace jump
        2 sigma / R inside each drop."""
        p1, p2 = self._drops()
        phi = np.minimum(p1 + p2, 1.0)
        u = np.zeros((3, self.L, self.L, self.L))
        u[2] = 0.5 * self.speed * (p1 - p2)
        if self.noise > 0.0:
            u += fourier_velocity(self.L, self.L, self.L, amplitude=self.noise, seed=self.seed)
        rho = phi * 1.0 + (1.0 - phi) / self.ratio
        return phi, u, 3.0 * (2.0 * self.sigma / self.R) * (p1 + p2) / rho

    def phi0(self):
        return self.fields()[0]

    def u0(self):
        return self.fields()[1]

    def pstar_init(self):
        return self.fields()[2]

    def params(self) -> dict:
        rho_g = 1.0 / self.ratio
        return dict(nx=self.L, ny=self.L, nz=self.L, wall_z=0, rho_l=1.0, rho_g=rho_g, mu_l=self.nu,
                    mu_g=self.nu * rho_g, sigma=self.sigma, width=self.width, mobility=self.mobility,
                    gravity=(0.0, 0.0, 0.0), rho_ref=1.0, body=(0.0, 0.0, 0.0))

    def coarse_params(self) -> dict:
        """Parameters of the same flow on a 2x coarser grid in acoustic scaling (dx and dt doubled,
        lattice velocities unchanged): nu, sigma and D halve in lattice units; the interface keeps
        W lattice units (so it is twice as wide physically)."""
        p = self.params()
        p.update(nx=self.L // 2, ny=self.L // 2, nz=self.L // 2, mu_l=p["mu_l"] / 2, mu_g=p["mu_g"] / 2,
                 sigma=p["sigma"] / 2, mobility=p["mobility"] / 2)
        return p


def rescaled_collision(col: Collision, L: int) -> Collision:
    """The same physical collision on an L^3 grid in acoustic scaling (lattice velocities kept,
    dx and dt scaled by f = col.L / L): lengths (R, gap, offset, the initial profile's width)
    scale by 1/f, nu, sigma and D by 1/f in lattice units; the solver's interface width stays
    col.width lattice units, as on every grid.  The seeded Fourier noise has the same physical
    modes at every L."""
    f = col.L / L
    pw = col.width if col.profile_width is None else col.profile_width
    return dataclasses.replace(col, L=L, R=col.R / f, gap=col.gap / f, offset=col.offset / f, nu=col.nu / f,
                               sigma=col.sigma / f, mobility=col.mobility / f, profile_width=pw / f,
                               name=f"{col.name}_at_{L}")


def collision_set(n=200, seed=7, L=128, R=20.0):
    """Seeded head-on collisions: gap ~ U[6, 18], lateral offset ~ U[-1, 1] (nodes), speed
    0.05 * U[0.9, 1.1], Fourier velocity noise of amplitude 0.001."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        out.append(Collision(L=L, R=R, speed=0.05 * float(rng.uniform(0.9, 1.1)), gap=float(rng.uniform(6.0, 18.0)),
                             offset=float(rng.uniform(-1.0, 1.0)), noise=0.001, seed=seed * 10000 + k,
                             name=f"collision_{k}"))
    return out
