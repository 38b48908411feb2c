"""Seeded synthetic inputs for the discrete-DtN Schroedinger time-stepper.

This module holds workload descriptions and random input generators only.
It contains none of the method's arithmetic (no Hamiltonian, no DtN map, no
integrator), so that both the CUDA path and the CPU oracle can draw the same
inputs from it without sharing any computation.

Grid convention (a reading; the paper gives only box extents, Sec. 4.2 and
Sec. 4.3): an interior axis of N nodes with spacing h has node coordinates
x_i = (i - (N-1)/2) * h, i = 0..N-1.  Arrays are laid out as
[orbital][z][y][x] with x fastest.

Workloads (sizes, spacing, step counts) follow the five configurations the
project is measured on; all inputs are synthetic and seeded with
``20190806 + workload number``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

SEED_BASE = 20190806


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: grid, ABC order, integrator and potential recipe."""

    number: int
    name: str
    n: int                      # interior nodes per axis (cube)
    h: float                    # grid spacing
    n_orb: int                  # orbitals (batch b)
    order: int                  # 0 or 1 (rational order of the ABC)
    s: float                    # interpolation point s0 (order 0) or s1 (order 1)
    dt: float
    steps: int
    potential: str              # "zero" | "harmonic_bumps" | "smooth_random" | "none"
    meanfield: Optional[Tuple[float, float, float]] = None   # (a, b, alpha)
    precision: str = "c64"      # "fp64" | "c64" | "tf32x3"
    points: Tuple[float, ...] = ()   # order 2: the four interpolation points
    fit1: str = "limit"         # order 1: "limit" | "two_point" | "hermite"
    s1b: float = 0.0            # order 1, two-point fit: the second point
    radius: int = 1             # stencil radius per axis (1, or 3: Sec. 4.2's 7-point scheme)

    @property
    def interp(self):
        """The interpolation argument of the context: s, or the four order-2 points."""
        return self.points if self.order == 2 else self.s

    @property
    def seed(self) -> int:
        return SEED_BASE + self.number

    @property
    def shape(self) -> Tuple[int, int, int]:
        return (self.n, self.n, self.n)


WORKLOADS = {
    1: Workload(1, "free-16cube-order0-fp64", 16, 0.5, 1, 0, 1.0, 0.01, 300, "zero",
                precision="fp64"),
    2: Workload(2, "harmonic-64cube-order1-single", 64, 0.4, 1, 1, 1.0, 0.005, 2000,
                "harmonic_bumps", precision="c64"),
    3: Workload(3, "meanfield-64cube-32orb-order1", 64, 0.4, 32, 1, 1.0, 0.005, 1000,
                "none", meanfield=(-1.0, 0.8, 1.0 / 6.0), precision="fp16x3"),
    4: Workload(4, "adjoint-48cube-order1", 48, 0.4, 1, 1, 1.0, 0.005, 1000,
                "smooth_random", precision="c64"),
    5: Workload(5, "meanfield-96cube-128orb-order1", 96, 0.35, 128, 1, 1.0, 0.004, 500,
                "none", meanfield=(-1.0, 0.8, 1.0 / 6.0), precision="fp16x3"),
    # the next-row variants on the benchmark grid and potential
    6: Workload(6, "harmonic-64cube-order2-single", 64, 0.4, 1, 2, 1.0, 0.005, 500,
                "harmonic_bumps", precision="c64", points=(1.0, 2.0, 3.0, 10.0)),
    7: Workload(7, "harmonic-64cube-order1-twopoint-single", 64, 0.4, 1, 1, 1.0, 0.005, 500,
                "harmonic_bumps", precision="c64", fit1="two_point", s1b=2.0),
    8: Workload(8, "harmonic-64cube-order1-hermite-single", 64, 0.4, 1, 1, 1.0, 0.005, 500,
                "harmonic_bumps", precision="c64", fit1="hermite"),
    # Sec. 4.2's 3D experiment: box [-1.5, 1.5]^3 at h = 0.1 (31^3, 7-point scheme per axis,
    # n_Gamma = 14166), free packet exp(-|x|^2 + 5 i x1) (eq:15 at t = 0), dt = 0.001,
    # first order fitted at s = 1, 2
    9: Workload(9, "paper-free-31cube-r3-order1-twopoint", 31, 0.1, 1, 1, 1.0, 0.001, 600,
                "zero", precision="c64", fit1="two_point", s1b=2.0, radius=3),
    # the same experiment with the second order at s = 1, 2, 3, 10 (FP64: the fit at
    # radius 3 needs it)
    10: Workload(10, "paper-free-31cube-r3-order2", 31, 0.1, 1, 2, 1.0, 0.001, 600,
                 "zero", precision="fp64", points=(1.0, 2.0, 3.0, 10.0), radius=3),
}


def axis_coords(n: int, h: float) -> np.ndarray:
    """Node coordinates of one axis, centred on the box."""
    return (np.arange(n, dtype=np.float64) - 0.5 * (n - 1)) * h


def mesh(shape: Tuple[int, int, int], h: float):
    """Return (X, Y, Z) arrays of shape (Nz, Ny, Nx)."""
    nx, ny, nz = shape
    z = axis_coords(nz, h)[:, None, None]
    y = axis_coords(ny, h)[None, :, None]
    x = axis_coords(nx, h)[None, None, :]
    return np.broadcast_arrays(x, y, z)


def _normalize(psi: np.ndarray, h: float) -> np.ndarray:
    nrm = math.sqrt(float(np.sum(np.abs(psi) ** 2)) * h ** 3)
    return psi / nrm


def gaussian_packet(shape, h, center, k, width, phase=0.0) -> np.ndarray:
    """exp(-|x-c|^2/w^2 + i k.(x-c) + i*phase), h^3-normalised (complex128)."""
    X, Y, Z = mesh(shape, h)
    dx, dy, dz = X - center[0], Y - center[1], Z - center[2]
    r2 = dx * dx + dy * dy + dz * dz
    arg = -r2 / (width * width) + 1j * (k[0] * dx + k[1] * dy + k[2] * dz) + 1j * phase
    return _normalize(np.exp(arg), h)


def _unit_vector(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def harmonic_bumps(shape, h, rng, omega=0.3, n_bumps=8) -> np.ndarray:
    """0.5*omega^2*r^2 plus seeded Gaussian bumps (amplitude in [-0.5, 0.5])."""
    X, Y, Z = mesh(shape, h)
    half = 0.5 * (np.array(shape) - 1) * h
    V = 0.5 * omega * omega * (X * X + Y * Y + Z * Z)
    for _ in range(n_bumps):
        amp = rng.uniform(-0.5, 0.5)
        wid = rng.uniform(1.0, 2.0)
        c = rng.uniform(-0.6, 0.6, size=3) * half
        V = V + amp * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (wid * wid))
    return V


def smooth_random(shape, h, rng, n_gauss=6, vmax=0.3) -> np.ndarray:
    """Sum of seeded Gaussians rescaled so that max|V| = vmax."""
    X, Y, Z = mesh(shape, h)
    half = 0.5 * (np.array(shape) - 1) * h
    V = np.zeros_like(X)
    for _ in range(n_gauss):
        amp = rng.uniform(-1.0, 1.0)
        wid = rng.uniform(1.0, 3.0)
        c = rng.uniform(-0.6, 0.6, size=3) * half
        V = V + amp * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (wid * wid))
    return V * (vmax / np.max(np.abs(V)))


def orbital_set(shape, h, rng, n_orb) -> np.ndarray:
    """Gaussian-modulated plane waves, Gram-Schmidt orthonormalised (h^3 product)."""
    X, Y, Z = mesh(shape, h)
    half = 0.5 * (np.array(shape) - 1) * h
    out = np.empty((n_orb,) + X.shape, dtype=np.complex128)
    for j in range(n_orb):
        c = rng.uniform(-0.5, 0.5, size=3) * half
        w = rng.uniform(1.5, 3.0)
        k = _unit_vector(rng) * rng.uniform(0.0, 1.0)
        r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        out[j] = np.exp(-r2 / (w * w) + 1j * (k[0] * X + k[1] * Y + k[2] * Z))
    for j in range(n_orb):
        v = out[j]
        for i in range(j):
            v = v - out[i] * (np.vdot(out[i], v) * h ** 3)
        out[j] = _normalize(v, h)
    return out


def make_inputs(w: Workload, n: Optional[int] = None, n_orb: Optional[int] = None):
    """Seeded (psi0 [b,Nz,Ny,Nx] complex128, V_ext [Nz,Ny,Nx] float64) for a workload.

    ``n`` and ``n_orb`` shrink the grid / batch for small test cases while keeping
    the workload's recipe (positions scale with the box)."""
    n = w.n if n is None else n
    b = w.n_orb if n_orb is None else n_orb
    shape = (n, n, n)
    rng = np.random.default_rng(w.seed)
    half = 0.5 * (n - 1) * w.h
    if w.potential == "zero" or w.potential == "none":
        V = np.zeros((n, n, n))
    elif w.potential == "harmonic_bumps":
        V = harmonic_bumps(shape, w.h, rng)
    elif w.potential == "smooth_random":
        V = smooth_random(shape, w.h, rng)
    else:
        raise ValueError(w.potential)
    if w.number in (9, 10):
        # the paper's packet: eq:15 at t = 0 with k0 = 5 (sigma^2 = 1/2, centre 0)
        psi = gaussian_packet(shape, w.h, (0.0, 0.0, 0.0), (5.0, 0.0, 0.0), 1.0)[None]
    elif w.number == 1:
        theta = rng.uniform(0.0, 2.0 * math.pi)
        # centre offset 2 at the 16^3, h=0.5 box (half-width 3.75), scaled with the box
        xc = (-2.0 * half / 3.75, 0.0, 0.0)
        psi = gaussian_packet(shape, w.h, xc, (1.5, 0.0, 0.0), 1.5, theta)[None]
    elif w.meanfield is not None:
        psi = orbital_set(shape, w.h, rng, b)
    else:
        theta = rng.uniform(0.0, 2.0 * math.pi)
        k = 2.0 * _unit_vector(rng)
        psi = gaussian_packet(shape, w.h, (0.0, 0.0, 0.0), k, 1.5, theta)[None]
        if b > 1:
            psi = np.concatenate([psi] + [
                gaussian_packet(shape, w.h, rng.uniform(-0.3, 0.3, 3) * half,
                                2.0 * _unit_vector(rng), 1.5, rng.uniform(0, 2 * math.pi))[None]
                for _ in range(b - 1)])
    return np.ascontiguousarray(psi), np.ascontiguousarray(V)


def random_state(shape, n_orb, rng) -> np.ndarray:
    """Unstructured complex test state (for operator-level parity cases)."""
    nx, ny, nz = shape
    return (rng.normal(size=(n_orb, nz, ny, nx)) + 1j * rng.normal(size=(n_orb, nz, ny, nx)))
