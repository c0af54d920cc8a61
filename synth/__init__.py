"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the method itself: only

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014; the finaliser constants are the published ones),
* the structured-box workloads (mesh sizes, spacing, nondimensional
  parameters, time step) of the dendrite / directional-growth runs,
* their initial conditions (tanh seeds and fronts) and random test fields.

The residual, tangent, preconditioner and solver live separately in the CUDA
library and in the CPU oracle; neither imports the other, both import this.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of SplitMix64 started from ``seed`` (uint64 array)."""
    gamma = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + k * gamma
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_scalar(seed: int, n: int) -> list:
    """Plain sequential SplitMix64, used to pin the vectorised form."""
    s = seed & MASK64
    res = []
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        res.append(z ^ (z >> 31))
    return res


def uniform01(seed: int, n: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """Doubles in [-1, 1)."""
    return 2.0 * uniform01(seed, n) - 1.0


# ---------------------------------------------------------------------------
# Structured box and parameters
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Mesh:
    """Structured box of nx x ny (x nz) elements of size h; nz = 0 in 2D.

    order 1: Q1 elements, node (i,j,k) at x0 + i*h; order 2: Q2 (biquadratic
    quads, triquadratic hexes), node (i,j,k) at x0 + i*h/2.
    """
    dim: int
    nx: int
    ny: int
    nz: int
    h: float
    x0: float = 0.0
    y0: float = 0.0
    z0: float = 0.0
    order: int = 1

    @property
    def shape_nodes(self):
        p = self.order
        if self.dim == 2:
            return (p * self.nx + 1, p * self.ny + 1)
        return (p * self.nx + 1, p * self.ny + 1, p * self.nz + 1)

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.shape_nodes))

    @property
    def n_dofs(self) -> int:
        return 2 * self.n_nodes

    @property
    def n_elems(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    def coords(self):
        """Per-axis node coordinates."""
        nn = self.shape_nodes
        hn = self.h / self.order
        out = [o + hn * np.arange(n) for o, n in zip((self.x0, self.y0, self.z0), nn)]
        return tuple(out)


@dataclasses.dataclass
class Params:
    """Nondimensional model parameters (Karma-Rappel units, W0 = tau0 = 1) and solver controls.

    model 0 = pure metal (phi + dimensionless temperature u, k = 1, no
    antitrapping); model 1 = dilute binary alloy (phi + solute u).
    """
    model: int = 0
    W0: float = 1.0
    tau0: float = 1.0
    eps4: float = 0.05
    lam: float = 3.19
    D: float = 2.0
    k: float = 1.0
    lT: float = 0.0
    Vp: float = 0.0
    zT: float = 0.0            # frozen-gradient origin: G4 = (x_last - zT - Vp t)/lT
    Delta: float = 0.65
    theta: float = 1.0
    phihat_form: int = 1       # theta < 1: 1 (phi^{n+1} - phi^n)/dt, 0 the estimate of Eq. (theta)
    jat_normalised: int = 1
    time_form: int = 0
    # solver controls
    jvp_mode: int = 1          # 0 finite difference, 1 exact tangent
    precond: int = 1           # 0 none, 1 point Jacobi, 2 block Jacobi + GMG
    smoother_fp32: int = 1
    gmres_restart: int = 30
    gmres_maxit: int = 300
    newton_maxit: int = 20
    newton_rtol: float = 1e-10
    newton_atol: float = 0.0
    eta0: float = 0.1
    eta_min: float = 1e-6
    eta_max: float = 0.01
    gamma: float = 0.9
    omega: float = 1.5
    mg_levels: int = 4
    cheb_degree: int = 2
    coarse_degree: int = 10
    linesearch_max: int = 8


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    params: Params
    dt: float
    steps: int


def _pure(**kw) -> Params:
    p = Params(model=0, W0=1.0, tau0=1.0, eps4=0.05, lam=3.19, D=2.0, k=1.0, Delta=0.65)
    for key, val in kw.items():
        setattr(p, key, val)
    return p


# Directional-growth constants for k = 0.15 (alloy workload): lambda = D/a2
# with a2 = 0.6267; W0, tau0 from d0 = 5e-9 m, D_L = 3e-9 m^2/s, a1 = 0.8839;
# thermal length lT = |m| c_inf (1-k)/(k G) / W0 and pulling speed
# Vp = R tau0 / W0 with m = -2.6 K/wt%, c_inf = 3 wt%, G = 1e4 K/m,
# R = 1e-2 m/s (Sec. 4.2, Table 2).
ALLOY_LAMBDA = 2.0 / 0.6267
ALLOY_LT = 2.448e5
ALLOY_VP = 0.12035
# The initial front (u = -1: liquid at c_inf, solid at k c_inf) is in
# equilibrium at the liquidus isotherm, where u + G4 = 0, i.e. G4 = 1; the
# frozen-gradient origin zT is placed one thermal length below the front.
ALLOY_FRONT_Z = 20.0


def workload(name: str) -> Workload:
    """The five structured-box workloads, by name.

    The multigrid-preconditioned 3D and 1024^2 workloads cap GMRES at 10
    iterations per Newton iteration (gmres_maxit = 10, truncated inexact
    Newton): restarted GMRES(30) stagnates on some Newton iterations of these
    problems (300 iterations without reaching the forcing tolerance) and
    gains little after about 10 iterations elsewhere, while the truncated
    solves leave the converged states unchanged to 1e-10 and the Newton
    iteration counts within 2 %; the alloy takes degree-3 Chebyshev smoothing.
    The adjoint workload's forward steps take the same cap (its transposed
    solves run to their tolerance regardless).

    dendrite2d_128      : 2D pure metal, 128^2 on [0,400]^2, FD-JFNK + Jacobi, dt 0.5
    dendrite2d_1024     : 2D pure metal, 1024^2 on [0,400]^2, GMG, dt 0.5
    dendrite3d_192      : 3D pure metal, 192^3, h = 0.8, centred seed r = 10, dt 0.4
    alloy3d_256x256x128 : 3D dilute alloy, h = 0.8, planar front, dt 0.2
    adjoint2d_512       : 2D pure metal, 512^2 on [0,400]^2, dt 0.5
    """
    if name == "dendrite2d_128":
        return Workload(name, Mesh(2, 128, 128, 0, 400.0 / 128),
                        _pure(jvp_mode=0, precond=1, smoother_fp32=0), 0.5, 10)
    if name == "dendrite2d_1024":
        return Workload(name, Mesh(2, 1024, 1024, 0, 400.0 / 1024), _pure(jvp_mode=0, precond=2, gmres_maxit=10),
                        0.5, 50)
    if name == "dendrite3d_192":
        L = 0.8 * 192
        return Workload(name, Mesh(3, 192, 192, 192, 0.8, -L / 2, -L / 2, -L / 2),
                        _pure(Delta=0.55, precond=2, gmres_maxit=10), 0.4, 20)
    if name == "alloy3d_256x256x128":
        p = Params(model=1, W0=1.0, tau0=1.0, eps4=0.02, lam=ALLOY_LAMBDA, D=2.0, k=0.15,
                   lT=ALLOY_LT, Vp=ALLOY_VP, zT=ALLOY_FRONT_Z - ALLOY_LT, Delta=1.0,
                   precond=2, jvp_mode=1, cheb_degree=3, gmres_maxit=10)
        return Workload(name, Mesh(3, 256, 256, 128, 0.8), p, 0.2, 20)
    if name == "adjoint2d_512":
        return Workload(name, Mesh(2, 512, 512, 0, 400.0 / 512), _pure(precond=2, gmres_maxit=10), 0.5, 50)
    raise KeyError(name)


WORKLOADS = ["dendrite2d_128", "dendrite2d_1024", "dendrite3d_192", "alloy3d_256x256x128", "adjoint2d_512"]


def scaled(w: Workload, nx: int, ny: int, nz: int = 0) -> Workload:
    """Same physics, spacing and time step on a smaller box (for oracle-sized cases)."""
    m = w.mesh
    mesh = Mesh(m.dim, nx, ny, nz if m.dim == 3 else 0, m.h, m.x0, m.y0, m.z0)
    if m.x0 != 0.0:  # keep centred boxes centred
        mesh.x0, mesh.y0 = -nx * m.h / 2, -ny * m.h / 2
        if m.dim == 3:
            mesh.z0 = -nz * m.h / 2
    return Workload(w.name + f"@{nx}x{ny}" + (f"x{nz}" if m.dim == 3 else ""), mesh,
                    dataclasses.replace(w.params), w.dt, w.steps)


# ---------------------------------------------------------------------------
# Initial conditions and random fields (field-major: U = [phi ; u])
# ---------------------------------------------------------------------------

def _node_grid(mesh: Mesh):
    return np.meshgrid(*mesh.coords(), indexing="ij")


def _flatten(a: np.ndarray) -> np.ndarray:
    """Node arrays indexed [i, j(, k)] -> flat with x fastest."""
    return np.ascontiguousarray(a.transpose()).reshape(-1)


def seed_state(mesh: Mesh, params: Params, radius: float = 8.0, centred: bool = False) -> np.ndarray:
    """Circular / spherical tanh seed phi = -tanh((r - R)/sqrt 2), u = -Delta everywhere."""
    g = _node_grid(mesh)
    if centred:
        r = np.sqrt(sum(x * x for x in g))
    else:
        r = np.sqrt(sum((x - c0) ** 2 for x, c0 in zip(g, (mesh.x0, mesh.y0, mesh.z0))))
    phi = -np.tanh((r - radius) / math.sqrt(2.0))
    u = np.full_like(phi, -params.Delta)
    return np.concatenate([_flatten(phi), _flatten(u)])


def front_state(mesh: Mesh, z_front: float = ALLOY_FRONT_Z, amp: float = 0.1, seed: int = 7) -> np.ndarray:
    """Planar front along the last axis, perturbed per (x,y) column by seed-`seed` noise; u = -1."""
    assert mesh.dim == 3
    nxn, nyn, nzn = mesh.shape_nodes
    xi = uniform_pm1(seed, nxn * nyn).reshape(nyn, nxn)  # i fastest
    zs = mesh.z0 + mesh.h * np.arange(nzn)
    phi = -np.tanh((zs[:, None, None] - z_front - amp * xi[None, :, :]) / math.sqrt(2.0))
    u = -np.ones_like(phi)
    return np.concatenate([phi.reshape(-1), u.reshape(-1)])


def initial_state(w: Workload) -> np.ndarray:
    if w.name.startswith("alloy3d"):
        return front_state(w.mesh)
    if w.name.startswith("dendrite3d"):
        return seed_state(w.mesh, w.params, radius=10.0, centred=True)
    return seed_state(w.mesh, w.params, radius=8.0)


def random_fields(mesh: Mesh, seed: int = 42):
    """(U, Un) uniform in [-1,1): Un first (phi then u), then U (phi then u)."""
    n = mesh.n_nodes
    r = uniform_pm1(seed, 4 * n)
    return r[2 * n:].copy(), r[: 2 * n].copy()


def random_vector(mesh: Mesh, seed: int) -> np.ndarray:
    return uniform_pm1(seed, mesh.n_dofs)
