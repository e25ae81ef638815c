"""Seeded synthetic workloads shared by the tests, the bench and the oracle runs.

This module holds *inputs only*: model parameters, grid sizes, time steps, ranks and
the seeded draw of per-trajectory pulse parameters.  It contains none of the method's
arithmetic (no Hamiltonian, kernel, field formula or propagation), so that the CPU
oracle and the CUDA path can both take their inputs from here without sharing code.

Workloads (all atomic units; tight-binding stand-ins for the paper's first-principles
kernels, which are not available):

  tiny_nb2_l12   two-band model, 12x12 k-grid (Nk=144, Nb=2, N=576), one trajectory,
                 2000 RK4 steps of dt=0.2, Gaussian*cos pulse E0=1e-3, w=0.1, t0=200,
                 sigma=60.  The parity workload; the paper's MoS2 runs use the same
                 narrow-pulse linear-response setup (Sec. "SVD acceleration of TD-aGW").
  mos2size_nb4_l36_channel
                 the same model with channel-wise factors: dense diagonal channels,
                 off-diagonal channels truncated to rank 65 (5 % of Nk).
  mos2size_nb4_l36
                 four-band model (two copies, energy offsets 0 and 0.03 Ha), 36x36 grid
                 (Nk=1296, N=20736 -- the size of the paper's 2v+2c, 36x36 MoS2 kernel,
                 Appendix A), one trajectory, 10000 steps, truncation rank 1024 (~5%,
                 the rank the paper finds sufficient for linear absorption).
  angle_nb4_l36  the mos2-size model driven along 60 directions (1 .. 60 degrees), strong
                 sin^2 pulse, 2000 steps each, rank 1024: the angle-resolved HHG sweep.
  sweep_nb2_l24  two-band, 24x24 grid (N=2304), rank 256, 256 trajectories with seeded
                 pulse parameters and uneven lengths 500..4000 steps (field sweep).
  prec_nb4_l48   four-band, 48x48 grid (N=36864), rank 2048, 64 trajectories, 5000 steps.
  adj_nb2_l36    two-band, 36x36 grid (N=5184), rank 512, 32 trajectories, 20000 steps.

Seeded trajectory parameters: numpy default_rng(20250208); E0 = 10**U(-4,-2),
omega ~ U(0.06, 0.16), sigma ~ U(30, 120), t0 = 200, steps ~ integers U[500, 4000].
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
import numpy as np

TRAJ_SEED = 20250208
SKETCH_SEED = 1


@dataclass(frozen=True)
class ModelParams:
    L: int = 12                 # k-grid is L x L
    nb_copies: int = 1          # copies of the two-band model; Nb = 2 * nb_copies
    offsets: tuple = (0.0, 0.0, 0.0, 0.0)   # energy offset of each copy (Ha)
    Delta: float = 0.08
    t: float = 0.05
    m: float = 0.1
    a: float = 6.0              # lattice constant (bohr)
    r0: float = 20.0            # Rytova-Keldysh screening length (bohr)
    exchange: float = 0.0       # scale of the exchange term (0: direct kernel only)

    @property
    def Nb(self) -> int:
        return 2 * self.nb_copies

    @property
    def Nk(self) -> int:
        return self.L * self.L

    @property
    def N(self) -> int:
        return self.Nb * self.Nb * self.Nk


@dataclass(frozen=True)
class Pulse:
    """Pulse parameters.  kind: 0 Gaussian*cos, 1 constant, 2 sin^2 envelope * sin."""
    E0: float = 1e-3
    omega: float = 0.1
    t0: float = 200.0
    sigma: float = 60.0
    T_pulse: float = 0.0
    dir_x: float = 1.0
    dir_y: float = 0.0
    kind: int = 0


@dataclass(frozen=True)
class Workload:
    name: str
    model: ModelParams
    dt: float
    steps: tuple            # per-trajectory step counts
    pulses: tuple           # per-trajectory Pulse
    rank: int = 0
    oversample: int = 64
    power_iters: int = 2

    @property
    def B(self) -> int:
        return len(self.steps)


def draw_pulses(B: int, seed: int = TRAJ_SEED, uneven: bool = True,
                fixed_steps: int | None = None):
    """Seeded per-trajectory pulse parameters and lengths (field-sweep distributions)."""
    rng = np.random.default_rng(seed)
    E0 = 10.0 ** rng.uniform(-4.0, -2.0, size=B)
    omega = rng.uniform(0.06, 0.16, size=B)
    sigma = rng.uniform(30.0, 120.0, size=B)
    steps = rng.integers(500, 4001, size=B)
    if fixed_steps is not None:
        steps = np.full(B, fixed_steps)
    pulses = tuple(Pulse(E0=float(E0[b]), omega=float(omega[b]), t0=200.0,
                         sigma=float(sigma[b]), kind=0) for b in range(B))
    return pulses, tuple(int(s) for s in steps)


def tiny_nb2_l12(steps: int = 2000) -> Workload:
    return Workload("tiny_nb2_l12", ModelParams(L=12), 0.2, (steps,), (Pulse(),))


def mos2size_nb4_l36(steps: int = 10000) -> Workload:
    mp = ModelParams(L=36, nb_copies=2, offsets=(0.0, 0.03, 0.0, 0.0))
    return Workload("mos2size_nb4_l36", mp, 0.2, (steps,), (Pulse(),), rank=1024)


def early_pulses(B: int, seed: int = TRAJ_SEED):
    """Seeded Gaussian*cos pulses that peak within the first 12 time units (t0 = 6,
    sigma 1.5-3), amplitudes 1e-4 .. 1e-2 (log-uniform), frequencies 0.06-0.16 and field
    directions spread over the plane: short runs that still see the whole pulse, for
    comparing kernel forms over a few dozen steps."""
    rng = np.random.default_rng(seed + 7)
    E0 = 10.0 ** rng.uniform(-4.0, -2.0, size=B)
    omega = rng.uniform(0.06, 0.16, size=B)
    sigma = rng.uniform(1.5, 3.0, size=B)
    ang = rng.uniform(0.0, np.pi, size=B)
    return tuple(Pulse(E0=float(E0[b]), omega=float(omega[b]), t0=6.0, sigma=float(sigma[b]),
                       dir_x=float(np.cos(ang[b])), dir_y=float(np.sin(ang[b])), kind=0) for b in range(B))


def mos2size_channel(steps: int = 10000) -> Workload:
    """The mos2-size model with the channel-wise compression: dense diagonal channels and
    every off-diagonal channel truncated to 5 % of Nk (65 of 1296 singular values), the
    "K_0^diag-ch + 5 % K_0^off-ch" kernel of the paper's TDA spectra."""
    mp = ModelParams(L=36, nb_copies=2, offsets=(0.0, 0.03, 0.0, 0.0))
    return Workload("mos2size_nb4_l36_channel", mp, 0.2, (steps,), (Pulse(),), rank=65)


def angle_nb4_l36(B: int = 60, steps: int = 2000) -> Workload:
    """Angle-resolved HHG sweep (Appendix C) at the mos2 size: B field directions evenly
    spaced over 1 .. 60 degrees, strong sin^2-envelope pulse (E0 5e-3, omega 0.1, the whole
    run long), rank 1024."""
    mp = ModelParams(L=36, nb_copies=2, offsets=(0.0, 0.03, 0.0, 0.0))
    th = np.deg2rad(np.linspace(1.0, 60.0, B))
    pulses = tuple(Pulse(E0=5e-3, omega=0.1, T_pulse=steps * 0.2, dir_x=float(np.cos(a)),
                         dir_y=float(np.sin(a)), kind=2) for a in th)
    return Workload("angle_nb4_l36", mp, 0.2, (steps,) * B, pulses, rank=1024)


def sweep_nb2_l24(B: int = 256) -> Workload:
    pulses, steps = draw_pulses(B)
    return Workload("sweep_nb2_l24", ModelParams(L=24), 0.2, steps, pulses, rank=256)


def prec_nb4_l48(B: int = 64, steps: int = 5000) -> Workload:
    pulses, _ = draw_pulses(B)
    mp = ModelParams(L=48, nb_copies=2, offsets=(0.0, 0.03, 0.0, 0.0))
    return Workload("prec_nb4_l48", mp, 0.2, (steps,) * B, pulses, rank=2048)


def adj_nb2_l36(B: int = 32, steps: int = 20000) -> Workload:
    pulses, _ = draw_pulses(B)
    return Workload("adj_nb2_l36", ModelParams(L=36), 0.2, (steps,) * B, pulses, rank=512)


def small_model(L: int, nb_copies: int = 1) -> ModelParams:
    """Reduced grids for parity tests (same model family, fewer k-points)."""
    offs = (0.0, 0.03, 0.0, 0.0) if nb_copies == 2 else (0.0, 0.0, 0.0, 0.0)
    return ModelParams(L=L, nb_copies=nb_copies, offsets=offs)


def random_state(N: int, seed: int, scale: float = 1e-2) -> np.ndarray:
    """Seeded complex test vector (not a physical density matrix)."""
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(N) + 1j * rng.standard_normal(N))


def gaussian_sketch(N: int, cols: int, seed: int = SKETCH_SEED) -> np.ndarray:
    """Seeded complex Gaussian test matrix (N x cols), unit variance per entry."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((N, cols)) + 1j * rng.standard_normal((N, cols))) / np.sqrt(2.0)


def random_factors(N: int, r: int, seed: int, s0: float = 0.05, decay: float = 3.0):
    """Seeded synthetic low-rank factors (U, S, V, diag) of kernel-like magnitude:
    Gaussian columns of norm ~1, S decaying geometrically from s0 by `decay` e-folds,
    diag constant.  Inputs for parity runs of the low-rank apply; not a decomposition."""
    rng = np.random.default_rng(seed)
    U = (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) / np.sqrt(2 * N)
    V = (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) / np.sqrt(2 * N)
    S = s0 * np.exp(-decay * np.arange(r) / max(r, 1))
    diag = np.full(N, -0.0134 + 0.0j)
    return U, S, V, diag


def as_dict(w: Workload) -> dict:
    d = asdict(w)
    d["N"] = w.model.N
    return d
