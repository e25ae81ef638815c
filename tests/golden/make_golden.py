"""Writes tests/golden/oracle_tiny_nb2_l12.txt from the FP64 oracle alone (no CUDA path).

The paper prints no values for the synthetic lattice model, so this file is a regression
fixture of the oracle, not a pin: tests/test_golden.py recomputes every value and fails on
any drift, so that a change to the oracle's arithmetic has to be made on purpose (and the
fixture rewritten with this script, the commit naming the passage that justifies it).

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import channel as oc  # noqa: E402
from oracle import hhg as oh  # noqa: E402
from oracle import kernel as ok  # noqa: E402
from oracle import lowrank as olr  # noqa: E402
from oracle import model as om  # noqa: E402
from oracle import propagate as op  # noqa: E402

OUT = os.path.join(HERE, "oracle_tiny_nb2_l12.txt")
STEPS = 400
EVERY = 40
ENTRIES = [(0, 0), (0, 1), (5, 9), (17, 300), (123, 456), (575, 2), (288, 289), (401, 401)]


def compute() -> dict:
    """Every fixture value, keyed by its line label."""
    w = wl.tiny_nb2_l12(steps=STEPS)
    mdl = om.Model(w.model)
    K = ok.dense_kernel(mdl)
    s = op.half_step_samples(w.pulses[0], w.dt, STEPS)
    out = {}
    # Appendix B: W(q = 0) as the mini-cell average; Eq. bse-direct-def entries
    p = w.model
    out["W0"] = [float(ok.cell_average_W0(np.pi / (p.L * p.a), p.Nk * p.a * p.a, p.r0))]
    out["K_entries"] = [v for r, c in ENTRIES for v in (K[r, c].real, K[r, c].imag)]
    # Eq. tdagw with the dense kernel (Eq. sigma-from-k)
    obs, _ = op.rk4(mdl, lambda v: K @ v, s, w.dt, STEPS)
    for z, name in enumerate(("P_full", "J_full", "occ_full")):
        out[name] = list(obs[::EVERY, z])
    # Eq. svd_acc at rank 29 (exact truncated SVD of K^off, Eq. svd_diag_offdiag)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, 29)
    obs_lr, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, w.dt, STEPS)
    out["P_lowrank29"] = list(obs_lr[::EVERY, 0])
    # Eq. svd-channel-wise: dense diagonal channels, off-diagonal channels at rank 9
    D, Uc, Sc, Vc = oc.channel_svd(K, mdl.Nb, 9)
    obs_ch, _ = op.rk4(mdl, lambda v: oc.apply_channel(D, Uc, Sc, Vc, v), s, w.dt, STEPS)
    out["P_channel9"] = list(obs_ch[::EVERY, 0])
    # HHG(w) of the dense run's current (Sec. "SVD acceleration of TD-aGW")
    omega = oh.harmonic_grid(w.pulses[0].omega, 8.0, 8)
    out["HHG_full"] = list(oh.hhg_spectrum(obs[:, 1], w.dt, omega))
    return out


def write(values: dict, path: str = OUT):
    lines = [
        "# FP64 oracle values for tiny_nb2_l12 (two-band 12 x 12 model, N = 576, dt = 0.2,",
        f"# Gaussian * cos pulse E0 1e-3, w 0.1, t0 200, sigma 60), {STEPS} RK4 steps, every {EVERY}th",
        "# step.  Written by tests/golden/make_golden.py from oracle/ only; a regression fixture",
        "# (the paper prints no values for this model).  Lines: label then values (%.17g).",
        "# W0: Appendix B average; K_entries: Eq. bse-direct-def at (row, col) = "
        + " ".join(f"({r},{c})" for r, c in ENTRIES) + " as re im pairs;",
        "# P/J/occ_full: Eq. tdagw with the dense kernel; P_lowrank29: Eq. svd_acc, rank 29;",
        "# P_channel9: Eq. svd-channel-wise, off-diagonal rank 9; HHG_full: HHG(w) of J_full at",
        "# 8 frequencies up to the 8th harmonic.",
    ]
    for k, v in values.items():
        lines.append(k + " " + " ".join(f"{float(x):.17g}" for x in v))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def read(path: str = OUT) -> dict:
    vals = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        vals[k] = [float(x) for x in v]
    return vals


if __name__ == "__main__":
    write(compute())
    print("wrote", OUT)
