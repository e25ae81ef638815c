"""Register-spill budget of the hot-path kernels (CPU only: nvcc cross-compiles sm_103a).

Compiles the translation units of the propagation paths with the library's own flags plus
`-Xptxas -v` and checks, per kernel, the spill stores ptxas reports against a budget: zero
for the kernels that do not spill today, and today's figure for the few that do (their
measured speed includes it).  A change that makes a hot kernel spill more fails here,
before any GPU time is spent on it."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_05635_gb300", "csrc")

UNITS = ["lr_persistent", "ch_persistent", "batched", "batched_tc", "adjoint", "kernels_step",
         "hhg", "channel"]

# fragment of the mangled kernel name -> largest allowed spill stores (bytes)
BUDGET = {
    "lr_persistent_kernelILi2E": 0, "lr_persistent_kernelILi4E": 0,
    "ch_persistent_kernelILi2E": 16, "ch_persistent_kernelILi4E": 4,
    "batched_kernelILi2ELb0E": 0, "batched_kernelILi2ELb1E": 52,
    "batched_kernelILi4ELb0E": 100, "batched_kernelILi4ELb1E": 72,
    "batched_tc_kernelILi2ELb0E": 96, "batched_tc_kernelILi4ELb0E": 424,
    "batched_tc_kernelILi2ELb1E": 16, "batched_tc_kernelILi4ELb1E": 392,
    "adjoint_kernelILi2E": 0, "adjoint_kernelILi4E": 780,
    "stage_kernelIfLi2E": 0, "stage_kernelIfLi4E": 0,
    "gemv_kernelIfLi4ELi256E": 0, "vcols_kernelIfE": 0, "yreduce_kernelIfE": 0,
    "observables_kernelIfLi4E": 0, "hhg_kernel": 0,
    "ch_vpass_kernelIfE": 0, "ch_upass_kernelIfE": 0,
}


def _ptxas_report(unit: str, out_dir: str) -> str:
    from paper_2502_05635_gb300 import build as b
    cmd = ([b.nvcc()] + b.ARCH + b.FLAGS + ["-Xptxas", "-v", "-x", "cu", "-c",
           os.path.join(CSRC, unit + ".cu"), "-o", os.path.join(out_dir, unit + ".o")])
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout + r.stderr


def _spills(report: str) -> dict:
    out, cur = {}, None
    for line in report.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and cur:
            out[cur] = int(m.group(1))
            cur = None
    return out


def test_hot_kernels_stay_within_their_spill_budget():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
            reports = list(ex.map(lambda u: _ptxas_report(u, tmp), UNITS))
    spills = {}
    for rep in reports:
        spills.update(_spills(rep))
    for frag, limit in BUDGET.items():
        hits = {k: v for k, v in spills.items() if frag in k}
        assert hits, f"kernel {frag} not found in the ptxas report"
        for name, v in hits.items():
            assert v <= limit, f"{frag}: {v} bytes of spill stores (budget {limit})"
