"""Register budgets the kernels' occupancy rests on, read from ptxas's report (nvcc -Xptxas -v; no
GPU needed): the blend forward must fit four 256-thread CTAs per SM (<= 64 registers), the blend
backward four 4-warp CTAs (<= 128), the projection backward two 256-thread CTAs (<= 128), the loss
kernels three 256-thread CTAs (<= 85), the key emission 1024-thread CTAs (<= 64); none of the hot
kernels spills more than a few words (the projection backward's 80 bytes and the loss kernels'
4-20 bytes are the measured state)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_13086_gb300", "csrc")

# (source, mangled-name fragment, max registers, max spill-store bytes)
BUDGETS = [
    ("k_blend.cu", "k_blend_forwardILi16ELi16ELi256", 64, 0),
    ("k_blend.cu", "k_blend_backwardILi16ELi16", 128, 0),
    ("k_project.cu", "k_project_backwardILi1", 128, 128),
    ("k_project.cu", "2gs9k_project", 64, 0),
    ("k_loss.cu", "k_loss_forward", 85, 32),   # 80 registers, a few words spilled (measured so)
    ("k_loss.cu", "k_loss_backward", 85, 32),
    ("k_sort.cu", "k_emit", 64, 0),
    ("k_sort.cu", "k_sort_pass", 64, 0),
]


def ptxas_report(src, tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC,
                          "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c", os.path.join(CSRC, src),
                          "-o", str(tmp_path / (src + ".o"))], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr[-2000:]
    # per entry function: its spill line and its register line
    res = {}
    cur = None
    for line in out.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and cur:
            res.setdefault(cur, {})["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            res.setdefault(cur, {})["regs"] = int(m.group(1))
            cur = None
    return res


@pytest.mark.parametrize("src", sorted({b[0] for b in BUDGETS}))
def test_register_budgets(src, tmp_path):
    rep = ptxas_report(src, tmp_path)
    for s, frag, max_regs, max_spill in BUDGETS:
        if s != src:
            continue
        hits = {k: v for k, v in rep.items() if frag in k and "regs" in v}
        assert hits, f"{frag} not found in the ptxas report of {src}"
        for name, v in hits.items():
            assert v["regs"] <= max_regs, (name, v)
            assert v.get("spill", 0) <= max_spill, (name, v)
