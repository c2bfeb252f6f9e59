"""The ncu summaries under profiles/ stay runnable and traceable: every
bench.py command they quote parses with the bench's own options, and each
summary names the hash of the kernel source it was taken on (the bench
reports a kernel's DRAM traffic only while that hash matches)."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(text: str) -> list[str]:
    """Indented command blocks, with backslash continuations joined."""
    cmds, cur = [], ""
    for line in text.splitlines():
        if line.startswith("    ") and line.strip():
            cur += " " + line.strip().rstrip("\\").strip()
            if not line.rstrip().endswith("\\"):
                cmds.append(cur.strip())
                cur = ""
        elif cur:
            cmds.append(cur.strip())
            cur = ""
    if cur:
        cmds.append(cur.strip())
    return cmds


def test_there_are_profiles():
    assert len(PROFILES) >= 3


@pytest.mark.parametrize("path", PROFILES, ids=os.path.basename)
def test_quoted_bench_commands_parse(path, monkeypatch):
    with open(path) as f:
        cmds = [c for c in _commands(f.read()) if "bench.py" in c]
    assert cmds, "no bench.py command quoted"
    for c in cmds:
        argv = shlex.split(c)
        i = next(j for j, a in enumerate(argv) if a.endswith("bench.py"))
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv[i + 1:])
        bench.parse_args()  # an unknown or malformed option exits here


@pytest.mark.parametrize("path", PROFILES, ids=os.path.basename)
def test_summary_names_its_kernel_source(path):
    with open(path) as f:
        text = f.read()
    assert re.search(r"kernel_source_sha256: [0-9a-f]{64}", text)
    assert "--clock-control none" in text
