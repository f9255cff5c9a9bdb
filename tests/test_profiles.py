"""Every command recorded in profiles/ runs committed files with options that
bench.py still accepts (a renamed or removed flag would leave a summary whose
command no longer reproduces it)."""
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _bench_invocations():
    out = []
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        text = open(os.path.join(PROFILES, name)).read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^\n`>&|]*)", text):
            out.append((name, shlex.split(m.group(1))))
    return out


def test_profiles_record_their_commands():
    names = [n for n in os.listdir(PROFILES) if n.endswith(".md")]
    assert names
    for n in names:
        text = open(os.path.join(PROFILES, n)).read()
        assert "ncu " in text and "--clock-control none" in text, n
        assert "python bench.py" in text, n


@pytest.mark.parametrize("name,args", _bench_invocations())
def test_recorded_bench_arguments_parse(name, args, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", *args])
    ns = bench.parse()
    assert ns.workload in bench.WORKLOADS, (name, args)
