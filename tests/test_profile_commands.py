"""The bench.py command lines quoted in profiles/ (the commands that made
each ncu summary and timing) still parse with bench.py's current options.
CPU only: nothing is run."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def quoted_commands():
    cmds = set()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for m in re.finditer(r"python bench\.py([^`\n\\]*)", open(path).read()):
            cmds.add((os.path.basename(path), m.group(1).strip()))
    return sorted(cmds)


def test_profiles_quote_bench_commands():
    assert len(quoted_commands()) >= 5


@pytest.mark.parametrize("profile,args", quoted_commands())
def test_quoted_command_parses(profile, args, monkeypatch):
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    monkeypatch.setattr(sys, "argv", ["bench.py", *shlex.split(args)])
    bench.parse()  # argparse exits on an unknown or malformed option
