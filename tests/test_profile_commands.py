"""The ncu summaries under profiles/ and the README state the bench.py
commands their figures come from; every such command must still be accepted
by bench.py's argument parser (options and choices), so that each recipe can
be run again from the committed files.  Each summary states at least one
bench.py command."""
import glob
import os
import shlex

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(path):
    out = []
    for line in open(path, encoding="utf-8"):
        t = line.strip()
        if t.startswith("python bench.py"):
            out.append(t)
    return out


def test_every_profile_has_a_committed_command():
    assert PROFILES
    for p in PROFILES:
        assert _commands(p), os.path.basename(p)


@pytest.mark.parametrize("path", PROFILES + [os.path.join(ROOT, "README.md")], ids=os.path.basename)
def test_stated_bench_commands_parse(path):
    parser = bench.make_parser()
    for cmd in _commands(path):
        # after "python bench.py", without a trailing comment (the README's lines)
        argv = shlex.split(cmd.split("#", 1)[0])[2:]
        try:
            parser.parse_args(argv)
        except SystemExit as e:  # argparse reports an unknown option or a bad choice this way
            pytest.fail(f"{os.path.basename(path)}: {cmd!r} is not accepted by bench.py ({e})")
