"""The ncu summaries under profiles/ name the command that made them; those commands must run the
committed files: every bench.py flag they use is one bench.py accepts, every test file they name
exists and their -k expression selects a test in it."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _summaries():
    return [os.path.join(PROFILES, f) for f in sorted(os.listdir(PROFILES)) if f.endswith((".md", ".txt"))]


def _bench_flags():
    out = subprocess.run([sys.executable, "bench.py", "--help"], cwd=ROOT, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr[-1000:]
    return set(re.findall(r"--[a-z0-9][a-z0-9-]*", out.stdout))


def test_every_summary_names_its_command():
    for path in _summaries():
        text = open(path).read()
        assert "Command" in text or "command" in text, path
        assert re.search(r"python (bench\.py|-m pytest)", text), path


def test_bench_commands_use_existing_flags():
    flags = _bench_flags()
    for path in _summaries():
        for line in open(path).read().splitlines():
            if "python bench.py" not in line:
                continue
            used = set(re.findall(r"--[a-z0-9][a-z0-9-]*", line.split("python bench.py", 1)[1]))
            assert used <= flags, (path, used - flags)


def test_pytest_commands_select_existing_tests():
    for path in _summaries():
        for line in open(path).read().splitlines():
            m = re.search(r"python -m pytest (\S+\.py)(.*)", line)
            if not m:
                continue
            test_file = os.path.join(ROOT, m.group(1))
            assert os.path.exists(test_file), (path, m.group(1))
            k = re.search(r"-k\s+(\S+)", m.group(2))
            if k:
                names = re.findall(r"^def (test_\w+)", open(test_file).read(), re.M)
                assert any(k.group(1) in n for n in names), (path, k.group(1))
