"""The ncu summaries under profiles/ give the commands that made them; the
bench.py invocations among them must still parse against bench.py's
options, and traffic.json must hold DRAM bytes per lattice update near the
algorithmic 72 B (FP32) / 36 B (16-bit) for the kernels it names."""
import glob
import json
import os
import shlex

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_commands():
    cmds = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for line in text.splitlines():
            if "python bench.py" not in line:
                continue
            args = shlex.split(line.split("python bench.py", 1)[1])
            args = [a for a in args if a not in ("&&",)]
            cmds.append((os.path.basename(path), args))
    return cmds


@pytest.mark.parametrize("name,args", bench_commands())
def test_profile_commands_parse(name, args):
    assert bench.parse(args) is not None, name


def test_profile_summaries_name_their_commands():
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read()
        assert "ncu " in text and "--clock-control none" in text, path


def test_traffic_record_is_plausible():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kernel, r in rec.items():
        algorithmic = 72.0 if "float" in kernel else 36.0
        assert 0.8 * algorithmic < r["dram_bytes_per_lu"] < 1.2 * algorithmic, kernel
        assert r["dram_bytes_per_lu"] == pytest.approx(
            r["dram_read_bytes_per_lu"] + r["dram_write_bytes_per_lu"], abs=0.02), kernel
        assert len(r["source_sha"]) == 16


def test_kernel_hash_ignores_comments_only():
    """bench.sources_sha hashes the step kernels' code without comments and
    spacing: a comment edit keeps a traffic record, a code edit drops it."""
    a = 'x = y + 1; // note\n/* block */ s = "//kept";  z = \'"\';\n'
    b = 'x = y + 1;   // another note\ns = "//kept"; z = \'"\';'
    c = 'x = y + 2; s = "//kept"; z = \'"\';'
    assert bench.code_of(a) == bench.code_of(b) != bench.code_of(c)
    assert '"//kept"' in bench.code_of(a)
