"""The GPU suite again, on the checked build of libddsg.

The checked build (-DDDSG_CHECKED) tests every table index its kernels derive
(cell offset, directory slot, device row against its component, staged block,
dimension, point and component ids) before the access and records a failed test
in a check word instead of touching memory out of bounds. It stands in for a
memory sanitizer. This test builds that variant and runs every other GPU test
file against it in a child process (DDSG_VARIANT=checked); the suite's
conftest then requires the check word to be clean after each test. The
full-size workloads are left out (they cover sizes, not new index paths).
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_gpu_suite_passes_on_the_checked_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if os.environ.get("DDSG_VARIANT") == "checked":
        pytest.skip("already running on the checked build")
    sys.path.insert(0, ROOT)
    from paper_2202_06555_gb300 import build as B
    B.build(variant="checked")
    files = sorted(f for f in os.listdir(HERE)
                   if f.startswith("test_gpu_") and f.endswith(".py")
                   and f not in ("test_gpu_checked_build.py", "test_gpu_full_size.py"))
    env = dict(os.environ, DDSG_VARIANT="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"]
                       + [os.path.join(HERE, f) for f in files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-30:])
    assert r.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
    print(tail.splitlines()[-1])


def test_checked_build_reports_itself():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = ("import paper_2202_06555_gb300 as G; L = G.load(); "
            "print(L.ddsg_checked_build(), L.ddsg_version().decode(), G.take_check_word())")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, DDSG_VARIANT="checked"))
    assert out.returncode == 0, out.stderr
    assert out.stdout.split()[0] == "1" and "checked" in out.stdout, out.stdout
    rel = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, DDSG_VARIANT="release"))
    assert rel.returncode == 0 and rel.stdout.split()[0] == "0", rel.stdout + rel.stderr
