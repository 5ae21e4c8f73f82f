"""The library path has no fallback: without libspx.so the binding raises,
and without a CUDA device an Engine cannot be created (the C library reports
an error; nothing runs on the host instead)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(code):
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, cwd=ROOT)


def test_missing_library_raises():
    r = run("from paper_2203_14362_gb300 import spx\n"
            "try:\n"
            "    spx.load('/nonexistent/libspx.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    assert r.returncode == 0 and "raised: libspx.so not found" in r.stdout, r.stdout + r.stderr


def test_engine_needs_a_device():
    # on a host without a visible GPU, spx_create fails with a status; no host path takes over
    r = run("import os\n"
            "os.environ['CUDA_VISIBLE_DEVICES'] = ''\n"
            "from paper_2203_14362_gb300 import spx\n"
            "try:\n"
            "    spx.Engine(0)\n"
            "    print('created')\n"
            "except spx.SpxError as e:\n"
            "    print('refused:', e.status)\n")
    assert r.returncode == 0, r.stderr
    assert "refused:" in r.stdout and "created" not in r.stdout, r.stdout
