"""The bounds-checked build (libgputx_debug.so, compiled with -DGPUTX_DEBUG)
runs the parity cases of every executor: each index a gather or scatter
takes is checked on the device, and a failed check would fail the bulk with
GPUTX_EBOUNDS.  The cases run in a child process that loads the debug
library (GPUTX_DEBUG=1) and compare with the oracle as in the release tests."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

# small cases of every strategy and schema: debit-credit (uniform, hot
# accounts, the TPL executors' pick), order-entry, subscriber, the batcher,
# incremental 0-set execution, the served mix
CASES = [
    ("tests/test_gpu_dc.py", "config1 or hot_chain or back_to_back"),
    ("tests/test_gpu_schemas.py", "not full_size and not sweep"),
    ("tests/test_gpu_batch.py", "uneven or graph"),
    ("tests/test_gpu_relaxed.py", ""),
    ("tests/test_gpu_pool.py", "debit_credit_stream or mixed_schema"),
    ("tests/test_gpu_serve.py", "served_stream_equals or mixed_schemas_served"),
]


@pytest.mark.parametrize("path,expr", CASES)
def test_parity_cases_under_the_debug_build(path, expr):
    from paper_1103_3105_gb300 import _build
    _build.build(debug=True)
    env = dict(os.environ, GPUTX_DEBUG="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", path]
    if expr:
        cmd += ["-k", expr]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail


def test_debug_library_is_the_one_loaded():
    """GPUTX_DEBUG=1 selects the debug library and nothing else."""
    from paper_1103_3105_gb300 import _build
    _build.build(debug=True)
    code = ("import paper_1103_3105_gb300 as G, os; G.lib(); "
            "print(os.path.basename(G.LIB_PATH))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, GPUTX_DEBUG="1"),
                         capture_output=True, text=True, timeout=300)
    assert out.stdout.strip() == "libgputx_debug.so", out.stdout + out.stderr
