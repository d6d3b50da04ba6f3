"""The bounds-checked build (-DLBM_CHECKED) in place of a memory checker: every shared
and global access of the step kernels and every bulk copy is checked (range inside the
stage or the population array, 16-byte rules of cp.async.bulk); a failed check records
LBM_ECHECK and skips the access.  A child process runs every kernel path and job layout on
small and degenerate lattices (tests/checked_cases.py) against the checked library: no
check may fail, and the stored states must equal the normal library's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_checked_build_passes_all_layouts(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08163_gb300 import build, lbm
    checked = build.build(checked=True)
    build.build()
    lbm.load()
    out_checked = str(tmp_path / "checked.npz")
    env = dict(os.environ, LBM_LIBRARY=checked,
               PYTHONPATH=os.pathsep.join([HERE, ROOT, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), out_checked],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    sys.path.insert(0, HERE)
    import checked_cases
    out_normal = str(tmp_path / "normal.npz")
    checked_cases.run(lbm, out_normal)
    a, b = np.load(out_checked), np.load(out_normal)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), f"{k}: checked and normal builds differ"
    print(f"{len(checked_cases.CASES)} layouts x 3 steps: no check failed, states bit-identical")
