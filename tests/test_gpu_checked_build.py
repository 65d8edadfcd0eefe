"""Bounds test with the checked library (liblpic_check.so, built with
LPIC_CHECK=1: every data-dependent shared-memory index of the gather and the
current boxes is tested against its box, and an index outside raises
LPIC_ST_BOUNDS instead of being accessed).  The cases of checked_cases.py run
in a child process on the checked library: no status bit may be raised, and
their fields and currents must match those of the product library run here
(the tests only observe; the two builds may fuse multiplies and adds of the
push differently, so the match is to float rounding carried over the steps,
not bitwise)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13507_b300 import build, lpic
    build.build()
    lpic.load()


def test_checked_library_raises_no_bounds_status_and_matches(tmp_path):
    import numpy as np
    from paper_2607_13507_b300 import build
    from pic_cases import rel_l2
    checked = build.build(checked=True)
    env = dict(os.environ, LPIC_LIBRARY=checked)
    dir_c, dir_p = tmp_path / "checked", tmp_path / "product"
    dir_c.mkdir()
    dir_p.mkdir()
    res = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), str(dir_c)], env=env,
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    got = json.loads(res.stdout.strip().splitlines()[-1])
    sys.path.insert(0, HERE)
    import checked_cases
    ref = checked_cases.run_cases(str(dir_p))
    assert set(got) == set(ref)
    for name in ref:
        assert got[name] == 0, (name, got[name])
        assert ref[name] == 0, name
        a, b = np.load(dir_c / (name + ".npz")), np.load(dir_p / (name + ".npz"))
        assert set(a.files) == set(b.files)
        for k in a.files:
            if np.linalg.norm(b[k].astype(np.float64)) > 0:
                assert rel_l2(a[k], b[k]) < 1e-3, (name, k, rel_l2(a[k], b[k]))
