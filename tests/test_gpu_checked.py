"""The index-checked build (libpcg_checked.so, -DPCG_CHECKED; a stand-in for a memory
checker, which is not available here), GB300 only.  Its kernels check every index they turn
into an address and record a code instead of making the access when a check fails.  The
same set of solves -- stencils with one and two unknowns per thread, variable coefficients,
CSR, Jacobi, mixed precision, a variable shift, the TMA-staged sweep, the persistent
kernel, a batch, a served request, a system in slabs -- runs with the ordinary and the
checked build: no check may fail, and every result must have the same bits."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(tmp_path, lib, name):
    out = tmp_path / f"{name}.npz"
    env = dict(os.environ)
    if lib:
        env["PCG_LIBRARY"] = lib
    else:
        env.pop("PCG_LIBRARY", None)
    subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_cases.py"), str(out)], env=env,
                   check=True, timeout=900)
    return np.load(out)


def test_checked_build_runs_clean_and_changes_no_result(tmp_path):
    import torch
    assert torch.cuda.is_available()
    from paper_1706_05988_gb300 import build
    build.build()
    lib_checked = build.build(checked=True)
    plain = _run(tmp_path, None, "plain")
    checked = _run(tmp_path, lib_checked, "checked")
    assert int(plain["checked_build"][0]) == 0 and int(checked["checked_build"][0]) == 1
    assert int(checked["check_code"][0]) == 0, f"index check {int(checked['check_code'][0])} failed"
    keys = [k for k in plain.files if k not in ("check_code", "checked_build")]
    assert len(keys) >= 30
    for k in keys:
        assert np.array_equal(plain[k], checked[k]), k
