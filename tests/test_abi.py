"""The C-ABI library builds, loads and exports what include/marnoldi.h declares (no GPU).

Also exercises the host-side validation of marnoldi_setup / marnoldi_solve,
which runs before any device work and needs no GPU.
"""

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1307_3218_gb300 as m
from paper_1307_3218_gb300 import build as mbuild
from tbsynth import config_c1, tiny_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "marnoldi.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = []
    for stmt in src.split(";"):
        s = " ".join(stmt.split())
        if s.startswith("typedef") or "marnoldi_" not in s:
            continue
        mm = re.search(r"\b(marnoldi_\w+)\s*\(", s)
        if mm:
            names.append(mm.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = mbuild.build()
    return m.load(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("marnoldi_setup", "marnoldi_solve", "marnoldi_density", "marnoldi_energy",
                 "marnoldi_green", "marnoldi_column_stats", "marnoldi_last_error",
                 "marnoldi_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", mbuild.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T marnoldi_" in ln}
    assert exported == set(declared_functions())


def _setup_args(t):
    return [t.n_block_rows, t.row_ptr.copy(), t.col_idx.copy(), t.H.copy(), t.S.copy()]


def _expect(code, t, **kw):
    args = _setup_args(t)
    for k, v in kw.items():
        idx = {"rp": 1, "ci": 2, "H": 3, "S": 4}[k]
        args[idx] = v
    with pytest.raises(m.MarnoldiError) as ei:
        m.marnoldi_setup(*args, precision=m.MARNOLDI_FP64, stream=0)
    assert ei.value.code == code, str(ei.value)
    return str(ei.value)


def test_setup_validation_on_host(lib):
    t = tiny_system(8, seed=0)
    # asymmetric H values
    H = t.H.copy()
    H[1, 0, 1] += 1.0
    assert "symmetric" in _expect(m.marnoldi.MARNOLDI_EINVAL, t, H=H)
    # NaN
    S = t.S.copy()
    S[0, 2, 2] = np.nan
    assert "finite" in _expect(m.marnoldi.MARNOLDI_EINVAL, t, S=S)
    # unsorted column indices in a row
    ci = t.col_idx.copy()
    r0, r1 = t.row_ptr[0], t.row_ptr[1]
    if r1 - r0 >= 2:
        ci[r0], ci[r0 + 1] = ci[r0 + 1], ci[r0]
        _expect(m.marnoldi.MARNOLDI_EINVAL, t, ci=ci)
    # column index out of range
    ci = t.col_idx.copy()
    ci[-1] = t.n_block_rows + 3
    _expect(m.marnoldi.MARNOLDI_EINVAL, t, ci=ci)
    # S not positive definite: inflate the overlaps
    S = t.S.copy()
    rows = np.repeat(np.arange(t.n_block_rows), np.diff(t.row_ptr))
    off = rows != t.col_idx
    S[off] *= 40.0
    assert "positive definite" in _expect(m.marnoldi.MARNOLDI_ENOTSPD, t, S=S)
    # S_jj <= 0
    S = t.S.copy()
    diag = np.nonzero(rows == t.col_idx)[0][0]
    S[diag, 1, 1] = -1.0
    _expect(m.marnoldi.MARNOLDI_ENOTSPD, t, S=S)
    assert "S_jj" in m.marnoldi_last_error(None)


def test_setup_rejects_missing_mirror_block(lib):
    t = config_c1()
    # drop block (0, J) but keep (J, 0): rebuild row 0 without its last off-diagonal block
    r0, r1 = t.row_ptr[0], t.row_ptr[1]
    keep = np.ones(t.nnzb, bool)
    last = r1 - 1 if t.col_idx[r1 - 1] != 0 else r1 - 2
    keep[last] = False
    rp = t.row_ptr.copy()
    rp[1:] -= 1
    with pytest.raises(m.MarnoldiError) as ei:
        m.marnoldi_setup(t.n_block_rows, rp, t.col_idx[keep], t.H[keep], t.S[keep], stream=0)
    assert ei.value.code == m.marnoldi.MARNOLDI_EINVAL
    assert "mirror" in str(ei.value)


def test_null_context_calls(lib):
    assert lib.marnoldi_solve(None, None, -1, 30, 0, 1.0, 0.1, None) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_energy(None, None, None, None) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_density(None, None, None) == m.marnoldi.MARNOLDI_EINVAL
    assert lib.marnoldi_set_batch(None, 4) == m.marnoldi.MARNOLDI_EINVAL
    lib.marnoldi_destroy(None)
    assert lib.marnoldi_kernel_kinds() >= 9


def test_package_fails_loudly_without_library(tmp_path):
    from paper_1307_3218_gb300 import marnoldi as mm
    saved = mm._LIB
    mm._LIB = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            mm.load(str(tmp_path / "missing.so"))
    finally:
        mm._LIB = saved


def test_count_noalloc_binding_rejects_host_arrays():
    """The binding refuses what the C entry point cannot check: host arrays and CPU tensors
    (and, on a GPU, wrong dtypes, devices, strides or lengths) never reach the kernel."""
    import torch

    import paper_1307_3218_gb300 as pm
    x = np.zeros(16)
    with pytest.raises(pm.MarnoldiError) as ei:
        pm.marnoldi_count_noalloc(x, x, None, 4, 4, 0.0, 0.1, x)
    assert ei.value.code == pm.marnoldi.MARNOLDI_EINVAL
    t = torch.zeros(16, dtype=torch.float64)
    with pytest.raises(pm.MarnoldiError) as ei:
        pm.marnoldi_count_noalloc(t, t, None, 4, 4, 0.0, 0.1, t)
    assert ei.value.code == pm.marnoldi.MARNOLDI_EINVAL
    with pytest.raises(pm.MarnoldiError) as ei:          # oversize, before any tensor check
        pm.marnoldi_count_noalloc(t, t, None, 16_777_217, 1, 0.0, 0.1, t)
    assert "16777216" in str(ei.value)
