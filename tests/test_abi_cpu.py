"""The C-ABI library builds, loads and exports every entry point include/ocn.h declares.

No compute calls are made (this runs on machines without a GPU); only pure
host-side entry points (version, argument validation of the grid) are invoked.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ocn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ocn_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libocn():
    from paper_2502_14148_gb300 import build, ocn
    build.build()
    return ocn.lib()


def test_every_declared_symbol_is_exported(libocn):
    from paper_2502_14148_gb300 import ocn
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(libocn, n), n
    assert sorted(ocn.EXPORTS) == names


def test_abi_version_and_grid_validation(libocn):
    from paper_2502_14148_gb300 import ocn
    assert libocn.ocn_abi_version() == 2
    zf = np.linspace(-1, 0, 9)
    g = ocn.Grid(16, 12, 8, 1.0, 1.0, zf)          # host-only call
    assert g._h
    for bad in [(15, 12, 8), (10, 12, 8), (16, 12, 0), (2, 12, 8)]:
        with pytest.raises(ocn.OcnError) as ei:
            ocn.Grid(*bad, 1.0, 1.0, np.linspace(-1, 0, max(bad[2], 0) + 1))
        assert ei.value.status == -1
    with pytest.raises(ocn.OcnError):
        ocn.Grid(16, 12, 8, 1.0, 1.0, zf[::-1])       # descending faces
    assert "ascending" in libocn.ocn_last_error().decode()
    with pytest.raises(ocn.OcnError) as ei:           # a level of 2^32 cells: beyond 32-bit level offsets
        ocn.Grid(65536, 65536, 8, 1.0, 1.0, zf)
    assert ei.value.status == -1 and "2^31" in libocn.ocn_last_error().decode()
    assert ocn.Grid(32768, 49152, 1, 1.0, 1.0, np.linspace(-1, 0, 2))._h   # 1.6e9 cells per level: allowed


def test_no_oracle_in_the_product_path():
    """The CUDA library and its binding never import, link or call the oracle."""
    pat = re.compile(r"(from|import)\s+oracle|liboracle|ocn_oracle|\borc_[a-z_]+\s*\(")
    pkg = os.path.join(ROOT, "paper_2502_14148_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f), encoding="utf-8").read()
                assert not pat.search(txt), f


def test_no_cpu_fallback_without_a_gpu():
    """Without a CUDA device every compute object refuses to be created: there is no CPU path."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2502_14148_gb300 import inputs, ocn
    p = inputs.config("cbl_256", Nx=16, Ny=16, Nz=8)
    for make in (lambda: ocn.Model(p),
                 lambda: ocn.Ensemble(inputs.ensemble_configs(n=2, sizes=(16,), depths=(8,))),
                 lambda: ocn.MLP(inputs.MLP_SIZES, max_batch=128)):
        with pytest.raises(RuntimeError, match="no CPU path"):
            make()


def test_transfer_and_bounds_calls_reject_bad_arguments(libocn):
    """The batched transfer calls, the transfer wait and the bounds-status call refuse a null
    model before touching the device (host-only paths)."""
    vp = C.c_void_p
    fids = (C.c_int * 1)(0)
    ptrs = (vp * 1)(None)
    nb = (C.c_size_t * 1)(4)
    assert libocn.ocn_set_fields(None, 1, fids, ptrs, nb, 0) == -1
    assert libocn.ocn_get_fields(None, 1, fids, ptrs, nb, 2) == -1
    assert libocn.ocn_wait_transfers(None) == -1
    st, chk = C.c_uint(7), C.c_int(7)
    assert libocn.ocn_bounds_status(None, C.byref(st), C.byref(chk)) == -1
    assert "null" in libocn.ocn_last_error().decode()


def test_library_variant_is_selected_by_environment(tmp_path):
    """OCN_LIBRARY names the build the binding loads (the bounds-checked variant in its GPU test); a
    missing file is an error that names it, never a fallback to another build."""
    import subprocess
    import sys
    missing = str(tmp_path / "libocn_missing.so")
    code = "from paper_2502_14148_gb300 import ocn; ocn.lib()"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, OCN_LIBRARY=missing),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "libocn_missing.so is missing" in r.stderr
