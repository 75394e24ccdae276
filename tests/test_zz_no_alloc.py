"""ocn_project_noalloc, the projection for callers that cannot allocate device memory.

Plug-ins whose host application owns all device memory, and loops that must not
allocate while running, call this entry point with the velocity and pressure
arrays they already hold; its work arrays live in a fixed array inside the
library.  This file is named so that pytest collects it last.  It checks, through
the C ABI, that two calls in a row on different inputs each match the projection
of the regular entry point (ocn_project on a model with the same grid), within
the tolerances the other GPU tests use, and that sizes above the stated limits
are refused.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2502_14148_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ocn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_14148_gb300 import build, ocn as mod
    build.build()
    return mod


def _params(precision, Nx=48, Ny=36, Nz=20):
    p = dict(Nx=Nx, Ny=Ny, Nz=Nz, Lx=48.0, Ly=30.0, Lz=20.0, precision=precision, weno_order=5,
             closure="none", tracers=["b"], eos="buoyancy_tracer",
             z_faces=inputs.tanh_faces(Nz, 20.0, 1.5), top_flux={}, bottom_flux={})
    return p


def _noalloc(ocn, p, st, stream):
    import torch
    dt = torch.float32 if p["precision"] == 32 else torch.float64
    dev = torch.device("cuda")
    u, v, w = (torch.as_tensor(st[x], dtype=dt, device=dev).contiguous() for x in "uvw")
    pr = torch.empty((p["Nz"], p["Ny"], p["Nx"]), dtype=dt, device=dev)
    zf = np.ascontiguousarray(p["z_faces"], dtype=np.float64)
    err = C.c_char_p()
    torch.cuda.synchronize()
    st_ = ocn.lib().ocn_project_noalloc(p["precision"], p["Nx"], p["Ny"], p["Nz"], p["Lx"], p["Ly"],
                                        zf.ctypes.data_as(C.POINTER(C.c_double)),
                                        C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr()), C.c_void_p(w.data_ptr()),
                                        C.c_void_p(pr.data_ptr()), C.c_void_p(stream.cuda_stream), C.byref(err))
    assert st_ == 0, err.value
    stream.synchronize()
    return {"u": u.cpu().numpy(), "v": v.cpu().numpy(), "w": w.cpu().numpy(), "p": pr.cpu().numpy()}


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_projection_matches_ocn_project_twice(ocn, precision):
    import torch
    p = _params(precision)
    tol = 1e-11 if precision == 64 else 2e-5
    stream = torch.cuda.Stream()
    for seed in (71, 72):                       # two calls in a row, different inputs
        st = inputs.random_state(p, seed=seed)
        if precision == 32:
            st = {k: x.astype(np.float32).astype(np.float64) for k, x in st.items()}
        got = _noalloc(ocn, p, st, stream)
        m = ocn.Model(p)
        m.set(project=False, **st)
        m.project()
        for name in ("u", "v", "w", "p"):
            ref = m.get_numpy(name).astype(np.float64)
            err = np.abs(got[name] - ref).max() / np.abs(ref).max()
            assert err < tol, (seed, name, err)


def test_noalloc_rejects_sizes_above_its_limit(ocn):
    import torch
    p = _params(32, Nx=512, Ny=512, Nz=8)       # (512/2+1)*512*8 > OCN_NOALLOC_MAX_MODES
    zf = np.ascontiguousarray(p["z_faces"], dtype=np.float64)
    err = C.c_char_p()
    dummy = torch.empty(4, device="cuda")
    st = ocn.lib().ocn_project_noalloc(32, p["Nx"], p["Ny"], p["Nz"], p["Lx"], p["Ly"],
                                       zf.ctypes.data_as(C.POINTER(C.c_double)),
                                       *(C.c_void_p(dummy.data_ptr()) for _ in range(4)), None, C.byref(err))
    assert st == -1 and b"OCN_NOALLOC_MAX_MODES" in err.value


def test_noalloc_refuses_a_stream_under_capture(ocn):
    """Every call uploads its grid tables from host memory, which a captured graph could not
    replay faithfully; a stream that is being captured is refused before anything is enqueued,
    and the capture itself still ends cleanly."""
    import torch
    p = _params(32)
    dev = torch.device("cuda")
    u, v, w, pr = (torch.zeros((p["Nz"], p["Ny"], p["Nx"]), device=dev) for _ in range(4))
    x = torch.zeros(8, device=dev)
    zf = np.ascontiguousarray(p["z_faces"], dtype=np.float64)
    err = C.c_char_p()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        x.add_(1.0)
        st = ocn.lib().ocn_project_noalloc(32, p["Nx"], p["Ny"], p["Nz"], p["Lx"], p["Ly"],
                                           zf.ctypes.data_as(C.POINTER(C.c_double)),
                                           *(C.c_void_p(t.data_ptr()) for t in (u, v, w, pr)),
                                           C.c_void_p(stream.cuda_stream), C.byref(err))
    assert st == -7 and b"captured" in err.value, (st, err.value)
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
