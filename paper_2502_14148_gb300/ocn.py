"""Thin ctypes binding of the C ABI in ``include/ocn.h``.

Argument marshalling only: every step of the time integration runs in the CUDA
kernels of ``_lib/libocn.so``.  PyTorch supplies the device arena and the CUDA
stream.  There is no CPU fallback: if the library or a GPU is missing, the
constructors raise.

The parameter dictionary uses the keys of :mod:`paper_2502_14148_gb300.inputs`
(the names follow the paper's ``RectilinearGrid`` / ``NonhydrostaticModel``
keywords: size, extent, advection order, closure, coriolis, buoyancy, tracers,
boundary fluxes).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libocn.so")

OCN_FIELD_U, OCN_FIELD_V, OCN_FIELD_W, OCN_FIELD_TRACER0 = 0, 1, 2, 3
OCN_FIELD_P, OCN_FIELD_G, OCN_FIELD_NU_E = 10, 20, 30
OCN_FIELD_TRACER_REF0, OCN_FIELD_RAW = 40, 0x100
OCN_OPT_GRAPHS, OCN_OPT_SYNC_CHECK, OCN_OPT_KERNEL_TIMING, OCN_OPT_TENDENCY_VARIANT = 1, 2, 3, 4
OCN_HOST_ASYNC = 2
TENDENCY_VARIANTS = 7
KERNEL_CLASSES = ["closure", "tendency", "div_fftx", "fft_y", "tridiag", "gauge", "ifftx", "correct", "column_closure",
                  "vertical"]
STEPPERS = {"rk3": 0, "qab2": 1}
COLUMN_FEATURES = 32
MAX_TRACERS = 4
CLOSURES = {"none": 0, "scalar": 1, "smagorinsky": 2, "amd": 3}
EOS = {"buoyancy_tracer": 0, "linear_ts": 1}
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_NONFINITE", -5: "ERR_CFL",
          -6: "ERR_TIMEOUT", -7: "ERR_UNSUPPORTED", -8: "ERR_STATE"}

# Entry points declared in include/ocn.h (checked by the CPU test suite).
EXPORTS = ["ocn_abi_version", "ocn_last_error", "ocn_grid_create", "ocn_grid_destroy", "ocn_model_create",
           "ocn_model_destroy", "ocn_model_arena_bytes", "ocn_model_bind_arena", "ocn_set_field", "ocn_get_field",
           "ocn_set_fields", "ocn_get_fields", "ocn_wait_transfers", "ocn_bounds_status",
           "ocn_project", "ocn_time_step", "ocn_compute_tendencies", "ocn_diagnostics", "ocn_set_option",
           "ocn_launches_per_step", "ocn_kernel_times", "ocn_project_noalloc", "ocn_autotune", "ocn_profiles",
           "ocn_regrid", "ocn_ensemble_create", "ocn_ensemble_destroy", "ocn_ensemble_arena_bytes",
           "ocn_ensemble_bind_arena", "ocn_ensemble_member", "ocn_ensemble_time_step", "ocn_ensemble_set_option",
           "ocn_ensemble_autotune", "ocn_ensemble_launches_per_step", "ocn_mlp_create", "ocn_mlp_destroy",
           "ocn_mlp_arena_bytes", "ocn_mlp_bind_arena", "ocn_mlp_num_params", "ocn_mlp_set_params",
           "ocn_mlp_get_params", "ocn_mlp_forward", "ocn_mlp_gradients", "ocn_mlp_adam", "ocn_mlp_train_step",
           "ocn_gemm_bf16", "ocn_set_column_closure", "ocn_closure_features", "ocn_column_fluxes",
           "ocn_coarse_grain", "ocn_set_time_stepper", "ocn_set_vertical_diffusivity", "ocn_gemm_timeout_test",
           "ocn_fp32_fma_peak", "ocn_set_column_closure_mode"]
OCN_OPT_ENSEMBLE_MODE, OCN_ENSEMBLE_CONCURRENT, OCN_ENSEMBLE_SEQUENTIAL, OCN_ENSEMBLE_BATCHED = 5, 0, 1, 2
OCN_OPT_ENSEMBLE_BRANCHES = 6
ENSEMBLE_MODES = {"concurrent": OCN_ENSEMBLE_CONCURRENT, "sequential": OCN_ENSEMBLE_SEQUENTIAL,
                  "batched": OCN_ENSEMBLE_BATCHED}


class OcnError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("Nx", C.c_int), ("Ny", C.c_int), ("Nz", C.c_int), ("Lx", C.c_double), ("Ly", C.c_double),
                ("z_faces", C.POINTER(C.c_double))]


class ModelDesc(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("weno_order", C.c_int), ("closure", C.c_int),
        ("nu", C.c_double), ("kappa", C.c_double),
        ("Cs", C.c_double), ("Cb", C.c_double), ("Pr", C.c_double),
        ("C_amd", C.c_double), ("f", C.c_double),
        ("n_tracers", C.c_int), ("eos", C.c_int),
        ("g", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("T0", C.c_double), ("S0", C.c_double),
        ("top_flux", C.c_double * (2 + MAX_TRACERS)), ("bottom_flux", C.c_double * (2 + MAX_TRACERS)),
        ("fp64_pivots", C.c_int),
    ]


class ColumnClosureDesc(C.Structure):
    _fields_ = [("mu", C.c_float * COLUMN_FEATURES), ("sigma", C.c_float * COLUMN_FEATURES),
                ("out_scale", C.c_float * 3), ("N2_background", C.c_double)]


_lib = None


def lib(path: str = None):
    """Load libocn.so (raises if it has not been built: there is no fallback).  The environment
    variable OCN_LIBRARY selects another build of the same library (the bounds-checked
    libocn_checked.so)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("OCN_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2502_14148_gb300.build`")
    L = C.CDLL(path)
    vp, sz = C.c_void_p, C.c_size_t
    L.ocn_abi_version.restype = C.c_int
    L.ocn_last_error.restype = C.c_char_p
    L.ocn_grid_create.argtypes = [C.POINTER(GridDesc), C.POINTER(vp)]
    L.ocn_grid_destroy.argtypes = [vp]
    L.ocn_model_create.argtypes = [vp, C.POINTER(ModelDesc), vp, C.POINTER(vp)]
    L.ocn_model_destroy.argtypes = [vp]
    L.ocn_model_arena_bytes.argtypes = [vp, C.POINTER(sz)]
    L.ocn_model_bind_arena.argtypes = [vp, vp, sz]
    L.ocn_set_field.argtypes = [vp, C.c_int, vp, sz, C.c_int]
    L.ocn_get_field.argtypes = [vp, C.c_int, vp, sz, C.c_int]
    L.ocn_set_fields.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(vp), C.POINTER(sz), C.c_int]
    L.ocn_get_fields.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(vp), C.POINTER(sz), C.c_int]
    L.ocn_wait_transfers.argtypes = [vp]
    L.ocn_bounds_status.argtypes = [vp, C.POINTER(C.c_uint), C.POINTER(C.c_int)]
    L.ocn_project.argtypes = [vp]
    L.ocn_time_step.argtypes = [vp, C.c_double, C.c_int]
    L.ocn_compute_tendencies.argtypes = [vp]
    L.ocn_diagnostics.argtypes = [vp, C.c_double, C.POINTER(C.c_double), C.c_int]
    L.ocn_set_option.argtypes = [vp, C.c_int, C.c_longlong]
    L.ocn_launches_per_step.argtypes = [vp, C.POINTER(C.c_int)]
    L.ocn_kernel_times.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.ocn_autotune.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    dp = C.POINTER(C.c_double)
    L.ocn_profiles.argtypes = [vp, dp, C.c_int]
    L.ocn_regrid.argtypes = [dp, C.c_int, dp, dp, C.c_int, dp]
    L.ocn_ensemble_create.argtypes = [C.c_int, C.POINTER(GridDesc), C.POINTER(ModelDesc), vp, C.POINTER(vp)]
    L.ocn_ensemble_destroy.argtypes = [vp]
    L.ocn_ensemble_destroy.restype = None
    L.ocn_ensemble_arena_bytes.argtypes = [vp, C.POINTER(sz)]
    L.ocn_ensemble_bind_arena.argtypes = [vp, vp, sz]
    L.ocn_ensemble_member.argtypes = [vp, C.c_int, C.POINTER(vp)]
    L.ocn_ensemble_time_step.argtypes = [vp, C.c_double, C.c_int]
    L.ocn_ensemble_set_option.argtypes = [vp, C.c_int, C.c_longlong]
    L.ocn_ensemble_autotune.argtypes = [vp, C.POINTER(C.c_int)]
    L.ocn_ensemble_launches_per_step.argtypes = [vp, C.POINTER(C.c_int)]
    L.ocn_project_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.POINTER(C.c_double), vp, vp, vp, vp, vp, C.POINTER(C.c_char_p)]
    ip = C.POINTER(C.c_int)
    L.ocn_mlp_create.argtypes = [C.c_int, ip, C.c_int, vp, C.POINTER(vp)]
    L.ocn_mlp_destroy.argtypes = [vp]
    L.ocn_mlp_destroy.restype = None
    L.ocn_mlp_arena_bytes.argtypes = [vp, C.POINTER(sz)]
    L.ocn_mlp_bind_arena.argtypes = [vp, vp, sz]
    L.ocn_mlp_num_params.argtypes = [vp, C.POINTER(sz)]
    L.ocn_mlp_set_params.argtypes = [vp, vp, sz, C.c_int]
    L.ocn_mlp_get_params.argtypes = [vp, vp, sz, C.c_int]
    L.ocn_mlp_forward.argtypes = [vp, vp, C.c_int, vp]
    L.ocn_mlp_gradients.argtypes = [vp, vp, vp, vp, C.c_int, vp, dp]
    L.ocn_mlp_adam.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, C.c_double]
    L.ocn_mlp_train_step.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double, dp]
    L.ocn_set_column_closure.argtypes = [vp, vp, C.POINTER(ColumnClosureDesc)]
    L.ocn_set_column_closure_mode.argtypes = [vp, C.c_int]
    L.ocn_set_time_stepper.argtypes = [vp, C.c_int, C.c_double]
    L.ocn_set_vertical_diffusivity.argtypes = [vp, dp, dp, C.c_int]
    L.ocn_closure_features.argtypes = [vp, C.c_double, vp]
    L.ocn_column_fluxes.argtypes = [vp, C.c_int, vp]
    L.ocn_coarse_grain.argtypes = [vp, C.c_int, C.c_int, vp, sz]
    L.ocn_gemm_timeout_test.argtypes = [vp, vp]
    L.ocn_fp32_fma_peak.argtypes = [dp, vp]
    L.ocn_gemm_bf16.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, C.c_int, vp, C.c_int, vp, vp]
    for name in EXPORTS:
        if name not in ("ocn_abi_version", "ocn_last_error", "ocn_grid_destroy", "ocn_model_destroy", "ocn_ensemble_destroy",
                        "ocn_mlp_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


@contextlib.contextmanager
def _stream_scope(device, stream):
    """Run the enclosed launches on the library's stream, ordered after everything the caller has
    already queued on its current stream (inputs it produced are ready), and order the caller's
    later work after them (outputs are ready for it)."""
    import torch
    caller = torch.cuda.current_stream(device)
    stream.wait_stream(caller)
    with torch.cuda.device(device), torch.cuda.stream(stream):
        yield caller
    caller.wait_stream(stream)


def _hand_over(t, caller):
    """A tensor made on the library's stream and returned: its memory is not reused before the
    caller's stream is done with it."""
    t.record_stream(caller)
    return t


def _check(st: int, where: str):
    if st != 0:
        raise OcnError(st, where, lib().ocn_last_error().decode())


class Grid:
    """RectilinearGrid: x, y periodic and uniform, z bounded with given face heights."""

    def __init__(self, Nx: int, Ny: int, Nz: int, Lx: float, Ly: float, z_faces):
        self.Nx, self.Ny, self.Nz, self.Lx, self.Ly = int(Nx), int(Ny), int(Nz), float(Lx), float(Ly)
        self._zf = np.ascontiguousarray(z_faces, dtype=np.float64)
        d = GridDesc(self.Nx, self.Ny, self.Nz, self.Lx, self.Ly, self._zf.ctypes.data_as(C.POINTER(C.c_double)))
        h = C.c_void_p()
        _check(lib().ocn_grid_create(C.byref(d), C.byref(h)), "ocn_grid_create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ocn_grid_destroy(self._h)
            self._h = None


def model_desc(p: dict) -> ModelDesc:
    """The C model descriptor of a workload dict."""
    d = ModelDesc()
    tracers = list(p.get("tracers", ["b"]))
    d.precision = int(p.get("precision", 32))
    d.weno_order = int(p.get("weno_order", 5))
    d.closure = CLOSURES[p.get("closure", "none")]
    d.nu, d.kappa = float(p.get("nu", 0.0)), float(p.get("kappa", 0.0))
    d.Cs, d.Cb, d.Pr = float(p.get("Cs", 0.16)), float(p.get("Cb", 1.0)), float(p.get("Pr", 1.0))
    d.C_amd = float(p.get("C_amd", 1.0 / 12.0))
    d.f = float(p.get("f", 0.0))
    d.n_tracers = len(tracers)
    d.eos = EOS[p.get("eos", "buoyancy_tracer")]
    d.g, d.alpha, d.beta = float(p.get("g", 9.81)), float(p.get("alpha", 2e-4)), float(p.get("beta", 8e-4))
    d.T0, d.S0 = float(p.get("T0", 20.0)), float(p.get("S0", 35.0))
    for n, name in enumerate(["u", "v"] + tracers):
        d.top_flux[n] = float(p.get("top_flux", {}).get(name, 0.0))
        d.bottom_flux[n] = float(p.get("bottom_flux", {}).get(name, 0.0))
    d.fp64_pivots = int(p.get("fp64_pivots", -1))
    return d


def shape_key(p: dict) -> list:
    """What a tendency tile choice depends on: grid size, precision, order, closure, tracer count."""
    return [int(p["Nx"]), int(p["Ny"]), int(p["Nz"]), int(p.get("precision", 32)), int(p.get("weno_order", 5)),
            str(p.get("closure", "none")), len(p.get("tracers", ["b"]))]


def _tuning_cache(path: str, key: str, value=None):
    """Read (value None) or write one entry of a JSON tuning cache; the file maps keys to choices."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    if value is None:
        return data.get(key)
    data[key] = value
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return value


def _device_name(device) -> str:
    import torch
    return torch.cuda.get_device_name(device)


def grid_desc(p: dict):
    zf = np.ascontiguousarray(p["z_faces"], dtype=np.float64)
    d = GridDesc(int(p["Nx"]), int(p["Ny"]), int(p["Nz"]), float(p["Lx"]), float(p["Ly"]),
                 zf.ctypes.data_as(C.POINTER(C.c_double)))
    return d, zf


class Model:
    """NonhydrostaticModel on the GPU.  ``params``: a workload dict (see inputs.config)."""

    def __init__(self, params: dict, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        p = dict(params)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._setup(p)
        self.grid = Grid(p["Nx"], p["Ny"], p["Nz"], p["Lx"], p["Ly"], p["z_faces"])
        d = model_desc(p)
        self._desc = d
        self._owner = True
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            h = C.c_void_p()
            _check(lib().ocn_model_create(self.grid._h, C.byref(d), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                   "ocn_model_create")
            self._h = h
            nbytes = C.c_size_t()
            _check(lib().ocn_model_arena_bytes(self._h, C.byref(nbytes)), "ocn_model_arena_bytes")
            self.arena_bytes = nbytes.value
            with torch.cuda.stream(self.stream):
                self.arena = torch.empty(self.arena_bytes, dtype=torch.uint8, device=self.device)
            _check(lib().ocn_model_bind_arena(self._h, C.c_void_p(self.arena.data_ptr()), self.arena_bytes),
                   "ocn_model_bind_arena")
        self._apply_schemes(p)

    def _apply_schemes(self, p: dict):
        """The workload keys for the time stepper and vertical diffusivities (as the oracle reads them)."""
        if p.get("timestepper", "rk3") != "rk3" or "chi" in p:
            self.set_time_stepper(p.get("timestepper", "rk3"), p.get("chi", 0.1))
        if p.get("nu_z") is not None or p.get("kappa_z") is not None:
            self.set_vertical_diffusivity(p.get("nu_z"), p.get("kappa_z"), bool(p.get("vertical_implicit", False)))

    def set_time_stepper(self, scheme: str = "rk3", chi: float = 0.1):
        _check(lib().ocn_set_time_stepper(self._h, STEPPERS[scheme], float(chi)), "ocn_set_time_stepper")
        self.params["timestepper"], self.params["chi"] = scheme, float(chi)

    def set_vertical_diffusivity(self, nu=None, kappa=None, implicit: bool = False):
        """Diffusivity profiles at the Nz+1 w-faces (scalars broadcast) for u, v, w (nu) and tracers (kappa)."""
        def arr(x):
            if x is None:
                return None, None
            a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), (self.Nz + 1,)))
            return a, a.ctypes.data_as(C.POINTER(C.c_double))
        a_nu, p_nu = arr(nu)
        a_ka, p_ka = arr(kappa)
        _check(lib().ocn_set_vertical_diffusivity(self._h, p_nu, p_ka, int(bool(implicit))),
               "ocn_set_vertical_diffusivity")

    def _setup(self, p: dict):
        import torch
        self.params = p
        self.tracers = list(p.get("tracers", ["b"]))
        self.precision = int(p.get("precision", 32))
        self.dtype = torch.float32 if self.precision == 32 else torch.float64
        self.np_dtype = np.float32 if self.precision == 32 else np.float64
        self.Nx, self.Ny, self.Nz = int(p["Nx"]), int(p["Ny"]), int(p["Nz"])

    @classmethod
    def borrowed(cls, handle, params: dict, device, stream, owner):
        """A handle owned by someone else (an ensemble member): never destroyed here."""
        m = cls.__new__(cls)
        m._setup(dict(params))
        m.device, m.stream, m._h, m._owner, m._keep = device, stream, handle, False, owner
        return m

    def __del__(self):
        if getattr(self, "_h", None) and getattr(self, "_owner", False):
            lib().ocn_model_destroy(self._h)
        self._h = None

    # ------------------------------------------------------------------ fields
    def fid(self, name: str) -> int:
        if name.startswith("G_"):
            return OCN_FIELD_G + self.fid(name[2:])
        if name.startswith("raw_"):
            return OCN_FIELD_RAW | self.fid(name[4:])
        if name.startswith("ref_"):
            return OCN_FIELD_TRACER_REF0 + self.tracers.index(name[4:])
        table = {"u": OCN_FIELD_U, "v": OCN_FIELD_V, "w": OCN_FIELD_W, "p": OCN_FIELD_P, "nu_e": OCN_FIELD_NU_E}
        if name in table:
            return table[name]
        return OCN_FIELD_TRACER0 + self.tracers.index(name)

    def shape(self, name: str):
        if name.startswith("ref_"):
            return (self.Nz,)
        if name.startswith("raw_"):
            name = name[4:]
        base = name[2:] if name.startswith("G_") else name
        return (self.Nz + 1 if base == "w" else self.Nz, self.Ny, self.Nx)

    def set(self, project: bool = True, **fields):
        """set!: copy fields in (numpy or torch); projects the velocity unless project=False."""
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            for name, arr in fields.items():
                t = torch.as_tensor(arr).to(device=self.device, dtype=self.dtype).contiguous()
                assert tuple(t.shape) == self.shape(name), (name, tuple(t.shape))
                _check(lib().ocn_set_field(self._h, self.fid(name), C.c_void_p(t.data_ptr()),
                                           t.numel() * t.element_size(), 1), "ocn_set_field")
                self.stream.synchronize()
        if project and any(k in fields for k in ("u", "v", "w")):
            self.project()

    def get(self, name: str):
        """A device tensor copy of a field."""
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            out = torch.empty(self.shape(name), dtype=self.dtype, device=self.device)
            _check(lib().ocn_get_field(self._h, self.fid(name), C.c_void_p(out.data_ptr()),
                                       out.numel() * out.element_size(), 1), "ocn_get_field")
        self.stream.synchronize()
        return _hand_over(out, caller)

    def get_numpy(self, name: str) -> np.ndarray:
        return self.get(name).cpu().numpy()

    def set_host(self, name: str, host_tensor):
        """Copy from (pinned) host memory through the C ABI's host path."""
        _check(lib().ocn_set_field(self._h, self.fid(name), C.c_void_p(host_tensor.data_ptr()),
                                   host_tensor.numel() * host_tensor.element_size(), 0), "ocn_set_field")

    def get_host(self, name: str, host_tensor):
        _check(lib().ocn_get_field(self._h, self.fid(name), C.c_void_p(host_tensor.data_ptr()),
                                   host_tensor.numel() * host_tensor.element_size(), 0), "ocn_get_field")

    def _many(self, tensors: dict):
        n = len(tensors)
        fids = (C.c_int * n)(*[self.fid(k) for k in tensors])
        ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in tensors.values()])
        nbytes = (C.c_size_t * n)(*[t.numel() * t.element_size() for t in tensors.values()])
        return n, fids, ptrs, nbytes

    def set_host_many(self, tensors: dict, wait: bool = True):
        """Copy several fields from (pinned) host memory in one call (ocn_set_fields); with
        wait=False the call only enqueues (OCN_HOST_ASYNC) and the tensors must stay unchanged
        until wait_transfers()."""
        n, fids, ptrs, nbytes = self._many(tensors)
        _check(lib().ocn_set_fields(self._h, n, fids, ptrs, nbytes, 0 if wait else OCN_HOST_ASYNC), "ocn_set_fields")

    def get_host_many(self, tensors: dict, wait: bool = True):
        """Copy several fields into (pinned) host memory in one call (ocn_get_fields); with
        wait=False the data is there once wait_transfers() has returned."""
        n, fids, ptrs, nbytes = self._many(tensors)
        _check(lib().ocn_get_fields(self._h, n, fids, ptrs, nbytes, 0 if wait else OCN_HOST_ASYNC), "ocn_get_fields")

    def wait_transfers(self):
        _check(lib().ocn_wait_transfers(self._h), "ocn_wait_transfers")

    def bounds_status(self):
        """(status word, checked): the out-of-range index bits recorded by the bounds-checked
        library variant since the last call (cleared by the call), and whether the loaded library
        is that variant."""
        st, chk = C.c_uint(0), C.c_int(0)
        _check(lib().ocn_bounds_status(self._h, C.byref(st), C.byref(chk)), "ocn_bounds_status")
        return int(st.value), bool(chk.value)

    def checkpoint(self) -> dict:
        """Device copies of everything a bitwise restart needs (state, raw tracer anomalies, profiles,
        and for QAB2 the previous tendencies, restored last)."""
        names = ["u", "v", "w"] + [f"raw_{t}" for t in self.tracers] + [f"ref_{t}" for t in self.tracers]
        if self.params.get("timestepper", "rk3") == "qab2":
            names += ["G_u", "G_v", "G_w"] + [f"G_{t}" for t in self.tracers]
        return {n: self.get(n).clone() for n in names}

    def restore(self, ckpt: dict):
        self.set(project=False, **ckpt)

    # ------------------------------------------------------------------ stepping
    def project(self):
        _check(lib().ocn_project(self._h), "ocn_project")

    def time_step(self, dt: float, nsteps: int = 1):
        """time_step!: nsteps RK3 steps (enqueued on the model stream)."""
        _check(lib().ocn_time_step(self._h, float(dt), int(nsteps)), "ocn_time_step")

    def compute_tendencies(self) -> dict:
        _check(lib().ocn_compute_tendencies(self._h), "ocn_compute_tendencies")
        return {n: self.get("G_" + n) for n in ["u", "v", "w"] + self.tracers}

    def diagnostics(self, dt: float = 0.0, check: bool = False) -> dict:
        nt = len(self.tracers)
        out = (C.c_double * (nt + 6))()
        st = lib().ocn_diagnostics(self._h, float(dt), out, nt + 6)
        if check or st not in (0, -4, -5):
            _check(st, "ocn_diagnostics")
        d = {f"sum_{t}": out[n] for n, t in enumerate(self.tracers)}
        d.update(sum_u=out[nt], sum_v=out[nt + 1], sum_w=out[nt + 2], max_div=out[nt + 3], cfl=out[nt + 4],
                 nonfinite=int(out[nt + 5]), status=STATUS.get(st, st))
        return d

    def set_option(self, option: int, value: int):
        _check(lib().ocn_set_option(self._h, int(option), int(value)), "ocn_set_option")

    def launches_per_step(self) -> int:
        n = C.c_int()
        _check(lib().ocn_launches_per_step(self._h, C.byref(n)), "ocn_launches_per_step")
        return n.value

    def profiles(self) -> dict:
        """Coarse-graining profiles: level means of b, u, v and mean face fluxes of b, u, v."""
        Nz = self.Nz
        out = (C.c_double * (3 * Nz + 3 * (Nz + 1)))()
        _check(lib().ocn_profiles(self._h, out, len(out)), "ocn_profiles")
        a = np.frombuffer(out, dtype=np.float64).copy()
        F = a[3 * Nz:]
        return {"b": a[:Nz], "u": a[Nz:2 * Nz], "v": a[2 * Nz:3 * Nz],
                "Fb": F[:Nz + 1], "Fu": F[Nz + 1:2 * (Nz + 1)], "Fv": F[2 * (Nz + 1):]}

    # ------------------------------------------------------------ learned column closure
    def set_column_closure(self, mlp, mu=None, sigma=None, out_scale=(1.0, 1.0, 1.0), N2_background=0.0,
                           mode=None):
        """Attach a trained network (an MLP of shape 32-128-128-128-16) as the learned column closure;
        mlp=None removes it (the model's own closure remains).  mode "flux" (explicit face fluxes)
        or "diffusivity" (outputs 0, 1 are eddy diffusivities applied by the implicit column solve);
        None keeps the current mode."""
        if mode is not None:
            _check(lib().ocn_set_column_closure_mode(self._h, {"flux": 0, "diffusivity": 1}[mode]),
                   "ocn_set_column_closure_mode")
        if mlp is None:
            _check(lib().ocn_set_column_closure(self._h, None, None), "ocn_set_column_closure")
            self._colc = None
            return
        d = ColumnClosureDesc()
        mu = np.zeros(COLUMN_FEATURES) if mu is None else np.asarray(mu, np.float64)
        sigma = np.ones(COLUMN_FEATURES) if sigma is None else np.asarray(sigma, np.float64)
        for q in range(COLUMN_FEATURES):
            d.mu[q] = float(mu[q]); d.sigma[q] = float(sigma[q])
        for q in range(3):
            d.out_scale[q] = float(out_scale[q])
        d.N2_background = float(N2_background)
        _check(lib().ocn_set_column_closure(self._h, mlp._h, C.byref(d)), "ocn_set_column_closure")
        self._colc = mlp          # keep the network alive while attached

    def closure_features(self, N2_background: float):
        """Raw column features of every w-face, a device tensor [(Nz+1)*Ny*Nx][32]."""
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            X = torch.empty(((self.Nz + 1) * self.Ny * self.Nx, COLUMN_FEATURES), dtype=torch.float32,
                            device=self.device)
            _check(lib().ocn_closure_features(self._h, float(N2_background), C.c_void_p(X.data_ptr())),
                   "ocn_closure_features")
        self.stream.synchronize()
        return _hand_over(X, caller)

    def column_fluxes(self, learned: bool = False):
        """Face fluxes of b, ubar, vbar [3][Nz+1][Ny][Nx]: the model's closure (default) or the learned one."""
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            F = torch.empty((3, self.Nz + 1, self.Ny, self.Nx), dtype=torch.float32, device=self.device)
            _check(lib().ocn_column_fluxes(self._h, 1 if learned else 0, C.c_void_p(F.data_ptr())),
                   "ocn_column_fluxes")
        self.stream.synchronize()
        return _hand_over(F, caller)

    def coarse_grain(self, cx: int, cy: int) -> dict:
        """Box filter onto cx x cy columns: coarse u, v, w, b and subfilter fluxes tau [3][Nz+1][cy][cx]
        (device FP64 tensors)."""
        import torch
        Nz = self.Nz
        n = cx * cy
        with _stream_scope(self.device, self.stream) as caller:
            out = torch.empty(n * (7 * Nz + 4), dtype=torch.float64, device=self.device)
            _check(lib().ocn_coarse_grain(self._h, int(cx), int(cy), C.c_void_p(out.data_ptr()), out.numel()),
                   "ocn_coarse_grain")
        self.stream.synchronize()
        _hand_over(out, caller)
        res, o = {}, 0
        for name, levels in (("u", Nz), ("v", Nz), ("w", Nz + 1), ("b", Nz)):
            res[name] = out[o:o + levels * n].view(levels, cy, cx); o += levels * n
        res["tau"] = out[o:].view(3, Nz + 1, cy, cx)
        return res

    def kernel_times(self) -> dict:
        """{kernel class: (launches, summed ms)} recorded while OCN_OPT_KERNEL_TIMING is on."""
        n = len(KERNEL_CLASSES)
        counts = (C.c_int * n)()
        ms = (C.c_double * n)()
        _check(lib().ocn_kernel_times(self._h, counts, ms), "ocn_kernel_times")
        return {k: (counts[i], ms[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def autotune(self, cache: str = None):
        """Time every tendency tile variant on the current state, keep the fastest.
        Returns (best index, [ms per launch of each variant]).  With ``cache`` (a JSON file path)
        a choice stored there for this device and model shape is applied without timing (ms is
        then None), and a new choice is stored."""
        key = json.dumps(["model", lib().ocn_abi_version(), _device_name(self.device), shape_key(self.params)])
        if cache:
            v = _tuning_cache(cache, key)
            if v is not None:
                self.set_option(OCN_OPT_TENDENCY_VARIANT, int(v))
                return int(v), None
        best = C.c_int()
        ms = (C.c_double * TENDENCY_VARIANTS)()
        _check(lib().ocn_autotune(self._h, C.byref(best), ms), "ocn_autotune")
        if cache:
            _tuning_cache(cache, key, best.value)
        return best.value, list(ms)

    def synchronize(self):
        self.stream.synchronize()


def regrid(zf_in, values, zf_out) -> np.ndarray:
    """Conservative regridding of cell averages between ascending face lists (library host code)."""
    dp = C.POINTER(C.c_double)
    zi = np.ascontiguousarray(zf_in, dtype=np.float64); v = np.ascontiguousarray(values, dtype=np.float64)
    zo = np.ascontiguousarray(zf_out, dtype=np.float64); out = np.zeros(zo.size - 1)
    _check(lib().ocn_regrid(zi.ctypes.data_as(dp), v.size, v.ctypes.data_as(dp), zo.ctypes.data_as(dp), out.size,
                            out.ctypes.data_as(dp)), "ocn_regrid")
    return out


class Ensemble:
    """Many independent members (uneven sizes and forcings) stepped together on one GPU."""

    def __init__(self, params_list, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.params = [dict(p) for p in params_list]
        self._mode, self._branches = "concurrent", 4
        n = len(self.params)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        grids = (GridDesc * n)()
        models = (ModelDesc * n)()
        self._zf = []
        for i, p in enumerate(self.params):
            gd, zf = grid_desc(p)
            self._zf.append(zf)
            grids[i] = gd
            models[i] = model_desc(p)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            h = C.c_void_p()
            _check(lib().ocn_ensemble_create(n, grids, models, C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                   "ocn_ensemble_create")
            self._h = h
            nb = C.c_size_t()
            _check(lib().ocn_ensemble_arena_bytes(self._h, C.byref(nb)), "ocn_ensemble_arena_bytes")
            self.arena_bytes = nb.value
            with torch.cuda.stream(self.stream):
                self.arena = torch.empty(self.arena_bytes, dtype=torch.uint8, device=self.device)
            _check(lib().ocn_ensemble_bind_arena(self._h, C.c_void_p(self.arena.data_ptr()), self.arena_bytes),
                   "ocn_ensemble_bind_arena")
        self.members = []
        for i, p in enumerate(self.params):
            mh = C.c_void_p()
            _check(lib().ocn_ensemble_member(self._h, i, C.byref(mh)), "ocn_ensemble_member")
            member = Model.borrowed(mh, p, self.device, self.stream, self)
            member._apply_schemes(p)
            self.members.append(member)

    def __del__(self):
        if getattr(self, "_h", None):
            for m in getattr(self, "members", []):
                m._h = None
            lib().ocn_ensemble_destroy(self._h)
            self._h = None

    def time_step(self, dt: float, nsteps: int = 1):
        _check(lib().ocn_ensemble_time_step(self._h, float(dt), int(nsteps)), "ocn_ensemble_time_step")

    def set_mode(self, mode: str = None, sequential: bool = None):
        """'concurrent' (one graph per step, a branch per member), 'batched' (one graph per step,
        each kernel one launch over all members) or 'sequential' (members one after another);
        ``sequential=True/False`` selects 'sequential' / 'concurrent'."""
        if mode is None:
            mode = "sequential" if sequential else "concurrent"
        if mode not in ENSEMBLE_MODES:
            raise ValueError(f"unknown ensemble mode {mode!r}")
        _check(lib().ocn_ensemble_set_option(self._h, OCN_OPT_ENSEMBLE_MODE, ENSEMBLE_MODES[mode]),
               "ocn_ensemble_set_option")
        self._mode = mode

    def set_branches(self, n: int):
        """Batched mode: split each group of members into n graph branches (1..64)."""
        _check(lib().ocn_ensemble_set_option(self._h, OCN_OPT_ENSEMBLE_BRANCHES, int(n)), "ocn_ensemble_set_option")
        self._branches = int(n)

    def autotune(self, cache: str = None):
        """Choose the members' tendency tile variants in context (see ocn_ensemble_autotune); returns
        them.  With ``cache`` (a JSON file path) the choices stored there for this device, mode,
        branch count and member list are applied without timing, and new choices are stored."""
        key = json.dumps(["ensemble", lib().ocn_abi_version(), _device_name(self.device), self._mode, self._branches,
                          [shape_key(p) for p in self.params]])
        if cache:
            v = _tuning_cache(cache, key)
            if v is not None and len(v) == len(self.members):
                for m, x in zip(self.members, v):
                    m.set_option(OCN_OPT_TENDENCY_VARIANT, int(x))
                return [int(x) for x in v]
        v = (C.c_int * len(self.members))()
        _check(lib().ocn_ensemble_autotune(self._h, v), "ocn_ensemble_autotune")
        if cache:
            _tuning_cache(cache, key, list(v))
        return list(v)

    def launches_per_step(self) -> int:
        n = C.c_int()
        _check(lib().ocn_ensemble_launches_per_step(self._h, C.byref(n)), "ocn_ensemble_launches_per_step")
        return n.value

    def synchronize(self):
        self.stream.synchronize()


def gemm_bf16(A, B, status=None, stream=None):
    """D = A B^T on the tensor cores (A [M][K], B [N][K] BF16 CUDA tensors) -> FP32 [M][N]."""
    import torch
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
    A, B = A.contiguous(), B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    _check(lib().ocn_gemm_bf16(M, N, K, C.c_void_p(A.data_ptr()), K, C.c_void_p(B.data_ptr()), K,
                               C.c_void_p(D.data_ptr()), N,
                               C.c_void_p(status.data_ptr()) if status is not None else None,
                               C.c_void_p(s.cuda_stream)), "ocn_gemm_bf16")
    return D


class MLP:
    """The learned column closure's network on the tensor cores (see ocn_mlp_* in include/ocn.h)."""

    def __init__(self, sizes, max_batch: int, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.sizes = tuple(int(x) for x in sizes)
        self.max_batch = int(max_batch)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            arr = (C.c_int * len(self.sizes))(*self.sizes)
            h = C.c_void_p()
            _check(lib().ocn_mlp_create(len(self.sizes) - 1, arr, self.max_batch, C.c_void_p(self.stream.cuda_stream),
                                        C.byref(h)), "ocn_mlp_create")
            self._h = h
            nb = C.c_size_t()
            _check(lib().ocn_mlp_arena_bytes(self._h, C.byref(nb)), "ocn_mlp_arena_bytes")
            with torch.cuda.stream(self.stream):
                self.arena = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
            base = self.arena.data_ptr()
            aligned = (base + 255) // 256 * 256
            _check(lib().ocn_mlp_bind_arena(self._h, C.c_void_p(aligned), nb.value), "ocn_mlp_bind_arena")
            n = C.c_size_t()
            _check(lib().ocn_mlp_num_params(self._h, C.byref(n)), "ocn_mlp_num_params")
            self.nparams = n.value

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ocn_mlp_destroy(self._h)
            self._h = None

    @staticmethod
    def flatten(params) -> np.ndarray:
        """[(W_l [n_out][n_in], b_l)] -> the flat FP32 parameter layout."""
        return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32)])
                               for W, b in params]).astype(np.float32)

    def unflatten(self, flat) -> list:
        out, o = [], 0
        for l in range(len(self.sizes) - 1):
            ni, no = self.sizes[l], self.sizes[l + 1]
            W = np.asarray(flat[o:o + no * ni]).reshape(no, ni); o += no * ni
            b = np.asarray(flat[o:o + no]); o += no
            out.append((W, b))
        return out

    def set_params(self, params):
        flat = np.ascontiguousarray(self.flatten(params) if isinstance(params, (list, tuple)) else params,
                                    dtype=np.float32)
        assert flat.size == self.nparams
        _check(lib().ocn_mlp_set_params(self._h, C.c_void_p(flat.ctypes.data), flat.size, 0), "ocn_mlp_set_params")

    def get_params(self) -> list:
        flat = np.zeros(self.nparams, dtype=np.float32)
        _check(lib().ocn_mlp_get_params(self._h, C.c_void_p(flat.ctypes.data), flat.size, 0), "ocn_mlp_get_params")
        return self.unflatten(flat)

    def _dev(self, a):
        import torch
        return torch.as_tensor(a).to(device=self.device, dtype=torch.float32).contiguous()

    def forward(self, X):
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            X = self._dev(X)
            Y = torch.empty((X.shape[0], self.sizes[-1]), dtype=torch.float32, device=self.device)
            _check(lib().ocn_mlp_forward(self._h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(Y.data_ptr())),
                   "ocn_mlp_forward")
        self.stream.synchronize()
        return _hand_over(Y, caller)

    def gradients(self, X, T, mask):
        """(loss, flat FP32 gradient tensor) of the masked mean-square loss."""
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            X, T, m = self._dev(X), self._dev(T), self._dev(mask)
            g = torch.empty(self.nparams, dtype=torch.float32, device=self.device)
            loss = C.c_double()
            _check(lib().ocn_mlp_gradients(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                           C.c_void_p(m.data_ptr()), X.shape[0], C.c_void_p(g.data_ptr()),
                                           C.byref(loss)), "ocn_mlp_gradients")
        return loss.value, _hand_over(g, caller)

    def adam(self, grads, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            g = self._dev(grads)
            _check(lib().ocn_mlp_adam(self._h, C.c_void_p(g.data_ptr()), float(lr), float(beta1), float(beta2),
                                      float(eps)), "ocn_mlp_adam")
            self.stream.synchronize()

    def train_step(self, X, T, mask, lr) -> float:
        """One Adam step on (X, T) (device tensors or arrays); returns the loss before the step."""
        import torch
        with _stream_scope(self.device, self.stream) as caller:
            X, T, m = self._dev(X), self._dev(T), self._dev(mask)
            loss = C.c_double()
            _check(lib().ocn_mlp_train_step(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                            C.c_void_p(m.data_ptr()), X.shape[0], float(lr), C.byref(loss)),
                   "ocn_mlp_train_step")
        return loss.value


def fp32_fma_peak(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device (TFLOP/s, FMA = 2 flops)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    _check(lib().ocn_fp32_fma_peak(C.byref(out), C.c_void_p(s.cuda_stream)), "ocn_fp32_fma_peak")
    return out.value
