"""ctypes binding of the C ABI in include/fsolve.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and does
nothing but convert arguments: torch tensors become device pointers
(``data_ptr()``), a torch stream (or None = the current stream) becomes a
``cudaStream_t``, and a non-zero ``fs_status`` becomes an ``FsError`` carrying
``fs_last_error()``.  All computation happens in ``libfsolve.so``.  There is no
fallback: if the library is missing, ``load()`` raises.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsolve.so")

FS_F32 = 0
FS_F64 = 1

FS_OK = 0
STATUS_NAMES = {
    0: "FS_OK", -1: "FS_ERR_ARG", -2: "FS_ERR_SIZE", -3: "FS_ERR_NOMEM", -4: "FS_ERR_BUDGET",
    -5: "FS_ERR_CUDA", -6: "FS_ERR_TIMEOUT", -7: "FS_ERR_BUSY", -8: "FS_ERR_NODEV",
}

FS_OP_POISSON = 0
FS_OP_DIFFUSION = 1
FS_OP_WAVE = 2
FS_OP_DIFFUSION_ADVANCE = 3
FS_OP_WAVE_ADVANCE = 4

_vp = ctypes.c_void_p


class FsRequest(ctypes.Structure):
    """struct fs_request of include/fsolve.h."""

    _fields_ = [("op", ctypes.c_int), ("plan", _vp), ("state", _vp), ("in_u", _vp), ("in_v", _vp),
                ("out_u", _vp), ("out_v", _vp), ("D", ctypes.c_double), ("c", ctypes.c_double),
                ("t", ctypes.c_double), ("keep", ctypes.c_int), ("parent", ctypes.c_uint64)]


class FsOrbitSource(ctypes.Structure):
    """fs_orbit_source of include/fsolve.h."""

    _fields_ = [("A", ctypes.c_double), ("sigma", ctypes.c_double), ("radius", ctypes.c_double),
                ("Omega", ctypes.c_double), ("gamma", ctypes.c_double), ("x_min", ctypes.c_double),
                ("y_min", ctypes.c_double)]


class FsTuneResult(ctypes.Structure):
    """fs_tune_result of include/fsolve.h."""

    _fields_ = [("e_row", ctypes.c_int), ("e_col", ctypes.c_int), ("rows", ctypes.c_int), ("cols", ctypes.c_int),
                ("us_default", ctypes.c_double), ("us_tuned", ctypes.c_double), ("candidates", ctypes.c_int)]


# Entry points declared in include/fsolve.h: name -> (restype, argtypes)
_SIGS = {
    "fs_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.POINTER(_vp)]),
    "fs_plan_destroy": (ctypes.c_int, [_vp]),
    "fs_plan_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_size_t)]),
    "fs_tune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_int, ctypes.POINTER(FsTuneResult)]),
    "fs_tune_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.POINTER(FsTuneResult)]),
    "fs_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "fs_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "fs_tune_cache_clear": (ctypes.c_int, []),
    "fs_plan_tiles": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "fs_poisson_solve": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "fs_poisson_solve_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               _vp, _vp, _vp]),
    "fs_diffusion_solve": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "fs_wave_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "fs_operator_factors": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, _vp, _vp]),
    "fs_rows_forward": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "fs_columns_apply": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "fs_rows_inverse": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "fs_poisson_solve_c": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "fs_diffusion_solve_c": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "fs_wave_solve_c": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "fs_state_create": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "fs_state_destroy": (ctypes.c_int, [_vp]),
    "fs_state_reset": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "fs_state_set_source": (ctypes.c_int, [_vp, _vp, _vp]),
    "fs_state_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "fs_state_save": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    "fs_state_load": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    "fs_diffusion_advance": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "fs_wave_advance": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp]),
    "fs_rk4_create": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.POINTER(FsOrbitSource), _vp, _vp,
                                     ctypes.c_double, _vp, ctypes.POINTER(_vp)]),
    "fs_rk4_step": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _vp]),
    "fs_rk4_output": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "fs_rk4_mean": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "fs_rk4_time": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "fs_rk4_destroy": (ctypes.c_int, [_vp]),
    "fs_batch_submit": (ctypes.c_int, [ctypes.POINTER(FsRequest), ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                       _vp]),
    "fs_batch_wait": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int]),
    "fs_serve_start": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
    "fs_serve_enqueue": (ctypes.c_int, [ctypes.POINTER(FsRequest), ctypes.POINTER(ctypes.c_uint64)]),
    "fs_serve_replay": (ctypes.c_int, [ctypes.POINTER(FsRequest), ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "fs_serve_poll": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.c_int]),
    "fs_serve_latency": (ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "fs_serve_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
    "fs_serve_stop": (ctypes.c_int, []),
    "fs_last_error": (ctypes.c_char_p, []),
    "fs_size_supported": (ctypes.c_int, [ctypes.c_int]),
    "fs_radix_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "fs_kernel_launches": (ctypes.c_uint64, []),
    "fs_device_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "fs_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "fs_profile_report": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int]),
}

PROFILE_CLASSES = ("row_r2c", "column", "row_c2r", "factor", "small", "batch")

_lib = None


class FsError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def load(path=None):
    """Load libfsolve.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C entry points this binding marshals."""
    return sorted(_SIGS)


def _check(status, where):
    if status != FS_OK:
        msg = _lib.fs_last_error()
        raise FsError(status, where, msg.decode() if msg else "")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return ctypes.c_void_p(t.data_ptr())


# Geometry of the handles this binding created: plan -> (nx, ny, dtype), and
# state / RK4 integrator -> its plan, so that every field argument can be
# checked against the grid before its pointer reaches the library.
_plans = {}
_owner = {}


def _key(h):
    return h.value if isinstance(h, ctypes.c_void_p) else h


def _plan_geom(plan):
    """(nx, ny, dtype) of a plan this binding created, else None (unchecked)."""
    return _plans.get(_key(plan))


def _owner_geom(h):
    plan = _owner.get(_key(h))
    return None if plan is None else _plan_geom(plan)


def _torch_dtype(dtype, cplx):
    import torch

    return {(FS_F32, False): torch.float32, (FS_F64, False): torch.float64,
            (FS_F32, True): torch.complex64, (FS_F64, True): torch.complex128}[(dtype, bool(cplx))]


def _field(t, geom, where, name, cplx=False):
    """Device pointer of a field argument, after checking that the tensor is a
    contiguous [ny][nx] field of the plan's element type in device memory (or
    host memory pinned by CUDA); raw integer pointers are passed unchecked."""
    if t is None or isinstance(t, int) or geom is None:
        return _ptr(t)
    nx, ny, dtype = geom
    want = _torch_dtype(dtype, cplx)
    bad = None
    if t.dtype != want:
        bad = f"dtype {t.dtype}, the plan needs {want}"
    elif t.numel() != nx * ny:
        bad = f"{t.numel()} elements, the grid has {ny} x {nx}"
    elif not t.is_contiguous():
        bad = "not contiguous"
    elif not (t.is_cuda or t.is_pinned()):
        bad = "neither device memory nor pinned host memory"
    if bad:
        raise FsError(-1, where, f"{name}: {bad}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(s):
    if s is None:
        import torch

        s = torch.cuda.current_stream()
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ entry points
def fs_plan_create(nx, ny, lx, ly, dtype):
    load()
    h = _vp()
    _check(_lib.fs_plan_create(int(nx), int(ny), float(lx), float(ly), int(dtype), ctypes.byref(h)),
           "fs_plan_create")
    _plans[h.value] = (int(nx), int(ny), int(dtype))
    return h


def fs_plan_destroy(plan):
    load()
    _check(_lib.fs_plan_destroy(plan), "fs_plan_destroy")
    _plans.pop(_key(plan), None)


def fs_plan_info(plan):
    load()
    nx, ny, dt, path = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ws = ctypes.c_size_t()
    _check(_lib.fs_plan_info(plan, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(dt),
                             ctypes.byref(path), ctypes.byref(ws)), "fs_plan_info")
    return {"nx": nx.value, "ny": ny.value, "dtype": dt.value, "path": path.value,
            "workspace_bytes": ws.value}


def fs_poisson_solve(plan, f, u, stream=None):
    load()
    g, w = _plan_geom(plan), "fs_poisson_solve"
    _check(_lib.fs_poisson_solve(plan, _field(f, g, w, "f"), _field(u, g, w, "u"), _stream(stream)), w)


def fs_poisson_solve_static(nx, ny, lx, ly, f, u, stream=None):
    load()
    g, w = (int(nx), int(ny), FS_F32), "fs_poisson_solve_static"
    _check(_lib.fs_poisson_solve_static(int(nx), int(ny), float(lx), float(ly), _field(f, g, w, "f"),
                                        _field(u, g, w, "u"), _stream(stream)), w)


def fs_diffusion_solve(plan, u0, D, t, u, stream=None):
    load()
    g, w = _plan_geom(plan), "fs_diffusion_solve"
    _check(_lib.fs_diffusion_solve(plan, _field(u0, g, w, "u0"), float(D), float(t), _field(u, g, w, "u"),
                                   _stream(stream)), w)


def fs_wave_solve(plan, u0, v0, c, t, u, stream=None):
    load()
    g, w = _plan_geom(plan), "fs_wave_solve"
    _check(_lib.fs_wave_solve(plan, _field(u0, g, w, "u0"), _field(v0, g, w, "v0"), float(c), float(t),
                              _field(u, g, w, "u"), _stream(stream)), w)


def fs_tune(nx, ny, lx, ly, dtype, reps=10):
    """Autotune a grid's passes on this GPU; returns the chosen configuration."""
    load()
    r = FsTuneResult()
    _check(_lib.fs_tune(int(nx), int(ny), float(lx), float(ly), int(dtype), int(reps), ctypes.byref(r)), "fs_tune")
    return {k: getattr(r, k) for k, _ in FsTuneResult._fields_}


def fs_tune_batch(nx, ny, lx, ly, dtype, nprob=8, reps=5):
    """Autotune a grid's register tiles inside a batch; returns the chosen pair."""
    load()
    r = FsTuneResult()
    _check(_lib.fs_tune_batch(int(nx), int(ny), float(lx), float(ly), int(dtype), int(nprob), int(reps),
                              ctypes.byref(r)), "fs_tune_batch")
    return {k: getattr(r, k) for k, _ in FsTuneResult._fields_}


def fs_tune_cache_load(path):
    load()
    return _lib.fs_tune_cache_load(os.fsencode(path))


def fs_tune_cache_save(path):
    load()
    return _lib.fs_tune_cache_save(os.fsencode(path))


def fs_tune_cache_clear():
    load()
    return _lib.fs_tune_cache_clear()


def fs_plan_tiles(plan):
    """(e_row, e_col, rows, cols) of a plan."""
    load()
    v = [ctypes.c_int() for _ in range(4)]
    _check(_lib.fs_plan_tiles(plan, *[ctypes.byref(x) for x in v]), "fs_plan_tiles")
    return tuple(x.value for x in v)


def _slab(t, n, dtype, cplx, where, name):
    """Pointer of a slab buffer with n elements of the plan's type (checked
    like whole fields; raw integers pass unchecked)."""
    return _field(t, None if dtype is None else (n, 1, dtype), where, name, cplx)


def fs_operator_factors(plan, op, out, D=0.0, c=0.0, t=0.0, fp64=False, stream=None):
    """The FP32 column pass's multiplier for every half-spectrum element into
    out [nx/2+1][ny] (float32); fp64=True evaluates it in FP64 instead."""
    load()
    g, w = _plan_geom(plan), "fs_operator_factors"
    n = (g[0] // 2 + 1) * g[1] if g else 0
    _check(_lib.fs_operator_factors(plan, int(op), float(D), float(c), float(t), 1 if fp64 else 0,
                                    _slab(out, n, g[2] if g else None, False, w, "out"), _stream(stream)), w)


def fs_rows_forward(plan, nrows, f, spec, stream=None):
    """x transforms of nrows real rows f [nrows][nx] -> spec [nx/2+1][nrows] (complex)."""
    load()
    g, w = _plan_geom(plan), "fs_rows_forward"
    nx, dt = (g[0], g[2]) if g else (None, None)
    _check(_lib.fs_rows_forward(plan, int(nrows), _slab(f, (nx or 0) * nrows, dt, False, w, "f"),
                                _slab(spec, ((nx or 0) // 2 + 1) * nrows, dt, True, w, "spec"), _stream(stream)), w)


def fs_columns_apply(plan, a0, ncols, op, spec_cols, D=0.0, c=0.0, t=0.0, stream=None):
    """Forward y transform, operator, inverse y transform of the x frequencies
    a0 .. a0+ncols-1; spec_cols [ncols][ny] (complex), in place."""
    load()
    g, w = _plan_geom(plan), "fs_columns_apply"
    ny, dt = (g[1], g[2]) if g else (None, None)
    _check(_lib.fs_columns_apply(plan, int(a0), int(ncols), int(op), float(D), float(c), float(t),
                                 _slab(spec_cols, (ny or 0) * ncols, dt, True, w, "spec_cols"), _stream(stream)), w)


def fs_rows_inverse(plan, nrows, spec, u, stream=None):
    """Inverse x transforms of spec [nx/2+1][nrows] (complex) -> real rows u [nrows][nx]."""
    load()
    g, w = _plan_geom(plan), "fs_rows_inverse"
    nx, dt = (g[0], g[2]) if g else (None, None)
    _check(_lib.fs_rows_inverse(plan, int(nrows), _slab(spec, ((nx or 0) // 2 + 1) * nrows, dt, True, w, "spec"),
                                _slab(u, (nx or 0) * nrows, dt, False, w, "u"), _stream(stream)), w)


def fs_poisson_solve_c(plan, f, u, stream=None):
    """Complex fields: f, u are complex64/complex128 tensors [ny][nx]."""
    load()
    g, w = _plan_geom(plan), "fs_poisson_solve_c"
    _check(_lib.fs_poisson_solve_c(plan, _field(f, g, w, "f", True), _field(u, g, w, "u", True),
                                   _stream(stream)), w)


def fs_diffusion_solve_c(plan, u0, D, t, u, stream=None):
    load()
    g, w = _plan_geom(plan), "fs_diffusion_solve_c"
    _check(_lib.fs_diffusion_solve_c(plan, _field(u0, g, w, "u0", True), float(D), float(t),
                                     _field(u, g, w, "u", True), _stream(stream)), w)


def fs_wave_solve_c(plan, u0, v0, c, t, u, stream=None):
    load()
    g, w = _plan_geom(plan), "fs_wave_solve_c"
    _check(_lib.fs_wave_solve_c(plan, _field(u0, g, w, "u0", True), _field(v0, g, w, "v0", True), float(c),
                                float(t), _field(u, g, w, "u", True), _stream(stream)), w)


def fs_state_create(plan, u0, v0=None, stream=None):
    load()
    h = _vp()
    g, w = _plan_geom(plan), "fs_state_create"
    _check(_lib.fs_state_create(plan, _field(u0, g, w, "u0"), _field(v0, g, w, "v0"), _stream(stream),
                                ctypes.byref(h)), w)
    _owner[h.value] = plan
    return h


def fs_state_destroy(state):
    load()
    _check(_lib.fs_state_destroy(state), "fs_state_destroy")
    _owner.pop(_key(state), None)


def fs_state_reset(state, u0, v0=None, stream=None):
    load()
    g, w = _owner_geom(state), "fs_state_reset"
    _check(_lib.fs_state_reset(state, _field(u0, g, w, "u0"), _field(v0, g, w, "v0"), _stream(stream)), w)


def fs_state_set_source(state, s, stream=None):
    """Attach a constant source field (None detaches it) to a kept state."""
    load()
    g, w = _owner_geom(state), "fs_state_set_source"
    _check(_lib.fs_state_set_source(state, _field(s, g, w, "s"), _stream(stream)), w)


def fs_rk4_create(plan, c, src, u0=None, v0=None, t0=0.0, stream=None):
    """RK4 integrator of the wave equation with an orbiting source.

    `src` has the fields of fs_orbit_source (e.g. workloads.OrbitSource)."""
    load()
    s = FsOrbitSource(float(src.A), float(src.sigma), float(src.radius), float(src.Omega), float(src.gamma),
                      float(src.x_min), float(src.y_min))
    h = _vp()
    g, w = _plan_geom(plan), "fs_rk4_create"
    _check(_lib.fs_rk4_create(plan, float(c), ctypes.byref(s), _field(u0, g, w, "u0"), _field(v0, g, w, "v0"),
                              float(t0), _stream(stream), ctypes.byref(h)), w)
    _owner[h.value] = plan
    return h


def fs_rk4_step(rk, dt, nsteps, stream=None):
    load()
    _check(_lib.fs_rk4_step(rk, float(dt), int(nsteps), _stream(stream)), "fs_rk4_step")


def fs_rk4_output(rk, u_out, v_out=None, stream=None):
    load()
    g, w = _owner_geom(rk), "fs_rk4_output"
    _check(_lib.fs_rk4_output(rk, _field(u_out, g, w, "u_out"), _field(v_out, g, w, "v_out"), _stream(stream)), w)


def fs_rk4_mean(rk, stream=None):
    load()
    m = ctypes.c_double()
    _check(_lib.fs_rk4_mean(rk, ctypes.byref(m), _stream(stream)), "fs_rk4_mean")
    return m.value


def fs_rk4_time(rk):
    load()
    t = ctypes.c_double()
    _check(_lib.fs_rk4_time(rk, ctypes.byref(t)), "fs_rk4_time")
    return t.value


def fs_rk4_destroy(rk):
    load()
    _check(_lib.fs_rk4_destroy(rk), "fs_rk4_destroy")
    _owner.pop(_key(rk), None)


def fs_state_save(state, stream=None):
    """Checkpoint of a kept state as bytes (host memory)."""
    load()
    n = ctypes.c_size_t()
    _check(_lib.fs_state_bytes(state, ctypes.byref(n)), "fs_state_bytes")
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.fs_state_save(state, buf, n.value, _stream(stream)), "fs_state_save")
    return buf.raw


def fs_state_load(state, data, stream=None):
    """Restore a checkpoint (bytes from fs_state_save) into a compatible state."""
    load()
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(_lib.fs_state_load(state, buf, len(data), _stream(stream)), "fs_state_load")


def fs_diffusion_advance(state, D, t, u_out, stream=None):
    load()
    g, w = _owner_geom(state), "fs_diffusion_advance"
    _check(_lib.fs_diffusion_advance(state, float(D), float(t), _field(u_out, g, w, "u_out"), _stream(stream)), w)


def fs_wave_advance(state, c, t, u_out, v_out=None, stream=None):
    load()
    g, w = _owner_geom(state), "fs_wave_advance"
    _check(_lib.fs_wave_advance(state, float(c), float(t), _field(u_out, g, w, "u_out"),
                                _field(v_out, g, w, "v_out"), _stream(stream)), w)


def fs_request(op, plan=None, state=None, in_u=None, in_v=None, out_u=None, out_v=None, D=0.0, c=0.0, t=0.0,
               keep=0, parent=0):
    """Marshal one batch / serving request (tensors -> device pointers)."""

    geom = _plan_geom(plan) if plan is not None else (_owner_geom(state) if state is not None else None)

    def p(x, name):
        v = _field(x, geom, "fs_request", name)
        return v.value if isinstance(v, ctypes.c_void_p) else v

    return FsRequest(int(op), plan, state, p(in_u, "in_u"), p(in_v, "in_v"), p(out_u, "out_u"), p(out_v, "out_v"),
                     float(D), float(c), float(t), int(keep), int(parent))


def fs_request_array(reqs):
    """Marshal a list of FsRequest once into a C array (reusable across submits)."""
    return (FsRequest * len(reqs))(*reqs)


def fs_batch_submit(reqs, stream=None):
    """Submit a list of FsRequest (or an array from fs_request_array); returns the ticket."""
    load()
    arr = reqs if isinstance(reqs, ctypes.Array) else (FsRequest * len(reqs))(*reqs)
    ticket = ctypes.c_uint64()
    _check(_lib.fs_batch_submit(arr, len(reqs), ctypes.byref(ticket), _stream(stream)), "fs_batch_submit")
    return ticket.value


def fs_batch_wait(ticket, timeout_us=-1):
    load()
    _check(_lib.fs_batch_wait(ctypes.c_uint64(ticket), int(timeout_us)), "fs_batch_wait")


SERVE_STATS = ("batches", "completed", "max_in_flight", "overlapped_batches", "peak_bytes", "bytes_used",
               "queued", "kept", "failed")


def fs_serve_start(hbm_budget_bytes, slots=2, max_batch=64):
    load()
    _check(_lib.fs_serve_start(int(hbm_budget_bytes), int(slots), int(max_batch)), "fs_serve_start")


def fs_serve_enqueue(req):
    load()
    t = ctypes.c_uint64()
    _check(_lib.fs_serve_enqueue(ctypes.byref(req), ctypes.byref(t)), "fs_serve_enqueue")
    return t.value


def fs_serve_replay(reqs, arrival_s):
    """Open-loop driver: enqueue reqs[i] at arrival_s[i] s; returns the tickets."""
    load()
    n = len(reqs)
    arr = (FsRequest * n)(*reqs)
    ts = (ctypes.c_double * n)(*[float(x) for x in arrival_s])
    out = (ctypes.c_uint64 * n)()
    _check(_lib.fs_serve_replay(arr, ts, n, out), "fs_serve_replay")
    return [out[i] for i in range(n)]


def fs_serve_poll(cap=1024, timeout_us=0):
    """Finished tickets (possibly empty)."""
    load()
    buf = (ctypes.c_uint64 * cap)()
    n = ctypes.c_int()
    st = _lib.fs_serve_poll(buf, cap, ctypes.byref(n), int(timeout_us))
    if st not in (FS_OK, -6):
        _check(st, "fs_serve_poll")
    return [buf[i] for i in range(n.value)]


def fs_serve_latency(ticket):
    load()
    v = ctypes.c_double()
    _check(_lib.fs_serve_latency(ctypes.c_uint64(ticket), ctypes.byref(v)), "fs_serve_latency")
    return v.value


def fs_serve_stats():
    load()
    n = len(SERVE_STATS)
    buf = (ctypes.c_uint64 * n)()
    _check(_lib.fs_serve_stats(buf, n), "fs_serve_stats")
    return {SERVE_STATS[i]: int(buf[i]) for i in range(n)}


def fs_serve_stop():
    load()
    _check(_lib.fs_serve_stop(), "fs_serve_stop")


def fs_last_error():
    load()
    m = _lib.fs_last_error()
    return m.decode() if m else ""


def fs_size_supported(n):
    load()
    return bool(_lib.fs_size_supported(int(n)))


def fs_radix_plan(L, e):
    load()
    buf = (ctypes.c_int * 8)()
    n = _lib.fs_radix_plan(int(L), int(e), buf, 8)
    return [buf[i] for i in range(n)]


def fs_device_status():
    """Device error code of the kernels' bounded waits (0 = none); cleared on read."""
    load()
    code = ctypes.c_int()
    _lib.fs_device_status(ctypes.byref(code))
    return code.value


def fs_kernel_launches():
    load()
    return int(_lib.fs_kernel_launches())


def fs_profile_enable(on):
    load()
    _check(_lib.fs_profile_enable(1 if on else 0), "fs_profile_enable")


def fs_profile_report():
    """{class name: (launches, total device ms)} of the recorded launches."""
    load()
    n = len(PROFILE_CLASSES)
    counts = (ctypes.c_uint64 * n)()
    ms = (ctypes.c_double * n)()
    k = _lib.fs_profile_report(counts, ms, n)
    return {PROFILE_CLASSES[i]: (int(counts[i]), float(ms[i])) for i in range(k)}
