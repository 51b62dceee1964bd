"""ctypes binding of libwt.so: argument marshalling only.

Every function here has the name of the C entry point it calls (wt_create,
wt_fit, ...).  Device buffers come from torch tensors (data_ptr) and
streams from torch.cuda streams; no computation happens in Python.  The
library must be built (``build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwt.so")

WT_OK, WT_ERR_ARG, WT_ERR_GEOMETRY, WT_ERR_ILL_CONDITIONED, WT_ERR_NOT_SPD = 0, 1, 2, 3, 4
WT_ERR_OOM, WT_ERR_CUDA, WT_ERR_TIMEOUT, WT_ERR_STATE, WT_ERR_NAN, WT_ERR_UNSUPPORTED = 5, 6, 7, 8, 9, 10
WT_ERR_ACCURACY = 11
WT_FP32, WT_FP64 = 0, 1
WT_Z_MIRROR = 0
STATUS_NAMES = {0: "WT_OK", 1: "WT_ERR_ARG", 2: "WT_ERR_GEOMETRY", 3: "WT_ERR_ILL_CONDITIONED",
                4: "WT_ERR_NOT_SPD", 5: "WT_ERR_OOM", 6: "WT_ERR_CUDA", 7: "WT_ERR_TIMEOUT",
                8: "WT_ERR_STATE", 9: "WT_ERR_NAN", 10: "WT_ERR_UNSUPPORTED", 11: "WT_ERR_ACCURACY"}


class wt_grid(C.Structure):
    _fields_ = [("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("Nx", C.c_int), ("Ny", C.c_int), ("Nz", C.c_int),
                ("eps_r", C.c_double), ("zbc", C.c_int)]


class wt_column(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z0", C.c_double), ("z1", C.c_double),
                ("radius", C.c_double), ("resistivity", C.c_double),
                ("terminal_top", C.c_int), ("driven", C.c_int), ("n_sources", C.c_int)]


class wt_fit_opts(C.Structure):
    _fields_ = [("n_az", C.c_int), ("n_h", C.c_int), ("tikhonov", C.c_double),
                ("v_w", C.c_double), ("az0", C.c_double), ("refine", C.c_int)]


class wt_tracks(C.Structure):
    _fields_ = [("n_tracks", C.c_int), ("n_steps", C.c_int), ("n_out", C.c_int),
                ("dt", C.c_double), ("charge", C.c_double),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p), ("q", C.c_void_p)]


class wt_shaper(C.Structure):
    _fields_ = [("tau", C.c_double), ("order", C.c_int), ("gain", C.c_double), ("noise_rms", C.c_double)]


class wt_tuning(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("nb", "lb", "nch", "nepi", "r_xy", "r_z", "x_direct", "two_pass",
                                       "store_vec", "table_rows", "table_flags")]


class wt_feature_opts(C.Structure):
    _fields_ = [("lo", C.c_float), ("hi", C.c_float), ("cfd", C.c_float)]


WT_N_FEATURES = 6
FEATURE_NAMES = ("amplitude", "t_peak", "charge", "t_lo", "t_hi", "t_cfd")


class wt_info(C.Structure):
    _fields_ = [("n_columns", C.c_int), ("n_sources", C.c_int), ("n_colloc", C.c_int), ("n_t", C.c_int),
                ("rank", C.c_int), ("cond_estimate", C.c_double), ("boundary_residual", C.c_double),
                ("asymmetry", C.c_double), ("trunc_rel", C.c_double), ("mu_min", C.c_double),
                ("mu_max", C.c_double), ("fit_seconds", C.c_double), ("relax_seconds", C.c_double),
                ("grad_trunc_rel", C.c_double), ("Nx", C.c_int), ("Ny", C.c_int), ("Nz", C.c_int),
                ("fit_correction", C.c_double), ("fit_refined", C.c_int)]


# name -> (restype, argtypes); the ABI of include/wt.h
SIGNATURES = {
    "wt_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(wt_grid), C.c_int]),
    "wt_add_columns": (C.c_int, [C.c_void_p, C.POINTER(wt_column), C.c_int]),
    "wt_fit": (C.c_int, [C.c_void_p, C.POINTER(wt_fit_opts), C.POINTER(C.c_double)]),
    "wt_relax": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int]),
    "wt_extend": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "wt_sample_H": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double), C.c_int,
                              C.POINTER(C.c_double)]),
    "wt_eq1": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(wt_tracks), C.c_void_p, C.c_void_p]),
    "wt_eq1_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(wt_tracks), C.c_void_p, C.c_void_p]),
    "wt_eq1_direct": (C.c_int, [C.c_void_p, C.POINTER(wt_tracks), C.c_void_p, C.c_void_p]),
    "wt_eq1_loss": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(wt_tracks), C.POINTER(C.c_double)]),
    "wt_eq1_loss_grad": (C.c_int, [C.c_void_p, C.POINTER(wt_tracks), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]),
    "wt_set_resistivity_profile": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_int]),
    "wt_eq1_loss_grad_profile": (C.c_int, [C.c_void_p, C.POINTER(wt_tracks), C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "wt_static_field": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "wt_drift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double]
                 + [C.c_void_p] * 7),
    "wt_shape": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double, C.POINTER(wt_shaper),
                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "wt_batch_run": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p), C.c_void_p]),
    "wt_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(wt_tuning)]),
    "wt_sync": (C.c_int, [C.c_void_p, C.c_void_p]),
    "wt_eq1_tangents": (C.c_int, [C.c_void_p, C.POINTER(wt_tracks), C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    "wt_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double,
                              C.POINTER(wt_feature_opts), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "wt_get_charges": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "wt_get_capacitance": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "wt_get_modes": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "wt_get_info": (C.c_int, [C.c_void_p, C.POINTER(wt_info)]),
    "wt_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "wt_get_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "wt_get_grad_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "wt_last_error": (C.c_char_p, [C.c_void_p]),
    "wt_destroy": (None, [C.c_void_p]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libwt.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} missing: build the CUDA library first (paper_2605_13987_gb300.build.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class WTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code, ctx):
    if code != WT_OK:
        lib = load_library()
        raise WTError(code, lib.wt_last_error(ctx).decode(errors="replace"))


def _dptr(a):
    return C.c_double_p if False else a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


# ---------------------------------------------------------------- C names
def wt_create(grid, cuda_device=0):
    lib = load_library()
    ctx = C.c_void_p()
    # any z boundary but the mirror reaches the library as an unknown code, which it rejects
    g = wt_grid(grid.Lx, grid.Ly, grid.Lz, grid.Nx, grid.Ny, grid.Nz, grid.eps_r,
                WT_Z_MIRROR if getattr(grid, "zbc", "mirror") == "mirror" else -1)
    _check(lib.wt_create(C.byref(ctx), C.byref(g), int(cuda_device)), None)
    return ctx


def wt_add_columns(ctx, columns):
    lib = load_library()
    arr = (wt_column * len(columns))(*[wt_column(c.x, c.y, c.z0, c.z1, c.radius, c.resistivity,
                                                 int(c.terminal_top), int(c.driven), int(c.n_sources))
                                       for c in columns])
    _check(lib.wt_add_columns(ctx, arr, len(columns)), ctx)


def wt_fit(ctx, n_az=4, n_h=2, tikhonov=0.0, v_w=1.0, az0=0.0, refine=0):
    lib = load_library()
    o = wt_fit_opts(int(n_az), int(n_h), float(tikhonov), float(v_w), float(az0), int(refine))
    cond = C.c_double(0.0)
    _check(lib.wt_fit(ctx, C.byref(o), C.byref(cond)), ctx)
    return cond.value


def wt_relax(ctx, times):
    lib = load_library()
    t = np.ascontiguousarray(times, dtype=np.float64)
    _check(lib.wt_relax(ctx, _dptr(t), len(t)), ctx)


def wt_extend(ctx, precision, H, stream=None):
    """H: torch tensor (cuda: asynchronous on `stream`; cpu: synchronous copy-out) or numpy array."""
    lib = load_library()
    nbytes = H.numel() * H.element_size() if hasattr(H, "numel") else H.nbytes
    st = _stream_handle(stream) if (hasattr(H, "is_cuda") and H.is_cuda) else None
    _check(lib.wt_extend(ctx, int(precision), _ptr(H), nbytes, st), ctx)


def wt_sample_H(ctx, xyz, times):
    lib = load_library()
    p = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    t = np.ascontiguousarray(times, dtype=np.float64).ravel()
    out = np.zeros((len(t), len(p), 3))
    _check(lib.wt_sample_H(ctx, _dptr(p), len(p), _dptr(t), len(t), _dptr(out)), ctx)
    return out


def _tracks_struct(tracks):
    """wt_tracks over the arrays of a track dict (the dict keeps them alive)."""
    return wt_tracks(int(tracks["n_tracks"]), int(tracks["n_steps"]), int(tracks["n_out"]),
                     float(tracks["dt"]), float(tracks.get("charge", 1.0)),
                     _ptr(tracks["x"]), _ptr(tracks["y"]), _ptr(tracks["z"]),
                     _ptr(tracks["vx"]), _ptr(tracks["vy"]), _ptr(tracks["vz"]), _ptr(tracks.get("q")))


def wt_eq1(ctx, H, tracks, i_out, stream=None):
    lib = load_library()
    tr = _tracks_struct(tracks)
    st = _stream_handle(stream) if (hasattr(i_out, "is_cuda") and i_out.is_cuda) else None
    _check(lib.wt_eq1(ctx, _ptr(H), C.byref(tr), _ptr(i_out), st), ctx)


def _noalloc_buffer(name, t, n_min, device, exact=False):
    """Checks a wt_eq1_noalloc argument: a contiguous float32 CUDA tensor on `device` holding at
    least (exactly, for H) n_min values; raises WTError(WT_ERR_ARG) otherwise."""
    import torch
    why = None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        why = "must be a CUDA tensor (the call stages nothing)"
    elif t.dtype != torch.float32:
        why = f"must be float32, not {t.dtype}"
    elif not t.is_contiguous():
        why = "must be contiguous"
    elif t.device.index != device:
        why = f"is on cuda:{t.device.index}, the context on cuda:{device}"
    elif (t.numel() != n_min) if exact else (t.numel() < n_min):
        why = f"holds {t.numel()} values, needs {'exactly ' if exact else ''}{n_min}"
    if why:
        raise WTError(WT_ERR_ARG, f"wt_eq1_noalloc: {name} {why}")


def wt_eq1_noalloc(ctx, H, tracks, i_out, stream=None, device=None):
    """Eq. 1 with no device allocation: every buffer a contiguous float32 CUDA tensor on the
    context's device (`device`, default: H's), sized as the call needs."""
    lib = load_library()
    info = wt_get_info(ctx)
    dev = H.device.index if device is None and hasattr(H, "device") else (device or 0)
    n_tr, n_st, n_out = int(tracks["n_tracks"]), int(tracks["n_steps"]), int(tracks["n_out"])
    _noalloc_buffer("H", H, info["n_t"] * 3 * info["Nx"] * info["Ny"] * info["Nz"], dev, exact=True)
    _noalloc_buffer("i_out", i_out, n_tr * n_out, dev)
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        _noalloc_buffer(k, tracks[k], n_tr * n_st, dev)
    if tracks.get("q") is not None:
        _noalloc_buffer("q", tracks["q"], n_tr, dev)
    tr = _tracks_struct(tracks)
    _check(lib.wt_eq1_noalloc(ctx, _ptr(H), C.byref(tr), _ptr(i_out), _stream_handle(stream)), ctx)


def wt_eq1_direct(ctx, tracks, i_out, stream=None):
    """Eq. 1 currents from the context's rank-r field form, without H."""
    lib = load_library()
    tr = _tracks_struct(tracks)
    st = _stream_handle(stream) if (hasattr(i_out, "is_cuda") and i_out.is_cuda) else None
    _check(lib.wt_eq1_direct(ctx, C.byref(tr), _ptr(i_out), st), ctx)


def wt_eq1_loss(ctx, precision, tracks):
    lib = load_library()
    tr = _tracks_struct(tracks)
    out = C.c_double(0.0)
    _check(lib.wt_eq1_loss(ctx, int(precision), C.byref(tr), C.byref(out)), ctx)
    return out.value


def wt_eq1_loss_grad(ctx, tracks):
    """(loss, grad[4]) with grad = dL/d(s_R, s_B, r, lambda)."""
    lib = load_library()
    tr = _tracks_struct(tracks)
    out = C.c_double(0.0)
    g = np.zeros(4)
    _check(lib.wt_eq1_loss_grad(ctx, C.byref(tr), C.byref(out), _dptr(g)), ctx)
    return out.value, g


def wt_set_resistivity_profile(ctx, column, rho):
    """Per-node resistivities [Ohm*m] of one column (None: back to uniform)."""
    lib = load_library()
    if rho is None:
        _check(lib.wt_set_resistivity_profile(ctx, int(column), None, 0), ctx)
        return
    r = np.ascontiguousarray(rho, dtype=np.float64)
    _check(lib.wt_set_resistivity_profile(ctx, int(column), _dptr(r), len(r)), ctx)


def wt_eq1_loss_grad_profile(ctx, tracks, delta):
    """(loss, dL/deps) along rho_j -> rho_j (1 + eps delta_j)."""
    lib = load_library()
    tr = _tracks_struct(tracks)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    out = C.c_double(0.0)
    g = C.c_double(0.0)
    _check(lib.wt_eq1_loss_grad_profile(ctx, C.byref(tr), _dptr(d), C.byref(out), C.byref(g)), ctx)
    return out.value, g.value


def wt_static_field(ctx, phi_cols, precision, E, stream=None):
    """Static field of the electrodes at phi_cols volts into the device tensor E [3, Nx, Ny, Nz]."""
    lib = load_library()
    p = np.ascontiguousarray(phi_cols, dtype=np.float64)
    _check(lib.wt_static_field(ctx, _dptr(p), int(precision), _ptr(E), E.numel() * E.element_size(),
                               _stream_handle(stream)), ctx)
    return E


def wt_drift(ctx, E, x0, smu, n_steps, dt, stream=None):
    """Drift tracks (dict of device tensors x, y, z, vx, vy, vz [n, n_steps])."""
    import torch
    lib = load_library()
    n = int(x0.shape[0])
    out = {k: torch.empty((n, n_steps), dtype=torch.float32, device=E.device) for k in ("x", "y", "z", "vx", "vy", "vz")}
    _check(lib.wt_drift(ctx, _ptr(E), _ptr(x0), _ptr(smu), n, int(n_steps), float(dt),
                        *[_ptr(out[k]) for k in ("x", "y", "z", "vx", "vy", "vz")], _stream_handle(stream)), ctx)
    return out


def wt_shape(ctx, i, dt, tau, order, gain=1.0, noise=None, noise_rms=0.0, out=None, stream=None):
    """CR-(RC)^n shaping of device currents i [n_tracks, n_out] (torch, FP32)."""
    import torch
    lib = load_library()
    if out is None:
        out = torch.empty_like(i)
    sh = wt_shaper(float(tau), int(order), float(gain), float(noise_rms))
    _check(lib.wt_shape(ctx, _ptr(i), int(i.shape[0]), int(i.shape[1]), float(dt), C.byref(sh), _ptr(noise),
                        _ptr(out), _stream_handle(stream)), ctx)
    return out


def wt_batch_run(ctxs, precision, H_list, stream=None):
    """Bulk extension of several relaxed contexts into their device buffers H_list."""
    lib = load_library()
    n = len(ctxs)
    carr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    harr = (C.c_void_p * n)(*[h.data_ptr() for h in H_list])
    _check(lib.wt_batch_run(carr, n, int(precision), harr, _stream_handle(stream)), ctxs[0])


def wt_get_tuning(ctx):
    lib = load_library()
    out = wt_tuning()
    _check(lib.wt_get_tuning(ctx, C.byref(out)), ctx)
    return {k: getattr(out, k) for k, _ in wt_tuning._fields_}


def wt_eq1_tangents(ctx, tracks, i_out=None, di_out=None):
    """(loss, grad[4]); fills the device tensors i_out [n_tracks, n_out] and
    di_out [4, n_tracks, n_out] (FP32) when given."""
    lib = load_library()
    tr = _tracks_struct(tracks)
    out = C.c_double(0.0)
    g = np.zeros(4)
    _check(lib.wt_eq1_tangents(ctx, C.byref(tr), _ptr(i_out), _ptr(di_out), C.byref(out), _dptr(g)), ctx)
    return out.value, g


def wt_features(ctx, x, t0, dt, lo=0.1, hi=0.9, cfd=0.5, dx=None, f_out=None, df_out=None, stream=None):
    """Signal features [n_tracks, 6] (FP64 device tensor) of the FP32 device
    waveforms x [n_tracks, n]; with tangents dx [n_dir, n_tracks, n] also
    their derivatives [n_dir, n_tracks, 6].  Returns (f, df or None)."""
    import torch
    lib = load_library()
    for t in (x, dx):
        if t is not None and (t.dtype != torch.float32 or not t.is_contiguous()):
            raise ValueError("waveforms and tangents must be contiguous float32 tensors")
    n_tracks, n = int(x.shape[0]), int(x.shape[1])
    n_dir = 0 if dx is None else int(dx.shape[0])
    if dx is not None and tuple(dx.shape[1:]) != (n_tracks, n):
        raise ValueError("tangents must have shape [n_dir, n_tracks, n]")
    if f_out is None:
        f_out = torch.empty((n_tracks, WT_N_FEATURES), dtype=torch.float64, device=x.device)
    if n_dir and df_out is None:
        df_out = torch.empty((n_dir, n_tracks, WT_N_FEATURES), dtype=torch.float64, device=x.device)
    o = wt_feature_opts(float(lo), float(hi), float(cfd))
    _check(lib.wt_features(ctx, _ptr(x), n_tracks, n, float(t0), float(dt), C.byref(o), _ptr(dx), n_dir,
                           _ptr(f_out), _ptr(df_out if n_dir else None), _stream_handle(stream)), ctx)
    return f_out, (df_out if n_dir else None)


def wt_sync(ctx, stream=None):
    """Wait for the context's work and report device-side failures of earlier asynchronous calls."""
    _check(load_library().wt_sync(ctx, _stream_handle(stream)), ctx)


def wt_get_charges(ctx, n_t, n_sources):
    lib = load_library()
    out = np.zeros((n_t, n_sources))
    _check(lib.wt_get_charges(ctx, _dptr(out)), ctx)
    return out


def wt_get_capacitance(ctx, n_sources):
    lib = load_library()
    out = np.zeros((n_sources, n_sources))
    _check(lib.wt_get_capacitance(ctx, _dptr(out)), ctx)
    return out


def wt_get_modes(ctx, n_sources):
    lib = load_library()
    out = np.zeros(n_sources - 1)
    _check(lib.wt_get_modes(ctx, _dptr(out)), ctx)
    return out


def wt_get_info(ctx):
    lib = load_library()
    info = wt_info()
    _check(lib.wt_get_info(ctx, C.byref(info)), ctx)
    return {k: getattr(info, k) for k, _ in wt_info._fields_}


def wt_set_timing(ctx, enable=True):
    _check(load_library().wt_set_timing(ctx, int(bool(enable))), ctx)


def wt_get_timing(ctx):
    """(ms[3], n_launches) of the last timed wt_extend."""
    ms = (C.c_double * 3)()
    n = C.c_int(0)
    _check(load_library().wt_get_timing(ctx, ms, C.byref(n)), ctx)
    return list(ms), n.value


def wt_get_grad_timing(ctx):
    ms = (C.c_double * 6)()
    _check(load_library().wt_get_grad_timing(ctx, ms), ctx)
    keys = ("base", "shared", "fit_tangent", "modal_tangent", "tangent_basis", "tangent_fields")
    return dict(zip(keys, list(ms)))


def wt_destroy(ctx):
    if ctx:
        load_library().wt_destroy(ctx)
