"""Python binding of the lbmwet C ABI (include/lbmwet.h): argument marshalling only.

Every computation runs in liblbmwet.so (CUDA kernels for sm_103a, plus its host-side setup); this
module converts numpy arrays and Python values to the C structs and pointers the ABI takes, and
turns non-OK status codes into exceptions.  The library is loaded from this package's directory;
importing this module fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbmwet.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_UNSTABLE, LBM_ERR_STATE = range(6)
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP64, LBM_FP32_DEV = 0, 1
LBM_EOS_PR, LBM_EOS_CS = 0, 1
LBM_WALL_IVD, LBM_WALL_VD, LBM_WALL_SF, LBM_WALL_GF = 0, 1, 2, 3
LBM_BODY_NONE, LBM_BODY_BALL, LBM_BODY_PLANE = 0, 1, 2


class lbm_eos(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double),
                ("T", C.c_double), ("omega", C.c_double)]


class lbm_config(C.Structure):
    _fields_ = [("lattice", C.c_int32), ("precision", C.c_int32),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("eos", lbm_eos), ("G", C.c_double), ("sigma", C.c_double),
                ("s_rho", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double), ("s_j", C.c_double),
                ("s_q", C.c_double), ("s_nu", C.c_double), ("s_pi", C.c_double), ("s_m", C.c_double),
                ("rho_l", C.c_double), ("rho_g", C.c_double), ("rho_ref", C.c_double),
                ("body_force", C.c_double * 3), ("wall_kind", C.c_int32), ("kappa", C.c_double),
                ("rho_w_const", C.c_double), ("body_kind", C.c_int32), ("body_center", C.c_double * 3),
                ("body_radius", C.c_double), ("drop_hint", C.c_double * 3),
                ("step_kernel", C.c_int32), ("Gw", C.c_double), ("theta_a", C.c_double)]


class lbm_obs(C.Structure):
    _fields_ = [("mass", C.c_double), ("rho_max", C.c_double), ("rho_min", C.c_double),
                ("u_max", C.c_double), ("theta_deg", C.c_double), ("drop_center", C.c_double * 3),
                ("drop_radius", C.c_double), ("n_interface", C.c_int64), ("step", C.c_int64)]


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lbmwet status {status}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1908_04443_gb300.build.build() "
                          "(this package has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    dp = C.POINTER(C.c_double)
    sig = {
        "lbm_coexistence": (C.c_int, [C.POINTER(lbm_eos), dp, dp]),
        "lbm_critical_temperature": (C.c_int, [C.POINTER(lbm_eos), dp]),
        "lbm_init": (C.c_int, [C.POINTER(lbm_config), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(H)]),
        "lbm_step": (C.c_int, [H, C.c_int64]),
        "lbm_enqueue_steps": (C.c_int, [H, C.c_int64]),
        "lbm_check": (C.c_int, [H]),
        "lbm_selftest_bounded_wait": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_int32)]),
        "lbm_probe_fp64_rate": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
        "lbm_release_cached_memory": (C.c_int, []),
        "lbm_memory_stats": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "lbm_check_guards": (C.c_int, [H, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "lbm_observables": (C.c_int, [H, C.POINTER(lbm_obs), C.c_void_p, C.c_void_p]),
        "lbm_fields_device": (C.c_int, [H, C.c_void_p, C.c_void_p]),
        "lbm_observables_noalloc": (C.c_int, [H, C.c_void_p, C.c_void_p, C.POINTER(lbm_obs)]),
        "lbm_wall_nodes": (C.c_int, [H, C.c_void_p, C.POINTER(C.c_int64)]),
        "lbm_get_state": (C.c_int, [H, C.c_void_p]),
        "lbm_set_state": (C.c_int, [H, C.c_void_p, C.c_int64]),
        "lbm_save_state": (C.c_int, [H, C.c_void_p, C.POINTER(C.c_size_t)]),
        "lbm_load_state": (C.c_int, [H, C.c_void_p, C.c_size_t]),
        "lbm_set_kappa": (C.c_int, [H, C.c_void_p]),
        "lbm_limiter_bounds": (C.c_int, [H, dp, dp]),
        "lbm_kernel_launches": (C.c_int64, [H]),
        "lbm_step_kernel_used": (C.c_int32, [H]),
        "lbm_destroy": (None, [H]),
        "lbm_last_error": (C.c_char_p, [H]),
        "lbm_status_string": (C.c_char_p, [C.c_int]),
        "lbm_record": (C.c_int, [H, C.c_int64, C.c_int64]),
        "lbm_adjoint": (C.c_int, [H, C.c_void_p, C.c_void_p]),
        "lbm_batch_init": (C.c_int, [C.c_int32, C.POINTER(lbm_config), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(C.c_void_p)]),
        "lbm_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
        "lbm_batch_enqueue_steps": (C.c_int, [C.c_void_p, C.c_int64]),
        "lbm_batch_observables": (C.c_int, [C.c_void_p, C.POINTER(lbm_obs)]),
        "lbm_batch_observables_fields": (C.c_int, [C.c_void_p, C.POINTER(lbm_obs), C.POINTER(C.c_void_p),
                                                   C.POINTER(C.c_void_p)]),
        "lbm_grid_shape": (C.c_int, [H, C.POINTER(C.c_int32)]),
        "lbm_d3q19_work_list": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                          C.POINTER(C.c_int64)]),
        "lbm_batch_handle": (C.c_void_p, [C.c_void_p, C.c_int32]),
        "lbm_batch_size": (C.c_int32, [C.c_void_p]),
        "lbm_batch_kernel_launches": (C.c_int64, [C.c_void_p]),
        "lbm_batch_step_kernel_used": (C.c_int32, [C.c_void_p]),
        "lbm_batch_instance_kernel": (C.c_int32, [C.c_void_p, C.c_int32]),
        "lbm_batch_autotune": (C.c_int, [C.c_void_p, C.c_int32]),
        "lbm_batch_tuning_report": (C.c_char_p, [C.c_void_p]),
        "lbm_batch_set_kernels": (C.c_int, [C.c_void_p, C.c_void_p]),
        "lbm_batch_autotune_forget": (None, []),
        "lbm_batch_last_error": (C.c_char_p, [C.c_void_p]),
        "lbm_batch_destroy": (None, [C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("lbm_coexistence", "lbm_critical_temperature", "lbm_init", "lbm_step", "lbm_enqueue_steps", "lbm_check",
            "lbm_selftest_bounded_wait", "lbm_probe_fp64_rate", "lbm_release_cached_memory", "lbm_memory_stats",
            "lbm_check_guards",
            "lbm_observables", "lbm_fields_device", "lbm_observables_noalloc", "lbm_wall_nodes", "lbm_get_state", "lbm_set_state",
            "lbm_save_state", "lbm_load_state", "lbm_set_kappa", "lbm_limiter_bounds", "lbm_kernel_launches",
            "lbm_step_kernel_used", "lbm_batch_step_kernel_used", "lbm_batch_instance_kernel", "lbm_batch_autotune",
            "lbm_batch_tuning_report", "lbm_batch_set_kernels", "lbm_batch_autotune_forget",
            "lbm_destroy", "lbm_last_error", "lbm_status_string", "lbm_record", "lbm_adjoint", "lbm_batch_init", "lbm_batch_step",
            "lbm_batch_enqueue_steps", "lbm_batch_observables", "lbm_batch_observables_fields", "lbm_grid_shape",
            "lbm_d3q19_work_list", "lbm_batch_handle", "lbm_batch_size",
            "lbm_batch_kernel_launches", "lbm_batch_last_error", "lbm_batch_destroy")


def library():
    return _lib


def _check(status: int, handle=None):
    if status != LBM_OK:
        msg = _lib.lbm_last_error(handle)
        raise LbmError(status, (msg or b"").decode() or _lib.lbm_status_string(status).decode())


def _mask_bytes(m) -> np.ndarray:
    """A solid mask as the C ABI takes it (one byte per node, nonzero = solid): a C-contiguous uint8
    array passes through uncopied, anything else is converted."""
    a = np.asarray(m).reshape(-1)
    if a.dtype == np.uint8 and a.flags.c_contiguous:
        return a
    return (a != 0).astype(np.uint8)


def _ptr(a: Optional[np.ndarray], dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


# ---- the ABI's entry points, same names -------------------------------------------------------

def lbm_coexistence(eos: lbm_eos):
    g, l = C.c_double(), C.c_double()
    _check(_lib.lbm_coexistence(C.byref(eos), C.byref(g), C.byref(l)))
    return g.value, l.value


def lbm_critical_temperature(eos: lbm_eos) -> float:
    t = C.c_double()
    _check(_lib.lbm_critical_temperature(C.byref(eos), C.byref(t)))
    return t.value


def lbm_init(cfg: lbm_config, solid_mask: np.ndarray, rho0=None, u0=None, kappa_per_wall=None, stream=None):
    n = cfg.nx * cfg.ny * cfg.nz
    mask, pm = _ptr(_mask_bytes(solid_mask), np.uint8)
    if mask.size != n:
        raise ValueError("solid_mask size does not match the grid")
    r, pr = _ptr(None if rho0 is None else np.asarray(rho0).reshape(-1), np.float64)
    if r is not None and r.size != n:
        raise ValueError("rho0 size does not match the grid")
    u, pu = _ptr(None if u0 is None else np.asarray(u0).reshape(-1), np.float64)
    if u is not None and u.size != (2 if cfg.lattice == LBM_D2Q9 else 3) * n:
        raise ValueError("u0 size does not match the grid (d * nodes, component-major)")
    k, pk = _ptr(None if kappa_per_wall is None else np.asarray(kappa_per_wall).reshape(-1), np.float64)
    h = C.c_void_p()
    st = _lib.lbm_init(C.byref(cfg), pm, pr, pu, pk, _stream_ptr(stream), C.byref(h))
    _check(st, None)
    return h


def lbm_step(h, n: int):
    _check(_lib.lbm_step(h, int(n)), h)


def lbm_enqueue_steps(h, n: int):
    _check(_lib.lbm_enqueue_steps(h, int(n)), h)


def lbm_check(h):
    _check(_lib.lbm_check(h), h)


def lbm_selftest_bounded_wait(polls: int = 1024, stream=None) -> bool:
    """Run the device's bounded-wait self-test: True if a wait that cannot complete gave up after
    `polls` polls and flagged the timeout (the expected outcome)."""
    t = C.c_int32(0)
    _check(_lib.lbm_selftest_bounded_wait(_stream_ptr(stream), int(polls), C.byref(t)))
    return bool(t.value)


def lbm_probe_fp64_rate(stream=None) -> float:
    """Measured FP64 fused multiply-add rate of the device in GFLOP/s (see the header)."""
    g = C.c_double(0.0)
    _check(_lib.lbm_probe_fp64_rate(_stream_ptr(stream), C.byref(g)))
    return float(g.value)


def lbm_release_cached_memory() -> None:
    """Return the unused memory of the library's device memory pools to the driver."""
    _check(_lib.lbm_release_cached_memory())


def lbm_memory_stats() -> Tuple[int, int]:
    """(bytes reserved, bytes in use) of the current device's memory pool."""
    r, u = C.c_int64(0), C.c_int64(0)
    _check(_lib.lbm_memory_stats(C.byref(r), C.byref(u)))
    return int(r.value), int(u.value)


def lbm_check_guards(h) -> Tuple[int, int]:
    """(guard bytes overwritten, padding bytes of the distributions no longer zero) of a handle:
    both 0 unless a kernel wrote outside its buffers."""
    g, p = C.c_int64(0), C.c_int64(0)
    _check(_lib.lbm_check_guards(h, C.byref(g), C.byref(p)), h)
    return int(g.value), int(p.value)


def lbm_grid_shape(h) -> Tuple[int, int, int, int]:
    """(nx, ny, nz, d) of a handle."""
    a = (C.c_int32 * 4)()
    _check(_lib.lbm_grid_shape(h, a), h)
    return int(a[0]), int(a[1]), int(a[2]), int(a[3])


def lbm_d3q19_work_list(mask) -> np.ndarray:
    """Work items of the TMA-staged D3Q19 z-march for a solid mask of shape (nz, ny, nx): an
    (items, 5) int32 array of rows (bx, by, z0, z1, solid).  Host code only (no device needed)."""
    m = np.asarray(mask)
    if m.ndim != 3:
        raise ValueError(f"mask must have shape (nz, ny, nx), got {m.shape}")
    nz, ny, nx = m.shape
    mb = _mask_bytes(m)
    mp = mb.ctypes.data_as(C.c_void_p)
    n = C.c_int64(0)
    _check(_lib.lbm_d3q19_work_list(mp, nx, ny, nz, None, 0, C.byref(n)))
    out = np.zeros((n.value, 5), np.int32)
    _check(_lib.lbm_d3q19_work_list(mp, nx, ny, nz, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
    return out


def _nodes_dim(h) -> Tuple[int, int]:
    nx, ny, nz, d = lbm_grid_shape(h)
    return nx * ny * nz, d


def _out_field(a, size: int, what: str):
    """A host output array the library writes `size` doubles into."""
    if a is None:
        return None
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous or not a.flags.writeable:
        raise ValueError(f"{what} must be a writeable C-contiguous float64 array")
    if a.size != size:
        raise ValueError(f"{what} must hold {size} values, not {a.size}")
    return a.ctypes.data


def lbm_observables(h, rho_host: Optional[np.ndarray] = None, u_host: Optional[np.ndarray] = None) -> lbm_obs:
    o = lbm_obs()
    n, d = _nodes_dim(h) if (rho_host is not None or u_host is not None) else (0, 0)
    pr = _out_field(rho_host, n, "rho_host")
    pu = _out_field(u_host, d * n, "u_host")
    _check(_lib.lbm_observables(h, C.byref(o), pr, pu), h)
    return o


def lbm_fields_device(h, rho_dev_ptr: Optional[int], u_dev_ptr: Optional[int]):
    _check(_lib.lbm_fields_device(h, rho_dev_ptr, u_dev_ptr), h)


def lbm_observables_noalloc(h, rho_dev_ptr: int, u_dev_ptr: int) -> lbm_obs:
    """Reductions of lbm_observables over caller-owned device fields, with no device allocation."""
    o = lbm_obs()
    _check(_lib.lbm_observables_noalloc(h, rho_dev_ptr, u_dev_ptr, C.byref(o)), h)
    return o


def lbm_wall_nodes(h) -> np.ndarray:
    cnt = C.c_int64()
    _check(_lib.lbm_wall_nodes(h, None, C.byref(cnt)), h)
    out = np.zeros(cnt.value, dtype=np.int64)
    _check(_lib.lbm_wall_nodes(h, out.ctypes.data_as(C.c_void_p), C.byref(cnt)), h)
    return out


def lbm_get_state(h, q: Optional[int] = None, n: Optional[int] = None) -> np.ndarray:
    """The post-streaming distributions, q * n doubles ([a][node]); q and n, if given, must be the
    handle's."""
    nn, d = _nodes_dim(h)
    qq = 9 if d == 2 else 19
    if (q is not None and q != qq) or (n is not None and n != nn):
        raise ValueError(f"the handle holds q = {qq} directions on n = {nn} nodes")
    out = np.zeros(qq * nn, dtype=np.float64)
    _check(_lib.lbm_get_state(h, out.ctypes.data_as(C.c_void_p)), h)
    return out


def lbm_set_state(h, f_post: np.ndarray, step: int = 0):
    nn, d = _nodes_dim(h)
    f, pf = _ptr(np.asarray(f_post).reshape(-1), np.float64)
    if f.size != (9 if d == 2 else 19) * nn:
        raise ValueError("f_post size does not match the handle's q * n")
    _check(_lib.lbm_set_state(h, pf, int(step)), h)


def lbm_save_state(h) -> bytes:
    nb = C.c_size_t(0)
    _check(_lib.lbm_save_state(h, None, C.byref(nb)), h)
    buf = C.create_string_buffer(nb.value)
    _check(_lib.lbm_save_state(h, buf, C.byref(nb)), h)
    return buf.raw


def lbm_load_state(h, data: bytes):
    buf = C.create_string_buffer(data, len(data))
    _check(_lib.lbm_load_state(h, buf, len(data)), h)


def lbm_set_kappa(h, kappa_per_wall: np.ndarray):
    k, pk = _ptr(np.asarray(kappa_per_wall).reshape(-1), np.float64)
    cnt = C.c_int64()
    _check(_lib.lbm_wall_nodes(h, None, C.byref(cnt)), h)
    if k.size != cnt.value:
        raise ValueError(f"kappa_per_wall must hold one value per wall node ({cnt.value})")
    _check(_lib.lbm_set_kappa(h, pk), h)


def lbm_limiter_bounds(h):
    g, l = C.c_double(), C.c_double()
    _check(_lib.lbm_limiter_bounds(h, C.byref(g), C.byref(l)), h)
    return g.value, l.value


def lbm_kernel_launches(h) -> int:
    return int(_lib.lbm_kernel_launches(h))


KERNEL_NAMES = {0: "auto", 1: "tile", 2: "ymarch", 3: "pair", 4: "ztma"}


def lbm_step_kernel_used(h) -> str:
    """"tile", "ymarch" or "pair" (D2Q9), "auto" for D3Q19 (its z-march)."""
    return KERNEL_NAMES[int(_lib.lbm_step_kernel_used(h))]


def lbm_destroy(h):
    _lib.lbm_destroy(h)


def lbm_record(h, n_steps: int, ckpt_every: int):
    _check(_lib.lbm_record(h, int(n_steps), int(ckpt_every)), h)


def lbm_adjoint(h, drho_final_dev_ptr: int, n_wall: int) -> np.ndarray:
    """dL/dkappa per wall node; drho_final_dev_ptr is a device pointer to N doubles."""
    out = np.zeros(max(n_wall, 1), dtype=np.float64)
    _check(_lib.lbm_adjoint(h, drho_final_dev_ptr, out.ctypes.data_as(C.c_void_p)), h)
    return out[:n_wall]


def _bcheck(status: int, b=None):
    if status != LBM_OK:
        msg = _lib.lbm_batch_last_error(b)
        raise LbmError(status, (msg or b"").decode() or _lib.lbm_status_string(status).decode())


def lbm_batch_init(cfgs, masks, rho0s=None, kappas_per_wall=None, stream=None):
    n = len(cfgs)
    # the library reads nx * ny * nz bytes of every mask and as many doubles of every density
    if len(masks) != n or (rho0s is not None and len(rho0s) != n) or \
            (kappas_per_wall is not None and len(kappas_per_wall) != n):
        raise ValueError("one mask (and density, kappa array) per instance")
    for i, c in enumerate(cfgs):
        if min(c.nx, c.ny, c.nz) < 1:
            continue                    # rejected by the library's own checks
        nodes = c.nx * c.ny * c.nz
        if masks[i] is None or np.asarray(masks[i]).size != nodes:
            raise ValueError(f"instance {i}: solid mask missing or of the wrong size")
        if rho0s is not None and rho0s[i] is not None and np.asarray(rho0s[i]).size != nodes:
            raise ValueError(f"instance {i}: rho0 size does not match the grid")
    arr = (lbm_config * n)(*cfgs)
    keep = []

    def ptrs(items, dtype):
        if items is None:
            return None
        out = (C.c_void_p * n)()
        for i, a in enumerate(items):
            if a is None:
                out[i] = None
            else:
                x = np.ascontiguousarray(np.asarray(a).reshape(-1), dtype=dtype)
                keep.append(x)
                out[i] = x.ctypes.data
        return out

    pm = ptrs([_mask_bytes(m) for m in masks], np.uint8)
    pr = ptrs(rho0s, np.float64)
    pk = ptrs(kappas_per_wall, np.float64)
    b = C.c_void_p()
    _bcheck(_lib.lbm_batch_init(n, arr, pm, pr, pk, _stream_ptr(stream), C.byref(b)), None)
    return b


def lbm_batch_step(b, n: int):
    _bcheck(_lib.lbm_batch_step(b, int(n)), b)


def lbm_batch_enqueue_steps(b, n: int):
    _bcheck(_lib.lbm_batch_enqueue_steps(b, int(n)), b)


def lbm_batch_observables(b):
    n = _lib.lbm_batch_size(b)
    out = (lbm_obs * n)()
    _bcheck(_lib.lbm_batch_observables(b, out), b)
    return list(out)


def lbm_batch_observables_fields(b, rho_hosts=None, u_hosts=None):
    """Observables of every instance, and their density / velocity fields written into the given host
    arrays (lists of n arrays or None), with one synchronisation for the whole batch."""
    n = _lib.lbm_batch_size(b)
    out = (lbm_obs * n)()

    def ptrs(arrs, comp, what):
        if arrs is None:
            return None
        if len(arrs) != n:
            raise ValueError(f"{what}: one array (or None) per instance")
        p = (C.c_void_p * n)()
        for i, a in enumerate(arrs):
            if a is not None:
                nn, d = _nodes_dim(lbm_batch_handle(b, i))
                p[i] = _out_field(a, (d if comp else 1) * nn, f"{what}[{i}]")
        return p

    pr = ptrs(rho_hosts, False, "rho_hosts")
    pu = ptrs(u_hosts, True, "u_hosts")
    _bcheck(_lib.lbm_batch_observables_fields(b, out, pr, pu), b)
    return list(out)


def lbm_batch_handle(b, i: int):
    h = _lib.lbm_batch_handle(b, int(i))
    if not h:
        raise IndexError(i)
    return C.c_void_p(h)


def lbm_batch_size(b) -> int:
    return int(_lib.lbm_batch_size(b))


def lbm_batch_kernel_launches(b) -> int:
    return int(_lib.lbm_batch_kernel_launches(b))


def lbm_batch_step_kernel_used(b) -> str:
    return KERNEL_NAMES[int(_lib.lbm_batch_step_kernel_used(b))]


def lbm_batch_instance_kernel(b, i: int) -> str:
    return KERNEL_NAMES[int(_lib.lbm_batch_instance_kernel(b, int(i)))]


def lbm_batch_set_kernels(b, kinds):
    """Step instance i with kernel kinds[i] ("tile", "ymarch" or "pair")."""
    names = {"tile": 1, "ymarch": 2, "pair": 3}
    arr = np.ascontiguousarray([names[k] if isinstance(k, str) else int(k) for k in kinds], dtype=np.int32)
    _bcheck(_lib.lbm_batch_set_kernels(b, arr.ctypes.data_as(C.c_void_p)), b)


def lbm_batch_autotune_forget():
    _lib.lbm_batch_autotune_forget()


def lbm_batch_autotune(b, trial_steps: int = 16) -> str:
    """Time the candidate kernels per size class and step each class with the fastest (see the
    header); returns the tuning report."""
    _bcheck(_lib.lbm_batch_autotune(b, int(trial_steps)), b)
    return (_lib.lbm_batch_tuning_report(b) or b"").decode()


def lbm_batch_destroy(b):
    _lib.lbm_batch_destroy(b)


# ---- configuration helpers ----------------------------------------------------------------------

def make_eos(kind: str, a: float, b: float, R: float = 1.0, T: float = 0.0, omega: float = 0.344) -> lbm_eos:
    return lbm_eos(kind={"PR": LBM_EOS_PR, "CS": LBM_EOS_CS}[kind], a=a, b=b, R=R, T=T, omega=omega)


def make_config(lattice: str, precision: str, shape: Sequence[int], eos: lbm_eos, *, G=-1.0, sigma=0.12,
                s_rho=1.0, s_e=0.8, s_eps=0.8, s_j=1.0, s_q=1.1, s_nu=1.0 / 0.95, s_pi=1.1, s_m=1.1,
                rho_l=0.0, rho_g=0.0, rho_ref=0.0, body_force=(0.0, 0.0, 0.0), wall="IVD", kappa=0.0,
                rho_w_const=1.0, body=None, drop_hint=(0.0, 0.0, 0.0), step_kernel="auto", Gw=0.0,
                theta_a=90.0) -> lbm_config:
    """Build an lbm_config.  `shape` is the numpy shape (ny, nx) or (nz, ny, nx).  `body` is
    ("ball", center, radius) or ("plane", wall_y) or None.  `step_kernel` is "auto", "tile",
    "ymarch", "pair" or "ztma" (work decomposition, see lbm_step_kernel in the header).  `wall` is
    "IVD" (parameter kappa), "VD" (rho_w_const), "SF" (Gw) or "GF" (theta_a, degrees; D2Q9)."""
    if len(shape) == 2:
        nz, (ny, nx) = 1, shape
    else:
        nz, ny, nx = shape
    cfg = lbm_config()
    cfg.lattice = {"D2Q9": LBM_D2Q9, "D3Q19": LBM_D3Q19}[lattice]
    cfg.precision = {"fp64": LBM_FP64, "fp32": LBM_FP32_DEV}[precision]
    cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
    cfg.eos = eos
    cfg.G, cfg.sigma = G, sigma
    cfg.s_rho, cfg.s_e, cfg.s_eps, cfg.s_j, cfg.s_q, cfg.s_nu, cfg.s_pi, cfg.s_m = s_rho, s_e, s_eps, s_j, s_q, s_nu, s_pi, s_m
    cfg.rho_l, cfg.rho_g, cfg.rho_ref = rho_l, rho_g, rho_ref
    for i in range(3):
        cfg.body_force[i] = body_force[i] if i < len(body_force) else 0.0
        cfg.drop_hint[i] = drop_hint[i] if i < len(drop_hint) else 0.0
    cfg.wall_kind = {"IVD": LBM_WALL_IVD, "VD": LBM_WALL_VD, "SF": LBM_WALL_SF, "GF": LBM_WALL_GF}[wall]
    cfg.Gw = Gw
    cfg.theta_a = theta_a
    cfg.kappa = kappa
    cfg.rho_w_const = rho_w_const
    cfg.step_kernel = {"auto": 0, "tile": 1, "ymarch": 2, "pair": 3, "ztma": 4}[step_kernel]
    cfg.body_kind = LBM_BODY_NONE
    if body is not None:
        if body[0] == "ball":
            cfg.body_kind = LBM_BODY_BALL
            for i, c in enumerate(body[1]):
                cfg.body_center[i] = c
            cfg.body_radius = body[2]
        else:
            cfg.body_kind = LBM_BODY_PLANE
            cfg.body_center[1] = body[1]
    return cfg


class Simulation:
    """Owns one lbm_handle.  Thin convenience over the entry points above."""

    def __init__(self, cfg: lbm_config, solid_mask, rho0=None, u0=None, kappa_per_wall=None, stream=None):
        self.cfg = cfg
        self.q = 9 if cfg.lattice == LBM_D2Q9 else 19
        self.d = 2 if cfg.lattice == LBM_D2Q9 else 3
        self.n = cfg.nx * cfg.ny * cfg.nz
        self.shape = (cfg.ny, cfg.nx) if self.d == 2 else (cfg.nz, cfg.ny, cfg.nx)
        self.h = lbm_init(cfg, solid_mask, rho0, u0, kappa_per_wall, stream)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def enqueue(self, n: int = 1):
        lbm_enqueue_steps(self.h, n)

    def check(self):
        lbm_check(self.h)

    def check_guards(self) -> Tuple[int, int]:
        return lbm_check_guards(self.h)

    def observables(self, fields: bool = False):
        if not fields:
            return lbm_observables(self.h), None, None
        rho = np.zeros(self.n)
        u = np.zeros(self.d * self.n)
        o = lbm_observables(self.h, rho, u)
        return o, rho.reshape(self.shape), u.reshape((self.d,) + self.shape)

    def get_state(self) -> np.ndarray:
        return lbm_get_state(self.h, self.q, self.n).reshape((self.q,) + self.shape)

    def set_state(self, f_post, step: int = 0):
        lbm_set_state(self.h, f_post, step)

    def wall_nodes(self) -> np.ndarray:
        return lbm_wall_nodes(self.h)

    def limiter_bounds(self):
        return lbm_limiter_bounds(self.h)

    def launches(self) -> int:
        return lbm_kernel_launches(self.h)

    def step_kernel(self) -> str:
        return lbm_step_kernel_used(self.h)

    def close(self):
        if self.h is not None:
            lbm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
