"""Thin Python binding of the C ABI in include/lens.h (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names; device buffers are torch tensors (their
data_ptr() is passed) and streams are torch.cuda.Stream objects (their
cuda_stream handle is passed).  Importing this module loads the compiled
library and raises if it is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblens.so")

LENS_OK, LENS_EINVAL, LENS_ENOMEM, LENS_ENOTFOUND, LENS_ECAPACITY, LENS_ECUDA, LENS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
LENS_DPIE, LENS_SIS, LENS_POINT = 0, 1, 2
LENS_FP64, LENS_MIXED = 0, 1
LENS_CHI2_SRC_MAPPED, LENS_CHI2_SRC_MU, LENS_CHI2_SRC_PLAIN = 0, 1, 2
LENS_REPAIR_RATIO_DEFAULT = 0.16  # lens.h

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = ("lens_create", "lens_destroy", "lens_set_fp64_threshold", "lens_set_repair_ratio", "lens_mem_used", "lens_model_bytes",
           "lens_model_upload",
           "lens_model_release", "lens_grad_map", "lens_hessian_map", "lens_potential_map", "lens_grad_map_host", "lens_hessian_map_host",
           "lens_cset_create", "lens_cset_release",
           "lens_chi2_source", "lens_chi2_source_nocache", "lens_chi2_source_scaled", "lens_cset_scaling_cache", "lens_mcmc_step", "lens_mcmc_step_dev", "lens_chi2_autotune", "lens_chi2_image",
           "lens_find_images", "lens_chi2_image_noalloc", "lens_selftest_wait", "lens_selftest_math", "lens_wait", "lens_strerror",
           "lens_last_error", "lens_server_create", "lens_server_destroy", "lens_server_submit",
           "lens_server_progress", "lens_server_cancel", "lens_server_stats")
LENS_REQ_MAP, LENS_REQ_CHI2_SOURCE, LENS_REQ_CHI2_IMAGE = 0, 1, 2


class LensError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.lens_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_lib.lens_strerror(code).decode()} ({code}): {msg}")


class lens_halo(C.Structure):
    _fields_ = [("type", C.c_int32), ("x0", C.c_double), ("y0", C.c_double), ("theta", C.c_double),
                ("eps", C.c_double), ("rcore", C.c_double), ("rcut", C.c_double), ("b0", C.c_double)]


HALO_BYTES = C.sizeof(lens_halo)  # one row of the halo table


class lens_grid(C.Structure):
    _fields_ = [("xmin", C.c_double), ("xmax", C.c_double), ("ymin", C.c_double), ("ymax", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


class lens_constraints(C.Structure):
    _fields_ = [("nsrc", C.c_int32), ("img_off", C.POINTER(C.c_int32)), ("x", C.POINTER(C.c_double)),
                ("y", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("dls_ds", C.POINTER(C.c_double))]


class lens_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("handle", C.c_int64), ("grid", lens_grid), ("dls_ds", C.c_double),
                ("precision", C.c_int32), ("hessian", C.c_int32), ("variant", C.c_int32), ("P", C.c_int32),
                ("params", C.POINTER(C.c_double)), ("result", C.c_void_p)]


class lens_completion(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("status", C.c_int32), ("queue_ms", C.c_double), ("latency_ms", C.c_double)]


class lens_server_info(C.Structure):
    _fields_ = [("queued", C.c_int32), ("inflight", C.c_int32), ("pool_bytes", C.c_size_t),
                ("pool_used", C.c_size_t), ("pool_peak", C.c_size_t)]


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, i64 = C.c_void_p, C.c_int64
    sig = {
        "lens_create": (C.c_int, [C.POINTER(vp), C.c_int, C.c_size_t]),
        "lens_destroy": (C.c_int, [vp]),
        "lens_set_fp64_threshold": (C.c_int, [vp, C.c_double]),
        "lens_set_repair_ratio": (C.c_int, [vp, C.c_double]),
        "lens_mem_used": (C.c_size_t, [vp]),
        "lens_model_bytes": (C.c_size_t, [vp, i64]),
        "lens_model_upload": (C.c_int, [vp, C.POINTER(lens_halo), C.c_int32, C.POINTER(i64)]),
        "lens_model_release": (C.c_int, [vp, i64]),
        "lens_grad_map": (C.c_int, [vp, i64, C.POINTER(lens_grid), C.c_double, C.c_int32, vp, vp]),
        "lens_hessian_map": (C.c_int, [vp, i64, C.POINTER(lens_grid), C.c_double, C.c_int32, vp, vp]),
        "lens_potential_map": (C.c_int, [vp, i64, C.POINTER(lens_grid), C.c_double, C.c_int32,
                                         C.POINTER(C.c_double), vp, vp]),
        "lens_grad_map_host": (C.c_int, [vp, i64, C.POINTER(lens_grid), C.c_double, C.c_int32, vp, vp]),
        "lens_hessian_map_host": (C.c_int, [vp, i64, C.POINTER(lens_grid), C.c_double, C.c_int32, vp, vp]),
        "lens_cset_create": (C.c_int, [vp, i64, C.POINTER(lens_constraints), C.POINTER(C.c_int32), C.POINTER(i64)]),
        "lens_cset_release": (C.c_int, [vp, i64]),
        "lens_chi2_source": (C.c_int, [vp, i64, vp, C.c_int32, C.c_int32, vp, vp]),
        "lens_mcmc_step_dev": (C.c_int, [vp, i64, vp, vp, C.c_int32, C.c_int32, vp, C.c_double, C.c_uint64,
                                         vp, C.c_int32, vp, vp, vp]),
        "lens_chi2_source_nocache": (C.c_int, [vp, i64, vp, C.c_int32, C.c_int32, vp, vp]),
        "lens_chi2_source_scaled": (C.c_int, [vp, i64, vp, C.c_int32, C.c_int32, vp, vp]),
        "lens_cset_scaling_cache": (C.c_int, [vp, i64, C.c_double, C.c_double, C.c_int32]),
        "lens_mcmc_step": (C.c_int, [vp, i64, vp, vp, C.c_int32, C.c_int32, vp, C.c_double, C.c_uint64,
                                     C.c_uint64, C.c_int32, vp, vp, vp]),
        "lens_chi2_autotune": (C.c_int, [vp, i64, vp, C.c_int32, vp, vp, C.POINTER(C.c_int32),
                                         C.POINTER(C.c_float)]),
        "lens_chi2_image": (C.c_int, [vp, i64, C.POINTER(lens_grid), vp, C.c_int32, vp, vp, vp]),
        "lens_find_images": (C.c_int, [vp, i64, C.POINTER(lens_grid), vp, C.c_int32, vp, C.c_int32, vp, vp]),
        "lens_chi2_image_noalloc": (C.c_int, [vp, i64, C.POINTER(lens_grid), vp, C.c_int32, vp, vp, vp]),
        "lens_selftest_wait": (C.c_int, [vp, C.c_int32, vp]),
        "lens_selftest_math": (C.c_int, [vp, vp, C.c_int32, vp, vp]),
        "lens_wait": (C.c_int, [vp, vp, i64]),
        "lens_server_create": (C.c_int, [vp, C.c_int32, C.c_size_t, C.POINTER(vp)]),
        "lens_server_destroy": (C.c_int, [vp]),
        "lens_server_submit": (C.c_int, [vp, C.POINTER(lens_request), C.POINTER(i64)]),
        "lens_server_progress": (C.c_int, [vp, C.POINTER(lens_completion), C.c_int32, C.POINTER(C.c_int32)]),
        "lens_server_cancel": (C.c_int, [vp, i64]),
        "lens_server_stats": (C.c_int, [vp, C.POINTER(lens_server_info)]),
        "lens_strerror": (C.c_char_p, [C.c_int]),
        "lens_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load_library()


def _check(rc, where):
    if rc != LENS_OK:
        raise LensError(rc, where)
    return rc


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_grid(g):
    if isinstance(g, lens_grid):
        return g
    return lens_grid(g["xmin"], g["xmax"], g["ymin"], g["ymax"], g["nx"], g["ny"])


# lens_halo as a numpy record: int32 type, 4 bytes of padding, 7 doubles
_HALO_DTYPE = np.dtype({"names": ["type", "x0", "y0", "theta", "eps", "rcore", "rcut", "b0"],
                        "formats": ["<i4"] + ["<f8"] * 7,
                        "offsets": [0, 8, 16, 24, 32, 40, 48, 56], "itemsize": 64})
assert _HALO_DTYPE.itemsize == C.sizeof(lens_halo)


def halos_from_table(table):
    """Halo table rows (type, x0, y0, theta, eps, rcore, rcut, b0) as a
    contiguous lens_halo array (numpy record array with the C layout)."""
    t = np.asarray(table, dtype=np.float64).reshape(-1, 8)
    arr = np.zeros(len(t), dtype=_HALO_DTYPE)
    arr["type"] = t[:, 0].astype(np.int32)
    for k, name in enumerate(_HALO_DTYPE.names[1:], start=1):
        arr[name] = t[:, k]
    return arr


class Context:
    """Owns a lens_ctx; the methods mirror the C calls."""

    def __init__(self, device=0, mem_budget_bytes=0):
        self.h = C.c_void_p()
        _check(_lib.lens_create(C.byref(self.h), int(device), int(mem_budget_bytes)), "lens_create")

    def close(self):
        if self.h:
            _lib.lens_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_fp64_threshold(self, b0):
        _check(_lib.lens_set_fp64_threshold(self.h, float(b0)), "lens_set_fp64_threshold")

    def set_repair_ratio(self, r):
        _check(_lib.lens_set_repair_ratio(self.h, float(r)), "lens_set_repair_ratio")

    def mem_used(self):
        return int(_lib.lens_mem_used(self.h))

    def model_bytes(self, model):
        return int(_lib.lens_model_bytes(self.h, int(model)))

    def model_upload(self, table):
        arr = halos_from_table(table)
        out = C.c_int64()
        _check(_lib.lens_model_upload(self.h, arr.ctypes.data_as(C.POINTER(lens_halo)), len(arr), C.byref(out)),
               "lens_model_upload")
        return out.value

    def model_release(self, model):
        _check(_lib.lens_model_release(self.h, int(model)), "lens_model_release")

    def grad_map(self, model, grid, dls_ds, precision, out, stream=None):
        g = make_grid(grid)
        _check(_lib.lens_grad_map(self.h, int(model), C.byref(g), float(dls_ds), int(precision), _ptr(out),
                                  _stream(stream)), "lens_grad_map")
        return out

    def hessian_map(self, model, grid, dls_ds, precision, out, stream=None):
        g = make_grid(grid)
        _check(_lib.lens_hessian_map(self.h, int(model), C.byref(g), float(dls_ds), int(precision), _ptr(out),
                                     _stream(stream)), "lens_hessian_map")
        return out

    def potential_map(self, model, grid, dls_ds, precision, out, beta=None, stream=None):
        """Lensing potential [ny][nx] into `out`, and with beta = (x, y) the
        time-delay (Fermat) surface as a second plane ([2][ny][nx])."""
        g = make_grid(grid)
        b = None if beta is None else (C.c_double * 2)(float(beta[0]), float(beta[1]))
        _check(_lib.lens_potential_map(self.h, int(model), C.byref(g), float(dls_ds), int(precision), b, _ptr(out),
                                       _stream(stream)), "lens_potential_map")
        return out

    def grad_map_host(self, model, grid, dls_ds, precision, out, stream=None):
        """Deflection map into page-locked host memory `out` (e.g. a torch
        tensor with pin_memory=True), band by band as the GPU finishes."""
        g = make_grid(grid)
        _check(_lib.lens_grad_map_host(self.h, int(model), C.byref(g), float(dls_ds), int(precision), _ptr(out),
                                       _stream(stream)), "lens_grad_map_host")
        return out

    def hessian_map_host(self, model, grid, dls_ds, precision, out, stream=None):
        """Six-plane Hessian map into page-locked host memory `out`."""
        g = make_grid(grid)
        _check(_lib.lens_hessian_map_host(self.h, int(model), C.byref(g), float(dls_ds), int(precision),
                                          _ptr(out), _stream(stream)), "lens_hessian_map_host")
        return out

    def cset_create(self, model, cons, var_halo):
        off = np.ascontiguousarray(cons["img_off"], dtype=np.int32)
        x = np.ascontiguousarray(cons["x"], dtype=np.float64)
        y = np.ascontiguousarray(cons["y"], dtype=np.float64)
        s = np.ascontiguousarray(cons["sigma"], dtype=np.float64)
        d = np.ascontiguousarray(cons["dls_ds"], dtype=np.float64)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        c = lens_constraints(len(off) - 1, off.ctypes.data_as(C.POINTER(C.c_int32)), dp(x), dp(y), dp(s), dp(d))
        var = (C.c_int32 * 2)(int(var_halo[0]), int(var_halo[1]))
        out = C.c_int64()
        _check(_lib.lens_cset_create(self.h, int(model), C.byref(c), var, C.byref(out)), "lens_cset_create")
        return out.value

    def cset_release(self, cset):
        _check(_lib.lens_cset_release(self.h, int(cset)), "lens_cset_release")

    def chi2_source(self, cset, params, P, variant, chi2, stream=None):
        _check(_lib.lens_chi2_source(self.h, int(cset), _ptr(params), int(P), int(variant), _ptr(chi2),
                                     _stream(stream)), "lens_chi2_source")
        return chi2

    def chi2_source_scaled(self, cset, params, P, variant, out, stream=None):
        """chi2 of P sets of 16 parameters: the 14 of chi2_source, then the
        members' b0 and r_cut factors (see lens.h)."""
        _check(_lib.lens_chi2_source_scaled(self.h, int(cset), _ptr(params), int(P), int(variant), _ptr(out),
                                            _stream(stream)), "lens_chi2_source_scaled")
        return out

    def cset_scaling_cache(self, cset, ft_min, ft_max, nodes=32):
        """Static sums at Chebyshev points of the members' r_cut factor (see
        lens.h); nodes = 0 drops them."""
        _check(_lib.lens_cset_scaling_cache(self.h, int(cset), float(ft_min), float(ft_max), int(nodes)),
               "lens_cset_scaling_cache")

    def mcmc_step(self, cset, params, chi2, W, sigma, temperature, seed, step, scratch, accepted=None,
                  variant=0, stream=None):
        """One Metropolis step of W chains, params [W][14 or 16] and chi2 [W]
        updated in place on the device (see lens.h)."""
        nparams = int(params.shape[-1])
        _check(_lib.lens_mcmc_step(self.h, int(cset), _ptr(params), _ptr(chi2), int(W), nparams, _ptr(sigma),
                                   float(temperature), int(seed) & (2**64 - 1), int(step) & (2**64 - 1),
                                   int(variant), _ptr(scratch), None if accepted is None else _ptr(accepted),
                                   _stream(stream)), "lens_mcmc_step")

    def mcmc_step_dev(self, cset, params, chi2, W, sigma, temperature, seed, step_counter, scratch, accepted=None,
                      variant=0, stream=None):
        """mcmc_step with the step counter in device memory (step_counter: a
        device tensor of one int64 / uint64, advanced by 1 by every step;
        see lens.h)."""
        nparams = int(params.shape[-1])
        _check(_lib.lens_mcmc_step_dev(self.h, int(cset), _ptr(params), _ptr(chi2), int(W), nparams, _ptr(sigma),
                                       float(temperature), int(seed) & (2**64 - 1), _ptr(step_counter),
                                       int(variant), _ptr(scratch), None if accepted is None else _ptr(accepted),
                                       _stream(stream)), "lens_mcmc_step_dev")

    def chi2_source_nocache(self, cset, params, P, variant, chi2, stream=None):
        _check(_lib.lens_chi2_source_nocache(self.h, int(cset), _ptr(params), int(P), int(variant), _ptr(chi2),
                                             _stream(stream)), "lens_chi2_source_nocache")
        return chi2

    def chi2_autotune(self, cset, params, P, chi2, stream=None):
        """Pick and keep the fastest launch shape of chi2_source for this set;
        returns (threads*100 + CTAs-per-SM cap, best ms)."""
        cfg, ms = C.c_int32(), C.c_float()
        _check(_lib.lens_chi2_autotune(self.h, int(cset), _ptr(params), int(P), _ptr(chi2), _stream(stream),
                                       C.byref(cfg), C.byref(ms)), "lens_chi2_autotune")
        return cfg.value, ms.value

    def chi2_image(self, cset, grid, params, P, chi2, nfound=None, stream=None):
        g = make_grid(grid)
        rc = _lib.lens_chi2_image(self.h, int(cset), C.byref(g), _ptr(params), int(P), _ptr(chi2), _ptr(nfound),
                                  _stream(stream))
        if rc not in (LENS_OK, LENS_ECAPACITY):
            raise LensError(rc, "lens_chi2_image")
        return rc

    def find_images(self, cset, grid, params, P, images, count, stream=None):
        """images: device double [P][max_per_set][3]; count: device int32 [P]."""
        g = make_grid(grid)
        rc = _lib.lens_find_images(self.h, int(cset), C.byref(g), _ptr(params), int(P), _ptr(images),
                                   int(images.shape[1]), _ptr(count), _stream(stream))
        if rc not in (LENS_OK, LENS_ECAPACITY):
            raise LensError(rc, "lens_find_images")
        return rc

    def chi2_image_noalloc(self, cset, grid, params, P, chi2, nfound=None, stream=None):
        """lens_chi2_image with all working memory in the library's fixed
        device array: for loops that may not allocate device memory at call
        time.  Overlapping calls race on that array."""
        g = make_grid(grid)
        rc = _lib.lens_chi2_image_noalloc(self.h, int(cset), C.byref(g), _ptr(params), int(P), _ptr(chi2),
                                          _ptr(nfound), _stream(stream))
        if rc not in (LENS_OK, LENS_ECAPACITY):
            raise LensError(rc, "lens_chi2_image_noalloc")
        return rc

    def selftest_wait(self, polls=64, stream=None):
        """Run the bounded-wait failure path once (see lens.h)."""
        _check(_lib.lens_selftest_wait(self.h, int(polls), _stream(stream)), "lens_selftest_wait")

    def selftest_math(self, x, out, stream=None):
        """rcp, 1/x, rsqrt, CUDA rsqrt of the device doubles x into out [4][n] (see lens.h)."""
        _check(_lib.lens_selftest_math(self.h, _ptr(x), int(x.numel()), _ptr(out), _stream(stream)),
               "lens_selftest_math")

    def wait(self, stream=None, timeout_ms=60000):
        return _check(_lib.lens_wait(self.h, _stream(stream), int(timeout_ms)), "lens_wait")


class Server:
    """Request loop of a context (lens_server_*): map and chi2 requests run on
    `slots` streams of its own, admitted by the device memory of its pool.
    Results land in page-locked host tensors given at submit."""

    def __init__(self, ctx, slots=4, pool_bytes=1 << 30):
        self.ctx = ctx
        self.h = C.c_void_p()
        _check(_lib.lens_server_create(ctx.h, int(slots), int(pool_bytes), C.byref(self.h)), "lens_server_create")
        self._done = (lens_completion * 256)()

    def close(self):
        if self.h:
            _lib.lens_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _submit(self, req, keep=None):
        t = C.c_int64()
        _check(_lib.lens_server_submit(self.h, C.byref(req), C.byref(t)), "lens_server_submit")
        return t.value

    def submit_map(self, model, grid, dls_ds, precision, hessian, result):
        """result: pinned host tensor of (6 if hessian else 2) x ny x nx elements."""
        r = lens_request(LENS_REQ_MAP, int(model), make_grid(grid), float(dls_ds), int(precision), int(bool(hessian)),
                         0, 0, None, C.c_void_p(result.data_ptr()))
        return self._submit(r)

    def submit_chi2_source(self, cset, params, variant, result):
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 14)
        r = lens_request(LENS_REQ_CHI2_SOURCE, int(cset), lens_grid(), 0.0, 0, 0, int(variant), len(p),
                         p.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(result.data_ptr()))
        return self._submit(r)

    def submit_chi2_image(self, cset, grid, params, result):
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 14)
        r = lens_request(LENS_REQ_CHI2_IMAGE, int(cset), make_grid(grid), 0.0, 0, 0, 0, len(p),
                         p.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(result.data_ptr()))
        return self._submit(r)

    def progress(self):
        """Retire finished requests and admit queued ones; returns a list of
        (ticket, status, queue_ms, latency_ms)."""
        n = C.c_int32()
        rc = _lib.lens_server_progress(self.h, self._done, len(self._done), C.byref(n))
        out = [(d.ticket, d.status, d.queue_ms, d.latency_ms) for d in self._done[:n.value]]
        if rc != LENS_OK and not out:
            raise LensError(rc, "lens_server_progress")
        return out

    def cancel(self, ticket):
        _check(_lib.lens_server_cancel(self.h, int(ticket)), "lens_server_cancel")

    def stats(self):
        i = lens_server_info()
        _check(_lib.lens_server_stats(self.h, C.byref(i)), "lens_server_stats")
        return {"queued": i.queued, "inflight": i.inflight, "pool_bytes": i.pool_bytes, "pool_used": i.pool_used,
                "pool_peak": i.pool_peak}


def strerror(code):
    return _lib.lens_strerror(int(code)).decode()
