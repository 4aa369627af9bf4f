"""ctypes binding of libvlasov.so (include/vlasov.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels; this module converts
Python arguments (torch tensors, integers) to the C ABI and raises
``VlasovError`` on a non-zero status. There is no CPU fallback: ``lib()``
raises if the shared library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvlasov.so")
MAX_SPECIES = 4
NSTATS = 13  # VL_NSTATS

VL_OK, VL_EINVAL, VL_ECUDA, VL_ENOCONV, VL_ENUMERIC, VL_ENOTSUP = range(6)

EXPORTED = ["vlasov_work_bytes", "vlasov_init", "vlasov_free", "vl_last_error", "pfc_advect_x",
            "pfc_advect_xy", "pfc_advect_v", "pfc_advect_v_static", "moments", "moment_fit", "moment_fit_solve", "moment_fit_exchange", "moment_fit_wide", "fluid_step", "fluid_step_species",
            "fluid_step_closure", "maxwell_step", "vl_read_stats", "vl_reset_stats", "vl_sync_status", "vl_launch_count", "vl_fma_peak", "mlp_init", "mlp_set_weights",
            "mlp_get_weights", "mlp_set_harvest", "mlp_harvest_count", "mlp_normalize", "mlp_train", "mlp_forward",
            "mlp_grad"]
MLP_NPARAM = 19520  # VL_MLP_NPARAM
MLP_SAMPLE = 24     # VL_MLP_SAMPLE


class VlasovError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libvlasov status %d: %s" % (status, msg))
        self.status = status


class VlDesc(ctypes.Structure):
    _fields_ = [
        ("nvdim", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("x0", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("bc_y", ctypes.c_int),
        ("nspecies", ctypes.c_int),
        ("q", ctypes.c_double * MAX_SPECIES),
        ("m", ctypes.c_double * MAX_SPECIES),
        ("nv", (ctypes.c_int * 3) * MAX_SPECIES),
        ("vmin", (ctypes.c_double * 3) * MAX_SPECIES),
        ("vmax", (ctypes.c_double * 3) * MAX_SPECIES),
        ("precision", ctypes.c_int),
        ("nshear", ctypes.c_int),
        ("c", ctypes.c_double),
        ("ion_background", ctypes.c_double),
        ("fit_tol", ctypes.c_double),
        ("fit_max_iter", ctypes.c_int),
    ]


_LIB = None
_vp = ctypes.c_void_p
_dpp = ctypes.POINTER(ctypes.c_void_p)


def lib():
    """Load libvlasov.so (raises if it is missing: no fallback path exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libvlasov.so not built: run paper_2109_06743_gb300.build.build() "
                           "(or __graft_entry__.build()) first")
    L = ctypes.CDLL(LIB_PATH)
    D = ctypes.POINTER(VlDesc)
    L.vlasov_work_bytes.argtypes = [D]
    L.vlasov_work_bytes.restype = ctypes.c_size_t
    L.vlasov_init.argtypes = [D, _dpp, _vp, _vp, _vp, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
    L.vlasov_free.argtypes = [_vp]
    L.vl_last_error.argtypes = [_vp]
    L.vl_last_error.restype = ctypes.c_char_p
    L.pfc_advect_x.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp]
    L.pfc_advect_xy.argtypes = [_vp, ctypes.c_int, ctypes.c_double, _vp, _vp]
    L.pfc_advect_v.argtypes = [_vp, ctypes.c_int, ctypes.c_double, _vp, _vp]
    L.pfc_advect_v_static.argtypes = [D, ctypes.c_int, _vp, _vp, ctypes.c_longlong, ctypes.c_double, _vp, _vp]
    L.moments.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    L.moment_fit.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.moment_fit_solve.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp]
    L.moment_fit_exchange.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
    L.fluid_step.argtypes = [_vp, ctypes.c_double, _dpp, _dpp, _vp]
    L.fluid_step_species.argtypes = [_vp, ctypes.c_int, ctypes.c_double, _vp, _vp, _vp]
    L.maxwell_step.argtypes = [_vp, ctypes.c_double, _dpp, _vp]
    L.fluid_step_closure.argtypes = [_vp, ctypes.c_double, _vp]
    L.vl_read_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong), _vp]
    L.vl_reset_stats.argtypes = [_vp, _vp]
    L.vl_sync_status.argtypes = [_vp, _vp]
    L.vl_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp, _vp]
    F = ctypes.POINTER(ctypes.c_float)
    L.mlp_init.argtypes = [_vp, ctypes.c_ulonglong]
    L.mlp_set_weights.argtypes = [_vp, F]
    L.mlp_get_weights.argtypes = [_vp, F]
    L.mlp_set_harvest.argtypes = [_vp, _vp, ctypes.c_longlong, _vp]
    L.mlp_harvest_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong), _vp]
    L.mlp_normalize.argtypes = [_vp, _vp, ctypes.c_longlong, _vp]
    L.mlp_train.argtypes = [_vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                            ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double), _vp]
    L.mlp_forward.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp]
    L.mlp_grad.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, ctypes.POINTER(ctypes.c_double), _vp]
    L.vl_launch_count.argtypes = []
    L.vl_launch_count.restype = ctypes.c_longlong
    for name in EXPORTED:
        getattr(L, name)
        if name not in ("vlasov_work_bytes", "vl_last_error", "vl_launch_count"):
            getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


def ptr(x):
    """Device (or host) address of a tensor, or an int/None passed through."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def stream_handle(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _ptr_array(xs):
    arr = (ctypes.c_void_p * MAX_SPECIES)()
    for i, x in enumerate(xs):
        arr[i] = ptr(x)
    return arr


def _check(ctx, st):
    if st != VL_OK:
        raise VlasovError(st, lib().vl_last_error(ctx).decode())


def make_desc(cfg) -> VlDesc:
    """vl_desc from a workloads.Config."""
    d = VlDesc()
    d.nvdim, d.nx, d.ny = cfg.nvdim, cfg.nx, cfg.ny
    d.x0, d.dx, d.y0, d.dy = cfg.x0, cfg.dx, cfg.y0, cfg.dy
    d.bc_y = cfg.bc_y
    d.nspecies = len(cfg.species)
    for s, sp in enumerate(cfg.species):
        d.q[s], d.m[s] = sp.q, sp.m
        for a in range(3):
            d.nv[s][a] = sp.nv[a]
            d.vmin[s][a] = sp.vmin[a]
            d.vmax[s][a] = sp.vmax[a]
    d.precision = cfg.precision
    d.nshear = cfg.nshear
    d.c = cfg.c or 0.0
    d.ion_background = cfg.ion_background
    d.fit_tol = cfg.fit_tol
    d.fit_max_iter = cfg.fit_max_iter
    return d


def vlasov_work_bytes(desc: VlDesc) -> int:
    return int(lib().vlasov_work_bytes(ctypes.byref(desc)))


def vlasov_init(desc, f_list, fluid, yee, eb, work, work_bytes):
    ctx = ctypes.c_void_p()
    st = lib().vlasov_init(ctypes.byref(desc), None if f_list is None else _ptr_array(f_list), ptr(fluid), ptr(yee),
                           ptr(eb), ptr(work),
                           work_bytes, ctypes.byref(ctx))
    _check(None, st)
    return ctx


def vlasov_free(ctx):
    lib().vlasov_free(ctx)


def pfc_advect_x(ctx, species, axis, dt, stream=None):
    _check(ctx, lib().pfc_advect_x(ctx, species, axis, dt, stream_handle(stream)))


def pfc_advect_xy(ctx, species, dt, f_out, stream=None):
    """x then y sweep, out of place into f_out; the context's f of the
    species becomes f_out (the caller swaps its buffers)."""
    _check(ctx, lib().pfc_advect_xy(ctx, species, dt, ptr(f_out), stream_handle(stream)))


def pfc_advect_v(ctx, species, dt, mom_out=None, stream=None):
    _check(ctx, lib().pfc_advect_v(ctx, species, dt, ptr(mom_out), stream_handle(stream)))


STATIC_SCRATCH_CELLS = 32768  # VL_STATIC_SCRATCH_CELLS


def pfc_advect_v_static(desc, species, f, eb, ncell, dt, mom_out=None, stream=None):
    """Context-free velocity pass on `ncell` cells with the library's static
    scratch (no allocation); errors come from vl_last_error(NULL)."""
    _check(None, lib().pfc_advect_v_static(ctypes.byref(desc), species, ptr(f), ptr(eb), int(ncell), dt,
                                           ptr(mom_out), stream_handle(stream)))


def moments(ctx, species, mom_out, stream=None):
    _check(ctx, lib().moments(ctx, species, ptr(mom_out), stream_handle(stream)))


def moment_fit(ctx, species, vmom, use_mlp=False, theta_v=None, theta_f=None, mom_out=None, stream=None):
    _check(ctx, lib().moment_fit(ctx, species, ptr(vmom), int(bool(use_mlp)), ptr(theta_v), ptr(theta_f),
                                 ptr(mom_out), stream_handle(stream)))


def moment_fit_solve(ctx, species, vmom, use_mlp=False, theta_v=None, theta_f=None, stream=None):
    _check(ctx, lib().moment_fit_solve(ctx, species, ptr(vmom), int(bool(use_mlp)), ptr(theta_v), ptr(theta_f),
                                       stream_handle(stream)))


def moment_fit_exchange(ctx, species, vmom, mom_out=None, stream=None):
    _check(ctx, lib().moment_fit_exchange(ctx, species, ptr(vmom), ptr(mom_out), stream_handle(stream)))


def moment_fit_wide(ctx, species, wide):
    """wide: None (chosen on the device), False/0 or True/1."""
    _check(ctx, lib().moment_fit_wide(ctx, species, -1 if wide is None else int(bool(wide))))


def fluid_step(ctx, dt, mom_t, mom_t1, stream=None):
    _check(ctx, lib().fluid_step(ctx, dt, _ptr_array(mom_t), _ptr_array(mom_t1), stream_handle(stream)))


def fluid_step_closure(ctx, dt, stream=None):
    """One SSP-RK3 step of the gradient-closure fluid model (Sec. 2.3)."""
    _check(ctx, lib().fluid_step_closure(ctx, dt, stream_handle(stream)))


def maxwell_step(ctx, h, mom=None, stream=None):
    arr = None if mom is None else _ptr_array(mom)
    _check(ctx, lib().maxwell_step(ctx, h, arr, stream_handle(stream)))


def vl_read_stats(ctx, stream=None):
    out = (ctypes.c_longlong * NSTATS)()
    _check(ctx, lib().vl_read_stats(ctx, out, stream_handle(stream)))
    return list(out)


def vl_reset_stats(ctx, stream=None):
    _check(ctx, lib().vl_reset_stats(ctx, stream_handle(stream)))


def vl_launch_count():
    return int(lib().vl_launch_count())


# ---- MLP warm start ------------------------------------------------------------------

def mlp_init(ctx, seed=0):
    _check(ctx, lib().mlp_init(ctx, int(seed)))


def mlp_set_weights(ctx, w):
    """w: numpy float32 array of MLP_NPARAM values (host)."""
    import numpy as np
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert w.size == MLP_NPARAM
    _check(ctx, lib().mlp_set_weights(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))


def mlp_get_weights(ctx):
    import numpy as np
    w = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check(ctx, lib().mlp_get_weights(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return w


def mlp_set_harvest(ctx, samples, capacity, stream=None):
    _check(ctx, lib().mlp_set_harvest(ctx, ptr(samples), int(capacity), stream_handle(stream)))


def mlp_harvest_count(ctx, stream=None):
    n = ctypes.c_longlong(0)
    _check(ctx, lib().mlp_harvest_count(ctx, ctypes.byref(n), stream_handle(stream)))
    return n.value


def mlp_normalize(ctx, samples, n, stream=None):
    _check(ctx, lib().mlp_normalize(ctx, ptr(samples), int(n), stream_handle(stream)))


def mlp_train(ctx, samples, n, steps, batch=4096, lr=1e-3, seed=0, record_loss=False, stream=None):
    """Returns the per-step losses if record_loss, else None."""
    loss = (ctypes.c_double * max(1, steps))() if record_loss else None
    _check(ctx, lib().mlp_train(ctx, ptr(samples), int(n), int(steps), int(batch), float(lr), int(seed),
                                loss, stream_handle(stream)))
    return list(loss)[:steps] if record_loss else None


def mlp_forward(ctx, x, n, y, stream=None):
    _check(ctx, lib().mlp_forward(ctx, ptr(x), int(n), ptr(y), stream_handle(stream)))


def mlp_grad(ctx, samples, n, grad, stream=None):
    loss = ctypes.c_double(0.0)
    _check(ctx, lib().mlp_grad(ctx, ptr(samples), int(n), ptr(grad), ctypes.byref(loss), stream_handle(stream)))
    return loss.value


def vl_sync_status(ctx, stream=None):
    """Wait for the stream; raises VlasovError(VL_ENUMERIC) if a kernel found
    non-finite or negative fit targets since the status was last reported."""
    _check(ctx, lib().vl_sync_status(ctx, stream_handle(stream)))


def vl_fma_peak(precision, sink, stream=None):
    """Measured FMA operations per second of the current device (FP32 or
    FP64); sink: an 8-byte device tensor the probe never writes."""
    out = ctypes.c_double(0.0)
    _check(None, lib().vl_fma_peak(int(precision), ctypes.byref(out), ptr(sink), stream_handle(stream)))
    return out.value


def fluid_step_species(ctx, species, dt, mom_t, mom_t1, stream=None):
    _check(ctx, lib().fluid_step_species(ctx, species, dt, ptr(mom_t), ptr(mom_t1), stream_handle(stream)))
