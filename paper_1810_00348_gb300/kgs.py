"""ctypes binding of libkgs.so (include/kgs.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; there is no
Python or CPU fallback.  If libkgs.so has not been built (``python -m
paper_1810_00348_gb300.build``) or no CUDA device is usable, the calls fail
with an exception.

The function names follow the C ABI: ``kgs_setup``, ``kgs_set_initial``,
``kgs_iterate``, ``kgs_moments``, ``kgs_moments_device``, ``kgs_rho_w``,
``kgs_set_rho_w``, ``kgs_save``, ``kgs_load``, ``kgs_info``,
``kgs_set_profiling``, ``kgs_profile``, ``kgs_destroy``, ``kgs_strerror``.
Problems come from ``paper_1810_00348_gb300.inputs.Problem``.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkgs.so")

KGS_OK = 0
KGS_NOTCONVERGED = 1
KGS_EINVAL = -1
KGS_ENOMEM = -2
KGS_ECUDA = -3
KGS_EDIVERGED = -4
KGS_ETIMEOUT = -5
KGS_EFORMAT = -6
KGS_FP64 = 0
KGS_MIXED = 1

_dp = ctypes.POINTER(ctypes.c_double)


class KgsGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", _dp), ("dy", _dp), ("dz", _dp)]


class KgsVgrid(ctypes.Structure):
    _fields_ = [("nvx", ctypes.c_int), ("nvy", ctypes.c_int), ("nvz", ctypes.c_int),
                ("xi_x", _dp), ("xi_y", _dp), ("xi_z", _dp), ("w_x", _dp), ("w_y", _dp), ("w_z", _dp)]


class KgsGas(ctypes.Structure):
    _fields_ = [("Kn", ctypes.c_double), ("Pr", ctypes.c_double), ("omega", ctypes.c_double)]


class KgsBc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int * 6), ("T_w", ctypes.c_double * 6), ("U_w", (ctypes.c_double * 3) * 6),
                ("rho_in", ctypes.c_double), ("U_in", ctypes.c_double * 3), ("T_in", ctypes.c_double),
                ("T_solid", ctypes.c_double)]


class KgsOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("wall_norm", ctypes.c_int), ("mass_rescale", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("tol", ctypes.c_double), ("v_per_cta", ctypes.c_int),
                ("block_z", ctypes.c_int), ("stream", ctypes.c_void_p), ("q_lagged", ctypes.c_int),
                ("vz_begin", ctypes.c_int), ("vz_end", ctypes.c_int), ("order", ctypes.c_int),
                ("dev_source", ctypes.c_int)]


class KgsInfo(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nvx", ctypes.c_int), ("nvy", ctypes.c_int), ("nvz", ctypes.c_int),
                ("n_fluid", ctypes.c_longlong), ("phase_points", ctypes.c_longlong),
                ("iteration", ctypes.c_int), ("n_stages", ctypes.c_int),
                ("v_per_cta", ctypes.c_int), ("block_z", ctypes.c_int), ("precision", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("last_residual", ctypes.c_double)]


# exported symbols and their C signatures (restype, argtypes)
SIGNATURES = {
    "kgs_setup": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(KgsGrid),
                                 ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(KgsVgrid), ctypes.POINTER(KgsGas),
                                 ctypes.POINTER(KgsBc), ctypes.POINTER(KgsOpts)]),
    "kgs_set_initial": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "kgs_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp]),
    "kgs_moments": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "kgs_moments_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "kgs_rho_w": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "kgs_set_rho_w": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "kgs_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "kgs_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "kgs_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(KgsInfo)]),
    "kgs_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "kgs_profile": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)]),
    "kgs_destroy": (None, [ctypes.c_void_p]),
    "kgs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "kgs_sweep_sums": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "kgs_close_sums": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _dp]),
    "kgs_iterate_noalloc": (ctypes.c_int, [ctypes.POINTER(KgsGrid), ctypes.POINTER(ctypes.c_uint8),
                                           ctypes.POINTER(KgsVgrid), ctypes.POINTER(KgsGas), ctypes.POINTER(KgsBc),
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _dp,
                                           ctypes.c_void_p]),
}

_lib = None


class KgsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, load().kgs_strerror(code).decode(), code))


def load(path: str = LIB_PATH):
    """Load libkgs.so and declare every exported signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libkgs.so is not built (run python -m paper_1810_00348_gb300.build)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc, where, allow=()):
    if rc != KGS_OK and rc not in allow:
        raise KgsError(rc, where)
    return rc


def _arr(x, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


class Context:
    """Handle of one kgs_ctx (one problem on the current CUDA device)."""

    def __init__(self, handle, prob, keep):
        self.handle = handle
        self.prob = prob
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None):
            kgs_destroy(self)

    @property
    def shape(self):
        return (self.prob.nz, self.prob.ny, self.prob.nx)


def _problem_structs(prob, keep):
    """ABI structs (grid, vgrid, gas, bc, solid pointer) of an inputs.Problem;
    arrays referenced by pointers are appended to ``keep``."""

    def p(a):
        a = _arr(a)
        keep.append(a)
        return a.ctypes.data_as(_dp)

    g = KgsGrid(prob.nx, prob.ny, prob.nz, p(prob.dx), p(prob.dy), p(prob.dz))
    v = KgsVgrid(len(prob.xi_x), len(prob.xi_y), len(prob.xi_z), p(prob.xi_x), p(prob.xi_y), p(prob.xi_z),
                 p(prob.w_x), p(prob.w_y), p(prob.w_z))
    gas = KgsGas(prob.Kn, prob.Pr, prob.omega)
    bc = KgsBc()
    for s in range(6):
        bc.type[s] = int(prob.face_type[s])
        bc.T_w[s] = float(prob.T_w[s])
        for d in range(3):
            bc.U_w[s][d] = float(prob.U_w[s][d])
    bc.rho_in, bc.T_in, bc.T_solid = prob.rho_in, prob.T_in, prob.T_solid
    for d in range(3):
        bc.U_in[d] = float(prob.U_in[d])
    solid_p = ctypes.POINTER(ctypes.c_uint8)()
    if prob.solid is not None:
        sol = _arr(prob.solid, np.uint8).reshape(-1)
        keep.append(sol)
        solid_p = sol.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    return g, v, gas, bc, solid_p


def kgs_setup(prob, precision=KGS_FP64, max_iters=1000, tol=1e-8, v_per_cta=0, block_z=0, stream=None,
              vz=(0, 0), dev_source=0):
    """kgs_setup for an ``inputs.Problem``; stream is a cudaStream_t value (int) or None; vz = (begin, end)
    sweeps only those velocity planes (a part of a velocity-space partition); dev_source = 1 selects the
    deviation-form FP32 source (kgs_opts.dev_source)."""
    lib = load()
    keep = []
    g, v, gas, bc, solid_p = _problem_structs(prob, keep)
    opts = KgsOpts(precision, int(prob.wall_mode), int(prob.mass_rescale), max_iters, tol, v_per_cta, block_z,
                   ctypes.c_void_p(stream) if stream else None, int(getattr(prob, "q_lagged", 0)),
                   int(vz[0]), int(vz[1]), int(getattr(prob, "order", 1)), int(dev_source))
    h = ctypes.c_void_p()
    _check(lib.kgs_setup(ctypes.byref(h), ctypes.byref(g), solid_p, ctypes.byref(v), ctypes.byref(gas),
                         ctypes.byref(bc), ctypes.byref(opts)), "kgs_setup")
    return Context(h, prob, None)


def kgs_set_initial(ctx, macros=None):
    if macros is None:
        return _check(load().kgs_set_initial(ctx.handle, _dp()), "kgs_set_initial")
    m = _arr(macros).reshape(-1)
    return _check(load().kgs_set_initial(ctx.handle, m.ctypes.data_as(_dp)), "kgs_set_initial")


def kgs_iterate(ctx, n_iters=1):
    """Returns (rc, iterations_done, residual); KGS_NOTCONVERGED and
    KGS_EDIVERGED are returned, other errors raise."""
    done = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = load().kgs_iterate(ctx.handle, int(n_iters), ctypes.byref(done), ctypes.byref(res))
    _check(rc, "kgs_iterate", allow=(KGS_NOTCONVERGED, KGS_EDIVERGED))
    return rc, done.value, res.value


def kgs_moments(ctx, out=None):
    n = ctx.prob.ncell
    if out is None:
        out = np.empty(8 * n)
    _check(load().kgs_moments(ctx.handle, out.ctypes.data_as(_dp)), "kgs_moments")
    return out.reshape((8,) + ctx.shape)


def kgs_moments_device(ctx, dev_ptr):
    return _check(load().kgs_moments_device(ctx.handle, ctypes.c_void_p(dev_ptr)), "kgs_moments_device")


def kgs_rho_w(ctx):
    out = np.empty(6 * ctx.prob.ncell)
    _check(load().kgs_rho_w(ctx.handle, out.ctypes.data_as(_dp)), "kgs_rho_w")
    return out.reshape((6,) + ctx.shape)


def kgs_set_rho_w(ctx, rho_w):
    a = _arr(rho_w).reshape(-1)
    return _check(load().kgs_set_rho_w(ctx.handle, a.ctypes.data_as(_dp)), "kgs_set_rho_w")


def kgs_save(ctx):
    n = ctypes.c_size_t(0)
    _check(load().kgs_save(ctx.handle, None, ctypes.byref(n)), "kgs_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().kgs_save(ctx.handle, buf, ctypes.byref(n)), "kgs_save")
    return buf.raw[: n.value]


def kgs_load(ctx, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    return load().kgs_load(ctx.handle, buf, len(data))


def kgs_info(ctx):
    info = KgsInfo()
    _check(load().kgs_info(ctx.handle, ctypes.byref(info)), "kgs_info")
    return {name: getattr(info, name) for name, _ in KgsInfo._fields_}


def kgs_set_profiling(ctx, enable=True):
    return _check(load().kgs_set_profiling(ctx.handle, 1 if enable else 0), "kgs_set_profiling")


def kgs_profile(ctx):
    ms = ctypes.c_double(0.0)
    sl = ctypes.c_longlong(0)
    kl = ctypes.c_longlong(0)
    _check(load().kgs_profile(ctx.handle, ctypes.byref(ms), ctypes.byref(sl), ctypes.byref(kl)), "kgs_profile")
    return ms.value, sl.value, kl.value


def kgs_sweep_sums(ctx, sums_dev):
    """One sweep of the context's velocities: per-cell sums [19][ncell] (FP64) written to the device
    pointer sums_dev (int); the state does not change."""
    return _check(load().kgs_sweep_sums(ctx.handle, ctypes.c_void_p(sums_dev)), "kgs_sweep_sums")


def kgs_close_sums(ctx, sums_dev):
    """Closure from the summed per-cell sums at the device pointer sums_dev; returns (rc, residual).
    KGS_EDIVERGED is returned, other errors raise."""
    res = ctypes.c_double(0.0)
    rc = load().kgs_close_sums(ctx.handle, ctypes.c_void_p(sums_dev), ctypes.byref(res))
    _check(rc, "kgs_close_sums", allow=(KGS_EDIVERGED,))
    return rc, res.value


def kgs_destroy(ctx):
    if ctx.handle:
        load().kgs_destroy(ctx.handle)
        ctx.handle = None


def kgs_strerror(code):
    return load().kgs_strerror(int(code)).decode()


# ---- raw-pointer variants (pinned host or device buffers owned by the caller) ----

def kgs_save_ptr(ctx, ptr, nbytes):
    n = ctypes.c_size_t(nbytes)
    _check(load().kgs_save(ctx.handle, ctypes.c_void_p(ptr), ctypes.byref(n)), "kgs_save")
    return n.value


def kgs_save_size(ctx):
    n = ctypes.c_size_t(0)
    _check(load().kgs_save(ctx.handle, None, ctypes.byref(n)), "kgs_save")
    return n.value


def kgs_load_ptr(ctx, ptr, nbytes):
    return _check(load().kgs_load(ctx.handle, ctypes.c_void_p(ptr), nbytes), "kgs_load")


def kgs_moments_ptr(ctx, ptr):
    return _check(load().kgs_moments(ctx.handle, ctypes.cast(ctypes.c_void_p(ptr), _dp)), "kgs_moments")


def kgs_iterate_noalloc(prob, macros_in, rho_w_in, macros_out, rho_w_out, M0=0.0, precision=KGS_FP64,
                        stream=None):
    """kgs_iterate_noalloc with device pointers (ints) for the four state
    buffers; returns (rc, residual).  KGS_EDIVERGED is returned, other errors
    raise."""
    keep = []
    g, v, gas, bc, solid_p = _problem_structs(prob, keep)
    res = ctypes.c_double(0.0)
    rc = load().kgs_iterate_noalloc(ctypes.byref(g), solid_p, ctypes.byref(v), ctypes.byref(gas),
                                    ctypes.byref(bc), int(precision), int(prob.wall_mode), float(M0),
                                    ctypes.c_void_p(macros_in), ctypes.c_void_p(rho_w_in),
                                    ctypes.c_void_p(macros_out), ctypes.c_void_p(rho_w_out), ctypes.byref(res),
                                    ctypes.c_void_p(stream) if stream else None)
    _check(rc, "kgs_iterate_noalloc", allow=(KGS_EDIVERGED,))
    return rc, res.value


# ---- batches ----

class KgsProblem(ctypes.Structure):
    _fields_ = [("grid", KgsGrid), ("solid", ctypes.POINTER(ctypes.c_uint8)), ("vgrid", KgsVgrid),
                ("gas", KgsGas), ("bc", KgsBc), ("wall_norm", ctypes.c_int), ("mass_rescale", ctypes.c_int),
                ("q_lagged", ctypes.c_int)]


SIGNATURES.update({
    "kgs_autotune": (ctypes.c_int, [ctypes.POINTER(KgsProblem), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
    "kgs_batch_setup": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(KgsProblem),
                                       ctypes.POINTER(KgsOpts)]),
    "kgs_batch_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp]),
    "kgs_batch_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp]),
    "kgs_batch_set_initial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp]),
    "kgs_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(KgsInfo)]),
    "kgs_batch_profile": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_longlong)]),
    "kgs_batch_fault": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int]),
    "kgs_batch_solve": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(KgsProblem),
                                       ctypes.POINTER(KgsOpts), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), _dp]),
    "kgs_batch_destroy": (None, [ctypes.c_void_p]),
})


def _problem(prob, keep):
    g, v, gas, bc, solid_p = _problem_structs(prob, keep)
    return KgsProblem(g, solid_p, v, gas, bc, int(prob.wall_mode), int(prob.mass_rescale),
                      int(getattr(prob, "q_lagged", 0)))


def kgs_autotune(prob, precision=KGS_MIXED):
    """Returns (v_per_cta, block_z) chosen by timing on the current device."""
    keep = []
    p = _problem(prob, keep)
    vpc, bz = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().kgs_autotune(ctypes.byref(p), int(precision), ctypes.byref(vpc), ctypes.byref(bz)), "kgs_autotune")
    return vpc.value, bz.value


class Batch:
    """Handle of one kgs_batch."""

    def __init__(self, handle, probs):
        self.handle = handle
        self.probs = probs

    def __del__(self):
        if getattr(self, "handle", None):
            kgs_batch_destroy(self)


def kgs_batch_setup(probs, precision=KGS_MIXED, max_iters=1000, tol=1e-8, v_per_cta=0, block_z=0, stream=None):
    keep = []
    arr = (KgsProblem * len(probs))(*[_problem(p, keep) for p in probs])
    opts = KgsOpts(precision, 0, 0, max_iters, tol, v_per_cta, block_z, ctypes.c_void_p(stream) if stream else None)
    h = ctypes.c_void_p()
    _check(load().kgs_batch_setup(ctypes.byref(h), len(probs), arr, ctypes.byref(opts)), "kgs_batch_setup")
    return Batch(h, probs)


def kgs_batch_iterate(b, n_iters=1):
    """Returns (rc, iterations per instance, residual per instance); the
    status codes KGS_NOTCONVERGED, KGS_EDIVERGED and KGS_ETIMEOUT are
    returned, other errors raise."""
    n = len(b.probs)
    done = (ctypes.c_int * n)()
    res = (ctypes.c_double * n)()
    rc = load().kgs_batch_iterate(b.handle, int(n_iters), done, res)
    _check(rc, "kgs_batch_iterate", allow=(KGS_NOTCONVERGED, KGS_EDIVERGED, KGS_ETIMEOUT))
    return rc, list(done), list(res)


def kgs_batch_solve(probs, tol=1e-6, max_iters=1000, v_per_cta=0, block_z=0, stream=None):
    """kgs_batch_solve: mixed then FP64 per instance.  Returns (rc, batch, iterations in the mixed phase,
    iterations in the FP64 phase, final residuals); the batch holds the FP64 results.  KGS_NOTCONVERGED
    is returned, other errors raise."""
    keep = []
    n = len(probs)
    arr = (KgsProblem * n)(*[_problem(p, keep) for p in probs])
    opts = KgsOpts(KGS_MIXED, 0, 0, max_iters, tol, v_per_cta, block_z, ctypes.c_void_p(stream) if stream else None)
    h = ctypes.c_void_p()
    im = (ctypes.c_int * n)()
    idd = (ctypes.c_int * n)()
    res = (ctypes.c_double * n)()
    rc = load().kgs_batch_solve(ctypes.byref(h), n, arr, ctypes.byref(opts), im, idd, res)
    _check(rc, "kgs_batch_solve", allow=(KGS_NOTCONVERGED,))
    return rc, Batch(h, probs), list(im), list(idd), list(res)


def kgs_batch_moments(b, i):
    p = b.probs[i]
    out = np.empty(8 * p.ncell)
    _check(load().kgs_batch_moments(b.handle, int(i), out.ctypes.data_as(_dp)), "kgs_batch_moments")
    return out.reshape(8, p.nz, p.ny, p.nx)


def kgs_batch_set_initial(b, i, macros=None):
    if macros is None:
        return _check(load().kgs_batch_set_initial(b.handle, int(i), _dp()), "kgs_batch_set_initial")
    m = _arr(macros).reshape(-1)
    return _check(load().kgs_batch_set_initial(b.handle, int(i), m.ctypes.data_as(_dp)), "kgs_batch_set_initial")


def kgs_batch_info(b, i):
    info = KgsInfo()
    _check(load().kgs_batch_info(b.handle, int(i), ctypes.byref(info)), "kgs_batch_info")
    return {name: getattr(info, name) for name, _ in KgsInfo._fields_}


def kgs_batch_profile(b):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    kl = ctypes.c_longlong(0)
    _check(load().kgs_batch_profile(b.handle, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(kl)),
           "kgs_batch_profile")
    return ms.value, n.value, kl.value


def kgs_batch_fault(b, spin_limit=20000000, unpublished_item=-1):
    return _check(load().kgs_batch_fault(b.handle, int(spin_limit), int(unpublished_item)), "kgs_batch_fault")


SIGNATURES["kgs_solve"] = (ctypes.c_int, [ctypes.POINTER(KgsProblem), _dp, ctypes.c_double, ctypes.c_int, _dp,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp,
                                          ctypes.c_void_p])


def kgs_solve(prob, initial=None, tol=1e-6, max_iters=5000, stream=None):
    """Mixed iterations while they make progress, then FP64 to tol.  Returns
    (rc, macros [8, nz, ny, nx], mixed iterations, FP64 iterations,
    residual); KGS_NOTCONVERGED is returned, other errors raise."""
    keep = []
    p = _problem(prob, keep)
    out = np.empty(8 * prob.ncell)
    init = None if initial is None else _arr(initial).reshape(-1)
    nm, nd = ctypes.c_int(0), ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = load().kgs_solve(ctypes.byref(p), init.ctypes.data_as(_dp) if init is not None else _dp(), float(tol),
                          int(max_iters), out.ctypes.data_as(_dp), ctypes.byref(nm), ctypes.byref(nd),
                          ctypes.byref(res), ctypes.c_void_p(stream) if stream else None)
    _check(rc, "kgs_solve", allow=(KGS_NOTCONVERGED,))
    return rc, out.reshape(8, prob.nz, prob.ny, prob.nx), nm.value, nd.value, res.value


def kgs_batch_destroy(b):
    if b.handle:
        load().kgs_batch_destroy(b.handle)
        b.handle = None


# ---- learned initial guess (kgs_net_*, kgs_surrogate_*) ----
_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p
SIGNATURES.update({
    "kgs_net_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.c_ulonglong, _vp]),
    "kgs_net_num_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "kgs_net_get": (ctypes.c_int, [_vp, ctypes.c_int, _fp]),
    "kgs_net_set_params": (ctypes.c_int, [_vp, _fp]),
    "kgs_net_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "kgs_net_train_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_float, _fp]),
    "kgs_net_destroy": (None, [_vp]),
    "kgs_surrogate_features": (ctypes.c_int, [ctypes.c_int] * 6 + [_vp, _vp, ctypes.c_double, ctypes.c_double,
                                                                   _vp, _vp, _vp]),
    "kgs_surrogate_target": (ctypes.c_int, [ctypes.c_longlong, _vp, _vp, _vp, _vp]),
    "kgs_surrogate_apply": (ctypes.c_int, [ctypes.c_longlong, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int), _vp]),
})


class Net:
    """Handle of one kgs_net; channels = (input, hidden..., output)."""

    def __init__(self, handle, channels):
        self.handle = handle
        self.channels = tuple(channels)

    def __del__(self):
        if getattr(self, "handle", None):
            kgs_net_destroy(self)


def _sp(stream):
    return ctypes.c_void_p(stream) if stream else None


def kgs_net_create(channels, seed=0, stream=None):
    ch = (ctypes.c_int * len(channels))(*channels)
    h = ctypes.c_void_p()
    _check(load().kgs_net_create(ctypes.byref(h), len(channels) - 1, ch, int(seed), _sp(stream)), "kgs_net_create")
    return Net(h, channels)


def kgs_net_num_params(net):
    r, p = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(load().kgs_net_num_params(net.handle, ctypes.byref(r), ctypes.byref(p)), "kgs_net_num_params")
    return r.value, p.value


def kgs_net_get(net, what=0):
    """Parameters (what=0) or gradients (what=1) as one float32 vector in the
    host layout: per layer W[27][Cout][Cin] then b[Cout]."""
    n, _ = kgs_net_num_params(net)
    out = np.empty(n, np.float32)
    _check(load().kgs_net_get(net.handle, int(what), out.ctypes.data_as(_fp)), "kgs_net_get")
    return out


def kgs_net_set_params(net, flat):
    f = _arr(flat, np.float32)
    return _check(load().kgs_net_set_params(net.handle, f.ctypes.data_as(_fp)), "kgs_net_set_params")


def kgs_net_forward(net, x_ptr, shape, y_ptr):
    """x_ptr, y_ptr: device addresses of [B][D][H][W][C] float32 tensors."""
    B, D, H, W = shape
    return _check(load().kgs_net_forward(net.handle, ctypes.c_void_p(x_ptr), B, D, H, W, ctypes.c_void_p(y_ptr)),
                  "kgs_net_forward")


def kgs_net_train_step(net, x_ptr, target_ptr, mask_ptr, shape, lr):
    """One Adam step (lr <= 0: gradients only); returns the loss before it."""
    B, D, H, W = shape
    loss = ctypes.c_float(0.0)
    _check(load().kgs_net_train_step(net.handle, ctypes.c_void_p(x_ptr), ctypes.c_void_p(target_ptr),
                                     ctypes.c_void_p(mask_ptr) if mask_ptr else None, B, D, H, W,
                                     float(lr), ctypes.byref(loss)), "kgs_net_train_step")
    return loss.value


def kgs_net_destroy(net):
    if net.handle:
        load().kgs_net_destroy(net.handle)
        net.handle = None


def kgs_surrogate_features(fine_shape, coarse_shape, coarse_ptr, solid_ptr, kn, u_lid, x_ptr, up_ptr, stream=None):
    """fine_shape, coarse_shape: (nx, ny, nz)."""
    return _check(load().kgs_surrogate_features(*fine_shape, *coarse_shape, ctypes.c_void_p(coarse_ptr),
                                                ctypes.c_void_p(solid_ptr) if solid_ptr else None, float(kn),
                                                float(u_lid), ctypes.c_void_p(x_ptr), ctypes.c_void_p(up_ptr),
                                                _sp(stream)), "kgs_surrogate_features")


def kgs_surrogate_target(ncell, fine_ptr, up_ptr, target_ptr, stream=None):
    return _check(load().kgs_surrogate_target(int(ncell), ctypes.c_void_p(fine_ptr), ctypes.c_void_p(up_ptr),
                                              ctypes.c_void_p(target_ptr), _sp(stream)), "kgs_surrogate_target")


def kgs_surrogate_apply(ncell, up_ptr, y_ptr, macros_ptr, stream=None):
    """Returns the number of cells whose guess is not a physical state."""
    bad = ctypes.c_int(0)
    _check(load().kgs_surrogate_apply(int(ncell), ctypes.c_void_p(up_ptr), ctypes.c_void_p(y_ptr),
                                      ctypes.c_void_p(macros_ptr), ctypes.byref(bad), _sp(stream)),
           "kgs_surrogate_apply")
    return bad.value
