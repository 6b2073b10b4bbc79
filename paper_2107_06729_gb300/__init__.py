"""GB300-native demag-extrapolated explicit LLG integrator (arXiv 2107.06729).

Thin ctypes binding over the C ABI of ``libmmx.so`` (``include/mmx.h``):
the module-level functions carry the same names as the C entry points and
only marshal arguments; every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: if ``libmmx.so`` is missing or
fails to load, every call raises.

Magnetisation buffers are torch tensors (CUDA or pinned/regular CPU memory)
or numpy arrays of shape ``[3, nz, ny, nx]`` and dtype float64 (MMX_FP64) or
float32 (MMX_FP32_MIXED).  Fields are in A/m, lengths in m, times in s.
"""
import ctypes
import os

from . import workloads  # noqa: F401  (seeded input generators)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmx.so")

MMX_OK = 0
MMX_WARN_HMIN = 1
MMX_ERR_ARG = -1
MMX_ERR_OOM = -2
MMX_ERR_CUDA = -3
MMX_ERR_NONFINITE = -4
MMX_ERR_TIMEOUT = -5
MMX_ERR_STATE = -6
MMX_FP64 = 0
MMX_FP32_MIXED = 1
MMX_NPROF = 6
METHODS = {"RK4": 0, "HEUN12": 1, "RK23": 2, "RKF45": 3, "RKCK45": 4, "RKDP54": 5, "RKF56": 6, "ABM2": 7}
PROFILE_CLASSES = ["x_forward_fft", "yz_fft_tensor_multiply", "x_inverse_fft", "llg_stage", "llg_last_stage", "controller"]


class mmx_mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class mmx_material(ctypes.Structure):
    _fields_ = [("Ms", ctypes.c_double), ("A", ctypes.c_double), ("K", ctypes.c_double),
                ("ku", ctypes.c_double * 3), ("alpha", ctypes.c_double), ("gamma", ctypes.c_double)]


class mmx_field(ctypes.Structure):
    _fields_ = [("H0", ctypes.c_double * 3), ("pulse_H", ctypes.c_double * 3),
                ("t_on", ctypes.c_double), ("t_off", ctypes.c_double)]


class mmx_integrator(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("extrap_order", ctypes.c_int), ("adaptive", ctypes.c_int),
                ("h", ctypes.c_double), ("tol", ctypes.c_double), ("hmin", ctypes.c_double),
                ("hmax", ctypes.c_double), ("cmin", ctypes.c_double), ("cmax", ctypes.c_double),
                ("safety", ctypes.c_double)]


class mmx_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("h", ctypes.c_double), ("last_err", ctypes.c_double),
                ("accepted", ctypes.c_longlong), ("rejected", ctypes.c_longlong),
                ("exact_evals", ctypes.c_longlong), ("extrap_evals", ctypes.c_longlong),
                ("forced_accepts", ctypes.c_longlong), ("attempts", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong)]


class mmx_plan(ctypes.Structure):
    _fields_ = [("yz_pass", ctypes.c_int), ("x_rows", ctypes.c_int), ("xi_tma", ctypes.c_int),
                ("tuned", ctypes.c_int), ("kernels_per_demag", ctypes.c_int),
                ("demag_us", ctypes.c_double)]


# every entry point declared in include/mmx.h, with its C signature
_VP = ctypes.c_void_p
SIGNATURES = {
    "mmx_create": (ctypes.c_int, [ctypes.POINTER(mmx_mesh), ctypes.POINTER(mmx_material),
                                  ctypes.POINTER(mmx_field), ctypes.POINTER(mmx_integrator),
                                  ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
    "mmx_set_m": (ctypes.c_int, [_VP, _VP]),
    "mmx_get_m": (ctypes.c_int, [_VP, _VP]),
    "mmx_set_time": (ctypes.c_int, [_VP, ctypes.c_double]),
    "mmx_demag": (ctypes.c_int, [_VP, _VP, _VP]),
    "mmx_run": (ctypes.c_int, [_VP, ctypes.c_double]),
    "mmx_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "mmx_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(mmx_stats)]),
    "mmx_save_state": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_size_t)]),
    "mmx_load_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "mmx_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int]),
    "mmx_get_profile": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "mmx_get_plan": (ctypes.c_int, [_VP, ctypes.POINTER(mmx_plan)]),
    "mmx_demag_static": (ctypes.c_int, [ctypes.POINTER(mmx_mesh), ctypes.c_double, ctypes.c_int, _VP, _VP, _VP]),
    "mmx_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP), _VP, ctypes.POINTER(_VP)]),
    "mmx_batch_run": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "mmx_batch_last_error": (ctypes.c_char_p, [_VP]),
    "mmx_batch_destroy": (None, [_VP]),
    "mmx_last_error": (ctypes.c_char_p, [_VP]),
    "mmx_destroy": (None, [_VP]),
    # learned residual correction (include/mmx_residual.h)
    "mmx_rnet_create": (ctypes.c_int, [ctypes.c_longlong, _VP, ctypes.POINTER(_VP)]),
    "mmx_rnet_set_params": (ctypes.c_int, [_VP, _VP]),
    "mmx_rnet_get_params": (ctypes.c_int, [_VP, _VP]),
    "mmx_rnet_forward": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "mmx_rnet_train_step": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_double)]),
    "mmx_rnet_get_grads": (ctypes.c_int, [_VP, _VP]),
    "mmx_rnet_get_activation": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_size_t]),
    "mmx_rnet_last_error": (ctypes.c_char_p, [_VP]),
    "mmx_rnet_destroy": (None, [_VP]),
    "mmx_residual_sample": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double), _VP,
                                           ctypes.c_double, _VP, _VP]),
    "mmx_set_residual": (ctypes.c_int, [_VP, _VP]),
    "mmx_set_residual_check": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double]),
    "mmx_residual_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
}

MMX_RNET_PARAMS = 63171

_lib = None


class MMXError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libmmx error %d: %s" % (code, msg))
        self.code = code


def lib():
    """Loads libmmx.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmmx.so is not built (run __graft_entry__.build()); "
                              "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, ctx=None, allow_warn=True):
    if rc < 0 or (rc > 0 and not allow_warn):
        msg = lib().mmx_last_error(ctx)
        raise MMXError(rc, msg.decode() if msg else "")
    return rc


def _ptr(buf):
    """Raw address of a torch tensor or numpy array (contiguous)."""
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    if hasattr(buf, "ctypes"):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return buf.ctypes.data
    raise TypeError("expected a torch tensor or numpy array")


# ---------------------------------------------------------------- C names --
def mmx_create(mesh, material, field, integrator, precision, cuda_stream=None):
    """Returns an opaque context handle (int).  See include/mmx.h."""
    out = _VP()
    rc = lib().mmx_create(ctypes.byref(mesh), ctypes.byref(material), ctypes.byref(field),
                          ctypes.byref(integrator), int(precision), cuda_stream, ctypes.byref(out))
    _check(rc, None)
    return out.value


def mmx_set_m(ctx, m):
    return _check(lib().mmx_set_m(ctx, _ptr(m)), ctx)


def mmx_get_m(ctx, m):
    return _check(lib().mmx_get_m(ctx, _ptr(m)), ctx)


def mmx_set_time(ctx, t):
    return _check(lib().mmx_set_time(ctx, float(t)), ctx)


def mmx_demag(ctx, m_dev, H_dev):
    return _check(lib().mmx_demag(ctx, _ptr(m_dev), _ptr(H_dev)), ctx)


def mmx_run(ctx, t_end):
    return _check(lib().mmx_run(ctx, float(t_end)), ctx)


def mmx_step(ctx, n_accepted):
    return _check(lib().mmx_step(ctx, int(n_accepted)), ctx)


def mmx_get_stats(ctx):
    s = mmx_stats()
    _check(lib().mmx_get_stats(ctx, ctypes.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in mmx_stats._fields_}


def mmx_save_state(ctx):
    n = ctypes.c_size_t(0)
    _check(lib().mmx_save_state(ctx, None, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().mmx_save_state(ctx, buf, ctypes.byref(n)), ctx)
    return buf.raw[:n.value]


def mmx_load_state(ctx, blob):
    buf = ctypes.create_string_buffer(blob, len(blob))
    return _check(lib().mmx_load_state(ctx, buf, len(blob)), ctx)


def mmx_set_profiling(ctx, enable):
    return _check(lib().mmx_set_profiling(ctx, int(enable)), ctx)


def mmx_get_profile(ctx):
    ms = (ctypes.c_double * MMX_NPROF)()
    n = (ctypes.c_longlong * MMX_NPROF)()
    _check(lib().mmx_get_profile(ctx, ms, n), ctx)
    return {PROFILE_CLASSES[i]: (ms[i], n[i]) for i in range(MMX_NPROF)}


def mmx_get_plan(ctx):
    p = mmx_plan()
    _check(lib().mmx_get_plan(ctx, ctypes.byref(p)), ctx)
    return {k: getattr(p, k) for k, _ in mmx_plan._fields_}


def mmx_demag_static(mesh, Ms, precision, m_dev, H_dev, cuda_stream=None):
    """Allocation-free exact demag (see include/mmx.h); mesh is an mmx_mesh."""
    rc = lib().mmx_demag_static(ctypes.byref(mesh), float(Ms), int(precision), _ptr(m_dev), _ptr(H_dev),
                                cuda_stream)
    return _check(rc, None)


def mmx_batch_create(members, cuda_stream=None):
    """Groups context handles into a batch run by one graph launch."""
    arr = (_VP * len(members))(*members)
    out = _VP()
    _check(lib().mmx_batch_create(len(members), arr, cuda_stream, ctypes.byref(out)), None)
    return out.value


def mmx_batch_run(batch, t_end):
    """Integrates member i to t_end[i]; returns (overall code, per-member
    codes).  Raises on an error of the batch itself; member errors are left
    in the codes (text from each member's mmx_last_error)."""
    n = len(t_end)
    te = (ctypes.c_double * n)(*[float(t) for t in t_end])
    st = (ctypes.c_int * n)()
    rc = lib().mmx_batch_run(batch, te, st)
    msg = mmx_batch_last_error(batch)
    if rc < 0 and msg:
        raise MMXError(rc, msg)
    return rc, list(st)


def mmx_batch_last_error(batch=None):
    msg = lib().mmx_batch_last_error(batch)
    return msg.decode() if msg else ""


def mmx_batch_destroy(batch):
    if batch:
        lib().mmx_batch_destroy(batch)


def mmx_last_error(ctx=None):
    msg = lib().mmx_last_error(ctx)
    return msg.decode() if msg else ""


def mmx_destroy(ctx):
    if ctx:
        lib().mmx_destroy(ctx)


# ------------------------------------------- learned residual (mmx_residual.h) --
def _rcheck(rc, net):
    if rc < 0:
        raise MMXError(rc, mmx_rnet_last_error(net))
    return rc


def mmx_rnet_create(max_cells, cuda_stream=None):
    out = _VP()
    rc = lib().mmx_rnet_create(int(max_cells), cuda_stream, ctypes.byref(out))
    if rc < 0:
        raise MMXError(rc, "mmx_rnet_create failed")
    return out.value


def mmx_rnet_set_params(net, params):
    """params: host float32 array of MMX_RNET_PARAMS values."""
    return _rcheck(lib().mmx_rnet_set_params(net, _ptr(params)), net)


def mmx_rnet_get_params(net, params):
    return _rcheck(lib().mmx_rnet_get_params(net, _ptr(params)), net)


def mmx_rnet_forward(net, n, x_dev, r_dev=None):
    """n = (nx, ny, nz); x_dev float32 [6][cells], r_dev float32 [3][cells] or None."""
    return _rcheck(lib().mmx_rnet_forward(net, *n, _ptr(x_dev), _ptr(r_dev) if r_dev is not None else None), net)


def mmx_rnet_train_step(net, n, x_dev, target_dev, lr):
    """One Adam step; returns the loss before the update."""
    loss = ctypes.c_double()
    _rcheck(lib().mmx_rnet_train_step(net, *n, _ptr(x_dev), _ptr(target_dev), float(lr), ctypes.byref(loss)), net)
    return loss.value


def mmx_rnet_get_grads(net, grads):
    return _rcheck(lib().mmx_rnet_get_grads(net, _ptr(grads)), net)


def mmx_rnet_get_activation(net, layer, dst):
    """dst: host array (uint16 for layers 0-3, float32 for layer 4) of the exact size."""
    return _rcheck(lib().mmx_rnet_get_activation(net, int(layer), _ptr(dst), dst.nbytes), net)


def mmx_rnet_last_error(net=None):
    msg = lib().mmx_rnet_last_error(net)
    return msg.decode() if msg else ""


def mmx_rnet_destroy(net):
    if net:
        lib().mmx_rnet_destroy(net)


def mmx_residual_sample(ctx, p, m_nodes_dev, t_nodes, m_dev, t, x_dev, target_dev):
    """Training pair (x, target) of the residual net from ctx's exact demag."""
    tn = (ctypes.c_double * (p + 1))(*[float(v) for v in t_nodes])
    rc = lib().mmx_residual_sample(ctx, int(p), _ptr(m_nodes_dev), tn, _ptr(m_dev), float(t), _ptr(x_dev),
                                   _ptr(target_dev))
    return _check(rc, ctx)


def mmx_set_residual_check(ctx, every, tol):
    return _check(lib().mmx_set_residual_check(ctx, int(every), float(tol)), ctx)


def mmx_residual_stats(ctx):
    out = (ctypes.c_longlong * 4)()
    _check(lib().mmx_residual_stats(ctx, out), ctx)
    return {"fallbacks": out[0], "checks": out[1], "check_fails": out[2], "net_ok": out[3]}


def mmx_set_residual(ctx, net):
    """Attaches the residual net (handle) to ctx's extrapolated stages; None detaches."""
    return _check(lib().mmx_set_residual(ctx, net), ctx)


class RNet:
    """Owner of one residual net (the C calls above underneath)."""

    def __init__(self, max_cells, params=None, stream=None):
        handle = stream
        if stream is not None and hasattr(stream, "cuda_stream"):
            handle = stream.cuda_stream
        self.handle = mmx_rnet_create(max_cells, handle)
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        import numpy as np
        mmx_rnet_set_params(self.handle, np.ascontiguousarray(params, dtype=np.float32))

    def params(self):
        import numpy as np
        out = np.empty(MMX_RNET_PARAMS, dtype=np.float32)
        mmx_rnet_get_params(self.handle, out)
        return out

    def grads(self):
        import numpy as np
        out = np.empty(MMX_RNET_PARAMS, dtype=np.float32)
        mmx_rnet_get_grads(self.handle, out)
        return out

    def forward(self, x, r=None):
        """x: CUDA float32 tensor [6, nz, ny, nx]; returns r [3, nz, ny, nx]."""
        if r is None:
            r = x.new_empty((3,) + tuple(x.shape[1:]))
        mmx_rnet_forward(self.handle, (x.shape[3], x.shape[2], x.shape[1]), x, r)
        return r

    def train_step(self, x, target, lr):
        return mmx_rnet_train_step(self.handle, (x.shape[3], x.shape[2], x.shape[1]), x, target, lr)

    def activation(self, layer, cells):
        """Layer 0-3: the BF16 input of that layer as float32 [cells, channels];
        layer 4: the output r as float32 [3, cells]."""
        import numpy as np
        if layer == 4:
            out = np.empty((3, cells), dtype=np.float32)
            mmx_rnet_get_activation(self.handle, 4, out)
            return out
        raw = np.empty((cells, 16 if layer == 0 else 32), dtype=np.uint16)
        mmx_rnet_get_activation(self.handle, layer, raw)
        return (raw.astype(np.uint32) << 16).view(np.float32)

    def close(self):
        if getattr(self, "handle", None):
            mmx_rnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- marshalling --
def make_structs(mesh, material, field, integrator):
    """Builds the C structs from the dict descriptions used in ``workloads``."""
    M = mmx_mesh(*mesh["n"], *mesh["d"])
    A = mmx_material()
    A.Ms = material["Ms"]
    A.A = material.get("A", 0.0)
    A.K = material.get("K", 0.0)
    for i, v in enumerate(material.get("ku", (1.0, 0.0, 0.0))):
        A.ku[i] = v
    A.alpha = material["alpha"]
    A.gamma = material["gamma"]
    F = mmx_field()
    for i in range(3):
        F.H0[i] = field.get("H0", (0.0, 0.0, 0.0))[i]
        F.pulse_H[i] = field.get("pulse", (0.0, 0.0, 0.0))[i]
    F.t_on = field.get("t_on", 0.0)
    F.t_off = field.get("t_off", 0.0)
    I = mmx_integrator()
    I.method = METHODS[integrator["method"]]
    I.extrap_order = integrator.get("extrap_order", -1)
    I.adaptive = int(bool(integrator.get("adaptive", False)))
    I.h = integrator["h"]
    I.tol = integrator.get("tol", 1e-5)
    I.hmin = integrator.get("hmin", 1e-15)
    I.hmax = integrator.get("hmax", 3e-12)
    I.cmin = integrator.get("cmin", 0.01)
    I.cmax = integrator.get("cmax", 2.0)
    I.safety = integrator.get("safety", 0.8)
    return M, A, F, I


class Context:
    """Convenience owner of one mmx context (the C calls above underneath)."""

    def __init__(self, mesh, material, field, integrator, precision="fp64", stream=None):
        self.precision = MMX_FP64 if precision in ("fp64", MMX_FP64) else MMX_FP32_MIXED
        self.shape = (3, mesh["n"][2], mesh["n"][1], mesh["n"][0])
        self._structs = make_structs(mesh, material, field, integrator)
        handle = stream
        if stream is not None and hasattr(stream, "cuda_stream"):
            handle = stream.cuda_stream
        self.handle = mmx_create(*self._structs, self.precision, handle)

    @property
    def dtype_name(self):
        return "float64" if self.precision == MMX_FP64 else "float32"

    def set_m(self, m):
        return mmx_set_m(self.handle, m)

    def get_m(self, out):
        return mmx_get_m(self.handle, out)

    def set_time(self, t):
        return mmx_set_time(self.handle, t)

    def demag(self, m_dev, H_dev):
        return mmx_demag(self.handle, m_dev, H_dev)

    def run(self, t_end):
        return mmx_run(self.handle, t_end)

    def step(self, n):
        return mmx_step(self.handle, n)

    def stats(self):
        return mmx_get_stats(self.handle)

    def save_state(self):
        return mmx_save_state(self.handle)

    def load_state(self, blob):
        return mmx_load_state(self.handle, blob)

    def set_profiling(self, on):
        return mmx_set_profiling(self.handle, on)

    def set_residual_check(self, every, tol):
        return mmx_set_residual_check(self.handle, every, tol)

    def residual_stats(self):
        return mmx_residual_stats(self.handle)

    def set_residual(self, net):
        """Attaches an RNet (kept alive here) to the extrapolated stages; None detaches."""
        mmx_set_residual(self.handle, net.handle if net is not None else None)
        self._rnet = net

    def plan(self):
        return mmx_get_plan(self.handle)

    def profile(self):
        return mmx_get_profile(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            mmx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owner of a batch over existing Context objects (kept alive here)."""

    def __init__(self, contexts, stream=None):
        self.contexts = list(contexts)
        handle = stream
        if stream is not None and hasattr(stream, "cuda_stream"):
            handle = stream.cuda_stream
        self.handle = mmx_batch_create([c.handle for c in self.contexts], handle)

    def run(self, t_end):
        """t_end: one time for every member, or a sequence of len(members)."""
        if not hasattr(t_end, "__len__"):
            t_end = [t_end] * len(self.contexts)
        rc, status = mmx_batch_run(self.handle, t_end)
        for c, r in zip(self.contexts, status):
            if r < 0:
                raise MMXError(r, mmx_last_error(c.handle))
        return rc, status

    def close(self):
        if getattr(self, "handle", None):
            mmx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
