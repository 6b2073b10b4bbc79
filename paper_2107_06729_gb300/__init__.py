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
MMX_NPROF = 5
METHODS = {"RK4": 0, "HEUN12": 1, "RK23": 2, "RKF45": 3, "RKCK45": 4, "RKDP54": 5, "RKF56": 6, "ABM2": 7}
PROFILE_CLASSES = ["x_forward_fft", "yz_fft_tensor_multiply", "x_inverse_fft", "llg_stage", "llg_last_stage"]


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
                ("cluster_ctas", ctypes.c_int), ("tuned", ctypes.c_int), ("kernels_per_demag", ctypes.c_int),
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
}

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
    return _check(lib().mmx_set_profiling(ctx, int(bool(enable))), ctx)


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
