"""Python binding of the C ABI in include/sesc.h (argument marshalling only).

Every step of the right-hand side runs in the CUDA library libsesc.so; this
module only checks tensor shapes / dtypes / devices, passes raw device pointers
and the current CUDA stream, and turns error codes into exceptions. There is no
fallback: if the library is missing or fails to load, an exception is raised.

Tensors are torch CUDA tensors (PyTorch provides device memory and streams).
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsesc.so")
# the bounds-checked build (python -m paper_2011_03338_gb300.build --bounds): selected
# for a process by SESC_LIBRARY=<path>
BOUNDS_LIB_PATH = os.path.join(_HERE, "libsesc_bounds.so")

(SESC_OK, SESC_EINVAL, SESC_ENOMEM, SESC_ECUDA, SESC_ENONPERMISSIBLE, SESC_ENONFINITE, SESC_ETOOLARGE,
 SESC_ETIMEOUT, SESC_EBOUNDS) = range(9)
BC_PERIODIC, BC_WALL, BC_OUTFLOW, BC_HALO = 0, 1, 2, 3
NODES = {"gauss": 0, "lgl": 1, "lobatto": 1}

# Every exported symbol of the library, in header order.
SYMBOLS = ("sesc_create", "sesc_destroy", "sesc_num_elements", "sesc_num_coeffs", "sesc_indicator",
           "sesc_rhs", "sesc_rk_stage", "sesc_dt", "sesc_rk3_step", "sesc_rk_stage_ex", "sesc_ssprk54_step",
           "sesc_status", "sesc_reset_status", "sesc_level_counts", "sesc_halo_bytes", "sesc_pack_halo",
           "sesc_set_halo", "sesc_stage_finish",
           "sesc_rhs_vjp", "sesc_rk_stage_vjp", "sesc_set_timing", "sesc_kernel_times", "sesc_rhs_static",
           "sesc_batch_create", "sesc_batch_destroy", "sesc_batch_offsets", "sesc_batch_num_groups",
           "sesc_batch_group_of", "sesc_batch_rhs", "sesc_batch_dt", "sesc_batch_rk3_step", "sesc_batch_use_graph",
           "sesc_batch_grids", "sesc_batch_set_grids", "sesc_batch_autotune", "sesc_batch_fused",
           "sesc_batch_set_fused", "sesc_batch_set_barrier_cap", "sesc_batch_status",
           "sesc_batch_reset_status", "sesc_strerror", "sesc_set_stage_cap", "sesc_set_indicator_filter")
KERNEL_KINDS = ("indicator", "face_flux", "update", "dt")


class sesc_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("M", ctypes.c_int32), ("nel", ctypes.c_int32 * 3),
                ("xlo", ctypes.c_double * 3), ("xhi", ctypes.c_double * 3), ("bc", ctypes.c_int32 * 6),
                ("gamma", ctypes.c_double), ("tauA", ctypes.c_double), ("tauS", ctypes.c_double),
                ("alphaH", ctypes.c_double), ("alphaL", ctypes.c_double), ("betaL", ctypes.c_double),
                ("cfl", ctypes.c_double), ("node_family", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("elem_size", ctypes.c_double * 3)]


class SescError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (code {code})")


_lib = None


def load():
    """Load libsesc.so, or the library the environment variable SESC_LIBRARY names
    (the bounds-checked build); raises if it is missing: there is no CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("SESC_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.sesc_create.argtypes = [ctypes.POINTER(sesc_config), ctypes.POINTER(P)]
    lib.sesc_create.restype = I
    lib.sesc_destroy.argtypes = [P]
    lib.sesc_destroy.restype = None
    lib.sesc_num_elements.argtypes = [P]
    lib.sesc_num_elements.restype = L
    lib.sesc_num_coeffs.argtypes = [P]
    lib.sesc_num_coeffs.restype = L
    lib.sesc_indicator.argtypes = [P, P, P, P, P, P, P]
    lib.sesc_indicator.restype = I
    lib.sesc_rhs.argtypes = [P, P, P, P, P, P]
    lib.sesc_rhs.restype = I
    lib.sesc_rk_stage.argtypes = [P, P, P, P, D, D, D, P, P, P, P]
    lib.sesc_rk_stage.restype = I
    lib.sesc_dt.argtypes = [P, P, P, P]
    lib.sesc_dt.restype = I
    lib.sesc_rk3_step.argtypes = [P, P, P, P, P]
    lib.sesc_rk3_step.restype = I
    lib.sesc_rk_stage_ex.argtypes = [P, P, D, P, D, P, D, D, D, P, P, P]
    lib.sesc_rk_stage_ex.restype = I
    lib.sesc_ssprk54_step.argtypes = [P, P, P, P, P]
    lib.sesc_ssprk54_step.restype = I
    lib.sesc_status.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.sesc_status.restype = I
    lib.sesc_reset_status.argtypes = [P, P]
    lib.sesc_reset_status.restype = I
    lib.sesc_level_counts.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.sesc_level_counts.restype = I
    lib.sesc_halo_bytes.argtypes = [P, I]
    lib.sesc_halo_bytes.restype = L
    lib.sesc_pack_halo.argtypes = [P, I, P, P]
    lib.sesc_pack_halo.restype = I
    lib.sesc_set_halo.argtypes = [P, I, P]
    lib.sesc_set_halo.restype = I
    lib.sesc_stage_finish.argtypes = [P, P, P, P, D, D, D, P, I, P]
    lib.sesc_stage_finish.restype = I
    lib.sesc_rhs_vjp.argtypes = [P, P, P, P, P, P]
    lib.sesc_rhs_vjp.restype = I
    lib.sesc_rk_stage_vjp.argtypes = [P, P, P, P, D, D, D, P, P, P, P]
    lib.sesc_rk_stage_vjp.restype = I
    lib.sesc_set_timing.argtypes = [P, I]
    lib.sesc_set_timing.restype = I
    lib.sesc_kernel_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    lib.sesc_kernel_times.restype = I
    lib.sesc_rhs_static.argtypes = [ctypes.POINTER(sesc_config), P, P, P]
    lib.sesc_rhs_static.restype = I
    lib.sesc_batch_create.argtypes = [ctypes.POINTER(sesc_config), I, ctypes.POINTER(P)]
    lib.sesc_batch_create.restype = I
    lib.sesc_batch_destroy.argtypes = [P]
    lib.sesc_batch_destroy.restype = None
    lib.sesc_batch_offsets.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.sesc_batch_offsets.restype = I
    lib.sesc_batch_num_groups.argtypes = [P]
    lib.sesc_batch_num_groups.restype = I
    lib.sesc_batch_group_of.argtypes = [P, I]
    lib.sesc_batch_group_of.restype = I
    lib.sesc_batch_rhs.argtypes = [P, P, P, P]
    lib.sesc_batch_rhs.restype = I
    lib.sesc_batch_dt.argtypes = [P, P, P, P]
    lib.sesc_batch_dt.restype = I
    lib.sesc_batch_rk3_step.argtypes = [P, P, P, P, P]
    lib.sesc_batch_rk3_step.restype = I
    lib.sesc_batch_use_graph.argtypes = [P, I]
    lib.sesc_batch_use_graph.restype = I
    lib.sesc_batch_grids.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.sesc_batch_grids.restype = I
    lib.sesc_batch_set_grids.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.sesc_batch_set_grids.restype = I
    lib.sesc_batch_autotune.argtypes = [P, P, I, P]
    lib.sesc_batch_autotune.restype = I
    lib.sesc_batch_fused.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.sesc_batch_fused.restype = I
    lib.sesc_batch_set_fused.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.sesc_batch_set_fused.restype = I
    lib.sesc_batch_set_barrier_cap.argtypes = [P, L]
    lib.sesc_batch_set_barrier_cap.restype = I
    lib.sesc_batch_status.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.sesc_batch_status.restype = I
    lib.sesc_batch_reset_status.argtypes = [P, P]
    lib.sesc_batch_reset_status.restype = I
    lib.sesc_set_stage_cap.argtypes = [P, L]
    lib.sesc_set_stage_cap.restype = I
    lib.sesc_set_indicator_filter.argtypes = [P, I]
    lib.sesc_set_indicator_filter.restype = I
    lib.sesc_strerror.argtypes = [I]
    lib.sesc_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code):
    return load().sesc_strerror(int(code)).decode()


def make_config(cfg):
    """sesc_config from a dict with the fields of include/sesc.h (nel/xlo/xhi/bc
    given for the first `dim` directions; node family 'gauss' or 'lgl'; precision
    'fp64' or 'fp32_split'; scheme 'multi_level' or 'single_level')."""
    c = sesc_config()
    d = int(cfg["dim"])
    c.dim, c.M = d, int(cfg["M"])
    for a in range(3):
        c.nel[a] = int(cfg["nel"][a]) if a < d else 1
        c.xlo[a] = float(cfg["xlo"][a]) if a < d else 0.0
        c.xhi[a] = float(cfg["xhi"][a]) if a < d else 1.0
    for i in range(6):
        c.bc[i] = int(cfg["bc"][i]) if i < 2 * d else 0
    for k in ("gamma", "tauA", "tauS", "alphaH", "alphaL", "betaL", "cfl"):
        setattr(c, k, float(cfg[k]))
    fam = cfg.get("family", "gauss")
    c.node_family = NODES[fam] if isinstance(fam, str) else int(fam)
    prec = cfg.get("precision", "fp64")
    c.precision = {"fp64": 0, "fp32_split": 1}[prec] if isinstance(prec, str) else int(prec)
    sch = cfg.get("scheme", "multi_level")
    c.scheme = {"multi_level": 0, "single_level": 1}[sch] if isinstance(sch, str) else int(sch)
    es = cfg.get("elem_size")
    for a in range(3):
        c.elem_size[a] = float(es[a]) if (es is not None and a < d) else 0.0
    return c


def on_device(t, index):
    """True when tensor t lives on CUDA device `index` (the device the library's
    kernels, stream and scratch belong to for this call)."""
    dev = getattr(t, "device", None)
    return dev is not None and dev.type == "cuda" and dev.index == index


def rhs_static(cfg, u, dudt, stream=None):
    """sesc_rhs_static: dudt = R(u) without any device allocation, for callers that
    must not have the library allocate (see include/sesc.h). u, dudt: contiguous
    float64 CUDA tensors of E * (d+2) * M^d entries. Raises SescError (code
    SESC_ETOOLARGE when the problem does not fit the static scratch)."""
    import torch
    lib = load()
    c = make_config(cfg)
    n = 1
    for a in range(int(cfg["dim"])):
        n *= int(cfg["nel"][a])
    n *= (int(cfg["dim"]) + 2) * int(cfg["M"]) ** int(cfg["dim"])
    for name, t in (("u", u), ("dudt", dudt)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() == n):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor with {n} elements")
        # the entry point runs on the current device (its scratch, stream and launches)
        if not on_device(t, torch.cuda.current_device()):
            raise ValueError(f"{name} must be on the current CUDA device (cuda:{torch.cuda.current_device()})")
    rc = lib.sesc_rhs_static(ctypes.byref(c), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(dudt.data_ptr()),
                             _stream(stream))
    if rc != SESC_OK:
        raise SescError(rc, "sesc_rhs_static")


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Solver:
    """One problem on one device: a handle of the C ABI."""

    def __init__(self, cfg):
        import torch
        self.lib = load()
        self.cfg = dict(cfg)
        self.dim, self.M = int(cfg["dim"]), int(cfg["M"])
        self.nv = self.dim + 2
        self.md = self.M ** self.dim
        self.nl = self.M.bit_length()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._c = make_config(cfg)
        h = ctypes.c_void_p()
        rc = self.lib.sesc_create(ctypes.byref(self._c), ctypes.byref(h))
        if rc != SESC_OK:
            raise SescError(rc, "sesc_create")
        self.h = h
        self.E = int(self.lib.sesc_num_elements(h))
        self.S = int(self.lib.sesc_num_coeffs(h))

    # -- helpers -------------------------------------------------------------
    def _ptr(self, t, shape, dtype=None, name="tensor", allow_none=False):
        import torch
        if t is None:
            if allow_none:
                return None
            raise ValueError(f"{name} is required")
        dtype = dtype or torch.float64
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if not on_device(t, self.device.index):
            raise ValueError(f"{name} must be on the handle's device {self.device}")
        if t.dtype != dtype or not t.is_contiguous() or t.numel() != int(__import__("math").prod(shape)):
            raise ValueError(f"{name} must be a contiguous {dtype} tensor with {shape} elements")
        return ctypes.c_void_p(t.data_ptr())

    @property
    def state_shape(self):
        return (self.E, self.nv, self.md)

    def _check(self, rc, what):
        if rc != SESC_OK:
            raise SescError(rc, what)

    # -- entry points ----------------------------------------------------------
    def indicator(self, u, coeffs=None, theta=None, decision=None, abar=None, stream=None):
        import torch
        self._check(self.lib.sesc_indicator(
            self.h, self._ptr(u, self.state_shape, name="u"),
            self._ptr(coeffs, (self.E, 2, self.S), name="coeffs", allow_none=True),
            self._ptr(theta, (self.E, self.nl, self.md), name="theta", allow_none=True),
            self._ptr(decision, (self.E,), dtype=torch.uint8, name="decision", allow_none=True),
            self._ptr(abar, (self.E, self.md), name="abar", allow_none=True), _stream(stream)), "sesc_indicator")

    def rhs(self, u, dudt, frozen=None, coeffs_out=None, stream=None):
        self._check(self.lib.sesc_rhs(
            self.h, self._ptr(u, self.state_shape, name="u"), self._ptr(dudt, self.state_shape, name="dudt"),
            self._ptr(frozen, (self.E, 2, self.S), name="frozen", allow_none=True),
            self._ptr(coeffs_out, (self.E, 2, self.S), name="coeffs_out", allow_none=True), _stream(stream)),
            "sesc_rhs")

    def rk_stage(self, u0, us, uout, a, b, dt=0.0, dt_dev=None, frozen=None, coeffs_out=None, stream=None):
        self._check(self.lib.sesc_rk_stage(
            self.h, self._ptr(u0, self.state_shape, name="u0", allow_none=True),
            self._ptr(us, self.state_shape, name="us"), self._ptr(uout, self.state_shape, name="uout"),
            float(a), float(b), float(dt), self._ptr(dt_dev, (1,), name="dt_dev", allow_none=True),
            self._ptr(frozen, (self.E, 2, self.S), name="frozen", allow_none=True),
            self._ptr(coeffs_out, (self.E, 2, self.S), name="coeffs_out", allow_none=True),
            _stream(stream)), "sesc_rk_stage")

    def rhs_vjp(self, u, dudt_bar, u_bar, frozen=None, stream=None):
        self._check(self.lib.sesc_rhs_vjp(
            self.h, self._ptr(u, self.state_shape, name="u"),
            self._ptr(frozen, (self.E, 2, self.S), name="frozen", allow_none=True),
            self._ptr(dudt_bar, self.state_shape, name="dudt_bar"), self._ptr(u_bar, self.state_shape, name="u_bar"),
            _stream(stream)), "sesc_rhs_vjp")

    def rk_stage_vjp(self, us, uout_bar, us_bar, a, b, dt=0.0, dt_dev=None, frozen=None, u0_bar=None, stream=None):
        self._check(self.lib.sesc_rk_stage_vjp(
            self.h, self._ptr(us, self.state_shape, name="us"),
            self._ptr(frozen, (self.E, 2, self.S), name="frozen", allow_none=True),
            self._ptr(uout_bar, self.state_shape, name="uout_bar"), float(a), float(b), float(dt),
            self._ptr(dt_dev, (1,), name="dt_dev", allow_none=True),
            self._ptr(us_bar, self.state_shape, name="us_bar"),
            self._ptr(u0_bar, self.state_shape, name="u0_bar", allow_none=True), _stream(stream)),
            "sesc_rk_stage_vjp")

    def dt(self, u, dt_dev, stream=None):
        self._check(self.lib.sesc_dt(self.h, self._ptr(u, self.state_shape, name="u"),
                                     self._ptr(dt_dev, (1,), name="dt_dev"), _stream(stream)), "sesc_dt")

    def rk3_step(self, u, uout, dt_dev=None, stream=None):
        self._check(self.lib.sesc_rk3_step(
            self.h, self._ptr(u, self.state_shape, name="u"), self._ptr(uout, self.state_shape, name="uout"),
            self._ptr(dt_dev, (1,), name="dt_dev", allow_none=True), _stream(stream)), "sesc_rk3_step")

    def rk_stage_ex(self, us, uout, a=0.0, u0=None, c=0.0, u2=None, b=1.0, g=1.0, dt=0.0, dt_dev=None,
                    stream=None):
        """uout = a u0 + c u2 + b (us + g dt R(us))."""
        self._check(self.lib.sesc_rk_stage_ex(
            self.h, self._ptr(u0, self.state_shape, name="u0", allow_none=True), float(a),
            self._ptr(u2, self.state_shape, name="u2", allow_none=True), float(c),
            self._ptr(us, self.state_shape, name="us"), float(b), float(g), float(dt),
            self._ptr(dt_dev, (1,), name="dt_dev", allow_none=True),
            self._ptr(uout, self.state_shape, name="uout"), _stream(stream)), "sesc_rk_stage_ex")

    def ssprk54_step(self, u, uout, dt_dev=None, stream=None):
        self._check(self.lib.sesc_ssprk54_step(
            self.h, self._ptr(u, self.state_shape, name="u"), self._ptr(uout, self.state_shape, name="uout"),
            self._ptr(dt_dev, (1,), name="dt_dev", allow_none=True), _stream(stream)), "sesc_ssprk54_step")

    # -- partitioned meshes ----------------------------------------------------
    def halo_bytes(self, side):
        return int(self.lib.sesc_halo_bytes(self.h, int(side)))

    def pack_halo(self, side, dst, stream=None):
        """Pack the element-face states of side `side` into dst (a CUDA tensor of
        halo_bytes(side) bytes)."""
        self._check(self.lib.sesc_pack_halo(self.h, int(side), self._buf(dst, self.halo_bytes(side), "dst"),
                                            _stream(stream)), "sesc_pack_halo")

    def set_halo(self, side, src):
        """Use src (the neighbour's packed states of its opposite side) as the ghost
        states of halo side `side`; the tensor must stay alive while it is in use."""
        self._check(self.lib.sesc_set_halo(self.h, int(side), self._buf(src, self.halo_bytes(side), "src")),
                    "sesc_set_halo")

    def stage_finish(self, us, out, u0=None, a=0.0, b=1.0, dt=0.0, dt_dev=None, mode=1, stream=None):
        """Interface fluxes and update after indicator(us): mode 0 out = R(us), mode 1
        out = a u0 + b (us + dt R(us))."""
        self._check(self.lib.sesc_stage_finish(
            self.h, self._ptr(u0, self.state_shape, name="u0", allow_none=True),
            self._ptr(us, self.state_shape, name="us"), self._ptr(out, self.state_shape, name="out"),
            float(a), float(b), float(dt), self._ptr(dt_dev, (1,), name="dt_dev", allow_none=True), int(mode),
            _stream(stream)), "sesc_stage_finish")

    def _buf(self, t, nbytes, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
                and t.numel() * t.element_size() == nbytes):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of {nbytes} bytes")
        if not on_device(t, self.device.index):
            raise ValueError(f"{name} must be on the handle's device {self.device}")
        return ctypes.c_void_p(t.data_ptr())

    def status(self):
        """(code, counters): synchronises the device."""
        c = (ctypes.c_int64 * 16)()
        rc = self.lib.sesc_status(self.h, c)
        return rc, list(c)

    def reset_status(self, stream=None):
        self._check(self.lib.sesc_reset_status(self.h, _stream(stream)), "sesc_reset_status")

    def set_stage_cap(self, polls):
        """Bound (polls) of the wait for an element's staging copy; 0 makes the staged
        kernels give up on every element (SESC_ETIMEOUT from status)."""
        self._check(self.lib.sesc_set_stage_cap(self.h, int(polls)), "sesc_set_stage_cap")

    def set_indicator_filter(self, on):
        """Certified FP32 pass of an FP64 handle's indicator (on by default): the same
        coefficients bit for bit on or off; status()[1][12] counts the elements it
        decided."""
        self._check(self.lib.sesc_set_indicator_filter(self.h, 1 if on else 0), "sesc_set_indicator_filter")

    def level_counts(self):
        """[16] element counts per level mask (bit l: level 2^l carries weight) over the
        indicator evaluations since the last reset_status (synchronises)."""
        c = (ctypes.c_int64 * 16)()
        self._check(self.lib.sesc_level_counts(self.h, c), "sesc_level_counts")
        return list(c)

    def set_timing(self, enable):
        self._check(self.lib.sesc_set_timing(self.h, 1 if enable else 0), "sesc_set_timing")

    def kernel_times(self):
        """{kind: (total ms, launch groups)} since the last read (synchronises)."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        self._check(self.lib.sesc_kernel_times(self.h, ms, n), "sesc_kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.sesc_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BATCH_KERNEL_KINDS = ("indicator", "face_flux", "update", "dt")


class Batch:
    """Many independent problems advanced together: a batch of the C ABI.

    The states of all problems live in one contiguous float64 CUDA tensor;
    problem k occupies entries offsets[k] .. offsets[k+1]-1 in the layout of a
    single problem ([E][d+2][M^d]). view(u, k) returns that slice reshaped."""

    def __init__(self, cfgs):
        import torch
        self.lib = load()
        self.cfgs = [dict(c) for c in cfgs]
        self.n = len(self.cfgs)
        arr = (sesc_config * self.n)(*[make_config(c) for c in self.cfgs])
        self._arr = arr
        h = ctypes.c_void_p()
        rc = self.lib.sesc_batch_create(arr, self.n, ctypes.byref(h))
        if rc != SESC_OK:
            raise SescError(rc, "sesc_batch_create")
        self.h = h
        off = (ctypes.c_int64 * (self.n + 1))()
        self._check(self.lib.sesc_batch_offsets(h, off), "sesc_batch_offsets")
        self.offsets = list(off)
        self.total = self.offsets[-1]
        self.ngroups = int(self.lib.sesc_batch_num_groups(h))
        self.group_of = [int(self.lib.sesc_batch_group_of(h, k)) for k in range(self.n)]
        self.device = torch.device("cuda", torch.cuda.current_device())

    def _check(self, rc, what):
        if rc != SESC_OK:
            raise SescError(rc, what)

    def _ptr(self, t, n, name, allow_none=False):
        import torch
        if t is None:
            if allow_none:
                return None
            raise ValueError(f"{name} is required")
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() == n):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor with {n} elements")
        if not on_device(t, self.device.index):
            raise ValueError(f"{name} must be on the batch's device {self.device}")
        return ctypes.c_void_p(t.data_ptr())

    def shape(self, k):
        c = self.cfgs[k]
        d, M = int(c["dim"]), int(c["M"])
        E = 1
        for a in range(d):
            E *= int(c["nel"][a])
        return (E, d + 2, M ** d)

    def view(self, u, k):
        """Problem k's part of a concatenated state tensor, shaped [E][d+2][M^d]."""
        return u[self.offsets[k]:self.offsets[k + 1]].view(self.shape(k))

    def rhs(self, u, dudt, stream=None):
        self._check(self.lib.sesc_batch_rhs(self.h, self._ptr(u, self.total, "u"),
                                            self._ptr(dudt, self.total, "dudt"), _stream(stream)), "sesc_batch_rhs")

    def dt(self, u, dt_dev=None, stream=None):
        self._check(self.lib.sesc_batch_dt(self.h, self._ptr(u, self.total, "u"),
                                           self._ptr(dt_dev, self.n, "dt_dev", True), _stream(stream)),
                    "sesc_batch_dt")

    def rk3_step(self, u, uout, dt_dev=None, stream=None):
        self._check(self.lib.sesc_batch_rk3_step(self.h, self._ptr(u, self.total, "u"),
                                                 self._ptr(uout, self.total, "uout"),
                                                 self._ptr(dt_dev, self.n, "dt_dev", True), _stream(stream)),
                    "sesc_batch_rk3_step")

    def use_graph(self, enable=True):
        self._check(self.lib.sesc_batch_use_graph(self.h, 1 if enable else 0), "sesc_batch_use_graph")

    def grids(self):
        """[[indicator, face_flux, update, dt] grid sizes] per group."""
        g = (ctypes.c_int32 * (4 * self.ngroups))()
        self._check(self.lib.sesc_batch_grids(self.h, g), "sesc_batch_grids")
        return [list(g[4 * i:4 * i + 4]) for i in range(self.ngroups)]

    def set_grids(self, grids):
        flat = [int(x) for row in grids for x in row]
        g = (ctypes.c_int32 * len(flat))(*flat)
        self._check(self.lib.sesc_batch_set_grids(self.h, g), "sesc_batch_set_grids")

    def autotune(self, u, reps=3, stream=None):
        self._check(self.lib.sesc_batch_autotune(self.h, self._ptr(u, self.total, "u"), int(reps),
                                                 _stream(stream)), "sesc_batch_autotune")
        return self.grids()

    def fused(self):
        """Per group: the grid of its one-launch stage, 0 when it runs three launches."""
        g = (ctypes.c_int32 * self.ngroups)()
        self._check(self.lib.sesc_batch_fused(self.h, g), "sesc_batch_fused")
        return list(g)

    def set_fused(self, grids):
        g = (ctypes.c_int32 * self.ngroups)(*[int(x) for x in grids])
        self._check(self.lib.sesc_batch_set_fused(self.h, g), "sesc_batch_set_fused")

    def set_barrier_cap(self, polls):
        self._check(self.lib.sesc_batch_set_barrier_cap(self.h, int(polls)), "sesc_batch_set_barrier_cap")

    def status(self):
        """(code, [[16 counters] per problem]): synchronises the device."""
        c = (ctypes.c_int64 * (16 * self.n))()
        rc = self.lib.sesc_batch_status(self.h, c)
        return rc, [list(c[16 * k:16 * k + 16]) for k in range(self.n)]

    def reset_status(self, stream=None):
        self._check(self.lib.sesc_batch_reset_status(self.h, _stream(stream)), "sesc_batch_reset_status")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.sesc_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
