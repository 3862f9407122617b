"""Python binding of libssht (see include/ssht.h).  Argument marshalling only: every step of
every transform runs in the CUDA library; there is no CPU path.  If the library is missing
the first call raises.

Low-level functions carry the C names (``ssht_plan``, ``ssht_inverse``, ...) and take raw
pointers; ``Plan`` wraps them for torch tensors (device memory and streams come from torch).
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# SSHT_LIBRARY names another build of the library (the bounds-checked lib/libssht_debug.so)
LIB_PATH = os.environ.get("SSHT_LIBRARY") or os.path.join(HERE, "lib", "libssht.so")

FP64, FP32, TF32X3, BF16X6 = 0, 1, 2, 3
FLAG_REAL = 1
FLAG_RISBO = 2
FLAG_TUNE = 4
FLAG_SPIN_PAIR = 8
RECOMPUTE, CACHE = 0, 1
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32x3": TF32X3, "bf16x6": BF16X6}
ERRORS = {0: "SSHT_OK", -1: "SSHT_EINVAL", -2: "SSHT_ENOMEM", -3: "SSHT_ECUDA", -4: "SSHT_ETIMEOUT",
          -5: "SSHT_EUNSUPPORTED"}
EXPORTS = ("ssht_plan", "ssht_plan_ex", "ssht_plan_destroy", "ssht_plan_workspace_bytes", "ssht_inverse",
           "ssht_forward", "ssht_adjoint", "ssht_forward_triangular", "ssht_wigner_delta", "ssht_plan_check", "ssht_plan_profile",
           "ssht_plan_profile_read", "ssht_plan_profile_trace", "ssht_wigner_delta_noalloc", "ssht_group_create", "ssht_group_destroy",
           "ssht_group_layout", "ssht_group_buckets", "ssht_group_inverse", "ssht_group_forward",
           "ssht_group_adjoint", "ssht_group_capture", "ssht_group_replay", "ssht_group_check",
           "ssht_debug_fail_allocation", "ssht_plan_set_wait_limit", "ssht_plan_tile_config",
           "ssht_group_bucket_tile_config", "ssht_debug_bounds", "ssht_debug_noalloc_wait_limit", "ssht_last_error",
           "ssht_version")
STAGES = ("delta", "inverse", "project", "fft", "torus", "pack", "delta_inverse")


class SshtError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s (%s): %s" % (what, ERRORS.get(code, code), _lib().ssht_last_error().decode()))
        self.code = code


class PlanDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("s", ctypes.c_int), ("batch", ctypes.c_int), ("precision", ctypes.c_int),
                ("delta_mode", ctypes.c_int), ("flags", ctypes.c_int)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libssht.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i = ctypes.c_void_p, ctypes.c_int
        sig = {
            "ssht_plan": ([ctypes.POINTER(vp), i, i, i], i),
            "ssht_plan_ex": ([ctypes.POINTER(vp), ctypes.POINTER(PlanDesc)], i),
            "ssht_plan_destroy": ([vp], i),
            "ssht_plan_workspace_bytes": ([vp, ctypes.POINTER(ctypes.c_size_t)], i),
            "ssht_inverse": ([vp, vp, vp, vp], i),
            "ssht_forward": ([vp, vp, vp, vp], i),
            "ssht_adjoint": ([vp, vp, vp, vp], i),
            "ssht_forward_triangular": ([vp, vp, vp, vp], i),
            "ssht_wigner_delta": ([vp, vp, vp], i),
            "ssht_plan_check": ([vp], i),
            "ssht_plan_profile": ([vp, i], i),
            "ssht_plan_profile_read": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong), i,
                                        ctypes.POINTER(ctypes.c_longlong)], i),
            "ssht_plan_profile_trace": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), i, ctypes.POINTER(i)], i),
            "ssht_wigner_delta_noalloc": ([i, vp, vp], i),
            "ssht_group_create": ([ctypes.POINTER(vp), i, ctypes.POINTER(i), ctypes.POINTER(i), i, i, i], i),
            "ssht_group_destroy": ([vp], i),
            "ssht_group_layout": ([vp, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)], i),
            "ssht_group_buckets": ([vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                    ctypes.POINTER(i)], i),
            "ssht_group_inverse": ([vp, vp, vp, vp], i),
            "ssht_group_forward": ([vp, vp, vp, vp], i),
            "ssht_group_adjoint": ([vp, vp, vp, vp], i),
            "ssht_group_capture": ([vp, vp, vp, vp, vp], i),
            "ssht_group_replay": ([vp, vp], i),
            "ssht_group_check": ([vp], i),
            "ssht_debug_fail_allocation": ([i], i),
            "ssht_debug_noalloc_wait_limit": ([ctypes.c_longlong], i),
            "ssht_plan_set_wait_limit": ([vp, ctypes.c_longlong], i),
            "ssht_plan_tile_config": ([vp, ctypes.POINTER(i)], i),
            "ssht_group_bucket_tile_config": ([vp, i, ctypes.POINTER(i)], i),
            "ssht_debug_bounds": ([ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)], i),
            "ssht_last_error": ([], ctypes.c_char_p),
            "ssht_version": ([], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


def _check(rc, what):
    if rc != 0:
        raise SshtError(rc, what)


# ---- C-named wrappers (raw pointers as ints) -------------------------------------------------

def ssht_plan(L, s, batch):
    h = ctypes.c_void_p()
    _check(_lib().ssht_plan(ctypes.byref(h), L, s, batch), "ssht_plan")
    return h


def ssht_plan_ex(L, s, batch, precision=FP64, delta_mode=RECOMPUTE, flags=0):
    h = ctypes.c_void_p()
    d = PlanDesc(L, s, batch, precision, delta_mode, flags)
    _check(_lib().ssht_plan_ex(ctypes.byref(h), ctypes.byref(d)), "ssht_plan_ex")
    return h


def ssht_plan_destroy(h):
    return _lib().ssht_plan_destroy(h)


def ssht_inverse(h, flm_ptr, f_ptr, stream=0):
    _check(_lib().ssht_inverse(h, flm_ptr, f_ptr, stream), "ssht_inverse")


def ssht_forward(h, f_ptr, flm_ptr, stream=0):
    _check(_lib().ssht_forward(h, f_ptr, flm_ptr, stream), "ssht_forward")


def ssht_adjoint(h, g_ptr, flm_ptr, stream=0):
    _check(_lib().ssht_adjoint(h, g_ptr, flm_ptr, stream), "ssht_adjoint")


def ssht_forward_triangular(h, f_ptr, flm_ptr, stream=0):
    _check(_lib().ssht_forward_triangular(h, f_ptr, flm_ptr, stream), "ssht_forward_triangular")


def ssht_wigner_delta(h, out_ptr, stream=0):
    _check(_lib().ssht_wigner_delta(h, out_ptr, stream), "ssht_wigner_delta")


def ssht_wigner_delta_noalloc(L, out_ptr, stream=0):
    """Delta table for L <= 512 without any device allocation (fixed scratch inside the library)."""
    rc = _lib().ssht_wigner_delta_noalloc(int(L), out_ptr, stream)
    if rc != 0:
        raise SshtError(rc, "ssht_wigner_delta_noalloc")


def ssht_plan_check(h):
    _check(_lib().ssht_plan_check(h), "ssht_plan_check")


def ssht_debug_fail_allocation(n):
    """Test hook: the n-th device allocation of the library from now on fails (0 disables)."""
    _check(_lib().ssht_debug_fail_allocation(int(n)), "ssht_debug_fail_allocation")


def ssht_debug_noalloc_wait_limit(ns):
    """Test hook: the spin limit of ssht_wigner_delta_noalloc's waits (0 restores the default)."""
    _check(_lib().ssht_debug_noalloc_wait_limit(int(ns)), "ssht_debug_noalloc_wait_limit")


def ssht_debug_bounds():
    """Index checks of the bounds-checked build: (count, site, index, extent) of the kernel
    accesses found outside their buffers since the last call; raises in release builds."""
    c, k, x, e = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib().ssht_debug_bounds(ctypes.byref(c), ctypes.byref(k), ctypes.byref(x), ctypes.byref(e)),
           "ssht_debug_bounds")
    return c.value, k.value, x.value, e.value


def ssht_plan_set_wait_limit(h, ns):
    _check(_lib().ssht_plan_set_wait_limit(h, int(ns)), "ssht_plan_set_wait_limit")


def ssht_plan_tile_config(h):
    cfg = (ctypes.c_int * 4)()
    _check(_lib().ssht_plan_tile_config(h, cfg), "ssht_plan_tile_config")
    return {"slice": cfg[0], "stages": cfg[1], "inv_order": cfg[2], "fwd_order": cfg[3]}


def ssht_group_bucket_tile_config(h, bucket):
    cfg = (ctypes.c_int * 4)()
    _check(_lib().ssht_group_bucket_tile_config(h, int(bucket), cfg), "ssht_group_bucket_tile_config")
    return {"slice": cfg[0], "stages": cfg[1], "inv_order": cfg[2], "fwd_order": cfg[3]}


def ssht_plan_profile(h, enable):
    _check(_lib().ssht_plan_profile(h, int(bool(enable))), "ssht_plan_profile")


def ssht_plan_profile_read(h):
    """Returns ({stage: (ms, count)}, launches) since profiling was enabled."""
    n = len(STAGES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    launches = ctypes.c_longlong()
    _check(_lib().ssht_plan_profile_read(h, ms, cnt, n, ctypes.byref(launches)), "ssht_plan_profile_read")
    return {name: (ms[k], cnt[k]) for k, name in enumerate(STAGES)}, launches.value


def ssht_plan_profile_trace(h, cap=8192):
    """Returns the stage brackets since profiling was enabled or last read, in recording order:
    a list of (stage name, lane, start ms, end ms), lane 0 the caller's stream and 1 the plan's
    second stream, times after the earliest bracket's start."""
    stage = (ctypes.c_int * cap)()
    lane = (ctypes.c_int * cap)()
    t0 = (ctypes.c_double * cap)()
    t1 = (ctypes.c_double * cap)()
    n = ctypes.c_int()
    _check(_lib().ssht_plan_profile_trace(h, stage, lane, t0, t1, cap, ctypes.byref(n)), "ssht_plan_profile_trace")
    return [(STAGES[stage[k]], lane[k], t0[k], t1[k]) for k in range(n.value)]


def ssht_plan_workspace_bytes(h):
    n = ctypes.c_size_t()
    _check(_lib().ssht_plan_workspace_bytes(h, ctypes.byref(n)), "ssht_plan_workspace_bytes")
    return n.value


def ssht_last_error():
    return _lib().ssht_last_error().decode()


def ssht_version():
    return _lib().ssht_version()


# ---- torch-facing plan --------------------------------------------------------------------

class Plan:
    """A transform plan for ``batch`` fields of band-limit ``L`` (exclusive) and spin ``s``.

    Tensors: coefficients ``[batch, L*L]``, samples ``[batch, L, 2L-1]`` (complex128 for
    precision ``fp64``, complex64 otherwise), on the plan's CUDA device or on the host.
    ``real=True`` (spin 0): real fields, samples real (float64 / float32), coefficients complex
    with sf_{l,-m} = (-1)^m conj(sf_lm).  ``recursion="risbo"`` makes Delta with the Risbo
    recursion the paper uses instead of the default three-term relation in m'.
    """

    def __init__(self, L, s, batch=1, precision="fp64", delta_mode="recompute", real=False, recursion="column",
                 tune=False, spin_pair=False):
        self.L, self.s, self.batch = int(L), int(s), int(batch)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.delta_mode = {"recompute": RECOMPUTE, "cache": CACHE}[delta_mode] if isinstance(delta_mode, str) else int(delta_mode)
        self.real = bool(real)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.complex128 if self.precision == FP64 else torch.complex64
        self.grid_dtype = (torch.float64 if self.precision == FP64 else torch.float32) if self.real else self.dtype
        if recursion not in ("column", "risbo"):
            raise ValueError("recursion must be 'column' or 'risbo'")
        self.spin_pair = bool(spin_pair)
        flags = (FLAG_REAL if self.real else 0) | (FLAG_RISBO if recursion == "risbo" else 0) | (FLAG_TUNE if tune else 0)
        flags |= FLAG_SPIN_PAIR if self.spin_pair else 0
        self._h = ssht_plan_ex(self.L, self.s, self.batch, self.precision, self.delta_mode, flags)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            ssht_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def N(self):
        return 2 * self.L - 1

    def coeff_shape(self):
        return (self.batch, 2, self.L * self.L) if self.spin_pair else (self.batch, self.L * self.L)

    def grid_shape(self):
        return (self.batch, self.L, self.N)

    def _arg(self, t, shape, name, dtype=None):
        dtype = self.dtype if dtype is None else dtype
        if t.dtype != dtype:
            raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
        if tuple(t.shape) != shape and not (self.batch == 1 and tuple(t.shape) == shape[1:]):
            raise ValueError("%s must have shape %s, got %s" % (name, shape, tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.is_cuda and t.device != self.device:
            raise ValueError("%s is on %s, the plan on %s" % (name, t.device, self.device))
        return t.data_ptr()

    def _out(self, out, ref, ref_shape, shape, dtype=None):
        if out is None:
            batched = ref.dim() == len(ref_shape)
            out = torch.empty(shape if batched else shape[1:], dtype=self.dtype if dtype is None else dtype,
                              device=ref.device)
        return out

    @staticmethod
    def _stream(stream, t):
        # the calling thread's current CUDA stream, whether the data is on the device or on the
        # host: a plan owns one workspace, so all its calls must go to one stream in order
        if stream is not None:
            return int(stream)
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0

    def inverse(self, flm, out=None, stream=None):
        out = self._out(out, flm, self.coeff_shape(), self.grid_shape(), self.grid_dtype)
        ssht_inverse(self._h, self._arg(flm, self.coeff_shape(), "flm"),
                     self._arg(out, self.grid_shape(), "f", self.grid_dtype), self._stream(stream, flm))
        return out

    def forward(self, f, out=None, stream=None):
        out = self._out(out, f, self.grid_shape(), self.coeff_shape())
        ssht_forward(self._h, self._arg(f, self.grid_shape(), "f", self.grid_dtype),
                     self._arg(out, self.coeff_shape(), "flm"), self._stream(stream, f))
        return out

    def adjoint(self, g, out=None, stream=None):
        out = self._out(out, g, self.grid_shape(), self.coeff_shape())
        ssht_adjoint(self._h, self._arg(g, self.grid_shape(), "g", self.grid_dtype),
                     self._arg(out, self.coeff_shape(), "flm"), self._stream(stream, g))
        return out

    def forward_triangular(self, f, out=None, stream=None):
        """The paper's triangular forward (FP64 plans; unstable at high band-limit)."""
        out = self._out(out, f, self.grid_shape(), self.coeff_shape())
        ssht_forward_triangular(self._h, self._arg(f, self.grid_shape(), "f", self.grid_dtype),
                                self._arg(out, self.coeff_shape(), "flm"), self._stream(stream, f))
        return out

    def wigner_delta(self, out=None, stream=None):
        n = self.L * (self.L + 1) * (2 * self.L + 1) // 6
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=self.device)
        if out.dtype != torch.float64 or out.numel() != n or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of %d elements" % n)
        ssht_wigner_delta(self._h, out.data_ptr(), self._stream(stream, out))
        return out

    def check(self):
        ssht_plan_check(self._h)

    def tile_config(self):
        """Shape of the tensor-core contraction (fields per launch, stages, work orders)."""
        return ssht_plan_tile_config(self._h)

    def set_wait_limit(self, ns):
        """Spin limit of the plan's device-side waits in nanoseconds (<= 0: the default, 1 s)."""
        ssht_plan_set_wait_limit(self._h, ns)

    def workspace_bytes(self):
        return ssht_plan_workspace_bytes(self._h)

    def profile(self, enable=True):
        ssht_plan_profile(self._h, enable)

    def profile_read(self):
        return ssht_plan_profile_read(self._h)

    def profile_trace(self):
        return ssht_plan_profile_trace(self._h)


class InverseFunction(torch.autograd.Function):
    """Differentiable inverse transform; the backward pass is ssht_adjoint (A^H of the linear map),
    which recomputes Delta^l instead of storing anything from the forward pass."""

    @staticmethod
    def forward(ctx, flm, plan):
        ctx.plan = plan
        return plan.inverse(flm.contiguous())

    @staticmethod
    def backward(ctx, grad_f):
        return ctx.plan.adjoint(grad_f.contiguous()), None


def inverse(flm, plan):
    """Inverse transform with autograd support."""
    return InverseFunction.apply(flm, plan)


# ---- groups of uneven fields ------------------------------------------------------------------

def ssht_group_create(Ls, ss, precision=FP32, delta_mode=RECOMPUTE, tune=True):
    n = len(Ls)
    h = ctypes.c_void_p()
    La = (ctypes.c_int * n)(*[int(x) for x in Ls])
    sa = (ctypes.c_int * n)(*[int(x) for x in ss])
    _check(_lib().ssht_group_create(ctypes.byref(h), n, La, sa, int(precision), int(delta_mode), int(bool(tune))),
           "ssht_group_create")
    return h


def ssht_group_layout(h, n):
    order = (ctypes.c_int * n)()
    co = (ctypes.c_longlong * (n + 1))()
    go = (ctypes.c_longlong * (n + 1))()
    _check(_lib().ssht_group_layout(h, order, co, go), "ssht_group_layout")
    return list(order), list(co), list(go)


def ssht_group_buckets(h):
    cap = ctypes.c_int(0)
    _check(_lib().ssht_group_buckets(h, ctypes.byref(cap), None, None, None, None), "ssht_group_buckets")
    nb = cap.value
    arr = [(ctypes.c_int * nb)() for _ in range(4)]
    cap = ctypes.c_int(nb)
    _check(_lib().ssht_group_buckets(h, ctypes.byref(cap), *arr), "ssht_group_buckets")
    return [(arr[0][k], arr[1][k], arr[2][k], arr[3][k]) for k in range(nb)]


class Group:
    """Fields of uneven band-limit L_i and spin s_i transformed together (buckets by (L, s), one
    shared Delta table per L, buckets on concurrent streams, optional autotuned contraction per
    bucket, and inverse + forward capturable into one CUDA graph).

    Data travels in flat complex tensors in the group's order: ``pack_coeffs`` / ``unpack_*``
    convert from and to per-field lists (on the device, by slicing)."""

    def __init__(self, Ls, ss, precision="fp32", delta_mode="recompute", tune=True):
        self.Ls, self.ss = [int(x) for x in Ls], [int(x) for x in ss]
        self.n = len(self.Ls)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        dm = {"recompute": RECOMPUTE, "cache": CACHE}[delta_mode] if isinstance(delta_mode, str) else int(delta_mode)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.complex128 if self.precision == FP64 else torch.complex64
        self._h = ssht_group_create(self.Ls, self.ss, self.precision, dm, tune)
        self.order, self.coff, self.goff = ssht_group_layout(self._h, self.n)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().ssht_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def buckets(self):
        """[(L, s, fields, precision)] per bucket, precision after tuning."""
        return ssht_group_buckets(self._h)

    def bucket_tile_config(self, i):
        """Tensor-core shape of bucket i (SshtError for a bucket on CUDA cores)."""
        return ssht_group_bucket_tile_config(self._h, i)

    def empty_coeffs(self):
        return torch.empty(self.coff[-1], dtype=self.dtype, device=self.device)

    def empty_grid(self):
        return torch.empty(self.goff[-1], dtype=self.dtype, device=self.device)

    def pack_coeffs(self, flms, out=None):
        """Per-field coefficient tensors [L_i^2] (caller's order) -> one flat tensor (group order)."""
        out = self.empty_coeffs() if out is None else out
        for k, i in enumerate(self.order):
            out[self.coff[k]:self.coff[k + 1]].copy_(flms[i].reshape(-1))
        return out

    def unpack_coeffs(self, flat):
        res = [None] * self.n
        for k, i in enumerate(self.order):
            res[i] = flat[self.coff[k]:self.coff[k + 1]]
        return res

    def unpack_grid(self, flat):
        res = [None] * self.n
        for k, i in enumerate(self.order):
            L = self.Ls[i]
            res[i] = flat[self.goff[k]:self.goff[k + 1]].view(L, 2 * L - 1)
        return res

    def _stream(self):
        return torch.cuda.current_stream().cuda_stream

    def inverse(self, flm_flat, out=None):
        out = self.empty_grid() if out is None else out
        _check(_lib().ssht_group_inverse(self._h, flm_flat.data_ptr(), out.data_ptr(), self._stream()), "ssht_group_inverse")
        return out

    def forward(self, f_flat, out=None):
        out = self.empty_coeffs() if out is None else out
        _check(_lib().ssht_group_forward(self._h, f_flat.data_ptr(), out.data_ptr(), self._stream()), "ssht_group_forward")
        return out

    def adjoint(self, f_flat, out=None):
        out = self.empty_coeffs() if out is None else out
        _check(_lib().ssht_group_adjoint(self._h, f_flat.data_ptr(), out.data_ptr(), self._stream()), "ssht_group_adjoint")
        return out

    def capture(self, flm_flat, f_flat, flm_out_flat):
        """Capture inverse (flm -> f) then forward (f -> flm_out) into one CUDA graph."""
        _check(_lib().ssht_group_capture(self._h, flm_flat.data_ptr(), f_flat.data_ptr(), flm_out_flat.data_ptr(),
                                         self._stream()), "ssht_group_capture")

    def replay(self):
        _check(_lib().ssht_group_replay(self._h, self._stream()), "ssht_group_replay")

    def check(self):
        _check(_lib().ssht_group_check(self._h), "ssht_group_check")
