"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every step of the method runs in the CUDA kernels behind the C ABI; this module
converts Python / numpy / torch arguments into the plain pointers and sizes the
ABI takes and turns status codes into exceptions.  PyTorch is used for device
memory (output tensors) and streams.  There is no CPU fallback: if the library
is missing or a call fails, an exception is raised.
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY may point at another build of the same ABI (e.g. a tuning variant)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "liblbm.so")

EOS = {"none": 0, "cs": 1, "piecewise": 2}
STORE = {"fp32": 0, "fp16": 1}
LAYOUT = {"auto": 0, "single": 1}
BC = {"periodic": 0, "wall": 1}
RATE_NAMES = ("s0", "s1", "s2", "s2b", "s3", "s3b", "s4", "s4b", "s5", "s6")
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_UNSTABLE",
          5: "LBM_ERR_EOS_RANGE", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_STATE"}


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 3), ("eos", ctypes.c_int32), ("eos_p", ctypes.c_double * 5),
        ("G", ctypes.c_double), ("G_ads", ctypes.c_double), ("kappa", ctypes.c_double), ("sigma", ctypes.c_double),
        ("s", ctypes.c_double * 10), ("variable_nu", ctypes.c_int32),
        ("nu_l", ctypes.c_double), ("nu_v", ctypes.c_double), ("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double),
        ("g", ctypes.c_double * 3), ("psi_ext_rho", ctypes.c_double), ("zchunk", ctypes.c_int32),
        ("store", ctypes.c_int32), ("onepass", ctypes.c_int32), ("store_layout", ctypes.c_int32),
    ]


_lib = None


def lib():
    """Load liblbm.so (built in-tree by paper_2306_16274_gb300.build) and declare the ABI."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2306_16274_gb300.build` "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P, V, I32, I64, D = ctypes.c_void_p, None, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "lbm_default_params": (V, [ctypes.POINTER(lbm_params)]),
        "lbm_create": (I32, [ctypes.POINTER(lbm_params), P, ctypes.POINTER(P)]),
        "lbm_init_fields": (I32, [P, P, P, P, I32]),
        "lbm_step": (I32, [P, I32]),
        "lbm_sync": (I32, [P]),
        "lbm_get_moments": (I32, [P, P, P, P, I32]),
        "lbm_get_psi": (I32, [P, P, I32]),
        "lbm_get_populations": (I32, [P, P, I32]),
        "lbm_set_populations": (I32, [P, P, I32]),
        "lbm_set_stream": (I32, [P, P]),
        "lbm_set_kernel_timing": (I32, [P, I32]),
        "lbm_get_kernel_timing": (I32, [P, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "lbm_step_count": (I64, [P]),
        "lbm_device_bytes": (ctypes.c_size_t, [P]),
        "lbm_estimate_bytes": (I32, [ctypes.POINTER(lbm_params), I32, ctypes.POINTER(ctypes.c_size_t)]),
        "lbm_contact": (I32, [P, ctypes.c_float, P, I32]),
        "lbm_destroy": (V, [P]),
        "lbm_last_error": (ctypes.c_char_p, [P]),
        "lbm_status_string": (ctypes.c_char_p, [I32]),
        "lbm_field_totals_noalloc": (I32, [P, P, I64, P, P]),
        "lbm_batch_create": (I32, [ctypes.POINTER(P), I32, P, ctypes.POINTER(P)]),
        "lbm_batch_step": (I32, [P, I32]),
        "lbm_batch_sync": (I32, [P]),
        "lbm_batch_tune": (I32, [P, I32, ctypes.POINTER(I32), I32]),
        "lbm_batch_info": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "lbm_batch_group": (I32, [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                  ctypes.POINTER(I32)]),
        "lbm_batch_set_group": (I32, [P, I32, I32, I32]),
        "lbm_batch_destroy": (V, [P]),
        "lbm_batch_last_error": (ctypes.c_char_p, [P]),
        "lbm_debug_bounds_violations": (ctypes.c_uint64, []),
        "lbm_staged_copies": (I32, [P]),
        "lbm_debug_stage_timeout": (I32, [P, I32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


@dataclass
class Params:
    """Mirror of lbm_params.  shape = (nx, ny, nz); bc per axis "periodic" / "wall";
    eos "none" / "cs" (eos_p = a, b, R, T) / "piecewise" (rho1, rho2, theta_v, theta_m, theta_l);
    rates: s0 .. s6 of Eq. e12 (defaults from the paper, filled in by the library);
    store "fp32" or "fp16" (shifted FP16 population store); onepass: one pass per step over two
    population copies (periodic, no solids, FP32), or "staged" for the same step with each plane's
    populations staged by tensor copies (nx a multiple of 32, ny of 4); store_layout "auto" (FP16 slots of cells x and
    x + nx/2 share a word where nx is even, x periodic and no mask is given) or "single"."""
    lattice: int = 19
    shape: tuple = (32, 32, 32)
    bc: tuple = ("periodic", "periodic", "periodic")
    eos: str = "none"
    eos_p: tuple = ()
    G: float = -1.0
    G_ads: float = 0.0
    kappa: float = 0.0
    sigma: float = 0.1
    rates: dict = field(default_factory=dict)
    variable_nu: bool = False
    nu_l: float = 0.0
    nu_v: float = 0.0
    rho_l: float = 1.0
    rho_v: float = 0.0
    g: tuple = (0.0, 0.0, 0.0)
    psi_ext_rho: float = -1.0
    zchunk: int = 0
    store: str = "fp32"
    onepass: bool = False
    store_layout: str = "auto"

    def to_c(self):
        c = lbm_params()
        lib().lbm_default_params(ctypes.byref(c))
        c.lattice = int(self.lattice)
        c.nx, c.ny, c.nz = (int(v) for v in self.shape)
        for a in range(3):
            b = self.bc[a]
            c.bc[a] = BC[b] if isinstance(b, str) else int(b)
        c.eos = EOS[self.eos] if isinstance(self.eos, str) else int(self.eos)
        for k, v in enumerate(self.eos_p):
            c.eos_p[k] = float(v)
        c.G, c.G_ads, c.kappa, c.sigma = float(self.G), float(self.G_ads), float(self.kappa), float(self.sigma)
        for k, name in enumerate(RATE_NAMES):
            if name in self.rates:
                c.s[k] = float(self.rates[name])
        c.variable_nu = 1 if self.variable_nu else 0
        c.nu_l, c.nu_v, c.rho_l, c.rho_v = float(self.nu_l), float(self.nu_v), float(self.rho_l), float(self.rho_v)
        for k in range(3):
            c.g[k] = float(self.g[k])
        c.psi_ext_rho = float(self.psi_ext_rho)
        c.zchunk = int(self.zchunk)
        c.store = STORE[self.store] if isinstance(self.store, str) else int(self.store)
        c.onepass = 2 if self.onepass == "staged" else (1 if self.onepass else 0)
        c.store_layout = LAYOUT[self.store_layout] if isinstance(self.store_layout, str) else int(self.store_layout)
        return c

    @property
    def ncell(self):
        nx, ny, nz = self.shape
        return int(nx) * int(ny) * int(nz)


def field_totals_noalloc(rho, u, totals, stream=None):
    """lbm_field_totals_noalloc: FP64 (sum rho, sum rho u_x, sum rho u_y, sum rho u_z) of caller-held
    CUDA tensors rho (n floats) and u (3 n floats) into the caller's CUDA tensor `totals` (4 doubles),
    enqueued on `stream`.  For callers that cannot allocate device memory while they run (a
    pre-budgeted pool allocator, a real-time loop that may not block on cudaMalloc): the library uses
    a fixed scratch array instead of cudaMalloc, so n is limited to LBM_NOALLOC_MAX_CELLS = 33554432
    and calls that overlap on one GPU race.  The first call on a device sets up the scratch address;
    make it before any stream capture.  All three tensors must be contiguous and on the current CUDA
    device, rho and u float32, totals float64 (ValueError otherwise; nothing is converted or copied,
    since a copy would allocate)."""
    torch = _torch()
    for name, t, dt in (("rho", rho, torch.float32), ("u", u, torch.float32), ("totals", totals, torch.float64)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device (cuda:{torch.cuda.current_device()}), "
                             f"got {t.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    L = lib()
    n = int(rho.numel())
    if int(u.numel()) != 3 * n or int(totals.numel()) != 4:
        raise ValueError("u must hold 3 n floats and totals 4 doubles")
    st = L.lbm_field_totals_noalloc(rho.data_ptr(), u.data_ptr(), n, totals.data_ptr(),
                                    ctypes.c_void_p(_stream_handle(stream)))
    if st != 0:
        raise LBMError(st, L.lbm_last_error(None).decode())


def estimate_bytes(params, with_solid=False):
    """lbm_estimate_bytes: device bytes a Simulation of `params` holds once initialised from device
    memory (with a solid mask if with_solid), computed without allocating."""
    L = lib()
    c = params.to_c()
    out = ctypes.c_size_t()
    st = L.lbm_estimate_bytes(ctypes.byref(c), 1 if with_solid else 0, ctypes.byref(out))
    if st != 0:
        raise LBMError(st, L.lbm_last_error(None).decode())
    return int(out.value)


CONTACT_FIELDS = ("wet", "floor", "xmin", "xmax", "ymin", "ymax")


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    if stream is None:
        torch = _torch()
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a, n, dtype, name):
    """(pointer, on_device, keepalive) for a torch tensor or array-like holding n elements."""
    if a is None:
        return None, None, None
    mod = type(a).__module__
    if mod.startswith("torch"):
        torch = _torch()
        t = a.detach().contiguous()
        want = {np.float32: torch.float32, np.uint8: torch.uint8}[dtype]
        if t.dtype != want:
            t = t.to(want)
        if t.numel() != n:
            raise ValueError(f"{name}: expected {n} elements, got {t.numel()}")
        return t.data_ptr(), bool(t.is_cuda), t
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.size != n:
        raise ValueError(f"{name}: expected {n} elements, got {arr.size}")
    return arr.ctypes.data, False, arr


class Simulation:
    """One lattice-Boltzmann domain on the current CUDA device (wraps an lbm_ctx)."""

    def __init__(self, params: Params, stream=None):
        self.params = params
        self._L = lib()
        self._c = params.to_c()
        self.Q = int(params.lattice)
        self.n = params.ncell
        self.stream = _stream_handle(stream)
        ctx = ctypes.c_void_p()
        st = self._L.lbm_create(ctypes.byref(self._c), ctypes.c_void_p(self.stream), ctypes.byref(ctx))
        if st != 0:
            raise LBMError(st, self._L.lbm_last_error(None).decode())
        self._ctx = ctx

    # ---------------------------------------------------------------- helpers
    def _check(self, st):
        if st != 0:
            raise LBMError(st, self._L.lbm_last_error(self._ctx).decode())

    def _same_side(self, flags):
        flags = [f for f in flags if f is not None]
        if flags and any(f != flags[0] for f in flags):
            raise ValueError("all arrays of one call must be on the device or all on the host")
        return int(flags[0]) if flags else 1

    # ---------------------------------------------------------------- ABI calls
    def init_fields(self, rho, u, solid=None):
        pr, dr, kr = _ptr(rho, self.n, np.float32, "rho")
        pu, du, ku = _ptr(u, 3 * self.n, np.float32, "u")
        ps, ds, ks = _ptr(solid, self.n, np.uint8, "solid")
        on_dev = self._same_side([dr, du, ds])
        self._check(self._L.lbm_init_fields(self._ctx, pr, pu, ps, on_dev))
        return self

    def step(self, n=1):
        self._check(self._L.lbm_step(self._ctx, int(n)))
        return self

    def sync(self):
        self._check(self._L.lbm_sync(self._ctx))

    def moments(self, device=True, sums=True):
        """(rho, u, sums): rho (nz, ny, nx), u (3, nz, ny, nx) as torch CUDA tensors (device=True)
        or numpy arrays; sums = FP64 (sum rho, sum rho u_x, sum rho u_y, sum rho u_z) over fluid cells."""
        nx, ny, nz = self.params.shape
        s = (ctypes.c_double * 4)()
        if device:
            torch = _torch()
            rho = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
            u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
            self._check(self._L.lbm_get_moments(self._ctx, rho.data_ptr(), u.data_ptr(), s if sums else None, 1))
        else:
            rho = np.empty((nz, ny, nx), dtype=np.float32)
            u = np.empty((3, nz, ny, nx), dtype=np.float32)
            self._check(self._L.lbm_get_moments(self._ctx, rho.ctypes.data, u.ctypes.data, s if sums else None, 0))
        return rho, u, (np.array(list(s)) if sums else None)

    def moments_into(self, rho, u, sums=None):
        """Fill caller-owned buffers (torch CUDA tensors or host arrays); sums: ctypes double[4] or None."""
        pr, dr, kr = _ptr(rho, self.n, np.float32, "rho") if rho is not None else (None, None, None)
        pu, du, ku = _ptr(u, 3 * self.n, np.float32, "u") if u is not None else (None, None, None)
        on_dev = self._same_side([dr, du])
        self._check(self._L.lbm_get_moments(self._ctx, pr, pu, sums, on_dev))

    def psi(self, device=True):
        nx, ny, nz = self.params.shape
        if device:
            torch = _torch()
            out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
            self._check(self._L.lbm_get_psi(self._ctx, out.data_ptr(), 1))
        else:
            out = np.empty((nz, ny, nx), dtype=np.float32)
            self._check(self._L.lbm_get_psi(self._ctx, out.ctypes.data, 0))
        return out

    def populations(self, device=True):
        nx, ny, nz = self.params.shape
        if device:
            torch = _torch()
            out = torch.empty((self.Q, nz, ny, nx), dtype=torch.float32, device="cuda")
            self._check(self._L.lbm_get_populations(self._ctx, out.data_ptr(), 1))
        else:
            out = np.empty((self.Q, nz, ny, nx), dtype=np.float32)
            self._check(self._L.lbm_get_populations(self._ctx, out.ctypes.data, 0))
        return out

    def contact(self, rho_threshold, out=None):
        """lbm_contact: liquid cells (rho > rho_threshold) touching solids and the liquid footprint on a
        bottom wall.  With out=None the call synchronises and returns a dict over CONTACT_FIELDS; with
        `out` an int32 CUDA tensor of 6 elements (e.g. a row of a larger buffer) it only enqueues."""
        if out is None:
            h = (ctypes.c_int32 * 6)()
            self._check(self._L.lbm_contact(self._ctx, float(rho_threshold), h, 0))
            return dict(zip(CONTACT_FIELDS, list(h)))
        torch = _torch()
        if out.dtype != torch.int32 or out.numel() != 6 or not out.is_cuda or not out.is_contiguous():
            raise ValueError("out must be a contiguous int32 CUDA tensor of 6 elements")
        self._check(self._L.lbm_contact(self._ctx, float(rho_threshold), out.data_ptr(), 1))
        return out

    def set_populations(self, f):
        p, d, k = _ptr(f, self.Q * self.n, np.float32, "f")
        self._check(self._L.lbm_set_populations(self._ctx, p, int(d)))

    def set_stream(self, stream):
        self.stream = _stream_handle(stream)
        self._check(self._L.lbm_set_stream(self._ctx, ctypes.c_void_p(self.stream)))

    def set_kernel_timing(self, enable=True):
        self._check(self._L.lbm_set_kernel_timing(self._ctx, 1 if enable else 0))

    def kernel_timing(self):
        """({'psi': ms, 'collide': ms}, {'psi': launches, 'collide': launches}) since timing was enabled."""
        ms = (ctypes.c_double * 2)()
        n = (ctypes.c_int64 * 2)()
        self._check(self._L.lbm_get_kernel_timing(self._ctx, ms, n))
        return {"psi": ms[0], "collide": ms[1]}, {"psi": n[0], "collide": n[1]}

    @property
    def staged(self):
        """True when the one-pass step stages populations with tensor copies (lbm_staged_copies)."""
        return bool(self._L.lbm_staged_copies(self._ctx))

    def debug_stage_timeout(self, enable=True):
        """lbm_debug_stage_timeout: make the staged step's waits run out (to test the timeout path)."""
        self._check(self._L.lbm_debug_stage_timeout(self._ctx, 1 if enable else 0))

    @property
    def step_count(self):
        return int(self._L.lbm_step_count(self._ctx))

    @property
    def device_bytes(self):
        return int(self._L.lbm_device_bytes(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.lbm_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many Simulations advanced together (lbm_batch_*): one launch per kernel and group per step,
    runs of steps replayed from one CUDA graph.  The Simulations stay owned by the caller and must
    outlive the Batch."""

    def __init__(self, sims, stream=None):
        self._L = lib()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s._ctx.value for s in self.sims])
        out = ctypes.c_void_p()
        self.stream = _stream_handle(stream)
        st = self._L.lbm_batch_create(arr, len(self.sims), ctypes.c_void_p(self.stream), ctypes.byref(out))
        if st != 0:
            raise LBMError(st, self._L.lbm_last_error(None).decode())
        self._b = out

    def _check(self, st):
        if st != 0:
            raise LBMError(st, self._L.lbm_batch_last_error(self._b).decode())

    def step(self, n=1):
        self._check(self._L.lbm_batch_step(self._b, int(n)))
        return self

    def sync(self):
        self._check(self._L.lbm_batch_sync(self._b))

    def tune(self, trial_steps=3):
        """Pick the tile shape and then the z-chunk per group by timing; returns the z-chunks
        (0 = automatic); groups() gives the shapes."""
        g = ctypes.c_int32()
        self._check(self._L.lbm_batch_info(self._b, ctypes.byref(g), None, None))
        out = (ctypes.c_int32 * max(g.value, 1))()
        self._check(self._L.lbm_batch_tune(self._b, int(trial_steps), out, g.value))
        return list(out)[:g.value]

    def groups(self):
        """[{lattice, solids, shape, zchunk}] per group (shape: index of LBM_BATCH_SHAPES)."""
        n = self.info()["groups"]
        out = []
        for k in range(n):
            v = [ctypes.c_int32() for _ in range(4)]
            self._check(self._L.lbm_batch_group(self._b, k, *[ctypes.byref(x) for x in v]))
            out.append(dict(zip(("lattice", "solids", "shape", "zchunk"), [x.value for x in v])))
        return out

    def set_group(self, group, shape, zchunk=0):
        self._check(self._L.lbm_batch_set_group(self._b, int(group), int(shape), int(zchunk)))

    def info(self):
        g, t, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self._L.lbm_batch_info(self._b, ctypes.byref(g), ctypes.byref(t), ctypes.byref(m)))
        return {"groups": g.value, "tiles": t.value, "graph_mode": m.value}

    def close(self):
        if getattr(self, "_b", None):
            self._L.lbm_batch_destroy(self._b)
            self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
