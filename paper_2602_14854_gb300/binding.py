"""Thin ctypes binding of libddlra.so (the C ABI declared in include/ddlra.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The library is loaded from the package's ``lib/`` folder; when it is missing
the binding raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libddlra.so")

DD_OK = 0
STATUS_NAMES = {0: "DD_OK", 1: "DD_ERR_ARG", 2: "DD_ERR_CUDA", 3: "DD_ERR_RANK_CAP",
                4: "DD_ERR_NONFINITE", 5: "DD_ERR_COMPLETION", 6: "DD_ERR_STATE",
                7: "DD_ERR_TIMEOUT"}
DD_RANK_FIXED, DD_RANK_TOL = 0, 1
DD_EULER, DD_RK4 = 0, 1
DD_FP64, DD_MIXED, DD_TF32, DD_BF16 = 0, 1, 2, 3
PRECISIONS = {"fp64": DD_FP64, "mixed": DD_MIXED, "tf32": DD_TF32, "bf16": DD_BF16}
PRODUCTS = {"fp64": 0, "tensor": 1, "auto": 2}

# every symbol include/ddlra.h declares
EXPORTS = ["dd_dlra_create", "dd_dlra_step", "dd_dlra_set_graph", "dd_dlra_scalar_flux",
           "dd_dlra_ranks", "dd_dlra_info", "dd_dlra_get_factors", "dd_dlra_set_factors",
           "dd_dlra_sync", "dd_dlra_destroy", "dd_last_error", "dd_profile_slots",
           "dd_profile_slot_name", "dd_dlra_profile", "dd_dlra_profile_work",
           "dd_dlra_scalar_flux_noalloc", "dd_dlra_tuning",
           "dd_dlra_create_batch", "dd_dlra_instance", "dd_selftest_wait",
           "dd_dlra_last_error", "dd_set_allocator", "dd_dlra_scalar_flux_instance"]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double)]


class Tiling(C.Structure):
    _fields_ = [("tx", C.c_int), ("ty", C.c_int), ("xcuts", _ip), ("ycuts", _ip)]


class Quadrature(C.Structure):
    _fields_ = [("n", C.c_int), ("omega_x", _dp), ("omega_y", _dp), ("w", _dp),
                ("n_polar", C.c_int), ("n_azimuth", C.c_int)]


class Fields(C.Structure):
    _fields_ = [("sigma_s", _dp), ("sigma_a", _dp), ("source", _dp),
                ("inflow_g", _dp * 4), ("inflow_h", _dp * 4)]


INFLOW_SIDES = ("x_lo", "x_hi", "y_lo", "y_hi")


class Options(C.Structure):
    _fields_ = [("rank_mode", C.c_int), ("rank", C.c_int), ("tol", C.c_double),
                ("r_min", C.c_int), ("r_max", C.c_int), ("r_aug_max", C.c_int),
                ("integrator", C.c_int), ("c_adv", C.c_double), ("dt", C.c_double),
                ("tau", C.c_double), ("precision", C.c_int), ("mass_fix", C.c_int),
                ("splitting", C.c_int), ("kstep_split", C.c_int), ("products", C.c_int),
                ("autotune", C.c_int)]


_lib = None


def load(path: str | None = None):
    """Load libddlra.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libddlra.so not built ({p}); run __graft_entry__.build()")
    lib = C.CDLL(p)
    vp = C.c_void_p
    lib.dd_dlra_create.argtypes = [C.POINTER(Grid), C.POINTER(Tiling), C.POINTER(Quadrature),
                                   C.POINTER(Fields), _dp, C.POINTER(Options), vp,
                                   C.POINTER(vp)]
    lib.dd_dlra_step.argtypes = [vp, C.c_int]
    lib.dd_dlra_set_graph.argtypes = [vp, C.c_int]
    lib.dd_dlra_scalar_flux.argtypes = [vp, vp, C.c_int]
    lib.dd_dlra_scalar_flux_instance.argtypes = [vp, C.c_int, vp, C.c_int]
    lib.dd_dlra_ranks.argtypes = [vp, _ip, _ip]
    lib.dd_dlra_info.argtypes = [vp, _ip, _ip, _ip]
    lib.dd_dlra_get_factors.argtypes = [vp, C.c_int, _dp, _dp, _dp, _ip]
    lib.dd_dlra_set_factors.argtypes = [vp, C.c_int, C.c_int, _dp, _dp, _dp]
    lib.dd_dlra_sync.argtypes = [vp]
    lib.dd_dlra_destroy.argtypes = [vp]
    lib.dd_dlra_destroy.restype = None
    lib.dd_last_error.restype = C.c_char_p
    lib.dd_dlra_last_error.argtypes = [vp]
    lib.dd_dlra_last_error.restype = C.c_char_p
    lib.dd_set_allocator.argtypes = [vp]
    lib.dd_profile_slots.argtypes = []
    lib.dd_profile_slot_name.argtypes = [C.c_int]
    lib.dd_profile_slot_name.restype = C.c_char_p
    lib.dd_dlra_profile.argtypes = [vp, C.c_int, _dp, _ip]
    lib.dd_dlra_profile_work.argtypes = [vp, C.c_int, _dp, _ip, _dp]
    lib.dd_dlra_scalar_flux_noalloc.argtypes = [vp, vp]
    lib.dd_dlra_tuning.argtypes = [vp, _ip, _dp]
    lib.dd_dlra_create_batch.argtypes = [C.c_int, C.POINTER(Grid), C.POINTER(Tiling),
                                         C.POINTER(Quadrature), C.POINTER(Fields),
                                         C.POINTER(_dp), C.POINTER(Options), vp, C.POINTER(vp)]
    lib.dd_dlra_instance.argtypes = [vp, C.c_int, _ip, _ip, _ip, _ip, _ip]
    for name in EXPORTS:
        if name not in ("dd_dlra_destroy", "dd_last_error", "dd_dlra_last_error",
                        "dd_profile_slot_name"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _RELEASE_FN), ("ctx", C.c_void_p)]


_allocator_keep = None    # the callbacks in effect (kept alive while the library may call them)


def set_allocator(alloc=None, release=None):
    """dd_set_allocator: ``alloc(nbytes) -> int`` device address (256-byte aligned) and
    ``release(address)`` supply the device memory of solvers created from now on (e.g.
    ``torch.cuda.caching_allocator_alloc`` / ``caching_allocator_delete``); no arguments
    restores cudaMalloc / cudaFree.  A solver releases its memory through the callbacks in
    effect when it was created, so keep them alive until those solvers are closed."""
    global _allocator_keep
    lib = load()
    if alloc is None and release is None:
        _check(lib, lib.dd_set_allocator(None))
        return
    if alloc is None or release is None:
        raise ValueError("set_allocator needs both alloc and release")

    def _a(nbytes, ctx):
        try:
            return int(alloc(int(nbytes)))
        except Exception:           # noqa: BLE001 - a failed allocation is reported as NULL
            return None

    def _r(ptr, ctx):
        release(int(ptr))

    a = Allocator(_ALLOC_FN(_a), _RELEASE_FN(_r), None)
    _check(lib, lib.dd_set_allocator(C.byref(a)))
    _allocator_keep = (_allocator_keep or []) + [a]


class DDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(lib, st):
    if st != DD_OK:
        raise DDError(st, lib.dd_last_error().decode())


def selftest_wait(polls: int) -> bool:
    """dd_selftest_wait: run the tensor-core kernels' bounded wait on a barrier nothing
    completes for at most ``polls`` polls; True when the timeout reached the host as the
    status bit the production kernels set."""
    lib = load()
    out = C.c_int(0)
    _check(lib, lib.dd_selftest_wait(C.c_uint(int(polls)), C.byref(out)))
    return bool(out.value)


def _choice(what, value, table):
    """The library's code for an option value; an unknown value is refused here."""
    if value not in table:
        raise ValueError(f"{what} {value!r}: one of {sorted(table)}")
    return table[value]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Solver:
    """DD-DLRA solver on one problem; wraps a dd_dlra_t handle."""

    def __init__(self, wl, tau: float = 1e-5, stream: int = 0, use_graph: bool = False,
                 precision: str = "fp64", products: str = "fp64", autotune: bool = False):
        """wl: one workload, or a list of workloads sharing the direction table (a batch).
        products: "fp64", "tensor" or "auto" (dd_options.products); autotune: time the
        launch choices at creation (dd_options.autotune)."""
        lib = load()
        self.lib = lib
        wls = list(wl) if isinstance(wl, (list, tuple)) else [wl]
        self.wls = wls
        self.wl = wls[0]
        self._keep = []
        n = len(wls)
        grids = (Grid * n)()
        tils = (Tiling * n)()
        flds = (Fields * n)()
        opts = (Options * n)()
        g0s = (_dp * n)()
        for i, w in enumerate(wls):
            xc = np.ascontiguousarray(w.xcuts, dtype=np.int32)
            yc = np.ascontiguousarray(w.ycuts, dtype=np.int32)
            ss, sa, q, g0 = _d(w.sigma_s), _d(w.sigma_a), _d(w.source), _d(w.g0)
            self._keep += [xc, yc, ss, sa, q, g0]
            grids[i] = Grid(w.nx, w.ny, w.x0, w.x1, w.y0, w.y1)
            tils[i] = Tiling(len(xc) - 1, len(yc) - 1, xc.ctypes.data_as(_ip),
                             yc.ctypes.data_as(_ip))
            ig, ih = (_dp * 4)(), (_dp * 4)()
            for j, side in enumerate(INFLOW_SIDES):
                if side in w.inflow:
                    gs, hs = _d(w.inflow[side][0]), _d(w.inflow[side][1])
                    self._keep += [gs, hs]
                    ig[j], ih[j] = _ptr(gs), _ptr(hs)
            flds[i] = Fields(_ptr(ss), _ptr(sa), _ptr(q), ig, ih)
            fixed = w.rank_mode == "fixed"
            if w.rank_mode not in ("fixed", "tol"):
                raise ValueError(f"rank_mode {w.rank_mode!r}: 'fixed' or 'tol'")
            opts[i] = Options(DD_RANK_FIXED if fixed else DD_RANK_TOL, w.rank, w.tol, w.r_min,
                              w.r_max, w.r_aug_max,
                              _choice("integrator", w.integrator, {"euler": DD_EULER, "rk4": DD_RK4}),
                              w.c_adv, w.dt, tau, _choice("precision", precision, PRECISIONS),
                              1 if w.mass_fix else 0,
                              _choice("splitting", w.splitting, {"lie": 0, "strang": 1}),
                              _choice("kstep_split", w.kstep_split, {"eigen": 0, "flux": 1}),
                              _choice("products", products, PRODUCTS), 1 if autotune else 0)
            g0s[i] = _ptr(g0)
        w0 = wls[0]
        ox, oy, w = _d(w0.omega_x), _d(w0.omega_y), _d(w0.w)
        self._keep += [ox, oy, w, grids, tils, flds, opts, g0s]
        quad = Quadrature(w0.n, _ptr(ox), _ptr(oy), _ptr(w), w0.n_mu, w0.n_phi)
        h = C.c_void_p()
        if n == 1:
            st = lib.dd_dlra_create(C.byref(grids[0]), C.byref(tils[0]), C.byref(quad),
                                    C.byref(flds[0]), g0s[0], C.byref(opts[0]),
                                    C.c_void_p(stream), C.byref(h))
        else:
            st = lib.dd_dlra_create_batch(n, grids, tils, C.byref(quad), flds, g0s, opts,
                                          C.c_void_p(stream), C.byref(h))
        _check(lib, st)
        self.h = h
        nsub, nd, rc = C.c_int(), C.c_int(), C.c_int()
        _check(lib, lib.dd_dlra_info(h, C.byref(nsub), C.byref(nd), C.byref(rc)))
        self.nsub, self.n, self.r_cap = nsub.value, nd.value, rc.value
        self.layout = []
        for i in range(n):
            a, b, c, d, e = (C.c_int() for _ in range(5))
            _check(lib, lib.dd_dlra_instance(h, i, C.byref(a), C.byref(b), C.byref(c), C.byref(d),
                                             C.byref(e)))
            self.layout.append((a.value, b.value, c.value, d.value, e.value))
        self.ncells_out = sum(w.nx * w.ny for w in wls)
        if use_graph:
            _check(lib, lib.dd_dlra_set_graph(h, 1))

    def tuning(self):
        """The launch choices in use and the autotuner's timings (dd_dlra_tuning):
        ({"oz_spatial", "oz_angular", "chunks_spatial", "chunks_angular"}, ms[8])."""
        ch = np.zeros(6, dtype=np.int32)
        ms = np.zeros(8)
        _check(self.lib, self.lib.dd_dlra_tuning(self.h, ch.ctypes.data_as(_ip), _ptr(ms)))
        return ({"oz_spatial": int(ch[0]), "oz_angular": int(ch[1]),
                 "chunks_spatial": int(ch[2]), "chunks_angular": int(ch[3]),
                 "oz_gram_spatial": int(ch[4]), "oz_gram_angular": int(ch[5])}, ms.tolist())

    def step(self, nsteps: int = 1):
        _check(self.lib, self.lib.dd_dlra_step(self.h, int(nsteps)))

    def sync(self):
        _check(self.lib, self.lib.dd_dlra_sync(self.h))

    def scalar_flux(self, out=None):
        """Host numpy array (synchronising), or write into a device pointer ``out``
        (an int address, e.g. a torch tensor's data_ptr())."""
        if out is not None:
            _check(self.lib, self.lib.dd_dlra_scalar_flux(self.h, C.c_void_p(out), 1))
            return None
        rho = np.empty(self.ncells_out)
        _check(self.lib, self.lib.dd_dlra_scalar_flux(self.h, rho.ctypes.data_as(C.c_void_p), 0))
        return rho

    def scalar_flux_instance(self, i, out=None):
        """Problem i's density alone (dd_dlra_scalar_flux_instance): a host numpy array
        (synchronising), or written into the device pointer ``out``."""
        if out is not None:
            _check(self.lib, self.lib.dd_dlra_scalar_flux_instance(self.h, int(i), C.c_void_p(out), 1))
            return None
        if not 0 <= int(i) < len(self.layout):        # the library refuses it (DD_ERR_ARG)
            _check(self.lib, self.lib.dd_dlra_scalar_flux_instance(self.h, int(i), None, 0))
        _, _, _, nx, ny = self.layout[i]
        rho = np.empty(nx * ny)
        _check(self.lib, self.lib.dd_dlra_scalar_flux_instance(
            self.h, int(i), rho.ctypes.data_as(C.c_void_p), 0))
        return rho

    def scalar_flux_noalloc(self, out):
        """Density into the device pointer ``out`` without any allocation (see
        dd_dlra_scalar_flux_noalloc in include/ddlra.h)."""
        _check(self.lib, self.lib.dd_dlra_scalar_flux_noalloc(self.h, C.c_void_p(out)))

    def ranks(self):
        st = np.empty(self.nsub, dtype=np.int32)
        it = np.empty(2 * self.nsub, dtype=np.int32)
        _check(self.lib, self.lib.dd_dlra_ranks(self.h, st.ctypes.data_as(_ip),
                                                it.ctypes.data_as(_ip)))
        return st, it.reshape(2, self.nsub)

    def instance_flux(self, rho, i):
        """Problem i's density out of the concatenated output of scalar_flux()."""
        _, _, off, nx, ny = self.layout[i]
        return rho[off:off + nx * ny]

    def subdomain_cells(self, k):
        for i, (k0, ns, _, _, _) in enumerate(self.layout):
            if k0 <= k < k0 + ns:
                wl = self.wls[i]
                kk = k - k0
                TX = len(wl.xcuts) - 1
                I, J = kk % TX, kk // TX
                return (wl.xcuts[I + 1] - wl.xcuts[I]) * (wl.ycuts[J + 1] - wl.ycuts[J])
        raise IndexError(k)

    def get_factors(self, k):
        N = self.subdomain_cells(k)
        U = np.empty((N, self.r_cap))
        S = np.empty((self.r_cap, self.r_cap))
        V = np.empty((self.n, self.r_cap))
        r = C.c_int()
        _check(self.lib, self.lib.dd_dlra_get_factors(self.h, k, _ptr(U), _ptr(S), _ptr(V),
                                                       C.byref(r)))
        r = r.value
        U = U.reshape(-1)[:N * r].reshape(N, r)
        S = S.reshape(-1)[:r * r].reshape(r, r)
        V = V.reshape(-1)[:self.n * r].reshape(self.n, r)
        return U, S, V

    def set_factors(self, k, U, S, V):
        U, S, V = _d(U), _d(S), _d(V)
        r = S.shape[0]
        _check(self.lib, self.lib.dd_dlra_set_factors(self.h, k, r, _ptr(U), _ptr(S), _ptr(V)))

    def profile(self, nsteps: int, work: bool = False):
        """Advance nsteps steps with a CUDA event pair around every kernel launch;
        returns {kernel: (total_ms, launches)}, or with work=True {kernel: (total_ms,
        launches, algorithmic_flops)}."""
        ns = self.lib.dd_profile_slots()
        ms = np.zeros(ns)
        cnt = np.zeros(ns, dtype=np.int32)
        fl = np.zeros(ns)
        if work:
            _check(self.lib, self.lib.dd_dlra_profile_work(self.h, int(nsteps), _ptr(ms),
                                                            cnt.ctypes.data_as(_ip), _ptr(fl)))
        else:
            _check(self.lib, self.lib.dd_dlra_profile(self.h, int(nsteps), _ptr(ms),
                                                       cnt.ctypes.data_as(_ip)))
        out = {}
        for i in range(ns):
            if cnt[i]:
                name = self.lib.dd_profile_slot_name(i).decode()
                out[name] = (float(ms[i]), int(cnt[i]), float(fl[i])) if work else \
                    (float(ms[i]), int(cnt[i]))
        return out

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dd_dlra_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
