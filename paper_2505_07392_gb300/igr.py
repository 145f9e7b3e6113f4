"""ctypes binding of the C ABI in include/igr.h.

Argument marshalling only: every step of the stage runs in libigr.so's CUDA
kernels. PyTorch supplies device memory (its caching allocator backs the
context's buffers through the igr_allocator callbacks) and the stream.
Importing this module does not load the library; the first call does, and
it raises if libigr.so has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# IGR_LIBRARY selects another build of the same library (the bounds-checking
# libigr_debug.so); the default is the in-tree libigr.so
LIB_PATH = os.environ.get("IGR_LIBRARY") or os.path.join(HERE, "libigr.so")

# enums of igr.h
OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
F64, F32, F32_F16STORE, F32_BF16STORE, F32_F16INC, F32_BF16INC = range(6)
DT_F64, DT_F32, DT_F16, DT_BF16 = range(4)
KC_SOURCE, KC_JACOBI, KC_FLUX, KC_OTHER = range(4)

# f16inc / bf16inc: the state q^n in FP32, 16-bit stage increments, Sigma and b
PRECISIONS = {"f64": F64, "f32": F32, "f16": F32_F16STORE, "bf16": F32_BF16STORE,
              "f16inc": F32_F16INC, "bf16inc": F32_BF16INC}
STATUS = {0: "IGR_OK", 1: "IGR_ERR_INVALID_ARG", 2: "IGR_ERR_OOM", 3: "IGR_ERR_CUDA",
          4: "IGR_ERR_NONFINITE", 5: "IGR_ERR_TIMEOUT", 6: "IGR_ERR_UNSUPPORTED"}


class Jet(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("cx", "cy", "radius", "rho", "w", "p", "edge_width")]


class Allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)),
                ("user", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("gamma", C.c_double), ("alpha", C.c_double), ("cfl", C.c_double),
                ("sweeps", C.c_int), ("prec", C.c_int), ("bc", C.c_int * 6),
                ("jets", C.POINTER(Jet)), ("njets", C.c_int), ("host_rk_base", C.c_int),
                ("order", C.c_int), ("sigma_solver", C.c_int), ("mu", C.c_double), ("zeta", C.c_double)]


class IGRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


class Diagnostics(C.Structure):
    """igr_diagnostics."""
    _fields_ = [("mass", C.c_double), ("momentum", C.c_double * 3), ("energy", C.c_double),
                ("rho_min", C.c_double), ("p_min", C.c_double), ("sigma_absmax", C.c_double),
                ("b_norm", C.c_double), ("sigma_residual", C.c_double)]


def lib():
    """The loaded libigr.so with argument types set."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2505_07392_gb300.build` (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        p, i, d = C.c_void_p, C.c_int, C.c_double
        sigs = {
            "igr_create": (i, [C.POINTER(Config), C.POINTER(Allocator), p, C.POINTER(p)]),
            "igr_memory_bytes": (C.c_size_t, [C.POINTER(Config)]),
            "igr_destroy": (i, [p]),
            "igr_set_state": (i, [p, p, p, i, i]),
            "igr_get_state": (i, [p, p, p, i, i]),
            "igr_set_conserved": (i, [p, p, i, i]),
            "igr_step_host": (i, [p, p, p, i, i]),
            "igr_step": (i, [p, i, d, C.POINTER(d)]),
            "igr_solve_sigma": (i, [p, p, p, i, i]),
            "igr_rhs": (i, [p, p, p, p, i]),
            "igr_get_dt": (i, [p, C.POINTER(d)]),
            "igr_rk_combine": (i, [p, p, p, p, p, C.c_longlong, i, d]),
            "igr_solve_sigma_noalloc": (i, [C.POINTER(Config), p, p, i, p]),
            "igr_noalloc_max_cells": (C.c_size_t, [i]),
            "igr_noalloc_last_error": (C.c_char_p, []),
            "igr_adjoint_step": (i, [p, p, p, p, p, p, p, C.POINTER(d), d, i]),
            "igr_set_tiles": (i, [p, i, i, i]),
            "igr_get_tiles": (i, [p, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
            "igr_set_kernel_forms": (i, [p, i, i]),
            "igr_get_kernel_forms": (i, [p, C.POINTER(i), C.POINTER(i)]),
            "igr_autotune": (i, [p, i]),
            "igr_create_batch": (i, [C.POINTER(Config), i, C.POINTER(Allocator), p, C.POINTER(p)]),
            "igr_batch_instance": (p, [p, i]),
            "igr_step_batch": (i, [p, i]),
            "igr_autotune_batch": (i, [p, i]),
            "igr_sync_batch": (i, [p]),
            "igr_batch_last_error": (C.c_char_p, [p]),
            "igr_destroy_batch": (i, [p]),
            "igr_sync": (i, [p]),
            "igr_get_flags": (i, [p, C.POINTER(i)]),
            "igr_diagnose": (i, [p, C.POINTER(Diagnostics)]),
            "igr_debug_bounds_hits": (i, [C.POINTER(C.c_ulonglong), i]),
            "igr_debug_bounds_selftest": (i, []),
            "igr_profile_enable": (i, [p, i]),
            "igr_profile_read": (i, [p, i, C.POINTER(C.c_longlong), C.POINTER(d)]),
            "igr_last_error": (C.c_char_p, [p]),
            "igr_version": (C.c_char_p, []),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def make_config(case, precision: str = "f32", host_rk_base: bool = False):
    """Config struct (and the jet array it points to) from an inputs.Case."""
    jets = (Jet * max(1, len(case.jets)))(*[Jet(*j) for j in case.jets])
    cfg = Config(int(case.nx), int(case.ny), int(case.nz), float(case.dx), float(case.gamma),
                 float(case.alpha), float(case.cfl), int(case.sweeps), PRECISIONS[precision],
                 (C.c_int * 6)(*[int(b) for b in case.bc]), jets, len(case.jets), int(host_rk_base),
                 int(getattr(case, "order", 5)), int(getattr(case, "sigma_solver", 0)),
                 float(getattr(case, "mu", 0.0)), float(getattr(case, "zeta", 0.0)))
    return cfg, jets


def memory_bytes(case, precision: str = "f32", host_rk_base: bool = False) -> int:
    cfg, _jets = make_config(case, precision, host_rk_base)
    return int(lib().igr_memory_bytes(C.byref(cfg)))


def storage_torch_dtype(precision: str):
    """Element type of Sigma and b (and of the increments of the increment modes)."""
    import torch
    return {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16,
            "bf16": torch.bfloat16, "f16inc": torch.float16, "bf16inc": torch.bfloat16}[precision]


def state_torch_dtype(precision: str):
    """Element type of the state q: the storage type, FP32 in the increment modes."""
    import torch
    return torch.float32 if precision.endswith("inc") else storage_torch_dtype(precision)


def compute_torch_dtype(precision: str):
    import torch
    return torch.float64 if precision == "f64" else torch.float32


_TORCH_DT = None


def _dt_code(t):
    import torch
    global _TORCH_DT
    if _TORCH_DT is None:
        _TORCH_DT = {torch.float64: DT_F64, torch.float32: DT_F32, torch.float16: DT_F16,
                     torch.bfloat16: DT_BF16}
    return _TORCH_DT[t]


_NP_DT = {np.dtype(np.float64): DT_F64, np.dtype(np.float32): DT_F32, np.dtype(np.float16): DT_F16}


def autotune_key(case, precision: str, host_rk_base: bool, device_name: str) -> str:
    """What a tuned launch shape depends on: grid shape, storage precision,
    scheme variant, RK base placement and GPU model."""
    visc = float(getattr(case, "mu", 0.0)) > 0 or float(getattr(case, "zeta", 0.0)) > 0
    return "%dx%dx%d:%s:order%d:solver%d:visc%d:hostbase%d:%s" % (
        case.nx, case.ny, case.nz, precision, int(getattr(case, "order", 5)),
        int(getattr(case, "sigma_solver", 0)), int(visc), int(bool(host_rk_base)), device_name)


def autotune_cache_load(path: str) -> dict:
    """The stored launch shapes ({} when the file is missing or unreadable)."""
    import json
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def autotune_cache_store(path: str, key: str, value: dict) -> None:
    """Add one entry, written to a temporary file and renamed into place."""
    import json
    d = autotune_cache_load(path)
    d[key] = value
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Solver:
    """One IGR context on the current CUDA device and PyTorch's current stream."""

    def __init__(self, case, precision: str = "f32", stream=None, torch_allocator: bool = True,
                 host_rk_base: bool = False):
        """host_rk_base keeps the RK base q^n in pinned host memory (igr_config)."""
        import torch
        self.case = case
        self.precision = precision
        self.host_rk_base = bool(host_rk_base)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.n = case.nx * case.ny * case.nz
        self.shape = (case.nz, case.ny, case.nx)
        self._cfg, self._jets = make_config(case, precision, host_rk_base)
        self._alloc = None
        if torch_allocator:
            dev, st = self.device.index, self.stream

            @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
            def _a(nbytes, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, st))
                except Exception:
                    return None

            @C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
            def _f(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc = Allocator(_a, _f, None)
        h = C.c_void_p()
        s = lib().igr_create(C.byref(self._cfg), C.byref(self._alloc) if self._alloc else None,
                             C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if s != OK:
            raise IGRError(s, lib().igr_last_error(None).decode())
        self.h = h

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            lib().igr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, s):
        if s != OK:
            raise IGRError(s, lib().igr_last_error(self.h).decode())

    # -- state
    def set_state(self, q, sigma=None):
        """q: (5, nz, ny, nx) torch CUDA tensor (any float dtype) or a numpy
        array in the storage dtype (host); sigma likewise or None (zero)."""
        import torch
        if isinstance(q, torch.Tensor):
            q = q.contiguous()
            if sigma is not None:
                sigma = sigma.to(q.dtype).contiguous()
            self._check(lib().igr_set_state(self.h, C.c_void_p(q.data_ptr()),
                                            C.c_void_p(sigma.data_ptr()) if sigma is not None else None,
                                            _dt_code(q.dtype), 1))
            # the copy is asynchronous on the solver's stream
            if self.stream != torch.cuda.current_stream(self.device):
                q.record_stream(self.stream)
                if sigma is not None:
                    sigma.record_stream(self.stream)
        else:
            q = np.ascontiguousarray(q)
            sp = None
            if sigma is not None:
                sigma = np.ascontiguousarray(sigma, dtype=q.dtype)
                sp = sigma.ctypes.data_as(C.c_void_p)
            self._check(lib().igr_set_state(self.h, q.ctypes.data_as(C.c_void_p), sp,
                                            _NP_DT[q.dtype], 0))

    def set_conserved(self, q):
        """Replace q alone and keep Sigma (igr_set_conserved); q as for
        set_state."""
        import torch
        if isinstance(q, torch.Tensor):
            q = q.contiguous()
            self._check(lib().igr_set_conserved(self.h, C.c_void_p(q.data_ptr()), _dt_code(q.dtype), 1))
            if self.stream != torch.cuda.current_stream(self.device):
                q.record_stream(self.stream)
        else:
            q = np.ascontiguousarray(q)
            self._check(lib().igr_set_conserved(self.h, q.ctypes.data_as(C.c_void_p), _NP_DT[q.dtype], 0))

    def step_host(self, q_in: np.ndarray, q_out: Optional[np.ndarray] = None, nsteps: int = 1):
        """igr_step_host: q_in (host, storage dtype) in, nsteps steps, the
        final q into q_out (default: q_in, in place). Sigma stays on the device."""
        q_in = np.ascontiguousarray(q_in)
        q_out = q_in if q_out is None else q_out
        assert q_out.flags.c_contiguous and q_out.dtype == q_in.dtype and q_out.shape == q_in.shape
        self._check(lib().igr_step_host(self.h, q_in.ctypes.data_as(C.c_void_p), q_out.ctypes.data_as(C.c_void_p),
                                        int(nsteps), _NP_DT[q_in.dtype]))
        return q_out

    def get_state(self, dtype=None):
        """(q, sigma) as new CUDA tensors (default: the state dtype)."""
        import torch
        dtype = dtype or state_torch_dtype(self.precision)
        q = torch.empty((5,) + self.shape, dtype=dtype, device=self.device)
        s = torch.empty(self.shape, dtype=dtype, device=self.device)
        self._check(lib().igr_get_state(self.h, C.c_void_p(q.data_ptr()), C.c_void_p(s.data_ptr()),
                                        _dt_code(dtype), 1))
        return q, s

    def get_state_host(self, q_out: np.ndarray, sigma_out: Optional[np.ndarray] = None):
        """Copy the state into host arrays of the storage dtype."""
        self._check(lib().igr_get_state(self.h, q_out.ctypes.data_as(C.c_void_p),
                                        sigma_out.ctypes.data_as(C.c_void_p) if sigma_out is not None else None,
                                        _NP_DT[q_out.dtype], 0))

    # -- stepping
    def step(self, nsteps: int = 1, fixed_dt: float = 0.0, sync: bool = True):
        """Advance nsteps; returns the elapsed simulated time if sync."""
        if sync:
            t = C.c_double(0.0)
            self._check(lib().igr_step(self.h, int(nsteps), float(fixed_dt), C.byref(t)))
            return t.value
        self._check(lib().igr_step(self.h, int(nsteps), float(fixed_dt), None))
        return None

    def dt(self) -> float:
        d = C.c_double()
        self._check(lib().igr_get_dt(self.h, C.byref(d)))
        return d.value

    def sync(self):
        self._check(lib().igr_sync(self.h))

    def diagnose(self) -> dict:
        """FP64 totals, extrema and the Sigma residual of the current state
        (igr_diagnose)."""
        d = Diagnostics()
        self._check(lib().igr_diagnose(self.h, C.byref(d)))
        return {"mass": d.mass, "momentum": tuple(d.momentum), "energy": d.energy,
                "rho_min": d.rho_min, "p_min": d.p_min, "sigma_absmax": d.sigma_absmax,
                "b_norm": d.b_norm, "sigma_residual": d.sigma_residual}

    def flags(self) -> int:
        """Warnings since the last call (IGR_WARN_FACE_POSITIVITY = 2)."""
        f = C.c_int()
        self._check(lib().igr_get_flags(self.h, C.byref(f)))
        return f.value

    # -- stand-alone operators on caller buffers (CUDA; q in the state dtype,
    #    sigma in the storage dtype)
    def solve_sigma(self, q, sigma, sweeps: int):
        """In place on sigma: b from q, then `sweeps` warm-started Jacobi sweeps."""
        self._check(lib().igr_solve_sigma(self.h, C.c_void_p(q.data_ptr()), C.c_void_p(sigma.data_ptr()),
                                          int(sweeps), _dt_code(sigma.dtype)))
        return sigma

    def rhs(self, q, sigma):
        """L(q; Sigma) as a new (5, nz, ny, nx) tensor in the arithmetic dtype."""
        import torch
        out = torch.empty((5,) + self.shape, dtype=compute_torch_dtype(self.precision), device=self.device)
        self._check(lib().igr_rhs(self.h, C.c_void_p(q.data_ptr()), C.c_void_p(sigma.data_ptr()),
                                  C.c_void_p(out.data_ptr()), _dt_code(sigma.dtype)))
        return out

    def rk_combine(self, qn, qs, L, stage: int, dt: float):
        """The stage kernel's RK combination on flat tensors (storage dtype; L in
        the arithmetic dtype); returns a new tensor."""
        import torch
        out = torch.empty_like(qn)
        self._check(lib().igr_rk_combine(self.h, C.c_void_p(qn.data_ptr()), C.c_void_p(qs.data_ptr()),
                                         C.c_void_p(L.data_ptr()), C.c_void_p(out.data_ptr()),
                                         int(qn.numel()), int(stage), float(dt)))
        return out

    # -- adjoint
    def adjoint_step(self, q_n, sigma_n, lam_q, lam_sigma, dt: float):
        """Adjoint of one SSP-RK3 step with fixed dt from the stored state
        (q_n, sigma_n): returns (lam_q_n, lam_sigma_n, grad_jet_w)."""
        import torch
        ct = compute_torch_dtype(self.precision)
        lam_q = lam_q.to(ct).contiguous()
        lam_sigma = lam_sigma.to(ct).contiguous()
        out_q = torch.empty_like(lam_q)
        out_s = torch.empty_like(lam_sigma)
        nj = len(self.case.jets)
        gw = (C.c_double * max(1, nj))()
        self._check(lib().igr_adjoint_step(self.h, C.c_void_p(q_n.data_ptr()), C.c_void_p(sigma_n.data_ptr()),
                                           C.c_void_p(lam_q.data_ptr()), C.c_void_p(lam_sigma.data_ptr()),
                                           C.c_void_p(out_q.data_ptr()), C.c_void_p(out_s.data_ptr()),
                                           gw if nj else None, float(dt), _dt_code(q_n.dtype)))
        return out_q, out_s, [gw[j] for j in range(nj)]

    # -- launch shapes
    def set_tiles(self, zc_source: int, zc_jacobi: int, zc_flux: int):
        self._check(lib().igr_set_tiles(self.h, int(zc_source), int(zc_jacobi), int(zc_flux)))

    def tiles(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._check(lib().igr_get_tiles(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def set_kernel_forms(self, source_vec4: int = -1, jacobi_vec4: int = -1):
        """Forms of the source and Jacobi kernels: -1 default rule, 0 one
        cell per thread, 1 four cells per thread (nx % 4 == 0)."""
        self._check(lib().igr_set_kernel_forms(self.h, int(source_vec4), int(jacobi_vec4)))

    def kernel_forms(self):
        a, b = C.c_int(), C.c_int()
        self._check(lib().igr_get_kernel_forms(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def autotune(self, reps: int = 3, cache: Optional[str] = None):
        """igr_autotune, or the launch shape stored for the same problem and
        GPU in the JSON file `cache` (default: $IGR_AUTOTUNE_CACHE; none when
        unset). A tuned shape is stored there for the next context."""
        path = cache if cache is not None else os.environ.get("IGR_AUTOTUNE_CACHE")
        key = None
        if path:
            import torch
            key = autotune_key(self.case, self.precision, getattr(self, "host_rk_base", False),
                               torch.cuda.get_device_name(self.device))
            hit = autotune_cache_load(path).get(key)
            if hit:
                self.set_tiles(*hit["tiles"])
                self.set_kernel_forms(*hit["forms"])
                return self.tiles()
        self._check(lib().igr_autotune(self.h, int(reps)))
        if key:
            autotune_cache_store(path, key, {"tiles": list(self.tiles()), "forms": list(self.kernel_forms())})
        return self.tiles()

    # -- per-kernel timing
    def profile(self, on: bool = True):
        self._check(lib().igr_profile_enable(self.h, int(on)))

    def profile_read(self, kernel_class: int):
        n, ms = C.c_longlong(), C.c_double()
        self._check(lib().igr_profile_read(self.h, int(kernel_class), C.byref(n), C.byref(ms)))
        return int(n.value), float(ms.value)


class _Instance(Solver):
    """A context owned by a Batch (not destroyed on its own)."""

    def __init__(self, case, precision, handle, stream):
        import torch
        self.case = case
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        self.n = case.nx * case.ny * case.nz
        self.shape = (case.nz, case.ny, case.nx)
        self.h = handle

    def close(self):
        self.h = None


class Batch:
    """Independent instances advanced together (igr_create_batch): one CUDA
    graph per step with a branch per instance, replayed."""

    def __init__(self, cases, precision: str = "f16", stream=None, torch_allocator: bool = True):
        import torch
        self.cases = list(cases)
        self.precision = precision
        self.stream = stream or torch.cuda.current_stream()
        made = [make_config(c, precision) for c in self.cases]
        self._jets = [m[1] for m in made]
        cfgs = (Config * len(made))(*[m[0] for m in made])
        self._cfgs = cfgs
        helper = Solver.__new__(Solver)
        self._alloc = None
        if torch_allocator:
            dev = torch.cuda.current_device()

            @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
            def _a(nbytes, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, self.stream))
                except Exception:
                    return None

            @C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
            def _f(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc = Allocator(_a, _f, None)
        h = C.c_void_p()
        s = lib().igr_create_batch(cfgs, len(made), C.byref(self._alloc) if self._alloc else None,
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if s != OK:
            raise IGRError(s, lib().igr_last_error(None).decode())
        self.h = h
        self.instances = [_Instance(c, precision, lib().igr_batch_instance(h, i), self.stream)
                          for i, c in enumerate(self.cases)]

    def step(self, nsteps: int = 1, sync: bool = False):
        s = lib().igr_step_batch(self.h, int(nsteps))
        if s != OK:
            raise IGRError(s, lib().igr_batch_last_error(self.h).decode())
        if sync:
            self.sync()

    def autotune(self, reps: int = 3):
        """igr_autotune_batch: every instance's launch shape for the batch
        (each distinct problem tuned alone, then the z-chunks of each kernel
        class scaled together over the whole batch). Returns each instance's
        (zc_source, zc_jacobi, zc_flux)."""
        s = lib().igr_autotune_batch(self.h, int(reps))
        if s != OK:
            raise IGRError(s, lib().igr_batch_last_error(self.h).decode())
        return [inst.tiles() for inst in self.instances]

    def sync(self):
        s = lib().igr_sync_batch(self.h)
        if s != OK:
            raise IGRError(s, lib().igr_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            for inst in self.instances:
                inst.h = None
            lib().igr_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
