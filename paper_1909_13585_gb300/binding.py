"""ctypes binding of libtobk.so: the C-ABI of include/tobk.h, one Python function per C entry point
with the same name, plus `Solver`, a thin owner of a handle that marshals numpy arrays and torch
tensors (device pointers, stream) into those calls.  No computation happens here: every step of the
solver runs in the library's CUDA kernels.  Importing fails loudly if the library is missing."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtobk.so")

TOBK_OK, TOBK_E_ARG, TOBK_E_STATE, TOBK_E_NOMEM, TOBK_E_CUDA, TOBK_E_NOT_CONVERGED, \
    TOBK_E_BREAKDOWN, TOBK_E_TIMEOUT, TOBK_E_NONFINITE = range(9)
TOBK_FP64, TOBK_FP32_VCYCLE = 0, 1
TOBK_ELEMENT_PLAIN, TOBK_ELEMENT_INCOMPATIBLE = 0, 1
TOBK_FIELD_U, TOBK_FIELD_MODES, TOBK_FIELD_ADJOINT, TOBK_FIELD_ADJOINT_RHS, TOBK_FIELD_FINE_ADJOINT, \
    TOBK_FIELD_COARSE_ADJOINT, TOBK_FIELD_PROLONGATED = range(7)


class tobk_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nel", C.c_int * 3), ("nu", C.c_double), ("E0", C.c_double),
                ("Emin", C.c_double), ("penal", C.c_double), ("mg_levels", C.c_int),
                ("eig_level", C.c_int), ("num_modes", C.c_int), ("precision", C.c_int),
                ("rtol", C.c_double), ("max_iter", C.c_int), ("omega", C.c_double),
                ("nu_pre", C.c_int), ("nu_post", C.c_int), ("eig_tol", C.c_double),
                ("eig_max_iter", C.c_int), ("max_rhs", C.c_int), ("eig_inner_iters", C.c_int),
                ("fuse_load_adjoint", C.c_int), ("smoother", C.c_int), ("cheb_ratio", C.c_double),
                ("kaczmarz_sweeps", C.c_int), ("ritz_levels", C.c_int), ("fine_steps", C.c_int),
                ("element", C.c_int), ("eig_gram_tc", C.c_int), ("consistent_sens", C.c_int), ("early_fine", C.c_int)]


class tobk_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("num_rhs", C.c_int),
                ("rel_residual", C.c_double), ("time_ms", C.c_double), ("status_detail", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_H = C.c_void_p
_P = C.c_void_p
_SIGS = {
    "tobk_default_desc": (C.c_int, [C.POINTER(tobk_desc)]),
    "tobk_create": (C.c_int, [C.POINTER(tobk_desc), C.c_void_p, C.POINTER(_H)]),
    "tobk_destroy": (None, [_H]),
    "tobk_last_error": (C.c_char_p, [_H]),
    "tobk_set_densities": (C.c_int, [_H, _P, C.c_int64, C.c_int]),
    "tobk_set_load": (C.c_int, [_H, _P, C.c_int64, C.c_int]),
    "tobk_set_fixed": (C.c_int, [_H, _P, C.c_int64, C.c_int]),
    "tobk_set_initial_guess": (C.c_int, [_H, _P, C.c_int64, C.c_int]),
    "tobk_solve_equilibrium": (C.c_int, [_H, C.POINTER(C.c_double), C.POINTER(tobk_solve_info)]),
    "tobk_compute_buckling": (C.c_int, [_H, _P, C.POINTER(tobk_solve_info)]),
    "tobk_compute_sensitivities": (C.c_int, [_H, _P, _P, C.c_int, C.POINTER(tobk_solve_info)]),
    "tobk_get_field": (C.c_int, [_H, C.c_int, _P, C.c_int64, C.c_int]),
    "tobk_level_info": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int64)]),
    "tobk_apply_K": (C.c_int, [_H, C.c_int, _P, _P, C.c_int]),
    "tobk_apply_G": (C.c_int, [_H, C.c_int, _P, _P, C.c_int]),
    "tobk_solve": (C.c_int, [_H, C.c_int, _P, _P, C.c_int, C.POINTER(tobk_solve_info)]),
    "tobk_get_element_matrices": (C.c_int, [_H, C.c_int, C.c_int, _P, C.c_int64]),
    "tobk_residual_noalloc": (C.c_int, [C.POINTER(tobk_desc), _P, _P, _P, _P, C.c_int, _P, C.c_void_p]),
    "tobk_gram_tc": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_int64, C.c_int64, _P, C.c_void_p]),
    "tobk_batch_create": (C.c_int, [C.POINTER(tobk_desc), C.c_int, C.c_int, C.c_void_p, C.POINTER(_H)]),
    "tobk_batch_destroy": (None, [_H]),
    "tobk_batch_last_error": (C.c_char_p, [_H]),
    "tobk_batch_layout": (C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "tobk_batch_set_designs": (C.c_int, [_H, _P, _P, C.c_int]),
    "tobk_batch_solve": (C.c_int, [_H, _P, _P, C.c_int, C.POINTER(tobk_solve_info)]),
    "tobk_batch_autotune": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "tobk_batch_set_variants": (C.c_int, [_H, C.c_int, C.c_int]),
    "tobk_unet_default_desc": (C.c_int, [C.c_void_p]),
    "tobk_unet_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(_H)]),
    "tobk_unet_destroy": (None, [_H]),
    "tobk_unet_last_error": (C.c_char_p, [_H]),
    "tobk_unet_num_params": (C.c_int64, [_H]),
    "tobk_unet_set_output_scale": (C.c_int, [_H, C.c_double]),
    "tobk_unet_output_scale": (C.c_double, [_H]),
    "tobk_unet_design_scale": (C.c_int, [_H, _P, _P, C.POINTER(C.c_double)]),
    "tobk_unet_get_state": (C.c_int, [_H, _P, _P, _P, C.POINTER(C.c_longlong), C.c_int]),
    "tobk_unet_set_state": (C.c_int, [_H, _P, _P, _P, C.c_longlong, C.c_int]),
    "tobk_unet_predict": (C.c_int, [_H, _P, _P, _P, _P]),
    "tobk_unet_loss_grad": (C.c_int, [_H, _P, _P, _P, _P, C.POINTER(C.c_float), _P]),
    "tobk_unet_train_step": (C.c_int, [_H, _P, _P, _P, _P, C.c_int, C.c_float, C.POINTER(C.c_float)]),
    "tobk_unet_set_tensor_cores": (C.c_int, [_H, C.c_int]),
    "tobk_conv3_bf16": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int, C.c_int, _P, C.c_void_p]),
    "tobk_launch_count": (C.c_longlong, []),
    "tobk_profile_enable": (C.c_int, [_H, C.c_int]),
    "tobk_phase_enable": (C.c_int, [_H, C.c_int]),
    "tobk_phase_read": (C.c_int, [_H, C.POINTER(C.c_double), C.c_int]),
    "tobk_profile_read": (C.c_int, [_H, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
}

PHASES = ("eigen", "eigen_precond", "eigen_rr", "prolong", "fine_solve", "rq", "eigen_iters")
KERNEL_CLASSES = ("fine_smooth", "fine_residual", "fine_cg_matvec", "coarse", "transfer", "coarsest",
                  "vector", "eigen_dense", "eigen_block")


def launch_count():
    return int(load().tobk_launch_count())

EXPORTED = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Loads libtobk.so and declares every entry point; raises if the library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtobk.so not found at {path}: run __graft_entry__.build() or "
                           "python -m paper_1909_13585_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TobkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tobk error {code}: {msg}")
        self.code = code


def _ptr(a):
    """(pointer, on_device) of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def _arr(a, kind):
    """(pointer, on_device, element count) of a contiguous array of the element type the C-ABI
    expects: kind "f64" (densities, loads, displacements) or "u8" (fixed-DOF masks)."""
    ok = {"f64": ("float64",), "u8": ("uint8", "bool")}[kind]
    name = str(a.dtype).replace("torch.", "")
    if name not in ok:
        raise TypeError(f"expected {kind} data, got {a.dtype}")
    ptr, dev = _ptr(a)
    return ptr, dev, int(a.size if isinstance(a, np.ndarray) else a.numel())


class Solver:
    """Owner of one tobk handle.  Arrays may be numpy (host) or torch tensors (host or device).

    `problem` is any object with dim, nel, nu, E0, Emin, penal, mg_levels, eig_level, num_modes,
    x, f, fixed (e.g. synthetic.Problem)."""

    def __init__(self, problem=None, *, stream=None, precision=TOBK_FP64, rtol=1e-8, max_iter=500,
                 omega=0.6, nu_pre=2, nu_post=2, eig_tol=1e-8, eig_max_iter=200, max_rhs=None,
                 desc=None, **overrides):
        self.lib = load()
        d = tobk_desc()
        self.lib.tobk_default_desc(C.byref(d))
        if problem is not None:
            d.dim = problem.dim
            d.nel[0], d.nel[1] = problem.nel[0], problem.nel[1]
            d.nel[2] = problem.nel[2] if problem.dim == 3 else 1
            d.nu, d.E0, d.Emin, d.penal = problem.nu, problem.E0, problem.Emin, problem.penal
            d.mg_levels, d.eig_level, d.num_modes = problem.mg_levels, problem.eig_level, problem.num_modes
        d.precision, d.rtol, d.max_iter, d.omega = precision, rtol, max_iter, omega
        d.nu_pre, d.nu_post, d.eig_tol, d.eig_max_iter = nu_pre, nu_post, eig_tol, eig_max_iter
        d.max_rhs = max_rhs if max_rhs is not None else d.num_modes + 4
        for k, v in overrides.items():
            setattr(d, k, v)
        if desc is not None:
            d = desc
        self.desc = d
        h = _H()
        s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = self.lib.tobk_create(C.byref(d), C.c_void_p(s), C.byref(h))
        if rc != TOBK_OK:
            raise TobkError(rc, self.lib.tobk_last_error(None).decode())
        self.h = h
        self.dim = d.dim
        self.q = d.num_modes
        info = (C.c_int64 * 5)()
        self.lib.tobk_level_info(self.h, 1, info)
        self.n, self.m = int(info[3]), int(info[4])
        if problem is not None:
            self.set_problem(problem)

    # -- lifetime --------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.tobk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != TOBK_OK and rc not in allow:
            raise TobkError(rc, self.lib.tobk_last_error(self.h).decode())
        return rc

    # -- inputs ----------------------------------------------------------------------------------
    def set_problem(self, p):
        self.set_fixed(np.ascontiguousarray(p.fixed, dtype=np.uint8))
        self.set_load(np.ascontiguousarray(p.f, dtype=np.float64))
        self.set_densities(np.ascontiguousarray(p.x, dtype=np.float64))

    def set_densities(self, x):
        ptr, dev, cnt = _arr(x, "f64")
        self._check(self.lib.tobk_set_densities(self.h, ptr, cnt, dev))

    def set_load(self, f):
        ptr, dev, cnt = _arr(f, "f64")
        self._check(self.lib.tobk_set_load(self.h, ptr, cnt, dev))

    def set_fixed(self, fixed):
        ptr, dev, cnt = _arr(fixed, "u8")
        self._check(self.lib.tobk_set_fixed(self.h, ptr, cnt, dev))

    def set_initial_guess(self, u0):
        if u0 is None:
            self._check(self.lib.tobk_set_initial_guess(self.h, None, 0, 0))
            return
        ptr, dev, cnt = _arr(u0, "f64")
        self._check(self.lib.tobk_set_initial_guess(self.h, ptr, cnt, dev))

    # -- the method ------------------------------------------------------------------------------
    def solve_equilibrium(self, allow_not_converged=False):
        J = C.c_double()
        info = tobk_solve_info()
        self._check(self.lib.tobk_solve_equilibrium(self.h, C.byref(J), C.byref(info)),
                    (TOBK_E_NOT_CONVERGED,) if allow_not_converged else ())
        return J.value, info.as_dict()

    def compute_buckling(self):
        lam = np.zeros(self.q)
        info = tobk_solve_info()
        self._check(self.lib.tobk_compute_buckling(self.h, lam.ctypes.data, C.byref(info)))
        return lam, info.as_dict()

    def compute_sensitivities(self, dlam=None, dJ=None):
        if dlam is None:
            dlam = np.zeros((self.q, self.m))
        if dJ is None:
            dJ = np.zeros(self.m)
        p1, d1 = _ptr(dlam)
        p2, d2 = _ptr(dJ)
        assert d1 == d2
        info = tobk_solve_info()
        self._check(self.lib.tobk_compute_sensitivities(self.h, p1, p2, d1, C.byref(info)))
        return dlam, dJ, info.as_dict()

    def get_field(self, which, out=None):
        size = self.n if which == TOBK_FIELD_U else self.q * self.n
        if out is None:
            out = np.zeros(size)
        ptr, dev = _ptr(out)
        self._check(self.lib.tobk_get_field(self.h, which, ptr, size, dev))
        return out

    # -- unit level (device tensors) -------------------------------------------------------------
    def level_info(self, level):
        info = (C.c_int64 * 5)()
        self._check(self.lib.tobk_level_info(self.h, level, info))
        return dict(nel=tuple(int(v) for v in info[:3]), n=int(info[3]), m=int(info[4]))

    def apply_K(self, level, v, y, nrhs=1):
        self._check(self.lib.tobk_apply_K(self.h, level, v.data_ptr(), y.data_ptr(), nrhs))

    def apply_G(self, level, v, y, nrhs=1):
        self._check(self.lib.tobk_apply_G(self.h, level, v.data_ptr(), y.data_ptr(), nrhs))

    def solve(self, level, B, X, nrhs=1, allow_not_converged=False):
        info = tobk_solve_info()
        self._check(self.lib.tobk_solve(self.h, level, B.data_ptr(), X.data_ptr(), nrhs, C.byref(info)),
                    (TOBK_E_NOT_CONVERGED,) if allow_not_converged else ())
        return info.as_dict()

    def profile(self, enable=True):
        self._check(self.lib.tobk_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            cnt, ms, units = C.c_longlong(), C.c_double(), C.c_double()
            self._check(self.lib.tobk_profile_read(self.h, k, C.byref(cnt), C.byref(ms), C.byref(units)))
            out[name] = dict(launches=int(cnt.value), ms=float(ms.value), dof_rhs=float(units.value))
        return out

    def phase_timing(self, enable=True):
        self._check(self.lib.tobk_phase_enable(self.h, 1 if enable else 0))

    def phase_read(self):
        out = (C.c_double * len(PHASES))()
        self._check(self.lib.tobk_phase_read(self.h, out, len(PHASES)))
        return {k: float(v) for k, v in zip(PHASES, out)}

    def element_matrices(self, level, which, out):
        self._check(self.lib.tobk_get_element_matrices(self.h, level, which, out.data_ptr(), out.numel()))
        return out


def problem_desc(lib, problem, **overrides):
    """A tobk_desc for a problem object (synthetic.Problem-like), defaults from tobk_default_desc."""
    d = tobk_desc()
    lib.tobk_default_desc(C.byref(d))
    d.dim = problem.dim
    d.nel[0], d.nel[1] = problem.nel[0], problem.nel[1]
    d.nel[2] = problem.nel[2] if problem.dim == 3 else 1
    d.nu, d.E0, d.Emin, d.penal = problem.nu, problem.E0, problem.Emin, problem.penal
    d.mg_levels, d.eig_level, d.num_modes = problem.mg_levels, problem.eig_level, problem.num_modes
    for k, v in overrides.items():
        setattr(d, k, v)
    return d


class Batch:
    """Owner of a tobk_batch: many independent 2D designs solved together (tobk_batch_* calls).
    Packed arrays follow `layout()`; arrays may be numpy (host) or torch tensors (host or device)."""

    def __init__(self, problems, nrhs, *, stream=None, **overrides):
        self.lib = load()
        n = len(problems)
        descs = (tobk_desc * n)()
        for i, p in enumerate(problems):
            descs[i] = problem_desc(self.lib, p, **overrides)
        h = _H()
        s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = self.lib.tobk_batch_create(descs, n, nrhs, C.c_void_p(s), C.byref(h))
        if rc != TOBK_OK:
            raise TobkError(rc, "tobk_batch_create failed")
        self.h = h
        self.nd = n
        self.nrhs = nrhs
        dof = (C.c_int64 * (n + 1))()
        elem = (C.c_int64 * (n + 1))()
        self.lib.tobk_batch_layout(self.h, dof, elem)
        self.dof_offsets = np.array(dof[:], dtype=np.int64)
        self.elem_offsets = np.array(elem[:], dtype=np.int64)

    def close(self):
        if getattr(self, "h", None):
            self.lib.tobk_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != TOBK_OK and rc not in allow:
            raise TobkError(rc, self.lib.tobk_batch_last_error(self.h).decode())
        return rc

    def set_designs(self, x, fixed):
        px, dx = _ptr(x)
        pf, df = _ptr(fixed)
        assert dx == df
        self._check(self.lib.tobk_batch_set_designs(self.h, px, pf, dx))

    def solve(self, B, X, allow_not_converged=False):
        pb, db = _ptr(B)
        px, dx = _ptr(X)
        assert db == dx
        infos = (tobk_solve_info * self.nd)()
        rc = self._check(self.lib.tobk_batch_solve(self.h, pb, px, db, infos),
                         (TOBK_E_NOT_CONVERGED,) if allow_not_converged else ())
        return [i.as_dict() for i in infos], rc

    def autotune(self):
        f, c = C.c_int(), C.c_int()
        self._check(self.lib.tobk_batch_autotune(self.h, C.byref(f), C.byref(c)))
        return f.value, c.value

    def set_variants(self, fine, coarse):
        self._check(self.lib.tobk_batch_set_variants(self.h, fine, coarse))


class tobk_unet_desc(C.Structure):
    _fields_ = [("nel", C.c_int * 3), ("levels", C.c_int), ("channels", C.c_int * 4), ("in_channels", C.c_int),
                ("out_channels", C.c_int), ("penal", C.c_double), ("E0", C.c_double), ("Emin", C.c_double),
                ("nu", C.c_double), ("loss", C.c_int), ("seed", C.c_ulonglong)]


TOBK_UNET_LOSS_MSE, TOBK_UNET_LOSS_ENERGY = 0, 1


class UNet:
    """Owner of a tobk_unet (the learned warm start): device tensors in, device tensors out."""

    def __init__(self, nel=(128, 64, 64), levels=4, channels=(16, 32, 64, 64), seed=1234, *, stream=None,
                 penal=3.0, E0=1.0, Emin=1e-6, nu=0.3, loss=TOBK_UNET_LOSS_ENERGY):
        self.lib = load()
        d = tobk_unet_desc()
        self.lib.tobk_unet_default_desc(C.byref(d))
        for a in range(3):
            d.nel[a] = nel[a]
        d.levels = levels
        for l in range(4):
            d.channels[l] = channels[l] if l < levels else 0
        d.penal, d.E0, d.Emin, d.seed, d.nu, d.loss = penal, E0, Emin, seed, nu, loss
        h = _H()
        s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = self.lib.tobk_unet_create(C.byref(d), C.c_void_p(s), C.byref(h))
        if rc != TOBK_OK:
            raise TobkError(rc, "tobk_unet_create failed")
        self.h = h
        self.stream = stream
        self.nel, self.levels, self.channels = tuple(nel), levels, tuple(channels[:levels])
        self.num_params = int(self.lib.tobk_unet_num_params(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.tobk_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != TOBK_OK:
            raise TobkError(rc, self.lib.tobk_unet_last_error(self.h).decode())

    def set_output_scale(self, c):
        self._check(self.lib.tobk_unet_set_output_scale(self.h, float(c)))

    def output_scale(self):
        return float(self.lib.tobk_unet_output_scale(self.h))

    def design_scale(self, x, f):
        s = C.c_double()
        self._check(self.lib.tobk_unet_design_scale(self.h, x.data_ptr(), f.data_ptr(), C.byref(s)))
        return s.value

    def _check_state_arrays(self, *arrays):
        for a in arrays:
            if a is None:
                continue
            n = a.numel() if hasattr(a, "numel") else a.size
            dt = str(a.dtype)
            if n != self.num_params or "float32" not in dt:
                raise ValueError(f"network state arrays must be float32 of length {self.num_params}, got {dt} of {n}")

    def get_state(self, params, m=None, v=None):
        self._check_state_arrays(params, m, v)
        step = C.c_longlong()
        pp, dev = _ptr(params)
        self._check(self.lib.tobk_unet_get_state(self.h, pp, _ptr(m)[0] if m is not None else None,
                                                 _ptr(v)[0] if v is not None else None, C.byref(step), dev))
        return step.value

    def set_state(self, params, m=None, v=None, step=0):
        self._check_state_arrays(params, m, v)
        pp, dev = _ptr(params)
        self._check(self.lib.tobk_unet_set_state(self.h, pp, _ptr(m)[0] if m is not None else None,
                                                 _ptr(v)[0] if v is not None else None, step, dev))

    def set_tensor_cores(self, mode=1):
        """Inference convolutions: 0 / False the FP32 direct convolution, 1 / True the tensor cores on
        large levels (default), 2 the tensor cores on every level."""
        self._check(self.lib.tobk_unet_set_tensor_cores(self.h, int(mode)))

    def predict(self, x, f, fixed, u0):
        self._check(self.lib.tobk_unet_predict(self.h, x.data_ptr(), f.data_ptr(), fixed.data_ptr(), u0.data_ptr()))

    def loss_grad(self, x, f, target, fixed, grad=None):
        loss = C.c_float()
        self._check(self.lib.tobk_unet_loss_grad(self.h, x.data_ptr(), f.data_ptr(), target.data_ptr(),
                                                 fixed.data_ptr(), C.byref(loss),
                                                 grad.data_ptr() if grad is not None else None))
        return loss.value

    def train_step(self, x, f, target, fixed, nbatch, lr):
        loss = C.c_float()
        self._check(self.lib.tobk_unet_train_step(self.h, x.data_ptr(), f.data_ptr(), target.data_ptr(),
                                                  fixed.data_ptr(), nbatch, lr, C.byref(loss)))
        return loss.value


def conv3_bf16(inp, weight, bias, out, relu=True, stream=None):
    """One 3x3x3 convolution on the tensor cores (tobk_conv3_bf16): inp [Cin][D][H][W], weight
    [Cout][Cin][27], bias [Cout] (or None), out [Cout][D][H][W]; FP32 CUDA tensors."""
    lib = load()
    cin, D, H, W = inp.shape
    cout = weight.shape[0]
    s = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib.tobk_conv3_bf16(inp.data_ptr(), cin, D, H, W, weight.data_ptr(),
                             bias.data_ptr() if bias is not None else None, cout, 1 if relu else 0, out.data_ptr(),
                             C.c_void_p(s))
    if rc != TOBK_OK:
        raise TobkError(rc, "tobk_conv3_bf16 failed")
