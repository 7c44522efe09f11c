"""Thin ctypes binding of liblskum (include/lskum.h): argument marshalling only.

Every step of an iteration runs in the library's CUDA kernels.  The binding
fails loudly when the compiled library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

INTERIOR, WALL, OUTER = 0, 1, 2
JVP_EXACT, JVP_INCREMENT = 0, 1
SCHEME_LUSGS, SCHEME_EXPLICIT = 0, 1
LUSGS_ANANDH, LUSGS_MANISH = 0, 1
ORDER_COLOUR, ORDER_WALL_FIRST, ORDER_SERIAL = 0, 1, 2
FARFIELD_FREESTREAM, FARFIELD_KINETIC = 0, 1
FIELD_U, FIELD_Q, FIELD_QX, FIELD_QY, FIELD_R, FIELD_D, FIELD_DUS, FIELD_DU = range(8)
OK, ERR_ARG, ERR_STENCIL, ERR_NONPOSITIVE, ERR_DIVERGED, ERR_CUDA, ERR_TIMEOUT, ERR_OOM = 0, -1, -2, -3, -4, -5, -6, -7
STATUS = {0: "LSKUM_OK", -1: "LSKUM_ERR_ARG", -2: "LSKUM_ERR_STENCIL", -3: "LSKUM_ERR_NONPOSITIVE",
          -4: "LSKUM_ERR_DIVERGED", -5: "LSKUM_ERR_CUDA", -6: "LSKUM_ERR_TIMEOUT", -7: "LSKUM_ERR_OOM"}


class LskumError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lskum_cloud(C.Structure):
    _fields_ = [("n_points", C.c_int32), ("x", C.c_void_p), ("y", C.c_void_p), ("flag", C.c_void_p),
                ("nx", C.c_void_p), ("ny", C.c_void_p), ("nbr_off", C.c_void_p), ("nbr_idx", C.c_void_p)]


class lskum_opts(C.Structure):
    _fields_ = [("mach", C.c_double), ("aoa_deg", C.c_double), ("cfl", C.c_double), ("cfl_ramp_iters", C.c_double),
                ("inner_iters", C.c_int32), ("jvp", C.c_int32), ("precision", C.c_int32),
                ("first_order_iters", C.c_int32), ("scheme", C.c_int32), ("lusgs", C.c_int32),
                ("ordering", C.c_int32), ("farfield", C.c_int32)]


_lib = None


def load():
    """Load liblskum.so (built by ``python -m paper_2406_07441_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"liblskum is not built ({LIB} missing): run python -m paper_2406_07441_gb300.build")
    L = C.CDLL(LIB)
    vp, i32, d, st = C.c_void_p, C.c_int32, C.c_double, C.c_int
    P = C.POINTER
    L.lskum_create.argtypes = [P(lskum_cloud), P(lskum_opts), vp, P(vp)]
    L.lskum_set_state.argtypes = [vp, vp, vp, vp, vp]
    L.lskum_set_conserved.argtypes = [vp, vp]
    L.lskum_run.argtypes = [vp, i32, d, P(i32)]
    L.lskum_enqueue.argtypes = [vp, i32, d]
    L.lskum_wait.argtypes = [vp, P(i32)]
    L.lskum_stream.argtypes = [vp]
    L.lskum_stream.restype = vp
    L.lskum_get_state.argtypes = [vp, vp, vp, vp, vp]
    L.lskum_get_field.argtypes = [vp, i32, vp]
    L.lskum_get_residuals.argtypes = [vp, vp, i32, P(i32)]
    L.lskum_get_forces.argtypes = [vp, P(d), P(d)]
    L.lskum_get_order.argtypes = [vp, vp, vp, P(i32)]
    L.lskum_get_info.argtypes = [vp, P(i32), P(i32), P(i32)]
    L.lskum_time_phases.argtypes = [vp, i32, vp]
    L.lskum_autotune.argtypes = [vp, i32, P(i32), P(i32), P(d)]
    L.lskum_density_norm_noalloc.argtypes = [vp, i32, vp, vp]
    L.lskum_selftest_fpint.argtypes = [i32, vp, vp, vp, i32]
    L.lskum_batch_create.argtypes = [P(lskum_cloud), P(lskum_opts), i32, vp, P(vp)]
    L.lskum_get_case_residuals.argtypes = [vp, i32, vp, i32, P(i32)]
    L.lskum_get_case_residuals4.argtypes = [vp, i32, vp, i32, P(i32)]
    L.lskum_get_case_forces.argtypes = [vp, i32, P(d), P(d)]
    L.lskum_get_case_info.argtypes = [vp, i32, P(i32), P(i32), P(i32), P(i32), P(i32), P(i32)]
    L.lskum_get_wall_distance.argtypes = [vp, vp]
    L.lskum_validate.argtypes = [P(lskum_cloud), P(lskum_opts), i32, P(i32), P(i32)]
    L.lskum_get_field_dev.argtypes = [vp, i32, vp, vp]
    L.lskum_set_conserved_dev.argtypes = [vp, vp, vp]
    L.lskum_set_host_io.argtypes = [vp, i32]
    L.lskum_get_host_io.argtypes = [vp, vp, vp]
    L.lskum_set_start_iters.argtypes = [vp, i32]
    L.lskum_set_launch_shape.argtypes = [vp, i32, i32]
    u64 = C.c_uint64
    L.lskum_mlp_n_params.argtypes = []
    L.lskum_mlp_n_params.restype = i32
    L.lskum_mlp_create.argtypes = [u64, i32, vp, P(vp)]
    L.lskum_mlp_get_params.argtypes = [vp, vp, vp]
    L.lskum_mlp_set_params.argtypes = [vp, vp, vp]
    L.lskum_mlp_features.argtypes = [vp, vp, i32, vp]
    L.lskum_mlp_forward.argtypes = [vp, vp, i32, vp]
    L.lskum_mlp_loss_grads.argtypes = [vp, vp, vp, i32, P(C.c_float), vp]
    L.lskum_mlp_adam.argtypes = [vp, vp, C.c_float]
    L.lskum_mlp_add_samples.argtypes = [vp, vp, i32, u64]
    L.lskum_mlp_time_forward.argtypes = [vp, i32, i32, P(d)]
    L.lskum_mlp_n_samples.argtypes = [vp, P(i32)]
    L.lskum_mlp_train.argtypes = [vp, i32, i32, C.c_float, u64, vp]
    L.lskum_mlp_predict.argtypes = [vp, vp, vp]
    L.lskum_mlp_set_wait_test.argtypes = [vp, i32, d]
    L.lskum_mlp_last_error.argtypes = [vp]
    L.lskum_mlp_last_error.restype = C.c_char_p
    L.lskum_mlp_destroy.argtypes = [vp]
    L.lskum_mlp_destroy.restype = None
    L.lskum_last_error.argtypes = [vp]
    L.lskum_last_error.restype = C.c_char_p
    L.lskum_destroy.argtypes = [vp]
    L.lskum_destroy.restype = None
    for f in ("lskum_create", "lskum_set_state", "lskum_set_conserved", "lskum_run", "lskum_enqueue", "lskum_wait",
              "lskum_get_state", "lskum_get_field", "lskum_get_residuals", "lskum_get_forces", "lskum_get_order",
              "lskum_get_info", "lskum_time_phases", "lskum_density_norm_noalloc", "lskum_selftest_fpint",
              "lskum_batch_create",
              "lskum_get_case_residuals", "lskum_get_case_residuals4", "lskum_get_case_forces", "lskum_get_case_info", "lskum_autotune",
              "lskum_get_wall_distance", "lskum_validate", "lskum_set_start_iters", "lskum_get_field_dev", "lskum_set_conserved_dev", "lskum_set_launch_shape",
              "lskum_set_host_io", "lskum_get_host_io", "lskum_mlp_create", "lskum_mlp_get_params",
              "lskum_mlp_set_params", "lskum_mlp_features", "lskum_mlp_forward", "lskum_mlp_loss_grads",
              "lskum_mlp_adam", "lskum_mlp_add_samples", "lskum_mlp_time_forward", "lskum_mlp_n_samples", "lskum_mlp_train",
              "lskum_mlp_predict", "lskum_mlp_set_wait_test"):
        getattr(L, f).restype = st
    _lib = L
    return L


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _cloud_struct(cloud, keep):
    """The C view of a cloud; nx / ny may be None (the library then computes
    the normals from the wall and outer polygons)."""
    arrs = [np.ascontiguousarray(cloud.x, np.float64), np.ascontiguousarray(cloud.y, np.float64),
            np.ascontiguousarray(cloud.flag, np.uint8),
            None if cloud.nx is None else np.ascontiguousarray(cloud.nx, np.float64),
            None if cloud.ny is None else np.ascontiguousarray(cloud.ny, np.float64),
            np.ascontiguousarray(cloud.nbr_off, np.int32), np.ascontiguousarray(cloud.nbr_idx, np.int32)]
    keep.extend(a for a in arrs if a is not None)
    return lskum_cloud(int(len(cloud.x)), *[None if a is None else a.ctypes.data for a in arrs])


FPINT_MUL, FPINT_EXP, FPINT_ERFCX_HALF, FPINT_MUL_FP64 = 0, 1, 2, 3


def selftest_fpint(op, a, b=None):
    """The kernels' integer-pipe FP64 arithmetic evaluated on the device
    (include/lskum.h, lskum_selftest_fpint): op FPINT_MUL a*b (integer
    multiply), FPINT_EXP exp(a), FPINT_ERFCX_HALF erfcx(min(|a|, 9))/2,
    FPINT_MUL_FP64 a*b on the FP64 unit."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty_like(a)
    s = load().lskum_selftest_fpint(int(op), _p(a), None if bb is None else _p(bb), _p(out), int(a.size))
    if s != 0:
        raise LskumError(s, f"lskum_selftest_fpint: status {s}")
    return out


def validate(clouds, conditions, **kw):
    """Host-only dry run of create (see lskum_validate): returns (n_colours,
    n_levels) or raises LskumError; no GPU is needed."""
    L = load()
    keep = []
    cl = (lskum_cloud * len(clouds))(*[_cloud_struct(c, keep) for c in clouds])
    o = dict(cfl=100.0, cfl_ramp_iters=0.0, inner_iters=3, jvp=JVP_EXACT, precision=0, first_order_iters=0,
             scheme=SCHEME_LUSGS, lusgs=LUSGS_ANANDH, ordering=ORDER_COLOUR, farfield=FARFIELD_FREESTREAM)
    o.update(kw)
    op = (lskum_opts * len(clouds))(*[lskum_opts(m, a, o["cfl"], o["cfl_ramp_iters"], o["inner_iters"], o["jvp"],
                                                 o["precision"], o["first_order_iters"], o["scheme"], o["lusgs"],
                                                 o["ordering"], o["farfield"]) for m, a in conditions])
    nc, nl = C.c_int32(), C.c_int32()
    s = L.lskum_validate(cl, op, len(clouds), C.byref(nc), C.byref(nl))
    if s != 0:
        raise LskumError(s, L.lskum_last_error(None).decode())
    return nc.value, nl.value


class Solver:
    """One context of liblskum for one cloud and one flow condition.

    ``Solver.batch(clouds, conditions, ...)`` builds one context that solves
    several (cloud, (mach, aoa_deg)) cases together."""

    def __init__(self, cloud, mach, aoa_deg, cfl=100.0, inner_iters=3, jvp=JVP_EXACT, cfl_ramp_iters=0.0,
                 first_order_iters=0, precision=0, scheme=SCHEME_LUSGS, lusgs=LUSGS_ANANDH,
                 ordering=ORDER_COLOUR, farfield=FARFIELD_FREESTREAM, stream=None, _cases=None):
        L = load()
        keep = []
        clouds = _cases[0] if _cases else [cloud]
        conds = _cases[1] if _cases else [(mach, aoa_deg)]
        if len(clouds) != len(conds) or not clouds:
            raise ValueError("one (mach, aoa_deg) per cloud")
        cl = (lskum_cloud * len(clouds))(*[_cloud_struct(c, keep) for c in clouds])
        op = (lskum_opts * len(clouds))(*[lskum_opts(m, a, cfl, cfl_ramp_iters, inner_iters, jvp, precision,
                                                     first_order_iters, scheme, lusgs, ordering, farfield)
                                          for m, a in conds])
        h = C.c_void_p()
        if _cases:
            s = L.lskum_batch_create(cl, op, len(clouds), C.c_void_p(stream), C.byref(h))
        else:
            s = L.lskum_create(cl, op, C.c_void_p(stream), C.byref(h))
        if s != 0:
            raise LskumError(s, L.lskum_last_error(None).decode())
        self._h = h
        self.n = int(sum(c.n for c in clouds))
        self.n_cases = len(clouds)
        self.conditions = list(conds)
        self.mach, self.aoa_deg = conds[0]

    @classmethod
    def batch(cls, clouds, conditions, **kw):
        return cls(None, None, None, _cases=(list(clouds), list(conditions)), **kw)

    def case_residuals(self, cs):
        n = C.c_int32(0)
        self._check(load().lskum_get_case_residuals(self._h, int(cs), None, 0, C.byref(n)))
        h = np.empty(max(n.value, 1))
        self._check(load().lskum_get_case_residuals(self._h, int(cs), _p(h), n.value, C.byref(n)))
        return h[:n.value]

    def case_residuals4(self, cs):
        """[n][4] norms of the four residual components per iteration (column 0: density)."""
        n = C.c_int32(0)
        self._check(load().lskum_get_case_residuals4(self._h, int(cs), None, 0, C.byref(n)))
        h = np.empty((max(n.value, 1), 4))
        self._check(load().lskum_get_case_residuals4(self._h, int(cs), _p(h), n.value, C.byref(n)))
        return h[:n.value]

    def residuals4(self):
        return self.case_residuals4(0)

    def case_forces(self, cs):
        cl, cd = C.c_double(), C.c_double()
        self._check(load().lskum_get_case_forces(self._h, int(cs), C.byref(cl), C.byref(cd)))
        return cl.value, cd.value

    def case_info(self, cs):
        a, b, c, d, e, f = (C.c_int32() for _ in range(6))
        self._check(load().lskum_get_case_info(self._h, int(cs), C.byref(a), C.byref(b), C.byref(c), C.byref(d),
                                               C.byref(e), C.byref(f)))
        return dict(first_point=a.value, n_points=b.value, iters=c.value, stopped=bool(d.value), status=e.value,
                    bad_point=f.value)

    def _check(self, s):
        if s != 0:
            raise LskumError(s, load().lskum_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().lskum_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- state ---
    def set_state(self, rho, u, v, p):
        a = [np.ascontiguousarray(t, np.float64) for t in (rho, u, v, p)]
        self._check(load().lskum_set_state(self._h, *[_p(t) for t in a]))

    def set_conserved(self, U):
        U = np.ascontiguousarray(U, np.float64).reshape(self.n, 4)
        self._check(load().lskum_set_conserved(self._h, _p(U)))

    def field_dev(self, which, out_ptr, stream=None):
        """Copy a field into device memory at out_ptr (caller order), ordered on `stream`."""
        self._check(load().lskum_get_field_dev(self._h, int(which), C.c_void_p(out_ptr), C.c_void_p(stream)))

    def set_conserved_dev(self, U_ptr, stream=None):
        """Set the conserved state from device memory at U_ptr ([N][4], caller order)."""
        self._check(load().lskum_set_conserved_dev(self._h, C.c_void_p(U_ptr), C.c_void_p(stream)))

    def get_state(self):
        out = [np.empty(self.n) for _ in range(4)]
        self._check(load().lskum_get_state(self._h, *[_p(t) for t in out]))
        return tuple(out)

    def field(self, which):
        out = np.empty(self.n if which == FIELD_D else (self.n, 4))
        self._check(load().lskum_get_field(self._h, int(which), _p(out)))
        return out

    # --- iterations ---
    def run(self, max_iters, target_drop=0.0, check=True):
        done = C.c_int32(0)
        s = load().lskum_run(self._h, int(max_iters), float(target_drop), C.byref(done))
        if check:
            self._check(s)
        return done.value if check else (s, done.value)

    def enqueue(self, max_iters, target_drop=0.0):
        self._check(load().lskum_enqueue(self._h, int(max_iters), float(target_drop)))

    def wait(self):
        done = C.c_int32(0)
        self._check(load().lskum_wait(self._h, C.byref(done)))
        return done.value

    def stream(self):
        return load().lskum_stream(self._h)

    # --- outputs ---
    def residuals(self):
        n = C.c_int32(0)
        self._check(load().lskum_get_residuals(self._h, None, 0, C.byref(n)))
        h = np.empty(max(n.value, 1))
        self._check(load().lskum_get_residuals(self._h, _p(h), n.value, C.byref(n)))
        return h[:n.value]

    def forces(self):
        cl, cd = C.c_double(), C.c_double()
        self._check(load().lskum_get_forces(self._h, C.byref(cl), C.byref(cd)))
        return cl.value, cd.value

    def order(self):
        col = np.empty(self.n, np.int32)
        order = np.empty(self.n, np.int32)
        nc = C.c_int32(0)
        self._check(load().lskum_get_order(self._h, _p(col), _p(order), C.byref(nc)))
        return col, order, nc.value

    PHASES = ("grad", "residual", "norm", "sweep_fwd", "sweep_bwd", "update")

    def time_phases(self, reps):
        """Mean device ms per iteration of each phase (CUDA events, library stream)."""
        ms = np.zeros(6)
        self._check(load().lskum_time_phases(self._h, int(reps), _p(ms)))
        return dict(zip(self.PHASES, ms.tolist()))

    def autotune(self, trial_iters=5):
        """Pick the fastest launch shape by timing real iterations; the state
        and histories are restored.  Returns (threads per point, sweep lanes
        per point, ms per iteration)."""
        a, b, t = C.c_int32(), C.c_int32(), C.c_double()
        self._check(load().lskum_autotune(self._h, int(trial_iters), C.byref(a), C.byref(b), C.byref(t)))
        return a.value, b.value, t.value

    def wall_distance(self):
        """Distance of every point to its case's wall polygon (as the warm-start network sees it)."""
        d = np.empty(self.n)
        self._check(load().lskum_get_wall_distance(self._h, _p(d)))
        return d

    def set_launch_shape(self, tpp, sweep_lanes):
        self._check(load().lskum_set_launch_shape(self._h, int(tpp), int(sweep_lanes)))

    def set_host_io(self, direct):
        """1: host arrays straight to / from the device's reorder kernels
        (where the device reads pageable host memory); 0: staging copies."""
        self._check(load().lskum_set_host_io(self._h, int(direct)))

    def host_io(self):
        """(direct in use, direct supported)."""
        a, b = C.c_int32(), C.c_int32()
        self._check(load().lskum_get_host_io(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_start_iters(self, first_order_iters):
        self._check(load().lskum_set_start_iters(self._h, int(first_order_iters)))

    def info(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(load().lskum_get_info(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return dict(n_points=a.value, n_colours=b.value, launches_per_iter=c.value)


class Mlp:
    """The warm-start network (include/lskum_mlp.h): BF16 tensor-core
    training and inference kernels with FP32 accumulation."""

    def __init__(self, seed=0, max_batch=65536, stream=None):
        L = load()
        h = C.c_void_p()
        s = L.lskum_mlp_create(C.c_uint64(seed), int(max_batch), C.c_void_p(stream), C.byref(h))
        if s != 0:
            raise LskumError(s, L.lskum_mlp_last_error(None).decode())
        self._h = h
        self.n_params = int(L.lskum_mlp_n_params())

    def _check(self, s):
        if s != 0:
            raise LskumError(s, load().lskum_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().lskum_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.empty(self.n_params, np.float32)
        B = np.empty(48, np.float32)
        self._check(load().lskum_mlp_get_params(self._h, _p(p), _p(B)))
        return p, B.reshape(16, 3)

    def set_params(self, params, fourier=None):
        p = np.ascontiguousarray(params, np.float32)
        B = None if fourier is None else np.ascontiguousarray(fourier, np.float32).reshape(48)
        self._check(load().lskum_mlp_set_params(self._h, _p(p), None if B is None else _p(B)))

    def features(self, in5):
        a = np.ascontiguousarray(in5, np.float32).reshape(-1, 5)
        X = np.empty((a.shape[0], 34), np.float32)
        self._check(load().lskum_mlp_features(self._h, _p(a), a.shape[0], _p(X)))
        return X

    def forward(self, X):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, 34)
        out = np.empty((X.shape[0], 4), np.float32)
        self._check(load().lskum_mlp_forward(self._h, _p(X), X.shape[0], _p(out)))
        return out

    def loss_grads(self, X, T):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, 34)
        T = np.ascontiguousarray(T, np.float32).reshape(-1, 4)
        g = np.empty(self.n_params, np.float32)
        loss = C.c_float()
        self._check(load().lskum_mlp_loss_grads(self._h, _p(X), _p(T), X.shape[0], C.byref(loss), _p(g)))
        return loss.value, g

    def adam(self, grads, lr):
        g = np.ascontiguousarray(grads, np.float32)
        self._check(load().lskum_mlp_adam(self._h, _p(g), C.c_float(lr)))

    def time_forward(self, n, reps=10):
        """Mean device ms of the forward pass over n points."""
        ms = C.c_double()
        self._check(load().lskum_mlp_time_forward(self._h, int(n), int(reps), C.byref(ms)))
        return ms.value

    def add_samples(self, solver, per_case, seed=0):
        self._check(load().lskum_mlp_add_samples(self._h, solver._h, int(per_case), C.c_uint64(seed)))

    def n_samples(self):
        n = C.c_int32()
        self._check(load().lskum_mlp_n_samples(self._h, C.byref(n)))
        return n.value

    def train(self, epochs, batch, lr, seed=0):
        losses = np.zeros(max(int(epochs), 1), np.float32)
        self._check(load().lskum_mlp_train(self._h, int(epochs), int(batch), C.c_float(lr), C.c_uint64(seed),
                                           _p(losses)))
        return losses[:int(epochs)]

    def set_wait_test(self, skip_products, wait_limit_s=1.0):
        """Failure-path test of the bounded tensor-core waits (see lskum_mlp_set_wait_test)."""
        self._check(load().lskum_mlp_set_wait_test(self._h, int(skip_products), float(wait_limit_s)))

    def predict(self, solver):
        """Warm-start the solver's state; returns per case whether the prediction was kept."""
        warm = np.zeros(solver.n_cases, np.int32)
        self._check(load().lskum_mlp_predict(self._h, solver._h, _p(warm)))
        return warm.astype(bool)


def unflatten_params(p):
    """Parameter vector -> [(W_l [out, in], b_l [out])] of the 34-128-128-128-128-4 network."""
    dims = [(34, 128), (128, 128), (128, 128), (128, 128), (128, 4)]
    out, o = [], 0
    for fin, fout in dims:
        W = np.asarray(p[o:o + fin * fout]).reshape(fout, fin)
        o += fin * fout
        b = np.asarray(p[o:o + fout])
        o += fout
        out.append((W, b))
    return out
