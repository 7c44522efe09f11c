"""ctypes binding of the plain FP64 CPU oracle (``lskum_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path never
does.  ``build()`` compiles the C source with gcc (-O2, no fused multiply-add,
no fast-math) next to this file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lskum_oracle.c")
LIB = os.path.join(HERE, "liblskum_oracle.so")

JVP_EXACT, JVP_INCREMENT = 0, 1
FARFIELD_FREESTREAM, FARFIELD_KINETIC = 0, 1
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Cloud(C.Structure):
    _fields_ = [("n", C.c_int32), ("x", C.c_void_p), ("y", C.c_void_p), ("flag", C.c_void_p),
                ("nx", C.c_void_p), ("ny", C.c_void_p), ("off", C.c_void_p), ("idx", C.c_void_p),
                ("farfield", C.c_int32), ("uinf", C.c_double * 4)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        d, i32, vp = C.c_double, C.c_int32, C.c_void_p
        P = C.POINTER
        L.o_prim_to_cons.argtypes = [d, d, d, d, vp]
        L.o_cons_to_prim.argtypes = [vp, P(d), P(d), P(d), P(d)]
        L.o_prim_to_q.argtypes = [d, d, d, d, vp]
        L.o_q_to_prim.argtypes = [vp, P(d), P(d), P(d), P(d), P(d)]
        L.o_euler_flux.argtypes = [d, d, d, d, d, d, vp]
        L.o_split_flux.argtypes = [d, d, d, d, d, d, d, C.c_int, vp]
        L.o_split_flux_cons.argtypes = [vp, d, d, C.c_int, vp]
        L.o_split_jvp_exact.argtypes = [vp, vp, d, d, C.c_int, vp]
        L.o_split_jvp_increment.argtypes = [vp, vp, d, d, C.c_int, vp]
        L.o_color_order.argtypes = [i32, vp, vp, vp, vp, vp]
        L.o_color_order.restype = C.c_int
        L.o_q_gradients.argtypes = [P(_Cloud), vp, C.c_int, vp, vp]
        L.o_q_gradient_pass.argtypes = [P(_Cloud), vp, vp, vp, vp, vp]
        L.o_residual.argtypes = [P(_Cloud), vp, vp, vp, vp, d, vp, vp]
        L.o_sweeps.argtypes = [P(_Cloud), vp, vp, vp, vp, vp, C.c_int, vp, vp]
        L.o_update.argtypes = [P(_Cloud), vp, vp, vp]
        L.o_update.restype = i32
        L.o_residual_norm.argtypes = [P(_Cloud), vp]
        L.o_residual_norm.restype = d
        L.o_forces.argtypes = [P(_Cloud), vp, d, d, P(d), P(d)]
        L.o_freestream.argtypes = [d, d, vp]
        L.o_initial_state.argtypes = [P(_Cloud), d, d, vp]
        L.o_q_from_state.argtypes = [P(_Cloud), vp, vp]
        L.o_cfl_at.argtypes = [d, d, i32]
        L.o_cfl_at.restype = d
        L.o_run.argtypes = [P(_Cloud), vp, vp, d, d, i32, i32, i32, i32, d, i32,
                            vp, vp, vp, vp, vp, vp, vp, vp, vp, P(d), P(i32)]
        L.o_run.restype = i32
        L.o_explicit_step.argtypes = [P(_Cloud), vp, d, vp, vp, vp]
        L.o_manish_terms.argtypes = [P(_Cloud), vp, d, vp, vp, vp]
        L.o_run_manish.argtypes = [P(_Cloud), vp, vp, d, d, i32, i32, i32, i32, i32, d, i32,
                                   vp, vp, vp, vp, vp, vp, vp, vp, vp, P(d), P(i32)]
        L.o_run_manish.restype = i32
        L.o_run_explicit.argtypes = [P(_Cloud), d, d, i32, i32, i32, d, i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                     P(d), P(i32)]
        L.o_run_explicit.restype = i32
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------------------
# point-wise functions
# ---------------------------------------------------------------------------

def prim_to_cons(rho, u, v, p):
    U = np.zeros(4)
    lib().o_prim_to_cons(rho, u, v, p, _p(U))
    return U


def cons_to_prim(U):
    U = _f64(U)
    r, u, v, p = (C.c_double() for _ in range(4))
    lib().o_cons_to_prim(_p(U), C.byref(r), C.byref(u), C.byref(v), C.byref(p))
    return r.value, u.value, v.value, p.value


def prim_to_q(rho, u, v, p):
    q = np.zeros(4)
    lib().o_prim_to_q(rho, u, v, p, _p(q))
    return q


def q_to_prim(q):
    q = _f64(q)
    out = [C.c_double() for _ in range(5)]
    lib().o_q_to_prim(_p(q), *[C.byref(o) for o in out])
    return tuple(o.value for o in out)  # rho, u, v, p, beta


def euler_flux(rho, u, v, p, dx, dy):
    G = np.zeros(4)
    lib().o_euler_flux(rho, u, v, p, dx, dy, _p(G))
    return G


def split_flux(rho, u, v, p, dx, dy, sign, beta=None):
    if beta is None:
        beta = rho / (2.0 * p)
    G = np.zeros(4)
    lib().o_split_flux(rho, u, v, p, beta, dx, dy, int(sign), _p(G))
    return G


def split_flux_cons(U, dx, dy, sign):
    U = _f64(U)
    G = np.zeros(4)
    lib().o_split_flux_cons(_p(U), dx, dy, int(sign), _p(G))
    return G


def split_jvp(U, dU, dx, dy, sign, mode=JVP_EXACT):
    U = _f64(U)
    dU = _f64(dU)
    out = np.zeros(4)
    f = lib().o_split_jvp_exact if mode == JVP_EXACT else lib().o_split_jvp_increment
    f(_p(U), _p(dU), dx, dy, int(sign), _p(out))
    return out


def freestream(mach, aoa_deg):
    U = np.zeros(4)
    lib().o_freestream(mach, aoa_deg, _p(U))
    return U


# ---------------------------------------------------------------------------
# cloud-wide steps
# ---------------------------------------------------------------------------

class Oracle:
    """One cloud, the canonical sweep order, and the steps of Alg. 1 on it."""

    def __init__(self, cloud, ordering=0, farfield=FARFIELD_FREESTREAM, mach=0.0, aoa_deg=0.0):
        """ordering 0: the sweep order of Alg. 6 (points stably sorted by
        colour); 1: Alg. 4 (wall points by colour, then interior points by
        colour, then outer points); 2: Alg. 2 (wall, interior and outer
        points, each in index order; no colours).  farfield 0: outer points frozen at the
        free stream; 1: the kinetic far field with the free stream of
        (mach, aoa_deg) and the cloud's outward normals at outer points."""
        self.cloud = cloud
        self.n = cloud.n
        self._keep = [np.ascontiguousarray(cloud.x, np.float64), np.ascontiguousarray(cloud.y, np.float64),
                      np.ascontiguousarray(cloud.flag, np.uint8), np.ascontiguousarray(cloud.nx, np.float64),
                      np.ascontiguousarray(cloud.ny, np.float64), np.ascontiguousarray(cloud.nbr_off, np.int32),
                      np.ascontiguousarray(cloud.nbr_idx, np.int32)]
        k = self._keep
        self.c = _Cloud(self.n, *[a.ctypes.data for a in k])
        self.farfield = int(farfield)
        self.c.farfield = self.farfield
        if self.farfield == FARFIELD_KINETIC:
            for j, v in enumerate(freestream(mach, aoa_deg)):
                self.c.uinf[j] = v
        self.colour = np.zeros(self.n, np.int32)
        self.order = np.zeros(self.n, np.int32)
        self.rank = np.zeros(self.n, np.int32)
        self.ncolours = lib().o_color_order(self.n, _p(k[5]), _p(k[6]), _p(self.colour), _p(self.order),
                                            _p(self.rank))
        group = np.where(cloud.flag == 1, 0, np.where(cloud.flag == 0, 1, 2))
        if ordering == 1:
            key = group.astype(np.int64) * (self.ncolours + 1) + self.colour
            self.order[:] = np.argsort(key, kind="stable").astype(np.int32)
            self.rank[self.order] = np.arange(self.n, dtype=np.int32)
        elif ordering == 2:
            self.order[:] = np.argsort(group, kind="stable").astype(np.int32)
            self.rank[self.order] = np.arange(self.n, dtype=np.int32)

    def initial_state(self, mach, aoa_deg):
        U = np.zeros((self.n, 4))
        lib().o_initial_state(C.byref(self.c), mach, aoa_deg, _p(U))
        return U

    def q_from_state(self, U):
        U = _f64(U, (self.n, 4))
        q = np.zeros((self.n, 4))
        lib().o_q_from_state(C.byref(self.c), _p(U), _p(q))
        return q

    def q_gradients(self, q, K):
        q = _f64(q, (self.n, 4))
        qx = np.zeros((self.n, 4))
        qy = np.zeros((self.n, 4))
        lib().o_q_gradients(C.byref(self.c), _p(q), int(K), _p(qx), _p(qy))
        return qx, qy

    def q_gradient_pass(self, q, px=None, py=None):
        """One pass of Eq. 16 from the previous iterate (px, py); first order if None."""
        q = _f64(q, (self.n, 4))
        qx = np.zeros((self.n, 4))
        qy = np.zeros((self.n, 4))
        if px is None:
            lib().o_q_gradient_pass(C.byref(self.c), _p(q), None, None, _p(qx), _p(qy))
        else:
            px, py = _f64(px, (self.n, 4)), _f64(py, (self.n, 4))
            lib().o_q_gradient_pass(C.byref(self.c), _p(q), _p(px), _p(py), _p(qx), _p(qy))
        return qx, qy

    def residual(self, q, qx, qy, U, cfl):
        q, qx, qy, U = (_f64(a, (self.n, 4)) for a in (q, qx, qy, U))
        R = np.zeros((self.n, 4))
        D = np.zeros(self.n)
        lib().o_residual(C.byref(self.c), _p(q), _p(qx), _p(qy), _p(U), float(cfl), _p(R), _p(D))
        return R, D

    def sweeps(self, U, R, D, jvp=JVP_EXACT):
        U, R = _f64(U, (self.n, 4)), _f64(R, (self.n, 4))
        D = _f64(D)
        dUs = np.zeros((self.n, 4))
        dU = np.zeros((self.n, 4))
        lib().o_sweeps(C.byref(self.c), _p(self.order), _p(self.rank), _p(U), _p(R), _p(D), int(jvp),
                       _p(dUs), _p(dU))
        return dUs, dU

    def update(self, U, dU):
        U = _f64(U, (self.n, 4)).copy()
        dU = _f64(dU, (self.n, 4))
        q = np.zeros((self.n, 4))
        bad = lib().o_update(C.byref(self.c), _p(U), _p(dU), _p(q))
        return U, q, int(bad)

    def residual_norm(self, R):
        R = _f64(R, (self.n, 4))
        return float(lib().o_residual_norm(C.byref(self.c), _p(R)))

    def forces(self, U, mach, aoa_deg):
        U = _f64(U, (self.n, 4))
        cl, cd = C.c_double(), C.c_double()
        lib().o_forces(C.byref(self.c), _p(U), mach, aoa_deg, C.byref(cl), C.byref(cd))
        return cl.value, cd.value

    def explicit_step(self, U, R, cfl):
        """The explicit (forward Euler) increment of the residual R at state U."""
        U = _f64(U, (self.n, 4))
        R = _f64(R, (self.n, 4))
        D = np.zeros(self.n)
        dU = np.zeros((self.n, 4))
        lib().o_explicit_step(C.byref(self.c), _p(U), float(cfl), _p(R), _p(D), _p(dU))
        return dU, D

    def manish_terms(self, U, cfl, dU_prev=None):
        """Diagonal D and lagged term S of the revised LU-SGS of Manish et al."""
        U = _f64(U, (self.n, 4))
        D = np.zeros(self.n)
        S = np.zeros((self.n, 4))
        prev = None if dU_prev is None else _f64(dU_prev, (self.n, 4))
        lib().o_manish_terms(C.byref(self.c), _p(U), float(cfl), None if prev is None else _p(prev), _p(D), _p(S))
        return D, S

    def run_manish(self, U, iters, cfl=100.0, K=3, jvp=JVP_EXACT, sigma=-1, target=0.0, ramp=0.0, n0=0,
                   hist0=0.0, first_order=0):
        """The revised LU-SGS of Manish et al.; as run() otherwise."""
        n = self.n
        U = _f64(U, (n, 4)).copy()
        w = {k: np.zeros((n, 4)) for k in ("q", "qx", "qy", "R", "dUs", "dU")}
        D = np.zeros(n)
        hist = np.zeros(max(1, iters))
        h0 = C.c_double(hist0)
        done = C.c_int32(0)
        st = lib().o_run_manish(C.byref(self.c), _p(self.order), _p(self.rank), float(cfl), float(ramp), int(K),
                                int(jvp), int(first_order), int(sigma), int(iters), float(target), int(n0), _p(U),
                                _p(w["q"]), _p(w["qx"]), _p(w["qy"]), _p(w["R"]), _p(D), _p(w["dUs"]), _p(w["dU"]),
                                _p(hist), C.byref(h0), C.byref(done))
        return dict(U=U, hist=hist[:done.value], hist0=h0.value, done=done.value, status=int(st), D=D, **w)

    def run_explicit(self, U, iters, cfl=0.5, K=3, target=0.0, ramp=0.0, n0=0, hist0=0.0, first_order=0):
        """Explicit solver: as run() with the forward Euler step in place of the sweeps."""
        n = self.n
        U = _f64(U, (n, 4)).copy()
        w = {k: np.zeros((n, 4)) for k in ("q", "qx", "qy", "R", "dU")}
        D = np.zeros(n)
        hist = np.zeros(max(1, iters))
        h0 = C.c_double(hist0)
        done = C.c_int32(0)
        st = lib().o_run_explicit(C.byref(self.c), float(cfl), float(ramp), int(K), int(first_order), int(iters),
                                  float(target), int(n0), _p(U), _p(w["q"]), _p(w["qx"]), _p(w["qy"]), _p(w["R"]),
                                  _p(D), _p(w["dU"]), _p(hist), C.byref(h0), C.byref(done))
        return dict(U=U, hist=hist[:done.value], hist0=h0.value, done=done.value, status=int(st), D=D,
                    dUs=np.zeros((n, 4)), **w)

    def run(self, U, iters, cfl=100.0, K=3, jvp=JVP_EXACT, target=0.0, ramp=0.0, n0=0, hist0=0.0, first_order=0):
        """Alg. 1 for up to `iters` iterations.  Returns a dict with the new state,
        the norm history and the last iteration's intermediates."""
        n = self.n
        U = _f64(U, (n, 4)).copy()
        w = {k: np.zeros((n, 4)) for k in ("q", "qx", "qy", "R", "dUs", "dU")}
        D = np.zeros(n)
        hist = np.zeros(max(1, iters))
        h0 = C.c_double(hist0)
        done = C.c_int32(0)
        st = lib().o_run(C.byref(self.c), _p(self.order), _p(self.rank), float(cfl), float(ramp), int(K), int(jvp),
                         int(first_order), int(iters), float(target), int(n0), _p(U), _p(w["q"]), _p(w["qx"]), _p(w["qy"]),
                         _p(w["R"]), _p(D), _p(w["dUs"]), _p(w["dU"]), _p(hist), C.byref(h0), C.byref(done))
        return dict(U=U, hist=hist[:done.value], hist0=h0.value, done=done.value, status=int(st), D=D, **w)
