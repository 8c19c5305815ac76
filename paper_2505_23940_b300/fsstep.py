"""ctypes binding of the C ABI in include/fs.h (argument marshalling only).

Every step of the solver runs in the CUDA library libfsstep.so; this module
loads it (failing loudly when it is missing), mirrors the C structs, and keeps
torch tensors as the caller-owned device buffers the ABI expects.  torch is
used for device memory and streams only.
"""
import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_void_p

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libfsstep.so")

FS_OK, FS_ERR_ARG, FS_ERR_CUDA, FS_ERR_DIVERGED, FS_ERR_TIMEOUT, FS_ERR_UNSUPPORTED, FS_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6
PERIODIC, NOSLIP, FREESLIP, INFLOW, OUTFLOW = 0, 1, 2, 3, 4
CENTRAL2, UPWIND1 = 0, 1
FE, RK3 = 0, 1
FP64, MIXED = 0, 1
PESKIN4, ROMA3 = 0, 1


class FsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fs error %d: %s" % (code, msg))
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int * 3), ("xf", POINTER(c_double) * 3), ("bc", (c_int * 2) * 3),
                ("bc_val", ((c_double * 3) * 2) * 3), ("nu", c_double), ("rho", c_double),
                ("conv_scheme", c_int), ("time_scheme", c_int), ("precision", c_int),
                ("body_force", POINTER(c_double))]


class State(ctypes.Structure):
    _fields_ = [("u", c_void_p * 3), ("p", c_void_p), ("body", c_void_p)]


class BodyDesc(ctypes.Structure):
    _fields_ = [("nm", c_int), ("X0", POINTER(c_double)), ("Y0", POINTER(c_double)), ("ds", POINTER(c_double)),
                ("centre", c_double * 2), ("omega", c_double), ("mass", c_double), ("stiffness", c_double),
                ("damping", c_double), ("active", c_int * 2), ("delta_kernel", c_int), ("ncontour", c_int),
                ("contour_start", POINTER(c_int))]


class ParamGrad(ctypes.Structure):
    _fields_ = [("body_force", c_void_p), ("stiffness", c_void_p)]


_LIB = None


def lib():
    """Load libfsstep.so once; raise if it has not been built (there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIBPATH):
            raise ImportError("libfsstep.so is not built: run paper_2505_23940_b300/build.py")
        L = ctypes.CDLL(LIBPATH)
        L.fs_create_grid.argtypes = [POINTER(GridDesc), c_void_p, POINTER(c_void_p)]
        L.fs_destroy_grid.argtypes = [c_void_p]
        L.fs_set_stream.argtypes = [c_void_p, c_void_p]
        L.fs_field_extent.argtypes = [c_void_p, c_int, POINTER(c_int)]
        L.fs_set_ib_markers.argtypes = [c_void_p, POINTER(BodyDesc)]
        L.fs_step.argtypes = [c_void_p, POINTER(State), c_double, c_int]
        L.fs_step_record.argtypes = [c_void_p, POINTER(State), c_double, POINTER(c_void_p), POINTER(c_void_p)]
        L.fs_step_adjoint_recorded.argtypes = [c_void_p, POINTER(State), POINTER(c_void_p), POINTER(c_void_p),
                                               POINTER(State), POINTER(ParamGrad), c_double]
        L.fs_step_adjoint.argtypes = [c_void_p, POINTER(State), POINTER(State), POINTER(c_double),
                                      POINTER(ParamGrad), c_double]
        L.fs_ib_face_count.argtypes = [c_void_p, POINTER(c_int)]
        L.fs_step_adjoint_dev.argtypes = [c_void_p, POINTER(State), POINTER(State), c_void_p,
                                          POINTER(ParamGrad), c_double]
        L.fs_solve_pressure.argtypes = [c_void_p, c_void_p, c_void_p]
        L.fs_solve_pressure_cg.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, POINTER(c_int),
                                           POINTER(c_double)]
        L.fs_forces.argtypes = [c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_double)]
        L.fs_diagnostics.argtypes = [c_void_p, POINTER(State), POINTER(c_double)]
        L.fs_kernel_launches.argtypes = [c_void_p]
        L.fs_kernel_launches.restype = c_longlong
        L.fs_last_error.restype = ctypes.c_char_p
        L.fs_profile_begin.argtypes = [c_void_p, ctypes.c_char_p]
        L.fs_profile_end.argtypes = [c_void_p, ctypes.c_char_p, c_int]
        L.fs_set_tuning.argtypes = [c_void_p, ctypes.c_char_p, c_int]
        L.fs_set_body_force.argtypes = [c_void_p, c_void_p]
        L.fs_set_stiffness.argtypes = [c_void_p, c_double]
        L.fs_set_coupling.argtypes = [c_void_p, c_int, c_double]
        L.fs_set_les.argtypes = [c_void_p, c_double]
        L.fs_set_ib_boxes.argtypes = [c_void_p, c_int, POINTER(c_double), c_int, POINTER(c_double), POINTER(c_double),
                                      c_int]
        L.fs_coupling_stats.argtypes = [c_void_p, POINTER(c_int), POINTER(c_double)]
        L.fs_forces_device.argtypes = [c_void_p, c_void_p]
        L.fs_device_status.argtypes = [c_void_p, POINTER(ctypes.c_uint)]
        L.fs_component_stats_noalloc.argtypes = [c_void_p, c_int, POINTER(c_int), c_double, c_void_p, c_void_p,
                                                 c_void_p]
        _LIB = L
    return _LIB


def check(rc):
    if rc != FS_OK:
        raise FsError(rc, lib().fs_last_error().decode())
    return rc


def _dptr(arr):
    import numpy as np
    a = np.ascontiguousarray(arr, dtype=np.float64)
    return a, a.ctypes.data_as(POINTER(c_double))


class Grid:
    """One solver grid on the current CUDA device (wraps fs_grid)."""

    def __init__(self, dim, n, xf, bc, bc_val=None, nu=0.0, rho=1.0, conv=CENTRAL2, scheme=FE,
                 precision=FP64, body_force=None, stream=None):
        L = lib()
        d = GridDesc()
        d.dim = dim
        n = list(n) + [1] * (3 - len(n))
        for i in range(3):
            d.n[i] = int(n[i])
        self._keep = []
        for i in range(dim):
            a, p = _dptr(xf[i])
            self._keep.append(a)
            d.xf[i] = p
        bc = list(bc) + [(PERIODIC, PERIODIC)] * (3 - len(bc))
        for i in range(3):
            for s in range(2):
                d.bc[i][s] = int(bc[i][s])
                vals = (bc_val[i][s] if bc_val is not None and i < len(bc_val) else [0.0, 0.0, 0.0])
                vals = list(vals) + [0.0] * (3 - len(vals))
                for c in range(3):
                    d.bc_val[i][s][c] = float(vals[c])
        d.nu, d.rho = float(nu), float(rho)
        d.conv_scheme, d.time_scheme, d.precision = int(conv), int(scheme), int(precision)
        if body_force is not None:
            a, p = _dptr(body_force)
            self._keep.append(a)
            d.body_force = p
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = c_void_p()
        check(L.fs_create_grid(byref(d), c_void_p(self.stream.cuda_stream), byref(h)))
        self.h = h
        self.dim = dim
        self.n = n
        self.scheme = int(scheme)
        self.has_boxes = False
        self.les_cs = 0.0
        self.precision = precision
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self.has_body = False

    def __del__(self):
        try:
            if getattr(self, "h", None) and _LIB is not None:
                _LIB.fs_destroy_grid(self.h)
                self.h = None
        except Exception:
            pass

    def extent(self, comp):
        e = (c_int * 3)()
        check(lib().fs_field_extent(self.h, comp, e))
        return tuple(e)

    def shape(self, comp):
        ex, ey, ez = self.extent(comp)
        return (ez, ey, ex)

    def zeros(self):
        return [torch.zeros(self.shape(c), dtype=self.dtype, device="cuda") for c in range(self.dim)]

    def set_body(self, X0, Y0, ds, centre, omega=0.0, mass=0.0, stiffness=0.0, damping=0.0,
                 active=(False, False), kernel=ROMA3, contours=None):
        """contours: first marker of each closed contour (several disjoint parts), or None."""
        b = BodyDesc()
        b.nm = len(X0)
        ax, px = _dptr(X0)
        ay, py = _dptr(Y0)
        ad, pd = _dptr(ds)
        b.X0, b.Y0, b.ds = px, py, pd
        b.centre[0], b.centre[1] = float(centre[0]), float(centre[1])
        b.omega, b.mass, b.stiffness, b.damping = float(omega), float(mass), float(stiffness), float(damping)
        b.active[0], b.active[1] = int(bool(active[0])), int(bool(active[1]))
        b.delta_kernel = int(kernel)
        starts = None
        if contours is not None and len(contours) > 1:
            starts = (c_int * len(contours))(*[int(a) for a in contours])
            b.ncontour = len(contours)
            b.contour_start = ctypes.cast(starts, POINTER(c_int))
        check(lib().fs_set_ib_markers(self.h, byref(b)))
        self.has_body = True
        self.nm = b.nm

    def _state(self, u, p=None, body=None):
        s = State()
        for c in range(self.dim):
            assert u[c].is_cuda and u[c].dtype == self.dtype and u[c].is_contiguous()
            assert tuple(u[c].shape) == self.shape(c)
            s.u[c] = u[c].data_ptr()
        s.p = p.data_ptr() if p is not None else None
        s.body = body.data_ptr() if body is not None else None
        return s

    def step(self, u, dt, nsteps=1, p=None, body=None):
        s = self._state(u, p, body)
        check(lib().fs_step(self.h, byref(s), float(dt), int(nsteps)))

    def step_adjoint(self, u_n, lam, dt, body_n=None, lam_body=None, dJdF=None, g_body_force=None,
                     g_stiffness=None):
        sn = self._state(u_n, None, body_n)
        sl = self._state(lam, None, lam_body)
        g = ParamGrad()
        g.body_force = g_body_force.data_ptr() if g_body_force is not None else None
        g.stiffness = g_stiffness.data_ptr() if g_stiffness is not None else None
        if torch.is_tensor(dJdF) and dJdF.is_cuda:
            # device sensitivities (2 contiguous float64 values): no host read
            assert dJdF.dtype == torch.float64 and dJdF.numel() >= 2 and dJdF.stride(-1) == 1
            check(lib().fs_step_adjoint_dev(self.h, byref(sn), byref(sl), c_void_p(dJdF.data_ptr()), byref(g),
                                            float(dt)))
            return
        dj = None
        if dJdF is not None:
            dj = (c_double * 2)(*[float(x) for x in dJdF])
        check(lib().fs_step_adjoint(self.h, byref(sn), byref(sl), dj, byref(g), float(dt)))

    @staticmethod
    def _ptrs(fields):
        return (c_void_p * 3)(*[c_void_p(x.data_ptr()) for x in fields], *([None] * (3 - len(fields))))

    def step_record(self, u, dt, v1, v2, p=None):
        """One RK3 step of u that leaves its two stage states in v1, v2 (lists shaped like u)."""
        s = self._state(u, p, None)
        check(lib().fs_step_record(self.h, byref(s), float(dt), self._ptrs(v1), self._ptrs(v2)))

    def step_adjoint_recorded(self, u_n, v1, v2, lam, dt, g_body_force=None):
        """step_adjoint of a step recorded by step_record from u_n (no recomputation)."""
        sn = self._state(u_n, None, None)
        sl = self._state(lam, None, None)
        g = ParamGrad()
        g.body_force = g_body_force.data_ptr() if g_body_force is not None else None
        g.stiffness = None
        check(lib().fs_step_adjoint_recorded(self.h, byref(sn), self._ptrs(v1), self._ptrs(v2), byref(sl),
                                             byref(g), float(dt)))

    def solve_pressure(self, rhs, p=None):
        p = torch.empty_like(rhs) if p is None else p
        check(lib().fs_solve_pressure(self.h, c_void_p(rhs.data_ptr()), c_void_p(p.data_ptr())))
        return p

    def solve_pressure_cg(self, rhs, p=None, tol=1e-12, maxit=100000, jacobi=False):
        """Krylov (CG) solve of D G p = rhs on an FP64 grid: returns (p, iterations, relative residual)."""
        p = torch.empty_like(rhs) if p is None else p
        it, rel = c_int(0), c_double(0.0)
        check(lib().fs_solve_pressure_cg(self.h, c_void_p(rhs.data_ptr()), c_void_p(p.data_ptr()), tol, maxit,
                                         1 if jacobi else 0, byref(it), byref(rel)))
        return p, it.value, rel.value

    def box_forces(self, with_q=False):
        """Force of the last step on the static 3-D box body: (F_x, F_y, F_z) [, q (nm, 3)]."""
        F = (c_double * 3)()
        tq = c_double()
        nm = self.n_box_markers
        q = (c_double * (3 * nm))() if with_q else None
        check(lib().fs_forces(self.h, F, byref(tq), q))
        if with_q:
            return (F[0], F[1], F[2]), [(q[3 * i], q[3 * i + 1], q[3 * i + 2]) for i in range(nm)]
        return F[0], F[1], F[2]

    def forces(self, with_q=False):
        F = (c_double * 2)()
        tq = c_double()
        q = (c_double * (2 * self.nm))() if with_q else None
        check(lib().fs_forces(self.h, F, byref(tq), q))
        out = (F[0], F[1]), tq.value
        if with_q:
            return out + ([(q[2 * i], q[2 * i + 1]) for i in range(self.nm)],)
        return out

    def set_body_force(self, fx):
        """fx: device float64 tensor with ny values (makes the profile a parameter)."""
        assert fx.is_cuda and fx.dtype == torch.float64 and fx.numel() == self.n[1]
        check(lib().fs_set_body_force(self.h, c_void_p(fx.contiguous().data_ptr())))

    def set_tuning(self, key, value):
        check(lib().fs_set_tuning(self.h, key.encode(), int(value)))

    def set_stream(self, stream):
        """Enqueue later work on a torch.cuda.Stream (e.g. a graph-capture branch)."""
        self.stream = stream
        check(lib().fs_set_stream(self.h, c_void_p(stream.cuda_stream)))

    def set_boxes(self, boxes, X, dV, kernel):
        """Static 3-D body: boxes (nb, 6), markers X (nm, 3), volumes dV (nm,), delta kernel."""
        import numpy as np
        b, bp = _dptr(np.asarray(boxes, dtype=np.float64).reshape(-1, 6))
        x, xp = _dptr(np.asarray(X, dtype=np.float64).reshape(-1, 3))
        v, vp = _dptr(np.asarray(dV, dtype=np.float64).reshape(-1))
        check(lib().fs_set_ib_boxes(self.h, b.shape[0], bp, x.shape[0], xp, vp, int(kernel)))
        self.n_box_markers = x.shape[0]
        self.has_boxes = True

    def set_les(self, cs):
        """Constant-coefficient Smagorinsky model with constant cs (0: off)."""
        check(lib().fs_set_les(self.h, float(cs)))
        self.les_cs = float(cs)

    def set_coupling(self, max_subiters, tol=1e-5):
        """Strong FSI coupling: sub-iterate each step up to max_subiters fluid solves (1 = weak)."""
        check(lib().fs_set_coupling(self.h, int(max_subiters), float(tol)))

    def ib_face_count(self):
        """IB faces classified by the last step (synchronises)."""
        n = c_int(0)
        check(lib().fs_ib_face_count(self.h, byref(n)))
        return n.value

    def coupling_stats(self):
        k, xi = c_int(0), c_double(0.0)
        check(lib().fs_coupling_stats(self.h, byref(k), byref(xi)))
        return k.value, xi.value

    def set_stiffness(self, k):
        check(lib().fs_set_stiffness(self.h, float(k)))

    def forces_device(self, out):
        """Copy {F_x, F_y, torque} of the last step into the device float64 tensor out (3 values)."""
        check(lib().fs_forces_device(self.h, c_void_p(out.data_ptr())))

    def diagnostics(self, u):
        s = self._state(u)
        out = (c_double * 3)()
        check(lib().fs_diagnostics(self.h, byref(s), out))
        return {"umax": out[0], "divmax": out[1], "ke": out[2]}

    def launches(self):
        return int(lib().fs_kernel_launches(self.h))

    def device_status(self):
        """Status bits set by kernels since the last call (0: nothing to report); synchronises."""
        v = ctypes.c_uint(0)
        check(lib().fs_device_status(self.h, byref(v)))
        return int(v.value)

    def profile_begin(self, filter_=""):
        check(lib().fs_profile_begin(self.h, filter_.encode()))

    def profile_end(self):
        """{kernel name: (launches, total ms)} of the launches since profile_begin (synchronises)."""
        buf = ctypes.create_string_buffer(1 << 16)
        check(lib().fs_profile_end(self.h, buf, len(buf)))
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms = line.split()
            out[name] = (int(cnt), float(ms))
        return out
