"""ctypes binding of include/lbe.h (argument marshalling only).

Every computation runs in liblbe.so.  Loading fails loudly when the library has not been
built (``python -m paper_1612_04488_gb300.build``); there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbe.so")

OK, NOT_CONVERGED, NAN, BAD_ARG, OOM, TIMEOUT, INTERNAL, UNSUPPORTED, CANCELLED = range(9)
POISEUILLE, THERMAL_TRANSPIRATION = 0, 1
CIS, SIS = 0, 1
FP64, FP32, BF16_REFINED, FP32_REFINED, DF32, BF16 = 0, 1, 2, 3, 4, 5


class Geometry(C.Structure):
    _fields_ = [("dim", C.c_int), ("ns", C.c_int), ("grid_kind", C.c_int), ("nx", C.c_int),
                ("ny", C.c_int), ("width", C.c_double)]


class Problem(C.Structure):
    _fields_ = [("geom", Geometry), ("delta", C.c_double), ("N", C.c_double), ("nv", C.c_int),
                ("vmax", C.c_double), ("M", C.c_int), ("R", C.c_double), ("forcing", C.c_int),
                ("scheme", C.c_int), ("precision", C.c_int), ("eps", C.c_double),
                ("max_iter", C.c_int)]


class Result(C.Structure):
    _fields_ = [("mass_flow", C.c_double), ("heat_flow", C.c_double), ("iters", C.c_int),
                ("status", C.c_int), ("last_rel_change", C.c_double), ("seconds", C.c_double),
                ("refinements", C.c_int)]


class Mixture(C.Structure):
    _fields_ = [("mass_ratio", C.c_double), ("diam_ratio", C.c_double), ("chi_A", C.c_double)]


class MixProblem(C.Structure):
    _fields_ = [("mix", Mixture), ("geom", Geometry), ("delta", C.c_double),
                ("N_A", C.c_double), ("N_B", C.c_double), ("nv", C.c_int), ("vmax", C.c_double),
                ("M", C.c_int), ("R", C.c_double), ("scheme", C.c_int), ("eps", C.c_double),
                ("max_iter", C.c_int), ("precision", C.c_int), ("solid_fraction", C.c_double)]


class MixResult(C.Structure):
    _fields_ = [("M_A", C.c_double), ("M_B", C.c_double), ("Q_A", C.c_double), ("Q_B", C.c_double),
                ("iters", C.c_int), ("status", C.c_int), ("N_A", C.c_double), ("N_B", C.c_double),
                ("fp64_iters", C.c_int)]


def mix_problem(mass_ratio, diam_ratio, chi_A, delta=1.0, ns=20, grid_kind=0, N_A=0.0, N_B=0.0, nv=16,
                vmax=6.0, M=16, R=4.5, scheme=SIS, eps=1e-8, max_iter=500, precision=FP64, dim=1, nx=0, ny=0,
                width=1.0, solid=0.0):
    geom = Geometry(dim, ns if dim == 1 else 0, grid_kind if dim == 1 else 0, nx, ny, width)
    return MixProblem(Mixture(mass_ratio, diam_ratio, chi_A), geom, delta, N_A, N_B, nv, vmax, M, R,
                      scheme, eps, max_iter, precision, solid)


def mix_cells(pb):
    return pb.geom.ns + 1 if pb.geom.dim == 1 else pb.geom.nx * pb.geom.ny


class Stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("cell_l_evals", C.c_uint64), ("dense_gemm_timed", C.c_uint64), ("dense_gemm_ms", C.c_double),
                ("sweep_timed", C.c_uint64), ("sweep_ms", C.c_double), ("sweep_bytes", C.c_double)]


def stats():
    s = Stats()
    lib().lbe_get_stats(C.byref(s))
    return {k: getattr(s, k) for k, _ in Stats._fields_}


def set_kernel_timing(on):
    lib().lbe_set_kernel_timing(1 if on else 0)


def debug_expire_waits(on):
    """Test hook: the tensor-core GEMM's first pipeline wait runs out (lbe_debug_expire_waits)."""
    lib().lbe_debug_expire_waits(1 if on else 0)


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblbe.so is not built; run python -m paper_1612_04488_gb300.build")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        L.lbe_create.argtypes = [C.POINTER(vp), ip, C.c_size_t]
        L.lbe_destroy.argtypes = [vp]
        L.lbe_status_str.argtypes = [ip]
        L.lbe_status_str.restype = C.c_char_p
        L.lbe_last_error.argtypes = [vp]
        L.lbe_last_error.restype = C.c_char_p
        L.lbe_problem_cells.argtypes = [C.POINTER(Problem)]
        L.lbe_solve.argtypes = [vp, C.POINTER(Problem), C.POINTER(Result), dp, dp]
        L.lbe_solve_batch.argtypes = [vp, C.POINTER(Problem), ip, C.POINTER(Result)]
        L.lbe_apply_L.argtypes = [vp, ip, C.c_double, ip, C.c_double, ip, ip, vp, vp, vp, vp, vp, vp, vp]
        L.lbe_sweep.argtypes = [vp, C.POINTER(Problem), vp, vp, vp, vp]
        L.lbe_diffusion.argtypes = [vp, C.POINTER(Problem), dp, dp, dp, dp, dp, dp, dp]
        L.lbe_fourier_omega.argtypes = [vp, ip, C.c_double, ip, C.c_double, C.c_double, C.c_double, ip, ip, dp, dp]
        L.lbe_submit.argtypes = [vp, C.POINTER(Problem), C.POINTER(C.c_uint64)]
        L.lbe_poll.argtypes = [vp, C.c_uint64, C.POINTER(Result), C.POINTER(C.c_int)]
        L.lbe_set_max_active.argtypes = [vp, ip]
        L.lbe_set_stream.argtypes = [vp, vp]
        L.lbe_apply_L_sym.argtypes = [vp, ip, C.c_double, ip, C.c_double, ip, ip, ip, vp, vp, vp, vp, vp, vp, vp]
        L.lbe_apply_L_noalloc.argtypes = [vp, ip, C.c_double, ip, C.c_double, ip, ip, vp, vp, vp, vp, vp]
        L.lbe_batch_create.argtypes = [vp, C.POINTER(Problem), ip, C.POINTER(vp)]
        L.lbe_batch_run.argtypes = [vp, C.POINTER(Result)]
        L.lbe_batch_destroy.argtypes = [vp]
        L.lbe_get_stats.argtypes = [C.POINTER(Stats)]
        L.lbe_solve_from.argtypes = [vp, C.POINTER(Problem), dp, C.POINTER(Result), C.POINTER(Result), dp, dp]
        L.lbe_cancel.argtypes = [vp, C.c_uint64]
        L.lbe_debug_expire_waits.argtypes = [ip]
        L.lbe_tuning_report.argtypes = [vp, C.c_char_p, C.c_size_t]
        L.lbe_mix_info.argtypes = [vp, C.POINTER(Mixture), ip, C.c_double, ip, C.c_double, dp, dp]
        L.lbe_mix_apply_L.argtypes = [vp, C.POINTER(Mixture), ip, C.c_double, ip, C.c_double, ip, C.c_double,
                                      vp, vp, vp, vp, vp, vp, vp]
        L.lbe_mix_solve.argtypes = [vp, C.POINTER(MixProblem), C.POINTER(MixResult), dp, dp]
        _lib = L
    return _lib


class LbeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (lib().lbe_status_str(status).decode(), msg))
        self.status = status


def problem(dim=1, ns=20, grid_kind=0, nx=64, ny=32, width=2.0, delta=1.0, N=0.0, nv=16,
            vmax=6.0, M=16, R=0.0, forcing=POISEUILLE, scheme=SIS, precision=FP64, eps=1e-8,
            max_iter=500):
    return Problem(Geometry(dim, ns, grid_kind, nx, ny, width), delta, N, nv, vmax, M, R,
                   forcing, scheme, precision, eps, max_iter)


def cells_of(pb):
    return lib().lbe_problem_cells(C.byref(pb))


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


class Context:
    """Owns an lbe_ctx on one CUDA device."""

    def __init__(self, device=0, hbm_budget=0):
        self.h = C.c_void_p()
        st = lib().lbe_create(C.byref(self.h), device, hbm_budget)
        if st != OK:
            raise LbeError(st, "lbe_create")

    def close(self):
        if self.h:
            lib().lbe_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def err(self):
        return lib().lbe_last_error(self.h).decode()

    def check(self, st, allow=(OK,)):
        if st not in allow:
            raise LbeError(st, self.err())
        return st

    def solve(self, pb, want_h=False, want_U=True):
        n = cells_of(pb)
        U = np.zeros(n) if want_U else None
        h = np.zeros(n * pb.nv ** 3) if want_h else None
        res = Result()
        st = lib().lbe_solve(self.h, C.byref(pb), C.byref(res), _dptr(U), _dptr(h))
        self.check(st, (OK, NOT_CONVERGED))
        return res, U, (h.reshape((n,) + (pb.nv,) * 3) if want_h else None)

    def solve_from(self, pb, h_in, prev=None, want_h=False, want_U=True):
        """lbe_solve_from: resume a solve from the iterate h_in (and the flow rates of prev)."""
        n = cells_of(pb)
        hin = np.ascontiguousarray(h_in, dtype=np.float64).reshape(-1)
        if hin.size != n * pb.nv ** 3:
            raise ValueError("h_in must hold cells * nv^3 values")
        U = np.zeros(n) if want_U else None
        h = np.zeros(n * pb.nv ** 3) if want_h else None
        res = Result()
        st = lib().lbe_solve_from(self.h, C.byref(pb), _dptr(hin), C.byref(prev) if prev is not None else None,
                                  C.byref(res), _dptr(U), _dptr(h))
        self.check(st, (OK, NOT_CONVERGED))
        return res, U, (h.reshape((n,) + (pb.nv,) * 3) if want_h else None)

    def solve_batch(self, pbs):
        arr = (Problem * len(pbs))(*pbs)
        res = (Result * len(pbs))()
        st = lib().lbe_solve_batch(self.h, arr, len(pbs), res)
        self.check(st, (OK, NOT_CONVERGED))
        return list(res)

    def apply_L(self, nv, vmax, M, R, precision, cells, delta_ptr, h_ptr, lplus_ptr, l_ptr,
                nd_ptr=None, G_ptr=None, stream=None):
        st = lib().lbe_apply_L(self.h, nv, vmax, M, R, precision, cells, delta_ptr, h_ptr,
                               lplus_ptr, l_ptr, nd_ptr, G_ptr, stream)
        return self.check(st)

    def apply_L_sym(self, nv, vmax, M, R, precision, parity, cells, delta_ptr, h_ptr, lplus_ptr, l_ptr,
                    nd_ptr=None, G_ptr=None, stream=None):
        st = lib().lbe_apply_L_sym(self.h, nv, vmax, M, R, precision, parity, cells, delta_ptr, h_ptr,
                                   lplus_ptr, l_ptr, nd_ptr, G_ptr, stream)
        return self.check(st)

    def apply_L_noalloc(self, nv, vmax, M, R, precision, cells, delta_ptr, h_ptr, lplus_ptr, l_ptr,
                        stream=None):
        st = lib().lbe_apply_L_noalloc(self.h, nv, vmax, M, R, precision, cells, delta_ptr, h_ptr,
                                       lplus_ptr, l_ptr, stream)
        return self.check(st)

    def mix_info(self, mix, nv, vmax, M, R, want_nu=False):
        """lbe_mix_info: (b_AA at delta = 1, N_A, N_B, mu1) and optionally nu_A, nu_B."""
        out = np.zeros(4)
        nu = np.zeros(2 * nv ** 3) if want_nu else None
        self.check(lib().lbe_mix_info(self.h, C.byref(mix), nv, vmax, M, R, _dptr(out), _dptr(nu)))
        return out, (nu.reshape((2,) + (nv,) * 3) if want_nu else None)

    def mix_apply_L(self, mix, nv, vmax, M, R, cells, delta, hA_ptr, hB_ptr, lpA_ptr, lA_ptr, lpB_ptr, lB_ptr,
                    stream=None):
        st = lib().lbe_mix_apply_L(self.h, C.byref(mix), nv, vmax, M, R, cells, delta, hA_ptr, hB_ptr, lpA_ptr,
                                   lA_ptr, lpB_ptr, lB_ptr, stream)
        return self.check(st)

    def mix_solve(self, pb, want_h=False, want_U=True):
        n = mix_cells(pb)
        U = np.zeros(2 * n) if want_U else None
        h = np.zeros(2 * n * pb.nv ** 3) if want_h else None
        res = MixResult()
        st = lib().lbe_mix_solve(self.h, C.byref(pb), C.byref(res), _dptr(U), _dptr(h))
        self.check(st, (OK, NOT_CONVERGED))
        return (res, U.reshape(2, n) if want_U else None,
                h.reshape((2, n) + (pb.nv,) * 3) if want_h else None)

    def sweep(self, pb, rhs_ptr, h_ptr, mom_ptr=None, stream=None):
        return self.check(lib().lbe_sweep(self.h, C.byref(pb), rhs_ptr, h_ptr, mom_ptr, stream))

    def fourier_omega(self, nv, vmax, M, R, delta, N, scheme, iters, e0):
        """Power-iteration ratios of the CIS / SIS Fourier-mode error map (lbe_fourier_omega);
        e0: complex or real array of nv^3 values (the start vector)."""
        e0 = np.asarray(e0).reshape(-1)
        buf = np.ascontiguousarray(np.concatenate([e0.real, e0.imag if np.iscomplexobj(e0) else 0 * e0.real]),
                                   dtype=np.float64)
        out = np.zeros(iters)
        st = lib().lbe_fourier_omega(self.h, nv, vmax, M, R, delta, N, scheme, iters,
                                     buf.ctypes.data_as(C.POINTER(C.c_double)),
                                     out.ctypes.data_as(C.POINTER(C.c_double)))
        self.check(st)
        return out

    def diffusion(self, pb, Uh, W1, W2, X12, G1, G2):
        n = cells_of(pb)
        out = np.zeros(n)
        arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
                for a in (Uh, W1, W2, X12, G1, G2)]
        st = lib().lbe_diffusion(self.h, C.byref(pb), *[_dptr(a) for a in arrs], _dptr(out))
        self.check(st)
        return out

    def submit(self, pb):
        t = C.c_uint64()
        self.check(lib().lbe_submit(self.h, C.byref(pb), C.byref(t)))
        return t.value

    def tuning_report(self):
        """The autotuner's decisions (lbe_tuning_report), one line each."""
        buf = C.create_string_buffer(1 << 16)
        lib().lbe_tuning_report(self.h, buf, len(buf))
        return [l for l in buf.value.decode().split("\n") if l]

    def cancel(self, ticket):
        self.check(lib().lbe_cancel(self.h, ticket))

    def poll(self, ticket):
        res = Result()
        done = C.c_int()
        self.check(lib().lbe_poll(self.h, ticket, C.byref(res), C.byref(done)))
        return bool(done.value), res

    def batch(self, pbs):
        return ResidentBatch(self, pbs)

    def set_stream(self, stream_handle):
        self.check(lib().lbe_set_stream(self.h, stream_handle))

    def set_max_active(self, n):
        self.check(lib().lbe_set_max_active(self.h, n))


class ResidentBatch:
    """lbe_batch_*: device state created once, re-solved from h = 0 on every run()."""

    def __init__(self, ctx, pbs):
        self.ctx = ctx
        self.n = len(pbs)
        self.h = C.c_void_p()
        arr = (Problem * self.n)(*pbs)
        ctx.check(lib().lbe_batch_create(ctx.h, arr, self.n, C.byref(self.h)))

    def run(self):
        res = (Result * self.n)()
        self.ctx.check(lib().lbe_batch_run(self.h, res), (OK, NOT_CONVERGED))
        return list(res)

    def close(self):
        if self.h:
            lib().lbe_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
