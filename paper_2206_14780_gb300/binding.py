"""Thin ctypes binding of include/sphvisc.h (argument marshalling only).

Every computation runs in libsphvisc.so; this module only converts torch
tensors to device pointers and C structs, and raises on a non-OK status.
There is no CPU fallback: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsphvisc.so")

SPH_OK = 0
SPH_NOALLOC_MAX_ROWS = 262144
STATUS = {0: "SPH_OK", 1: "SPH_ERR_INVALID", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_CAPACITY", 4: "SPH_ERR_NONFINITE",
          5: "SPH_ERR_TIMEOUT", 6: "SPH_NOT_CONVERGED", 7: "SPH_ERR_NOMEM"}
SPH_BC_DUMMY, SPH_BC_DYNAMIC = 0, 1
SPH_MEAN_HARMONIC, SPH_MEAN_ARITHMETIC = 0, 1
SPH_PREC_MIXED, SPH_PREC_FP64 = 0, 1
SPH_CONVERGED, SPH_STALLED, SPH_PROGRESSING = 0, 1, 2
SPH_SOLVER_BICGSTAB, SPH_SOLVER_CG = 0, 1
SPH_KERNEL_WENDLAND, SPH_KERNEL_GAUSSIAN = 0, 1

# every symbol include/sphvisc.h declares
EXPORTS = ["sph_build_neighbors", "sph_neighbors_info", "sph_neighbors_export", "sph_set_viscosity",
           "sph_neighbors_destroy", "sph_visc_setup", "sph_visc_apply", "sph_visc_apply_otf", "sph_visc_apply_noalloc", "sph_visc_residual", "sph_visc_solve",
           "sph_mu_papanastasiou", "sph_profile_enable", "sph_profile_read", "sph_last_error", "sph_version",
           "sph_batch_create", "sph_batch_solve", "sph_batch_info", "sph_batch_tiles", "sph_batch_set_tile",
           "sph_batch_destroy",
           "sph_mlp_create", "sph_mlp_set_params", "sph_mlp_get_params", "sph_mlp_destroy", "sph_mlp_features",
           "sph_mlp_targets", "sph_mlp_forward", "sph_mlp_grad", "sph_mlp_train_step", "sph_warm_start",
           "sph_mlp_residual_targets", "sph_mlp_set_mode", "sph_visc_solve_host", "sph_bicgstab_replay",
           "sph_shard_plan", "sph_shard_create", "sph_shard_info", "sph_shard_solve", "sph_shard_destroy",
           "sph_step", "sph_set_row_scale", "sph_row_norms", "sph_wall_row_scale",
           "sph_mlp_row_scale", "sph_mlp_scale_targets",
           "sph_shard_set_striping"]
MLP_NPARAMS = 9603


class sph_scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("ptype", ctypes.c_void_p), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("periodic", ctypes.c_int32 * 3), ("h", ctypes.c_float), ("kernel", ctypes.c_int32)]


class sph_visc_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("boundary", ctypes.c_int32), ("mean", ctypes.c_int32)]


class sph_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("eps_inner", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("merged_reductions", ctypes.c_int32), ("chunk", ctypes.c_int32), ("jacobi", ctypes.c_int32),
                ("apply_form", ctypes.c_int32), ("launch_mode", ctypes.c_int32), ("method", ctypes.c_int32)]


class sph_solve_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("state", ctypes.c_int8 * 3), ("stalled_any", ctypes.c_int8 * 3),
                ("true_rel_res", ctypes.c_double), ("true_rel_res_c", ctypes.c_double * 3)]


class sph_profile_counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("apply_launches", ctypes.c_int64), ("apply_ms", ctypes.c_double),
                ("apply_bytes", ctypes.c_int64), ("op_nnz", ctypes.c_int64),
                ("phase_launches", ctypes.c_int64 * 2), ("phase_ms", ctypes.c_double * 2),
                ("apply_variant", ctypes.c_int32 * 2), ("tune_us", (ctypes.c_float * 6) * 3),
                ("standalone_launches", ctypes.c_int64 * 2), ("standalone_ms", ctypes.c_double * 2),
                ("otf_bytes", ctypes.c_int64), ("apply_grid", ctypes.c_int32 * 2)]


class sph_state(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("mu", ctypes.c_void_p), ("ptype", ctypes.c_void_p), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("periodic", ctypes.c_int32 * 3), ("h", ctypes.c_float),
                ("kernel", ctypes.c_int32)]


class sph_step_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("rho0", ctypes.c_double), ("c0", ctypes.c_double),
                ("zeta", ctypes.c_double), ("g", ctypes.c_double * 3), ("boundary", ctypes.c_int32),
                ("mean", ctypes.c_int32), ("rheology", ctypes.c_int32), ("tau0", ctypes.c_double),
                ("mu0", ctypes.c_double), ("m", ctypes.c_double), ("max_neighbors", ctypes.c_int32),
                ("picard", ctypes.c_int32), ("picard_tol", ctypes.c_double)]


class sph_step_report(ctypes.Structure):
    _fields_ = [("half", sph_solve_report), ("full", sph_solve_report), ("picard_passes", ctypes.c_int32),
                ("picard_change", ctypes.c_double)]


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libsphvisc.so (built by paper_2206_14780_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2206_14780_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sph_build_neighbors": [ctypes.POINTER(sph_scene), i32, ctypes.POINTER(vp), vp],
        "sph_neighbors_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "sph_neighbors_export": [vp, vp, vp, vp],
        "sph_set_viscosity": [vp, vp, vp],
        "sph_neighbors_destroy": [vp],
        "sph_visc_setup": [vp, ctypes.POINTER(sph_visc_params), vp],
        "sph_visc_apply": [vp, ctypes.POINTER(sph_visc_params), vp, vp, vp],
        "sph_visc_apply_otf": [vp, ctypes.POINTER(sph_visc_params), vp, vp, vp],
        "sph_visc_apply_noalloc": [vp, ctypes.POINTER(sph_visc_params), vp, vp, vp],
        "sph_visc_residual": [vp, ctypes.POINTER(sph_visc_params), vp, vp, vp, vp],
        "sph_visc_solve": [vp, ctypes.POINTER(sph_visc_params), ctypes.POINTER(sph_solve_opts), vp, vp,
                           ctypes.POINTER(sph_solve_report), vp],
        "sph_mu_papanastasiou": [vp, vp, vp, dbl, dbl, dbl, vp, i32, vp],
        "sph_profile_enable": [vp, i32],
        "sph_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(sph_visc_params), i32, ctypes.POINTER(vp), vp],
        "sph_batch_solve": [vp, ctypes.POINTER(sph_solve_opts), ctypes.POINTER(vp), ctypes.POINTER(vp),
                            ctypes.POINTER(sph_solve_report), vp],
        "sph_batch_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float),
                           ctypes.POINTER(i32)],
        "sph_batch_tiles": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                            ctypes.POINTER(ctypes.c_float)],
        "sph_batch_set_tile": [vp, i32, vp],
        "sph_batch_destroy": [vp],
        "sph_mlp_create": [vp, ctypes.POINTER(vp)],
        "sph_mlp_set_params": [vp, vp],
        "sph_mlp_get_params": [vp, vp],
        "sph_mlp_destroy": [vp],
        "sph_mlp_features": [vp, ctypes.POINTER(sph_visc_params), vp, vp, ctypes.POINTER(dbl), vp],
        "sph_mlp_targets": [vp, vp, vp, vp, vp, vp, vp],
        "sph_mlp_forward": [vp, vp, i64, vp, vp],
        "sph_mlp_grad": [vp, vp, vp, vp, i64, i64, vp, vp, vp],
        "sph_mlp_train_step": [vp, vp, vp, vp, i64, i64, ctypes.c_float, ctypes.POINTER(ctypes.c_float), vp],
        "sph_warm_start": [vp, ctypes.POINTER(sph_visc_params), vp, vp, vp, vp, vp, vp],
        "sph_mlp_set_mode": [vp, ctypes.c_int32],
        "sph_mlp_residual_targets": [vp, ctypes.POINTER(sph_visc_params), vp, vp, vp, vp, ctypes.c_int, vp, vp,
                                     vp, ctypes.POINTER(dbl), vp],
        "sph_profile_read": [vp, ctypes.POINTER(sph_profile_counters), i32],
        "sph_bicgstab_replay": [vp, dbl, i32, i32, vp, vp, vp],
        "sph_shard_plan": [i64, vp, i32, i32, vp, vp, vp],
        "sph_shard_create": [vp, ctypes.POINTER(sph_visc_params), i32, ctypes.POINTER(vp), vp],
        "sph_shard_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), vp, vp, ctypes.POINTER(i64)],
        "sph_shard_solve": [vp, ctypes.POINTER(sph_solve_opts), vp, vp, ctypes.POINTER(sph_solve_report), vp],
        "sph_shard_destroy": [vp],
        "sph_shard_set_striping": [vp, i32],
        "sph_step": [ctypes.POINTER(sph_state), ctypes.POINTER(sph_step_params), ctypes.POINTER(sph_solve_opts),
                     ctypes.POINTER(vp), ctypes.POINTER(sph_step_report), vp],
        "sph_set_row_scale": [vp, vp, vp],
        "sph_row_norms": [vp, ctypes.POINTER(sph_visc_params), vp, vp],
        "sph_wall_row_scale": [vp, ctypes.POINTER(sph_visc_params), dbl, dbl, vp, vp],
        "sph_mlp_row_scale": [vp, ctypes.POINTER(sph_visc_params), vp, vp, vp, vp],
        "sph_mlp_scale_targets": [vp, ctypes.POINTER(sph_visc_params), dbl, dbl, vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.sph_last_error.restype = ctypes.c_char_p
    lib.sph_last_error.argtypes = []
    lib.sph_version.restype = ctypes.c_char_p
    lib.sph_version.argtypes = []
    _lib = lib
    return lib


def _check(status):
    if status != SPH_OK:
        raise SphError(status, _lib.sph_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def launch_count():
    """Kernels launched by the library so far (process-wide)."""
    load()
    c = sph_profile_counters()
    _check(_lib.sph_profile_read(None, ctypes.byref(c), 0))
    return c.launches


def bicgstab_replay(gamma0, eps, maxit, dots, stream=None):
    """sph_bicgstab_replay: the solver's scalar steps on given dots ([k][15] float64).
    Returns the [k + 1][20] table (alpha, omega, alpha', beta, state, stalled_any per
    component, iterations, done) after the initialisation and after each step."""
    load()
    g = np.ascontiguousarray(gamma0, np.float64).reshape(3)
    d = np.ascontiguousarray(dots, np.float64).reshape(-1, 15)
    out = np.empty((d.shape[0] + 1, 20), np.float64)
    _check(_lib.sph_bicgstab_replay(g.ctypes.data_as(ctypes.c_void_p), float(eps), int(maxit), int(d.shape[0]),
                                    d.ctypes.data_as(ctypes.c_void_p) if d.shape[0] else None,
                                    out.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return out


def shard_plan(layer, nlayers, ranks):
    """sph_shard_plan (host only): returns (virt [n] int64, rank_first_layer [ranks + 1],
    layer_first_virt [nlayers + 1])."""
    load()
    lay = np.ascontiguousarray(layer, np.int32)
    virt = np.empty(lay.size, np.int64)
    rfl = np.empty(ranks + 1, np.int32)
    lfv = np.empty(nlayers + 1, np.int64)
    _check(_lib.sph_shard_plan(lay.size, lay.ctypes.data_as(ctypes.c_void_p), int(nlayers), int(ranks),
                               virt.ctypes.data_as(ctypes.c_void_p), rfl.ctypes.data_as(ctypes.c_void_p),
                               lfv.ctypes.data_as(ctypes.c_void_p)))
    return virt, rfl, lfv


class Shard:
    """Owner of an sph_shard: one system partitioned over `ranks` sub-domains."""

    def __init__(self, nb, params, ranks, stream=None):
        load()
        h = ctypes.c_void_p()
        _check(_lib.sph_shard_create(nb.handle, ctypes.byref(params), int(ranks), ctypes.byref(h), _stream(stream)))
        self.handle = h
        self.ranks = int(ranks)
        self._nb = nb

    def info(self):
        ax, nl, ex = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        owned = np.empty(self.ranks, np.int64)
        halo = np.empty(self.ranks, np.int64)
        _check(_lib.sph_shard_info(self.handle, ctypes.byref(ax), ctypes.byref(nl),
                                   owned.ctypes.data_as(ctypes.c_void_p), halo.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(ex)))
        return dict(axis=ax.value, layers=nl.value, owned=owned.tolist(), halo=halo.tolist(), exchanged=ex.value)

    def set_striping(self, on):
        """sph_shard_set_striping: overlap each halo exchange with the interior slices' apply."""
        _check(_lib.sph_shard_set_striping(self.handle, int(bool(on))))

    def solve(self, opts, b, x, stream=None):
        rep = sph_solve_report()
        st = _lib.sph_shard_solve(self.handle, ctypes.byref(opts), _ptr(b), _ptr(x), ctypes.byref(rep),
                                  _stream(stream))
        if st not in (SPH_OK, 6):
            _check(st)
        return _report(rep)

    def close(self):
        if self.handle:
            _lib.sph_shard_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def visc_params(dt, boundary=SPH_BC_DUMMY, mean=SPH_MEAN_HARMONIC):
    return sph_visc_params(float(dt), int(boundary), int(mean))


def solve_opts(rtol=1e-6, eps_inner=2e-2, maxit=20000, max_refine=30, precision=SPH_PREC_MIXED,
               merged_reductions=0, chunk=8, jacobi=1, apply_form=0, launch_mode=0, method=0):
    """sph_solve_opts; method 0 = BiCGSTAB, 1 = the rotated conjugate gradient (SPH_SOLVER_CG)."""
    return sph_solve_opts(rtol, eps_inner, maxit, max_refine, precision, merged_reductions, chunk, jacobi,
                          apply_form, launch_mode, method)


def scene_tensors(scene, device="cuda"):
    """Copy a scene's particle arrays to the device (float32 pos[n,4], rho, mu, uint8 type)."""
    import torch

    return dict(pos=torch.from_numpy(np.ascontiguousarray(scene.pos, np.float32)).to(device),
                rho=torch.from_numpy(np.ascontiguousarray(scene.rho, np.float32)).to(device),
                mu=torch.from_numpy(np.ascontiguousarray(scene.mu, np.float32)).to(device),
                ptype=torch.from_numpy(np.ascontiguousarray(scene.ptype, np.uint8)).to(device))


class Neighbors:
    """Owner of one sph_neighbors handle (sph_build_neighbors ... sph_neighbors_destroy)."""

    def __init__(self, handle, n, keep):
        self.handle = handle
        self.n = n
        self._keep = keep

    def rebuild(self, pos, rho, mu, ptype, lo, hi, periodic, h, max_neighbors=128, stream=None, kernel=0):
        """sph_build_neighbors on this handle (rebuild in place, keeps the workspace)."""
        sc = _scene_struct(pos, rho, mu, ptype, lo, hi, periodic, h, kernel)
        handle = ctypes.c_void_p(self.handle.value if isinstance(self.handle, ctypes.c_void_p) else self.handle)
        _check(_lib.sph_build_neighbors(ctypes.byref(sc), int(max_neighbors), ctypes.byref(handle), _stream(stream)))
        self.handle = handle
        self.n = sc.n
        self._keep = (pos, rho, mu, ptype)

    def info(self):
        n, nnz, mc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.sph_neighbors_info(self.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(mc)))
        return n.value, nnz.value, mc.value

    def export(self, stream=None):
        import torch

        n, nnz, _ = self.info()
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        idx = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        _check(_lib.sph_neighbors_export(self.handle, _ptr(off), _ptr(idx), _stream(stream)))
        return off, idx[:nnz]

    def set_viscosity(self, mu, stream=None):
        _check(_lib.sph_set_viscosity(self.handle, _ptr(mu), _stream(stream)))

    def setup(self, params, stream=None):
        _check(_lib.sph_visc_setup(self.handle, ctypes.byref(params), _stream(stream)))

    def apply(self, params, v, y, stream=None):
        _check(_lib.sph_visc_apply(self.handle, ctypes.byref(params), _ptr(v), _ptr(y), _stream(stream)))

    def apply_otf(self, params, v, y, stream=None):
        """sph_visc_apply_otf: y = A v with the coefficients recomputed per pair."""
        _check(_lib.sph_visc_apply_otf(self.handle, ctypes.byref(params), _ptr(v), _ptr(y), _stream(stream)))

    def apply_noalloc(self, params, v, y, stream=None):
        """sph_visc_apply_noalloc: y = A v with no device allocation (needs setup first)."""
        _check(_lib.sph_visc_apply_noalloc(self.handle, ctypes.byref(params), _ptr(v), _ptr(y), _stream(stream)))

    def residual(self, params, x, b, r, stream=None):
        _check(_lib.sph_visc_residual(self.handle, ctypes.byref(params), _ptr(x), _ptr(b), _ptr(r),
                                      _stream(stream)))

    def solve(self, params, opts, b, x, stream=None, raise_on_nonconvergence=False):
        rep = sph_solve_report()
        st = _lib.sph_visc_solve(self.handle, ctypes.byref(params), ctypes.byref(opts), _ptr(b), _ptr(x),
                                 ctypes.byref(rep), _stream(stream))
        if st not in (SPH_OK, 6) or (st == 6 and raise_on_nonconvergence):
            _check(st)
        return dict(status=st, iters=rep.iters, refinements=rep.refinements, state=list(rep.state),
                    stalled_any=list(rep.stalled_any), true_rel_res=rep.true_rel_res,
                    true_rel_res_c=list(rep.true_rel_res_c))

    def set_row_scale(self, scale, stream=None):
        """sph_set_row_scale: scale (device float [n], caller order) multiplies the Jacobi
        diagonal's inverse in the mixed-precision solves; None clears it."""
        _check(_lib.sph_set_row_scale(self.handle, None if scale is None else _ptr(scale), _stream(stream)))

    def row_norms(self, params, out, stream=None):
        """sph_row_norms: squared norms of the rows of D^-1 A (device float [n], caller order)."""
        _check(_lib.sph_row_norms(self.handle, ctypes.byref(params), _ptr(out), _stream(stream)))

    def wall_row_scale(self, params, factor, power, out, stream=None):
        """sph_wall_row_scale: factor norm2^-power on dummy-wall rows, 1 elsewhere (device float [n])."""
        _check(_lib.sph_wall_row_scale(self.handle, ctypes.byref(params), float(factor), float(power), _ptr(out),
                                       _stream(stream)))

    def mu_papanastasiou(self, vel, wall_vel, tau0, mu0, m, mu_out, set_handle=True, stream=None):
        _check(_lib.sph_mu_papanastasiou(self.handle, _ptr(vel), _ptr(wall_vel), float(tau0), float(mu0), float(m),
                                         _ptr(mu_out), int(bool(set_handle)), _stream(stream)))

    def profile(self, on=True):
        _check(_lib.sph_profile_enable(self.handle, int(bool(on))))

    def profile_read(self, reset=False):
        c = sph_profile_counters()
        _check(_lib.sph_profile_read(self.handle, ctypes.byref(c), int(bool(reset))))
        return dict(launches=c.launches, apply_launches=c.apply_launches, apply_ms=c.apply_ms,
                    apply_bytes=c.apply_bytes, op_nnz=c.op_nnz, phase_launches=list(c.phase_launches),
                    phase_ms=list(c.phase_ms), apply_variant=list(c.apply_variant),
                    tune_us=[list(r) for r in c.tune_us], standalone_launches=list(c.standalone_launches),
                    standalone_ms=list(c.standalone_ms), otf_bytes=c.otf_bytes,
                    apply_grid=list(c.apply_grid))

    def close(self):
        if self.handle:
            _lib.sph_neighbors_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(t):
    """Pointer of a contiguous host (CPU) torch tensor or numpy array."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous host tensor")
        return ctypes.c_void_p(t.data_ptr())
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous host array")
    return ctypes.c_void_p(t.ctypes.data)


def solve_host(pos, rho, mu, ptype, lo, hi, periodic, h, params, opts, vel, b, x, nb=None, max_neighbors=128,
               stream=None):
    """sph_visc_solve_host on HOST arrays (torch CPU tensors, pinned for asynchronous copies, or
    numpy): neighbour build, x0 = v^n with the wall closure (vel given) or x, solve, x copied
    back.  nb: a Neighbors from an earlier call (or None: one is created).  Returns
    (report dict, Neighbors)."""
    load()
    sc = sph_scene()
    sc.n = int(pos.shape[0])
    sc.pos, sc.rho, sc.mu, sc.ptype = _host_ptr(pos), _host_ptr(rho), _host_ptr(mu), _host_ptr(ptype)
    for ax in range(3):
        sc.lo[ax] = float(lo[ax])
        sc.hi[ax] = float(hi[ax])
        sc.periodic[ax] = int(periodic[ax])
    sc.h = float(h)
    handle = ctypes.c_void_p(nb.handle.value if nb is not None else None)
    rep = sph_solve_report()
    st = _lib.sph_visc_solve_host(ctypes.byref(sc), int(max_neighbors), ctypes.byref(params), ctypes.byref(opts),
                                  _host_ptr(vel), _host_ptr(b), _host_ptr(x), ctypes.byref(handle),
                                  ctypes.byref(rep), _stream(stream))
    if nb is None and handle.value:
        nb = Neighbors(handle, sc.n, keep=())
    elif nb is not None:
        nb.handle = handle
        nb.n = sc.n
    if st not in (SPH_OK, 6):
        _check(st)
    return _report(rep), nb


def _scene_struct(pos, rho, mu, ptype, lo, hi, periodic, h, kernel=0):
    sc = sph_scene()
    sc.n = int(pos.shape[0])
    sc.pos, sc.rho, sc.mu, sc.ptype = _ptr(pos), _ptr(rho), _ptr(mu), _ptr(ptype)
    for ax in range(3):
        sc.lo[ax] = float(lo[ax])
        sc.hi[ax] = float(hi[ax])
        sc.periodic[ax] = int(periodic[ax])
    sc.h = float(h)
    sc.kernel = int(kernel)
    return sc


def _report(rep):
    return dict(status=rep.status, iters=rep.iters, refinements=rep.refinements, state=list(rep.state),
                stalled_any=list(rep.stalled_any), true_rel_res=rep.true_rel_res,
                true_rel_res_c=list(rep.true_rel_res_c))


class Batch:
    """Owner of an sph_batch (sph_batch_create ... sph_batch_destroy) over built Neighbors."""

    def __init__(self, neighbors, params, stream=None):
        load()
        self.nbs = list(neighbors)
        S = len(self.nbs)
        hs = (ctypes.c_void_p * S)(*[nb.handle.value if isinstance(nb.handle, ctypes.c_void_p) else nb.handle
                                    for nb in self.nbs])
        ps = (sph_visc_params * S)(*params)
        h = ctypes.c_void_p()
        _check(_lib.sph_batch_create(hs, ps, S, ctypes.byref(h), _stream(stream)))
        self.handle = h

    def solve(self, opts, bs, xs, stream=None):
        S = len(self.nbs)
        bp = (ctypes.c_void_p * S)(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * S)(*[x.data_ptr() for x in xs])
        reps = (sph_solve_report * S)()
        st = _lib.sph_batch_solve(self.handle, ctypes.byref(opts), bp, xp, reps, _stream(stream))
        if st not in (SPH_OK, 6):
            _check(st)
        return st, [_report(r) for r in reps]

    def set_tile(self, tile_slices, stream=None):
        _check(_lib.sph_batch_set_tile(self.handle, int(tile_slices), _stream(stream)))

    def info(self):
        v, g, grid = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        t = (ctypes.c_float * 8)()
        _check(_lib.sph_batch_info(self.handle, ctypes.byref(v), ctypes.byref(g), t, ctypes.byref(grid)))
        ts, nt = ctypes.c_int32(), ctypes.c_int32()
        cand, tms = (ctypes.c_int32 * 3)(), (ctypes.c_float * 3)()
        _check(_lib.sph_batch_tiles(self.handle, ctypes.byref(ts), ctypes.byref(nt), cand, tms))
        return dict(variant=v.value, graph=bool(g.value), graph_mode=g.value, tune_ms=list(t), grid=grid.value,
                    tile_slices=ts.value,
                    ntiles=nt.value, tile_candidates=list(cand), tile_tune_ms=list(tms))

    def close(self):
        if self.handle:
            _lib.sph_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """Owner of an sph_mlp (the learned warm-start network)."""

    def __init__(self, params=None):
        load()
        h = ctypes.c_void_p()
        if params is None:
            _check(_lib.sph_mlp_create(None, ctypes.byref(h)))
        else:
            p = np.ascontiguousarray(params, np.float32)
            assert p.size == MLP_NPARAMS
            _check(_lib.sph_mlp_create(p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self.handle = h

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == MLP_NPARAMS
        _check(_lib.sph_mlp_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)))

    def params(self):
        p = np.empty(MLP_NPARAMS, np.float32)
        _check(_lib.sph_mlp_get_params(self.handle, p.ctypes.data_as(ctypes.c_void_p)))
        return p

    def set_mode(self, mode):
        """sph_mlp_set_mode (MLP_HIGHPASS: the x0 correction is y - S y)."""
        _check(_lib.sph_mlp_set_mode(self.handle, int(mode)))

    def forward(self, feats, out, stream=None):
        _check(_lib.sph_mlp_forward(self.handle, _ptr(feats), int(feats.shape[0]), _ptr(out), _stream(stream)))

    def grad(self, feats, targets, mask, count, grad_out, loss_out, stream=None):
        _check(_lib.sph_mlp_grad(self.handle, _ptr(feats), _ptr(targets), _ptr(mask), int(feats.shape[0]),
                                 int(count), _ptr(grad_out), _ptr(loss_out), _stream(stream)))

    def train_step(self, feats, targets, mask, count, lr, stream=None):
        loss = ctypes.c_float()
        _check(_lib.sph_mlp_train_step(self.handle, _ptr(feats), _ptr(targets), _ptr(mask), int(feats.shape[0]),
                                       int(count), float(lr), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def close(self):
        if self.handle:
            _lib.sph_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_row_scale(nb, params, mlp, vel, scale, stream=None):
    """sph_mlp_row_scale: the learned wall-row scale (device float [n], caller order), or
    with scale None installed as the handle's row scale directly."""
    _check(_lib.sph_mlp_row_scale(nb.handle, ctypes.byref(params), mlp.handle, _ptr(vel), _ptr(scale),
                                  _stream(stream)))


def mlp_scale_targets(nb, params, factor, power, targets, mask, stream=None):
    """sph_mlp_scale_targets: (log s, 0, 0, 0) of the closed-form wall scale, wall-row mask."""
    _check(_lib.sph_mlp_scale_targets(nb.handle, ctypes.byref(params), float(factor), float(power), _ptr(targets),
                                      _ptr(mask), _stream(stream)))


def mlp_features(nb, params, vel, feats, stream=None):
    """sph_mlp_features: feats (device int16 [n,16] holding bf16 bits); returns U."""
    U = ctypes.c_double()
    _check(_lib.sph_mlp_features(nb.handle, ctypes.byref(params), _ptr(vel), _ptr(feats), ctypes.byref(U),
                                 _stream(stream)))
    return U.value


def mlp_targets(nb, vel, x_star, ptype, targets, mask, stream=None):
    _check(_lib.sph_mlp_targets(nb.handle, _ptr(vel), _ptr(x_star), _ptr(ptype), _ptr(targets), _ptr(mask),
                                _stream(stream)))


MLP_HIGHPASS = 1
RLOSS_JACOBI = 1
RLOSS_LOG = 2


def mlp_residual_targets(nb, params, mlp, vel, ptype, b, feats, targets, mask, flags=RLOSS_LOG, stream=None):
    """sph_mlp_residual_targets; returns the residual loss L."""
    L = ctypes.c_double()
    _check(_lib.sph_mlp_residual_targets(nb.handle, ctypes.byref(params), mlp.handle, _ptr(vel), _ptr(ptype), _ptr(b),
                                         int(flags), _ptr(feats), _ptr(targets), _ptr(mask), ctypes.byref(L),
                                         _stream(stream)))
    return L.value


def warm_start(nb, params, mlp, vel, ptype, b, x0, stream=None):
    """sph_warm_start; mlp=None gives v^n with the dummy-wall closure."""
    _check(_lib.sph_warm_start(nb.handle, ctypes.byref(params), mlp.handle if mlp is not None else None, _ptr(vel),
                               _ptr(ptype), _ptr(b), _ptr(x0), _stream(stream)))


def step_params(dt, rho0, c0, zeta=7.0, g=(0.0, 0.0, 0.0), boundary=SPH_BC_DUMMY, mean=SPH_MEAN_HARMONIC,
                rheology=None, max_neighbors=128, picard=0, picard_tol=0.0):
    """sph_step_params; rheology = (tau0, mu0, m) for Papanastasiou, None for Newtonian;
    picard: fixed-point passes bringing mu into the implicit system (0: lagged mu)."""
    p = sph_step_params()
    p.dt, p.rho0, p.c0, p.zeta = float(dt), float(rho0), float(c0), float(zeta)
    for k in range(3):
        p.g[k] = float(g[k])
    p.boundary, p.mean = int(boundary), int(mean)
    p.rheology = 0 if rheology is None else 1
    if rheology is not None:
        p.tau0, p.mu0, p.m = (float(v) for v in rheology)
    p.max_neighbors = int(max_neighbors)
    p.picard = int(picard)
    p.picard_tol = float(picard_tol)
    return p


class Stepper:
    """sph_step on a particle state held in device tensors (pos [n,4], vel [n,4], rho, mu
    float32, ptype uint8), advanced in place; owns the neighbour handle between steps."""

    def __init__(self, pos, vel, rho, mu, ptype, lo, hi, periodic, h, kernel=0):
        load()
        self.t = dict(pos=pos, vel=vel, rho=rho, mu=mu, ptype=ptype)
        st = sph_state()
        st.n = int(pos.shape[0])
        st.pos, st.vel, st.rho, st.mu, st.ptype = _ptr(pos), _ptr(vel), _ptr(rho), _ptr(mu), _ptr(ptype)
        for ax in range(3):
            st.lo[ax] = float(lo[ax])
            st.hi[ax] = float(hi[ax])
            st.periodic[ax] = int(periodic[ax])
        st.h = float(h)
        st.kernel = int(kernel)
        self.state = st
        self.handle = ctypes.c_void_p()

    def step(self, params, opts, stream=None):
        rep = sph_step_report()
        s = _lib.sph_step(ctypes.byref(self.state), ctypes.byref(params), ctypes.byref(opts),
                          ctypes.byref(self.handle), ctypes.byref(rep), _stream(stream))
        if s not in (SPH_OK, 6):
            _check(s)
        return dict(status=s, half=_report(rep.half), full=_report(rep.full), picard_passes=rep.picard_passes,
                    picard_change=rep.picard_change)

    def close(self):
        if self.handle:
            _lib.sph_neighbors_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_neighbors(pos, rho, mu, ptype, lo, hi, periodic, h, max_neighbors=128, stream=None, kernel=0):
    """sph_build_neighbors on device tensors; returns a Neighbors owner.  kernel: 0 Wendland, 1 Gaussian."""
    load()
    sc = _scene_struct(pos, rho, mu, ptype, lo, hi, periodic, h, kernel)
    handle = ctypes.c_void_p()
    _check(_lib.sph_build_neighbors(ctypes.byref(sc), int(max_neighbors), ctypes.byref(handle), _stream(stream)))
    return Neighbors(handle, sc.n, keep=(pos, rho, mu, ptype))


def build_for_scene(scene, max_neighbors=128, device="cuda", stream=None):
    t = scene_tensors(scene, device)
    return build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], scene.lo, scene.hi, scene.periodic, scene.h,
                           max_neighbors, stream, kernel=getattr(scene, "kernel", 0)), t
