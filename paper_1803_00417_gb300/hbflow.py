"""Thin ctypes binding of the hbflow C-ABI (include/hbflow.h).

Argument marshalling only: every stage of the step runs in the CUDA library.
Device memory and streams come from PyTorch.  The library must have been built
(``paper_1803_00417_gb300.build.build()``); there is no CPU fallback and
loading fails loudly without it.

Array layout helpers convert between the x-fastest, component-major device
layout and numpy arrays indexed ``[i, j(, k)]`` (axis a = direction a).
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhbflow.so")

HBF_OK = 0
HBF_ERR_NOT_CONVERGED = -4
FIELDS = dict(U=0, P=1, ETA=2, USTAR=3, UADV=4, UMAC=5, RHS=6, PHI_MAC=7, GP=8, LU=9, UL=10, UR=11,
              ETA_FACES=12, SLOPES=13, HATS=14, NRES0=15, VRES0=16, VCORR=17)
FP64, MIXED = 0, 1


class SolveStats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("converged", ctypes.c_int), ("r0", ctypes.c_double),
                ("rnorm", ctypes.c_double), ("bnorm", ctypes.c_double), ("guess", ctypes.c_int)]

    def as_dict(self):
        return dict(cycles=self.cycles, converged=bool(self.converged), r0=self.r0, rnorm=self.rnorm,
                    bnorm=self.bnorm, guess=int(self.guess))


class StepStats(ctypes.Structure):
    _fields_ = [("mac", SolveStats), ("visc", SolveStats), ("nodal", SolveStats)]

    def as_dict(self):
        return dict(mac=self.mac.as_dict(), visc=self.visc.as_dict(), nodal=self.nodal.as_dict())


class State(ctypes.Structure):
    """hbf_state: the checkpoint record of a context."""
    _fields_ = [("dim", ctypes.c_int32), ("precision", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("h", ctypes.c_double), ("t", ctypes.c_double), ("step", ctypes.c_int64),
                ("K", ctypes.c_double), ("nexp", ctypes.c_double), ("tau_y", ctypes.c_double),
                ("m", ctypes.c_double), ("reg_power", ctypes.c_int32), ("predictor_viscous", ctypes.c_int32),
                ("theta", ctypes.c_double), ("periodic", ctypes.c_int32 * 3), ("rho", ctypes.c_double), ("f", ctypes.c_double * 3), ("wall_u", ctypes.c_double * 18)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out

    @classmethod
    def from_dict(cls, d):
        s = cls()
        for name, typ in cls._fields_:
            v = d[name]
            if isinstance(v, list):
                getattr(s, name)[:] = v
            else:
                setattr(s, name, v)
        return s


class YieldInfo(ctypes.Structure):
    _fields_ = [("tau_max", ctypes.c_double), ("yielded", ctypes.c_int64), ("cells", ctypes.c_int64 * 3),
                ("zones", ctypes.c_int64 * 3)]

    def as_dict(self):
        kinds = ("stagnant", "plug", "attached")
        return dict(tau_max=self.tau_max, yielded=self.yielded,
                    cells={k: self.cells[i] for i, k in enumerate(kinds)},
                    zones={k: self.zones[i] for i, k in enumerate(kinds)})


class RunInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("t", ctypes.c_double), ("change", ctypes.c_double),
                ("tau_ratio", ctypes.c_double), ("t_c", ctypes.c_double), ("t_c_interp", ctypes.c_double),
                ("reached", ctypes.c_int32), ("not_converged", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None

SIGNATURES = {
    "hbf_init_grid": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p]),
    "hbf_set_rheology": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int]),
    "hbf_set_density": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "hbf_set_body_force": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "hbf_set_predictor_viscous": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_set_solver": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int]),
    "hbf_set_tail": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_set_fused_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_set_staged_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hbf_set_staged_op": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hbf_set_inner_drop": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "hbf_set_split_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_field_size": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_set_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "hbf_get_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "hbf_compute_viscosity": (ctypes.c_int, [ctypes.c_void_p]),
    "hbf_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "hbf_mac_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SolveStats)]),
    "hbf_advect_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "hbf_solve_viscous": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(SolveStats)]),
    "hbf_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(SolveStats)]),
    "hbf_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(StepStats)]),
    "hbf_cfl_dt": (ctypes.c_double, [ctypes.c_void_p, ctypes.c_double]),
    "hbf_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "hbf_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "hbf_cfl_dt_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_unet_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]),
    "hbf_unet_destroy": (None, [ctypes.c_void_p]),
    "hbf_unet_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hbf_unet_param_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "hbf_unet_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_unet_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_unet_get_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_unet_set_tensor_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_unet_tensor_status": (ctypes.c_int, [ctypes.c_void_p]),
    "hbf_unet_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_unet_loss": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double)]),
    "hbf_unet_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_unet_zero_grads": (ctypes.c_int, [ctypes.c_void_p]),
    "hbf_unet_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double]),
    "hbf_set_guess_model": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_set_guess_model_level": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "hbf_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_set_walls": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "hbf_step_change": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "hbf_yield": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(YieldInfo), ctypes.c_void_p]),
    "hbf_run_steady": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                      ctypes.POINTER(RunInfo)]),
    "hbf_run_cessation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                         ctypes.POINTER(RunInfo)]),
    "hbf_set_theta": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "hbf_set_periodic": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "hbf_centreline": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "hbf_vortex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]),
    "hbf_set_visc_guess": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_set_visc_guess_model": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "hbf_set_visc_record": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_restrict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "hbf_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "hbf_destroy": (None, [ctypes.c_void_p]),
    "hbf_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p]),
    "hbf_batch_destroy": (None, [ctypes.c_void_p]),
    "hbf_batch_cavity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "hbf_batch_set_dt": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "hbf_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hbf_batch_set_tiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "hbf_batch_set_tail": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_batch_get_tiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]),
    "hbf_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "hbf_batch_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hbf_batch_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "hbf_batch_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "hbf_batch_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "hbf_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}


def load(path=LIB_PATH):
    """Load the shared library and declare every exported signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"hbflow CUDA library not built ({path}); run paper_1803_00417_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HBFlowError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hbflow error {code}: {msg}")
        self.code = code


def to_device_layout(arrs):
    """List of numpy arrays indexed [i, j(, k)] -> flat x-fastest array."""
    if isinstance(arrs, np.ndarray):
        arrs = [arrs]
    return np.concatenate([np.ascontiguousarray(np.asarray(a, dtype=np.float64).T).ravel() for a in arrs])


def from_device_layout(flat, shape, ncomp):
    """Flat x-fastest array -> list of ``ncomp`` numpy arrays of ``shape``."""
    n = int(np.prod(shape))
    return [np.ascontiguousarray(flat[c * n:(c + 1) * n].reshape(shape[::-1]).T) for c in range(ncomp)]


def _ptr(x):
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        assert x.dtype in (np.float64, np.int32) and x.flags.c_contiguous
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(int(x))


class HBFlow:
    """One context of the library: a box of ``n`` cells of size ``h`` with wall
    velocities ``wall_u[a][s][c]`` (all faces are no-slip walls)."""

    def __init__(self, n, h, wall_u=None, precision=FP64, stream=None):
        self.lib = load()
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        self.h = float(h)
        nn = (ctypes.c_int64 * 3)(*(list(self.n) + [1] * (3 - self.d)))
        wu = np.zeros((3, 2, 3))
        if wall_u is not None:
            w = np.asarray(wall_u, dtype=np.float64).reshape(self.d, 2, self.d)
            wu[:self.d, :, :self.d] = w
        wuc = (ctypes.c_double * 18)(*wu.ravel())
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = stream
        ctx = ctypes.c_void_p()
        st = self.lib.hbf_init_grid(ctypes.byref(ctx), self.d, nn, self.h, wuc, int(precision),
                                    ctypes.c_void_p(stream))
        if st != HBF_OK:
            raise HBFlowError(st, "hbf_init_grid failed")
        self.ctx = ctx
        self._owned = True
        self.ncell = int(np.prod(self.n))
        self.node_shape = tuple(v + 1 for v in self.n)

    @classmethod
    def _borrow(cls, lib, ctx, n, h):
        """A view of a context owned by someone else (a batch's cavity)."""
        self = cls.__new__(cls)
        self.lib = lib
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        self.h = float(h)
        self.ctx = ctx
        self._owned = False
        self.ncell = int(np.prod(self.n))
        self.node_shape = tuple(v + 1 for v in self.n)
        return self

    def close(self):
        if getattr(self, "ctx", None):
            if getattr(self, "_owned", True):
                self.lib.hbf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow_nc=False):
        if st == HBF_OK or (allow_nc and st == HBF_ERR_NOT_CONVERGED):
            return st
        raise HBFlowError(st, self.lib.hbf_last_error(self.ctx).decode())

    # ---- configuration ------------------------------------------------------------
    def set_rheology(self, K, n, tau_y, m, reg_power=True):
        self._check(self.lib.hbf_set_rheology(self.ctx, K, n, tau_y, m, int(bool(reg_power))))

    def set_density(self, rho):
        self._check(self.lib.hbf_set_density(self.ctx, rho))

    def set_body_force(self, f):
        ff = (ctypes.c_double * 3)(*(list(f) + [0.0] * (3 - len(f))))
        self._check(self.lib.hbf_set_body_force(self.ctx, ff))

    def set_visc_guess(self, mode):
        self._check(self.lib.hbf_set_visc_guess(self.ctx, int(mode)))

    def set_visc_record(self, on):
        self._check(self.lib.hbf_set_visc_record(self.ctx, int(bool(on))))

    def restrict(self, kind, level, src_dev, dst_dev):
        """One level of the multigrid restriction (kind 0 cell vector, 1 cell
        scalar, 2 nodes) of device arrays."""
        self._check(self.lib.hbf_restrict(self.ctx, int(kind), int(level), _ptr(src_dev), _ptr(dst_dev)))

    def set_theta(self, theta):
        self._check(self.lib.hbf_set_theta(self.ctx, float(theta)))

    def set_periodic(self, periodic):
        per = (ctypes.c_int * 3)(*([int(bool(v)) for v in periodic] + [0] * (3 - len(periodic))))
        self._check(self.lib.hbf_set_periodic(self.ctx, per))

    def set_predictor_viscous(self, on):
        self._check(self.lib.hbf_set_predictor_viscous(self.ctx, int(bool(on))))

    def set_solver(self, rtol=1e-10, max_cycles=200, nu1=2, nu2=2, nu_bottom=40):
        self._check(self.lib.hbf_set_solver(self.ctx, rtol, max_cycles, nu1, nu2, nu_bottom))

    def set_fused_sweep(self, on):
        self._check(self.lib.hbf_set_fused_sweep(self.ctx, int(bool(on))))

    def set_staged_sweep(self, tile_x, tile_z=16):
        """TMA-staged finest-level viscous sweeps (tile_x 64 or 128; 0 off)."""
        self._check(self.lib.hbf_set_staged_sweep(self.ctx, int(tile_x), int(tile_z)))

    def set_inner_drop(self, drop):
        """Residual drop of each FP32 BiCGStab pass of the mixed viscous solve."""
        self._check(self.lib.hbf_set_inner_drop(self.ctx, float(drop)))

    def set_split_layout(self, on):
        """Colour-split layout of the FP32 finest-level vectors of the mixed
        viscous solve (1, the default where it applies) or the natural one (0)."""
        self._check(self.lib.hbf_set_split_layout(self.ctx, int(on)))

    def set_staged_op(self, rows, tile_z=16):
        """TMA-staged finest-level viscous operator (rows 4 or 8; 0 off)."""
        self._check(self.lib.hbf_set_staged_op(self.ctx, int(rows), int(tile_z)))

    def set_tail(self, max_cells):
        """Levels from the first one with at most max_cells cells run as one
        fused launch per V-cycle (0: none)."""
        self._check(self.lib.hbf_set_tail(self.ctx, int(max_cells)))

    # ---- fields -------------------------------------------------------------------
    def field_size(self, which):
        return int(self.lib.hbf_field_size(self.ctx, FIELDS[which]))

    def set_field(self, which, src):
        """src: flat float64 numpy array (host) or torch CUDA tensor (device)."""
        self._check(self.lib.hbf_set_field(self.ctx, FIELDS[which], _ptr(src)))
        self.sync()

    def get_field(self, which, dst=None):
        if dst is None:
            dst = np.empty(self.field_size(which), dtype=np.float64)
        self._check(self.lib.hbf_get_field(self.ctx, FIELDS[which], _ptr(dst)))
        self.sync()
        return dst

    def set_velocity(self, u):
        self.set_field("U", to_device_layout(u))

    def set_pressure(self, p):
        self.set_field("P", to_device_layout(p))

    def velocity(self, which="U"):
        return from_device_layout(self.get_field(which), self.n, self.d)

    def pressure(self):
        return from_device_layout(self.get_field("P"), self.node_shape, 1)[0]

    def cell_scalar(self, which):
        return from_device_layout(self.get_field(which), self.n, 1)[0]

    def face_field(self, which, ncomp):
        """Face arrays per axis a (list over a of lists over components)."""
        flat = self.get_field(which)
        out, off = [], 0
        for a in range(self.d):
            shape = tuple(self.n[b] + (1 if b == a else 0) for b in range(self.d))
            cnt = int(np.prod(shape)) * ncomp
            out.append(from_device_layout(flat[off:off + cnt], shape, ncomp))
            off += cnt
        return out

    # ---- stages -------------------------------------------------------------------
    def compute_viscosity(self):
        self._check(self.lib.hbf_compute_viscosity(self.ctx))

    def predict(self, dt):
        self._check(self.lib.hbf_predict(self.ctx, dt))

    def mac_project(self):
        s = SolveStats()
        self._check(self.lib.hbf_mac_project(self.ctx, ctypes.byref(s)), allow_nc=True)
        return s.as_dict()

    def advect_rhs(self, dt):
        self._check(self.lib.hbf_advect_rhs(self.ctx, dt))

    def solve_viscous(self, dt, rhs_dev, u_dev):
        s = SolveStats()
        self._check(self.lib.hbf_solve_viscous(self.ctx, dt, _ptr(rhs_dev), _ptr(u_dev), ctypes.byref(s)),
                    allow_nc=True)
        return s.as_dict()

    def project(self, dt, u_dev, p_dev):
        s = SolveStats()
        self._check(self.lib.hbf_project(self.ctx, dt, _ptr(u_dev), _ptr(p_dev), ctypes.byref(s)), allow_nc=True)
        return s.as_dict()

    def step(self, dt):
        s = StepStats()
        self._check(self.lib.hbf_step(self.ctx, dt, ctypes.byref(s)), allow_nc=True)
        return s.as_dict()

    def cfl_dt(self, cfl):
        return float(self.lib.hbf_cfl_dt(self.ctx, cfl))

    # ---- checkpoint, walls and the start-up / steady / cessation study -----------
    def get_state(self, with_fields=True):
        """(record dict, flat U, flat P) of hbf_get_state."""
        s = State()
        u = np.empty(self.d * self.ncell) if with_fields else None
        p = np.empty(int(np.prod(self.node_shape))) if with_fields else None
        self._check(self.lib.hbf_get_state(self.ctx, ctypes.byref(s), _ptr(u) if u is not None else None,
                                           _ptr(p) if p is not None else None))
        return s.as_dict(), u, p

    def set_state(self, record, u=None, p=None):
        s = State.from_dict(record)
        self._check(self.lib.hbf_set_state(self.ctx, ctypes.byref(s), _ptr(u) if u is not None else None,
                                           _ptr(p) if p is not None else None))

    def save_checkpoint(self, path):
        """``path``.json (the record) and ``path``.bin (U then P, float64)."""
        import json
        rec, u, p = self.get_state()
        with open(path + ".json", "w") as f:
            json.dump(rec, f)
        np.concatenate([u, p]).tofile(path + ".bin")

    def load_checkpoint(self, path):
        import json
        with open(path + ".json") as f:
            rec = json.load(f)
        data = np.fromfile(path + ".bin", dtype=np.float64)
        nu = self.d * self.ncell
        self.set_state(rec, np.ascontiguousarray(data[:nu]), np.ascontiguousarray(data[nu:]))
        return rec

    def set_walls(self, wall_u):
        wu = np.zeros((3, 2, 3))
        w = np.asarray(wall_u, dtype=np.float64).reshape(self.d, 2, self.d)
        wu[:self.d, :, :self.d] = w
        self._check(self.lib.hbf_set_walls(self.ctx, (ctypes.c_double * 18)(*wu.ravel())))

    def step_change(self):
        v = ctypes.c_double()
        self._check(self.lib.hbf_step_change(self.ctx, ctypes.byref(v)))
        return v.value

    def yield_info(self, labels=False):
        info = YieldInfo()
        lab = np.empty(self.ncell, dtype=np.int32) if labels else None
        self._check(self.lib.hbf_yield(self.ctx, ctypes.byref(info), _ptr(lab) if labels else None))
        out = info.as_dict()
        if labels:
            out["labels"] = from_device_layout(lab, self.n, 1)[0]
        return out

    def run_steady(self, dt, tol=1e-5, max_steps=100000):
        r = RunInfo()
        self._check(self.lib.hbf_run_steady(self.ctx, dt, tol, int(max_steps), ctypes.byref(r)))
        return r.as_dict()

    def run_cessation(self, dt, max_steps=100000, damp_steps=0):
        r = RunInfo()
        self._check(self.lib.hbf_run_cessation(self.ctx, dt, int(max_steps), int(damp_steps), ctypes.byref(r)))
        return r.as_dict()

    def centreline(self, comp, along):
        out = np.empty(self.n[along])
        self._check(self.lib.hbf_centreline(self.ctx, int(comp), int(along), _ptr(out)))
        return out

    def vortex(self, with_psi=False):
        """(x, y) of the primary vortex centre in the centre plane, psi there,
        and optionally psi on the plane's nodes (array indexed [a, b])."""
        na = self.n[0]
        nb = self.n[2] if self.d == 3 else self.n[1]
        psi = np.empty((na + 1) * (nb + 1)) if with_psi else None
        c = (ctypes.c_double * 2)()
        pc = ctypes.c_double()
        self._check(self.lib.hbf_vortex(self.ctx, _ptr(psi) if with_psi else None, c, ctypes.byref(pc)))
        out = dict(centre=(c[0], c[1]), psi=pc.value)
        if with_psi:
            out["field"] = psi.reshape(nb + 1, na + 1).T
        return out

    PROFILE_SLOTS = dict(visc_smooth=0, visc_resid=1, nodal_smooth=2, nodal_resid=3, mac_smooth=4,
                         mac_resid=5, explicit=6, bottom=7, transfer=8, reduce=9, vector=10, coarse=11,
                         guess=12)

    def profile_enable(self, level=1):
        """0 off, 1 finest-level solver kernels and explicit stages, 2 also
        bottom solves, transfers, reductions, vector updates, coarse levels."""
        self._check(self.lib.hbf_profile_enable(self.ctx, int(level)))

    def profile_read(self, slot):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self.lib.hbf_profile_read(self.ctx, self.PROFILE_SLOTS[slot], ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def launch_count(self):
        return int(self.lib.hbf_launch_count(self.ctx))

    def sync(self):
        self._check(self.lib.hbf_sync(self.ctx))


class UNet:
    """The learned initial-guess network (hbf_unet_*): a box of ``n`` points
    (each a multiple of 8).  Arrays passed in are torch CUDA float32 tensors of
    one value per point, x fastest."""

    def __init__(self, n, train=False, seed=0, stream=None):
        self.lib = load()
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        nn = (ctypes.c_int64 * 3)(*(list(self.n) + [1] * (3 - self.d)))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        net = ctypes.c_void_p()
        st = self.lib.hbf_unet_create(ctypes.byref(net), self.d, nn, int(bool(train)), int(seed),
                                      ctypes.c_void_p(stream))
        if st != HBF_OK:
            raise HBFlowError(st, "hbf_unet_create failed")
        self.net = net
        self.points = int(np.prod(self.n))

    def close(self):
        if getattr(self, "net", None):
            self.lib.hbf_unet_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != HBF_OK:
            raise HBFlowError(st, self.lib.hbf_unet_last_error(self.net).decode())

    def param_count(self):
        return int(self.lib.hbf_unet_param_count(self.net))

    def get_params(self):
        out = np.empty(self.param_count(), dtype=np.float32)
        self._check(self.lib.hbf_unet_get_params(self.net, ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self.lib.hbf_unet_set_params(self.net, ctypes.c_void_p(flat.ctypes.data)))

    def get_grads(self):
        out = np.empty(self.param_count(), dtype=np.float32)
        self._check(self.lib.hbf_unet_get_grads(self.net, ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_tensor_path(self, path):
        """0: mma.sync convolutions, 1: tcgen05 (TMEM accumulators)."""
        self._check(self.lib.hbf_unet_set_tensor_path(self.net, int(path)))

    def tensor_status(self):
        self._check(self.lib.hbf_unet_tensor_status(self.net))

    def forward(self, x_dev, y_dev=None):
        self._check(self.lib.hbf_unet_forward(self.net, _ptr(x_dev), _ptr(y_dev) if y_dev is not None else None))

    def loss(self, t_dev, mask_dev, gy_dev):
        v = ctypes.c_double()
        self._check(self.lib.hbf_unet_loss(self.net, _ptr(t_dev), _ptr(mask_dev), _ptr(gy_dev), ctypes.byref(v)))
        return v.value

    def backward(self, gy_dev):
        self._check(self.lib.hbf_unet_backward(self.net, _ptr(gy_dev)))

    def zero_grads(self):
        self._check(self.lib.hbf_unet_zero_grads(self.net))

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.hbf_unet_adam(self.net, lr, beta1, beta2, eps))


def set_visc_guess_model(sim, net, level=0):
    """Use ``net`` (a UNet, or None) for the viscous solve's learned direction
    (guess mode 2), evaluated on the cells of multigrid level ``level``."""
    st = sim.lib.hbf_set_visc_guess_model(sim.ctx, net.net if net is not None else None, int(level))
    sim._check(st)


def set_guess_model(sim, net, level=0):
    """Use ``net`` (a UNet, or None) for the nodal projection's initial guess,
    evaluated on the nodes of multigrid level ``level`` (0 = finest)."""
    st = sim.lib.hbf_set_guess_model_level(sim.ctx, net.net if net is not None else None, int(level))
    sim._check(st)


class Batch:
    """Many independent cavities advanced together (``hbf_batch_*``): ``ns`` is a
    list of cell counts (all of one dimension), ``hs`` their cell sizes,
    ``wall_us`` their wall velocities (as for :class:`HBFlow`, or None).  Each
    cavity is configured through :meth:`cavity`, which returns a borrowed
    :class:`HBFlow` view."""

    def __init__(self, ns, hs, wall_us=None, precision=FP64, stream=None):
        self.lib = load()
        self.ns = [tuple(int(v) for v in n) for n in ns]
        self.d = len(self.ns[0])
        assert all(len(n) == self.d for n in self.ns)
        self.hs = [float(h) for h in hs]
        k = len(self.ns)
        nn = (ctypes.c_int64 * (3 * k))(*[v for n in self.ns for v in (list(n) + [1] * (3 - self.d))])
        hh = (ctypes.c_double * k)(*self.hs)
        wu = np.zeros((k, 3, 2, 3))
        if wall_us is not None:
            for i, w in enumerate(wall_us):
                if w is not None:
                    wu[i, :self.d, :, :self.d] = np.asarray(w, dtype=np.float64).reshape(self.d, 2, self.d)
        wuc = (ctypes.c_double * (18 * k))(*wu.ravel())
        b = ctypes.c_void_p()
        st = self.lib.hbf_batch_create(ctypes.byref(b), self.d, k, nn, hh, wuc, int(precision),
                                       ctypes.c_void_p(stream) if stream is not None else None)
        if st != HBF_OK:
            raise HBFlowError(st, "hbf_batch_create failed")
        self.b = b
        self.ncav = k
        self._views = []
        for i in range(k):
            c = ctypes.c_void_p()
            self._check(self.lib.hbf_batch_cavity(self.b, i, ctypes.byref(c)))
            self._views.append(HBFlow._borrow(self.lib, c, self.ns[i], self.hs[i]))

    def close(self):
        if getattr(self, "b", None):
            for v in self._views:
                v.ctx = None
            self.lib.hbf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow_nc=False):
        if st == HBF_OK or (allow_nc and st == HBF_ERR_NOT_CONVERGED):
            return st
        raise HBFlowError(st, self.lib.hbf_batch_last_error(self.b).decode())

    def cavity(self, i):
        return self._views[i]

    def set_dt(self, dts):
        arr = (ctypes.c_double * self.ncav)(*[float(x) for x in dts])
        self._check(self.lib.hbf_batch_set_dt(self.b, arr))

    def step(self):
        """One step of every cavity; returns the per-cavity solver statistics."""
        stats = (StepStats * self.ncav)()
        self._check(self.lib.hbf_batch_step(self.b, ctypes.cast(stats, ctypes.c_void_p)), allow_nc=True)
        return [s.as_dict() for s in stats]

    def set_tiling(self, tile, blocks_per_sm):
        self._check(self.lib.hbf_batch_set_tiling(self.b, int(tile), int(blocks_per_sm)))

    def set_tail(self, max_cells):
        """Fuse the levels with at most ``max_cells`` cells per cavity (0: off)."""
        self._check(self.lib.hbf_batch_set_tail(self.b, int(max_cells)))

    def tiling(self):
        t, b, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        self._check(self.lib.hbf_batch_get_tiling(self.b, ctypes.byref(t), ctypes.byref(b), ctypes.byref(n)))
        return dict(tile=t.value, blocks_per_sm=b.value, tiles_level0=n.value)

    def autotune(self, reps=3):
        t, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.hbf_batch_autotune(self.b, int(reps), ctypes.byref(t), ctypes.byref(b),
                                                ctypes.byref(ms)))
        return dict(tile=t.value, blocks_per_sm=b.value, probe_ms=ms.value)

    PHASES = ("explicit_pre", "mac_solve", "explicit_post", "viscous_solve", "nodal_rhs", "nodal_solve",
              "update")

    def profile(self, on=True):
        """Start (and reset) or stop phase timing of the following steps."""
        self._check(self.lib.hbf_batch_profile(self.b, int(bool(on))))

    def profile_read(self):
        ms = (ctypes.c_double * 7)()
        trips = (ctypes.c_int64 * 3)()
        steps = ctypes.c_int64()
        self._check(self.lib.hbf_batch_profile_read(self.b, ms, trips, ctypes.byref(steps)))
        return dict(steps=steps.value, phase_ms=dict(zip(self.PHASES, list(ms))),
                    loop_trips=dict(zip(("mac", "visc", "nodal"), list(trips))))

    def launch_count(self):
        return int(self.lib.hbf_batch_launch_count(self.b))

    def sync(self):
        self._check(self.lib.hbf_batch_sync(self.b))
