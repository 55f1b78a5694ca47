"""ctypes binding of the C ABI declared in include/qttpdip.h.

Argument marshalling only: every computation runs in the CUDA library.  Device
buffers are torch CUDA tensors (PyTorch provides device memory and streams);
their data pointers and the current CUDA stream are handed to the C calls.
Importing this module never falls back to anything: if the shared library is
missing, `load()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqttpdip.so")

QP_OK, QP_INVALID_ARG, QP_OOM, QP_CUDA_ERROR = 0, -1, -2, -3
QP_NOT_CONVERGED, QP_BREAKDOWN, QP_LINESEARCH_FAIL, QP_TIMEOUT, QP_NOT_READY = -4, -5, -6, -7, -8
QP_F64, QP_F32, QP_BF16 = 0, 1, 2
QP_JACOBI_PCG, QP_QTT_PCG, QP_QTT_DIRECT = 0, 1, 2
QP_CG, QP_BICGSTAB = 0, 1
QTT_NOALLOC_MAX_VALUES = 1 << 22

SYMBOLS = ["qp_create", "qp_destroy", "qp_status_string", "qp_last_error", "ccp_assemble", "pdip_init",
           "newton_apply", "newton_rhs", "newton_solve", "newton_solve_batched", "newton_batch_plan", "newton_batch_qtt_tiles", "pdip_step", "pdip_measure", "pdip_solve", "pdip_init_warm",
           "ccp_advance", "qp_selftest_barrier", "mpnn_forward", "mpnn_grad", "mpnn_adam", "mpnn_warm_start", "qtt_from_host",
           "qtt_free", "qtt_get_dims", "qtt_get_ranks", "qtt_copy_cores_to_host", "qtt_apply", "qtt_set_tensor_cores",
           "qtt_round",
           "qtt_compress", "qtt_inverse", "qtt_apply_f32_noalloc"]


class Scene(C.Structure):
    _fields_ = [("M", C.c_int), ("pos", C.c_void_p), ("vel", C.c_void_p), ("omega", C.c_void_p),
                ("radius", C.c_void_p), ("inv_mass", C.c_void_p), ("inv_inertia", C.c_void_p),
                ("floor_z", C.c_double), ("gravity", C.c_double * 3), ("dt", C.c_double), ("delta", C.c_double),
                ("mu", C.c_double), ("slots", C.c_int), ("nwalls", C.c_int), ("wall_axis", C.c_int * 4),
                ("wall_sign", C.c_int * 4), ("wall_offset", C.c_double * 4)]


class Contacts(C.Structure):
    _fields_ = [("M", C.c_int), ("Nc", C.c_int), ("L", C.c_int), ("slots", C.c_int), ("P", C.c_longlong),
                ("body_a", C.c_void_p), ("body_b", C.c_void_p), ("phi", C.c_void_p), ("frame", C.c_void_p),
                ("point", C.c_void_p), ("arm_a", C.c_void_p), ("arm_b", C.c_void_p), ("key", C.c_void_p),
                ("r", C.c_void_p), ("plane", C.c_void_p)]


class State(C.Structure):
    _fields_ = [("gamma", C.c_void_p), ("lam", C.c_void_p), ("t", C.c_double)]


class BatchOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("inner_tol", C.c_double), ("max_outer", C.c_int),
                ("block_threads", C.c_int), ("split", C.c_int), ("precond", C.c_void_p), ("core_dtype", C.c_int),
                ("qtt_tile", C.c_int)]


class PrevContacts(C.Structure):
    _fields_ = [("Nc", C.c_int), ("slots", C.c_int), ("body_a", C.c_void_p), ("body_b", C.c_void_p),
                ("gamma", C.c_void_p), ("plane", C.c_void_p)]


class SolveOpts(C.Structure):
    _fields_ = [("precond", C.c_int), ("X", C.c_void_p), ("tol", C.c_double), ("maxit", C.c_int),
                ("mixed", C.c_int), ("inner_tol", C.c_double), ("max_outer", C.c_int), ("core_dtype", C.c_int),
                ("krylov", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("outer", C.c_int), ("rel_res", C.c_double),
                ("ms", C.c_double), ("fallback", C.c_int)]


class PdipOpts(C.Structure):
    _fields_ = [("nu", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("step_frac", C.c_double),
                ("max_halvings", C.c_int), ("solve", SolveOpts), ("qtt_refresh", C.c_int),
                ("qtt_eps", C.c_double), ("qtt_rmax", C.c_int)]


class PdipStats(C.Structure):
    _fields_ = [("status", C.c_int), ("eta", C.c_double), ("t", C.c_double), ("r_dual", C.c_double),
                ("r_t", C.c_double), ("s", C.c_double), ("halvings", C.c_int), ("solve", SolveStats),
                ("ms_refresh", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (built by build.build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_1808_02558_gb300.build.build())")
    lib = C.CDLL(path)
    vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "qp_create": (i, [C.POINTER(vp), i, vp]),
        "qp_destroy": (i, [vp]),
        "qp_status_string": (C.c_char_p, [i]),
        "qp_last_error": (i, [vp, C.c_char_p, i]),
        "ccp_assemble": (i, [vp, C.POINTER(Scene), C.POINTER(Contacts)]),
        "pdip_init": (i, [vp, C.POINTER(State), d]),
        "newton_apply": (i, [vp, C.POINTER(State), vp, vp, i]),
        "newton_rhs": (i, [vp, C.POINTER(State), vp]),
        "newton_solve": (i, [vp, C.POINTER(State), vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveStats)]),
        "pdip_step": (i, [vp, C.POINTER(State), C.POINTER(PdipOpts), C.POINTER(PdipStats)]),
        "pdip_measure": (i, [vp, C.POINTER(State), C.POINTER(d), C.POINTER(d)]),
        "pdip_solve": (i, [vp, C.POINTER(State), C.POINTER(PdipOpts), d, d, i, C.POINTER(PdipStats), C.POINTER(i)]),
        "pdip_init_warm": (i, [vp, C.POINTER(State), C.POINTER(PrevContacts), d, d]),
        "newton_solve_batched": (i, [i, C.POINTER(vp), C.POINTER(C.POINTER(State)), C.POINTER(vp), C.POINTER(vp),
                                     C.POINTER(BatchOpts), C.POINTER(SolveStats), C.POINTER(i)]),
        "newton_batch_plan": (i, [i, C.POINTER(ll), i, i, C.POINTER(i), C.POINTER(i)]),
        "newton_batch_qtt_tiles": (i, [vp, i, C.POINTER(i)]),
        "ccp_advance": (i, [vp, C.POINTER(Scene), C.POINTER(State), vp, vp, vp]),
        "qp_selftest_barrier": (i, [vp, ll, i, C.POINTER(i)]),
        "mpnn_forward": (i, [vp, vp, C.POINTER(C.c_float), vp]),
        "mpnn_grad": (i, [vp, vp, C.POINTER(C.c_float), vp, vp, C.POINTER(d)]),
        "mpnn_adam": (i, [vp, vp, vp, vp, vp, i, d, d, d, d]),
        "mpnn_warm_start": (i, [vp, C.POINTER(State), vp, d, d, d]),
        "qtt_from_host": (i, [vp, i, C.POINTER(i), C.POINTER(d), C.POINTER(vp)]),
        "qtt_free": (i, [vp, vp]),
        "qtt_get_dims": (i, [vp, C.POINTER(i), C.POINTER(ll)]),
        "qtt_get_ranks": (i, [vp, C.POINTER(i)]),
        "qtt_copy_cores_to_host": (i, [vp, C.POINTER(d)]),
        "qtt_apply": (i, [vp, vp, vp, vp, i, i]),
        "qtt_set_tensor_cores": (i, [vp, i]),
        "qtt_round": (i, [vp, vp, d, i, C.POINTER(vp)]),
        "qtt_compress": (i, [vp, C.POINTER(State), d, i, C.POINTER(vp)]),
        "qtt_inverse": (i, [vp, vp, d, i, i, vp, C.POINTER(vp)]),
        "qtt_apply_f32_noalloc": (i, [i, C.POINTER(i), vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def qtt_apply_f32_noalloc(ranks: list, cores, x, y, stream=None) -> int:
    """Context-free, allocation-free y = A x (float32 cores and vectors); returns the status.

    The C entry point sees raw device pointers only, so the buffer sizes are
    checked here: x and y hold 2^d float32 values, cores holds
    sum_k r_{k-1} * 4 * r_k float32 values, all contiguous CUDA tensors."""
    import torch

    lib = load()
    d = len(ranks) - 1
    if d < 1 or any(int(v) < 1 for v in ranks):
        raise ValueError("ranks must be d + 1 >= 2 positive integers")
    need = sum(int(ranks[k]) * 4 * int(ranks[k + 1]) for k in range(d))
    for name, t, n in (("cores", cores, need), ("x", x, 1 << d), ("y", y, 1 << d)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
        if t.numel() != n:
            raise ValueError(f"{name} has {t.numel()} values, expected {n}")
    r = (C.c_int * (d + 1))(*ranks)
    s = torch.cuda.current_stream() if stream is None else stream
    return lib.qtt_apply_f32_noalloc(d, r, C.c_void_p(cores.data_ptr()), C.c_void_p(x.data_ptr()),
                                     C.c_void_p(y.data_ptr()), C.c_void_p(s.cuda_stream))


class QPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _ptr(t) -> int:
    return int(t.data_ptr())


class QTT:
    """Handle to a context-owned QTT matrix."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.h = C.c_void_p(handle)

    @property
    def d(self) -> int:
        dd, nv = C.c_int(), C.c_longlong()
        self.ctx.lib.qtt_get_dims(self.h, C.byref(dd), C.byref(nv))
        return dd.value

    def ranks(self) -> list:
        r = (C.c_int * (self.d + 1))()
        self.ctx.lib.qtt_get_ranks(self.h, r)
        return list(r)

    def cores(self) -> list:
        """Cores as numpy arrays of shape (r_k, 4, r_{k+1})."""
        dd, nv = C.c_int(), C.c_longlong()
        self.ctx.lib.qtt_get_dims(self.h, C.byref(dd), C.byref(nv))
        buf = np.empty(nv.value, dtype=np.float64)
        self.ctx._check(self.ctx.lib.qtt_copy_cores_to_host(self.h, buf.ctypes.data_as(C.POINTER(C.c_double))),
                        "qtt_copy_cores_to_host")
        r = self.ranks()
        out, off = [], 0
        for k in range(dd.value):
            n = r[k] * 4 * r[k + 1]
            out.append(buf[off:off + n].reshape(r[k], 4, r[k + 1]).copy())
            off += n
        return out

    def free(self):
        if self.h and self.h.value:
            self.ctx.lib.qtt_free(self.ctx.h, self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """One library context on the current CUDA device and stream."""

    def __init__(self, device: int | None = None, stream=None):
        import torch

        self.lib = load()
        self.device = torch.cuda.current_device() if device is None else device
        s = torch.cuda.current_stream(self.device) if stream is None else stream
        self.stream = s
        h = C.c_void_p()
        self._check(self.lib.qp_create(C.byref(h), self.device, C.c_void_p(s.cuda_stream)), "qp_create", ctx=False)
        self.h = h
        self.contacts = None

    def _check(self, rc: int, what: str, ctx: bool = True, allow=()):
        if rc != QP_OK and rc not in allow:
            msg = ""
            if ctx:
                buf = C.create_string_buffer(512)
                self.lib.qp_last_error(self.h, buf, 512)
                msg = buf.value.decode()
            raise QPError(rc, f"{what}: {self.lib.qp_status_string(rc).decode()} {msg}")
        return rc

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.qp_destroy(self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- assembly
    def assemble(self, scene_dev: dict, floor_z, gravity, dt, delta, mu, slots=3, walls=()) -> Contacts:
        """scene_dev: dict of device float64 tensors pos/vel/omega (3, M) SoA and radius/inv_mass/inv_inertia (M,);
        walls: up to four side walls (axis, sign, offset)."""
        M = int(scene_dev["radius"].shape[0])
        walls = list(walls)
        ax = [int(w[0]) for w in walls] + [0] * (4 - len(walls))
        sg = [int(w[1]) for w in walls] + [1] * (4 - len(walls))
        off = [float(w[2]) for w in walls] + [0.0] * (4 - len(walls))
        sc = Scene(M, _ptr(scene_dev["pos"]), _ptr(scene_dev["vel"]), _ptr(scene_dev["omega"]),
                   _ptr(scene_dev["radius"]), _ptr(scene_dev["inv_mass"]), _ptr(scene_dev["inv_inertia"]),
                   float(floor_z), (C.c_double * 3)(*gravity), float(dt), float(delta), float(mu), int(slots),
                   len(walls), (C.c_int * 4)(*ax[:4]), (C.c_int * 4)(*sg[:4]), (C.c_double * 4)(*off[:4]))
        out = Contacts()
        self._check(self.lib.ccp_assemble(self.h, C.byref(sc), C.byref(out)), "ccp_assemble")
        self.contacts = out
        self.scene = (sc, scene_dev)
        return out

    def advance(self, st: State):
        """One time step of the assembled scene with impulses st.gamma; updates the
        scene's device tensors (pos, vel, omega) in place."""
        sc, dev = self.scene
        self._check(self.lib.ccp_advance(self.h, C.byref(sc), C.byref(st), _ptr(dev["pos"]), _ptr(dev["vel"]),
                                         _ptr(dev["omega"])), "ccp_advance")

    def selftest_barrier(self, budget: int, absent_block: int) -> int:
        """Device status of a cooperative launch in which one block skips the grid barrier."""
        status = C.c_int(0)
        self._check(self.lib.qp_selftest_barrier(self.h, int(budget), int(absent_block), C.byref(status)),
                    "qp_selftest_barrier")
        return status.value

    # ------------------------------------------------------------- learned warm start
    def mpnn_forward(self, params, feat_scale, out):
        sc = (C.c_float * 8)(*[float(v) for v in feat_scale])
        self._check(self.lib.mpnn_forward(self.h, _ptr(params), sc, _ptr(out) if out.numel() else None),
                    "mpnn_forward")

    def mpnn_grad(self, params, feat_scale, target, grad) -> float:
        sc = (C.c_float * 8)(*[float(v) for v in feat_scale])
        loss = C.c_double(0.0)
        self._check(self.lib.mpnn_grad(self.h, _ptr(params), sc, _ptr(target), _ptr(grad), C.byref(loss)),
                    "mpnn_grad")
        return loss.value

    def mpnn_adam(self, params, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.mpnn_adam(self.h, _ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr),
                                       float(beta1), float(beta2), float(eps)), "mpnn_adam")

    def mpnn_warm_start(self, st: State, out, out_scale, gn_min=1e-3, shrink=0.9):
        self._check(self.lib.mpnn_warm_start(self.h, C.byref(st), _ptr(out) if out.numel() else None,
                                             float(out_scale), float(gn_min), float(shrink)), "mpnn_warm_start")

    def pdip_init_warm(self, st: State, prev_a, prev_b, prev_gamma, prev_slots=3, gn0=1.0, shrink=0.9,
                       prev_plane=None):
        """Warm start from the previous step's pairs and impulses (device tensors
        the caller copied before re-assembly); prev_plane: the previous contacts'
        plane indices (needed with walls), or None."""
        pc = PrevContacts(int(prev_a.numel()), int(prev_slots), _ptr(prev_a), _ptr(prev_b), _ptr(prev_gamma),
                          _ptr(prev_plane) if prev_plane is not None else None)
        self._check(self.lib.pdip_init_warm(self.h, C.byref(st), C.byref(pc), float(gn0), float(shrink)),
                    "pdip_init_warm")

    # ------------------------------------------------------------- PDIP / Newton
    @staticmethod
    def state(gamma, lam, t=1.0) -> State:
        return State(_ptr(gamma), _ptr(lam), float(t))

    def pdip_init(self, st: State, gn0: float = 1.0):
        self._check(self.lib.pdip_init(self.h, C.byref(st), float(gn0)), "pdip_init")

    def newton_apply(self, st, x, y, dtype=QP_F64):
        sp = C.byref(st) if st is not None else None
        self._check(self.lib.newton_apply(self.h, sp, _ptr(x), _ptr(y), dtype), "newton_apply")

    def newton_rhs(self, st: State, rhs):
        self._check(self.lib.newton_rhs(self.h, C.byref(st), _ptr(rhs)), "newton_rhs")

    @staticmethod
    def solve_opts(precond=QP_JACOBI_PCG, X=None, tol=1e-10, maxit=20000, mixed=0, inner_tol=0.0, max_outer=0,
                   core_dtype=QP_F32, krylov=QP_CG) -> SolveOpts:
        return SolveOpts(precond, X.h.value if X is not None else None, tol, maxit, mixed, inner_tol, max_outer,
                         core_dtype, krylov)

    def newton_solve(self, st, rhs, dx, opts: SolveOpts, allow=(QP_NOT_CONVERGED, QP_BREAKDOWN)) -> SolveStats:
        stats = SolveStats()
        sp = C.byref(st) if st is not None else None
        self._check(self.lib.newton_solve(self.h, sp, _ptr(rhs), _ptr(dx), C.byref(opts), C.byref(stats)),
                    "newton_solve", allow=allow)
        return stats

    @staticmethod
    def pdip_opts(solve: SolveOpts, nu=10.0, alpha=0.01, beta=0.5, step_frac=0.99, max_halvings=60, qtt_refresh=0,
                  qtt_eps=1e-2, qtt_rmax=10) -> PdipOpts:
        return PdipOpts(nu, alpha, beta, step_frac, max_halvings, solve, qtt_refresh, qtt_eps, qtt_rmax)

    def pdip_step(self, st: State, opts: PdipOpts, allow=(QP_NOT_CONVERGED,)) -> PdipStats:
        stats = PdipStats()
        self._check(self.lib.pdip_step(self.h, C.byref(st), C.byref(opts), C.byref(stats)), "pdip_step", allow=allow)
        return stats

    def pdip_solve(self, st: State, opts: PdipOpts, gap_tol=1e-8, dual_tol=1e-8, max_iter=200,
                   allow=(QP_NOT_CONVERGED,)):
        """PDIP loop to the given tolerances; returns (stats, steps taken)."""
        stats = PdipStats()
        n = C.c_int(0)
        self._check(self.lib.pdip_solve(self.h, C.byref(st), C.byref(opts), float(gap_tol), float(dual_tol),
                                        int(max_iter), C.byref(stats), C.byref(n)), "pdip_solve", allow=allow)
        return stats, n.value

    def pdip_measure(self, st: State):
        eta, rd = C.c_double(), C.c_double()
        self._check(self.lib.pdip_measure(self.h, C.byref(st), C.byref(eta), C.byref(rd)), "pdip_measure")
        return eta.value, rd.value

    # ------------------------------------------------------------- QTT
    def qtt_from_cores(self, cores: list) -> QTT:
        d = len(cores)
        ranks = [1] + [int(G.shape[2]) for G in cores]
        flat = np.concatenate([np.ascontiguousarray(G, dtype=np.float64).reshape(-1) for G in cores])
        h = C.c_void_p()
        r = (C.c_int * (d + 1))(*ranks)
        self._check(self.lib.qtt_from_host(self.h, d, r, flat.ctypes.data_as(C.POINTER(C.c_double)), C.byref(h)),
                    "qtt_from_host")
        return QTT(self, h.value)

    def qtt_apply(self, A: QTT, x, y, core_dtype=QP_F64, vec_dtype=QP_F64):
        self._check(self.lib.qtt_apply(self.h, A.h, _ptr(x), _ptr(y), core_dtype, vec_dtype), "qtt_apply")

    def batch_qtt_tiles(self, block_threads: int) -> list:
        """Measured tile shapes (1 or 2 column items per thread) of the batched QTT
        passes for input ranks <= 4, <= 8, <= 16 and above."""
        t = (C.c_int * 4)()
        self._check(self.lib.newton_batch_qtt_tiles(self.h, int(block_threads), t), "newton_batch_qtt_tiles")
        return list(t)

    def qtt_set_tensor_cores(self, mode: int):
        """0: CUDA-core steps only; 1: tensor cores for dense cores (default); 2: every core that qualifies."""
        self._check(self.lib.qtt_set_tensor_cores(self.h, int(mode)), "qtt_set_tensor_cores")

    def qtt_round(self, A: QTT, eps: float, rmax: int = 1 << 30) -> QTT:
        h = C.c_void_p()
        self._check(self.lib.qtt_round(self.h, A.h, float(eps), int(min(rmax, 2**31 - 1)), C.byref(h)), "qtt_round")
        return QTT(self, h.value)

    def qtt_compress(self, st, eps: float, rmax: int) -> QTT:
        h = C.c_void_p()
        sp = C.byref(st) if st is not None else None
        self._check(self.lib.qtt_compress(self.h, sp, float(eps), int(rmax), C.byref(h)), "qtt_compress")
        return QTT(self, h.value)

    def qtt_inverse(self, S: QTT, eps: float, rmax: int, sweeps: int = 4, warm: QTT | None = None) -> QTT:
        h = C.c_void_p()
        self._check(self.lib.qtt_inverse(self.h, S.h, float(eps), int(rmax), int(sweeps),
                                         warm.h if warm is not None else None, C.byref(h)), "qtt_inverse")
        return QTT(self, h.value)


def newton_solve_batched(ctxs, states, rhs, dx, tol=1e-8, maxit=100000, inner_tol=1e-3, max_outer=60,
                         block_threads=0, split=0, allow=(QP_NOT_CONVERGED, QP_BREAKDOWN), precond=None,
                         core_dtype=QP_F32, qtt_tile=0):
    """Many scenes in one launch (clusters of two thread blocks: a large scene on
    both, small scenes one per block).  ctxs: Contexts on one device; states:
    State or None per scene; rhs, dx: device tensors; split: 0 automatic, 1 one
    block per scene, 2 every scene on two blocks; precond: None (Jacobi) or one
    QTT (or None) per scene; core_dtype: QP_F32 or QP_BF16 cores; qtt_tile: 0
    measured tile shapes, 1 one item per thread, 2 two items per thread.
    Returns (per-scene SolveStats list, block size used)."""
    lib = load()
    n = len(ctxs)
    ch = (C.c_void_p * n)(*[c.h.value for c in ctxs])
    sp = (C.POINTER(State) * n)(*[C.pointer(s) if s is not None else C.POINTER(State)() for s in states])
    rp = (C.c_void_p * n)(*[_ptr(t) for t in rhs])
    dp = (C.c_void_p * n)(*[_ptr(t) for t in dx])
    pre = None
    if precond is not None:
        pre = (C.c_void_p * n)(*[(x.h.value if x is not None else None) for x in precond])
    opts = BatchOpts(float(tol), int(maxit), float(inner_tol), int(max_outer), int(block_threads), int(split),
                     C.cast(pre, C.c_void_p) if pre is not None else None, int(core_dtype), int(qtt_tile))
    stats = (SolveStats * n)()
    used = C.c_int(0)
    rc = lib.newton_solve_batched(n, ch, sp, rp, dp, C.byref(opts), stats, C.byref(used))
    if rc != QP_OK and rc not in allow:
        ctxs[0]._check(rc, "newton_solve_batched")
    return list(stats), used.value


def newton_batch_plan(costs, num_sms, split=0):
    """The cluster jobs of newton_solve_batched for scenes of the given costs
    (host only): a list of (scene, -2) for a scene on both blocks or (a, b) for
    scene a and scene b (-1: none) on the two blocks, in launch order."""
    lib = load()
    n = len(costs)
    cost = (C.c_longlong * max(n, 1))(*[int(c) for c in costs])
    jobs = (C.c_int * max(2 * n, 2))()
    nj = C.c_int(0)
    rc = lib.newton_batch_plan(n, cost, int(num_sms), int(split), jobs, C.byref(nj))
    if rc != QP_OK:
        raise QPError(rc, "newton_batch_plan: " + lib.qp_status_string(rc).decode())
    return [(jobs[2 * j], jobs[2 * j + 1]) for j in range(nj.value)]
