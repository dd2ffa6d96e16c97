"""ctypes binding of ``libtnfem.so`` (C ABI in include/tnfem.h), argument marshalling only.

Every computation runs inside the library; this module converts Python values to the C
structs, keeps handles alive and frees them, and raises ``TnfemError`` on a non-OK status.
Importing it loads the library and raises ``ImportError`` if it has not been built
(``python -m paper_2501_12151_gb300.build``): there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from .workloads import Grid, Material, Load, SolveOpts

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtnfem.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libtnfem.so is not built ({_LIB_PATH}); run python -m paper_2501_12151_gb300.build")
lib = C.CDLL(_LIB_PATH)

STATUS = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "TIMEOUT", 6: "BUDGET", 7: "NUMERIC"}
LOAD_KIND = {"gravity": 0, "traction": 1, "fourier": 2, "manufactured": 3, "nodal": 4}


class TnfemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tnfem {STATUS.get(status, status)}: {msg}")
        self.status = status


class CGrid(C.Structure):
    _fields_ = [("dim", C.c_int), ("levels", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("clamped", C.c_int * 6), ("plane_stress", C.c_int), ("mapped", C.c_int),
                ("edges", (C.c_double * 3) * 3)]


class CMaterial(C.Structure):
    _fields_ = [("E", C.c_double * 2), ("split_x", C.c_double), ("nu", C.c_double)]


class CLoad(C.Structure):
    _fields_ = [("kind", C.c_int), ("rho", C.c_double), ("g", C.c_double), ("face", C.c_int),
                ("traction", C.c_double * 3), ("n_modes", C.c_int), ("amp", C.POINTER(C.c_double)),
                ("wave", C.POINTER(C.c_int)), ("phase", C.POINTER(C.c_double)), ("scale", C.c_double),
                ("nodal", C.c_void_p)]


class COpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("rank_cap", C.c_int), ("kickrank", C.c_int), ("max_sweeps", C.c_int),
                ("precision", C.c_int), ("refine_tol", C.c_double), ("max_refine", C.c_int),
                ("seed", C.c_uint64), ("local_maxit", C.c_int), ("no_precond", C.c_int),
                ("tensor_cores", C.c_int), ("local_rtol", C.c_double), ("cg_engine", C.c_int),
                ("timeout_us", C.c_int64)]


class CInfo(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("refines", C.c_int), ("max_rank", C.c_int), ("local_iters", C.c_longlong),
                ("max_res", C.c_double), ("max_dx", C.c_double), ("energy_err_est", C.c_double),
                ("t_solve_ms", C.c_double), ("flops", C.c_double), ("bytes_A", C.c_size_t),
                ("bytes_f", C.c_size_t), ("bytes_u", C.c_size_t), ("converged", C.c_int),
                ("t_phase_ms", C.c_double * 7)]

    PHASES = ("rhs", "residual", "solve", "svd", "enrich", "env", "other")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "t_phase_ms"}
        d["t_phase_ms"] = dict(zip(self.PHASES, list(self.t_phase_ms)))
        return d


class CRequestInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("message", C.c_char * 256), ("info", CInfo),
                ("queued_us", C.c_double), ("run_us", C.c_double), ("latency_us", C.c_double),
                ("start_us", C.c_double), ("end_us", C.c_double), ("worker", C.c_int),
                ("est_bytes", C.c_size_t), ("peak_bytes", C.c_size_t), ("ncores", C.c_int),
                ("ranks", C.c_int * 64), ("modes", C.c_int * 63), ("result_doubles", C.c_size_t)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_vp = C.c_void_p
_i = C.c_int
_d = C.c_double
_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int)
_pvp = C.POINTER(C.c_void_p)


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("tnfem_create", _i, [_i, _vp, ALLOC_FN, FREE_FN, _vp, _pvp])
_sig("tnfem_destroy", None, [_vp])
_sig("tnfem_last_error", C.c_char_p, [_vp])
_sig("tnfem_set_stream", _i, [_vp, _vp])
_sig("tnfem_kernel_launches", C.c_longlong, [_vp])
_sig("tnfem_set_hbm_budget", _i, [_vp, C.c_size_t])
_sig("tnfem_memory_stats", _i, [_vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), _i])
_sig("tnfem_op_barrier_probe", _i, [_vp, _i, _i, _d, _d])
_sig("tnfem_build_stiffness", _i, [_vp, C.POINTER(CGrid), C.POINTER(CMaterial), _pvp])
_sig("tnfem_build_mass", _i, [_vp, C.POINTER(CGrid), _pvp])
_sig("tnfem_build_load", _i, [_vp, C.POINTER(CGrid), C.POINTER(CMaterial), C.POINTER(CLoad), _i, _pvp])
_sig("tnfem_host_stiffness", _i, [C.POINTER(CGrid), C.POINTER(CMaterial), _pi, _pi, _pi, _pd, _pd])
_sig("tnfem_host_mass", _i, [C.POINTER(CGrid), _pi, _pi, _pi, _pd])
_sig("tnfem_host_load", _i, [C.POINTER(CGrid), C.POINTER(CMaterial), C.POINTER(CLoad), _i, _pi, _pi, _pi, _pd])
_sig("tnfem_solve", _i, [_vp, _vp, _vp, C.POINTER(COpts), _vp, _pvp, C.POINTER(CInfo)])
_sig("tnfem_eval_displacement", _i, [_vp, _vp, C.POINTER(C.c_int64), C.c_int64, _pd])
_sig("tnfem_eval_strain", _i, [_vp, _vp, C.POINTER(CGrid), C.POINTER(C.c_int64), C.c_int64, _pd])
_sig("tnfem_energy_norm", _i, [_vp, _vp, _vp, _vp, _pd])
_sig("tnfem_tt_dot", _i, [_vp, _vp, _vp, _pd])
_sig("tnfem_tt_norm", _i, [_vp, _vp, _pd])
_sig("tnfem_residual_norm", _i, [_vp, _vp, _vp, _vp, _pd])
_sig("tnfem_residual_norm_train", _i, [_vp, _vp, _vp, _vp, _pd])
_sig("tnfem_tt_round", _i, [_vp, _vp, _d, _i, _pvp])
_sig("tnfem_tt_axpy", _i, [_vp, _vp, _d, _vp, _pvp])
_sig("tnfem_mpo_apply", _i, [_vp, _vp, _vp, _pvp])
_sig("tnfem_tt_export", _i, [_vp, _vp, _pi, _pi, _pi, _pd])
_sig("tnfem_tt_import", _i, [_vp, _i, _pi, _pi, _pd, _pvp])
_sig("tnfem_mpo_export", _i, [_vp, _vp, _pi, _pi, _pi, _pd])
_sig("tnfem_mpo_import", _i, [_vp, _i, _pi, _pi, _pd, _pvp])
_sig("tnfem_free_tt", None, [_vp])
_sig("tnfem_free_mpo", None, [_vp])
_sig("tnfem_op_local_matvec", _i, [_vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp])
_sig("tnfem_op_env_left", _i, [_vp, _i, _i, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp])
_sig("tnfem_op_qr", _i, [_vp, _i, _i, _vp, _vp, _vp])
_sig("tnfem_op_qr_ext", _i, [_vp, _i, _i, _i, _vp, _vp, _vp])
_sig("tnfem_op_svd", _i, [_vp, _i, _i, _vp, _vp, _vp, _vp])
_sig("tnfem_op_local_matvec_noalloc", _i, [_vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp])
_ll = C.c_longlong
_sig("tnfem_op_gemm_f32", _i, [_vp, _i, _i, _i, _i, _i] + [_ll] * 9 + [C.c_float, _vp, _vp, C.c_float, _vp])
_sig("tnfem_op_gemm_f64", _i, [_vp, _i, _i, _i, _i, _i] + [_ll] * 9 + [C.c_double, _vp, _vp, C.c_double, _vp])
_sig("tnfem_op_local_matvec_f32", _i, [_vp, _i, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp])
_sig("tnfem_op_local_cg", _i, [_vp, _i, _i, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, C.c_double, _i,
                               C.POINTER(C.c_int), C.POINTER(C.c_int)])
_sig("tnfem_measure_fma_peak", _i, [_vp, _i, _pd])
_sig("tnfem_profile_start", _i, [_vp, _i])
_sig("tnfem_profile_read", _i, [_vp, _i, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _pd, _pd, _pd])

_sig("tnfem_server_start", _i, [_i, _i, C.c_size_t, _pvp])
_sig("tnfem_server_budget", _i, [_vp, C.POINTER(C.c_size_t)])
_sig("tnfem_serve_estimate", _i, [C.POINTER(CGrid), C.POINTER(COpts), C.POINTER(C.c_size_t)])
_sig("tnfem_submit", _i, [_vp, C.POINTER(CGrid), C.POINTER(CMaterial), C.POINTER(CLoad), _i, C.POINTER(COpts),
                          C.POINTER(C.c_uint64)])
_sig("tnfem_wait", _i, [_vp, C.c_uint64, C.c_int64, C.POINTER(CRequestInfo)])
_sig("tnfem_result_take", _i, [_vp, C.c_uint64, _pd])
_sig("tnfem_server_stop", _i, [_vp])
_sig("tnfem_cancel", _i, [_vp, C.c_uint64])
_sig("tnfem_server_stats", _i, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)])

PRECISIONS = {"fp64": 0, "mixed": 1, "mixed-local": 2, "mixed-tf32": 3}
PROF_CLASSES = {"contract32": 0, "contract64": 1, "krylov": 2, "qr": 3, "svd": 4, "other": 5, "cg32": 6, "cg64": 7}


# ---------------------------------------------------------------------------------------
# struct conversion
# ---------------------------------------------------------------------------------------

def c_grid(g: Grid) -> CGrid:
    cg = CGrid()
    cg.dim = g.dim
    cg.levels = g.levels
    for d in range(3):
        cg.lo[d] = float(g.lo[d]) if d < len(g.lo) else 0.0
        cg.hi[d] = float(g.hi[d]) if d < len(g.hi) else 1.0
    for f in range(6):
        cg.clamped[f] = 1 if (f < len(g.clamped) and g.clamped[f]) else 0
    cg.plane_stress = 1 if g.plane_stress else 0
    edges = getattr(g, "edges", None)
    quad = getattr(g, "quad", None)
    cg.mapped = 2 if quad is not None else (1 if edges is not None else 0)
    if quad is not None:
        # corners P0..P3 at unit-square (0,0), (1,0), (0,1), (1,1): lo = P0, edges = the bilinear
        # map's coefficients a = P1 - P0, b = P2 - P0, c = P3 - P2 - P1 + P0
        P = np.asarray(quad, dtype=float).reshape(4, -1)[:, :2]
        cg.lo[0], cg.lo[1], cg.lo[2] = P[0, 0], P[0, 1], 0.0
        for d, v in enumerate((P[1] - P[0], P[2] - P[0], P[3] - P[2] - P[1] + P[0])):
            cg.edges[d][0], cg.edges[d][1], cg.edges[d][2] = float(v[0]), float(v[1]), 0.0
    elif edges is not None:
        for d in range(min(3, len(edges))):
            for e in range(min(3, len(edges[d]))):
                cg.edges[d][e] = float(edges[d][e])
    return cg


def c_material(m: Material) -> CMaterial:
    cm = CMaterial()
    cm.E[0], cm.E[1] = float(m.E[0]), float(m.E[1])
    cm.split_x = float(m.split_x) if np.isfinite(m.split_x) else 1e300
    cm.nu = float(m.nu)
    return cm


class _Loads:
    """Keeps the host arrays of the load structs alive for the duration of a call."""

    def __init__(self, loads: Sequence[Load], dim: int):
        self.keep = []
        self.arr = (CLoad * max(1, len(loads)))()
        for i, ld in enumerate(loads):
            c = self.arr[i]
            c.kind = LOAD_KIND[ld.kind]
            c.rho = float(ld.rho)
            c.g = float(ld.g)
            c.face = int(ld.face)
            for k in range(3):
                c.traction[k] = float(ld.traction[k]) if k < len(ld.traction) else 0.0
            c.scale = float(ld.scale)
            if ld.kind == "fourier":
                amp = np.ascontiguousarray(ld.amp, dtype=np.float64)
                wave = np.ascontiguousarray(ld.wave, dtype=np.int32)
                phase = np.ascontiguousarray(ld.phase, dtype=np.float64)
                self.keep += [amp, wave, phase]
                c.n_modes = int(phase.shape[0])
                c.amp = amp.ctypes.data_as(_pd)
                c.wave = wave.ctypes.data_as(_pi)
                c.phase = phase.ctypes.data_as(_pd)
            if ld.kind == "nodal":
                if ld.nodal is None or not getattr(ld.nodal, "h", None):
                    raise ValueError("a nodal load needs a TT of the same context in Load.nodal")
                self.keep.append(ld.nodal)
                h = ld.nodal.h
                c.nodal = h.value if isinstance(h, C.c_void_p) else h
        self.n = len(loads)


def c_opts(o: SolveOpts, local_maxit: int = 500) -> COpts:
    co = COpts()
    co.tol = float(o.tol)
    co.rank_cap = int(o.rank_cap)
    co.kickrank = int(o.kickrank)
    co.max_sweeps = int(o.max_sweeps)
    co.precision = PRECISIONS[o.precision]
    co.refine_tol = float(o.refine_tol)
    co.max_refine = int(o.max_refine)
    co.seed = int(o.seed)
    co.local_maxit = int(local_maxit)
    co.no_precond = 0 if getattr(o, "precond", True) else 1
    co.tensor_cores = 1 if getattr(o, "tensor_cores", False) else 0
    co.local_rtol = float(getattr(o, "local_rtol", -1.0))
    co.cg_engine = 0 if getattr(o, "fused_cg", True) else 1
    co.timeout_us = int(getattr(o, "timeout_us", 0))
    return co


def _check(st: int, ctx=None):
    if st != 0:
        msg = lib.tnfem_last_error(ctx).decode() if ctx else ""
        raise TnfemError(st, msg)


def op_local_matvec_noalloc(stream: int, r0, n, r1, a0, a1, PhiL, A, PhiR, x, y):
    """Local matvec on device pointers with the library's static scratch array (allocates
    nothing; enqueued on ``stream`` without synchronising)."""
    _check(lib.tnfem_op_local_matvec_noalloc(C.c_void_p(stream), r0, n, r1, a0, a1, PhiL, A, PhiR, x, y))


# ---------------------------------------------------------------------------------------
# host-only builders (no GPU needed)
# ---------------------------------------------------------------------------------------

def _host_train(call, op: bool):
    nc = C.c_int()
    ranks = (C.c_int * 64)()
    modes = (C.c_int * 64)()
    _check(call(C.byref(nc), ranks, modes, None))
    d = nc.value
    sizes = [ranks[k] * modes[k] * (modes[k] if op else 1) * ranks[k + 1] for k in range(d)]
    buf = np.zeros(sum(sizes))
    _check(call(C.byref(nc), ranks, modes, buf.ctypes.data_as(_pd)))
    cores, off = [], 0
    for k in range(d):
        shp = (ranks[k], modes[k], modes[k], ranks[k + 1]) if op else (ranks[k], modes[k], ranks[k + 1])
        cores.append(buf[off:off + sizes[k]].reshape(shp).copy())
        off += sizes[k]
    return cores


def host_stiffness(grid: Grid, mat: Material):
    """Exact (un-rounded) stiffness operator cores and the BC shift s, built on the host."""
    cg, cm = c_grid(grid), c_material(mat)
    s = C.c_double()
    cores = _host_train(lambda n, r, m, c: lib.tnfem_host_stiffness(C.byref(cg), C.byref(cm), n, r, m, c,
                                                                     C.byref(s)), True)
    return cores, s.value


def host_mass(grid: Grid):
    cg = c_grid(grid)
    return _host_train(lambda n, r, m, c: lib.tnfem_host_mass(C.byref(cg), n, r, m, c), True)


def host_load(grid: Grid, mat: Material, loads: Sequence[Load]):
    cg, cm = c_grid(grid), c_material(mat)
    L = _Loads(loads, grid.dim)
    return _host_train(lambda n, r, m, c: lib.tnfem_host_load(C.byref(cg), C.byref(cm), L.arr, L.n, n, r, m, c),
                       False)


# ---------------------------------------------------------------------------------------
# device objects
# ---------------------------------------------------------------------------------------

class Context:
    """A library context on one CUDA device; device work goes to ``stream`` (a cudaStream_t
    handle as int, 0 for the default stream).  With ``torch_alloc`` every device allocation
    of the library is served by PyTorch's caching allocator."""

    def __init__(self, device: int = 0, stream: int = 0, torch_alloc: bool = False, alloc_hook=None, free_hook=None):
        self._cbs = None
        alloc = ALLOC_FN()
        free = FREE_FN()
        if alloc_hook is not None:
            # caller-supplied callbacks: alloc_hook(nbytes) -> device pointer (int) or 0 on failure,
            # free_hook(ptr)
            def _alloc(nbytes, user):
                p = alloc_hook(int(nbytes))
                return p or None

            def _free(ptr, user):
                free_hook(ptr)

            alloc = ALLOC_FN(_alloc)
            free = FREE_FN(_free)
            self._cbs = (alloc, free)
        elif torch_alloc:
            import torch

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or None)
                except Exception:
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            alloc = ALLOC_FN(_alloc)
            free = FREE_FN(_free)
            self._cbs = (alloc, free)
        h = C.c_void_p()
        _check(lib.tnfem_create(device, C.c_void_p(stream), alloc, free, None, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.tnfem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        _check(st, self.h)

    @property
    def launches(self) -> int:
        return int(lib.tnfem_kernel_launches(self.h))

    def set_hbm_budget(self, nbytes: int):
        """Device-memory budget of the context in bytes (0: none)."""
        self.check(lib.tnfem_set_hbm_budget(self.h, int(nbytes)))

    def memory_stats(self, reset_peak: bool = False):
        """(bytes held now, high-water mark)."""
        a, b = C.c_size_t(), C.c_size_t()
        self.check(lib.tnfem_memory_stats(self.h, C.byref(a), C.byref(b), 1 if reset_peak else 0))
        return a.value, b.value

    def barrier_probe(self, ctas: int, late_cta: int, late_ms: float, limit_ms: float) -> int:
        """Status of tnfem_op_barrier_probe (0 or the TNFEM_E_TIMEOUT code); raises on other errors."""
        st = lib.tnfem_op_barrier_probe(self.h, ctas, late_cta, late_ms, limit_ms)
        if st not in (0, 5):
            self.check(st)
        return st

    def set_stream(self, stream: int):
        self.check(lib.tnfem_set_stream(self.h, C.c_void_p(stream)))

    def fma_peak(self, precision: str) -> float:
        """Measured CUDA-core FMA rate in TFLOP/s ("fp64" or "fp32")."""
        v = C.c_double()
        self.check(lib.tnfem_measure_fma_peak(self.h, 0 if precision == "fp64" else 1, C.byref(v)))
        return v.value

    def profile_start(self, every: int = 1):
        """Time every ``every``-th launch of each kernel class with CUDA events (0 stops)."""
        self.check(lib.tnfem_profile_start(self.h, int(every)))

    def profile_read(self, cls: str) -> dict:
        """Launches seen / sampled, device ms, algorithmic flops and bytes of the sampled launches."""
        n, s = C.c_longlong(), C.c_longlong()
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        self.check(lib.tnfem_profile_read(self.h, PROF_CLASSES[cls], C.byref(n), C.byref(s), C.byref(ms),
                                          C.byref(fl), C.byref(by)))
        return {"launches": n.value, "sampled": s.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}

    # builders
    def stiffness(self, grid: Grid, mat: Material) -> "Mpo":
        out = C.c_void_p()
        cg, cm = c_grid(grid), c_material(mat)
        self.check(lib.tnfem_build_stiffness(self.h, C.byref(cg), C.byref(cm), C.byref(out)))
        return Mpo(self, out)

    def mass(self, grid: Grid) -> "Mpo":
        out = C.c_void_p()
        cg = c_grid(grid)
        self.check(lib.tnfem_build_mass(self.h, C.byref(cg), C.byref(out)))
        return Mpo(self, out)

    def load(self, grid: Grid, mat: Material, loads: Sequence[Load]) -> "TT":
        out = C.c_void_p()
        cg, cm = c_grid(grid), c_material(mat)
        L = _Loads(loads, grid.dim)
        self.check(lib.tnfem_build_load(self.h, C.byref(cg), C.byref(cm), L.arr, L.n, C.byref(out)))
        return TT(self, out)

    def solve(self, A: "Mpo", f: "TT", opts: SolveOpts, x0: Optional["TT"] = None, local_maxit: int = 500,
              allow_not_converged: bool = True):
        out = C.c_void_p()
        info = CInfo()
        co = c_opts(opts, local_maxit)
        st = lib.tnfem_solve(self.h, A.h, f.h, C.byref(co), x0.h if x0 else None, C.byref(out), C.byref(info))
        if st in (4, 5) and allow_not_converged and out.value:
            # not converged, or stopped at timeout_us: the last iterate and its info are returned
            d = info.as_dict()
            d["status"] = STATUS[st]
            return TT(self, out), d
        self.check(st)
        d = info.as_dict()
        d["status"] = STATUS[st]
        return TT(self, out), d

    def tt_import(self, cores: List[np.ndarray]) -> "TT":
        d = len(cores)
        ranks = (C.c_int * (d + 1))(*([cores[0].shape[0]] + [c.shape[2] for c in cores]))
        modes = (C.c_int * d)(*[c.shape[1] for c in cores])
        buf = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float64).ravel() for c in cores]))
        out = C.c_void_p()
        self.check(lib.tnfem_tt_import(self.h, d, ranks, modes, buf.ctypes.data_as(_pd), C.byref(out)))
        return TT(self, out)

    def mpo_import(self, cores: List[np.ndarray]) -> "Mpo":
        d = len(cores)
        ranks = (C.c_int * (d + 1))(*([cores[0].shape[0]] + [c.shape[3] for c in cores]))
        modes = (C.c_int * d)(*[c.shape[1] for c in cores])
        buf = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float64).ravel() for c in cores]))
        out = C.c_void_p()
        self.check(lib.tnfem_mpo_import(self.h, d, ranks, modes, buf.ctypes.data_as(_pd), C.byref(out)))
        return Mpo(self, out)

    # kernel-level entry points on device pointers (ints)
    def op_local_matvec(self, r0, n, r1, a0, a1, PhiL, A, PhiR, x, y):
        self.check(lib.tnfem_op_local_matvec(self.h, r0, n, r1, a0, a1, PhiL, A, PhiR, x, y))

    def op_env_left(self, ry0, ry1, rx0, rx1, n, a0, a1, Phi, y, A, x, out):
        self.check(lib.tnfem_op_env_left(self.h, ry0, ry1, rx0, rx1, n, a0, a1, Phi, y, A, x, out))

    def op_gemm_f32(self, engine, M, N, K, batch, strides, alpha, A, B, beta, Cp):
        self.check(lib.tnfem_op_gemm_f32(self.h, engine, M, N, K, batch, *strides, alpha, A, B, beta, Cp))

    def op_gemm_f64(self, engine, M, N, K, batch, strides, alpha, A, B, beta, Cp):
        self.check(lib.tnfem_op_gemm_f64(self.h, engine, M, N, K, batch, *strides, float(alpha), A, B, float(beta), Cp))

    def op_local_matvec_f32(self, engine, r0, n, r1, a0, a1, PhiL, A, PhiR, x, y):
        self.check(lib.tnfem_op_local_matvec_f32(self.h, engine, r0, n, r1, a0, a1, PhiL, A, PhiR, x, y))

    def op_local_cg(self, precision, precond, r0, n, r1, a0, a1, PhiL, A, PhiR, g, x, rtol, maxit):
        """Fused preconditioned CG on one local system; returns (iterations, state)."""
        its, st = C.c_int(0), C.c_int(0)
        prec = 0 if precision in ("fp64", 0) else 1
        self.check(lib.tnfem_op_local_cg(self.h, prec, int(precond), r0, n, r1, a0, a1, PhiL, A, PhiR, g, x, float(rtol), int(maxit),
                                         C.byref(its), C.byref(st)))
        return its.value, st.value

    def op_qr(self, m, n, A, Q, R):
        self.check(lib.tnfem_op_qr(self.h, m, n, A, Q, R))

    def op_qr_ext(self, m, rk, w, A, Q, R):
        self.check(lib.tnfem_op_qr_ext(self.h, m, rk, w, A, Q, R))

    def op_svd(self, m, n, A, U, S, Vt):
        self.check(lib.tnfem_op_svd(self.h, m, n, A, U, S, Vt))


class TT:
    """A tensor train held by the library (cores in device memory)."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    def __del__(self):
        try:
            if self.h:
                lib.tnfem_free_tt(self.h)
                self.h = None
        except Exception:
            pass

    def cores(self) -> List[np.ndarray]:
        nc = C.c_int()
        ranks = (C.c_int * 64)()
        modes = (C.c_int * 64)()
        self.ctx.check(lib.tnfem_tt_export(self.ctx.h, self.h, C.byref(nc), ranks, modes, None))
        d = nc.value
        sizes = [ranks[k] * modes[k] * ranks[k + 1] for k in range(d)]
        buf = np.zeros(sum(sizes))
        self.ctx.check(lib.tnfem_tt_export(self.ctx.h, self.h, C.byref(nc), ranks, modes, buf.ctypes.data_as(_pd)))
        out, off = [], 0
        for k in range(d):
            out.append(buf[off:off + sizes[k]].reshape(ranks[k], modes[k], ranks[k + 1]).copy())
            off += sizes[k]
        return out

    def ranks(self) -> List[int]:
        c = self.cores()
        return [1] + [x.shape[2] for x in c]

    def round(self, eps: float, rmax: int = 1 << 20) -> "TT":
        out = C.c_void_p()
        self.ctx.check(lib.tnfem_tt_round(self.ctx.h, self.h, eps, rmax, C.byref(out)))
        return TT(self.ctx, out)

    def axpy(self, beta: float, y: "TT") -> "TT":
        out = C.c_void_p()
        self.ctx.check(lib.tnfem_tt_axpy(self.ctx.h, self.h, beta, y.h, C.byref(out)))
        return TT(self.ctx, out)

    def dot(self, y: "TT") -> float:
        v = C.c_double()
        self.ctx.check(lib.tnfem_tt_dot(self.ctx.h, self.h, y.h, C.byref(v)))
        return v.value

    def norm(self) -> float:
        v = C.c_double()
        self.ctx.check(lib.tnfem_tt_norm(self.ctx.h, self.h, C.byref(v)))
        return v.value

    def displacement(self, nodes: np.ndarray) -> np.ndarray:
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        n, D = nodes.shape
        out = np.zeros((n, D))
        self.ctx.check(lib.tnfem_eval_displacement(self.ctx.h, self.h, nodes.ctypes.data_as(C.POINTER(C.c_int64)), n,
                                                   out.ctypes.data_as(_pd)))
        return out

    def strain(self, grid: Grid, elems: np.ndarray) -> np.ndarray:
        elems = np.ascontiguousarray(elems, dtype=np.int64)
        n = elems.shape[0]
        out = np.zeros((n, 3 if grid.dim == 2 else 6))
        cg = c_grid(grid)
        self.ctx.check(lib.tnfem_eval_strain(self.ctx.h, self.h, C.byref(cg),
                                             elems.ctypes.data_as(C.POINTER(C.c_int64)), n, out.ctypes.data_as(_pd)))
        return out


class Mpo:
    """A TT-operator held by the library."""

    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h

    def __del__(self):
        try:
            if self.h:
                lib.tnfem_free_mpo(self.h)
                self.h = None
        except Exception:
            pass

    def cores(self) -> List[np.ndarray]:
        nc = C.c_int()
        ranks = (C.c_int * 64)()
        modes = (C.c_int * 64)()
        self.ctx.check(lib.tnfem_mpo_export(self.ctx.h, self.h, C.byref(nc), ranks, modes, None))
        d = nc.value
        sizes = [ranks[k] * modes[k] * modes[k] * ranks[k + 1] for k in range(d)]
        buf = np.zeros(sum(sizes))
        self.ctx.check(lib.tnfem_mpo_export(self.ctx.h, self.h, C.byref(nc), ranks, modes, buf.ctypes.data_as(_pd)))
        out, off = [], 0
        for k in range(d):
            out.append(buf[off:off + sizes[k]].reshape(ranks[k], modes[k], modes[k], ranks[k + 1]).copy())
            off += sizes[k]
        return out

    def apply(self, x: TT) -> TT:
        out = C.c_void_p()
        self.ctx.check(lib.tnfem_mpo_apply(self.ctx.h, self.h, x.h, C.byref(out)))
        return TT(self.ctx, out)

    def energy_norm(self, u: TT, v: Optional[TT] = None) -> float:
        out = C.c_double()
        self.ctx.check(lib.tnfem_energy_norm(self.ctx.h, self.h, u.h, v.h if v else None, C.byref(out)))
        return out.value

    def residual_norm(self, f: TT, u: TT, route: str = "auto") -> float:
        """Relative residual ||f - A u||_2 / ||f||_2 of an approximate solution (step a9's check) in
        binary64: "auto" forms it on dense expansions where they fit (up to 2^22 unknowns), else as
        an orthogonalised residual train; "train" always takes the train route."""
        out = C.c_double()
        fn = lib.tnfem_residual_norm_train if route == "train" else lib.tnfem_residual_norm
        self.ctx.check(fn(self.ctx.h, self.h, f.h, u.h, C.byref(out)))
        return out.value


# ---------------------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------------------

def serve_estimate(grid: Grid, opts: SolveOpts) -> int:
    """Admission estimate (bytes) of one request."""
    cg, co = c_grid(grid), c_opts(opts)
    v = C.c_size_t()
    _check(lib.tnfem_serve_estimate(C.byref(cg), C.byref(co), C.byref(v)))
    return v.value


class Server:
    """Persistent request loop on one GPU (tnfem_server_*): ``submit`` queues a solve request and
    returns its id, ``wait`` blocks until it is done and returns (cores or None, info dict)."""

    def __init__(self, device: int = 0, workers: int = 2, hbm_budget: int = 0, local_maxit: int = 500):
        h = C.c_void_p()
        _check(lib.tnfem_server_start(device, workers, hbm_budget, C.byref(h)))
        self.h = h
        self.local_maxit = local_maxit

    @property
    def budget(self) -> int:
        v = C.c_size_t()
        _check(lib.tnfem_server_budget(self.h, C.byref(v)))
        return v.value

    def submit(self, grid: Grid, mat: Material, loads: Sequence[Load], opts: SolveOpts) -> int:
        cg, cm = c_grid(grid), c_material(mat)
        L = _Loads(loads, grid.dim)
        co = c_opts(opts, self.local_maxit)
        rid = C.c_uint64()
        _check(lib.tnfem_submit(self.h, C.byref(cg), C.byref(cm), L.arr, L.n, C.byref(co), C.byref(rid)))
        return rid.value

    def wait(self, rid: int, timeout_us: int = -1, take: bool = True):
        ri = CRequestInfo()
        _check(lib.tnfem_wait(self.h, rid, timeout_us, C.byref(ri)))
        d = {"status": STATUS[ri.status], "message": ri.message.decode(errors="replace"),
             "info": ri.info.as_dict(), "queued_us": ri.queued_us, "run_us": ri.run_us,
             "latency_us": ri.latency_us, "start_us": ri.start_us, "end_us": ri.end_us, "worker": ri.worker,
             "est_bytes": ri.est_bytes, "peak_bytes": ri.peak_bytes}
        cores = None
        if take:
            buf = np.zeros(max(1, ri.result_doubles))
            _check(lib.tnfem_result_take(self.h, rid, buf.ctypes.data_as(_pd)))
            if ri.result_doubles:
                cores, off = [], 0
                for k in range(ri.ncores):
                    shp = (ri.ranks[k], ri.modes[k], ri.ranks[k + 1])
                    sz = shp[0] * shp[1] * shp[2]
                    cores.append(buf[off:off + sz].reshape(shp).copy())
                    off += sz
        return cores, d

    def cancel(self, rid: int) -> bool:
        """Cancel a queued request; False when it was already admitted (or done)."""
        return lib.tnfem_cancel(self.h, rid) == 0

    def stats(self) -> dict:
        q, r, b = C.c_int(), C.c_int(), C.c_size_t()
        _check(lib.tnfem_server_stats(self.h, C.byref(q), C.byref(r), C.byref(b)))
        return {"queued": q.value, "running": r.value, "admitted_bytes": b.value}

    def stop(self):
        if getattr(self, "h", None):
            lib.tnfem_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
