"""Python binding of the C ABI in include/opt_gb300.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libopt_gb300.so``; PyTorch
only provides device memory (tensors whose data pointers are handed to the
library) and the current CUDA stream.  There is no CPU fallback: importing
this module without the built library, or creating a problem without a CUDA
device, raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int32, c_int64, c_void_p

import numpy as np

from . import build as _build

OPT_OK = 0
STATUS = {0: "OPT_OK", 1: "OPT_ERR_INVALID_ARG", 2: "OPT_ERR_OOM", 3: "OPT_ERR_CUDA",
          4: "OPT_ERR_NUMERIC", 5: "OPT_ERR_TIMEOUT", 6: "OPT_ERR_BUDGET", 7: "OPT_ERR_NOT_READY"}
OPT_ARAP_WARP_2D, OPT_POISSON_2D, OPT_ARAP_MESH = 0, 1, 2
OPT_ARAP_WARP_GRAPH, OPT_ARAP_VOLUME, OPT_EMBEDDED_DEFORMATION = 3, 4, 5


class GridDesc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("W", c_int32), ("H", c_int32),
                ("unknowns", c_void_p * 4), ("consts", c_void_p * 4), ("mask", c_void_p),
                ("handle_idx", c_void_p), ("handle_target", c_void_p), ("n_handles", c_int32),
                ("w_reg", c_float), ("w_fit", c_float)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("V", c_int32), ("E", c_int32), ("v0", c_void_p), ("v1", c_void_p),
                ("unknowns", c_void_p * 6), ("urshape", c_void_p * 3),
                ("handle_idx", c_void_p), ("handle_target", c_void_p), ("n_handles", c_int32),
                ("w_reg", c_float), ("w_fit", c_float)]


class VolumeDesc(ctypes.Structure):
    _fields_ = [("W", c_int32), ("H", c_int32), ("D", c_int32), ("unknowns", c_void_p * 6),
                ("urshape", c_void_p * 3), ("handle_idx", c_void_p), ("handle_target", c_void_p),
                ("n_handles", c_int32), ("w_reg", c_float), ("w_fit", c_float)]


class EmbeddedDesc(ctypes.Structure):
    _fields_ = [("V", c_int32), ("E", c_int32), ("v0", c_void_p), ("v1", c_void_p),
                ("unknowns", c_void_p * 12), ("urshape", c_void_p * 3),
                ("handle_idx", c_void_p), ("handle_target", c_void_p), ("n_handles", c_int32),
                ("w_reg", c_float), ("w_fit", c_float), ("w_rot", c_float)]


class GridDescF64(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("W", c_int32), ("H", c_int32),
                ("unknowns", c_void_p * 4), ("consts", c_void_p * 4), ("mask", c_void_p),
                ("handle_idx", c_void_p), ("handle_target", c_void_p), ("n_handles", c_int32),
                ("w_reg", c_double), ("w_fit", c_double)]


class GraphDescF64(ctypes.Structure):
    _fields_ = [("V", c_int32), ("E", c_int32), ("v0", c_void_p), ("v1", c_void_p),
                ("unknowns", c_void_p * 6), ("urshape", c_void_p * 3),
                ("handle_idx", c_void_p), ("handle_target", c_void_p), ("n_handles", c_int32),
                ("w_reg", c_double), ("w_fit", c_double)]


class SolveParams(ctypes.Structure):
    _fields_ = [("outer", c_int32), ("inner", c_int32), ("lambda0", c_double),
                ("lambda_min", c_double), ("lambda_max", c_double), ("diag_min", c_double),
                ("diag_max", c_double), ("eta", c_double), ("rel_tol", c_double),
                ("use_precond", c_int32), ("materialized", c_int32), ("use_graph", c_int32),
                ("tile_w", c_int32), ("persistent", c_int32), ("stream", c_void_p),
                ("pcg_form", c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("outer_done", c_int32), ("pcg_done", c_int32), ("accepted", c_int32),
                ("converged", c_int32), ("E0", c_double), ("E_final", c_double),
                ("lambda_final", c_double), ("E_history", POINTER(c_double)), ("ms", c_float)]


# (name, restype, argtypes) of every exported entry point
_SIGNATURES = [
    ("opt_solve_params_default", c_int32, [POINTER(SolveParams)]),
    ("opt_problem_create_grid", c_int32, [POINTER(GridDesc), POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_problem_create_graph", c_int32, [POINTER(GraphDesc), POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_problem_create_graph2d", c_int32, [POINTER(GraphDesc), POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_problem_create_volume", c_int32, [POINTER(VolumeDesc), POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_problem_create_embedded", c_int32, [POINTER(EmbeddedDesc), POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_problem_destroy", c_int32, [c_void_p]),
    ("opt_solve_gn", c_int32, [c_void_p, POINTER(SolveParams), POINTER(Report)]),
    ("opt_solve_lm", c_int32, [c_void_p, POINTER(SolveParams), POINTER(Report)]),
    ("opt_pcg_init", c_int32, [c_void_p, c_double, POINTER(c_double)]),
    ("opt_pcg_step", c_int32, [c_void_p, c_int32]),
    ("opt_pcg_get_state", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int32)]),
    ("opt_apply_jtj", c_int32, [c_void_p, c_void_p, c_void_p, c_double, POINTER(c_double)]),
    ("opt_eval_jtf", c_int32, [c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
    ("opt_eval_energy", c_int32, [c_void_p, POINTER(c_double)]),
    ("opt_profile_pcg", c_int32, [c_void_p, c_int32, c_void_p, POINTER(c_float)]),
    ("opt_profile_pcg_fused", c_int32, [c_void_p, c_int32, c_void_p, POINTER(c_float)]),
    ("opt_problem_set_chunking", c_int32, [c_void_p, c_int32]),
    ("opt_problem_autotune", c_int32, [c_void_p, POINTER(c_int32), POINTER(c_float)]),
    ("opt_problem_info", c_int32, [c_void_p, POINTER(c_int64), POINTER(c_int32), POINTER(c_int64)]),
    ("opt_batch_create", c_int32, [POINTER(c_void_p), c_int32, POINTER(c_void_p)]),
    ("opt_batch_destroy", c_int32, [c_void_p]),
    ("opt_batch_set_chunking", c_int32, [c_void_p, c_int32]),
    ("opt_batch_autotune", c_int32, [c_void_p, POINTER(SolveParams), POINTER(c_int32), POINTER(c_float)]),
    ("opt_batch_solve_gn", c_int32, [c_void_p, POINTER(SolveParams), POINTER(Report), POINTER(c_float)]),
    ("opt_batch_solve_lm", c_int32, [c_void_p, POINTER(SolveParams), POINTER(Report), POINTER(c_float)]),
    ("opt_server_create", c_int32, [ctypes.c_size_t, POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_server_destroy", c_int32, [c_void_p]),
    ("opt_server_submit_grid", c_int32, [c_void_p, POINTER(GridDesc), POINTER(ctypes.c_uint64)]),
    ("opt_server_submit_graph", c_int32, [c_void_p, POINTER(GraphDesc), POINTER(ctypes.c_uint64)]),
    ("opt_server_step", c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    ("opt_server_poll", c_int32, [c_void_p, ctypes.c_uint64, POINTER(Report)]),
    ("opt_server_set_max_active", c_int32, [c_void_p, c_int32]),
    ("opt_server_set_max_rounds", c_int32, [c_void_p, c_int32]),
    ("opt_problem_get_config", c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
    ("opt_problem_set_apply_form", c_int32, [c_void_p, c_int32]),
    ("opt_server_inject_rebuild_failure", c_int32, [c_void_p, c_int32]),
    ("opt_warp_apply_jtj_noalloc", c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                             c_int32, c_float, c_float, c_void_p, c_void_p, c_void_p,
                                             c_void_p]),
    ("opt_selftest_grid_barrier", c_int32, [c_int32, c_int32, POINTER(c_int32)]),
    ("opt_selftest_staging_wait", c_int32, [c_int32, POINTER(c_int32)]),
    ("opt_problem_create_grid_f64", c_int32, [POINTER(GridDescF64), POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_problem_create_graph_f64", c_int32, [POINTER(GraphDescF64), POINTER(SolveParams), POINTER(c_void_p)]),
    ("opt_problem_destroy_f64", c_int32, [c_void_p]),
    ("opt_solve_gn_f64", c_int32, [c_void_p, POINTER(SolveParams), POINTER(Report)]),
    ("opt_solve_lm_f64", c_int32, [c_void_p, POINTER(SolveParams), POINTER(Report)]),
    ("opt_apply_jtj_f64", c_int32, [c_void_p, c_void_p, c_void_p, c_double, POINTER(c_double)]),
    ("opt_eval_jtf_f64", c_int32, [c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
    ("opt_eval_energy_f64", c_int32, [c_void_p, POINTER(c_double)]),
    ("opt_profile_pcg_f64", c_int32, [c_void_p, c_int32, c_void_p, POINTER(c_float)]),
    ("opt_problem_info_f64", c_int32, [c_void_p, POINTER(c_int64), POINTER(c_int32), POINTER(c_int64)]),
    ("opt_measure_fp64_fma_rate", c_int32, [c_void_p, POINTER(c_double)]),
    ("opt_status_str", ctypes.c_char_p, [c_int32]),
    ("opt_last_error", ctypes.c_char_p, []),
]

_LIB = None


def load_library(path: str | None = None):
    """Loads the built solver library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA solver library not built ({path}); run paper_1604_06525_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class OptError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load_library()
        msg = lib.opt_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)} {msg}")
        self.status = status


def _check(status: int, where: str):
    if status != OPT_OK:
        raise OptError(status, where)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def default_params(**kw) -> SolveParams:
    p = SolveParams()
    _check(load_library().opt_solve_params_default(ctypes.byref(p)), "opt_solve_params_default")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def make_descriptor(prob, device):
    """Device tensors and the C descriptor of a synth problem instance.
    Returns (descriptor, unknown tensor, tensors to keep alive)."""
    import torch
    dev = torch.device(device)

    def f32(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)

    def i32(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.int32), device=dev)

    keep = []
    if prob.kind in ("warp", "poisson"):
        x = f32(prob.x0).reshape(-1, prob.H, prob.W).clone()
        d = GridDesc()
        d.W, d.H = prob.W, prob.H
        if prob.kind == "warp":
            d.kind = OPT_ARAP_WARP_2D
            consts = f32(prob.urshape)
            mask = None if prob.mask is None else torch.as_tensor(prob.mask, dtype=torch.uint8, device=dev)
            hidx = i32(prob.handle_idx)
            htgt = f32(prob.handle_target.reshape(-1))
            d.n_handles = int(prob.handle_idx.size)
            d.handle_idx = _ptr(hidx) if d.n_handles else None
            d.handle_target = _ptr(htgt) if d.n_handles else None
            d.w_reg, d.w_fit = prob.w_reg, prob.w_fit
            keep += [hidx, htgt]
            nx, nc = 3, 2
        else:
            d.kind = OPT_POISSON_2D
            consts = f32(prob.guide)
            mask = None if prob.mask is None else torch.as_tensor(prob.mask, dtype=torch.uint8, device=dev)
            d.n_handles = 0
            nx, nc = 4, 4
        for c in range(nx):
            d.unknowns[c] = _ptr(x[c])
        for c in range(nc):
            d.consts[c] = _ptr(consts[c])
        d.mask = _ptr(mask) if mask is not None else None
        keep += [consts, mask, x]
        return d, x, keep
    if prob.kind in ("mesh", "warp_graph"):
        nxg, dim = (6, 3) if prob.kind == "mesh" else (3, 2)
        x = f32(prob.x0).reshape(nxg, prob.V).clone()
        U = f32(prob.urshape)
        v0, v1 = i32(prob.v0), i32(prob.v1)
        hidx = i32(prob.handle_idx)
        htgt = f32(prob.handle_target.reshape(-1))
        d = GraphDesc()
        d.V, d.E = prob.V, int(prob.v0.size)
        d.v0, d.v1 = _ptr(v0), _ptr(v1)
        for c in range(nxg):
            d.unknowns[c] = _ptr(x[c])
        for c in range(dim):
            d.urshape[c] = _ptr(U[c])
        d.n_handles = int(prob.handle_idx.size)
        d.handle_idx = _ptr(hidx) if d.n_handles else None
        d.handle_target = _ptr(htgt) if d.n_handles else None
        d.w_reg, d.w_fit = prob.w_reg, prob.w_fit
        keep += [U, v0, v1, hidx, htgt, x]
        return d, x, keep
    if prob.kind == "embedded":
        x = f32(prob.x0).reshape(12, prob.V).clone()
        U = f32(prob.urshape)
        v0, v1 = i32(prob.v0), i32(prob.v1)
        hidx = i32(prob.handle_idx)
        htgt = f32(prob.handle_target.reshape(-1))
        d = EmbeddedDesc()
        d.V, d.E = prob.V, int(prob.v0.size)
        d.v0, d.v1 = _ptr(v0), _ptr(v1)
        for c in range(12):
            d.unknowns[c] = _ptr(x[c])
        for c in range(3):
            d.urshape[c] = _ptr(U[c])
        d.n_handles = int(prob.handle_idx.size)
        d.handle_idx = _ptr(hidx) if d.n_handles else None
        d.handle_target = _ptr(htgt) if d.n_handles else None
        d.w_reg, d.w_fit, d.w_rot = prob.w_reg, prob.w_fit, prob.w_rot
        keep += [U, v0, v1, hidx, htgt, x]
        return d, x, keep
    if prob.kind == "volume":
        x = f32(prob.x0).reshape(6, prob.V).clone()
        U = f32(prob.urshape)
        hidx = i32(prob.handle_idx)
        htgt = f32(prob.handle_target.reshape(-1))
        d = VolumeDesc()
        d.W, d.H, d.D = prob.W, prob.H, prob.D
        for c in range(6):
            d.unknowns[c] = _ptr(x[c])
        for c in range(3):
            d.urshape[c] = _ptr(U[c])
        d.n_handles = int(prob.handle_idx.size)
        d.handle_idx = _ptr(hidx) if d.n_handles else None
        d.handle_target = _ptr(htgt) if d.n_handles else None
        d.w_reg, d.w_fit = prob.w_reg, prob.w_fit
        keep += [U, hidx, htgt, x]
        return d, x, keep
    raise ValueError(prob.kind)


class Problem:
    """One planned problem on the current CUDA device (Fig. 4: plan once,
    solve many times).  `prob` is a synth.WarpProblem / PoissonProblem /
    MeshProblem; its arrays are copied to device tensors that this object
    owns (the unknowns stay caller-owned device memory from the library's
    point of view)."""

    def __init__(self, prob, device: str = "cuda", tile_w: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = load_library()
        self.kind = prob.kind
        self.device = torch.device(device)
        dev = self.device

        def f32(a):
            return torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)

        def i32(a):
            return torch.as_tensor(np.ascontiguousarray(a, np.int32), device=dev)

        self._keep = []
        h = c_void_p()
        d, self.x, self._keep = make_descriptor(prob, self.device)
        if prob.kind in ("warp", "poisson"):
            self.W, self.H = prob.W, prob.H
            plan = default_params(tile_w=tile_w)
            _check(self.lib.opt_problem_create_grid(ctypes.byref(d), ctypes.byref(plan), ctypes.byref(h)),
                   "opt_problem_create_grid")
        else:
            self.V = prob.V
            create = {"mesh": self.lib.opt_problem_create_graph, "warp_graph": self.lib.opt_problem_create_graph2d,
                      "volume": self.lib.opt_problem_create_volume,
                      "embedded": self.lib.opt_problem_create_embedded}[prob.kind]
            _check(create(ctypes.byref(d), None, ctypes.byref(h)), "opt_problem_create_graph")
        self.h = h

    @classmethod
    def from_template(cls, template, tile_w: int = 0):
        """Plans a problem over a device-resident template (template =
        make_descriptor(prob, device) + (kind,)): the constants are shared,
        only the unknowns are fresh -- the input path of a server request."""
        import torch
        d0, x0, keep, kind = template
        self = cls.__new__(cls)
        self.lib = load_library()
        self.kind = kind
        self.device = x0.device
        self.x = x0.clone()
        self._keep = [keep]
        d = type(d0).from_buffer_copy(d0)
        for c in range(self.x.shape[0]):
            d.unknowns[c] = _ptr(self.x[c])
        h = c_void_p()
        if kind in ("warp", "poisson"):
            self.W, self.H = d.W, d.H
            plan = default_params(tile_w=tile_w)
            _check(self.lib.opt_problem_create_grid(ctypes.byref(d), ctypes.byref(plan), ctypes.byref(h)),
                   "opt_problem_create_grid")
        elif kind == "mesh":
            self.V = d.V
            _check(self.lib.opt_problem_create_graph(ctypes.byref(d), None, ctypes.byref(h)), "opt_problem_create_graph")
        else:
            raise ValueError(f"templates of kind {kind} are not supported")
        self.h = h
        return self

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.opt_problem_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_unknowns(self) -> int:
        return int(self.x.numel())

    def _params(self, outer, inner, **kw) -> SolveParams:
        import torch
        kw.setdefault("stream", torch.cuda.current_stream(self.device).cuda_stream)
        return default_params(outer=outer, inner=inner, **kw)

    def _solve(self, fn, outer, inner, **kw) -> dict:
        p = self._params(outer, inner, **kw)
        hist = (c_double * (outer + 1))()
        rep = Report()
        rep.E_history = ctypes.cast(hist, POINTER(c_double))
        st = fn(self.h, ctypes.byref(p), ctypes.byref(rep))
        if st not in (OPT_OK, 4):
            _check(st, "solve")
        return {"status": STATUS[st], "outer_done": rep.outer_done, "pcg_done": rep.pcg_done,
                "accepted": rep.accepted, "converged": rep.converged, "E0": rep.E0,
                "E_final": rep.E_final, "lambda_final": rep.lambda_final,
                "E_history": list(hist[: rep.outer_done + 1]), "ms": rep.ms}

    def solve_gn(self, outer: int, inner: int, **kw) -> dict:
        """Gauss-Newton; x (self.x) is updated in place."""
        return self._solve(self.lib.opt_solve_gn, outer, inner, **kw)

    def solve_lm(self, outer: int, inner: int, **kw) -> dict:
        """Levenberg-Marquardt; x (self.x) is updated in place."""
        return self._solve(self.lib.opt_solve_lm, outer, inner, **kw)

    # parity hooks -----------------------------------------------------
    def apply_jtj(self, p, lam: float = 0.0):
        import torch
        p = torch.as_tensor(p, dtype=torch.float32, device=self.device).contiguous()
        q = torch.empty_like(p)
        pq = c_double()
        _check(self.lib.opt_apply_jtj(self.h, _ptr(p), _ptr(q), lam, ctypes.byref(pq)), "opt_apply_jtj")
        return q, pq.value

    def eval_jtf(self):
        import torch
        jtf = torch.empty_like(self.x)
        diag = torch.empty_like(self.x)
        E = c_double()
        _check(self.lib.opt_eval_jtf(self.h, _ptr(jtf), _ptr(diag), ctypes.byref(E)), "opt_eval_jtf")
        return jtf, diag, E.value

    def energy(self) -> float:
        E = c_double()
        _check(self.lib.opt_eval_energy(self.h, ctypes.byref(E)), "opt_eval_energy")
        return E.value

    def pcg_init(self, lam: float = 0.0) -> float:
        E = c_double()
        _check(self.lib.opt_pcg_init(self.h, lam, ctypes.byref(E)), "opt_pcg_init")
        return E.value

    def pcg_step(self, n: int):
        _check(self.lib.opt_pcg_step(self.h, n), "opt_pcg_step")

    def profile_pcg(self, n_iters: int) -> tuple:
        """Mean device ms per launch of (PCGInit, applyJTJ, vector update)."""
        import torch
        ms = (c_float * 3)()
        st = torch.cuda.current_stream(self.device).cuda_stream
        _check(self.lib.opt_profile_pcg(self.h, n_iters, st, ms), "opt_profile_pcg")
        return ms[0], ms[1], ms[2]

    def profile_pcg_fused(self, n_iters: int) -> tuple:
        """Mean device ms of (PCGInit, one single-reduction PCG iteration,
        the final step) for a wide-tile warp."""
        import torch
        ms = (c_float * 3)()
        st = torch.cuda.current_stream(self.device).cuda_stream
        _check(self.lib.opt_profile_pcg_fused(self.h, n_iters, st, ms), "opt_profile_pcg_fused")
        return ms[0], ms[1], ms[2]

    def set_chunking(self, units_per_block: int):
        _check(self.lib.opt_problem_set_chunking(self.h, units_per_block), "opt_problem_set_chunking")

    def autotune(self):
        """Picks the work granularity (and a mesh's apply form, a grid's tile
        width) with the fastest applyJTJ + update."""
        c, ms = c_int32(), c_float()
        _check(self.lib.opt_problem_autotune(self.h, ctypes.byref(c), ctypes.byref(ms)), "opt_problem_autotune")
        return c.value, ms.value

    def config(self) -> dict:
        """The launch configuration in use (opt_problem_get_config)."""
        tw, ch, af = c_int32(), c_int32(), c_int32()
        _check(self.lib.opt_problem_get_config(self.h, ctypes.byref(tw), ctypes.byref(ch), ctypes.byref(af)),
               "opt_problem_get_config")
        return {"tile_w": tw.value, "chunking": ch.value, "apply_form": af.value}

    def set_apply_form(self, form: int):
        _check(self.lib.opt_problem_set_apply_form(self.h, form), "opt_problem_set_apply_form")

    def pcg_state(self):
        import torch
        dl, r, p = (torch.empty_like(self.x) for _ in range(3))
        it = c_int32()
        _check(self.lib.opt_pcg_get_state(self.h, _ptr(dl), _ptr(r), _ptr(p), ctypes.byref(it)),
               "opt_pcg_get_state")
        return dl, r, p, it.value


def make_descriptor_f64(prob, device):
    """float64 device tensors and the C descriptor of a synth warp / Poisson /
    mesh instance.  Returns (descriptor, unknown tensor, tensors to keep alive)."""
    import torch
    dev = torch.device(device)

    def f64(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.float64), device=dev)

    def i32(a):
        return torch.as_tensor(np.ascontiguousarray(a, np.int32), device=dev)

    keep = []
    if prob.kind in ("warp", "poisson"):
        x = f64(prob.x0).reshape(-1, prob.H, prob.W).clone()
        d = GridDescF64()
        d.W, d.H = prob.W, prob.H
        mask = None if prob.mask is None else torch.as_tensor(prob.mask, dtype=torch.uint8, device=dev)
        if prob.kind == "warp":
            d.kind = OPT_ARAP_WARP_2D
            consts = f64(prob.urshape)
            hidx = i32(prob.handle_idx)
            htgt = f64(prob.handle_target.reshape(-1))
            d.n_handles = int(prob.handle_idx.size)
            d.handle_idx = _ptr(hidx) if d.n_handles else None
            d.handle_target = _ptr(htgt) if d.n_handles else None
            d.w_reg, d.w_fit = prob.w_reg, prob.w_fit
            keep += [hidx, htgt]
            nx, nc = 3, 2
        else:
            d.kind = OPT_POISSON_2D
            consts = f64(prob.guide)
            d.n_handles = 0
            nx, nc = 4, 4
        for c in range(nx):
            d.unknowns[c] = _ptr(x[c])
        for c in range(nc):
            d.consts[c] = _ptr(consts[c])
        d.mask = _ptr(mask) if mask is not None else None
        keep += [consts, mask, x]
        return d, x, keep
    if prob.kind == "mesh":
        x = f64(prob.x0).reshape(6, prob.V).clone()
        U = f64(prob.urshape)
        v0, v1 = i32(prob.v0), i32(prob.v1)
        hidx = i32(prob.handle_idx)
        htgt = f64(prob.handle_target.reshape(-1))
        d = GraphDescF64()
        d.V, d.E = prob.V, int(prob.v0.size)
        d.v0, d.v1 = _ptr(v0), _ptr(v1)
        for c in range(6):
            d.unknowns[c] = _ptr(x[c])
        for c in range(3):
            d.urshape[c] = _ptr(U[c])
        d.n_handles = int(prob.handle_idx.size)
        d.handle_idx = _ptr(hidx) if d.n_handles else None
        d.handle_target = _ptr(htgt) if d.n_handles else None
        d.w_reg, d.w_fit = prob.w_reg, prob.w_fit
        keep += [U, v0, v1, hidx, htgt, x]
        return d, x, keep
    raise ValueError(f"no float64 variant for {prob.kind}")


class ProblemF64(Problem):
    """The full float64 solver (opt_*_f64 in the C ABI) on a synth warp,
    Poisson or mesh instance; the same methods as Problem, float64 tensors."""

    def __init__(self, prob, device: str = "cuda"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = load_library()
        self.kind = prob.kind
        self.device = torch.device(device)
        h = c_void_p()
        d, self.x, self._keep = make_descriptor_f64(prob, self.device)
        if prob.kind in ("warp", "poisson"):
            self.W, self.H = prob.W, prob.H
            _check(self.lib.opt_problem_create_grid_f64(ctypes.byref(d), None, ctypes.byref(h)),
                   "opt_problem_create_grid_f64")
        else:
            self.V = prob.V
            _check(self.lib.opt_problem_create_graph_f64(ctypes.byref(d), None, ctypes.byref(h)),
                   "opt_problem_create_graph_f64")
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.opt_problem_destroy_f64(self.h)
            self.h = c_void_p()

    def solve_gn(self, outer: int, inner: int, **kw) -> dict:
        return self._solve(self.lib.opt_solve_gn_f64, outer, inner, **kw)

    def solve_lm(self, outer: int, inner: int, **kw) -> dict:
        return self._solve(self.lib.opt_solve_lm_f64, outer, inner, **kw)

    def apply_jtj(self, p, lam: float = 0.0):
        import torch
        p = torch.as_tensor(p, dtype=torch.float64, device=self.device).contiguous()
        q = torch.empty_like(p)
        pq = c_double()
        _check(self.lib.opt_apply_jtj_f64(self.h, _ptr(p), _ptr(q), lam, ctypes.byref(pq)), "opt_apply_jtj_f64")
        return q, pq.value

    def eval_jtf(self):
        import torch
        jtf = torch.empty_like(self.x)
        diag = torch.empty_like(self.x)
        E = c_double()
        _check(self.lib.opt_eval_jtf_f64(self.h, _ptr(jtf), _ptr(diag), ctypes.byref(E)), "opt_eval_jtf_f64")
        return jtf, diag, E.value

    def energy(self) -> float:
        E = c_double()
        _check(self.lib.opt_eval_energy_f64(self.h, ctypes.byref(E)), "opt_eval_energy_f64")
        return E.value

    def profile_pcg(self, n_iters: int) -> tuple:
        import torch
        ms = (c_float * 3)()
        st = torch.cuda.current_stream(self.device).cuda_stream
        _check(self.lib.opt_profile_pcg_f64(self.h, n_iters, st, ms), "opt_profile_pcg_f64")
        return ms[0], ms[1], ms[2]

    def _unsupported(self, *a, **k):
        raise NotImplementedError("not part of the float64 solver")

    pcg_init = pcg_step = set_chunking = autotune = pcg_state = _unsupported


def fp64_fma_rate() -> float:
    """Measured float64 FMA throughput of the current device, GFLOP/s."""
    import torch
    g = c_double()
    _check(load_library().opt_measure_fp64_fma_rate(torch.cuda.current_stream().cuda_stream, ctypes.byref(g)),
           "opt_measure_fp64_fma_rate")
    return g.value


class Batch:
    """Many planned problems solved together, one launch per solver phase for
    the whole batch (opt_batch_* in the C ABI).  The Problem objects must stay
    alive while the batch exists."""

    def __init__(self, problems):
        self.lib = load_library()
        self.problems = list(problems)
        arr = (c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        h = c_void_p()
        _check(self.lib.opt_batch_create(arr, len(self.problems), ctypes.byref(h)), "opt_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.opt_batch_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_chunking(self, tiles_per_chunk: int):
        _check(self.lib.opt_batch_set_chunking(self.h, tiles_per_chunk), "opt_batch_set_chunking")

    def autotune(self, inner: int = 4, **kw):
        import torch
        kw.setdefault("stream", torch.cuda.current_stream().cuda_stream)
        p = default_params(outer=1, inner=inner, **kw)
        chosen, best = c_int32(), c_float()
        _check(self.lib.opt_batch_autotune(self.h, ctypes.byref(p), ctypes.byref(chosen), ctypes.byref(best)),
               "opt_batch_autotune")
        return chosen.value, best.value

    def _solve(self, fn, outer, inner, **kw):
        import torch
        kw.setdefault("stream", torch.cuda.current_stream().cuda_stream)
        p = default_params(outer=outer, inner=inner, **kw)
        n = len(self.problems)
        hists = [(c_double * (outer + 1))() for _ in range(n)]
        reps = (Report * n)()
        for i in range(n):
            reps[i].E_history = ctypes.cast(hists[i], POINTER(c_double))
        ms = c_float()
        st = fn(self.h, ctypes.byref(p), reps, ctypes.byref(ms))
        if st not in (OPT_OK, 4):
            _check(st, "batch solve")
        out = []
        for i in range(n):
            r = reps[i]
            out.append({"outer_done": r.outer_done, "pcg_done": r.pcg_done, "accepted": r.accepted,
                        "converged": r.converged, "E0": r.E0, "E_final": r.E_final,
                        "lambda_final": r.lambda_final, "E_history": list(hists[i][: r.outer_done + 1])})
        return out, ms.value

    def solve_gn(self, outer: int, inner: int, **kw):
        """Returns (per-problem reports, device ms of the batched solve)."""
        return self._solve(self.lib.opt_batch_solve_gn, outer, inner, **kw)

    def solve_lm(self, outer: int, inner: int, **kw):
        return self._solve(self.lib.opt_batch_solve_lm, outer, inner, **kw)


class Server:
    """Continuous-batching LM server (opt_server_* in the C ABI).  submit()
    takes a synth problem instance, uploads its arrays and queues it; step()
    admits under the HBM budget and advances every admitted request by one LM
    outer iteration; poll() returns the report once the request finished.
    max_active > 0 caps the requests admitted at once (opt_server_set_max_active);
    max_rounds > 1 lets a step run several outer iterations when nothing waits
    (opt_server_set_max_rounds)."""

    def __init__(self, hbm_budget_bytes: int, outer: int = 10, inner: int = 10, rel_tol: float = 1e-6,
                 device: str = "cuda", max_active: int = 0, max_rounds: int = 1, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = load_library()
        self.device = torch.device(device)
        self.outer = outer
        p = default_params(outer=outer, inner=inner, rel_tol=rel_tol, **kw)
        h = c_void_p()
        _check(self.lib.opt_server_create(hbm_budget_bytes, ctypes.byref(p), ctypes.byref(h)), "opt_server_create")
        self.h = h
        self.inflight = {}
        if max_active:
            self.set_max_active(max_active)
        if max_rounds != 1:
            self.set_max_rounds(max_rounds)

    def set_max_active(self, max_active: int):
        _check(self.lib.opt_server_set_max_active(self.h, max_active), "opt_server_set_max_active")

    def set_max_rounds(self, max_rounds: int):
        _check(self.lib.opt_server_set_max_rounds(self.h, max_rounds), "opt_server_set_max_rounds")

    def inject_rebuild_failure(self, status: int):
        """Test hook: the next batch rebuild fails with `status` (host only)."""
        _check(self.lib.opt_server_inject_rebuild_failure(self.h, status), "opt_server_inject_rebuild_failure")

    def step_status(self):
        """As step(), but returns the status code instead of raising."""
        a, q = c_int32(), c_int32()
        st = self.lib.opt_server_step(self.h, ctypes.byref(a), ctypes.byref(q))
        return st, a.value, q.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.opt_server_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, prob, x=None) -> int:
        if prob.kind not in ("warp", "poisson", "mesh"):
            raise ValueError(f"the server takes warp, poisson and mesh requests, not {prob.kind}")
        d, xt, keep = make_descriptor(prob, self.device)
        if x is not None:
            xt.copy_(x)
        t = ctypes.c_uint64()
        if prob.kind == "mesh":
            _check(self.lib.opt_server_submit_graph(self.h, ctypes.byref(d), ctypes.byref(t)), "submit")
        else:
            _check(self.lib.opt_server_submit_grid(self.h, ctypes.byref(d), ctypes.byref(t)), "submit")
        self.inflight[t.value] = (xt, keep)
        return t.value

    def submit_template(self, template) -> int:
        """Queues a request that shares a prepared template's device constants
        (template = make_descriptor(prob, device) + (kind,)); only the
        unknowns are fresh."""
        d0, x0, keep, kind = template
        xt = x0.clone()
        d = type(d0).from_buffer_copy(d0)
        for c in range(xt.shape[0]):
            d.unknowns[c] = _ptr(xt[c])
        t = ctypes.c_uint64()
        fn = self.lib.opt_server_submit_graph if kind == "mesh" else self.lib.opt_server_submit_grid
        _check(fn(self.h, ctypes.byref(d), ctypes.byref(t)), "submit")
        self.inflight[t.value] = (xt, keep)
        return t.value

    def step(self):
        a, q = c_int32(), c_int32()
        _check(self.lib.opt_server_step(self.h, ctypes.byref(a), ctypes.byref(q)), "opt_server_step")
        return a.value, q.value

    def poll(self, ticket: int):
        """None while running, else (report dict, solution tensor)."""
        hist = (c_double * (self.outer + 2))()
        rep = Report()
        rep.E_history = ctypes.cast(hist, POINTER(c_double))
        st = self.lib.opt_server_poll(self.h, ticket, ctypes.byref(rep))
        if st == 7:
            return None
        xt, _ = self.inflight.pop(ticket)
        if st not in (OPT_OK, 4):
            _check(st, "opt_server_poll")
        return ({"status": STATUS[st], "outer_done": rep.outer_done, "pcg_done": rep.pcg_done,
                 "accepted": rep.accepted, "converged": rep.converged, "E0": rep.E0, "E_final": rep.E_final,
                 "lambda_final": rep.lambda_final, "E_history": list(hist[: rep.outer_done + 1])}, xt)
