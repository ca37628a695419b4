"""GB300 hp-multigrid preconditioned FGMRES for the condensed H(div)-HDG scheme.

Thin Python binding of the C ABI declared in ``include/hdg.h``: the functions
below have the same names as the C entry points and only marshal arguments
(torch tensors -> device pointers, the current CUDA stream, ctypes structs).
Every step of the computation runs in the library's CUDA kernels.  There is
no CPU fallback: if the shared library is missing or no GPU is present the
calls raise.

Typical use::

    import paper_2303_06762_gb300 as hdg
    ctx = hdg.hdg_setup_mesh_hierarchy(levels)          # list of meshes, coarsest first
    F = hdg.hdg_condense(ctx, hdg.Params(k=3, gamma=1e2), forcing)   # forcing: cuda tensor
    u, p, info = hdg.hdg_solve(ctx, F)
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from .build import LIB, build as _build

HDG_FP64 = 0
HDG_MIXED_FP32 = 1
HDG_MIXED_BF16 = 2
HDG_MIXED_FP16 = 3

_STATUS = {0: "HDG_OK", 1: "HDG_ERR_INVALID_ARG", 2: "HDG_ERR_OOM", 3: "HDG_ERR_CUDA",
           4: "HDG_ERR_SINGULAR", 5: "HDG_ERR_NOT_CONVERGED", 6: "HDG_ERR_BREAKDOWN",
           7: "HDG_ERR_NONFINITE", 8: "HDG_ERR_UNSUPPORTED", 9: "HDG_ERR_STATE", 10: "HDG_ERR_TIMEOUT"}

# every exported entry point of include/hdg.h
EXPORTS = ("hdg_default_solve_opts", "hdg_setup_mesh_hierarchy", "hdg_check_hierarchy", "hdg_condense", "hdg_load",
           "hdg_apply", "hdg_precond_apply", "hdg_solve", "hdg_recover", "hdg_adjoint", "hdg_get_sizes",
           "hdg_get_element_matrices", "hdg_level_apply", "hdg_smooth", "hdg_prolong_add",
           "hdg_restrict", "hdg_coarse_solve", "hdg_mg_h", "hdg_kernel_launches",
           "hdg_reference_tables", "hdg_restrict_noalloc", "hdg_set_wait_limit", "hdg_fp64_fma_probe", "hdg_postprocess", "hdg_boundary_facets", "hdg_apply_transpose", "hdg_apply_multi",
           "hdg_precond_apply_multi", "hdg_smooth_multi", "hdg_set_batched_tile", "hdg_tune_batched", "hdg_solve_multi", "hdg_solve_batched", "hdg_picard", "hdg_newton",
           "hdg_destroy",
           "hdg_status_string", "hdg_last_error")


class HdgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("n_vertices", ctypes.POINTER(ctypes.c_int64)),
                ("n_cells", ctypes.POINTER(ctypes.c_int64)),
                ("coords", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
                ("cells", ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))),
                ("parent", ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))),
                ("vertex_colour", ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)))]


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nu", ctypes.c_double), ("beta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("m_p", ctypes.c_int), ("m_h", ctypes.c_int),
                ("cycle", ctypes.c_int), ("vcycle_growth", ctypes.c_int), ("precision", ctypes.c_int),
                ("fused_coarse_cells", ctypes.c_int), ("nu_elem", ctypes.c_void_p), ("conv", ctypes.c_void_p),
                ("newton_u", ctypes.c_void_p), ("smoother", ctypes.c_int), ("jacobi_damping", ctypes.c_double),
                ("hp_additive", ctypes.c_int), ("dirichlet", ctypes.c_void_p), ("pseudo_dt_inv", ctypes.c_double)]


class HierarchyInfo(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("n_interior_facets", ctypes.c_int64), ("n_dof", ctypes.c_int64),
                ("n_patches", ctypes.c_int), ("n_colours", ctypes.c_int), ("max_patch_facets", ctypes.c_int),
                ("max_patch_cells", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("floor_rel", ctypes.c_double),
                ("uzawa_tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_it", ctypes.c_int),
                ("max_uzawa", ctypes.c_int), ("krylov", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("uzawa_its", ctypes.c_int), ("krylov_its_total", ctypes.c_int),
                ("krylov_its", ctypes.c_int * 64), ("res_mom", ctypes.c_double),
                ("dp_rel", ctypes.c_double), ("normF", ctypes.c_double), ("div_l2", ctypes.c_double),
                ("res_floor", ctypes.c_double)]

    def as_dict(self):
        return dict(uzawa_its=self.uzawa_its, krylov_its_total=self.krylov_its_total,
                    krylov_its=list(self.krylov_its[:self.uzawa_its]), res_mom=self.res_mom,
                    dp_rel=self.dp_rel, normF=self.normF, div_l2=self.div_l2, res_floor=self.res_floor)


class Sizes(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_levels", ctypes.c_int), ("n_cells", ctypes.c_int64),
                ("n_interior_facets", ctypes.c_int64), ("n_dof", ctypes.c_int64),
                ("n_dof_level", ctypes.c_int64 * 16), ("n_colours_level", ctypes.c_int * 16),
                ("n_lat", ctypes.c_int), ("n_boundary_facets", ctypes.c_int64)]


@dataclass
class Params:
    """Solver parameters (hdg_params); defaults follow Section 5 (m_p = m_h = 1, V-cycle)."""
    k: int = 2
    nu: float = 1.0
    beta: float = 0.0
    gamma: float = 1e2
    m_p: int = 1
    m_h: int = 1
    cycle: int = 1
    vcycle_growth: int = 2
    precision: int = HDG_FP64
    fused_coarse_cells: int = 0
    nu_elem: object = None          # optional CUDA float64 tensor [n_cells] of per-cell viscosity
    conv: object = None             # optional CUDA float64 tensor [n_cells, n_lat, 2]: Oseen field w_h
    newton_u: object = None         # optional CUDA float64 tensor [n_dof]: previous iterate (Newton step)
    smoother: int = 0               # 0 = block Gauss-Seidel, 1 = damped block Jacobi
    jacobi_damping: float = 0.5
    hp_additive: int = 0            # 1 = additive form of Algorithm 2
    dirichlet: object = None        # optional CUDA float64 tensor [n_boundary_facets, dpf]: boundary data
    pseudo_dt_inv: float = 0.0      # hdg_picard: pseudo-time continuation 1/dt* (0 = off)

    def to_c(self) -> _Params:
        ne = None if self.nu_elem is None else _ptr(self.nu_elem)
        cv = None if self.conv is None else _ptr(self.conv)
        nw = None if self.newton_u is None else _ptr(self.newton_u)
        return _Params(self.k, self.nu, self.beta, self.gamma, self.m_p, self.m_h, self.cycle,
                       self.vcycle_growth, self.precision, self.fused_coarse_cells, ne, cv, nw,
                       self.smoother, self.jacobi_damping, self.hp_additive,
                       None if self.dirichlet is None else _ptr(self.dirichlet), self.pseudo_dt_inv)


_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load (building first if needed) the shared library; raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        _build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.c_int
    sigs = {
        "hdg_default_solve_opts": (None, [ctypes.POINTER(SolveOpts)]),
        "hdg_setup_mesh_hierarchy": (I, [ctypes.POINTER(_MeshDesc), I, ctypes.POINTER(P)]),
        "hdg_check_hierarchy": (I, [ctypes.POINTER(_MeshDesc), I, ctypes.POINTER(HierarchyInfo), ctypes.c_char_p, I]),
        "hdg_apply_multi": (I, [P, I, P, P, P]),
        "hdg_precond_apply_multi": (I, [P, I, P, P, P]),
        "hdg_smooth_multi": (I, [P, I, I, P, P, I, I, P]),
        "hdg_set_batched_tile": (I, [P, I, I]),
        "hdg_tune_batched": (I, [P, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double), P]),
        "hdg_solve_multi": (I, [P, I, P, P, P, ctypes.POINTER(SolveOpts), P, P]),
        "hdg_solve_batched": (I, [P, I, P, P, P, ctypes.POINTER(SolveOpts), P, P]),
        "hdg_picard": (I, [P, ctypes.POINTER(_Params), P, ctypes.c_double, I, P, P, ctypes.POINTER(SolveOpts),
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), P]),
        "hdg_newton": (I, [P, ctypes.POINTER(_Params), P, ctypes.c_double, I, P, P, ctypes.POINTER(SolveOpts),
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), P]),
        "hdg_condense": (I, [P, ctypes.POINTER(_Params), P, P, P]),
        "hdg_load": (I, [P, P, P, P]),
        "hdg_apply": (I, [P, P, P, P]),
        "hdg_precond_apply": (I, [P, P, P, P]),
        "hdg_solve": (I, [P, P, P, P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), P]),
        "hdg_recover": (I, [P, P, P, P, P, P]),
        "hdg_adjoint": (I, [P, P, P, P, P, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveOpts),
                            ctypes.POINTER(SolveInfo), P]),
        "hdg_get_sizes": (I, [P, ctypes.POINTER(Sizes)]),
        "hdg_get_element_matrices": (I, [P, I, P, P]),
        "hdg_level_apply": (I, [P, I, P, P, P]),
        "hdg_smooth": (I, [P, I, P, P, I, I, P]),
        "hdg_prolong_add": (I, [P, I, P, P, P]),
        "hdg_restrict": (I, [P, I, P, P, P]),
        "hdg_restrict_noalloc": (I, [P, I, P, P, P]),
        "hdg_set_wait_limit": (I, [P, ctypes.c_int64]),
        "hdg_postprocess": (I, [P, P, P, P, P]),
        "hdg_boundary_facets": (I, [P, P]),
        "hdg_apply_transpose": (I, [P, I, P, P, P]),
        "hdg_fp64_fma_probe": (ctypes.c_int64, [I, ctypes.c_int64, P, P]),
        "hdg_coarse_solve": (I, [P, P, P, P]),
        "hdg_mg_h": (I, [P, P, P, P]),
        "hdg_kernel_launches": (ctypes.c_uint64, []),
        "hdg_reference_tables": (ctypes.c_int64, [I, P]),
        "hdg_destroy": (None, [P]),
        "hdg_status_string": (ctypes.c_char_p, [I]),
        "hdg_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    del D
    _lib = lib
    return lib


# ------------------------------------------------------------------ helpers
def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns an hdg_ctx handle; freed by close() or garbage collection."""

    def __init__(self, handle: ctypes.c_void_p, device: int):
        self.handle = handle
        self.device = device

    def check(self, st: int):
        if st != 0:
            msg = load_library().hdg_last_error(self.handle)
            raise HdgError(st, msg.decode() if msg else "")

    def sizes(self) -> Sizes:
        s = Sizes()
        self.check(load_library().hdg_get_sizes(self.handle, ctypes.byref(s)))
        return s

    def close(self):
        if self.handle:
            load_library().hdg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ C-ABI mirrors
def _mesh_desc(levels: Sequence):
    """The hdg_mesh_desc of `levels` and the arrays it points into (keep them alive)."""
    n = len(levels)
    keep = []
    nv = (ctypes.c_int64 * n)(*[int(m.coords.shape[0]) for m in levels])
    nc = (ctypes.c_int64 * n)(*[int(m.cells.shape[0]) for m in levels])
    co = (ctypes.POINTER(ctypes.c_double) * n)()
    ce = (ctypes.POINTER(ctypes.c_int32) * n)()
    pa = (ctypes.POINTER(ctypes.c_int32) * n)()
    vc = (ctypes.POINTER(ctypes.c_int32) * n)()
    for l, m in enumerate(levels):
        a = np.ascontiguousarray(m.coords, dtype=np.float64)
        b = np.ascontiguousarray(m.cells, dtype=np.int32)
        keep += [a, b]
        co[l] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        ce[l] = b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if l > 0:
            p = np.ascontiguousarray(m.parent, dtype=np.int32)
            keep.append(p)
            pa[l] = p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        col = getattr(m, "vertex_colour", None)
        if col is not None:
            c = np.ascontiguousarray(col, dtype=np.int32)
            keep.append(c)
            vc[l] = c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    keep += [nv, nc, co, ce, pa, vc]
    dim = int(levels[0].coords.shape[1])
    if dim not in (2, 3) or any(int(m.coords.shape[1]) != dim or int(m.cells.shape[1]) != dim + 1 for m in levels):
        raise ValueError("levels must all be triangulations (coords (nv,2), cells (nc,3)) or all "
                         "tetrahedrisations (coords (nv,3), cells (nc,4))")
    return _MeshDesc(dim, n, nv, nc, co, ce, pa, vc), keep


def hdg_check_hierarchy(levels: Sequence, k: int = 1) -> dict:
    """Host-only validation of a hierarchy (no GPU needed); returns the finest level's sizes
    for order k, raises HdgError with the reason otherwise."""
    desc, keep = _mesh_desc(levels)
    info = HierarchyInfo()
    msg = ctypes.create_string_buffer(512)
    st = load_library().hdg_check_hierarchy(ctypes.byref(desc), k, ctypes.byref(info), msg, len(msg))
    if st != 0:
        raise HdgError(st, msg.value.decode())
    return {name: getattr(info, name) for name, _ in HierarchyInfo._fields_}


def hdg_setup_mesh_hierarchy(levels: Sequence, device: int = 0) -> Context:
    """levels: objects with .coords (nv,2) float64, .cells (nc,3) int32, .parent (levels >= 1)
    and optional .vertex_colour, coarsest first; or tetrahedral levels, .coords (nv,3) and
    .cells (nc,4) (3D: edge patches, red-refined hierarchy)."""
    lib = load_library()
    desc, keep = _mesh_desc(levels)
    h = ctypes.c_void_p()
    st = lib.hdg_setup_mesh_hierarchy(ctypes.byref(desc), device, ctypes.byref(h))
    ctx = Context(h, device)
    ctx.check(st)
    ctx.level_cells = [int(m.cells.shape[0]) for m in levels]
    ctx.dim = int(levels[0].coords.shape[1])
    return ctx


def dofs_per_facet(dim: int, k: int) -> int:
    """Skeleton unknowns per facet: 2(k+1) on triangles, 3(k+1)(k+2)/2 on tetrahedra."""
    return 2 * (k + 1) if dim == 2 else 3 * (k + 1) * (k + 2) // 2


def union_slices(hierarchies: Sequence, k: int):
    """For a hierarchy built by workloads.mesh2d.disjoint_union(hierarchies): per mesh, the slice of
    the skeleton unknowns and the slice of the cells (pressures) on the finest level.  One solve of
    the union is the solve of all meshes' block-diagonal system with every kernel launch (and the
    preconditioner's captured graph) covering all meshes."""
    out, d0, c0 = [], 0, 0
    for h in hierarchies:
        cells = np.asarray(h[-1].cells)
        e = np.sort(np.concatenate([cells[:, [1, 2]], cells[:, [0, 2]], cells[:, [0, 1]]]).astype(np.int64), axis=1)
        _, cnt = np.unique(e, axis=0, return_counts=True)
        nd = int((cnt == 2).sum()) * 2 * (k + 1)
        out.append((slice(d0, d0 + nd), slice(c0, c0 + cells.shape[0])))
        d0 += nd
        c0 += cells.shape[0]
    return out


def hdg_condense(ctx: Context, params: Params, forcing=None, stream=None):
    """Condense; returns the condensed load F (cuda float64 tensor) when forcing is given."""
    import torch
    lib = load_library()
    p = params.to_c()
    F = None
    if forcing is not None:
        n = ctx.sizes().n_interior_facets * dofs_per_facet(getattr(ctx, "dim", 2), params.k)
        F = torch.empty(n, dtype=torch.float64, device=forcing.device)
        ctx.check(lib.hdg_condense(ctx.handle, ctypes.byref(p), _ptr(forcing), _ptr(F),
                                   _stream(stream)))
    else:
        ctx.check(lib.hdg_condense(ctx.handle, ctypes.byref(p), None, None, _stream(stream)))
    return F


def hdg_load(ctx: Context, forcing, F=None, stream=None):
    """Condensed load of lattice forcing [n_cells, n_lat, 2] with the current condensed operator."""
    import torch
    n = ctx.sizes().n_dof
    F = torch.empty(n, dtype=torch.float64, device=forcing.device) if F is None else F
    ctx.check(load_library().hdg_load(ctx.handle, _ptr(forcing), _ptr(F), _stream(stream)))
    return F


def hdg_apply(ctx: Context, x, y=None, stream=None):
    import torch
    y = torch.empty_like(x) if y is None else y
    ctx.check(load_library().hdg_apply(ctx.handle, _ptr(x), _ptr(y), _stream(stream)))
    return y


def hdg_apply_transpose(ctx: Context, x, y=None, level: int = -1, stream=None):
    """y = (A^eps)^T x on a level (-1: order k)."""
    import torch
    y = torch.empty_like(x) if y is None else y
    ctx.check(load_library().hdg_apply_transpose(ctx.handle, level, _ptr(x), _ptr(y), _stream(stream)))
    return y


def hdg_precond_apply(ctx: Context, r, z=None, stream=None):
    import torch
    z = torch.empty_like(r) if z is None else z
    ctx.check(load_library().hdg_precond_apply(ctx.handle, _ptr(r), _ptr(z), _stream(stream)))
    return z


def default_solve_opts() -> SolveOpts:
    o = SolveOpts()
    load_library().hdg_default_solve_opts(ctypes.byref(o))
    return o


def hdg_solve(ctx: Context, F, u=None, p=None, opts: Optional[SolveOpts] = None, stream=None,
              raise_on_nonconvergence: bool = True):
    """Uzawa + FGMRES; returns (u, p, info dict).  u, p are updated in place when given."""
    import torch
    s = ctx.sizes()
    u = torch.zeros(s.n_dof, dtype=torch.float64, device=F.device) if u is None else u
    p = torch.zeros(s.n_cells, dtype=torch.float64, device=F.device) if p is None else p
    info = SolveInfo()
    o = opts if opts is not None else default_solve_opts()
    st = load_library().hdg_solve(ctx.handle, _ptr(F), _ptr(u), _ptr(p), ctypes.byref(o),
                                  ctypes.byref(info), _stream(stream))
    if st != 0 and (st != 5 or raise_on_nonconvergence):
        ctx.check(st)
    d = info.as_dict()
    d["converged"] = st == 0
    return u, p, d


def hdg_apply_multi(ctx: Context, x, y=None, stream=None):
    """Y = A^eps X for X of shape [nrhs, n_dof] (CUDA float64)."""
    import torch
    y = torch.empty_like(x) if y is None else y
    ctx.check(load_library().hdg_apply_multi(ctx.handle, x.shape[0], _ptr(x), _ptr(y), _stream(stream)))
    return y


def hdg_precond_apply_multi(ctx: Context, r, z=None, stream=None):
    """Z = MG_hp(R) column by column for R of shape [nrhs, n_dof]."""
    import torch
    z = torch.empty_like(r) if z is None else z
    ctx.check(load_library().hdg_precond_apply_multi(ctx.handle, r.shape[0], _ptr(r), _ptr(z), _stream(stream)))
    return z


def hdg_smooth_multi(ctx: Context, level: int, g, u, n_sweeps: int = 1, reverse: bool = False, stream=None):
    """hdg_smooth for g, u of shape [nrhs, n] (u updated in place)."""
    ctx.check(load_library().hdg_smooth_multi(ctx.handle, level, g.shape[0], _ptr(g), _ptr(u), n_sweeps,
                                              1 if reverse else 0, _stream(stream)))
    return u


def hdg_set_batched_tile(ctx: Context, rows_per_thread: int = 0, threads: int = 0):
    """Force the batched order-k sweep's tile (0, 0 = autotuner)."""
    ctx.check(load_library().hdg_set_batched_tile(ctx.handle, rows_per_thread, threads))


def hdg_tune_batched(ctx: Context, nrhs: int, stream=None):
    """Run the batched-sweep autotuner now; returns (rows_per_thread, threads, ms per colour phase)."""
    rb, nt, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    ctx.check(load_library().hdg_tune_batched(ctx.handle, nrhs, ctypes.byref(rb), ctypes.byref(nt), ctypes.byref(ms),
                                              _stream(stream)))
    return rb.value, nt.value, ms.value


def hdg_solve_multi(ctx: Context, F, u=None, p=None, opts: Optional[SolveOpts] = None, stream=None,
                    raise_on_nonconvergence: bool = True):
    """hdg_solve for F of shape [nrhs, n_dof]; returns (u [nrhs, n_dof], p [nrhs, n_cells], [info dicts])."""
    import torch
    s = ctx.sizes()
    nrhs = F.shape[0]
    u = torch.zeros((nrhs, s.n_dof), dtype=torch.float64, device=F.device) if u is None else u
    p = torch.zeros((nrhs, s.n_cells), dtype=torch.float64, device=F.device) if p is None else p
    infos = (SolveInfo * nrhs)()
    o = opts if opts is not None else default_solve_opts()
    st = load_library().hdg_solve_multi(ctx.handle, nrhs, _ptr(F), _ptr(u), _ptr(p), ctypes.byref(o),
                                        ctypes.cast(infos, ctypes.c_void_p), _stream(stream))
    if st != 0 and (st != 5 or raise_on_nonconvergence):
        ctx.check(st)
    return u, p, [infos[r].as_dict() for r in range(nrhs)]


def hdg_solve_batched(ctxs: Sequence, Fs: Sequence, opts: Optional[SolveOpts] = None):
    """One load per context, all solved concurrently (one host thread and stream each).
    Returns ([u], [p], [info dicts], [status])."""
    import torch
    n = len(ctxs)
    us, ps = [], []
    for c, F in zip(ctxs, Fs):
        s = c.sizes()
        us.append(torch.zeros(s.n_dof, dtype=torch.float64, device=F.device))
        ps.append(torch.zeros(s.n_cells, dtype=torch.float64, device=F.device))
    P = ctypes.c_void_p
    handles = (P * n)(*[c.handle for c in ctxs])
    fp = (P * n)(*[F.data_ptr() for F in Fs])
    up = (P * n)(*[u.data_ptr() for u in us])
    pp = (P * n)(*[p.data_ptr() for p in ps])
    infos = (SolveInfo * n)()
    stat = (ctypes.c_int * n)()
    o = opts if opts is not None else default_solve_opts()
    torch.cuda.synchronize()
    st = load_library().hdg_solve_batched(ctypes.cast(handles, P), n, ctypes.cast(fp, P), ctypes.cast(up, P),
                                          ctypes.cast(pp, P), ctypes.byref(o), ctypes.cast(infos, P),
                                          ctypes.cast(stat, P))
    if st not in (0, 5):
        for c, sv in zip(ctxs, stat):
            if sv not in (0, 5):
                c.check(sv)
        raise HdgError(st, "hdg_solve_batched failed")
    return us, ps, [infos[i].as_dict() for i in range(n)], list(stat)


def hdg_picard(ctx: Context, params: Params, forcing, tol: float = 1e-8, max_steps: int = 50,
               opts: Optional[SolveOpts] = None, stream=None, raise_on_nonconvergence: bool = True):
    """Steady Navier-Stokes by Picard iteration; returns (u, p, steps, last ||u^n - u^(n-1)||)."""
    import torch
    s = ctx.sizes()
    k = params.k
    n_dof = s.n_interior_facets * 2 * (k + 1)
    u = torch.empty(n_dof, dtype=torch.float64, device=forcing.device)
    p = torch.empty(s.n_cells, dtype=torch.float64, device=forcing.device)
    steps = ctypes.c_int()
    dist = ctypes.c_double()
    c = params.to_c()
    o = opts if opts is not None else default_solve_opts()
    st = load_library().hdg_picard(ctx.handle, ctypes.byref(c), _ptr(forcing), tol, max_steps, _ptr(u), _ptr(p),
                                   ctypes.byref(o), ctypes.byref(steps), ctypes.byref(dist), _stream(stream))
    if st != 0 and (st != 5 or raise_on_nonconvergence):
        ctx.check(st)
    return u, p, steps.value, dist.value


def hdg_newton(ctx: Context, params: Params, forcing, u, p, tol: float = 1e-10, max_steps: int = 20,
               opts: Optional[SolveOpts] = None, stream=None, raise_on_nonconvergence: bool = True):
    """Newton steps from the iterate (u, p) of the context's current operator (updated in place);
    returns (u, p, steps, last ||u^n - u^(n-1)||)."""
    steps = ctypes.c_int()
    dist = ctypes.c_double()
    c = params.to_c()
    o = opts if opts is not None else default_solve_opts()
    st = load_library().hdg_newton(ctx.handle, ctypes.byref(c), _ptr(forcing), tol, max_steps, _ptr(u), _ptr(p),
                                   ctypes.byref(o), ctypes.byref(steps), ctypes.byref(dist), _stream(stream))
    if st != 0 and (st != 5 or raise_on_nonconvergence):
        ctx.check(st)
    return u, p, steps.value, dist.value


def hdg_recover(ctx: Context, u, forcing=None, stream=None):
    """Local fields of a skeleton solution: (L coefficients [nc, d*d, npk], u at the lattice [nc, nlat, d]);
    d = 2 on triangles, 3 on tetrahedra."""
    import torch
    s = ctx.sizes()
    k = s.k
    d = getattr(ctx, "dim", 2)
    if d == 2:
        npk, nlat = (k + 1) * (k + 2) // 2, (k + 2) * (k + 3) // 2
    else:
        npk, nlat = (k + 1) * (k + 2) * (k + 3) // 6, (k + 2) * (k + 3) * (k + 4) // 6
    L = torch.empty((s.n_cells, d * d, npk), dtype=torch.float64, device=u.device)
    ul = torch.empty((s.n_cells, nlat, d), dtype=torch.float64, device=u.device)
    ctx.check(load_library().hdg_recover(ctx.handle, _ptr(u), _ptr(forcing), _ptr(L), _ptr(ul),
                                         _stream(stream)))
    return L, ul


def hdg_boundary_facets(ctx: Context) -> np.ndarray:
    """Sorted global vertex pairs (triples on tetrahedra) of the finest level's boundary facets,
    the order of the Dirichlet data, shape [n_boundary_facets, dim] (int32)."""
    n = ctx.sizes().n_boundary_facets
    out = np.zeros((n, getattr(ctx, "dim", 2)), dtype=np.int32)
    ctx.check(load_library().hdg_boundary_facets(ctx.handle, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def hdg_postprocess(ctx: Context, u, forcing=None, stream=None):
    """u* of eq. stPost at each cell's degree-(k+1) lattice, shape [n_cells, n_lat, d]."""
    import torch
    s = ctx.sizes()
    d = getattr(ctx, "dim", 2)
    out = torch.empty((s.n_cells, s.n_lat, d), dtype=torch.float64, device=u.device)
    ctx.check(load_library().hdg_postprocess(ctx.handle, _ptr(u), _ptr(forcing), _ptr(out), _stream(stream)))
    return out


def hdg_adjoint(ctx: Context, forcing, u, u_target, opts: Optional[SolveOpts] = None, stream=None):
    """Adjoint gradients of J = 1/2 ||u_h - u_target||^2: returns (J, dJ/dforcing, dJ/dnu_cell, info)."""
    import torch
    s = ctx.sizes()
    gf = torch.empty_like(forcing)
    gn = torch.empty(s.n_cells, dtype=torch.float64, device=forcing.device)
    J = ctypes.c_double()
    info = SolveInfo()
    o = opts if opts is not None else default_solve_opts()
    ctx.check(load_library().hdg_adjoint(ctx.handle, _ptr(forcing), _ptr(u), _ptr(u_target), _ptr(gf),
                                         _ptr(gn), ctypes.byref(J), ctypes.byref(o), ctypes.byref(info),
                                         _stream(stream)))
    return J.value, gf, gn, info.as_dict()


def hdg_get_element_matrices(ctx: Context, level: int = -1, stream=None):
    import torch
    s = ctx.sizes()
    dim = getattr(ctx, "dim", 2)
    if level < 0:
        nloc = (dim + 1) * dofs_per_facet(dim, s.k)
        nc = s.n_cells
    else:
        nloc = (dim + 1) * dim
        nc = _level_cells(ctx, level)
    out = torch.empty((nc, nloc, nloc), dtype=torch.float64, device=f"cuda:{ctx.device}")
    ctx.check(load_library().hdg_get_element_matrices(ctx.handle, level, _ptr(out), _stream(stream)))
    return out


def _level_cells(ctx: Context, level: int) -> int:
    return ctx.level_cells[level]


def hdg_level_apply(ctx: Context, level: int, x, y=None, stream=None):
    import torch
    y = torch.empty_like(x) if y is None else y
    ctx.check(load_library().hdg_level_apply(ctx.handle, level, _ptr(x), _ptr(y), _stream(stream)))
    return y


def hdg_fp64_fma_probe(out, blocks_per_sm: int = 8, iters: int = 1 << 16, stream=None) -> int:
    """Enqueue the FP64 FMA-rate kernel (out: CUDA float64 tensor, >= 1 element); returns its FLOPs."""
    n = load_library().hdg_fp64_fma_probe(blocks_per_sm, iters, _ptr(out), _stream(stream))
    if n < 0:
        raise HdgError(1, "hdg_fp64_fma_probe: bad arguments or launch error")
    return int(n)


def hdg_set_wait_limit(ctx: Context, first_wait_ns: int):
    """Limit of the first bounded wait of the bulk-copy order-k sweep (0 = expire at once)."""
    ctx.check(load_library().hdg_set_wait_limit(ctx.handle, int(first_wait_ns)))


def hdg_smooth(ctx: Context, level: int, g, u, n_sweeps: int = 1, reverse: bool = False, stream=None):
    ctx.check(load_library().hdg_smooth(ctx.handle, level, _ptr(g), _ptr(u), n_sweeps, int(reverse),
                                        _stream(stream)))
    return u


def hdg_prolong_add(ctx: Context, level: int, uc, uf, stream=None):
    ctx.check(load_library().hdg_prolong_add(ctx.handle, level, _ptr(uc), _ptr(uf), _stream(stream)))
    return uf


def hdg_restrict(ctx: Context, level: int, rf, rc=None, stream=None):
    import torch
    if rc is None:
        rc = torch.empty(int(ctx.sizes().n_dof_level[level - 1]), dtype=torch.float64, device=rf.device)
    ctx.check(load_library().hdg_restrict(ctx.handle, level, _ptr(rf), _ptr(rc), _stream(stream)))
    return rc


def hdg_restrict_noalloc(ctx: Context, level: int, rf, rc, stream=None):
    """hdg_restrict with its temporaries in the library's fixed scratch array (no allocation)."""
    ctx.check(load_library().hdg_restrict_noalloc(ctx.handle, level, _ptr(rf), _ptr(rc),
                                                  _stream(stream)))
    return rc


def hdg_coarse_solve(ctx: Context, g, u=None, stream=None):
    import torch
    u = torch.empty_like(g) if u is None else u
    ctx.check(load_library().hdg_coarse_solve(ctx.handle, _ptr(g), _ptr(u), _stream(stream)))
    return u


def hdg_mg_h(ctx: Context, g, u=None, stream=None):
    import torch
    u = torch.empty_like(g) if u is None else u
    ctx.check(load_library().hdg_mg_h(ctx.handle, _ptr(g), _ptr(u), _stream(stream)))
    return u


def hdg_reference_tables(k: int) -> dict:
    """Reference-element tables R1..R16 used by the device condensation and recovery (host call)."""
    lib = load_library()
    n = lib.hdg_reference_tables(k, None)
    if n < 0:
        raise HdgError(1, "k out of range")
    buf = np.empty(n, dtype=np.float64)
    lib.hdg_reference_tables(k, buf.ctypes.data_as(ctypes.c_void_p))
    npk, nrt, nf, nlat = (k + 1) * (k + 2) // 2, (k + 1) * (k + 3), k + 1, (k + 2) * (k + 3) // 2
    nq, nfq = (k + 5) ** 2, (3 * k + 5) // 2
    shapes = dict(R1=(nrt, 2, 2, npk), R2=(3, nrt, 2, npk), R3=(3, npk, nf), R4=(nrt, 2, nrt, 2),
                  R5=(nrt, npk), R6=(nrt, 2, nlat), R7=(nrt, 2, nlat), R8=(nlat, nlat),
                  R9=(nq, nrt, 2), R10=(nq, nrt, 2, 2), R11=(nq, nlat), R12=(nq,),
                  R13=(3, nfq, nrt, 2), R14=(3, nfq, nlat), R15=(nfq, nf), R16=(nfq,))
    out, o = {}, 0
    for name, shp in shapes.items():
        m = int(np.prod(shp))
        out[name] = buf[o:o + m].reshape(shp)
        o += m
    assert o == n
    return out


def hdg_kernel_launches() -> int:
    return int(load_library().hdg_kernel_launches())


def hdg_destroy(ctx: Context):
    ctx.close()
