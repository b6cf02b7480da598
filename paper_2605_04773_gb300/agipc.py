"""Thin Python binding of the C ABI in include/agipc.h.

Argument marshalling only: every function passes torch CUDA tensors' device
pointers and the context's stream to libagipc.so, and every step of the
coarsened solve runs in the library's CUDA kernels.  There is no CPU
fallback: loading fails loudly when the library is missing or when no CUDA
device is present.

The function names mirror the C entry points (agipc_aggregate,
agipc_assemble_coarse, agipc_pcg, agipc_prolongate).  DeviceScene,
CoarsenedStep and FineStep only allocate output tensors and call those four
entry points in order.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_CAPACITY = -3
ERR_NONFINITE = -4
ERR_NOT_CONVERGED = -5
ERR_TIMEOUT = -6
ERR_BAD_INDEX = -7

_lib = None


class AgipcError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, status_string(code), code))
        self.code = code


class _PcgOptions(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("rhs_sign", ctypes.c_int32),
                ("use_x0", ctypes.c_int32), ("streamed", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libagipc.so (built by build.build()).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("libagipc.so is not built (%s); run paper_2605_04773_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.agipc_create.argtypes = [ctypes.POINTER(P), P, i32, i64, i64, i64]
    lib.agipc_destroy.argtypes = [P]
    lib.agipc_set_stream.argtypes = [P, P]
    lib.agipc_set_assembly_run.argtypes = [P, ctypes.c_int32]
    lib.agipc_aggregate.argtypes = [P, i32, i64, P, P, P, P]
    lib.agipc_assemble_coarse.argtypes = [P, i32, P, P, P, P, P, i64, i64, P, P, P, P, P, P, i64, P, P, P]
    lib.agipc_pcg.argtypes = [P, i32, P, P, P, P, P, P, P, ctypes.POINTER(_PcgOptions), P, P]
    lib.agipc_prolongate.argtypes = [P, i32, P, P, P]
    lib.agipc_status.argtypes = [P]
    lib.agipc_aggregate_static.argtypes = [P, i32, i64, P, P, P, P, P]
    lib.agipc_assemble_coarse_mixed.argtypes = [P, i32, P, P, P, P, P, i64, i64, P, P, i64, P, P, P, P, P, P, P, i64,
                                                P, P, P]
    lib.agipc_pcg_mixed.argtypes = [P, i32, P, P, P, P, P, P, P, P, ctypes.POINTER(_PcgOptions), i32, P, P]
    f64 = ctypes.c_double
    lib.agipc_precision_split.argtypes = [P, i64, P, P, i64, P, P, P, f64, P, P, P, P, P]
    D3 = ctypes.POINTER(ctypes.c_double)
    lib.agipc_prolongate_add.argtypes = [P, i32, P, P, P, P]
    lib.agipc_fine_assemble_stvk.argtypes = [P, i32, i64, P, P, P, D3, P, f64, P, P, P, P, i64, P, P, P, i64]
    lib.agipc_restrict.argtypes = [P, i32, P, P, P, P]
    lib.agipc_stvk_vjp.argtypes = [P, i32, i64, P, P, P, P, f64, P, P, P, P, P, P, i64]
    lib.agipc_stvk_workspace_bytes.argtypes = [i64]
    lib.agipc_stvk_workspace_bytes.restype = i64
    lib.agipc_batch_coarse_offsets.argtypes = [P, i32, i32, P, P, P, P]
    lib.agipc_strain_tags.argtypes = [P, i32, i64, P, P, P, P, f64, P, P, i64, i64, P]
    lib.agipc_affine_plan.argtypes = [P, i32, P, P, i32, P, P, P]
    lib.agipc_assemble_affine.argtypes = [P, i32, P, P, P, P, P, P, P, P, P, P, P, i64, i64, P, P, P, P, P, P, i64,
                                          P, P, P]
    lib.agipc_prolongate_affine.argtypes = [P, i32, P, P, P, P, P, P, P]
    lib.agipc_pcg_batched.argtypes = [P, i32, P, i32, P, P, P, P, P, P, P, ctypes.POINTER(_PcgOptions), i32, i32, P, P]
    lib.agipc_stvk_energy.argtypes = [P, i32, i64, P, P, P, P, f64, D3, P, f64, P, P, P, P]
    lib.agipc_max_abs.argtypes = [P, i64, P, P]
    lib.agipc_status_string.argtypes = [ctypes.c_int]
    lib.agipc_status_string.restype = ctypes.c_char_p
    for name in ("agipc_create", "agipc_destroy", "agipc_set_stream", "agipc_set_assembly_run", "agipc_aggregate",
                 "agipc_assemble_coarse", "agipc_pcg", "agipc_prolongate", "agipc_status", "agipc_aggregate_static",
                 "agipc_assemble_coarse_mixed", "agipc_pcg_mixed", "agipc_precision_split", "agipc_prolongate_add", "agipc_fine_assemble_stvk",
                 "agipc_restrict", "agipc_stvk_vjp", "agipc_batch_coarse_offsets", "agipc_pcg_batched", "agipc_strain_tags", "agipc_affine_plan", "agipc_assemble_affine",
                 "agipc_prolongate_affine", "agipc_stvk_energy", "agipc_max_abs"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().agipc_status_string(code).decode()


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(rc: int, what: str):
    if rc != OK:
        raise AgipcError(rc, what)


class Context:
    """agipc_create / agipc_destroy.  Bound to torch's current CUDA stream
    unless another stream is given."""

    def __init__(self, max_fine_nodes: int, max_edges: int, max_fine_nnzb: int, max_pairs: int, stream=None):
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("the coarsening library needs a CUDA device")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.agipc_create(ctypes.byref(h), ctypes.c_void_p(self.stream.cuda_stream), int(max_fine_nodes),
                                int(max_edges), int(max_fine_nnzb), int(max_pairs)), "agipc_create")
        self.handle = h
        self.max_fine_nodes = int(max_fine_nodes)

    def set_stream(self, stream):
        self.stream = stream
        _check(load().agipc_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)), "agipc_set_stream")

    def set_assembly_run(self, terms_per_lane: int):
        """agipc_set_assembly_run: terms per lane of the coarse assembly's
        reduction (4, 8, 16 or 32)."""
        _check(load().agipc_set_assembly_run(self.handle, int(terms_per_lane)), "agipc_set_assembly_run")
        self.assembly_run = int(terms_per_lane)

    def status(self) -> int:
        """Synchronize and return (and clear) the device-side status."""
        return int(load().agipc_status(self.handle))

    def check(self, allow=(OK,)):
        rc = self.status()
        if rc not in allow:
            raise AgipcError(rc, "device status")
        return rc

    def close(self):
        if getattr(self, "handle", None):
            load().agipc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def agipc_aggregate(ctx: Context, n_fine: int, edges, tags, labels, n_coarse_dev):
    _check(load().agipc_aggregate(ctx.handle, int(n_fine), int(edges.shape[0]), _ptr(edges), _ptr(tags), _ptr(labels),
                                  _ptr(n_coarse_dev)), "agipc_aggregate")


def agipc_assemble_coarse(ctx: Context, n_fine: int, labels, n_coarse_dev, fine_row_ptr, fine_col, fine_val,
                          pair_idx, pair_blk, g, coarse_row_ptr, coarse_col, coarse_val, coarse_nnzb_dev, g_c, dinv):
    _check(load().agipc_assemble_coarse(
        ctx.handle, int(n_fine), _ptr(labels), _ptr(n_coarse_dev), _ptr(fine_row_ptr), _ptr(fine_col), _ptr(fine_val),
        int(fine_col.shape[0]), int(pair_idx.shape[0]), _ptr(pair_idx), _ptr(pair_blk), _ptr(g), _ptr(coarse_row_ptr),
        _ptr(coarse_col), _ptr(coarse_val), int(coarse_col.shape[0]), _ptr(coarse_nnzb_dev), _ptr(g_c), _ptr(dinv)),
        "agipc_assemble_coarse")


def agipc_pcg(ctx: Context, max_rows: int, n_rows_dev, row_ptr, col, val, dinv, b, x, tol: float, max_iter: int,
              rhs_sign: int, iters_dev, relres_dev, use_x0: bool = False, streamed: bool = False):
    opt = _PcgOptions(float(tol), int(max_iter), int(rhs_sign), 1 if use_x0 else 0, 1 if streamed else 0)
    _check(load().agipc_pcg(ctx.handle, int(max_rows), _ptr(n_rows_dev), _ptr(row_ptr), _ptr(col), _ptr(val),
                            _ptr(dinv), _ptr(b), _ptr(x), ctypes.byref(opt), _ptr(iters_dev), _ptr(relres_dev)),
           "agipc_pcg")


def agipc_prolongate(ctx: Context, n_fine: int, labels, y, dx):
    _check(load().agipc_prolongate(ctx.handle, int(n_fine), _ptr(labels), _ptr(y), _ptr(dx)), "agipc_prolongate")


def agipc_precision_split(ctx: Context, val, val32, pair_idx, pair_blk, pair_gap, gap_limit: float, pair_idx32,
                          pair_blk32, pair_idx64, pair_blk64, counts_dev):
    _check(load().agipc_precision_split(
        ctx.handle, int(val.shape[0]), _ptr(val), _ptr(val32), int(pair_idx.shape[0]), _ptr(pair_idx),
        _ptr(pair_blk), _ptr(pair_gap), float(gap_limit), _ptr(pair_idx32), _ptr(pair_blk32), _ptr(pair_idx64),
        _ptr(pair_blk64), _ptr(counts_dev)), "agipc_precision_split")


def agipc_assemble_coarse_mixed(ctx: Context, n_fine: int, labels, n_coarse_dev, fine_row_ptr, fine_col, fine_val32,
                                pair_idx32, pair_blk32, pair_idx64, pair_blk64, g, coarse_row_ptr, coarse_col,
                                coarse_val, coarse_val32, coarse_nnzb_dev, g_c, dinv32):
    _check(load().agipc_assemble_coarse_mixed(
        ctx.handle, int(n_fine), _ptr(labels), _ptr(n_coarse_dev), _ptr(fine_row_ptr), _ptr(fine_col),
        _ptr(fine_val32), int(fine_col.shape[0]), int(pair_idx32.shape[0]), _ptr(pair_idx32), _ptr(pair_blk32),
        int(pair_idx64.shape[0]), _ptr(pair_idx64), _ptr(pair_blk64), _ptr(g), _ptr(coarse_row_ptr), _ptr(coarse_col),
        _ptr(coarse_val), _ptr(coarse_val32), int(coarse_col.shape[0]), _ptr(coarse_nnzb_dev), _ptr(g_c),
        _ptr(dinv32)), "agipc_assemble_coarse_mixed")


def agipc_pcg_mixed(ctx: Context, max_rows: int, n_rows_dev, row_ptr, col, val, val32, dinv32, b, x, tol: float,
                    max_iter: int, rhs_sign: int, refine_every: int, iters_dev, relres_dev, streamed: bool = False):
    opt = _PcgOptions(float(tol), int(max_iter), int(rhs_sign), 0, 1 if streamed else 0)
    _check(load().agipc_pcg_mixed(ctx.handle, int(max_rows), _ptr(n_rows_dev), _ptr(row_ptr), _ptr(col), _ptr(val),
                                  _ptr(val32), _ptr(dinv32), _ptr(b), _ptr(x), ctypes.byref(opt), int(refine_every),
                                  _ptr(iters_dev), _ptr(relres_dev)), "agipc_pcg_mixed")


def agipc_prolongate_add(ctx: Context, n_fine: int, labels, y, base, out):
    _check(load().agipc_prolongate_add(ctx.handle, int(n_fine), _ptr(labels), _ptr(y), _ptr(base), _ptr(out)),
           "agipc_prolongate_add")


def stvk_workspace(n_tets: int, device="cuda"):
    """A device workspace for agipc_fine_assemble_stvk / agipc_stvk_vjp."""
    nbytes = int(load().agipc_stvk_workspace_bytes(int(n_tets)))
    return torch.empty((nbytes + 7) // 8, dtype=torch.int64, device=device)


def agipc_fine_assemble_stvk(ctx: Context, n_fine: int, tets, X_rest, x, xhat_shift, E, nu: float, mass_h2,
                             g_extra, fine_row_ptr, fine_col, fine_val, g, workspace):
    shift = (ctypes.c_double * 3)(*[float(v) for v in xhat_shift])
    _check(load().agipc_fine_assemble_stvk(
        ctx.handle, int(n_fine), int(tets.shape[0]), _ptr(tets), _ptr(X_rest), _ptr(x), shift, _ptr(E), float(nu),
        _ptr(mass_h2), _ptr(g_extra), _ptr(fine_row_ptr), _ptr(fine_col), int(fine_col.shape[0]), _ptr(fine_val),
        _ptr(g), _ptr(workspace), 8 * int(workspace.numel())), "agipc_fine_assemble_stvk")


def agipc_restrict(ctx: Context, n_fine: int, labels, n_coarse_dev, v, v_c):
    _check(load().agipc_restrict(ctx.handle, int(n_fine), _ptr(labels), _ptr(n_coarse_dev), _ptr(v), _ptr(v_c)),
           "agipc_restrict")


def agipc_stvk_vjp(ctx: Context, n_fine: int, tets, X_rest, x, E, nu: float, mass_h2, lam, dx, dL_dE, dL_dX_rest,
                   workspace):
    _check(load().agipc_stvk_vjp(ctx.handle, int(n_fine), int(tets.shape[0]), _ptr(tets), _ptr(X_rest), _ptr(x),
                                 _ptr(E), float(nu), _ptr(mass_h2), _ptr(lam), _ptr(dx), _ptr(dL_dE),
                                 _ptr(dL_dX_rest), _ptr(workspace), 8 * int(workspace.numel())), "agipc_stvk_vjp")


def agipc_strain_tags(ctx: Context, n_fine: int, tets, X_rest, x_prev, x_cur, threshold: float, fine_row_ptr,
                      fine_col, tags):
    _check(load().agipc_strain_tags(ctx.handle, int(n_fine), int(tets.shape[0]), _ptr(tets), _ptr(X_rest),
                                    _ptr(x_prev), _ptr(x_cur), float(threshold), _ptr(fine_row_ptr), _ptr(fine_col),
                                    int(fine_col.shape[0]), int(tags.shape[0]), _ptr(tags)), "agipc_strain_tags")


def agipc_stvk_energy(ctx: Context, n_fine: int, tets, X_rest, x0, d, alpha: float, xhat_shift, E, nu: float,
                      mass_h2, g_extra, x_out, energy_dev):
    shift = (ctypes.c_double * 3)(*[float(v) for v in xhat_shift])
    _check(load().agipc_stvk_energy(ctx.handle, int(n_fine), int(tets.shape[0]), _ptr(tets), _ptr(X_rest), _ptr(x0),
                                    _ptr(d), float(alpha), shift, _ptr(E), float(nu), _ptr(mass_h2), _ptr(g_extra),
                                    _ptr(x_out), _ptr(energy_dev)), "agipc_stvk_energy")


def agipc_max_abs(ctx: Context, v, out_dev):
    _check(load().agipc_max_abs(ctx.handle, int(v.numel()), _ptr(v), _ptr(out_dev)), "agipc_max_abs")


BATCH_MAX_INSTANCES = 512
BATCH_TILES = (4, 5, 6, 8)
ASSEMBLY_RUNS = (4, 8, 16, 32)   # terms per lane of the coarse assembly's reduction


def agipc_batch_coarse_offsets(ctx: Context, n_inst: int, n_fine: int, vert_ptr, labels, n_coarse_dev, inst_row):
    _check(load().agipc_batch_coarse_offsets(ctx.handle, int(n_inst), int(n_fine), _ptr(vert_ptr), _ptr(labels),
                                             _ptr(n_coarse_dev), _ptr(inst_row)), "agipc_batch_coarse_offsets")


def agipc_pcg_batched(ctx: Context, n_inst: int, inst_row, max_rows: int, row_ptr, col, val, val32, dinv32, b, x,
                      tol: float, max_iter: int, rhs_sign: int, refine_every: int, blocks_per_lane: int, iters_dev,
                      relres_dev):
    opt = _PcgOptions(float(tol), int(max_iter), int(rhs_sign), 0)
    _check(load().agipc_pcg_batched(ctx.handle, int(n_inst), _ptr(inst_row), int(max_rows), _ptr(row_ptr), _ptr(col),
                                    _ptr(val), _ptr(val32), _ptr(dinv32), _ptr(b), _ptr(x), ctypes.byref(opt),
                                    int(refine_every), int(blocks_per_lane), _ptr(iters_dev), _ptr(relres_dev)),
           "agipc_pcg_batched")


AGGREGATE_STATIC_MAX_NODES = 1 << 20


def agipc_aggregate_static(stream, n_fine: int, edges, tags, labels, n_coarse_dev, status_dev):
    """The labeller for callers that cannot allocate GPU memory (no Context):
    its scratch is a fixed array inside the library, so n_fine is limited to
    AGGREGATE_STATIC_MAX_NODES and calls that overlap on the GPU race.
    status_dev (uint32 device scalar) receives the device-side error bits."""
    _check(load().agipc_aggregate_static(ctypes.c_void_p(stream.cuda_stream), int(n_fine), int(edges.shape[0]),
                                         _ptr(edges), _ptr(tags), _ptr(labels), _ptr(n_coarse_dev),
                                         _ptr(status_dev)), "agipc_aggregate_static")


# ---------------------------------------------------------------------------
# Allocation helpers (marshalling only)
# ---------------------------------------------------------------------------


class DeviceScene:
    """A scene's solve inputs as contiguous device tensors."""

    def __init__(self, sc, device="cuda"):
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)  # noqa: E731
        self.n = sc.n
        self.edges = t(sc.edges, torch.int32)
        self.tags = t(sc.tags, torch.uint8)
        self.row_ptr = t(sc.row_ptr, torch.int32)
        self.col = t(sc.col, torch.int32)
        self.val = t(sc.val.reshape(-1, 9), torch.float64)
        self.pair_idx = t(sc.pair_idx.reshape(-1, 4), torch.int32)
        self.pair_blk = t(sc.pair_blk.reshape(-1, 90), torch.float64)
        self.g = t(sc.g.reshape(-1, 3), torch.float64)

    @property
    def capacity(self) -> int:
        return 2 * int(self.col.shape[0]) + 16 * int(self.pair_idx.shape[0])

    def context(self) -> Context:
        return Context(self.n, self.edges.shape[0], self.col.shape[0], self.pair_idx.shape[0])


class CoarsenedStep:
    """Output buffers of one coarsened Newton-step solve and the four calls
    that fill them: aggregate -> assemble_coarse -> pcg -> prolongate."""

    def __init__(self, ctx: Context, ds: DeviceScene, tol: float, max_iter: int = 100000, streamed: bool = False):
        dev = ds.g.device
        n, cap = ds.n, ds.capacity
        i32 = dict(device=dev, dtype=torch.int32)
        f64 = dict(device=dev, dtype=torch.float64)
        self.ctx, self.ds, self.tol, self.max_iter = ctx, ds, tol, max_iter
        self.streamed = streamed   # the 16-warp streaming PCG (systems larger than shared memory)
        self.labels = torch.empty(n, **i32)
        self.n_c = torch.zeros(1, **i32)
        self.row_ptr = torch.empty(n + 1, **i32)
        self.col = torch.empty(cap, **i32)
        self.val = torch.empty(cap, 9, **f64)
        self.nnz = torch.zeros(1, **i32)
        self.g_c = torch.empty(n, 3, **f64)
        self.dinv = torch.empty(n, 9, **f64)
        self.y = torch.empty(n, 3, **f64)
        self.dx = torch.empty(n, 3, **f64)
        self.iters = torch.zeros(1, **i32)
        self.relres = torch.zeros(1, **f64)

    def aggregate(self, tags=None):
        ds = self.ds
        agipc_aggregate(self.ctx, ds.n, ds.edges, ds.tags if tags is None else tags, self.labels, self.n_c)

    def assemble(self):
        ds = self.ds
        agipc_assemble_coarse(self.ctx, ds.n, self.labels, self.n_c, ds.row_ptr, ds.col, ds.val, ds.pair_idx,
                              ds.pair_blk, ds.g, self.row_ptr, self.col, self.val, self.nnz, self.g_c, self.dinv)

    def solve(self):
        agipc_pcg(self.ctx, self.ds.n, self.n_c, self.row_ptr, self.col, self.val, self.dinv, self.g_c, self.y,
                  self.tol, self.max_iter, -1, self.iters, self.relres, streamed=self.streamed)

    def prolongate(self):
        agipc_prolongate(self.ctx, self.ds.n, self.labels, self.y, self.dx)

    def run(self, tags=None):
        self.aggregate(tags)
        self.assemble()
        self.solve()
        self.prolongate()

    def host(self):
        """Copy the results to host numpy arrays (synchronizes)."""
        nc = int(self.n_c.item())
        nnz = int(self.nnz.item())
        return dict(labels=self.labels.cpu().numpy(), n_c=nc, row_ptr=self.row_ptr[:nc + 1].cpu().numpy(),
                    col=self.col[:nnz].cpu().numpy(), val=self.val[:nnz].cpu().numpy().reshape(-1, 3, 3),
                    g_c=self.g_c[:nc].cpu().numpy(), dinv=self.dinv[:nc].cpu().numpy().reshape(-1, 3, 3),
                    y=self.y[:nc].cpu().numpy(), dx=self.dx.cpu().numpy(), iters=int(self.iters.item()),
                    relres=float(self.relres.item()))


SCENE_INPUTS = ("edges", "tags", "row_ptr", "col", "val", "pair_idx", "pair_blk", "g")


class HostPipeline:
    """Coarsened steps whose inputs arrive in pinned host memory, one after
    another, as a serving loop runs them: two sets of device input buffers;
    the host-to-device copies of step k+1 and the device-to-host copy of
    step k-1's dx run on a copy stream while step k's kernels run on the
    context's stream.  Both steps share the context (their kernels are
    ordered on its stream)."""

    def __init__(self, ctx: Context, buffers, tol: float, max_iter: int = 100000):
        if len(buffers) != 2:
            raise ValueError("two DeviceScene buffers are needed")
        self.ctx = ctx
        self.bufs = tuple(buffers)
        self.steps = [CoarsenedStep(ctx, b, tol, max_iter) for b in self.bufs]
        self.copy_stream = torch.cuda.Stream(device=self.bufs[0].g.device)
        self.copied = [torch.cuda.Event() for _ in range(2)]   # inputs of buffer set i are on the device
        self.free = [torch.cuda.Event() for _ in range(2)]     # buffer set i's step has run
        self.read = [torch.cuda.Event() for _ in range(2)]     # its dx has reached the host

    def run(self, host_inputs, dx_out):
        """Enqueue len(host_inputs) steps.  host_inputs[k] maps every name of
        SCENE_INPUTS to a pinned CPU tensor shaped like the DeviceScene's;
        dx_out[k] is a pinned CPU tensor [n, 3] that receives step k's dx.
        Asynchronous: synchronize (or read the context's status) before using
        dx_out."""
        comp = self.ctx.stream
        n = len(host_inputs)
        if len(dx_out) != n:
            raise ValueError("one dx buffer per step")
        for e in self.free + self.read:
            e.record(comp)

        def issue(k):
            # step k's inputs, once buffer set k % 2's previous step has run
            i = k % 2
            self.copy_stream.wait_event(self.free[i])
            with torch.cuda.stream(self.copy_stream):
                for f in SCENE_INPUTS:
                    getattr(self.bufs[i], f).copy_(host_inputs[k][f], non_blocking=True)
            self.copied[i].record(self.copy_stream)

        if n:
            issue(0)
        for k in range(n):
            i = k % 2
            if k + 1 < n:
                issue(k + 1)
            comp.wait_event(self.copied[i])
            comp.wait_event(self.read[i])     # step k-2's dx has left steps[i].dx
            self.steps[i].run()
            self.free[i].record(comp)
            self.copy_stream.wait_event(self.free[i])
            with torch.cuda.stream(self.copy_stream):
                dx_out[k].copy_(self.steps[i].dx, non_blocking=True)
            self.read[i].record(self.copy_stream)
        comp.wait_stream(self.copy_stream)    # the caller's synchronisation covers the last copies


class MixedDeviceScene(DeviceScene):
    """DeviceScene plus the precision form's inputs, made on the GPU by
    agipc_precision_split from the FP64 blocks, stencils and gaps: FP32 fine
    blocks and stencils, FP64 stencils of gaps below fp64_gap * dhat."""

    def __init__(self, sc, device="cuda", fp64_gap: float = 0.05):
        super().__init__(sc, device)
        dev = self.g.device
        P = int(self.pair_idx.shape[0])
        gap = np.asarray(sc.meta["pair_d"], dtype=np.float64) if P else np.zeros(0)
        self.pair_gap = torch.from_numpy(np.ascontiguousarray(gap)).to(device=dev)
        self.gap_limit = float(fp64_gap) * float(sc.meta["dhat"])
        self.val32 = torch.empty(self.val.shape[0], 9, device=dev, dtype=torch.float32)
        idx32 = torch.empty(P, 4, device=dev, dtype=torch.int32)
        blk32 = torch.empty(P, 90, device=dev, dtype=torch.float32)
        idx64 = torch.empty(P, 4, device=dev, dtype=torch.int32)
        blk64 = torch.empty(P, 90, device=dev, dtype=torch.float64)
        counts = torch.zeros(2, device=dev, dtype=torch.int32)
        ctx = self.context()
        agipc_precision_split(ctx, self.val, self.val32, self.pair_idx, self.pair_blk, self.pair_gap, self.gap_limit,
                              idx32, blk32, idx64, blk64, counts)
        ctx.check()
        ctx.close()
        n32, n64 = (int(c) for c in counts.cpu())
        self.pair_idx32, self.pair_blk32 = idx32[:n32], blk32[:n32]
        self.pair_idx64, self.pair_blk64 = idx64[:n64], blk64[:n64]


class MixedStep(CoarsenedStep):
    """The precision form of the step: FP32 blocks, SpMV and preconditioner,
    FP64 dot products, FP64 residual replacement every refine_every
    iterations against the FP64 master coarse matrix."""

    def __init__(self, ctx: Context, ds: MixedDeviceScene, tol: float, max_iter: int = 100000,
                 refine_every: int = 20, streamed: bool = False):
        super().__init__(ctx, ds, tol, max_iter, streamed=streamed)
        self.refine_every = refine_every
        self.val32 = torch.empty(ds.capacity, 9, device=ds.g.device, dtype=torch.float32)
        self.dinv32 = torch.empty(ds.n, 9, device=ds.g.device, dtype=torch.float32)

    def assemble(self):
        ds = self.ds
        agipc_assemble_coarse_mixed(self.ctx, ds.n, self.labels, self.n_c, ds.row_ptr, ds.col, ds.val32,
                                    ds.pair_idx32, ds.pair_blk32, ds.pair_idx64, ds.pair_blk64, ds.g, self.row_ptr,
                                    self.col, self.val, self.val32, self.nnz, self.g_c, self.dinv32)

    def solve(self):
        agipc_pcg_mixed(self.ctx, self.ds.n, self.n_c, self.row_ptr, self.col, self.val, self.val32, self.dinv32,
                        self.g_c, self.y, self.tol, self.max_iter, -1, self.refine_every, self.iters, self.relres,
                        streamed=self.streamed)

    def host(self):
        out = super().host()
        nnz = out["col"].size
        out["val32"] = self.val32[:nnz].cpu().numpy().reshape(-1, 3, 3)
        out["dinv32"] = self.dinv32[:out["n_c"]].cpu().numpy().reshape(-1, 3, 3)
        return out


class MixedFineStep:
    """The fine system (identity labels, contacts merged) solved in the
    precision form: FP32 blocks, SpMV and preconditioner, FP64 dots and
    residual replacement against the FP64 master."""

    def __init__(self, ctx: Context, ds: MixedDeviceScene, tol: float, max_iter: int = 100000,
                 refine_every: int = 20, streamed: bool = True):
        self.inner = MixedStep(ctx, ds, tol, max_iter, refine_every, streamed=streamed)
        self.inner.labels.copy_(torch.arange(ds.n, dtype=torch.int32, device=ds.g.device))
        self.inner.n_c.fill_(ds.n)

    def assemble(self):
        self.inner.assemble()

    def solve(self):
        self.inner.solve()

    def host(self):
        return self.inner.host()


class PostCoarsening:
    """Post-coarsening (Sec. 4.3): at most max_iter block-Jacobi PCG
    iterations on the fine system, started from the prolongated coarse step
    dx (agipc_pcg with an initial guess).  The fine system is the identity-
    label assembly (contacts merged, full storage)."""

    def __init__(self, ctx: Context, ds: DeviceScene, tol: float, max_iter: int = 10):
        self.fine = FineStep(ctx, ds, tol, max_iter)
        self.ctx, self.ds, self.tol, self.max_iter = ctx, ds, tol, max_iter
        self.x = torch.empty(ds.n, 3, device=ds.g.device, dtype=torch.float64)

    def assemble(self):
        self.fine.inner.assemble()

    def refine(self, dx):
        """x = dx, then up to max_iter PCG iterations on H x = -g."""
        f = self.fine.inner
        self.x.copy_(dx)
        agipc_pcg(self.ctx, self.ds.n, f.n_c, f.row_ptr, f.col, f.val, f.dinv, f.g_c, self.x, self.tol, self.max_iter,
                  -1, f.iters, f.relres, use_x0=True, streamed=f.streamed)
        return self.x


class FineStep:
    """The no-coarsening arm: identity labels (the fine system in full
    storage, contacts merged) and PCG on the fine matrix."""

    def __init__(self, ctx: Context, ds: DeviceScene, tol: float, max_iter: int = 100000, streamed: bool = True):
        self.inner = CoarsenedStep(ctx, ds, tol, max_iter, streamed=streamed)
        self.inner.labels.copy_(torch.arange(ds.n, dtype=torch.int32, device=ds.g.device))
        self.inner.n_c.fill_(ds.n)

    def run(self):
        self.inner.assemble()
        self.inner.solve()

    def host(self):
        return self.inner.host()


# ---------------------------------------------------------------------------
# Differentiation form
# ---------------------------------------------------------------------------

GRAVITY = (0.0, 0.0, -9.81)


class DiffDeviceProblem:
    """The differentiation form's constant inputs on the device: topology,
    fine upper BSR structure, current positions, M/h^2, contact terms."""

    def __init__(self, problem: dict, device="cuda"):
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)  # noqa: E731
        self.n = int(problem["n"])
        self.nu = float(problem["nu"])
        self.h = float(problem["h"])
        self.tets = t(problem["tets"], torch.int32)
        self.edges = t(problem["edges"], torch.int32)
        self.tags = t(problem["tags"], torch.uint8)
        self.row_ptr = t(problem["row_ptr"], torch.int32)
        self.col = t(problem["col"], torch.int32)
        self.x = t(problem["x"], torch.float64)
        self.mass_h2 = t(problem["mass_h2"], torch.float64)
        self.pair_idx = t(np.asarray(problem["pair_idx"]).reshape(-1, 4), torch.int32)
        self.pair_blk = t(np.asarray(problem["pair_blk"]).reshape(-1, 90), torch.float64)
        gp = problem.get("g_extra")
        if gp is None:
            gp = problem.get("g_pairs")
        self.g_extra = None if gp is None or not np.any(gp) else t(gp, torch.float64)
        self.xhat_shift = tuple(self.h * self.h * gv for gv in GRAVITY)

    @property
    def capacity(self) -> int:
        return 2 * int(self.col.shape[0]) + 16 * int(self.pair_idx.shape[0])

    def context(self) -> Context:
        return Context(self.n, self.edges.shape[0], self.col.shape[0], max(1, self.pair_idx.shape[0]))


class DiffStep:
    """Buffers and calls of the differentiation form.

    forward(E, X_rest): fine StVK assembly -> labels -> coarse assembly ->
    PCG -> x_next = x + U^T y.  backward(v): v_c = U v -> PCG on the same
    coarse system -> lambda = U^T lambda_c -> per-element VJP."""

    def __init__(self, ctx: Context, dp: DiffDeviceProblem, tol: float, max_iter: int = 100000,
                 adjoint_tol: float = None):
        dev = dp.x.device
        n, cap = dp.n, dp.capacity
        i32 = dict(device=dev, dtype=torch.int32)
        f64 = dict(device=dev, dtype=torch.float64)
        self.ctx, self.dp, self.tol, self.max_iter = ctx, dp, tol, max_iter
        self.adjoint_tol = tol if adjoint_tol is None else adjoint_tol
        self.fine_val = torch.empty(dp.col.shape[0], 9, **f64)
        self.g = torch.empty(n, 3, **f64)
        self.labels = torch.empty(n, **i32)
        self.n_c = torch.zeros(1, **i32)
        self.row_ptr = torch.empty(n + 1, **i32)
        self.col = torch.empty(cap, **i32)
        self.val = torch.empty(cap, 9, **f64)
        self.nnz = torch.zeros(1, **i32)
        self.g_c = torch.empty(n, 3, **f64)
        self.dinv = torch.empty(n, 9, **f64)
        self.y = torch.empty(n, 3, **f64)
        self.x_next = torch.empty(n, 3, **f64)
        self.dx = torch.empty(n, 3, **f64)
        self.iters = torch.zeros(1, **i32)
        self.relres = torch.zeros(1, **f64)
        self.v_c = torch.empty(n, 3, **f64)
        self.lam_c = torch.empty(n, 3, **f64)
        self.lam = torch.empty(n, 3, **f64)
        self.adj_iters = torch.zeros(1, **i32)
        self.adj_relres = torch.zeros(1, **f64)
        self.dL_dE = torch.empty(dp.tets.shape[0], **f64)
        self.dL_dX = torch.empty(n, 3, **f64)
        self.workspace = stvk_workspace(dp.tets.shape[0], dev)
        self.E = None
        self.X_rest = None

    def forward(self, E, X_rest):
        dp, ctx = self.dp, self.ctx
        self.E, self.X_rest = E, X_rest
        agipc_fine_assemble_stvk(ctx, dp.n, dp.tets, X_rest, dp.x, dp.xhat_shift, E, dp.nu, dp.mass_h2, dp.g_extra,
                                 dp.row_ptr, dp.col, self.fine_val, self.g, self.workspace)
        agipc_aggregate(ctx, dp.n, dp.edges, dp.tags, self.labels, self.n_c)
        agipc_assemble_coarse(ctx, dp.n, self.labels, self.n_c, dp.row_ptr, dp.col, self.fine_val, dp.pair_idx,
                              dp.pair_blk, self.g, self.row_ptr, self.col, self.val, self.nnz, self.g_c, self.dinv)
        agipc_pcg(ctx, dp.n, self.n_c, self.row_ptr, self.col, self.val, self.dinv, self.g_c, self.y, self.tol,
                  self.max_iter, -1, self.iters, self.relres)
        agipc_prolongate(ctx, dp.n, self.labels, self.y, self.dx)
        agipc_prolongate_add(ctx, dp.n, self.labels, self.y, dp.x, self.x_next)
        return self.x_next

    def backward(self, v):
        dp, ctx = self.dp, self.ctx
        v = v.contiguous()
        agipc_restrict(ctx, dp.n, self.labels, self.n_c, v, self.v_c)
        agipc_pcg(ctx, dp.n, self.n_c, self.row_ptr, self.col, self.val, self.dinv, self.v_c, self.lam_c,
                  self.adjoint_tol, self.max_iter, 1, self.adj_iters, self.adj_relres)
        agipc_prolongate(ctx, dp.n, self.labels, self.lam_c, self.lam)
        agipc_stvk_vjp(ctx, dp.n, dp.tets, self.X_rest, dp.x, self.E, dp.nu, dp.mass_h2, self.lam, self.dx,
                       self.dL_dE, self.dL_dX, self.workspace)
        return self.dL_dE, self.dL_dX


class CoarsenedStepFunction(torch.autograd.Function):
    """x_next = step(E, X_rest) with the hand-written adjoint as backward.
    Aggregation is piecewise constant in the parameters; x is data."""

    @staticmethod
    def forward(fctx, E, X_rest, step: DiffStep):
        fctx.step = step
        return step.forward(E.detach().contiguous(), X_rest.detach().contiguous()).clone()

    @staticmethod
    def backward(fctx, grad_x_next):
        dE, dX = fctx.step.backward(grad_x_next)
        return dE.clone(), dX.clone(), None


def coarsened_step(E, X_rest, step: DiffStep):
    """Differentiable coarsened Newton step (see CoarsenedStepFunction)."""
    return CoarsenedStepFunction.apply(E, X_rest, step)


class NewtonSolver:
    """The coarsened Newton loop with backtracking line search (the inner
    loop of Algorithm 1) on the StVK problem without contact.  Per
    iteration, on the device: fine assembly (agipc_fine_assemble_stvk), tags
    from the Green-strain increment against the previous iterate
    (agipc_strain_tags; at the first iteration against x_last, the previous
    time step), labels, coarse assembly, coarse PCG, prolongation,
    post-coarsening (at most post_iters fine PCG iterations from d) and
    |d|_inf; then alpha = 1, 1/2, ... until E(x_prev + alpha d) <
    E_prev (agipc_stvk_energy).  The loop stops when |d|_inf / h <= eps_d
    (default 1e-3 l, l the rest bounding-box diagonal).  The host reads two
    scalars per line-search trial and the status once per iteration."""

    def __init__(self, ctx: Context, dp: DiffDeviceProblem, E, X_rest, x_last, threshold: float = 5e-5,
                 tol: float = 1e-3, eps_d: float = None, max_newton: int = 50, post_iters: int = 10,
                 max_halvings: int = 30, max_iter: int = 100000):
        dev = dp.x.device
        n, cap = dp.n, dp.capacity
        i32 = dict(device=dev, dtype=torch.int32)
        f64 = dict(device=dev, dtype=torch.float64)
        self.ctx, self.dp = ctx, dp
        self.E = E.contiguous()
        self.X_rest = X_rest.contiguous()
        self.threshold, self.tol, self.max_newton = float(threshold), float(tol), int(max_newton)
        self.post_iters, self.max_halvings, self.max_iter = int(post_iters), int(max_halvings), int(max_iter)
        if eps_d is None:
            ext = (self.X_rest.max(0).values - self.X_rest.min(0).values).cpu().numpy()
            eps_d = 1e-3 * float(np.linalg.norm(ext))
        self.eps_d = float(eps_d)
        self.x_start = dp.x
        self.x = torch.empty(n, 3, **f64)
        self.x_trial = torch.empty(n, 3, **f64)
        self.x_before = torch.empty(n, 3, **f64)
        self.x_last = x_last.contiguous()
        self.fine_val = torch.empty(dp.col.shape[0], 9, **f64)
        self.g = torch.empty(n, 3, **f64)
        self.tags = torch.empty(dp.edges.shape[0], device=dev, dtype=torch.uint8)
        self.labels = torch.empty(n, **i32)
        self.n_c = torch.zeros(1, **i32)
        self.row_ptr = torch.empty(n + 1, **i32)
        self.col = torch.empty(cap, **i32)
        self.val = torch.empty(cap, 9, **f64)
        self.nnz = torch.zeros(1, **i32)
        self.g_c = torch.empty(n, 3, **f64)
        self.dinv = torch.empty(n, 9, **f64)
        self.y = torch.empty(n, 3, **f64)
        self.d = torch.empty(n, 3, **f64)
        self.iters = torch.zeros(1, **i32)
        self.relres = torch.zeros(1, **f64)
        # the fine system in full storage for the post-coarsening (identity labels)
        self.ident = torch.arange(n, **i32)
        self.n_ident = torch.full((1,), n, **i32)
        self.f_row_ptr = torch.empty(n + 1, **i32)
        self.f_col = torch.empty(cap, **i32)
        self.f_val = torch.empty(cap, 9, **f64)
        self.f_nnz = torch.zeros(1, **i32)
        self.f_g = torch.empty(n, 3, **f64)
        self.f_dinv = torch.empty(n, 9, **f64)
        self.p_iters = torch.zeros(1, **i32)
        self.p_relres = torch.zeros(1, **f64)
        self.scal = torch.zeros(2, **f64)       # [energy, |d|_inf]
        self.workspace = stvk_workspace(dp.tets.shape[0], dev)
        self.history = []

    def energy(self, x0, d=None, alpha: float = 0.0, x_out=None) -> float:
        dp = self.dp
        agipc_stvk_energy(self.ctx, dp.n, dp.tets, self.X_rest, x0, d, alpha, dp.xhat_shift, self.E, dp.nu,
                          dp.mass_h2, dp.g_extra, x_out, self.scal[:1])
        return float(self.scal[0].item())

    def direction(self, x, x_before):
        """Enqueue the steps from the fine assembly at x to d (post-coarsened)
        and |d|_inf; the coarse solve's status is checked on the host."""
        dp, ctx = self.dp, self.ctx
        agipc_fine_assemble_stvk(ctx, dp.n, dp.tets, self.X_rest, x, dp.xhat_shift, self.E, dp.nu, dp.mass_h2,
                                 dp.g_extra, dp.row_ptr, dp.col, self.fine_val, self.g, self.workspace)
        agipc_strain_tags(ctx, dp.n, dp.tets, self.X_rest, x_before, x, self.threshold, dp.row_ptr, dp.col, self.tags)
        agipc_aggregate(ctx, dp.n, dp.edges, self.tags, self.labels, self.n_c)
        agipc_assemble_coarse(ctx, dp.n, self.labels, self.n_c, dp.row_ptr, dp.col, self.fine_val, dp.pair_idx,
                              dp.pair_blk, self.g, self.row_ptr, self.col, self.val, self.nnz, self.g_c, self.dinv)
        agipc_pcg(ctx, dp.n, self.n_c, self.row_ptr, self.col, self.val, self.dinv, self.g_c, self.y, self.tol,
                  self.max_iter, -1, self.iters, self.relres)
        agipc_prolongate(ctx, dp.n, self.labels, self.y, self.d)
        if self.post_iters > 0:
            agipc_assemble_coarse(ctx, dp.n, self.ident, self.n_ident, dp.row_ptr, dp.col, self.fine_val, dp.pair_idx,
                                  dp.pair_blk, self.g, self.f_row_ptr, self.f_col, self.f_val, self.f_nnz, self.f_g,
                                  self.f_dinv)
            ctx.check()
            agipc_pcg(ctx, dp.n, self.n_ident, self.f_row_ptr, self.f_col, self.f_val, self.f_dinv, self.f_g, self.d,
                      self.tol, self.post_iters, -1, self.p_iters, self.p_relres, use_x0=True)
            ctx.check(allow=(OK, ERR_NOT_CONVERGED))   # the post-coarsening is capped on purpose
        else:
            ctx.check()
        agipc_max_abs(ctx, self.d, self.scal[1:])

    def run(self, keep_labels: bool = False):
        """The whole loop from the problem's x.  Returns dict(x, history,
        converged, stalled, iterations)."""
        dp = self.dp
        self.x.copy_(self.x_start)
        self.x_before.copy_(self.x_last)
        e_prev = self.energy(self.x)
        self.history = []
        converged = stalled = False
        for _ in range(self.max_newton):
            self.direction(self.x, self.x_before)
            dnorm = float(self.scal[1].item())
            alpha, e_new, trials = 1.0, None, 0
            for k in range(self.max_halvings + 1):
                e = self.energy(self.x, self.d, alpha, self.x_trial)
                trials = k + 1
                if e < e_prev:
                    e_new = e
                    break
                alpha *= 0.5
            rec = dict(e_prev=e_prev, n_c=int(self.n_c.item()), coarse_iters=int(self.iters.item()),
                       post_iters=int(self.p_iters.item()) if self.post_iters > 0 else 0, dnorm=dnorm,
                       alpha=alpha if e_new is not None else None, trials=trials, e_new=e_new)
            if keep_labels:
                rec["labels"] = self.labels.cpu().numpy()
                rec["d"] = self.d.cpu().numpy()
            self.history.append(rec)
            if e_new is None:
                converged = dnorm / dp.h <= self.eps_d
                stalled = not converged
                break
            # rotate: x_before <- x, x <- x_trial
            self.x_before, self.x, self.x_trial = self.x, self.x_trial, self.x_before
            e_prev = e_new
            if dnorm / dp.h <= self.eps_d:
                converged = True
                break
        self.ctx.check()
        return dict(x=self.x, history=self.history, converged=converged, stalled=stalled,
                    iterations=len(self.history))


# ---------------------------------------------------------------------------
# Batched form
# ---------------------------------------------------------------------------


class BatchDevice:
    """A Batch's inputs on the device.  Fine blocks and stencils are FP32
    (the batched form's precision); the gradient is FP64.  Instances whose
    numpy values are missing (NaN) get them from agipc_fine_assemble_stvk
    (FP64, then rounded), which evaluates the same StVK physics."""

    def __init__(self, batch, device="cuda"):
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)  # noqa: E731
        self.n = batch.n
        self.n_inst = batch.n_inst
        self.vert_ptr = t(batch.vert_ptr, torch.int32)
        self.edges = t(batch.edges, torch.int32)
        self.tags = t(batch.tags, torch.uint8)
        self.row_ptr = t(batch.row_ptr, torch.int32)
        self.col = t(batch.col, torch.int32)
        self.pair_idx = t(batch.pair_idx.reshape(-1, 4), torch.int32)
        self.pair_blk32 = t(batch.pair_blk.reshape(-1, 90), torch.float32)
        self.pair_idx64 = torch.zeros(0, 4, dtype=torch.int32, device=device)
        self.pair_blk64 = torch.zeros(0, 90, dtype=torch.float64, device=device)
        nnzb = int(batch.col.shape[0])
        missing = batch.val is None or bool(np.isnan(batch.val).any())
        self.ctx_max_pairs = max(1, int(batch.pair_idx.shape[0]))
        val = torch.empty(nnzb, 9, dtype=torch.float64, device=device)
        g = torch.empty(self.n, 3, dtype=torch.float64, device=device)
        if missing:
            ctx = Context(self.n, self.edges.shape[0], nnzb, self.ctx_max_pairs)
            tets = t(batch.tets, torch.int32)
            ws = stvk_workspace(tets.shape[0], device)
            shift = tuple(batch.h * batch.h * gv for gv in GRAVITY)
            agipc_fine_assemble_stvk(ctx, self.n, tets, t(batch.X_rest, torch.float64), t(batch.x, torch.float64),
                                     shift, t(batch.E, torch.float64), batch.nu, t(batch.mass_h2, torch.float64),
                                     t(batch.g_pairs, torch.float64), self.row_ptr, self.col, val, g, ws)
            ctx.check()
            ctx.close()
            del tets, ws
        if batch.val is not None:
            have = ~np.isnan(batch.val.reshape(nnzb, 9)).any(1)
            hv = torch.from_numpy(np.ascontiguousarray(batch.val.reshape(nnzb, 9)[have])).to(device)
            val[torch.from_numpy(np.nonzero(have)[0]).to(device)] = hv
            gh = ~np.isnan(batch.g).any(1)
            g[torch.from_numpy(np.nonzero(gh)[0]).to(device)] = torch.from_numpy(
                np.ascontiguousarray(batch.g[gh])).to(device)
        self.val32 = val.to(torch.float32)
        self.g = g
        del val

    @property
    def capacity(self) -> int:
        return 2 * int(self.col.shape[0]) + 16 * int(self.pair_idx.shape[0])

    def context(self) -> Context:
        return Context(self.n, self.edges.shape[0], self.col.shape[0], self.ctx_max_pairs)


class BatchedStep:
    """The batched coarsened step: labels of the concatenation -> instance
    offsets -> mixed coarse assembly -> per-instance batched PCG ->
    prolongation.  run() enqueues it; capture() records it in a CUDA graph
    that replay() launches as one unit."""

    def __init__(self, ctx: Context, bd: BatchDevice, tol: float, max_iter: int = 100000, refine_every: int = 20,
                 tile: int = 5):
        dev = bd.g.device
        n, cap = bd.n, bd.capacity
        i32 = dict(device=dev, dtype=torch.int32)
        f64 = dict(device=dev, dtype=torch.float64)
        self.ctx, self.bd, self.tol, self.max_iter, self.refine_every, self.tile = ctx, bd, tol, max_iter, \
            refine_every, tile
        self.labels = torch.empty(n, **i32)
        self.n_c = torch.zeros(1, **i32)
        self.inst_row = torch.zeros(bd.n_inst + 1, **i32)
        self.row_ptr = torch.empty(n + 1, **i32)
        self.col = torch.empty(cap, **i32)
        self.val = torch.empty(cap, 9, **f64)
        self.val32 = torch.empty(cap, 9, device=dev, dtype=torch.float32)
        self.nnz = torch.zeros(1, **i32)
        self.g_c = torch.empty(n, 3, **f64)
        self.dinv32 = torch.empty(n, 9, device=dev, dtype=torch.float32)
        self.y = torch.empty(n, 3, **f64)
        self.dx = torch.empty(n, 3, **f64)
        self.iters = torch.zeros(bd.n_inst, **i32)
        self.relres = torch.zeros(bd.n_inst, **f64)
        self.graph = None

    def run(self):
        bd, ctx = self.bd, self.ctx
        agipc_aggregate(ctx, bd.n, bd.edges, bd.tags, self.labels, self.n_c)
        agipc_batch_coarse_offsets(ctx, bd.n_inst, bd.n, bd.vert_ptr, self.labels, self.n_c, self.inst_row)
        self.assemble()
        self.solve()
        agipc_prolongate(ctx, bd.n, self.labels, self.y, self.dx)

    def assemble(self):
        bd = self.bd
        agipc_assemble_coarse_mixed(self.ctx, bd.n, self.labels, self.n_c, bd.row_ptr, bd.col, bd.val32, bd.pair_idx,
                                    bd.pair_blk32, bd.pair_idx64, bd.pair_blk64, bd.g, self.row_ptr, self.col,
                                    self.val, self.val32, self.nnz, self.g_c, self.dinv32)

    def solve(self, tile: int = None):
        agipc_pcg_batched(self.ctx, self.bd.n_inst, self.inst_row, self.bd.n, self.row_ptr, self.col, self.val,
                          self.val32, self.dinv32, self.g_c, self.y, self.tol, self.max_iter, -1, self.refine_every,
                          self.tile if tile is None else tile, self.iters, self.relres)

    def capture(self):
        """Record run() in a CUDA graph on a side stream (the context is
        switched to that stream for the capture and back afterwards)."""
        side = torch.cuda.Stream(device=self.bd.g.device)
        prev = self.ctx.stream
        side.wait_stream(prev)
        self.ctx.set_stream(side)
        graph = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(graph, stream=side):
                self.run()
        finally:
            self.ctx.set_stream(prev)
        prev.wait_stream(side)
        self.graph = graph
        return graph

    def replay(self):
        self.graph.replay()

    def host(self):
        nc = int(self.n_c.item())
        nnz = int(self.nnz.item())
        return dict(labels=self.labels.cpu().numpy(), n_c=nc, inst_row=self.inst_row.cpu().numpy(),
                    row_ptr=self.row_ptr[:nc + 1].cpu().numpy(), col=self.col[:nnz].cpu().numpy(),
                    val=self.val[:nnz].cpu().numpy().reshape(-1, 3, 3),
                    val32=self.val32[:nnz].cpu().numpy().reshape(-1, 3, 3), g_c=self.g_c[:nc].cpu().numpy(),
                    y=self.y[:nc].cpu().numpy(), dx=self.dx.cpu().numpy(), iters=self.iters.cpu().numpy(),
                    relres=self.relres.cpu().numpy())


def autotune_batched(step: BatchedStep, tiles=BATCH_TILES, runs=ASSEMBLY_RUNS, reps: int = 3, cache: str = None):
    """Pick the batched form's two launch shapes by timing each candidate on
    the step's own systems after one run(), median of reps launches: the
    coarse assembly's reduction run (terms per lane, agipc_set_assembly_run;
    the assembly alone on the step's labels) and the batched PCG's slice
    width (the solve alone).  The choices are cached per device and batch
    shape in a JSON file (default: next to the library) and set on the step
    and its context.  Returns (tile, timings_ms); the run and its timings
    are in step.assembly_run and step.assembly_ms."""
    import json
    dev = step.bd.g.device
    key = "%s|n_inst=%d|n=%d|nnzb=%d" % (torch.cuda.get_device_name(dev), step.bd.n_inst, step.bd.n,
                                          int(step.bd.col.shape[0]))
    path = cache or os.path.join(os.path.dirname(library_path()), "autotune_batched.json")
    table = {}
    if os.path.exists(path):
        try:
            table = json.load(open(path))
        except (OSError, ValueError):
            table = {}
    ent = table.get(key)
    if ent and ent.get("tile") in tiles and ent.get("assembly_run") in runs:
        step.tile = int(ent["tile"])
        step.ctx.set_assembly_run(int(ent["assembly_run"]))
        step.assembly_run, step.assembly_ms = int(ent["assembly_run"]), ent["assembly_ms"]
        return step.tile, ent["ms"]
    step.run()
    step.ctx.check()
    stream = torch.cuda.current_stream(dev)

    def median_ms(fn):
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            times.append(a.elapsed_time(b))
        step.ctx.check()
        return float(np.median(times))

    asm_ms = {}
    for r in runs:
        step.ctx.set_assembly_run(r)
        asm_ms[str(r)] = median_ms(step.assemble)
    run = int(min(asm_ms, key=asm_ms.get))
    step.ctx.set_assembly_run(run)
    step.assemble()
    ms = {}
    for tile in tiles:
        ms[str(tile)] = median_ms(lambda: step.solve(tile))
    best = int(min(ms, key=ms.get))
    step.tile = best
    step.assembly_run, step.assembly_ms = run, asm_ms
    table[key] = {"tile": best, "ms": ms, "assembly_run": run, "assembly_ms": asm_ms}
    try:
        with open(path + ".tmp", "w") as f:
            json.dump(table, f, indent=1)
        os.replace(path + ".tmp", path)
    except OSError:
        pass
    return best, ms


# ---------------------------------------------------------------------------
# Affine embedding
# ---------------------------------------------------------------------------


def agipc_affine_plan(ctx: Context, n_fine: int, labels, n_coarse_dev, threshold: int, coarse_base, coarse_k,
                      n_rows_dev):
    _check(load().agipc_affine_plan(ctx.handle, int(n_fine), _ptr(labels), _ptr(n_coarse_dev), int(threshold),
                                    _ptr(coarse_base), _ptr(coarse_k), _ptr(n_rows_dev)), "agipc_affine_plan")


def agipc_assemble_affine(ctx: Context, n_fine: int, labels, n_coarse_dev, X_rest, coarse_base, coarse_k, n_rows_dev,
                          label_row_ptr, label_col, fine_row_ptr, fine_col, fine_val, pair_idx, pair_blk, g, row_ptr,
                          col, val, nnzb_dev, g_c, dinv):
    _check(load().agipc_assemble_affine(
        ctx.handle, int(n_fine), _ptr(labels), _ptr(n_coarse_dev), _ptr(X_rest), _ptr(coarse_base), _ptr(coarse_k),
        _ptr(n_rows_dev), _ptr(label_row_ptr), _ptr(label_col), _ptr(fine_row_ptr), _ptr(fine_col), _ptr(fine_val),
        int(fine_col.shape[0]), int(pair_idx.shape[0]), _ptr(pair_idx), _ptr(pair_blk), _ptr(g), _ptr(row_ptr),
        _ptr(col), _ptr(val), int(col.shape[0]), _ptr(nnzb_dev), _ptr(g_c), _ptr(dinv)), "agipc_assemble_affine")


def agipc_prolongate_affine(ctx: Context, n_fine: int, labels, n_coarse_dev, X_rest, coarse_base, coarse_k, y, dx):
    _check(load().agipc_prolongate_affine(ctx.handle, int(n_fine), _ptr(labels), _ptr(n_coarse_dev), _ptr(X_rest),
                                          _ptr(coarse_base), _ptr(coarse_k), _ptr(y), _ptr(dx)),
           "agipc_prolongate_affine")


class AffineStep(CoarsenedStep):
    """The coarsened step with affine embedding of aggregates larger than
    `threshold` fine nodes: labels -> label-level assembly (structure) ->
    plan -> expanded Galerkin assembly -> PCG -> dx = P y."""

    def __init__(self, ctx: Context, ds: DeviceScene, X_rest, tol: float, threshold: int = 32,
                 max_iter: int = 100000):
        super().__init__(ctx, ds, tol, max_iter)
        dev = ds.g.device
        n = ds.n
        self.threshold = threshold
        self.X_rest = torch.as_tensor(np.ascontiguousarray(X_rest), dtype=torch.float64, device=dev)
        self.coarse_base = torch.zeros(n, dtype=torch.int32, device=dev)
        self.coarse_k = torch.zeros(n, dtype=torch.int32, device=dev)
        self.n_rows = torch.zeros(1, dtype=torch.int32, device=dev)
        cap = 16 * ds.capacity
        self.a_row_ptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
        self.a_col = torch.empty(cap, dtype=torch.int32, device=dev)
        self.a_val = torch.empty(cap, 9, dtype=torch.float64, device=dev)
        self.a_nnz = torch.zeros(1, dtype=torch.int32, device=dev)
        self.a_gc = torch.empty(n, 3, dtype=torch.float64, device=dev)
        self.a_dinv = torch.empty(n, 9, dtype=torch.float64, device=dev)

    def assemble(self):
        super().assemble()
        ds, ctx = self.ds, self.ctx
        agipc_affine_plan(ctx, ds.n, self.labels, self.n_c, self.threshold, self.coarse_base, self.coarse_k,
                          self.n_rows)
        agipc_assemble_affine(ctx, ds.n, self.labels, self.n_c, self.X_rest, self.coarse_base, self.coarse_k,
                              self.n_rows, self.row_ptr, self.col, ds.row_ptr, ds.col, ds.val, ds.pair_idx,
                              ds.pair_blk, ds.g, self.a_row_ptr, self.a_col, self.a_val, self.a_nnz, self.a_gc,
                              self.a_dinv)

    def solve(self):
        agipc_pcg(self.ctx, self.ds.n, self.n_rows, self.a_row_ptr, self.a_col, self.a_val, self.a_dinv, self.a_gc,
                  self.y, self.tol, self.max_iter, -1, self.iters, self.relres)

    def prolongate(self):
        agipc_prolongate_affine(self.ctx, self.ds.n, self.labels, self.n_c, self.X_rest, self.coarse_base,
                                self.coarse_k, self.y, self.dx)

    def host(self):
        nr = int(self.n_rows.item())
        nnz = int(self.a_nnz.item())
        out = super().host()
        out.update(n_rows=nr, a_row_ptr=self.a_row_ptr[:nr + 1].cpu().numpy(), a_col=self.a_col[:nnz].cpu().numpy(),
                   a_val=self.a_val[:nnz].cpu().numpy().reshape(-1, 3, 3), a_gc=self.a_gc[:nr].cpu().numpy(),
                   y=self.y[:nr].cpu().numpy(), coarse_base=self.coarse_base[:out["n_c"]].cpu().numpy(),
                   coarse_k=self.coarse_k[:out["n_c"]].cpu().numpy())
        return out
