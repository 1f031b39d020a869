"""Python binding of the KIFMM C ABI (include/kifmm.h).

Argument marshalling only: every step of the method runs in the CUDA library
(lib/libkifmm.so).  PyTorch provides device memory and the current stream.
There is no fallback: if the library is missing or a call fails, an
exception is raised.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libkifmm.so")

OK, ERR_ARG, ERR_CAPACITY, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = range(7)
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed_fp16": 3}
KERNELS = {"laplace": 0, "stokeslet": 1}
LIST_KINDS = {"U": 0, "V": 1, "W": 2, "X": 3}


class KifmmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


class PlanDesc(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("leaf_cap", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("precision", ctypes.c_int), ("coef", ctypes.c_double), ("n_max", ctypes.c_int64),
                ("n_systems_max", ctypes.c_int), ("dtype", ctypes.c_int), ("pinv_eps", ctypes.c_double),
                ("autotune", ctypes.c_int), ("direct_max", ctypes.c_int), ("m2l_eps", ctypes.c_double),
                ("cell", ctypes.c_double), ("kernel", ctypes.c_int), ("reuse_lists", ctypes.c_int)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_boxes", ctypes.c_int64), ("max_level", ctypes.c_int),
                ("n_systems", ctypes.c_int), ("n_u", ctypes.c_int64), ("n_v", ctypes.c_int64),
                ("n_w", ctypes.c_int64), ("n_x", ctypes.c_int64), ("sort_passes", ctypes.c_int),
                ("lists_reused", ctypes.c_int)]


STAGES = ["tree", "p2m", "m2m", "m2l", "p2l", "l2l", "leaf", "p2p", "out"]


class ProfileT(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(STAGES)), ("calls", ctypes.c_int64 * len(STAGES)),
                ("launches", ctypes.c_int64)]


class TuningT(ctypes.Structure):
    _fields_ = [("tuned", ctypes.c_int), ("m2l_stages", ctypes.c_int), ("leaf_tpl", ctypes.c_int * 16),
                ("leaf_groups", ctypes.c_int * 16), ("m2l_rank_out", ctypes.c_int), ("m2l_rank_in", ctypes.c_int),
                ("m2l_producers", ctypes.c_int), ("m2l_tiles", ctypes.c_int)]


_LIB = None
EXPORTS = ["kifmm_plan_create", "kifmm_plan_destroy", "kifmm_set_sources", "kifmm_evaluate",
           "kifmm_clump_reduce", "kifmm_backward", "kifmm_get_device_status", "kifmm_status_string",
           "kifmm_tree_info", "kifmm_copy_keys", "kifmm_copy_tree", "kifmm_copy_list",
           "kifmm_profile_enable", "kifmm_profile_read", "kifmm_copy_expansions", "kifmm_update_sources",
           "kifmm_get_tuning", "kifmm_energy_noalloc", "kifmm_refresh_sources", "kifmm_lr_stride", "kifmm_far_image_operator",
           "kifmm_copy_list_images", "kifmm_set_m2l_tuning", "kifmm_set_m2l_wait_bound"]


def load(path: str = LIB_PATH):
    """Load the library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise FileNotFoundError(f"KIFMM library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.kifmm_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(P)]
    lib.kifmm_plan_destroy.argtypes = [P]
    lib.kifmm_set_sources.argtypes = [P, I, P, P, P, P]
    lib.kifmm_evaluate.argtypes = [P, P, P, P, P]
    lib.kifmm_clump_reduce.argtypes = [P, I64, P, P, P, P, P, P, P, P]
    lib.kifmm_backward.argtypes = [P, P, P, P, P, P, P, P]
    lib.kifmm_get_device_status.argtypes = [P, ctypes.POINTER(I)]
    lib.kifmm_status_string.argtypes = [I]
    lib.kifmm_status_string.restype = ctypes.c_char_p
    lib.kifmm_tree_info.argtypes = [P, ctypes.POINTER(TreeInfo)]
    lib.kifmm_copy_keys.argtypes = [P, P, P, P]
    lib.kifmm_copy_tree.argtypes = [P, P, P, P, P, P, P]
    lib.kifmm_copy_list.argtypes = [P, I, P, P]
    lib.kifmm_profile_enable.argtypes = [P, I]
    lib.kifmm_profile_read.argtypes = [P, ctypes.POINTER(ProfileT)]
    lib.kifmm_copy_expansions.argtypes = [P, P, P, P]
    lib.kifmm_update_sources.argtypes = [P, P, P, P]
    lib.kifmm_refresh_sources.argtypes = [P, P, P, D, ctypes.POINTER(I), P]
    lib.kifmm_lr_stride.argtypes = [D, D, ctypes.POINTER(I64)]
    lib.kifmm_far_image_operator.argtypes = [I, D, P]
    lib.kifmm_set_m2l_tuning.argtypes = [P, I, I, I]
    lib.kifmm_set_m2l_wait_bound.argtypes = [P, I64]
    lib.kifmm_copy_list_images.argtypes = [P, I, P, P, P]
    for name in EXPORTS:
        getattr(lib, name).restype = ctypes.c_int if name != "kifmm_status_string" else ctypes.c_char_p
    _LIB = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().kifmm_status_string(code).decode()
    except Exception:
        return "unknown"


def _check(code: int, what: str):
    if code != OK:
        raise KifmmError(code, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """One precomputed KIFMM configuration (operators + workspace) on the
    current CUDA device."""

    def __init__(self, p: int = 6, leaf_cap: int = 128, max_depth: int = 20, precision: str = "fp32",
                 coef: float = 1.0, n_max: int = 1 << 20, n_systems_max: int = 1,
                 dtype: torch.dtype = torch.float32, pinv_eps: float = 0.0, autotune: bool = False,
                 direct_max: int = 0, m2l_eps: float = 0.0, cell: float = 0.0, kernel: str = "laplace",
                 reuse_lists: bool = False):
        lib = load()
        self.dtype = dtype
        self.precision = precision
        self.coef = coef
        d = PlanDesc(p=p, leaf_cap=leaf_cap, max_depth=max_depth, precision=PRECISIONS[precision], coef=coef,
                     n_max=n_max, n_systems_max=n_systems_max,
                     dtype=1 if dtype == torch.float64 else 0, pinv_eps=pinv_eps, autotune=int(autotune), direct_max=direct_max,
                     m2l_eps=m2l_eps, cell=cell, kernel=KERNELS[kernel], reuse_lists=int(reuse_lists))
        h = ctypes.c_void_p()
        _check(lib.kifmm_plan_create(ctypes.byref(d), ctypes.byref(h)), "kifmm_plan_create")
        self._h = h
        self.kernel = kernel
        self._ns = (6 * (p - 1) ** 2 + 2) * (3 if kernel == "stokeslet" else 1)  # expansion length
        self.n = 0
        self.n_systems = 0
        self._offsets = None
        # bumped whenever the plan's sources change: an autograd backward
        # checks that the plan still holds the sources of its forward
        self.generation = 0

    def close(self):
        if getattr(self, "_h", None):
            load().kifmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_sources(self, xyz: torch.Tensor, q: torch.Tensor, sys_offsets=None, stream=None):
        assert xyz.is_cuda and q.is_cuda and xyz.dtype == self.dtype and q.dtype == self.dtype
        xyz = xyz.contiguous()
        q = q.contiguous()
        n = xyz.shape[0]
        if sys_offsets is None:
            sys_offsets = [0, n]
        off = np.ascontiguousarray(np.asarray(sys_offsets, dtype=np.int64))
        _check(load().kifmm_set_sources(self._h, len(off) - 1, off.ctypes.data_as(ctypes.c_void_p),
                                        _ptr(xyz), _ptr(q), _stream(stream)), "kifmm_set_sources")
        self.n = n
        self.n_systems = len(off) - 1
        self._offsets = off
        self.generation += 1

    def update_sources(self, xyz: torch.Tensor, q: torch.Tensor, stream=None):
        """New positions/charges for the same particles, tree and lists frozen.
        Asynchronous on `stream`: a contiguous copy made here is recorded on
        that stream, so the allocator does not reuse it before the copy in is
        done."""
        assert xyz.is_cuda and q.is_cuda and xyz.dtype == self.dtype and q.dtype == self.dtype
        assert self.n == 0 or xyz.shape[0] == self.n  # n == 0: the library reports the state error
        xc, qc = xyz.contiguous(), q.contiguous()
        if stream is not None:
            for t, src in ((xc, xyz), (qc, q)):
                if t.data_ptr() != src.data_ptr():
                    t.record_stream(stream)
        _check(load().kifmm_update_sources(self._h, _ptr(xc), _ptr(qc), _stream(stream)), "kifmm_update_sources")
        self.generation += 1

    def refresh_sources(self, xyz: torch.Tensor, q: torch.Tensor, skin: float = 0.05, stream=None) -> bool:
        """update_sources if every particle is still within its leaf (grown by
        `skin` finest-level half-widths), else a full rebuild with the same
        systems.  Returns True if the tree was kept.  Synchronises."""
        assert xyz.is_cuda and q.is_cuda and xyz.dtype == self.dtype and q.dtype == self.dtype
        assert self.n == 0 or xyz.shape[0] == self.n  # n == 0: the library reports the state error
        reused = ctypes.c_int(0)
        _check(load().kifmm_refresh_sources(self._h, _ptr(xyz.contiguous()), _ptr(q.contiguous()), float(skin),
                                            ctypes.byref(reused), _stream(stream)), "kifmm_refresh_sources")
        self.generation += 1
        return bool(reused.value)

    def evaluate(self, pot=None, grad=None, energy=None, want_pot=True, want_grad=True, want_energy=False,
                 stream=None):
        """(pot [N], grad [N, 3], energy [n_systems] float64), None where not
        wanted.  A Stokeslet plan returns (velocity [N, 3], None, None)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if self.kernel == "stokeslet":
            if pot is None:
                pot = torch.empty(self.n, 3, dtype=self.dtype, device=dev)
            # grad / energy, if given, are refused by the library
            _check(load().kifmm_evaluate(self._h, _ptr(pot), _ptr(grad), _ptr(energy), _stream(stream)),
                   "kifmm_evaluate")
            return pot, None, None
        if pot is None and want_pot:
            pot = torch.empty(self.n, dtype=self.dtype, device=dev)
        if grad is None and want_grad:
            grad = torch.empty(self.n, 3, dtype=self.dtype, device=dev)
        if energy is None and want_energy:
            energy = torch.empty(self.n_systems, dtype=torch.float64, device=dev)
        _check(load().kifmm_evaluate(self._h, _ptr(pot), _ptr(grad), _ptr(energy), _stream(stream)),
               "kifmm_evaluate")
        return pot, grad, energy

    def clump_reduce(self, clump_offsets: torch.Tensor, xyz, q, grad, ref, force=None, torque=None, stream=None):
        nc = clump_offsets.shape[0] - 1
        if force is None:
            force = torch.empty(nc, 3, dtype=self.dtype, device=xyz.device)
        if torque is None:
            torque = torch.empty(nc, 3, dtype=self.dtype, device=xyz.device)
        _check(load().kifmm_clump_reduce(self._h, nc, _ptr(clump_offsets), _ptr(xyz), _ptr(q), _ptr(grad),
                                         _ptr(ref), _ptr(force), _ptr(torque), _stream(stream)),
               "kifmm_clump_reduce")
        return force, torque

    def backward(self, dL_dpot=None, grad=None, dq=None, dx=None, stream=None, dL_dgrad=None, dL_denergy=None):
        """Adjoint of evaluate on the plan's current tree and sources
        (kifmm_backward): for a loss with dL/dpot, dL/dgrad (each [N] / [N, 3]
        in the plan's dtype, or None) and dL/dU per system ([n_systems]
        float64, or None), returns (dq, dx).  grad is the forward gradient,
        needed for dx with dL_dpot or dL_denergy; dL_dgrad and dL_denergy read
        the last evaluate, which must have run on the current sources."""
        lib = load()
        c = lambda t: None if t is None else t.contiguous()
        dL_dpot, grad, dL_dgrad = c(dL_dpot), c(grad), c(dL_dgrad)
        if dL_denergy is not None:
            dL_denergy = dL_denergy.to(torch.float64).contiguous()
        for t in (dL_dpot, dL_dgrad, grad):
            assert t is None or (t.dtype == self.dtype and t.is_cuda)
        dev = torch.device("cuda", torch.cuda.current_device())
        if dq is None:
            dq = torch.empty(self.n, dtype=self.dtype, device=dev)
        if dx is None:
            dx = torch.empty(self.n, 3, dtype=self.dtype, device=dev)
        _check(lib.kifmm_backward(self._h, _ptr(dL_dpot), _ptr(dL_dgrad), _ptr(dL_denergy), _ptr(grad), _ptr(dq),
                                  _ptr(dx), _stream(stream)), "kifmm_backward")
        return dq, dx

    def device_status(self) -> int:
        c = ctypes.c_int(0)
        _check(load().kifmm_get_device_status(self._h, ctypes.byref(c)), "kifmm_get_device_status")
        return c.value

    # ---- profiling ----
    def profile(self, enable: bool = True):
        _check(load().kifmm_profile_enable(self._h, int(enable)), "kifmm_profile_enable")

    def tuning(self) -> dict:
        """Tile shapes in use (see kifmm_get_tuning)."""
        t = TuningT()
        _check(load().kifmm_get_tuning(self._h, ctypes.byref(t)), "kifmm_get_tuning")
        return {"tuned_leaf": bool(t.tuned & 1), "tuned_m2l": bool(t.tuned & 2), "m2l_stages": t.m2l_stages,
                "leaf_tiles": [(t.leaf_tpl[i], t.leaf_groups[i]) for i in range(16)],
                "m2l_ranks": (t.m2l_rank_out, t.m2l_rank_in), "m2l_producers": t.m2l_producers,
                "m2l_tiles": t.m2l_tiles}

    def set_m2l_wait_bound(self, polls: int):
        """Bound of the tensor-core M2L's barrier waits (see kifmm_set_m2l_wait_bound)."""
        _check(load().kifmm_set_m2l_wait_bound(self._h, polls), "kifmm_set_m2l_wait_bound")

    def set_m2l_tuning(self, producers: int, tiles: int, stages: int):
        """Pin the tensor-core M2L variant (see kifmm_set_m2l_tuning)."""
        _check(load().kifmm_set_m2l_tuning(self._h, producers, tiles, stages), "kifmm_set_m2l_tuning")

    def profile_read(self) -> dict:
        """Per-stage device milliseconds and bracket counts since the last
        read, and the number of kernels the library launched."""
        t = ProfileT()
        _check(load().kifmm_profile_read(self._h, ctypes.byref(t)), "kifmm_profile_read")
        return {"ms": dict(zip(STAGES, list(t.ms))), "calls": dict(zip(STAGES, list(t.calls))),
                "launches": t.launches}

    # ---- introspection ----
    def tree_info(self) -> dict:
        t = TreeInfo()
        _check(load().kifmm_tree_info(self._h, ctypes.byref(t)), "kifmm_tree_info")
        return {f: getattr(t, f) for f, _ in TreeInfo._fields_}

    def keys(self):
        n = self.n
        keys = np.empty(n, dtype=np.uint64)
        perm = np.empty(n, dtype=np.int64)
        lo_side = np.empty((self.n_systems, 4))
        _check(load().kifmm_copy_keys(self._h, keys.ctypes.data_as(ctypes.c_void_p),
                                      perm.ctypes.data_as(ctypes.c_void_p),
                                      lo_side.ctypes.data_as(ctypes.c_void_p)), "kifmm_copy_keys")
        return keys, perm, lo_side

    def tree(self) -> dict:
        nb = self.tree_info()["n_boxes"]
        out = {k: np.empty(nb, dtype=np.int64) for k in ("sys", "level", "first", "count", "parent")}
        out["coord"] = np.empty((nb, 3), dtype=np.int64)
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().kifmm_copy_tree(self._h, c(out["sys"]), c(out["level"]), c(out["coord"]), c(out["first"]),
                                      c(out["count"]), c(out["parent"])), "kifmm_copy_tree")
        return out

    def expansions(self):
        """(u, d, res) after the last evaluate (see kifmm_copy_expansions)."""
        nb = self.tree_info()["n_boxes"]
        lib = load()
        ns = self._ns
        u = np.empty((nb, ns))
        d = np.empty((nb, ns))
        res = np.empty((self.n, 4))
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib.kifmm_copy_expansions(self._h, c(u), c(d), c(res)), "kifmm_copy_expansions")
        return u, d, res

    def list_images(self, kind: str):
        """(ptr, idx, img): one list kind as CSR with the image of every entry
        ((n_x + 1) 9 + (n_y + 1) 3 + (n_z + 1), 13 = the cell itself), sorted
        by (box, image) (see kifmm_copy_list_images)."""
        nb = self.tree_info()["n_boxes"]
        ptr = np.empty(nb + 1, dtype=np.int64)
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().kifmm_copy_list_images(self._h, LIST_KINDS[kind], c(ptr), None, None), "kifmm_copy_list_images")
        idx = np.empty(max(int(ptr[-1]), 1), dtype=np.int64)
        img = np.empty(max(int(ptr[-1]), 1), dtype=np.int64)
        _check(load().kifmm_copy_list_images(self._h, LIST_KINDS[kind], c(ptr), c(idx), c(img)),
               "kifmm_copy_list_images")
        return ptr, idx[:int(ptr[-1])], img[:int(ptr[-1])]

    def list(self, kind: str):
        info = self.tree_info()
        nb = info["n_boxes"]
        ptr = np.empty(nb + 1, dtype=np.int64)
        _check(load().kifmm_copy_list(self._h, LIST_KINDS[kind], ptr.ctypes.data_as(ctypes.c_void_p), None),
               "kifmm_copy_list")
        idx = np.empty(max(int(ptr[-1]), 1), dtype=np.int64)
        _check(load().kifmm_copy_list(self._h, LIST_KINDS[kind], ptr.ctypes.data_as(ctypes.c_void_p),
                                      idx.ctypes.data_as(ctypes.c_void_p)), "kifmm_copy_list")
        return ptr, idx[:int(ptr[-1])]


def lr_stride(k_dem: float, k_lr: float) -> int:
    """Long-range force computation stride S = max(1, floor(sqrt(k_dem / k_lr)))
    (Eq. 2): evaluate the long-range forces at least once every S DEM steps.
    Host only (no device needed)."""
    s = ctypes.c_int64(0)
    _check(load().kifmm_lr_stride(float(k_dem), float(k_lr), ctypes.byref(s)), "kifmm_lr_stride")
    return s.value


def far_image_operator(p: int, cell: float) -> np.ndarray:
    """[n_s, n_s] far-image operator of a periodic cell of side `cell`
    (see kifmm_far_image_operator).  Host only."""
    ns = 6 * (p - 1) ** 2 + 2
    T = np.empty((ns, ns), dtype=np.float64)
    _check(load().kifmm_far_image_operator(int(p), float(cell), T.ctypes.data_as(ctypes.c_void_p)),
           "kifmm_far_image_operator")
    return T


def energy_noalloc(q: torch.Tensor, pot: torch.Tensor, out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """U = 1/2 sum q pot through kifmm_energy_noalloc (the library allocates
    nothing; ``out`` is a float64 device tensor whose first element receives
    U, created here if not given).  q and pot: float32 or float64 (the same),
    on one CUDA device; the call runs with that device current."""
    lib = load()
    if not hasattr(lib, "_noalloc_typed"):
        lib.kifmm_energy_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]
        lib.kifmm_energy_noalloc.restype = ctypes.c_int
        lib._noalloc_typed = True
    if not (q.is_cuda and pot.is_cuda and q.device == pot.device):
        raise ValueError("q and pot must be CUDA tensors on one device")
    if q.dtype not in (torch.float32, torch.float64) or pot.dtype != q.dtype:
        raise TypeError("q and pot must both be float32 or both float64")
    if q.numel() != pot.numel():
        raise ValueError("q and pot differ in size")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=q.device)
    if out.dtype != torch.float64 or out.device != q.device or out.numel() < 1 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 tensor of at least one element on q's device")
    dt = 1 if q.dtype == torch.float64 else 0
    with torch.cuda.device(q.device):
        qc, pc = q.contiguous(), pot.contiguous()
        if stream is not None:
            # the temporaries (if any) are read on `stream`: keep them alive until it has
            qc.record_stream(stream)
            pc.record_stream(stream)
        _check(lib.kifmm_energy_noalloc(q.numel(), dt, _ptr(qc), _ptr(pc), _ptr(out), _stream(stream)),
               "kifmm_energy_noalloc")
    return out


def _check_generation(ctx):
    if ctx.plan.generation != ctx.generation:
        raise RuntimeError("the plan's sources changed after this forward: backward needs the plan to "
                           "hold the forward's sources (one plan per differentiated evaluation)")


class KifmmPotential(torch.autograd.Function):
    """(pot, grad) = KIFMM(x, q) with gradients w.r.t. x and q through the
    adjoint passes (kifmm_backward), for losses on the potential and on the
    gradient (forces F = -q grad).  The tree is built (rebuild=True) or
    frozen (rebuild=False, kifmm_update_sources); the plan must still hold
    these sources when backward runs (tree-level recomputation, nothing
    stored besides the forward gradient)."""

    @staticmethod
    def forward(ctx, x, q, plan, rebuild=True):
        if rebuild:
            plan.set_sources(x.detach(), q.detach())
        else:
            plan.update_sources(x.detach(), q.detach())
        pot, grad, _ = plan.evaluate()
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.save_for_backward(grad)
        return pot, grad

    @staticmethod
    def backward(ctx, g_pot, g_grad):
        (grad,) = ctx.saved_tensors
        _check_generation(ctx)
        if g_grad is not None and not torch.any(g_grad != 0):
            g_grad = None
        if g_pot is None and g_grad is None:
            return None, None, None, None
        dq, dx = ctx.plan.backward(g_pot, grad, dL_dgrad=g_grad)
        return dx, dq, None, None


class KifmmEnergy(torch.autograd.Function):
    """Long-range energy per system, U_s = 1/2 sum_{i in s} q_i pot_i (Sec.
    2.4), as the library's energy output; its gradients w.r.t. x and q come
    from kifmm_backward's energy term (no arithmetic here)."""

    @staticmethod
    def forward(ctx, x, q, plan, rebuild=True):
        if rebuild:
            plan.set_sources(x.detach(), q.detach())
        else:
            plan.update_sources(x.detach(), q.detach())
        _, grad, energy = plan.evaluate(want_pot=False, want_energy=True)
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.save_for_backward(grad)
        return energy

    @staticmethod
    def backward(ctx, g_energy):
        (grad,) = ctx.saved_tensors
        _check_generation(ctx)
        dq, dx = ctx.plan.backward(None, grad, dL_denergy=g_energy)
        return dx, dq, None, None


def potential(x, q, plan, rebuild=True):
    """Differentiable potential (Eq. 1 with the Eq. 3 kernel, coef applied)."""
    pot, _ = KifmmPotential.apply(x, q, plan, rebuild)
    return pot


def field(x, q, plan, rebuild=True):
    """Differentiable (pot, grad); a loss on grad (e.g. on the forces
    -q grad) is differentiated through the adjoint of the gradient."""
    return KifmmPotential.apply(x, q, plan, rebuild)


def energy(x, q, plan, rebuild=True):
    """Differentiable long-range energy, summed over the plan's systems
    (KifmmEnergy gives the per-system values)."""
    return KifmmEnergy.apply(x, q, plan, rebuild).sum()
