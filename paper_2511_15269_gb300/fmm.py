"""Python binding of the GB300 FMM library (C ABI in include/fmm.h).

Argument marshalling only: every stage of the evaluation runs in the CUDA
kernels of libfmm_gb300.so.  Tensors are torch CUDA tensors (float64,
contiguous); work is enqueued on torch's current CUDA stream.  If the library
has not been built, loading fails with an error (there is no other path).
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libfmm_gb300.so")
_lib = None

FMM_OK, FMM_ERR_INVALID_ARG, FMM_ERR_CUDA, FMM_ERR_OOM, FMM_ERR_CAPACITY, FMM_ERR_TIMEOUT = range(6)
FMM_FP64, FMM_FP32C, FMM_FP64DF = 0, 1, 2
FMM_TIE_TARGET = 1
FMM_SAME_LEVEL = 2
FMM_POS_SOA = 4
FMM_OPT_SCHEDULE, FMM_OPT_M2M_ONE_LAUNCH, FMM_OPT_NEAR_SYMMETRIC, FMM_OPT_M2L_BLOCKS_PER_SM = 1, 2, 3, 4
FMM_MAX_P = 10

# exported entry points, in include/fmm.h order
ENTRY_POINTS = ["fmm_device_peaks", "fmm_last_error", "fmm_set_device_memory_limit", "fmm_device_memory_in_use",
                "fmm_set_pool_retention",
                "fmm_num_levels", "fmm_build_tree", "fmm_build_tree2", "fmm_tree_free",
                "fmm_tree_merge",
                "fmm_tree_point_offsets",
                "fmm_tree_set_precision", "fmm_tree_stats", "fmm_tree_status", "fmm_tree_set_option", "fmm_tree_set_wait_limit",
                "fmm_tree_export",
                "fmm_tree_profile", "fmm_tree_stage_times", "fmm_eval_potential", "fmm_eval_field",
                "fmm_eval_batched", "fmm_tree_workspace_bytes", "fmm_tree_set_workspace",
                "fmm_eval_potential_host", "fmm_eval_potential_static", "fmm_backward"]
STAGES = ["sort", "p2p", "p2m", "m2m", "m2l", "l2l", "l2p"]


class FmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("FMM error %d: %s" % (code, msg))
        self.code = code


class fmm_params(C.Structure):
    _fields_ = [("p", C.c_int), ("leaf_size", C.c_int), ("splits", C.c_int), ("theta", C.c_double),
                ("precision", C.c_int), ("flags", C.c_int)]


class fmm_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int), ("p", C.c_int), ("splits", C.c_int),
                ("leaf_size", C.c_int), ("precision", C.c_int), ("theta", C.c_double),
                ("n_boxes", C.c_int64), ("n_leaves", C.c_int64), ("n_m2l", C.c_int64),
                ("n_p2p", C.c_int64), ("n_p2p_pairs", C.c_int64), ("device_bytes", C.c_size_t),
                ("build_ms", C.c_double), ("kernel_launches", C.c_int64), ("n_trees", C.c_int),
                ("levels_src", C.c_int), ("n_sources", C.c_int64), ("n_targets", C.c_int64),
                ("n_src_leaves", C.c_int64)]


def library_path():
    return _LIB_PATH


def lib():
    """Loads libfmm_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libfmm_gb300.so not found at %s; build it with "
                              "paper_2511_15269_gb300.build.build()" % _LIB_PATH)
        L = C.CDLL(_LIB_PATH)
        vp, i64, i = C.c_void_p, C.c_int64, C.c_int
        L.fmm_last_error.restype = C.c_char_p
        L.fmm_device_peaks.argtypes = [vp, vp]
        L.fmm_set_device_memory_limit.argtypes = [C.c_size_t]
        L.fmm_device_memory_in_use.argtypes = [C.POINTER(C.c_size_t)]
        L.fmm_set_pool_retention.argtypes = [C.c_size_t]
        L.fmm_tree_set_wait_limit.argtypes = [vp, i64]
        L.fmm_tree_set_option.argtypes = [vp, i, i]
        L.fmm_num_levels.argtypes = [i64, i, i]
        L.fmm_num_levels.restype = i
        L.fmm_build_tree.argtypes = [vp, i64, C.POINTER(fmm_params), vp, C.POINTER(vp)]
        L.fmm_build_tree2.argtypes = [vp, i64, vp, i64, C.POINTER(fmm_params), vp, C.POINTER(vp)]
        L.fmm_tree_free.argtypes = [vp]
        L.fmm_tree_merge.argtypes = [vp, i, vp, C.POINTER(vp)]
        L.fmm_tree_point_offsets.argtypes = [vp, vp]
        L.fmm_tree_free.restype = None
        L.fmm_tree_set_precision.argtypes = [vp, i]
        L.fmm_tree_stats.argtypes = [vp, C.POINTER(fmm_stats)]
        L.fmm_tree_status.argtypes = [vp, vp]
        L.fmm_tree_export.argtypes = [vp] * 11
        L.fmm_tree_profile.argtypes = [vp, i]
        L.fmm_tree_stage_times.argtypes = [vp, vp, vp]
        L.fmm_eval_potential.argtypes = [vp, vp, vp, vp]
        L.fmm_eval_field.argtypes = [vp, vp, vp, vp, vp]
        L.fmm_eval_batched.argtypes = [vp, i, vp, vp, vp]
        L.fmm_tree_workspace_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.fmm_tree_set_workspace.argtypes = [vp, vp, C.c_size_t]
        L.fmm_eval_potential_host.argtypes = [vp, vp, vp, vp]
        L.fmm_eval_potential_static.argtypes = [vp, vp, vp, vp]
        L.fmm_backward.argtypes = [vp, vp, vp, vp, vp, vp]
        for f in ENTRY_POINTS:
            if f not in ("fmm_last_error", "fmm_num_levels", "fmm_tree_free"):
                getattr(L, f).restype = i
        _lib = L
    return _lib


def _check(rc):
    if rc != FMM_OK:
        raise FmmError(rc, lib().fmm_last_error().decode(errors="replace"))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, numel=None, what="tensor"):
    """Device pointer of a contiguous float64 tensor on the current CUDA
    device; `numel` (if given) is the number of doubles the library reads or
    writes through it, checked here because the kernels cannot."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s: expected a contiguous float64 CUDA tensor" % what)
    if t.device.index != torch.cuda.current_device():
        raise FmmError(FMM_ERR_INVALID_ARG, "%s is on cuda:%d, the current device is cuda:%d"
                       % (what, t.device.index, torch.cuda.current_device()))
    if numel is not None and t.numel() != numel:
        raise FmmError(FMM_ERR_INVALID_ARG, "%s has %d entries, the tree needs %d" % (what, t.numel(), numel))
    return C.c_void_p(t.data_ptr())


def fmm_device_peaks():
    """Measured FP32 / packed FP32x2 / FP64 FMA TFLOP/s and rsqrt Gop/s."""
    import numpy as np
    out = np.zeros(4)
    _check(lib().fmm_device_peaks(C.c_void_p(out.ctypes.data), _stream()))
    return {"fp32_fma_tflops": out[0], "fp32x2_fma_tflops": out[1], "fp64_fma_tflops": out[2],
            "rsqrt_gops": out[3]}


def fmm_last_error():
    return lib().fmm_last_error().decode(errors="replace")


def fmm_set_device_memory_limit(nbytes):
    """Caps the device memory the library holds (0: no cap)."""
    _check(lib().fmm_set_device_memory_limit(int(nbytes)))


def fmm_set_pool_retention(nbytes):
    """Unused device memory the library keeps for later builds (default 2 GiB)."""
    _check(lib().fmm_set_pool_retention(int(nbytes)))


def fmm_device_memory_in_use():
    v = C.c_size_t()
    _check(lib().fmm_device_memory_in_use(C.byref(v)))
    return v.value


def fmm_num_levels(n, leaf_size, splits=2):
    return lib().fmm_num_levels(int(n), int(leaf_size), int(splits))


class Tree:
    """Owner of an fmm_tree* built by fmm_build_tree / fmm_build_tree2.
    n_charges: length of q; n_out: length of u (both n for one point set)."""

    def __init__(self, handle, n, params, n_charges=None, n_out=None):
        self._h = handle
        self.n = n
        self.params = params
        self.n_charges = n if n_charges is None else n_charges
        self.n_out = n if n_out is None else n_out
        self.two_trees = n_charges is not None
        self._workspace = None  # a caller workspace attached with fmm_tree_set_workspace

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            lib().fmm_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self):
        return fmm_tree_stats(self)

    def set_precision(self, precision):
        fmm_tree_set_precision(self, precision)


def fmm_build_tree(pos, p, leaf_size, splits=2, theta=0.5, precision=FMM_FP32C, flags=0):
    """Builds the hierarchy of `pos` on the device: an N x 3 float64 CUDA
    tensor, or 3 x N with FMM_POS_SOA in flags."""
    pos = pos.contiguous()
    n = pos.shape[1] if flags & FMM_POS_SOA else pos.shape[0]
    prm = fmm_params(int(p), int(leaf_size), int(splits), float(theta), int(precision), int(flags))
    h = C.c_void_p()
    _check(lib().fmm_build_tree(_dev(pos, 3 * n, "pos"), n, C.byref(prm), _stream(), C.byref(h)))
    return Tree(h, n, prm)


def fmm_build_tree2(src_pos, trg_pos, p, leaf_size, splits=2, theta=0.5, precision=FMM_FP32C, flags=0):
    """Separate source and target hierarchies: evaluations take charges at
    src_pos (N_s x 3) and return potentials / fields at trg_pos (N_t x 3)."""
    src_pos, trg_pos = src_pos.contiguous(), trg_pos.contiguous()
    ns, nt = (src_pos.shape[1], trg_pos.shape[1]) if flags & FMM_POS_SOA else (src_pos.shape[0], trg_pos.shape[0])
    prm = fmm_params(int(p), int(leaf_size), int(splits), float(theta), int(precision), int(flags))
    h = C.c_void_p()
    _check(lib().fmm_build_tree2(_dev(src_pos, 3 * ns, "src_pos"), ns, _dev(trg_pos, 3 * nt, "trg_pos"), nt,
                                 C.byref(prm), _stream(), C.byref(h)))
    return Tree(h, ns + nt, prm, n_charges=ns, n_out=nt)


def fmm_tree_free(tree):
    tree.free()


def fmm_tree_merge(trees):
    """Batch of independent trees evaluated together (points concatenated in
    the given order); the inputs stay valid."""
    arr = (C.c_void_p * len(trees))(*[t.handle for t in trees])
    h = C.c_void_p()
    _check(lib().fmm_tree_merge(arr, len(trees), _stream(), C.byref(h)))
    n = sum(t.n for t in trees)
    return Tree(h, n, trees[0].params)


def fmm_tree_point_offsets(tree):
    import numpy as np
    st = fmm_tree_stats(tree)
    out = np.zeros(st["n_trees"] + 1, dtype=np.int64)
    _check(lib().fmm_tree_point_offsets(tree.handle, C.c_void_p(out.ctypes.data)))
    return out


def fmm_tree_set_precision(tree, precision):
    _check(lib().fmm_tree_set_precision(tree.handle, int(precision)))


def fmm_tree_stats(tree):
    s = fmm_stats()
    _check(lib().fmm_tree_stats(tree.handle, C.byref(s)))
    return {k: getattr(s, k) for k, _ in fmm_stats._fields_}


def fmm_tree_status(tree):
    _check(lib().fmm_tree_status(tree.handle, _stream()))


def fmm_tree_set_option(tree, option, value):
    """Launch option of later evaluations (FMM_OPT_*)."""
    _check(lib().fmm_tree_set_option(tree.handle, int(option), int(value)))


def fmm_tree_set_wait_limit(tree, cycles):
    """Cycle limit of the near-field kernels' bounded waits (0: give up at once)."""
    _check(lib().fmm_tree_set_wait_limit(tree.handle, int(cycles)))


def fmm_tree_export(tree):
    """Host copies of the hierarchy (numpy arrays)."""
    import numpy as np
    st = fmm_tree_stats(tree)
    nb, L = st["n_boxes"], st["levels"]
    n_avg = st["levels_src"] + L + 2 if tree.two_trees else L + 1
    out = dict(perm=np.zeros(st["n"], np.int32), box_start=np.zeros(nb, np.int64),
               box_count=np.zeros(nb, np.int64), center=np.zeros((nb, 3)), radius=np.zeros(nb),
               level_avg_radius=np.zeros(n_avg), m2l_trg=np.zeros(st["n_m2l"], np.int32),
               m2l_src=np.zeros(st["n_m2l"], np.int32), p2p_trg=np.zeros(st["n_p2p"], np.int32),
               p2p_src=np.zeros(st["n_p2p"], np.int32))
    keys = ["perm", "box_start", "box_count", "center", "radius", "level_avg_radius", "m2l_trg",
            "m2l_src", "p2p_trg", "p2p_src"]
    _check(lib().fmm_tree_export(tree.handle, *[C.c_void_p(out[k].ctypes.data) for k in keys]))
    return out


def fmm_tree_profile(tree, enable=True):
    _check(lib().fmm_tree_profile(tree.handle, int(bool(enable))))


def fmm_tree_stage_times(tree):
    """(dict stage -> summed ms, number of recorded calls)."""
    import numpy as np
    ms = np.zeros(len(STAGES))
    calls = C.c_int64()
    _check(lib().fmm_tree_stage_times(tree.handle, C.c_void_p(ms.ctypes.data), C.byref(calls)))
    return dict(zip(STAGES, ms.tolist())), calls.value


def fmm_eval_potential(tree, q, out=None):
    u = out if out is not None else torch.empty(tree.n_out, dtype=torch.float64, device=q.device)
    _check(lib().fmm_eval_potential(tree.handle, _dev(q, tree.n_charges, "q"), _dev(u, tree.n_out, "u"),
                                    _stream()))
    return u


def fmm_eval_field(tree, q, potential=True):
    f = torch.empty((tree.n_out, 3), dtype=torch.float64, device=q.device)
    u = torch.empty(tree.n_out, dtype=torch.float64, device=q.device) if potential else None
    _check(lib().fmm_eval_field(tree.handle, _dev(q, tree.n_charges, "q"),
                                _dev(u, tree.n_out, "u") if u is not None else None,
                                _dev(f, 3 * tree.n_out, "field"), _stream()))
    return (u, f) if potential else f


def fmm_eval_batched(batch, q_sets, u_sets=None):
    """Potentials of the batch's charge sets (one float64 CUDA tensor per
    set, in the order the trees were merged) in one evaluation."""
    offs = fmm_tree_point_offsets(batch)
    n = len(offs) - 1
    if len(q_sets) != n:
        raise FmmError(FMM_ERR_INVALID_ARG, "expected %d charge sets, got %d" % (n, len(q_sets)))
    if u_sets is None:
        u_sets = [torch.empty(int(offs[k + 1] - offs[k]), dtype=torch.float64, device=q_sets[k].device)
                  for k in range(n)]
    qp = (C.c_void_p * n)(*[_dev(q, int(offs[k + 1] - offs[k]), "q_sets[%d]" % k).value for k, q in enumerate(q_sets)])
    up = (C.c_void_p * n)(*[_dev(u, int(offs[k + 1] - offs[k]), "u_sets[%d]" % k).value for k, u in enumerate(u_sets)])
    _check(lib().fmm_eval_batched(batch.handle, n, qp, up, _stream()))
    return u_sets


def fmm_tree_workspace_bytes(tree):
    v = C.c_size_t()
    _check(lib().fmm_tree_workspace_bytes(tree.handle, C.byref(v)))
    return v.value


def fmm_tree_set_workspace(tree, workspace):
    """Evaluations of `tree` use `workspace` (a CUDA tensor of at least
    fmm_tree_workspace_bytes bytes, kept alive by the caller; the tree holds a
    reference) for their scratch; None gives the tree its own again."""
    if workspace is None:
        _check(lib().fmm_tree_set_workspace(tree.handle, None, 0))
        tree._workspace = None
        return
    if not (isinstance(workspace, torch.Tensor) and workspace.is_cuda and workspace.is_contiguous()):
        raise TypeError("workspace: expected a contiguous CUDA tensor")
    _check(lib().fmm_tree_set_workspace(tree.handle, C.c_void_p(workspace.data_ptr()),
                                        workspace.numel() * workspace.element_size()))
    tree._workspace = workspace


def fmm_eval_potential_host(tree, q_host, u_host=None):
    """Host-buffer evaluation: q_host, u_host are float64 CPU tensors (pinned is fastest)."""
    if u_host is None:
        u_host = torch.empty(tree.n_out, dtype=torch.float64, pin_memory=True)
    for t, n, what in ((q_host, tree.n_charges, "q_host"), (u_host, tree.n_out, "u_host")):
        if t.dtype != torch.float64 or t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise FmmError(FMM_ERR_INVALID_ARG, "%s: expected %d contiguous float64 host values" % (what, n))
    _check(lib().fmm_eval_potential_host(tree.handle, C.c_void_p(q_host.data_ptr()),
                                         C.c_void_p(u_host.data_ptr()), _stream()))
    return u_host


def fmm_eval_potential_static(tree, q, out=None):
    """fmm_eval_potential without device allocation in the library: the
    per-call scratch is the library's static device array (see fmm.h).
    `out` lets the caller pass a preallocated output."""
    u = out if out is not None else torch.empty(tree.n, dtype=torch.float64, device=q.device)
    _check(lib().fmm_eval_potential_static(tree.handle, _dev(q, tree.n, "q"), _dev(u, tree.n, "u"), _stream()))
    return u


def fmm_backward(tree, q, grad_u, need_q=True, need_pos=True):
    gq = torch.empty(tree.n, dtype=torch.float64, device=q.device) if need_q else None
    gp = torch.empty((tree.n, 3), dtype=torch.float64, device=q.device) if need_pos else None
    _check(lib().fmm_backward(tree.handle, _dev(q, tree.n, "q"), _dev(grad_u.contiguous(), tree.n, "grad_u"),
                              _dev(gq, tree.n, "grad_q") if gq is not None else None,
                              _dev(gp, 3 * tree.n, "grad_pos") if gp is not None else None, _stream()))
    return gq, gp


class FMMPotential(torch.autograd.Function):
    """u = FMM potential of charges q at the tree's points (Eq. 1-3).

    Gradients: dL/dq = K dL/du (fmm_backward) and dL/dpos from the fields of q
    and of dL/du, at the fixed hierarchy of the tree."""

    @staticmethod
    def forward(ctx, pos, q, tree):
        ctx.tree = tree
        ctx.save_for_backward(q)
        return fmm_eval_potential(tree, q.contiguous())

    @staticmethod
    def backward(ctx, grad_u):
        (q,) = ctx.saved_tensors
        need_pos, need_q = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gq, gp = fmm_backward(ctx.tree, q.contiguous(), grad_u.contiguous(), need_q=need_q,
                              need_pos=need_pos)
        return gp, gq, None


class FMMPotential2(torch.autograd.Function):
    """u = FMM potential at the targets of charges q at the sources of a
    source/target tree pair built by fmm_build_tree2.

    dL/dq = K^T dL/du is the potential at the sources of charges dL/du at the
    targets, evaluated with the reverse tree (sources and targets swapped), to
    FMM accuracy.  Position gradients are not offered for separate trees."""

    @staticmethod
    def forward(ctx, q, tree, tree_rev):
        ctx.tree_rev = tree_rev
        return fmm_eval_potential(tree, q.contiguous())

    @staticmethod
    def backward(ctx, grad_u):
        gq = fmm_eval_potential(ctx.tree_rev, grad_u.contiguous()) if ctx.needs_input_grad[0] else None
        return gq, None, None
