"""CPU FP64 oracle for the adaptive Laplace FMM of arXiv 2511.15269 (jaxFMM).

TEST INFRASTRUCTURE ONLY.  The oracle exists to check the CUDA path: only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  It shares no code with the CUDA library.

The C sources (``expansions.c``, ``tree.c``, ``fmm.c``) are compiled into
``liboracle.so`` by :func:`build` with ``-ffp-contract=off`` so that the FP64
expressions that decide the tree and the interaction lists are evaluated one
rounded operation at a time.  This module is a thin ctypes wrapper.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = ["expansions.c", "tree.c", "fmm.c"]
_lib = None


def build(force=False):
    """Compile the oracle shared library with gcc (OpenMP when available)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    hdr = os.path.join(_HERE, "fmm_oracle.h")
    if not force and os.path.exists(_SO):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(_SO) >= newest:
            return _SO
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", _SO + ".tmp"] + srcs + ["-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        d, i, i64, vp = C.c_double, C.c_int, C.c_int64, C.c_void_p
        L.orc_rhat.argtypes = [i, d, d, d, vp]
        L.orc_shat.argtypes = [i, d, d, d, vp]
        L.orc_grad_rhat.argtypes = [i, d, d, d, vp, vp]
        L.orc_wigner_d.argtypes = [i, d, vp]
        L.orc_rotate_azimuthal.argtypes = [i, i, d, vp, vp]
        L.orc_rotate_polar.argtypes = [i, i, d, vp, vp]
        for f in (L.orc_axial_m2m, L.orc_axial_m2l, L.orc_axial_l2l):
            f.argtypes = [i, d, vp, vp]
        L.orc_p2m.argtypes = [i, vp, vp, i64, vp, vp]
        L.orc_p2l.argtypes = [i, vp, vp, i64, vp, vp]
        for f in (L.orc_m2m, L.orc_m2l, L.orc_l2l):
            f.argtypes = [i, vp, vp, vp, vp]
        L.orc_l2p.argtypes = [i, vp, vp, vp, vp]
        L.orc_l2p.restype = d
        L.orc_m2p.argtypes = [i, vp, vp, vp]
        L.orc_m2p.restype = d
        L.orc_num_levels.argtypes = [i64, i, i]
        L.orc_num_levels.restype = i
        L.orc_tree_build.argtypes = [vp, i64, i, i, d, i]
        L.orc_tree_build.restype = vp
        L.orc_tree_free.argtypes = [vp]
        L.orc_tree_info.argtypes = [vp, vp]
        L.orc_tree_export.argtypes = [vp] + [vp] * 6
        L.orc_tree_export_lists.argtypes = [vp] * 5
        L.orc_fmm_eval.argtypes = [vp, i, vp, vp, i64, vp, vp]
        L.orc_fmm_eval_timed.argtypes = [vp, i, vp, vp, i64, vp, vp, vp]
        L.orc_set_num_threads.argtypes = [i]
        L.orc_direct.argtypes = [vp, vp, i64, vp, i64, vp, vp]
        L.orc_direct_vjp.argtypes = [vp, vp, vp, i64, vp, vp]
        L.orc_tree2_build.argtypes = [vp, i64, vp, i64, i, i, d, i]
        L.orc_tree2_build.restype = vp
        L.orc_tree2_free.argtypes = [vp]
        L.orc_tree2_source.argtypes = [vp]
        L.orc_tree2_source.restype = vp
        L.orc_tree2_target.argtypes = [vp]
        L.orc_tree2_target.restype = vp
        L.orc_tree2_info.argtypes = [vp, vp]
        L.orc_tree2_export_lists.argtypes = [vp] * 5
        L.orc_fmm2_eval.argtypes = [vp, i, vp, vp, vp]
        L.orc_direct2.argtypes = [vp, vp, i64, vp, i64, vp, vp]
        L.orc_num_threads.restype = i
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def ncoef(p):
    return (p + 1) * (p + 1)


def idx(n, m):
    """Storage index of real coefficient (n, m)."""
    return n * n + n + m


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """OpenMP threads of later oracle calls."""
    lib().orc_set_num_threads(int(n))


# ---- basis (App. A) ----
def rhat(p, v):
    out = np.zeros(ncoef(p))
    lib().orc_rhat(p, float(v[0]), float(v[1]), float(v[2]), _p(out))
    return out


def shat(p, v):
    out = np.zeros(ncoef(p))
    lib().orc_shat(p, float(v[0]), float(v[1]), float(v[2]), _p(out))
    return out


def grad_rhat(p, v):
    R = np.zeros(ncoef(p))
    G = np.zeros((ncoef(p), 3))
    lib().orc_grad_rhat(p, float(v[0]), float(v[1]), float(v[2]), _p(R), _p(G))
    return R, G


# ---- rotations and axial transforms (App. B) ----
def wigner_d(p, beta):
    """Array d[n, m + p, k + p] = d^n_{m,k}(beta)."""
    w = 2 * p + 1
    out = np.zeros((p + 1, w, w))
    lib().orc_wigner_d(p, float(beta), _p(out))
    return out


def rotate_azimuthal(p, coef, dphi, local=False):
    coef = _f64(coef)
    out = np.zeros_like(coef)
    lib().orc_rotate_azimuthal(p, int(local), float(dphi), _p(coef), _p(out))
    return out


def rotate_polar(p, coef, dtheta, local=False):
    coef = _f64(coef)
    out = np.zeros_like(coef)
    lib().orc_rotate_polar(p, int(local), float(dtheta), _p(coef), _p(out))
    return out


def axial(op, p, coef, r):
    coef = _f64(coef)
    out = np.zeros_like(coef)
    getattr(lib(), "orc_axial_" + op)(p, float(r), _p(coef), _p(out))
    return out


# ---- operators between centres ----
def p2m(p, pts, q, c):
    pts, q, c = _f64(pts), _f64(q), _f64(c)
    out = np.zeros(ncoef(p))
    lib().orc_p2m(p, _p(pts), _p(q), len(q), _p(c), _p(out))
    return out


def p2l(p, pts, q, c):
    pts, q, c = _f64(pts), _f64(q), _f64(c)
    out = np.zeros(ncoef(p))
    lib().orc_p2l(p, _p(pts), _p(q), len(q), _p(c), _p(out))
    return out


def _translate(name, p, coef, c_old, c_new):
    coef, a, b = _f64(coef), _f64(c_old), _f64(c_new)
    out = np.zeros(ncoef(p))
    getattr(lib(), name)(p, _p(coef), _p(a), _p(b), _p(out))
    return out


def m2m(p, C_, c_old, c_new):
    return _translate("orc_m2m", p, C_, c_old, c_new)


def m2l(p, C_, c_src, c_trg):
    return _translate("orc_m2l", p, C_, c_src, c_trg)


def l2l(p, D, c_old, c_new):
    return _translate("orc_l2l", p, D, c_old, c_new)


def l2p(p, D, c, x, grad=False):
    D, c, x = _f64(D), _f64(c), _f64(x)
    g = np.zeros(3)
    u = lib().orc_l2p(p, _p(D), _p(c), _p(x), _p(g))
    return (u, g) if grad else u


def m2p(p, C_, c, x):
    C_, c, x = _f64(C_), _f64(c), _f64(x)
    return lib().orc_m2p(p, _p(C_), _p(c), _p(x))


def num_levels(n, leaf_size, s=2):
    return lib().orc_num_levels(int(n), int(leaf_size), int(s))


class Tree:
    """Oracle hierarchy: median-split tree, geometry and interaction lists."""

    def __init__(self, pos, leaf_size, s=2, theta=0.5, tie_target=False, same_level=False):
        self.pos = _f64(pos).reshape(-1, 3)
        self.n = len(self.pos)
        self.leaf_size, self.s, self.theta = leaf_size, s, theta
        flags = (1 if tie_target else 0) | (2 if same_level else 0)
        h = lib().orc_tree_build(_p(self.pos), self.n, int(leaf_size), int(s), float(theta), flags)
        if not h:
            raise ValueError("oracle tree build rejected its arguments")
        self._h = h
        info = np.zeros(5, dtype=np.int64)
        lib().orc_tree_info(h, _p(info))
        self.L, self.n_boxes, self.n_m2l, self.n_p2p, self.n_leaves = (int(v) for v in info)
        self.perm = np.zeros(self.n, dtype=np.int32)
        self.box_start = np.zeros(self.n_boxes, dtype=np.int64)
        self.box_count = np.zeros(self.n_boxes, dtype=np.int64)
        self.center = np.zeros((self.n_boxes, 3))
        self.radius = np.zeros(self.n_boxes)
        self.level_avg_radius = np.zeros(self.L + 1)
        lib().orc_tree_export(h, _p(self.perm), _p(self.box_start), _p(self.box_count),
                              _p(self.center), _p(self.radius), _p(self.level_avg_radius))
        self.m2l_trg = np.zeros(self.n_m2l, dtype=np.int32)
        self.m2l_src = np.zeros(self.n_m2l, dtype=np.int32)
        self.p2p_trg = np.zeros(self.n_p2p, dtype=np.int32)
        self.p2p_src = np.zeros(self.n_p2p, dtype=np.int32)
        lib().orc_tree_export_lists(h, _p(self.m2l_trg), _p(self.m2l_src),
                                    _p(self.p2p_trg), _p(self.p2p_src))

    def level_offset(self, l):
        return sum(1 << (self.s * i) for i in range(l))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None

    def eval(self, q, p, targets=None, field=False):
        """FMM potential (and field = -grad u) at all points or at `targets`."""
        q = _f64(q)
        tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
        m = self.n if tg is None else len(tg)
        u = np.zeros(m)
        f = np.zeros((m, 3)) if field else None
        lib().orc_fmm_eval(self._h, int(p), _p(q), _p(tg), 0 if tg is None else m,
                           _p(u), _p(f))
        return (u, f) if field else u


    def eval_timed(self, q, p, targets):
        """Potential at `targets` plus the stage wall times (seconds) and the
        work of the stages restricted to the boxes feeding the targets:
        dict(sort, p2m, m2m, m2l, l2l, eval, n_m2l_done, n_l2l_done, n_eval)."""
        q = _f64(q)
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        u = np.zeros(len(tg))
        tm = np.zeros(9)
        lib().orc_fmm_eval_timed(self._h, int(p), _p(q), _p(tg), len(tg), _p(u), None, _p(tm))
        keys = ("sort", "p2m", "m2m", "m2l", "l2l", "eval", "n_m2l_done", "n_l2l_done", "n_eval")
        return u, dict(zip(keys, tm.tolist()))


class _Hierarchy:
    """Read-only view of one of the two hierarchies of a Tree2."""

    def __init__(self, h, n, s):
        info = np.zeros(5, dtype=np.int64)
        lib().orc_tree_info(h, _p(info))
        self.L, self.n_boxes, _, _, self.n_leaves = (int(v) for v in info)
        self.n, self.s = n, s
        self.perm = np.zeros(n, dtype=np.int32)
        self.box_start = np.zeros(self.n_boxes, dtype=np.int64)
        self.box_count = np.zeros(self.n_boxes, dtype=np.int64)
        self.center = np.zeros((self.n_boxes, 3))
        self.radius = np.zeros(self.n_boxes)
        self.level_avg_radius = np.zeros(self.L + 1)
        lib().orc_tree_export(h, _p(self.perm), _p(self.box_start), _p(self.box_count),
                              _p(self.center), _p(self.radius), _p(self.level_avg_radius))

    def level_offset(self, l):
        return sum(1 << (self.s * i) for i in range(l))


class Tree2:
    """Separate source and target hierarchies (Sec. II.B, final part) and the
    level-march lists between them.  M2L pairs use combined box ids (source
    boxes first, target box g at src.n_boxes + g); near-field pairs are
    (target leaf, source leaf)."""

    def __init__(self, src_pos, trg_pos, leaf_size, s=2, theta=0.5, tie_target=False):
        sp = _f64(src_pos).reshape(-1, 3)
        tp = _f64(trg_pos).reshape(-1, 3)
        self.src_pos, self.trg_pos = sp, tp
        self.leaf_size, self.s, self.theta = leaf_size, s, theta
        h = lib().orc_tree2_build(_p(sp), len(sp), _p(tp), len(tp), int(leaf_size), int(s),
                                  float(theta), 1 if tie_target else 0)
        if not h:
            raise ValueError("oracle tree build rejected its arguments")
        self._h = h
        self.src = _Hierarchy(lib().orc_tree2_source(h), len(sp), s)
        self.trg = _Hierarchy(lib().orc_tree2_target(h), len(tp), s)
        info = np.zeros(2, dtype=np.int64)
        lib().orc_tree2_info(h, _p(info))
        self.n_m2l, self.n_p2p = (int(v) for v in info)
        self.m2l_trg = np.zeros(self.n_m2l, dtype=np.int32)
        self.m2l_src = np.zeros(self.n_m2l, dtype=np.int32)
        self.p2p_trg = np.zeros(self.n_p2p, dtype=np.int32)
        self.p2p_src = np.zeros(self.n_p2p, dtype=np.int32)
        lib().orc_tree2_export_lists(h, _p(self.m2l_trg), _p(self.m2l_src),
                                     _p(self.p2p_trg), _p(self.p2p_src))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree2_free(h)
            self._h = None

    def eval(self, q, p, field=False):
        """FMM potential (and field) of charges q (source order) at the
        targets (target order)."""
        q = _f64(q)
        m = len(self.trg_pos)
        u = np.zeros(m)
        f = np.zeros((m, 3)) if field else None
        lib().orc_fmm2_eval(self._h, int(p), _p(q), _p(u), _p(f))
        return (u, f) if field else u


def direct2(src_pos, q, trg_pos, field=False):
    """Direct sum of Eq. 1-3 of charges q at src_pos, evaluated at trg_pos;
    zero distances contribute nothing."""
    sp, q, tp = _f64(src_pos).reshape(-1, 3), _f64(q), _f64(trg_pos).reshape(-1, 3)
    u = np.zeros(len(tp))
    f = np.zeros((len(tp), 3)) if field else None
    lib().orc_direct2(_p(sp), _p(q), len(q), _p(tp), len(tp), _p(u), _p(f))
    return (u, f) if field else u


def direct(pos, q, targets=None, field=False):
    """Direct sum of Eq. 1-3 at all points or at `targets` (original indices)."""
    pos, q = _f64(pos).reshape(-1, 3), _f64(q)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    m = len(q) if tg is None else len(tg)
    u = np.zeros(m)
    f = np.zeros((m, 3)) if field else None
    lib().orc_direct(_p(pos), _p(q), len(q), _p(tg), 0 if tg is None else m, _p(u), _p(f))
    return (u, f) if field else u


def direct_vjp(pos, q, g):
    """(dq, dpos) of <g, u(pos, q)> by the direct sum."""
    pos, q, g = _f64(pos).reshape(-1, 3), _f64(q), _f64(g)
    dq = np.zeros(len(q))
    dpos = np.zeros((len(q), 3))
    lib().orc_direct_vjp(_p(pos), _p(q), _p(g), len(q), _p(dq), _p(dpos))
    return dq, dpos


# ---- active shielding (Sec. III.B) ----
def _kernel_matrix(src_pos, trg_pos):
    """K[i, j]: potential at target i of a unit charge at source j (columns
    by the direct sum)."""
    sp = _f64(src_pos).reshape(-1, 3)
    K = np.zeros((len(_f64(trg_pos).reshape(-1, 3)), len(sp)))
    for j in range(len(sp)):
        e = np.zeros(len(sp))
        e[j] = 1.0
        K[:, j] = direct2(sp, e, trg_pos)
    return K


def shielding_loss(geo, q_sh, weights=(1.0, 0.2, 0.1)):
    """Loss of Sec. III.B with direct-sum potentials: (total, L_in, L_out, L_reg)."""
    src = np.concatenate([geo["ext"], geo["shield"]])
    q_all = np.concatenate([geo["q_ext"], q_sh])
    phi_in = direct2(src, q_all, geo["inside"])
    phi_out = direct2(geo["shield"], q_sh, geo["outside"])
    l_in = float(np.sum((phi_in - phi_in.mean()) ** 2))
    l_out = float(np.sum(phi_out ** 2))
    l_reg = float(np.sum(np.asarray(q_sh) ** 2))
    w_in, w_out, w_reg = weights
    return w_in * l_in + w_out * l_out + w_reg * l_reg, l_in, l_out, l_reg


def shielding_optimum(geo, weights=(1.0, 0.2, 0.1)):
    """Minimiser of the Sec. III.B loss, which is quadratic in the shield
    charges: with C the centring projector, A, B the direct-sum potential
    matrices of the shield at the inner and outer points and b the external
    potential at the inner points, the normal equations read
    (w_in A^T C A + w_out B^T B + w_reg I) q = -w_in A^T C b."""
    w_in, w_out, w_reg = weights
    A = _kernel_matrix(geo["shield"], geo["inside"])
    B = _kernel_matrix(geo["shield"], geo["outside"])
    b = direct2(geo["ext"], geo["q_ext"], geo["inside"])
    Ac = A - A.mean(axis=0, keepdims=True)
    bc = b - b.mean()
    H = w_in * Ac.T @ Ac + w_out * B.T @ B + w_reg * np.eye(A.shape[1])
    return np.linalg.solve(H, -w_in * Ac.T @ bc)
