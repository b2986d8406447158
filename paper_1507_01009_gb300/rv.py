"""Thin Python binding of librv (the C ABI in include/rv.h).

Only argument marshalling lives here: every step of the tree-gravity path
runs in librv's CUDA kernels. PyTorch provides device memory (the workspace
and the user's arrays) and streams. There is no CPU fallback: if librv.so is
missing or no GPU is present, loading fails with an error.

The ``rv_*`` functions mirror the C entry points one to one; ``Context`` and
``System`` are small conveniences over them.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build_lib

_LOCK = threading.Lock()
_LIB = None

RV_OK, RV_E_INVAL, RV_E_CUDA, RV_E_WORKSPACE, RV_E_STACK, RV_E_TIMEOUT, RV_E_NOTBUILT, RV_E_TOO_LARGE = range(8)
STATUS_NAMES = ["RV_OK", "RV_E_INVAL", "RV_E_CUDA", "RV_E_WORKSPACE", "RV_E_STACK", "RV_E_TIMEOUT", "RV_E_NOTBUILT",
                "RV_E_TOO_LARGE"]
EXPORTS = ["rv_default_config", "rv_workspace_size", "rv_create", "rv_destroy", "rv_set_workspace", "rv_build_tree",
           "rv_build_tree_members", "rv_tree_forces", "rv_tree_forces_rel", "rv_tree_forces_members",
           "rv_perturber_forces",
           "rv_system_forces", "rv_kdk_step", "rv_kdk_step_graph", "rv_energy",
           "rv_select_perturbers", "rv_select_perturbers_tidal", "rv_chain_perturber_forces", "rv_select_radius_static",
           "rv_block_start", "rv_block_steps", "rv_block_levels", "rv_block_count", "rv_chain_start_radius", "rv_get_tree", "rv_walk_stats", "rv_sync_status",
           "rv_profile_walk", "rv_walk_time", "rv_launch_count", "rv_last_error", "rv_mlp_param_bytes",
           "rv_mlp_scratch_bytes", "rv_mlp_init", "rv_mlp_forward", "rv_mlp_gradient", "rv_mlp_adam",
           "rv_mlp_samples", "rv_tree_forces_mlp", "rv_wait_selftest", "rv_mlp_fit_feature_box",
           "rv_mlp_set_feature_box", "rv_direct_fp64_scratch_bytes", "rv_direct_fp64", "rv_mlp_train_scratch_bytes",
           "rv_mlp_train", "rv_mlp_state_bytes", "rv_mlp_save", "rv_mlp_load", "rv_chain_absorb", "rv_chain_escape"]


class RvError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class rv_config(C.Structure):
    _fields_ = [("theta", C.c_float), ("eps_star", C.c_float), ("n_leaf", C.c_int32), ("group", C.c_int32),
                ("quadrupole", C.c_int32), ("tile", C.c_int32), ("mac", C.c_int32), ("alpha", C.c_float),
                ("softening", C.c_int32)]


class rv_blocks(C.Structure):
    _fields_ = [("dt_max", C.c_double), ("max_level", C.c_int32), ("tau_acc", C.c_float), ("tau_vel", C.c_float),
                ("eps", C.c_float), ("adapt", C.c_int32), ("level", C.c_void_p), ("substep", C.c_int64)]


class rv_tree_view(C.Structure):
    _fields_ = [("n", C.c_int64), ("ncell", C.c_int64), ("ngroup", C.c_int64), ("keys", C.c_void_p),
                ("perm", C.c_void_p), ("pos", C.c_void_p), ("cbox", C.c_void_p), ("clink", C.c_void_p),
                ("cmom", C.c_void_p), ("cparent", C.c_void_p), ("groups", C.c_void_p), ("bounds", C.c_void_p)]


class rv_mlp_train_cfg(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("t", C.c_void_p), ("steps", C.c_int32), ("batch", C.c_int32),
                ("step0", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("adam_eps", C.c_float), ("seed", C.c_uint64), ("fit_box", C.c_int32)]


class rv_chain_escape_result(C.Structure):
    _fields_ = [("escape_count", C.c_int32), ("terminate", C.c_int32), ("designated", C.c_int32),
                ("r_chain", C.c_double), ("r_escape", C.c_double)]


class rv_system(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("vx", C.c_void_p),
                ("vy", C.c_void_p), ("vz", C.c_void_p), ("m", C.c_void_p), ("ax", C.c_void_p), ("ay", C.c_void_p),
                ("az", C.c_void_p), ("pot", C.c_void_p), ("n_chain", C.c_int32), ("chain_m", C.c_void_p),
                ("chain_x", C.c_void_p), ("chain_v", C.c_void_p), ("chain_a", C.c_void_p),
                ("chain_pot", C.c_void_p), ("pert_mode", C.c_int32), ("pert_radius", C.c_float),
                ("pert_k", C.c_int32), ("n_members", C.c_int32), ("member_offsets", C.c_void_p),
                ("pert_gamma", C.c_float), ("n_chains", C.c_int32), ("chain_quad", C.c_int32)]


def lib_path() -> str:
    return build_lib.LIB


def load(build_if_missing: bool = True):
    """Load librv.so (building it first if asked). Raises if it cannot."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = build_lib.LIB
            if build_if_missing and build_lib.stale():
                build_lib.build()
            if not os.path.exists(path):
                raise RuntimeError(f"librv.so not found at {path}; run __graft_entry__.build()")
            L = C.CDLL(path)
            _declare(L)
            _LIB = L
    return _LIB


def _declare(L):
    vp, i64, i32, f32, f64 = C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_double
    L.rv_default_config.argtypes = [C.POINTER(rv_config)]
    L.rv_default_config.restype = None
    L.rv_workspace_size.argtypes = [i64, C.POINTER(rv_config)]
    L.rv_workspace_size.restype = C.c_size_t
    L.rv_create.argtypes = [C.POINTER(vp), i64, C.POINTER(rv_config)]
    L.rv_destroy.argtypes = [vp]
    L.rv_destroy.restype = None
    L.rv_set_workspace.argtypes = [vp, vp, C.c_size_t]
    L.rv_build_tree.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.rv_build_tree_members.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
    L.rv_tree_forces.argtypes = [vp, f32, f32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rv_tree_forces_rel.argtypes = [vp, f32, f32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rv_tree_forces_members.argtypes = [vp, f32, f32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rv_kdk_step_graph.argtypes = [vp, C.POINTER(rv_system), f64, i32, vp, vp]
    L.rv_perturber_forces.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rv_system_forces.argtypes = [vp, C.POINTER(rv_system), vp]
    L.rv_kdk_step.argtypes = [vp, C.POINTER(rv_system), f64, i32, vp]
    L.rv_energy.argtypes = [vp, C.POINTER(rv_system), vp, vp]
    L.rv_select_perturbers.argtypes = [vp, i64, vp, vp, vp, C.POINTER(C.c_float), i32, f32, i32, i32, vp, vp, vp]
    L.rv_chain_start_radius.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, C.POINTER(C.c_float), C.c_double,
                                        i32, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double), vp]
    L.rv_block_start.argtypes = [vp, C.POINTER(rv_system), C.POINTER(rv_blocks), vp]
    L.rv_block_steps.argtypes = [vp, C.POINTER(rv_system), C.POINTER(rv_blocks), i32, vp]
    L.rv_block_levels.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, C.POINTER(rv_blocks), i32, vp]
    L.rv_block_count.argtypes = [vp, C.POINTER(C.c_int64), vp]
    L.rv_chain_perturber_forces.argtypes = [vp, C.POINTER(rv_system), C.c_double, vp, vp, vp, vp]
    L.rv_select_perturbers_tidal.argtypes = [vp, i64, vp, vp, vp, vp, C.POINTER(C.c_float), f32, f32, f32, i32, vp,
                                             vp, vp]
    L.rv_select_radius_static.argtypes = [i64, vp, vp, vp, C.POINTER(C.c_float), f32, i32, vp, vp, vp]
    L.rv_get_tree.argtypes = [vp, C.POINTER(rv_tree_view), vp]
    L.rv_walk_stats.argtypes = [vp, C.POINTER(C.c_int64), vp]
    L.rv_sync_status.argtypes = [vp, vp]
    L.rv_profile_walk.argtypes = [vp, i32]
    L.rv_walk_time.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.rv_mlp_param_bytes.argtypes = []
    L.rv_mlp_param_bytes.restype = C.c_size_t
    L.rv_mlp_scratch_bytes.argtypes = [i64]
    L.rv_mlp_scratch_bytes.restype = C.c_size_t
    L.rv_mlp_init.argtypes = [vp, C.c_uint64, vp]
    L.rv_mlp_forward.argtypes = [vp, i64, vp, vp, vp]
    L.rv_mlp_gradient.argtypes = [vp, i64, vp, vp, vp, vp, vp, C.c_size_t, vp]
    L.rv_mlp_adam.argtypes = [vp, vp, i32, f32, f32, f32, f32, vp]
    L.rv_mlp_samples.argtypes = [vp, f32, f32, i64, C.c_uint64, vp, vp, vp, vp]
    L.rv_tree_forces_mlp.argtypes = [vp, vp, f32, f32, f32, vp, vp, vp, vp, vp, i32, vp, vp, vp]
    L.rv_wait_selftest.argtypes = [i64, i32, vp, vp]
    L.rv_mlp_fit_feature_box.argtypes = [vp, i64, vp, vp]
    L.rv_mlp_set_feature_box.argtypes = [vp, vp, vp, vp]
    L.rv_direct_fp64_scratch_bytes.argtypes = [i64]
    L.rv_direct_fp64_scratch_bytes.restype = C.c_size_t
    L.rv_direct_fp64.argtypes = [i64, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, C.c_size_t, vp]
    L.rv_mlp_train_scratch_bytes.argtypes = [i32]
    L.rv_mlp_train_scratch_bytes.restype = C.c_size_t
    L.rv_mlp_train.argtypes = [vp, C.POINTER(rv_mlp_train_cfg), vp, vp, C.c_size_t, vp]
    L.rv_mlp_state_bytes.argtypes = []
    L.rv_mlp_state_bytes.restype = C.c_size_t
    L.rv_mlp_save.argtypes = [vp, vp, C.c_size_t, vp]
    L.rv_mlp_load.argtypes = [vp, vp, C.c_size_t, vp]
    L.rv_chain_absorb.argtypes = [vp, i64, vp, vp, vp, i32, vp, vp, i32, vp, vp, vp, vp]
    L.rv_chain_escape.argtypes = [i32, vp, vp, vp, vp, i32, f64, f64, i32, vp, C.POINTER(rv_chain_escape_result)]
    L.rv_launch_count.argtypes = [vp]
    L.rv_launch_count.restype = C.c_int64
    L.rv_last_error.argtypes = [vp]
    L.rv_last_error.restype = C.c_char_p
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("rv_default_config", "rv_workspace_size", "rv_destroy", "rv_last_error", "rv_launch_count",
                        "rv_mlp_param_bytes", "rv_mlp_scratch_bytes", "rv_direct_fp64_scratch_bytes",
                        "rv_mlp_train_scratch_bytes", "rv_mlp_state_bytes"):
            f.restype = C.c_int


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def default_config(**kw) -> rv_config:
    cfg = rv_config()
    load().rv_default_config(C.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def workspace_size(n_max: int, cfg: rv_config) -> int:
    return int(load().rv_workspace_size(n_max, C.byref(cfg)))


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("librv takes CUDA tensors only")


def select_radius_static(x, y, z, centre, radius, cap=5000, idx=None, count=None, stream=None):
    """rv_select_radius_static: radius perturber search with no context and no
    device allocation inside librv (its scratch is a fixed array in the
    library). ``idx`` (int32 [cap]) and ``count`` (int32 [1]) may be passed in
    by a caller that must not allocate either; otherwise they are created here.
    Returns (idx, count); count holds the untruncated total (above cap: only
    the first cap indices were written)."""
    import torch
    _need_cuda(x, y, z, idx, count)
    if idx is None:
        idx = torch.empty(max(cap, 1), dtype=torch.int32, device=x.device)
    if count is None:
        count = torch.zeros(1, dtype=torch.int32, device=x.device)
    c3 = (C.c_float * 3)(*[float(v) for v in centre])
    st = load().rv_select_radius_static(int(x.shape[0]), _ptr(x), _ptr(y), _ptr(z), c3, float(radius), int(cap),
                                         _ptr(idx), _ptr(count), _stream(stream))
    if st != RV_OK:
        raise RvError(st, "rv_select_radius_static")
    return idx, count


class Context:
    """An rv_ctx with a torch-allocated workspace on the current device."""

    def __init__(self, n_max: int, theta: float = 0.5, eps_star: float = 0.01, n_leaf: int = 16,
                 group: int = 32, quadrupole: bool = True, tile: int = 64, mac: int = 0, alpha: float = 1e-3,
                 softening: int = 0):
        import torch
        self.L = load()
        self.cfg = default_config(theta=theta, eps_star=eps_star, n_leaf=n_leaf, group=group,
                                  quadrupole=int(bool(quadrupole)), tile=tile, mac=int(mac), alpha=float(alpha),
                                  softening=int(softening))
        self.n_max = int(n_max)
        h = C.c_void_p()
        st = self.L.rv_create(C.byref(h), self.n_max, C.byref(self.cfg))
        if st != RV_OK:
            raise RvError(st, "rv_create")
        self.h = h
        nbytes = workspace_size(self.n_max, self.cfg)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = (self.ws.data_ptr() + 255) & ~255
        self._ws_off = base - self.ws.data_ptr()
        self._check(self.L.rv_set_workspace(self.h, C.c_void_p(base), nbytes))
        self.n = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.rv_destroy(h)
            self.h = None

    def _check(self, st):
        if st != RV_OK:
            raise RvError(st, self.L.rv_last_error(self.h).decode())

    def last_error(self) -> str:
        return self.L.rv_last_error(self.h).decode()

    def launch_count(self) -> int:
        return int(self.L.rv_launch_count(self.h))

    def profile_walk(self, enable=True):
        self._check(self.L.rv_profile_walk(self.h, int(bool(enable))))

    def walk_time(self):
        """(summed ms, launches) of the walks recorded since profile_walk(True)."""
        t = C.c_double()
        k = C.c_int64()
        self._check(self.L.rv_walk_time(self.h, C.byref(t), C.byref(k)))
        return float(t.value), int(k.value)

    # --- tree ---
    def build_tree(self, x, y, z, m, stream=None):
        _need_cuda(x, y, z, m)
        n = int(x.shape[0])
        self._check(self.L.rv_build_tree(self.h, n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _stream(stream)))
        self.n = n

    def build_tree_members(self, offsets, x, y, z, m, stream=None):
        """Independent members stored one after another; offsets: host ints [n_members + 1]."""
        import numpy as np
        _need_cuda(x, y, z, m)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self._check(self.L.rv_build_tree_members(self.h, len(off) - 1, off.ctypes.data_as(C.c_void_p), _ptr(x),
                                                 _ptr(y), _ptr(z), _ptr(m), _stream(stream)))
        self.n = int(off[-1])

    def tree_forces_members(self, theta=None, eps_star=None, extra_xyzm=None, extra_eps=None, extra_member=None,
                            out=None, stream=None):
        import torch
        theta = self.cfg.theta if theta is None else theta
        eps_star = self.cfg.eps_star if eps_star is None else eps_star
        if out is None:
            out = [torch.empty(self.n, dtype=torch.float32, device="cuda") for _ in range(4)]
        k = 0 if extra_xyzm is None else int(extra_xyzm.shape[0])
        xout = torch.empty((max(k, 1), 4), dtype=torch.float32, device="cuda") if k else None
        _need_cuda(*out, extra_xyzm, extra_eps, extra_member)
        self._check(self.L.rv_tree_forces_members(self.h, float(theta), float(eps_star), k, _ptr(extra_xyzm),
                                                  _ptr(extra_eps), _ptr(extra_member), *[_ptr(o) for o in out],
                                                  _ptr(xout), _stream(stream)))
        return tuple(out) + ((xout[:k],) if k else ())

    def tree_forces(self, theta=None, eps_star=None, extra_xyzm=None, extra_eps=None, out=None, stream=None):
        """Returns (ax, ay, az, pot[, extra_out (k,4)]) as new or given CUDA tensors."""
        import torch
        theta = self.cfg.theta if theta is None else theta
        eps_star = self.cfg.eps_star if eps_star is None else eps_star
        if out is None:
            out = [torch.empty(self.n, dtype=torch.float32, device="cuda") for _ in range(4)]
        k = 0 if extra_xyzm is None else int(extra_xyzm.shape[0])
        xout = torch.empty((max(k, 1), 4), dtype=torch.float32, device="cuda") if k else None
        _need_cuda(*out, extra_xyzm, extra_eps)
        self._check(self.L.rv_tree_forces(self.h, float(theta), float(eps_star), k, _ptr(extra_xyzm),
                                          _ptr(extra_eps), *[_ptr(o) for o in out], _ptr(xout), _stream(stream)))
        return tuple(out) + ((xout[:k],) if k else ())

    def tree_forces_rel(self, alpha, ref, eps_star=None, out=None, stream=None):
        """Tree forces under the relative opening criterion with tolerance
        alpha and reference accelerations ref = (ax, ay, az) (CUDA FP32 [n]
        each, caller order; may be the output tensors themselves).
        Returns (ax, ay, az, pot)."""
        import torch
        eps_star = self.cfg.eps_star if eps_star is None else eps_star
        if out is None:
            out = [torch.empty(self.n, dtype=torch.float32, device="cuda") for _ in range(4)]
        _need_cuda(*out, *ref)
        self._check(self.L.rv_tree_forces_rel(self.h, float(alpha), float(eps_star), *[_ptr(r) for r in ref],
                                              *[_ptr(o) for o in out], _stream(stream)))
        return tuple(out)

    def tree_sizes(self, stream=None):
        """(stars, cells, groups) of the last tree (rv_get_tree, no copies)."""
        v = rv_tree_view()
        self._check(self.L.rv_get_tree(self.h, C.byref(v), _stream(stream)))
        return int(v.n), int(v.ncell), int(v.ngroup)

    def tree_view(self, stream=None) -> dict:
        """Copies of the last tree's arrays (as CUDA tensors)."""
        import torch
        v = rv_tree_view()
        self._check(self.L.rv_get_tree(self.h, C.byref(v), _stream(stream)))
        base = self.ws.data_ptr()

        def view(ptr, count, dtype, width=1):
            itemsize = torch.empty((), dtype=dtype).element_size()
            off = ptr - base
            nb = count * width * itemsize
            return self.ws[off:off + nb].view(dtype).reshape(count, width).clone() if width > 1 else \
                self.ws[off:off + nb].view(dtype).clone()

        n, nc, ng = v.n, v.ncell, v.ngroup
        return {
            "n": n, "ncell": nc, "ngroup": ng,
            "keys": view(v.keys, n, torch.int64),
            "perm": view(v.perm, n, torch.int32),
            "pos": view(v.pos, n, torch.float32, 4),
            "cbox": view(v.cbox, nc, torch.int32, 4),
            "clink": view(v.clink, nc, torch.int32, 4),
            "cmom": view(v.cmom, 3 * nc, torch.float32, 4).reshape(nc, 12),
            "cparent": view(v.cparent, nc, torch.int32),
            "groups": view(v.groups, ng, torch.int32, 8),
            "bounds": view(v.bounds, 5, torch.float64),
        }

    def walk_stats(self, stream=None):
        """(P2P pairs, M2P pairs) of the last walk."""
        return self.walk_stats3(stream)[:2]

    def walk_stats3(self, stream=None):
        """(P2P pairs, M2P pairs, deepest walk stack so far)."""
        out = (C.c_int64 * 3)()
        self._check(self.L.rv_walk_stats(self.h, out, _stream(stream)))
        return int(out[0]), int(out[1]), int(out[2])

    def sync_status(self, stream=None):
        self._check(self.L.rv_sync_status(self.h, _stream(stream)))

    # --- chain ---
    def perturber_forces(self, chain_m, chain_x, pert_m, pert_x, stream=None):
        """FP64 CUDA tensors in; dict of FP64 CUDA tensors out (see rv.h)."""
        import torch
        _need_cuda(chain_m, chain_x, pert_m, pert_x)
        nch, npt = int(chain_m.shape[0]), int(pert_m.shape[0])
        d = dict(a_pert=torch.zeros((max(npt, 1), 3), dtype=torch.float64, device="cuda"),
                 pot_pert=torch.zeros(max(npt, 1), dtype=torch.float64, device="cuda"),
                 a_chain=torch.zeros((nch, 3), dtype=torch.float64, device="cuda"),
                 pot_chain=torch.zeros(nch, dtype=torch.float64, device="cuda"),
                 out8=torch.zeros(16, dtype=torch.float64, device="cuda"))
        self._check(self.L.rv_perturber_forces(self.h, nch, _ptr(chain_m), _ptr(chain_x), npt, _ptr(pert_m),
                                               _ptr(pert_x), _ptr(d["a_pert"]), _ptr(d["pot_pert"]),
                                               _ptr(d["a_chain"]), _ptr(d["pot_chain"]), _ptr(d["out8"]),
                                               _stream(stream)))
        d["a_pert"], d["pot_pert"] = d["a_pert"][:npt], d["pot_pert"][:npt]
        return d

    def select_perturbers(self, x, y, z, centre, mode, radius=0.0, k=0, cap=5000, stream=None):
        import torch
        _need_cuda(x, y, z)
        idx = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        c3 = (C.c_float * 3)(*[float(v) for v in centre])
        self._check(self.L.rv_select_perturbers(self.h, int(x.shape[0]), _ptr(x), _ptr(y), _ptr(z), c3, int(mode),
                                                float(radius), int(k), int(cap), _ptr(idx), _ptr(cnt),
                                                _stream(stream)))
        return idx, cnt

    def select_perturbers_tidal(self, x, y, z, m, centre, m_chain, gamma_crit, r_crit, cap=5000, stream=None):
        """Eq. 2 tidal perturber search; returns (idx, count) CUDA int32 tensors."""
        import torch
        _need_cuda(x, y, z, m)
        idx = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        c3 = (C.c_float * 3)(*[float(v) for v in centre])
        self._check(self.L.rv_select_perturbers_tidal(self.h, int(x.shape[0]), _ptr(x), _ptr(y), _ptr(z), _ptr(m), c3,
                                                      float(m_chain), float(gamma_crit), float(r_crit), int(cap),
                                                      _ptr(idx), _ptr(cnt), _stream(stream)))
        return idx, cnt

    def chain_perturber_forces(self, sysobj, dt, chain_x, a_chain=None, pot_chain=None, stream=None):
        """Perturber pull on the chain members at chain_x (CUDA FP64 (M n_ch, 3)),
        the last force pass's perturbers predicted dt ahead. Returns (a_chain, pot_chain)."""
        import torch
        nk = sysobj.n_members * sysobj.chains_per_member * sysobj.n_chain
        a_chain = torch.empty(3 * nk, dtype=torch.float64, device="cuda") if a_chain is None else a_chain
        pot_chain = torch.empty(nk, dtype=torch.float64, device="cuda") if pot_chain is None else pot_chain
        _need_cuda(chain_x, a_chain, pot_chain)
        self._check(self.L.rv_chain_perturber_forces(self.h, C.byref(sysobj.c()), float(dt), _ptr(chain_x),
                                                     _ptr(a_chain), _ptr(pot_chain), _stream(stream)))
        return a_chain, pot_chain

    def chain_absorb(self, x, y, z, chain_m, chain_x, cap=5000, stream=None):
        """rv_chain_absorb (Eq. 4): (idx int32 [cap], count int32 [1] untruncated,
        r_chain float64 [1]) as CUDA tensors; chain_m (n_ch,), chain_x (n_ch, 3)."""
        import torch
        cm = torch.as_tensor(chain_m, dtype=torch.float64).to("cuda").contiguous()
        cx = torch.as_tensor(chain_x, dtype=torch.float64).to("cuda").reshape(-1).contiguous()
        idx = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        rch = torch.zeros(1, dtype=torch.float64, device="cuda")
        self._check(self.L.rv_chain_absorb(self.h, int(x.shape[0]), _ptr(x), _ptr(y), _ptr(z), int(cm.shape[0]),
                                           _ptr(cm), _ptr(cx), int(cap), _ptr(idx), _ptr(cnt), _ptr(rch),
                                           _stream(stream)))
        return idx, cnt, rch

    def chain_start_radius(self, pos, vel, m, centre, m_bh, alpha, beta, eps, n_sigma=50, stream=None) -> dict:
        """Eq. 1: returns r2m, sigma, r_sigma, r_infl, r_chain0 (pos/vel: CUDA (x, y, z) tuples)."""
        _need_cuda(*pos, *vel, m)
        c3 = (C.c_float * 3)(*[float(v) for v in centre])
        out = (C.c_double * 5)()
        self._check(self.L.rv_chain_start_radius(self.h, int(m.shape[0]), *[_ptr(t) for t in pos],
                                                 *[_ptr(t) for t in vel], _ptr(m), c3, float(m_bh), int(n_sigma),
                                                 float(alpha), float(beta), float(eps), out, _stream(stream)))
        return dict(zip(("r2m", "sigma", "r_sigma", "r_infl", "r_chain0"), list(out)))

    def block_start(self, sysobj, blocks, stream=None):
        b = blocks.c()
        self._check(self.L.rv_block_start(self.h, C.byref(sysobj.c()), C.byref(b), _stream(stream)))
        blocks.substep = int(b.substep)

    def block_steps(self, sysobj, blocks, nsub, stream=None):
        b = blocks.c()
        self._check(self.L.rv_block_steps(self.h, C.byref(sysobj.c()), C.byref(b), int(nsub), _stream(stream)))
        blocks.substep = int(b.substep)

    def block_levels(self, blocks, acc, vel, start=False, stream=None):
        """The level rule on device FP32 acc = (ax, ay, az), vel = (vx, vy, vz)."""
        _need_cuda(*acc, *vel)
        b = blocks.c()
        self._check(self.L.rv_block_levels(self.h, int(acc[0].shape[0]), *[_ptr(t) for t in acc],
                                           *[_ptr(t) for t in vel], C.byref(b), int(bool(start)), _stream(stream)))

    def block_count(self, stream=None) -> int:
        v = C.c_int64(0)
        self._check(self.L.rv_block_count(self.h, C.byref(v), _stream(stream)))
        return int(v.value)

    def system_forces(self, sysobj, stream=None):
        self._check(self.L.rv_system_forces(self.h, C.byref(sysobj.c()), _stream(stream)))

    def kdk_step(self, sysobj, dt, nsteps=1, stream=None):
        self._check(self.L.rv_kdk_step(self.h, C.byref(sysobj.c()), float(dt), int(nsteps), _stream(stream)))

    def kdk_step_graph(self, sysobj, dt, nsteps=1, energy_out=None, stream=None):
        """Graph-captured KDK steps; `stream` must be a torch.cuda.Stream (not the default stream)."""
        self._check(self.L.rv_kdk_step_graph(self.h, C.byref(sysobj.c()), float(dt), int(nsteps),
                                             _ptr(energy_out), _stream(stream)))

    def energy(self, sysobj, out=None, stream=None):
        import torch
        if out is None:
            out = torch.zeros(10 * max(1, sysobj.n_members), dtype=torch.float64, device="cuda")
        self._check(self.L.rv_energy(self.h, C.byref(sysobj.c()), _ptr(out), _stream(stream)))
        return out


class System:
    """Device state of stars (FP32, caller order) and an optional chain (FP64)."""

    def __init__(self, pos, vel, mass, chain_m=None, chain_x=None, chain_v=None, pert_mode=0, pert_radius=0.0,
                 pert_k=0, member_offsets=None, pert_gamma=0.0, chains_per_member=1, chain_quad=True):
        """pos/vel (3, n); mass (n,). member_offsets: host ints [M + 1] for M
        independent members stored one after another (None: one member).
        chain_* are member-major: chain_m (M n_ch,) or (n_ch,), chain_x/v
        (M n_ch, 3). pert_mode 1 radius, 2 k nearest, 3 tidal (Eq. 2,
        r_crit = pert_radius, gamma_crit = pert_gamma). chains_per_member: C
        chains in every member (chain arrays hold M C chains of n_ch members,
        member by member). chain_quad: the stars beyond the perturbers also
        feel each chain's quadrupole (rv_system.chain_quad)."""
        import torch
        f32 = dict(dtype=torch.float32, device="cuda")
        f64 = dict(dtype=torch.float64, device="cuda")
        pos = torch.as_tensor(pos)
        vel = torch.as_tensor(vel)
        self.n = int(pos.shape[1])
        # one block, rows x, y, z, vx, vy, vz, ax, ay, az, pot (each row a
        # contiguous array): the whole state moves in one copy
        self.state = torch.zeros((10, self.n), **f32)
        self.x, self.y, self.z, self.vx, self.vy, self.vz, self.ax, self.ay, self.az, self.pot = self.state.unbind(0)
        for a in range(3):
            self.state[a].copy_(pos[a].to(**f32))
            self.state[3 + a].copy_(vel[a].to(**f32))
        self.m = torch.as_tensor(mass).to(**f32).contiguous()
        self.n_chain = 0 if chain_m is None else int(len(chain_m))
        if self.n_chain:
            self.chain_m = torch.as_tensor(chain_m).to(**f64).contiguous()
            self.chain_x = torch.as_tensor(chain_x).to(**f64).reshape(-1).contiguous()
            self.chain_v = torch.as_tensor(chain_v).to(**f64).reshape(-1).contiguous()
            self.chain_a = torch.zeros(3 * self.n_chain, **f64)
            self.chain_pot = torch.zeros(self.n_chain, **f64)
        else:
            self.chain_m = self.chain_x = self.chain_v = self.chain_a = self.chain_pot = None
        self.pert_mode, self.pert_radius, self.pert_k = int(pert_mode), float(pert_radius), int(pert_k)
        self.pert_gamma = float(pert_gamma)
        import numpy as np
        if member_offsets is None:
            self.n_members, self.member_offsets = 1, None
        else:
            self.member_offsets = np.ascontiguousarray(member_offsets, dtype=np.int64)
            self.n_members = int(len(self.member_offsets) - 1)
        self.chains_per_member = int(chains_per_member)
        self.chain_quad = int(bool(chain_quad))
        if self.n_chain:
            self.n_chain //= self.n_members * self.chains_per_member   # members of each chain
        self._c = None

    def c(self) -> rv_system:
        s = rv_system()
        s.n = self.n
        for f in ("x", "y", "z", "vx", "vy", "vz", "m", "ax", "ay", "az", "pot"):
            setattr(s, f, getattr(self, f).data_ptr())
        s.n_chain = self.n_chain
        for f in ("chain_m", "chain_x", "chain_v", "chain_a", "chain_pot"):
            t = getattr(self, f)
            setattr(s, f, t.data_ptr() if t is not None else None)
        s.pert_mode, s.pert_radius, s.pert_k = self.pert_mode, self.pert_radius, self.pert_k
        s.pert_gamma = self.pert_gamma
        s.n_chains = self.chains_per_member
        s.chain_quad = self.chain_quad
        s.n_members = self.n_members
        s.member_offsets = None if self.member_offsets is None else self.member_offsets.ctypes.data
        self._c = s
        return s


class Blocks:
    """Block time-step state: levels (CUDA int8 [n]) and parameters (see rv_blocks)."""

    def __init__(self, n, dt_max, max_level, tau_acc=0.3, tau_vel=0.3, eps=0.01, adapt=True, level=None):
        import torch
        self.level = (torch.zeros(n, dtype=torch.int8, device="cuda") if level is None else
                      torch.as_tensor(level).to(dtype=torch.int8, device="cuda").contiguous())
        self.dt_max, self.max_level = float(dt_max), int(max_level)
        self.tau_acc, self.tau_vel, self.eps, self.adapt = float(tau_acc), float(tau_vel), float(eps), bool(adapt)
        self.substep = 0

    def c(self) -> rv_blocks:
        b = rv_blocks()
        b.dt_max, b.max_level = self.dt_max, self.max_level
        b.tau_acc, b.tau_vel, b.eps, b.adapt = self.tau_acc, self.tau_vel, self.eps, int(self.adapt)
        b.level = self.level.data_ptr()
        b.substep = self.substep
        self._c = b
        return b


# --------------------------------------------------------------------------
# learned cell-force correction
# --------------------------------------------------------------------------
MLP_PARAMS = 5768
MLP_LAYOUT = (("W1", (16, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 8)), ("b3", (8,)))


class Mlp:
    """Parameter block of the correction network on the current device."""

    def __init__(self, seed=1, stream=None):
        import torch
        self.L = load()
        self.block = torch.zeros(int(self.L.rv_mlp_param_bytes()), dtype=torch.uint8, device="cuda")
        self._scratch = None
        st = self.L.rv_mlp_init(_ptr(self.block), int(seed), _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_init")
        self.step = 0

    def master(self):
        """FP32 master parameters as a dict of CUDA tensors (views)."""
        w = self.block[:4 * MLP_PARAMS].view(torch_float32())
        out, o = {}, 0
        for k, shp in MLP_LAYOUT:
            sz = 1
            for s in shp:
                sz *= s
            out[k] = w[o:o + sz].view(*shp)
            o += sz
        return out

    def forward(self, x, stream=None):
        import torch
        y = torch.empty((x.shape[0], 3), dtype=torch.float32, device=x.device)
        st = self.L.rv_mlp_forward(_ptr(self.block), int(x.shape[0]), _ptr(x), _ptr(y), _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_forward")
        return y

    def gradient(self, x, t, stream=None):
        import torch
        n = int(x.shape[0])
        need = int(self.L.rv_mlp_scratch_bytes(n))
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = torch.empty(need, dtype=torch.uint8, device=x.device)
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        st = self.L.rv_mlp_gradient(_ptr(self.block), n, _ptr(x), _ptr(t), _ptr(grad), _ptr(loss),
                                    _ptr(self._scratch), self._scratch.numel(), _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_gradient")
        return grad, loss

    def adam(self, grad, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        self.step += 1
        st = self.L.rv_mlp_adam(_ptr(self.block), _ptr(grad), self.step, lr, b1, b2, eps, _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_adam")

    def fit_feature_box(self, x, stream=None):
        """The feature box becomes the per-feature range of the rows x (n, 16)."""
        st = self.L.rv_mlp_fit_feature_box(_ptr(self.block), int(x.shape[0]), _ptr(x), _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_fit_feature_box")

    def set_feature_box(self, lo, hi, stream=None):
        """Sets the feature box from 16 lower and 16 upper bounds (host)."""
        import numpy as np
        lo = np.ascontiguousarray(lo, dtype=np.float32)
        hi = np.ascontiguousarray(hi, dtype=np.float32)
        if lo.shape != (16,) or hi.shape != (16,):
            raise ValueError("feature box bounds need 16 values each")
        st = self.L.rv_mlp_set_feature_box(_ptr(self.block), lo.ctypes.data_as(C.c_void_p),
                                           hi.ctypes.data_as(C.c_void_p), _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_set_feature_box")

    def feature_box(self):
        """(lo, hi) as numpy arrays of 16."""
        box = self.block[-4 * 32:].view(torch_float32()).cpu().numpy()
        return box[:16].copy(), box[16:].copy()

    def train(self, x, t, steps, batch=4096, lr=1e-3, seed=0, b1=0.9, b2=0.999, eps=1e-8, fit_box=True,
              stream=None):
        """rv_mlp_train: `steps` Adam steps on SplitMix64-drawn minibatches of
        (x [n,16], t [n,3]), all on the device in one call; returns the
        per-step losses. With fit_box the feature box becomes the range of x."""
        import torch
        x = x.contiguous()
        t = t.contiguous()
        need = int(self.L.rv_mlp_train_scratch_bytes(int(batch)))
        scratch = torch.empty(max(need, 1), dtype=torch.uint8, device=x.device)
        losses = torch.empty(max(int(steps), 1), dtype=torch.float32, device=x.device)
        cfg = rv_mlp_train_cfg(n=int(x.shape[0]), x=_ptr(x), t=_ptr(t), steps=int(steps), batch=int(batch),
                               step0=self.step + 1, lr=float(lr), beta1=float(b1), beta2=float(b2),
                               adam_eps=float(eps), seed=int(seed), fit_box=int(bool(fit_box)))
        st = self.L.rv_mlp_train(_ptr(self.block), C.byref(cfg), _ptr(losses), _ptr(scratch), need,
                                 _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_train")
        self.step += int(steps)
        return [float(v) for v in losses[:int(steps)].cpu().tolist()]

    def save(self, stream=None) -> bytes:
        """rv_mlp_save: the whole network state as bytes."""
        n = int(self.L.rv_mlp_state_bytes())
        buf = (C.c_char * n)()
        st = self.L.rv_mlp_save(_ptr(self.block), C.cast(buf, C.c_void_p), n, _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_save")
        return bytes(buf)

    def load(self, state: bytes, step=None, stream=None):
        """rv_mlp_load: restores a state from save(); `step` sets the Adam step
        count the next training continues from."""
        buf = C.create_string_buffer(bytes(state), len(state))
        st = self.L.rv_mlp_load(_ptr(self.block), C.cast(buf, C.c_void_p), len(state), _stream(stream))
        if st != RV_OK:
            raise RvError(st, "rv_mlp_load")
        if step is not None:
            self.step = int(step)


def chain_escape(mass, pos, vel, massive, designated, r_chain0, gamma, n_absorbing):
    """rv_chain_escape (Eq. 5 and the membership rules; host only): returns
    dict escape (bool array), terminate, designated, r_chain, r_escape."""
    import numpy as np
    m = np.ascontiguousarray(mass, dtype=np.float64)
    x = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    v = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1)
    mv = np.ascontiguousarray(massive, dtype=np.int32)
    k = int(m.shape[0])
    esc = np.zeros(max(k, 1), dtype=np.int32)
    res = rv_chain_escape_result()
    st = load().rv_chain_escape(k, m.ctypes.data, x.ctypes.data, v.ctypes.data, mv.ctypes.data, int(designated),
                                float(r_chain0), float(gamma), int(n_absorbing), esc.ctypes.data, C.byref(res))
    if st != RV_OK:
        raise RvError(st, "rv_chain_escape")
    return {"escape": esc[:k].astype(bool), "terminate": int(res.terminate), "designated": int(res.designated),
            "r_chain": float(res.r_chain), "r_escape": float(res.r_escape), "escape_count": int(res.escape_count)}


def torch_float32():
    import torch
    return torch.float32


def direct_fp64(pos, mass, eps, targets, stream=None):
    """FP64 direct-summation acceleration and potential on `targets` from all
    bodies (see rv_direct_fp64). pos (3, n), mass (n,), eps scalar or (n,)
    (0: unsoftened), targets (nt,) indices; numpy or torch. Returns numpy
    (acc (3, nt), pot (nt,))."""
    import numpy as np
    import torch
    dev = dict(dtype=torch.float64, device="cuda")
    pos = torch.as_tensor(pos).to(**dev)
    n = int(pos.shape[1])
    x, y, z = (pos[a].contiguous() for a in range(3))
    m = torch.as_tensor(mass).to(**dev).contiguous()
    e = torch.as_tensor(eps, dtype=torch.float64)
    e = (e.expand(n) if e.dim() == 0 else e).to(**dev).contiguous()
    t = torch.as_tensor(np.asarray(targets, dtype=np.int64)).to(device="cuda").contiguous()
    nt = int(t.shape[0])
    out = [torch.empty(nt, **dev) for _ in range(4)]
    L = load()
    need = int(L.rv_direct_fp64_scratch_bytes(nt))
    scratch = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
    st = L.rv_direct_fp64(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(e), nt, _ptr(t), *[_ptr(o) for o in out],
                          _ptr(scratch), need, _stream(stream))
    if st != RV_OK:
        raise RvError(st, "rv_direct_fp64")
    o = [u.cpu().numpy() for u in out]
    return np.stack(o[:3]), o[3]


def wait_selftest(limit_cycles, arrive, stream=None):
    """Runs the bounded tensor-core completion wait once (see rv_wait_selftest):
    returns 1 if it ran out after limit_cycles, else 0."""
    import torch
    flag = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = load().rv_wait_selftest(int(limit_cycles), int(bool(arrive)), _ptr(flag), _stream(stream))
    if st != RV_OK:
        raise RvError(st, "rv_wait_selftest")
    return int(flag.item())


def mlp_samples(ctx, theta, eps_star, n, seed, stream=None):
    """Training samples from ctx's last tree: (x [n,16], t [n,3], pairs [n,2])."""
    import torch
    x = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    t = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    p = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    ctx._check(ctx.L.rv_mlp_samples(ctx.h, float(theta), float(eps_star), int(n), int(seed), _ptr(x), _ptr(t),
                                    _ptr(p), _stream(stream)))
    return x, t, p


def tree_forces_mlp(ctx, mlp, theta, theta_rec, eps_star, pair_cap=1 << 24, stream=None):
    """(ax, ay, az, pot, pairs, npairs) with the learned correction."""
    import torch
    n = ctx.n
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(4)]
    pairs = torch.empty((pair_cap, 2), dtype=torch.int32, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int32, device="cuda")
    gcorr = torch.empty(3 * max(n, 1), dtype=torch.float32, device="cuda")
    ctx._check(ctx.L.rv_tree_forces_mlp(ctx.h, _ptr(mlp.block), float(theta), float(theta_rec), float(eps_star),
                                        *[_ptr(o) for o in out], _ptr(pairs), int(pair_cap), _ptr(npairs),
                                        _ptr(gcorr), _stream(stream)))
    return (*out, pairs, npairs)
