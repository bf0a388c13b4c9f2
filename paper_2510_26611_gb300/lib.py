"""Thin ctypes binding of librs (include/rs.h), same names as the C ABI.

Only argument marshalling happens here: numpy arrays and CPU tensors are passed
as host pointers (RS_MEM_HOST), CUDA tensors as device pointers on the current
torch stream (RS_MEM_DEVICE).  Every computation runs in the library's kernels.
The library is built on first use; if it cannot be built or loaded, import of
this module raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import _build

RS_OK = 0
RS_ERR_INVALID = -1
RS_ERR_OOM = -2
RS_ERR_CUDA = -3
RS_ERR_TIMEOUT = -4
RS_ERR_BUSY = -5
RS_ERR_NOT_READY = -6
RS_ERR_UNSUPPORTED = -7
RS_MEM_HOST = 0
RS_MEM_DEVICE = 1
RS_FLAG_CLASH = 1
RS_FLAG_OUT_OF_GRID = 2

_STATUS_NAMES = {0: "RS_OK", -1: "RS_ERR_INVALID", -2: "RS_ERR_OOM", -3: "RS_ERR_CUDA",
                 -4: "RS_ERR_TIMEOUT", -5: "RS_ERR_BUSY", -6: "RS_ERR_NOT_READY",
                 -7: "RS_ERR_UNSUPPORTED"}


class RSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class rs_params(C.Structure):
    _fields_ = [("n", C.c_int32), ("b", C.c_double), ("sigma", C.c_double), ("R_l", C.c_int32),
                ("r_min", C.c_double), ("tau", C.c_double), ("short_tol", C.c_double),
                ("tucker_cap", C.c_int32), ("eps_r", C.c_double), ("galerkin", C.c_int32)]


class rs_protein_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("N", C.c_int32), ("R_l", C.c_int32), ("K", C.c_int32),
                ("b", C.c_double), ("h", C.c_double), ("sigma", C.c_double), ("r_c", C.c_double),
                ("h_s", C.c_double), ("quad_err", C.c_double), ("kind", C.c_int32),
                ("rank", C.c_int32 * 3), ("sv_gap", C.c_double * 3), ("sv_tail", C.c_double * 3),
                ("device_bytes", C.c_size_t)]


class rs_pair(C.Structure):
    _fields_ = [("prot", C.c_void_p), ("L", C.c_int32), ("lig_xyz", C.c_void_p),
                ("lig_q", C.c_void_p), ("P", C.c_int64), ("quat", C.c_void_p),
                ("trans", C.c_void_p), ("E_out", C.c_void_p), ("flags_out", C.c_void_p)]


class rs_batch_info(C.Structure):
    _fields_ = [("npairs", C.c_int32), ("ngroups", C.c_int32), ("nitems", C.c_int32),
                ("grid", C.c_int32), ("threads", C.c_int32), ("atoms_per_item", C.c_int32),
                ("tune_ms", C.c_double), ("mode", C.c_int32), ("warps_per_cta", C.c_int32),
                ("chunk_atoms", C.c_int64), ("nchunks", C.c_int32), ("streams", C.c_int32)]


class rs_request(C.Structure):
    _fields_ = [("protein_id", C.c_uint64), ("N", C.c_int32), ("prot_xyz", C.c_void_p),
                ("prot_q", C.c_void_p), ("params", rs_params), ("L", C.c_int32),
                ("lig_xyz", C.c_void_p), ("lig_q", C.c_void_p), ("P", C.c_int64),
                ("quat", C.c_void_p), ("trans", C.c_void_p)]


class rs_result(C.Structure):
    _fields_ = [("status", C.c_int), ("t_submit_ns", C.c_int64), ("t_admit_ns", C.c_int64),
                ("t_start_ns", C.c_int64), ("t_end_ns", C.c_int64), ("message", C.c_char * 160)]


class rs_serve_params(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_uint64), ("max_queue", C.c_int32),
                ("max_inflight_launches", C.c_int32), ("idle_wait_ms", C.c_int32),
                ("inject_alloc_failures", C.c_int32), ("group_min_atoms", C.c_int64),
                ("group_atoms_per_cell", C.c_double), ("hold_builds", C.c_int32)]


class rs_serve_stats(C.Structure):
    _fields_ = [("done", C.c_uint64), ("failed", C.c_uint64), ("launches", C.c_uint64),
                ("builds", C.c_uint64), ("cache_hits", C.c_uint64), ("evictions", C.c_uint64),
                ("queued", C.c_uint64), ("cached_proteins", C.c_uint64),
                ("budget_bytes", C.c_uint64), ("used_bytes", C.c_uint64),
                ("mean_requests_per_launch", C.c_double)]


def _load() -> C.CDLL:
    path = os.environ.get("RS_LIBRARY") or _build.build()
    lib = C.CDLL(path)
    vp, i32, i64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_int
    sig = {
        "rs_params_default": (None, [C.POINTER(rs_params)]),
        "rs_ctx_create": (st, [C.c_int, C.POINTER(vp)]),
        "rs_ctx_destroy": (None, [vp]),
        "rs_last_error": (C.c_char_p, []),
        "rs_version": (C.c_char_p, []),
        "rs_build_protein": (st, [vp, i32, vp, vp, C.POINTER(rs_params), C.c_int, vp, C.POINTER(vp)]),
        "rs_protein_free": (None, [vp]),
        "rs_protein_get_info": (st, [vp, C.POINTER(rs_protein_info)]),
        "rs_protein_get_table": (st, [vp, vp, vp, vp]),
        "rs_energy_poses": (st, [vp, vp, i32, vp, vp, i64, vp, vp, vp, vp, C.c_int, vp]),
        "rs_energy_grad_poses": (st, [vp, vp, i32, vp, vp, i64, vp, vp, vp, vp, vp, vp, C.c_int, vp]),
        "rs_energy_poses_noalloc": (st, [vp, i32, vp, vp, i64, vp, vp, vp, vp, vp]),
        "rs_fd_forces_poses": (st, [vp, vp, i32, vp, vp, i64, vp, vp, C.c_double, C.c_double, vp, vp, vp,
                                    vp, vp, vp, C.c_int, vp]),
        "rs_ppiem_scan": (st, [vp, vp, i32, vp, vp, i32, i32, i32, vp, vp, C.c_double, vp, vp, vp, vp, vp,
                               vp, vp, C.c_int, vp]),
        "rs_protein_local_box": (st, [vp, vp, vp, vp, C.c_double, C.POINTER(vp)]),
        "rs_protein_add_compress": (st, [vp, vp, i32, i32, C.c_double, vp, C.POINTER(vp)]),
        "rs_energy_poses_complex": (st, [vp, i32, vp, i32, vp, vp, i64, vp, vp, vp, vp, C.c_int, vp]),
        "rs_pgd_run": (st, [vp, vp, i32, vp, vp, i64, vp, vp, i32, C.c_double, C.c_double, i32,
                            vp, vp, vp, vp]),
        "rs_batch_create": (st, [vp, i32, C.POINTER(rs_pair), i32, C.POINTER(vp)]),
        "rs_batch_run": (st, [vp, vp]),
        "rs_batch_free": (None, [vp]),
        "rs_batch_get_info": (st, [vp, C.POINTER(rs_batch_info)]),
        "rs_serve_params_default": (None, [C.POINTER(rs_serve_params)]),
        "rs_request_validate": (st, [C.POINTER(rs_request)]),
        "rs_serve_create": (st, [C.c_int, C.POINTER(rs_serve_params), C.POINTER(vp)]),
        "rs_serve_submit": (st, [vp, C.POINTER(rs_request), vp, vp, C.POINTER(C.c_uint64)]),
        "rs_serve_poll": (st, [vp, C.c_uint64, C.POINTER(rs_result)]),
        "rs_serve_wait": (st, [vp, C.c_uint64, i32, C.POINTER(rs_result)]),
        "rs_serve_cancel": (st, [vp, C.c_uint64]),
        "rs_serve_release_builds": (st, [vp]),
        "rs_serve_get_stats": (st, [vp, C.POINTER(rs_serve_stats)]),
        "rs_serve_destroy": (None, [vp]),
        "rs_symeig_host": (st, [i32, vp, vp, vp]),
        "rs_qr_host": (st, [i32, i32, vp, vp]),
        "rs_set_wform_kernel": (C.c_int, [C.c_int]),
        "rs_set_build_gemm_kernel": (C.c_int, [C.c_int]),
        "rs_tc_error_count": (st, [C.c_int, C.POINTER(i32)]),
        "rs_diag_tc_contract": (st, [i32, i32, vp, vp, vp, vp, vp]),
        "rs_diag_tc_launch": (st, [C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]),
        "rs_diag_short_counts": (st, [C.c_int, C.c_int, vp, C.POINTER(C.c_double), C.c_int]),
        "rs_diag_pair_exp": (st, [i32, vp, vp]),
        "rs_stats_kernel_launches": (C.c_ulonglong, []),
        "rs_timing_enable": (st, [C.c_int]),
        "rs_timing_reset": (st, []),
        "rs_timing_count": (C.c_int, []),
        "rs_timing_get": (st, [C.c_int, C.c_char_p, C.c_size_t, C.POINTER(C.c_double),
                               C.POINTER(C.c_ulonglong), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
LIBRARY_PATH = _lib._name


def header_symbols() -> list[str]:
    """Function names declared in include/rs.h."""
    hdr = os.path.join(_build.ROOT, "include", "rs.h")
    text = open(hdr).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_0-9]+)\s*\(", text)))


def _check(status: int):
    if status != RS_OK:
        raise RSError(status, _lib.rs_last_error().decode())


def rs_last_error() -> str:
    return _lib.rs_last_error().decode()


def rs_version() -> str:
    return _lib.rs_version().decode()


def rs_params_default(**overrides) -> rs_params:
    p = rs_params()
    _lib.rs_params_default(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def rs_ctx_create(device: int = 0) -> int:
    h = C.c_void_p()
    _check(_lib.rs_ctx_create(device, C.byref(h)))
    return h.value


def rs_ctx_destroy(ctx: int) -> None:
    _lib.rs_ctx_destroy(ctx)


# ------------------------------------------------------------------ marshalling
def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _stream_ptr(stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def _host(x, dtype) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def _dev(x, dtype):
    import torch
    tdt = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
    if x.dtype != tdt or not x.is_contiguous():
        x = x.to(tdt).contiguous()
    return x


def _ptr(x):
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def rs_build_protein(ctx: int, xyz, q, params: rs_params | None = None, stream=None) -> int:
    """Algorithm TEP: returns a protein handle (free with rs_protein_free)."""
    if params is None:
        params = rs_params_default()
    h = C.c_void_p()
    if _is_cuda(xyz):
        xyz_, q_ = _dev(xyz, np.float64), _dev(q, np.float64)
        mem, sp = RS_MEM_DEVICE, _stream_ptr(stream)
    else:
        xyz_, q_ = _host(xyz, np.float64), _host(q, np.float64)
        mem, sp = RS_MEM_HOST, None
    N = int(q_.shape[0])
    if tuple(xyz_.shape) != (N, 3):
        raise RSError(RS_ERR_INVALID, f"xyz must be ({N}, 3), got {tuple(xyz_.shape)}")
    _check(_lib.rs_build_protein(ctx, N, _ptr(xyz_), _ptr(q_), C.byref(params), mem, sp, C.byref(h)))
    return h.value


def rs_protein_free(prot: int) -> None:
    _lib.rs_protein_free(prot)


def rs_protein_get_info(prot: int) -> dict:
    info = rs_protein_info()
    _check(_lib.rs_protein_get_info(prot, C.byref(info)))
    d = {k: getattr(info, k) for k, _ in info._fields_}
    for k in ("rank", "sv_gap", "sv_tail"):
        d[k] = list(d[k])
    return d


def rs_protein_get_table(prot: int):
    K = rs_protein_get_info(prot)["K"]
    t, a, il = np.zeros(K), np.zeros(K), np.zeros(K, dtype=np.uint8)
    _check(_lib.rs_protein_get_table(prot, t.ctypes.data, a.ctypes.data, il.ctypes.data))
    return t, a, il.astype(bool)


def _pose_call(grad: bool, ctx, prot, lig_xyz, lig_q, rot, trans, E_out, flags_out,
               dE_dt, dE_dw, stream):
    rdim = 3 if grad else 4
    if _is_cuda(rot):
        import torch
        dev = rot.device
        lx, lq = _dev(lig_xyz.to(dev), np.float64), _dev(lig_q.to(dev), np.float64)
        r, t = _dev(rot, np.float64), _dev(trans, np.float64)
        P = int(r.shape[0])
        E = E_out if E_out is not None else torch.empty(P, dtype=torch.float64, device=dev)
        f = flags_out if flags_out is not None else torch.empty(P, dtype=torch.uint8, device=dev)
        gt = gw = None
        if grad:
            gt = dE_dt if dE_dt is not None else torch.empty((P, 3), dtype=torch.float64, device=dev)
            gw = dE_dw if dE_dw is not None else torch.empty((P, 3), dtype=torch.float64, device=dev)
        mem, sp = RS_MEM_DEVICE, _stream_ptr(stream)
    else:
        lx, lq = _host(lig_xyz, np.float64), _host(lig_q, np.float64)
        r, t = _host(rot, np.float64), _host(trans, np.float64)
        P = int(r.shape[0])
        E = E_out if E_out is not None else np.empty(P)
        f = flags_out if flags_out is not None else np.empty(P, dtype=np.uint8)
        gt = gw = None
        if grad:
            gt = dE_dt if dE_dt is not None else np.empty((P, 3))
            gw = dE_dw if dE_dw is not None else np.empty((P, 3))
        mem, sp = RS_MEM_HOST, None
    L = int(lq.shape[0])
    if tuple(lx.shape) != (L, 3) or tuple(r.shape) != (P, rdim) or tuple(t.shape) != (P, 3):
        raise RSError(RS_ERR_INVALID, "shape mismatch in pose arguments")
    if grad:
        _check(_lib.rs_energy_grad_poses(ctx, prot, L, _ptr(lx), _ptr(lq), P, _ptr(r), _ptr(t),
                                         _ptr(E), _ptr(gt), _ptr(gw), _ptr(f), mem, sp))
        return E, gt, gw, f
    _check(_lib.rs_energy_poses(ctx, prot, L, _ptr(lx), _ptr(lq), P, _ptr(r), _ptr(t),
                                _ptr(E), _ptr(f), mem, sp))
    return E, f


def rs_energy_poses(ctx, prot, lig_xyz, lig_q, quat, trans, E_out=None, flags_out=None,
                    stream=None):
    """Algorithm PLIE over poses given by quaternions; returns (E, flags)."""
    return _pose_call(False, ctx, prot, lig_xyz, lig_q, quat, trans, E_out, flags_out, None,
                      None, stream)


def rs_energy_grad_poses(ctx, prot, lig_xyz, lig_q, rotvec, trans, E_out=None, dE_dt=None,
                         dE_dw=None, flags_out=None, stream=None):
    """Energies and exact gradients for poses given by rotation vectors;
    returns (E, dE_dt, dE_dw, flags)."""
    return _pose_call(True, ctx, prot, lig_xyz, lig_q, rotvec, trans, E_out, flags_out, dE_dt,
                      dE_dw, stream)


def rs_fd_forces_poses(ctx, prot, lig_xyz, lig_q, rotvec, trans, h: float = 0.0, r0: float = 0.0,
                       stream=None) -> dict:
    """The paper's backward-difference atom forces (Eq. differ_ligand) and their
    rigid-cluster resultants (Eq. Field_Xcenter, Eq. Field_phi) for poses given by
    rotation vectors.  Returns a dict with E, F (sum of atom forces), F0 (radial),
    Fphi (tangential at radius r0), M (moment about the centre) and flags, as CUDA
    tensors when rotvec is one, numpy arrays otherwise."""
    if _is_cuda(rotvec):
        import torch
        dev = rotvec.device
        lx, lq = _dev(lig_xyz.to(dev), np.float64), _dev(lig_q.to(dev), np.float64)
        r, t = _dev(rotvec, np.float64), _dev(trans, np.float64)
        P = int(r.shape[0])
        new = lambda *shape: torch.empty(shape, dtype=torch.float64, device=dev)
        f = torch.empty(P, dtype=torch.uint8, device=dev)
        mem, sp = RS_MEM_DEVICE, _stream_ptr(stream)
    else:
        lx, lq = _host(lig_xyz, np.float64), _host(lig_q, np.float64)
        r, t = _host(rotvec, np.float64), _host(trans, np.float64)
        P = int(r.shape[0])
        new = lambda *shape: np.empty(shape)
        f = np.empty(P, dtype=np.uint8)
        mem, sp = RS_MEM_HOST, None
    L = int(lq.shape[0])
    if tuple(lx.shape) != (L, 3) or tuple(r.shape) != (P, 3) or tuple(t.shape) != (P, 3):
        raise RSError(RS_ERR_INVALID, "shape mismatch in pose arguments")
    out = {"E": new(P), "F": new(P, 3), "F0": new(P, 3), "Fphi": new(P, 3), "M": new(P, 3), "flags": f}
    _check(_lib.rs_fd_forces_poses(ctx, prot, L, _ptr(lx), _ptr(lq), P, _ptr(r), _ptr(t), float(h), float(r0),
                                   _ptr(out["E"]), _ptr(out["F"]), _ptr(out["F0"]), _ptr(out["Fphi"]),
                                   _ptr(out["M"]), _ptr(f), mem, sp))
    return out


def rs_energy_poses_complex(ctx, mols, lig_xyz, lig_q, quat, trans, stream=None):
    """Energies of a ligand molecule against a complex of molecules (the sum of their
    RS potentials, Eq. EnergySum_Mcomplex); mols: protein handles.  Returns (E, flags)
    as CUDA tensors when quat is one, numpy arrays otherwise."""
    arr = (C.c_void_p * len(mols))(*[int(m) for m in mols])
    if _is_cuda(quat):
        import torch
        dev = quat.device
        lx, lq = _dev(lig_xyz.to(dev), np.float64), _dev(lig_q.to(dev), np.float64)
        r, t = _dev(quat, np.float64), _dev(trans, np.float64)
        P = int(r.shape[0])
        E = torch.empty(P, dtype=torch.float64, device=dev)
        f = torch.empty(P, dtype=torch.uint8, device=dev)
        mem, sp = RS_MEM_DEVICE, _stream_ptr(stream)
    else:
        lx, lq = _host(lig_xyz, np.float64), _host(lig_q, np.float64)
        r, t = _host(quat, np.float64), _host(trans, np.float64)
        P = int(r.shape[0])
        E, f = np.empty(P), np.empty(P, dtype=np.uint8)
        mem, sp = RS_MEM_HOST, None
    L = int(lq.shape[0])
    if tuple(lx.shape) != (L, 3) or tuple(r.shape) != (P, 4) or tuple(t.shape) != (P, 3):
        raise RSError(RS_ERR_INVALID, "shape mismatch in pose arguments")
    _check(_lib.rs_energy_poses_complex(ctx, len(mols), arr, L, _ptr(lx), _ptr(lq), P, _ptr(r), _ptr(t), _ptr(E),
                                        _ptr(f), mem, sp))
    return E, f


def rs_protein_local_box(ctx: int, parent: int, lo, hi, eps: float = 1e-7) -> int:
    """Local-box handle of a Tucker protein (scheme C): its potential restricted to
    the box [lo, hi] and re-truncated to lower ranks there; free with rs_protein_free."""
    l = np.ascontiguousarray(lo, dtype=np.float64).reshape(3)
    h = np.ascontiguousarray(hi, dtype=np.float64).reshape(3)
    out = C.c_void_p()
    _check(_lib.rs_protein_local_box(ctx, parent, l.ctypes.data, h.ctypes.data, float(eps), C.byref(out)))
    return out.value


def rs_protein_add_compress(ctx: int, parts, tucker_cap: int, eps_r: float = 1e-7, stream=None) -> int:
    """One Tucker handle for the sum of the parts' long-range tensors, re-truncated
    (add-and-compress), with the short range of the union of their atoms; free with
    rs_protein_free."""
    arr = (C.c_void_p * len(parts))(*[int(m) for m in parts])
    out = C.c_void_p()
    _check(_lib.rs_protein_add_compress(ctx, arr, len(parts), int(tucker_cap), float(eps_r), _stream_ptr(stream),
                                        C.byref(out)))
    return out.value


def rs_ppiem_scan(ctx, prot, lig_xyz, lig_q, quats, n_theta: int, n_phi: int, x_P=None,
                  margin: float = 0.0, stream=None) -> dict:
    """Pose scan of Algorithm PPIEM: contact offsets, energies and flags of every
    (orbit direction, self-rotation) pair, the best rotation per direction and the
    local minima over the direction grid.  CUDA tensors in, CUDA tensors out (host
    arrays otherwise).  Keys: s, E, flags ([D, n_rot]); E_best, rot_best, t_best,
    is_min ([D])."""
    D = int(n_theta) * int(n_phi)
    if _is_cuda(quats):
        import torch
        dev = quats.device
        lx, lq = _dev(lig_xyz.to(dev), np.float64), _dev(lig_q.to(dev), np.float64)
        qu = _dev(quats, np.float64)
        xp = _dev(x_P.to(dev), np.float64) if x_P is not None else None
        f64 = lambda *sh: torch.empty(sh, dtype=torch.float64, device=dev)
        u8 = lambda *sh: torch.empty(sh, dtype=torch.uint8, device=dev)
        i32 = lambda *sh: torch.empty(sh, dtype=torch.int32, device=dev)
        mem, sp = RS_MEM_DEVICE, _stream_ptr(stream)
    else:
        lx, lq, qu = _host(lig_xyz, np.float64), _host(lig_q, np.float64), _host(quats, np.float64)
        xp = _host(x_P, np.float64) if x_P is not None else None
        f64 = lambda *sh: np.empty(sh)
        u8 = lambda *sh: np.empty(sh, dtype=np.uint8)
        i32 = lambda *sh: np.empty(sh, dtype=np.int32)
        mem, sp = RS_MEM_HOST, None
    L, R = int(lq.shape[0]), int(qu.shape[0])
    if tuple(lx.shape) != (L, 3) or tuple(qu.shape) != (R, 4):
        raise RSError(RS_ERR_INVALID, "shape mismatch in scan arguments")
    out = {"s": f64(D, R), "E": f64(D, R), "flags": u8(D, R), "E_best": f64(D), "rot_best": i32(D),
           "t_best": f64(D, 3), "is_min": u8(D)}
    _check(_lib.rs_ppiem_scan(ctx, prot, L, _ptr(lx), _ptr(lq), int(n_theta), int(n_phi), R, _ptr(qu),
                              _ptr(xp) if xp is not None else None, float(margin), _ptr(out["s"]),
                              _ptr(out["E"]), _ptr(out["flags"]), _ptr(out["E_best"]), _ptr(out["rot_best"]),
                              _ptr(out["t_best"]), _ptr(out["is_min"]), mem, sp))
    return out


def rs_energy_poses_noalloc(prot, lig_xyz, lig_q, quat, trans, E_out=None, flags_out=None,
                            stream=None):
    """rs_energy_poses for callers that must not trigger any device allocation
    during the call: every argument is a CUDA tensor on the protein's GPU, the
    library's scratch is a fixed array (ligands of at most 4096 atoms), and
    concurrent calls must not overlap on the GPU.  Returns (E, flags)."""
    import torch
    for x in (lig_xyz, lig_q, quat, trans):
        if not _is_cuda(x):
            raise RSError(RS_ERR_INVALID, "rs_energy_poses_noalloc takes CUDA tensors only")
    if len({x.device for x in (lig_xyz, lig_q, quat, trans)}) != 1:
        raise RSError(RS_ERR_INVALID, "rs_energy_poses_noalloc: tensors on different GPUs")
    lx, lq = _dev(lig_xyz, np.float64), _dev(lig_q, np.float64)
    r, t = _dev(quat, np.float64), _dev(trans, np.float64)
    P, L = int(r.shape[0]), int(lq.shape[0])
    if tuple(lx.shape) != (L, 3) or tuple(r.shape) != (P, 4) or tuple(t.shape) != (P, 3):
        raise RSError(RS_ERR_INVALID, "shape mismatch in pose arguments")
    E = E_out if E_out is not None else torch.empty(P, dtype=torch.float64, device=r.device)
    f = flags_out if flags_out is not None else torch.empty(P, dtype=torch.uint8, device=r.device)
    if E.device != r.device or f.device != r.device:
        raise RSError(RS_ERR_INVALID, "rs_energy_poses_noalloc: outputs on another device")
    _check(_lib.rs_energy_poses_noalloc(prot, L, _ptr(lx), _ptr(lq), P, _ptr(r), _ptr(t),
                                        _ptr(E), _ptr(f), _stream_ptr(stream)))
    return E, f


def rs_pgd_run(ctx: int, prot: int, lig_xyz, lig_q, rotvec, trans, nsteps: int,
               eta_t: float = 0.1, eta_r: float = 0.02, max_halvings: int = 5, stream=None):
    """Projected gradient descent of Eq. Energy_Min; rotvec and trans (CUDA float64
    tensors [P, 3]) are updated in place.  Returns (E, flags, accepted_level)."""
    import torch
    for x in (lig_xyz, lig_q, rotvec, trans):
        if not _is_cuda(x):
            raise RSError(RS_ERR_INVALID, "rs_pgd_run takes CUDA tensors")
    if rotvec.dtype != torch.float64 or trans.dtype != torch.float64 or not rotvec.is_contiguous() \
            or not trans.is_contiguous():
        raise RSError(RS_ERR_INVALID, "rotvec and trans must be contiguous float64 (updated in place)")
    lx, lq = _dev(lig_xyz, np.float64), _dev(lig_q, np.float64)
    P, L = int(rotvec.shape[0]), int(lq.shape[0])
    E = torch.empty(P, dtype=torch.float64, device=rotvec.device)
    f = torch.empty(P, dtype=torch.uint8, device=rotvec.device)
    acc = torch.empty(P, dtype=torch.int32, device=rotvec.device)
    _check(_lib.rs_pgd_run(ctx, prot, L, _ptr(lx), _ptr(lq), P, _ptr(rotvec), _ptr(trans), nsteps,
                           eta_t, eta_r, max_halvings, _ptr(E), _ptr(f), _ptr(acc),
                           _stream_ptr(stream)))
    return E, f, acc


def rs_batch_create(ctx: int, pairs: list, autotune: int | bool = True):
    """pairs: list of dicts with keys prot (handle), lig_xyz, lig_q, quat, trans, E_out,
    flags_out (CUDA tensors; outputs preallocated).  Returns (handle, keepalive)."""
    arr = (rs_pair * len(pairs))()
    keep = []
    for i, p in enumerate(pairs):
        lx, lq = _dev(p["lig_xyz"], np.float64), _dev(p["lig_q"], np.float64)
        qu, tr = _dev(p["quat"], np.float64), _dev(p["trans"], np.float64)
        keep += [lx, lq, qu, tr, p["E_out"], p.get("flags_out")]
        arr[i] = rs_pair(p["prot"], int(lq.shape[0]), _ptr(lx), _ptr(lq), int(qu.shape[0]),
                         _ptr(qu), _ptr(tr), _ptr(p["E_out"]),
                         _ptr(p["flags_out"]) if p.get("flags_out") is not None else None)
    h = C.c_void_p()
    _check(_lib.rs_batch_create(ctx, len(pairs), arr, int(autotune), C.byref(h)))
    return h.value, keep


def rs_batch_run(batch: int, stream=None) -> None:
    _check(_lib.rs_batch_run(batch, _stream_ptr(stream)))


def rs_batch_free(batch: int) -> None:
    _lib.rs_batch_free(batch)


def rs_batch_get_info(batch: int) -> dict:
    info = rs_batch_info()
    _check(_lib.rs_batch_get_info(batch, C.byref(info)))
    return {k: getattr(info, k) for k, _ in info._fields_}


def rs_symeig_host(A: np.ndarray):
    """Eigenvalues (descending) and eigenvectors (columns) of the symmetric part of A,
    by the library's host eigensolver."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    lam = np.empty(n)
    W = np.empty((n, n))
    _check(_lib.rs_symeig_host(n, A.ctypes.data, lam.ctypes.data, W.ctypes.data))
    return lam, W


def rs_qr_host(A: np.ndarray):
    """Thin QR (Q n x k, R k x k upper) of A by the library's host routine for
    add-and-compress; columns dependent on the previous ones give zero columns of Q."""
    A = np.asarray(A, dtype=np.float64)
    n, k = A.shape
    Qc = np.ascontiguousarray(A.T)  # column-major A: row j of Qc is column j
    R = np.empty((k, k))
    _check(_lib.rs_qr_host(n, k, Qc.ctypes.data, R.ctypes.data))
    return np.ascontiguousarray(Qc.T), R


def rs_set_wform_kernel(mode: int) -> int:
    """W-form kernel of the cell-grouped pose paths: 1 tensor cores (default), 0 float
    pairs on the FP32 pipes.  Returns the previous mode."""
    return int(_lib.rs_set_wform_kernel(int(mode)))


def rs_set_build_gemm_kernel(mode: int) -> int:
    """Block products G Q of the Tucker build: 1 tensor cores (default), 0 float pairs
    on the FP32 pipes.  Returns the previous mode."""
    return int(_lib.rs_set_build_gemm_kernel(int(mode)))


def rs_tc_error_count(device: int = 0) -> int:
    out = C.c_int32(0)
    _check(_lib.rs_tc_error_count(int(device), C.byref(out)))
    return int(out.value)


def rs_diag_short_counts(device: int = 0, grad: bool = False, reset: bool = False) -> dict:
    """Pose-atoms, candidates screened and near pairs of the cell-grouped atoms kernel
    since the last reset (energy or gradient launches)."""
    out = np.zeros(3, dtype=np.uint64)
    ops = C.c_double(0.0)
    _check(_lib.rs_diag_short_counts(int(device), int(bool(grad)), out.ctypes.data, C.byref(ops),
                                     int(bool(reset))))
    return {"atoms": int(out[0]), "candidates": int(out[1]), "near": int(out[2]), "fp32_ops": float(ops.value)}


def rs_diag_pair_exp(x: np.ndarray) -> np.ndarray:
    """exp(x) by the build's float-pair exponential on the GPU (|x| <= 80)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    _check(_lib.rs_diag_pair_exp(int(x.size), x.ctypes.data, out.ctypes.data))
    return out


def rs_diag_tc_launch() -> dict:
    """Launch shape of the latest tensor-core W-form launch: CTAs, shared memory per
    CTA and CTAs per SM."""
    g, m, p = C.c_int64(0), C.c_int64(0), C.c_int32(0)
    _check(_lib.rs_diag_tc_launch(C.byref(g), C.byref(m), C.byref(p)))
    return {"grid": int(g.value), "smem": int(m.value), "per_sm": int(p.value)}


def rs_diag_tc_contract(RP: int, v: np.ndarray, W: np.ndarray, D: np.ndarray):
    """X = v W^T and Xd = v D^T for one tile (rows <= 128) through the tensor-core
    slicing, MMAs and combination of the pose kernels."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    rows = v.shape[0]
    X = np.empty((rows, RP))
    Xd = np.empty((rows, RP))
    _check(_lib.rs_diag_tc_contract(int(RP), int(rows), v.ctypes.data, W.ctypes.data, D.ctypes.data,
                                    X.ctypes.data, Xd.ctypes.data))
    return X, Xd


def rs_stats_kernel_launches() -> int:
    return int(_lib.rs_stats_kernel_launches())


def rs_timing_enable(mode: int = 1) -> None:
    _check(_lib.rs_timing_enable(mode))


def rs_timing_reset() -> None:
    _check(_lib.rs_timing_reset())


def rs_timing_count() -> int:
    return int(_lib.rs_timing_count())


def rs_timing_get(index: int) -> dict:
    buf = C.create_string_buffer(128)
    ms, n, work = C.c_double(), C.c_ulonglong(), C.c_double()
    _check(_lib.rs_timing_get(index, buf, 128, C.byref(ms), C.byref(n), C.byref(work)))
    return {"name": buf.value.decode(), "ms": ms.value, "launches": int(n.value), "work": work.value}


def rs_timing_all() -> dict:
    """All timing records keyed by kernel name."""
    out = {}
    for i in range(rs_timing_count()):
        r = rs_timing_get(i)
        out[r["name"]] = r
    return out


# ------------------------------------------------------------------ serving
def rs_serve_params_default(**overrides) -> rs_serve_params:
    p = rs_serve_params()
    _lib.rs_serve_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def make_request(protein_id: int, prot_xyz, prot_q, params: rs_params, lig_xyz, lig_q, quat,
                 trans):
    """An rs_request over host arrays, plus the float64 arrays it points into (the
    caller keeps them alive until the request is finished)."""
    arrs = [_host(prot_xyz, np.float64), _host(prot_q, np.float64), _host(lig_xyz, np.float64),
            _host(lig_q, np.float64), _host(quat, np.float64), _host(trans, np.float64)]
    px, pq, lx, lq, qu, tr = arrs
    r = rs_request()
    r.protein_id = protein_id
    r.N = pq.shape[0]
    r.prot_xyz, r.prot_q = px.ctypes.data, pq.ctypes.data
    r.params = params
    r.L = lq.shape[0]
    r.lig_xyz, r.lig_q = lx.ctypes.data, lq.ctypes.data
    r.P = tr.shape[0]
    r.quat, r.trans = (qu.ctypes.data if r.P else None), (tr.ctypes.data if r.P else None)
    return r, arrs


def rs_request_validate(r: rs_request) -> int:
    return _lib.rs_request_validate(C.byref(r) if r is not None else None)


def rs_serve_create(device: int = 0, params: rs_serve_params | None = None) -> int:
    h = C.c_void_p()
    _check(_lib.rs_serve_create(device, C.byref(params) if params is not None else None,
                                C.byref(h)))
    return h.value


def rs_serve_submit(server: int, req: rs_request, E_out: np.ndarray, flags_out: np.ndarray | None):
    rid = C.c_uint64()
    _check(_lib.rs_serve_submit(server, C.byref(req), E_out.ctypes.data,
                                flags_out.ctypes.data if flags_out is not None else None,
                                C.byref(rid)))
    return rid.value


def _result_dict(r: rs_result) -> dict:
    return {"status": r.status, "t_submit_ns": r.t_submit_ns, "t_admit_ns": r.t_admit_ns,
            "t_start_ns": r.t_start_ns, "t_end_ns": r.t_end_ns, "message": r.message.decode()}


def rs_serve_poll(server: int, req_id: int):
    """None while pending, else the result record (its 'status' is the request's)."""
    r = rs_result()
    s = _lib.rs_serve_poll(server, req_id, C.byref(r))
    if s == RS_ERR_NOT_READY:
        return None
    _check(s)
    return _result_dict(r)


def rs_serve_wait(server: int, req_id: int, timeout_ms: int = 60000) -> dict:
    r = rs_result()
    _check(_lib.rs_serve_wait(server, req_id, timeout_ms, C.byref(r)))
    return _result_dict(r)


def rs_serve_cancel(server: int, req_id: int) -> int:
    return _lib.rs_serve_cancel(server, req_id)


def rs_serve_get_stats(server: int) -> dict:
    st = rs_serve_stats()
    _check(_lib.rs_serve_get_stats(server, C.byref(st)))
    return {k: getattr(st, k) for k, _ in rs_serve_stats._fields_}


def rs_serve_destroy(server: int) -> None:
    _lib.rs_serve_destroy(server)


class Server:
    """Owns an rs_server; keeps each request's host arrays alive until it finishes."""

    def __init__(self, device: int = 0, **params):
        self.handle = rs_serve_create(device, rs_serve_params_default(**params))
        self._keep = {}

    def submit(self, protein_id, prot_xyz, prot_q, params, lig_xyz, lig_q, quat, trans):
        req, arrs = make_request(protein_id, prot_xyz, prot_q, params, lig_xyz, lig_q, quat, trans)
        P = req.P
        E = np.empty(P, dtype=np.float64)
        f = np.empty(P, dtype=np.uint8)
        rid = rs_serve_submit(self.handle, req, E, f)
        self._keep[rid] = (arrs, E, f)
        return rid

    def _finish(self, rid, res):
        arrs, E, f = self._keep.pop(rid)
        res["E"], res["flags"] = E, f
        return res

    def poll(self, rid):
        res = rs_serve_poll(self.handle, rid)
        return None if res is None else self._finish(rid, res)

    def wait(self, rid, timeout_ms: int = 60000):
        return self._finish(rid, rs_serve_wait(self.handle, rid, timeout_ms))

    def cancel(self, rid) -> int:
        s = rs_serve_cancel(self.handle, rid)
        if s == RS_OK:
            self._keep.pop(rid, None)
        return s

    def release_builds(self):
        _check(_lib.rs_serve_release_builds(self.handle))

    def stats(self) -> dict:
        return rs_serve_get_stats(self.handle)

    def close(self):
        if self.handle:
            rs_serve_destroy(self.handle)
            self.handle = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ handle owners
class Context:
    """Owns an rs_ctx."""

    def __init__(self, device: int = 0):
        self.handle = rs_ctx_create(device)
        self.device = device

    def close(self):
        if self.handle:
            rs_ctx_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Protein:
    """Owns an rs_protein built by Algorithm TEP."""

    def __init__(self, ctx: Context, xyz, q, params: rs_params | None = None, stream=None, handle=None):
        self.ctx = ctx
        self.handle = handle if handle is not None else rs_build_protein(ctx.handle, xyz, q, params, stream)
        self.info = rs_protein_get_info(self.handle)

    def local_box(self, lo, hi, eps: float = 1e-7) -> "Protein":
        """A local-box handle (scheme C) on [lo, hi]; see rs_protein_local_box."""
        return Protein(self.ctx, None, None, handle=rs_protein_local_box(self.ctx.handle, self.handle, lo, hi, eps))

    @staticmethod
    def add_compress(ctx: Context, parts, tucker_cap: int, eps_r: float = 1e-7) -> "Protein":
        """The sum of the parts' potentials as one Tucker protein; see rs_protein_add_compress."""
        h = rs_protein_add_compress(ctx.handle, [p.handle for p in parts], tucker_cap, eps_r)
        return Protein(ctx, None, None, handle=h)

    def energies(self, lig_xyz, lig_q, quat, trans, **kw):
        return rs_energy_poses(self.ctx.handle, self.handle, lig_xyz, lig_q, quat, trans, **kw)

    def ppiem_scan(self, lig_xyz, lig_q, quats, n_theta, n_phi, **kw):
        return rs_ppiem_scan(self.ctx.handle, self.handle, lig_xyz, lig_q, quats, n_theta, n_phi, **kw)

    def fd_forces(self, lig_xyz, lig_q, rotvec, trans, **kw):
        return rs_fd_forces_poses(self.ctx.handle, self.handle, lig_xyz, lig_q, rotvec, trans, **kw)

    def energies_grad(self, lig_xyz, lig_q, rotvec, trans, **kw):
        return rs_energy_grad_poses(self.ctx.handle, self.handle, lig_xyz, lig_q, rotvec, trans, **kw)

    def close(self):
        if self.handle:
            rs_protein_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
