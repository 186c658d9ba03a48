"""ctypes binding of libgfopt (argument marshalling only; every step runs in the CUDA
library).  Function names mirror the C ABI in include/gfopt.h.  Device buffers are passed as
torch tensors (their data_ptr) or raw integer addresses; streams as torch.cuda.Stream or
integer cudaStream_t handles.

The library is loaded from the package's _lib directory on first use; if it has not been
built, every call raises GfError -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgfopt.so")

GF_OK, GF_EINVAL, GF_ECUDA, GF_ESINGULAR, GF_ENOIMPROVE, GF_ETIMEOUT, GF_ENOMEM = range(7)
GF_C128, GF_C64 = 0, 1
GF_KIND_SINGLE, GF_KIND_BRUSH2, GF_KIND_PILLAR = 0, 1, 2
GF_DIR_FILL, GF_DIR_CLEAR = 1, 2
GF_NBANDS = 9
GF_UPDATE_TC, GF_UPDATE_DFMA, GF_UPDATE_TENSOR = 0, 1, 2
GF_BATCH_STAGED, GF_BATCH_PERSISTENT = 0, 1
BATCH_MAX = 64             # items per gf_batch

STATUS_NAMES = {GF_OK: "GF_OK", GF_EINVAL: "GF_EINVAL", GF_ECUDA: "GF_ECUDA",
                GF_ESINGULAR: "GF_ESINGULAR", GF_ENOIMPROVE: "GF_ENOIMPROVE",
                GF_ETIMEOUT: "GF_ETIMEOUT", GF_ENOMEM: "GF_ENOMEM"}

EXPORTS = ["gf_create", "gf_destroy", "gf_last_error", "gf_status_string", "gf_version",
           "gf_num_candidates", "gf_workspace_size", "gf_fill_g0", "gf_extract_bands",
           "gf_eval_candidates", "gf_select_topk", "gf_apply_update", "gf_profile_begin",
           "gf_profile_end", "gf_set_update_algo", "gf_refresh", "gf_refresh_workspace_size",
           "gf_fill_g0_static", "gf_batch_table_size", "gf_batch_create", "gf_batch_step",
           "gf_batch_set_schedule", "gf_batch_set_form", "gf_batch_selftest_timeout", "gf_batch_destroy", "gf_select_egreedy", "gf_lowrank_workspace_size",
           "gf_lowrank_init", "gf_lowrank_eval", "gf_lowrank_update", "gf_lowrank_count",
           "gf_lowrank_materialize", "gf3_num_unknowns", "gf3_num_candidates", "gf3_workspace_size",
           "gf3_fill_g0", "gf3_eval_candidates", "gf3_select_topk", "gf3_apply_update", "gf_selftest_timeout", "gf_select_selftest_bytes", "gf_select_selftest_timeout",
           "gf_fom", "gf3_fom", "gf_lowrank_fom", "gf_refresh_field", "gf_shard_rows", "gf_shard_fill_g0",
           "gf_shard_eval", "gf_shard_gather_rows", "gf_shard_apply_update", "gf_shard_pack_halo",
           "gf_shard_unpack_halo"]


class GfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gf_geom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double),
                ("wavelength", C.c_double), ("eps_bg", C.c_double), ("eps_mat", C.c_double),
                ("mon_x", C.c_double), ("mon_y", C.c_double)]


class gf_problem(C.Structure):
    _fields_ = [("geom", gf_geom), ("G", C.c_void_p), ("ldg", C.c_int64), ("E", C.c_void_p),
                ("bands", C.c_void_p)]


class gf_cand_spec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dir_mask", C.c_int32), ("k", C.c_int32),
                ("excl_radius", C.c_int32), ("tie_rel", C.c_double), ("aligned", C.c_int32), ("pad", C.c_int32)]


class gf_geom3d(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("pad", C.c_int32), ("dx", C.c_double),
                ("wavelength", C.c_double), ("eps_bg", C.c_double), ("eps_mat", C.c_double),
                ("mon_x", C.c_double), ("mon_y", C.c_double), ("mon_z", C.c_double)]


class gf_problem3d(C.Structure):
    _fields_ = [("geom", gf_geom3d), ("G", C.c_void_p), ("ldg", C.c_int64), ("E", C.c_void_p)]


class gf_lowrank(C.Structure):
    _fields_ = [("geom", gf_geom), ("E", C.c_void_p), ("bands", C.c_void_p), ("monrow", C.c_void_p),
                ("U", C.c_void_p), ("max_cols", C.c_int32)]


class gf_shard(C.Structure):
    _fields_ = [("geom", gf_geom), ("y0", C.c_int32), ("y1", C.c_int32), ("G", C.c_void_p), ("ldg", C.c_int64),
                ("E", C.c_void_p), ("bands", C.c_void_p), ("mon", C.c_void_p)]


class gf_refresh_report(C.Structure):
    _fields_ = [("e_residual", C.c_double), ("e_residual_after", C.c_double), ("e_iters", C.c_int32),
                ("e_replaced", C.c_int32)]


class gf_batch_item(C.Structure):
    _fields_ = [("prob", gf_problem), ("state", C.c_void_p), ("dfom", C.c_void_p), ("idx", C.c_void_p),
                ("val", C.c_void_p), ("status", C.c_void_p), ("fom_out", C.c_void_p),
                ("applied", C.c_void_p), ("ws", C.c_void_p), ("ws_bytes", C.c_size_t),
                ("epsilon", C.c_double), ("uniforms", C.c_void_p), ("step", C.c_void_p), ("horizon", C.c_int32)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libgfopt.so (once) and declare the signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise GfError(GF_EINVAL, f"{path} is missing: build it with __graft_entry__.build() "
                                     "(there is no CPU fallback)")
        lib = C.CDLL(path)
        P = C.c_void_p
        sig = {
            "gf_create": (C.c_int32, [C.POINTER(P), C.c_int32]),
            "gf_destroy": (None, [P]),
            "gf_last_error": (C.c_char_p, [P]),
            "gf_status_string": (C.c_char_p, [C.c_int32]),
            "gf_version": (C.c_char_p, []),
            "gf_num_candidates": (C.c_int64, [C.POINTER(gf_geom), C.POINTER(gf_cand_spec)]),
            "gf_workspace_size": (C.c_size_t, [C.POINTER(gf_geom), C.c_int32, C.c_int32,
                                               C.POINTER(gf_cand_spec)]),
            "gf_fill_g0": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, P, C.c_size_t, P]),
            "gf_extract_bands": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, P]),
            "gf_fom": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, C.c_int32, P, P]),
            "gf3_fom": (C.c_int32, [P, C.POINTER(gf_problem3d), C.c_int32, P, P]),
            "gf_lowrank_fom": (C.c_int32, [P, C.POINTER(gf_lowrank), P, P]),
            "gf_eval_candidates": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, C.c_int32, P,
                                               C.POINTER(gf_cand_spec), P, P]),
            "gf_select_topk": (C.c_int32, [P, C.POINTER(gf_geom), C.POINTER(gf_cand_spec), P,
                                           C.c_int64, P, P, P, P, C.c_size_t, P]),
            "gf_apply_update": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, C.c_int32, P,
                                            C.POINTER(gf_cand_spec), P, P, P, P, P, C.c_size_t, P]),
            "gf_profile_begin": (C.c_int32, [P, C.c_int32]),
            "gf_set_update_algo": (C.c_int32, [P, C.c_int32]),
            "gf_fill_g0_static": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, P]),
            "gf_refresh_workspace_size": (C.c_size_t, [C.POINTER(gf_geom), C.c_int32]),
            "gf_refresh": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, P, C.c_int32,
                                       C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_double,
                                       C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_double), P,
                                       C.c_size_t, P]),
            "gf_refresh_field": (C.c_int32, [P, C.POINTER(gf_problem), C.c_int32, P, C.c_double, C.c_int32,
                                             C.c_int32, C.c_double, C.POINTER(gf_refresh_report), P, C.c_size_t,
                                             P]),
            "gf_profile_end": (C.c_int32, [P, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                           C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "gf_select_egreedy": (C.c_int32, [P, C.POINTER(gf_geom), C.POINTER(gf_cand_spec), P, C.c_int64,
                                              C.c_double, P, P, P, P, P, C.c_size_t, P]),
            "gf_selftest_timeout": (C.c_int32, [P, C.c_int64, P, P]),
            "gf_select_selftest_bytes": (C.c_size_t, []),
            "gf_select_selftest_timeout": (C.c_int32, [P, C.c_int64, P, C.c_size_t, P, P]),
            "gf3_num_unknowns": (C.c_int64, [C.POINTER(gf_geom3d)]),
            "gf3_num_candidates": (C.c_int64, [C.POINTER(gf_geom3d)]),
            "gf3_workspace_size": (C.c_size_t, [C.POINTER(gf_geom3d), C.c_int32, C.POINTER(gf_cand_spec)]),
            "gf3_fill_g0": (C.c_int32, [P, C.POINTER(gf_problem3d), C.c_int32, P, C.c_size_t, P]),
            "gf3_eval_candidates": (C.c_int32, [P, C.POINTER(gf_problem3d), C.c_int32, P, C.POINTER(gf_cand_spec), P, P]),
            "gf3_select_topk": (C.c_int32, [P, C.POINTER(gf_geom3d), C.POINTER(gf_cand_spec), P, C.c_int64, P, P, P, P,
                                            C.c_size_t, P]),
            "gf3_apply_update": (C.c_int32, [P, C.POINTER(gf_problem3d), C.c_int32, P, C.POINTER(gf_cand_spec), P, P, P,
                                             P, P, C.c_size_t, P]),
            "gf_lowrank_workspace_size": (C.c_size_t, [C.POINTER(gf_geom), C.c_int32]),
            "gf_lowrank_init": (C.c_int32, [P, C.POINTER(gf_lowrank), P, C.c_size_t, P]),
            "gf_lowrank_eval": (C.c_int32, [P, C.POINTER(gf_lowrank), P, C.POINTER(gf_cand_spec), P, P]),
            "gf_lowrank_update": (C.c_int32, [P, C.POINTER(gf_lowrank), P, C.POINTER(gf_cand_spec), P, P, P, P, P,
                                              C.c_size_t, P]),
            "gf_lowrank_count": (C.c_int32, [P, C.POINTER(gf_lowrank), P, C.c_size_t, C.POINTER(C.c_int32),
                                             C.POINTER(C.c_int32), P]),
            "gf_lowrank_materialize": (C.c_int32, [P, C.POINTER(gf_lowrank), P, C.c_int64, P, C.c_size_t, P]),
            "gf_shard_rows": (C.c_int64, [C.POINTER(gf_shard)]),
            "gf_shard_fill_g0": (C.c_int32, [P, C.POINTER(gf_shard), C.c_int32, P, C.c_size_t, P]),
            "gf_shard_eval": (C.c_int32, [P, C.POINTER(gf_shard), C.c_int32, P, C.POINTER(gf_cand_spec), P, P]),
            "gf_shard_gather_rows": (C.c_int32, [P, C.POINTER(gf_shard), C.c_int32, P, C.POINTER(gf_cand_spec), P, P,
                                                 P, C.c_int64, P]),
            "gf_shard_apply_update": (C.c_int32, [P, C.POINTER(gf_shard), C.c_int32, P, C.POINTER(gf_cand_spec), P, P,
                                                  C.c_int64, P, P, P, P, C.c_size_t, P]),
            "gf_shard_pack_halo": (C.c_int32, [P, C.POINTER(gf_shard), P, P]),
            "gf_shard_unpack_halo": (C.c_int32, [P, C.POINTER(gf_shard), P, P]),
            "gf_batch_table_size": (C.c_size_t, [C.c_int32]),
            "gf_batch_create": (C.c_int32, [P, C.c_int32, C.POINTER(gf_batch_item), C.c_int32,
                                            C.POINTER(gf_cand_spec), P, C.c_size_t, P, C.POINTER(P)]),
            "gf_batch_step": (C.c_int32, [P, P]),
            "gf_batch_set_schedule": (C.c_int32, [P, C.c_int32]),
            "gf_batch_set_form": (C.c_int32, [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
            "gf_batch_selftest_timeout": (C.c_int32, [P, C.c_int64, P]),
            "gf_batch_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def geom_struct(g) -> gf_geom:
    return gf_geom(int(g.nx), int(g.ny), float(g.dx), float(g.wavelength), float(g.eps_bg),
                   float(g.eps_mat), float(g.mon_x), float(g.mon_y))


def spec_struct(s) -> gf_cand_spec:
    return gf_cand_spec(int(s.kind), int(s.dir_mask), int(s.k), int(s.excl_radius), float(s.tie_rel),
                        int(getattr(s, "aligned", False)), 0)


def geom3d_struct(g) -> gf_geom3d:
    return gf_geom3d(int(g.nx), int(g.ny), int(g.nz), 0, float(g.dx), float(g.wavelength), float(g.eps_bg),
                     float(g.eps_mat), float(g.mon_x), float(g.mon_y), float(g.mon_z))


def problem3d_struct(g, G, ldg, E) -> gf_problem3d:
    return gf_problem3d(geom3d_struct(g), _ptr(G), int(ldg), _ptr(E))


def problem_struct(g, G, ldg, E, bands) -> gf_problem:
    return gf_problem(geom_struct(g), _ptr(G), int(ldg), _ptr(E), _ptr(bands))


class Handle:
    """Owns a gf_handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.gf_create(C.byref(h), int(device))
        if st != GF_OK:
            raise GfError(st, self.lib.gf_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != GF_OK:
            raise GfError(st, self.lib.gf_last_error(self.h).decode())

    # ---- ABI mirrors
    def gf_num_candidates(self, geom, spec) -> int:
        g, s = geom_struct(geom), spec_struct(spec)
        return int(self.lib.gf_num_candidates(C.byref(g), C.byref(s)))

    def gf_workspace_size(self, geom, nlam, dtype, spec) -> int:
        g, s = geom_struct(geom), spec_struct(spec)
        return int(self.lib.gf_workspace_size(C.byref(g), int(nlam), int(dtype), C.byref(s)))

    def gf_fill_g0(self, prob: gf_problem, dtype, ws, ws_bytes, stream=None):
        self._check(self.lib.gf_fill_g0(self.h, C.byref(prob), int(dtype), _ptr(ws), int(ws_bytes),
                                        _stream(stream)))

    def gf_fill_g0_static(self, prob: gf_problem, dtype, stream=None):
        """gf_fill_g0 with its table in the library's fixed device array (no workspace)."""
        self._check(self.lib.gf_fill_g0_static(self.h, C.byref(prob), int(dtype), _stream(stream)))

    def gf_extract_bands(self, prob: gf_problem, dtype, stream=None):
        self._check(self.lib.gf_extract_bands(self.h, C.byref(prob), int(dtype), _stream(stream)))

    def gf_fom(self, probs, dtype, fom_out, stream=None):
        arr = (gf_problem * len(probs))(*probs)
        self._check(self.lib.gf_fom(self.h, arr, len(probs), int(dtype), _ptr(fom_out), _stream(stream)))

    def gf_eval_candidates(self, probs, dtype, state, spec, dfom, stream=None):
        arr = (gf_problem * len(probs))(*probs)
        s = spec_struct(spec)
        self._check(self.lib.gf_eval_candidates(self.h, arr, len(probs), int(dtype), _ptr(state),
                                                C.byref(s), _ptr(dfom), _stream(stream)))

    def gf_select_topk(self, geom, spec, dfom, ncand, idx, val, status, ws, ws_bytes, stream=None):
        g, s = geom_struct(geom), spec_struct(spec)
        self._check(self.lib.gf_select_topk(self.h, C.byref(g), C.byref(s), _ptr(dfom), int(ncand),
                                            _ptr(idx), _ptr(val), _ptr(status), _ptr(ws),
                                            int(ws_bytes), _stream(stream)))

    def gf_select_egreedy(self, geom, spec, dfom, ncand, epsilon, u, idx, val, status, ws, ws_bytes, stream=None):
        g, s = geom_struct(geom), spec_struct(spec)
        self._check(self.lib.gf_select_egreedy(self.h, C.byref(g), C.byref(s), _ptr(dfom), int(ncand), float(epsilon),
                                               _ptr(u), _ptr(idx), _ptr(val), _ptr(status), _ptr(ws), int(ws_bytes),
                                               _stream(stream)))

    def gf_apply_update(self, probs, dtype, state, spec, idx, status, fom_out, ws, ws_bytes,
                        stream=None, applied=None):
        arr = (gf_problem * len(probs))(*probs)
        s = spec_struct(spec)
        self._check(self.lib.gf_apply_update(self.h, arr, len(probs), int(dtype), _ptr(state),
                                             C.byref(s), _ptr(idx), _ptr(status), _ptr(fom_out),
                                             _ptr(applied), _ptr(ws), int(ws_bytes), _stream(stream)))

    def gf_set_update_algo(self, algo: int):
        self._check(self.lib.gf_set_update_algo(self.h, int(algo)))

    def gf_refresh_workspace_size(self, geom, restart: int) -> int:
        g = geom_struct(geom)
        return int(self.lib.gf_refresh_workspace_size(C.byref(g), int(restart)))

    def gf_refresh(self, prob: gf_problem, dtype, state, cols, restart, max_iter, tol, ws, ws_bytes,
                   stream=None):
        """Returns (resid list of 1 + len(cols), GMRES iterations per column, each stored
        column's own Eq. 2 residual)."""
        ns = len(cols)
        ca = (C.c_int32 * max(ns, 1))(*cols)
        res = (C.c_double * (ns + 1))()
        its = (C.c_int32 * max(ns, 1))()
        cres = (C.c_double * max(ns, 1))()
        self._check(self.lib.gf_refresh(self.h, C.byref(prob), int(dtype), _ptr(state), ns, ca, int(restart),
                                        int(max_iter), float(tol), res, its, cres, _ptr(ws), int(ws_bytes),
                                        _stream(stream)))
        return list(res), list(its)[:ns], list(cres)[:ns]

    def gf_refresh_field(self, prob: gf_problem, dtype, state, e_tol, restart, max_iter, tol, ws, ws_bytes,
                         stream=None) -> dict:
        rep = gf_refresh_report()
        self._check(self.lib.gf_refresh_field(self.h, C.byref(prob), int(dtype), _ptr(state), float(e_tol),
                                              int(restart), int(max_iter), float(tol), C.byref(rep), _ptr(ws),
                                              int(ws_bytes), _stream(stream)))
        return {"e_residual": rep.e_residual, "e_residual_after": rep.e_residual_after, "e_iters": rep.e_iters,
                "e_replaced": bool(rep.e_replaced)}

    def gf_selftest_timeout(self, timeout_ns: int, status, stream=None):
        self._check(self.lib.gf_selftest_timeout(self.h, int(timeout_ns), _ptr(status), _stream(stream)))

    def gf_select_selftest_bytes(self) -> int:
        return int(self.lib.gf_select_selftest_bytes())

    def gf_select_selftest_timeout(self, timeout_ns: int, ws, ws_bytes: int, status, stream=None):
        self._check(self.lib.gf_select_selftest_timeout(self.h, int(timeout_ns), _ptr(ws), int(ws_bytes), _ptr(status),
                                                        _stream(stream)))

    # ---- 3-D form
    def gf3_num_unknowns(self, geom) -> int:
        g = geom3d_struct(geom)
        return int(self.lib.gf3_num_unknowns(C.byref(g)))

    def gf3_num_candidates(self, geom) -> int:
        g = geom3d_struct(geom)
        return int(self.lib.gf3_num_candidates(C.byref(g)))

    def gf3_workspace_size(self, geom, dtype, spec) -> int:
        g, s = geom3d_struct(geom), spec_struct(spec)
        return int(self.lib.gf3_workspace_size(C.byref(g), int(dtype), C.byref(s)))

    def gf3_fill_g0(self, prob: gf_problem3d, dtype, ws, ws_bytes, stream=None):
        self._check(self.lib.gf3_fill_g0(self.h, C.byref(prob), int(dtype), _ptr(ws), int(ws_bytes), _stream(stream)))

    def gf3_fom(self, prob: gf_problem3d, dtype, fom_out, stream=None):
        self._check(self.lib.gf3_fom(self.h, C.byref(prob), int(dtype), _ptr(fom_out), _stream(stream)))

    def gf3_eval_candidates(self, prob: gf_problem3d, dtype, state, spec, dfom, stream=None):
        s = spec_struct(spec)
        self._check(self.lib.gf3_eval_candidates(self.h, C.byref(prob), int(dtype), _ptr(state), C.byref(s), _ptr(dfom),
                                                 _stream(stream)))

    def gf3_select_topk(self, geom, spec, dfom, ncand, idx, val, status, ws, ws_bytes, stream=None):
        g, s = geom3d_struct(geom), spec_struct(spec)
        self._check(self.lib.gf3_select_topk(self.h, C.byref(g), C.byref(s), _ptr(dfom), int(ncand), _ptr(idx),
                                             _ptr(val), _ptr(status), _ptr(ws), int(ws_bytes), _stream(stream)))

    def gf3_apply_update(self, prob: gf_problem3d, dtype, state, spec, idx, status, fom_out, ws, ws_bytes,
                         stream=None, applied=None):
        s = spec_struct(spec)
        self._check(self.lib.gf3_apply_update(self.h, C.byref(prob), int(dtype), _ptr(state), C.byref(s), _ptr(idx),
                                              _ptr(status), _ptr(fom_out), _ptr(applied), _ptr(ws), int(ws_bytes),
                                              _stream(stream)))

    # ---- deferred (low-rank) form
    def gf_lowrank_workspace_size(self, geom, max_cols: int) -> int:
        g = geom_struct(geom)
        return int(self.lib.gf_lowrank_workspace_size(C.byref(g), int(max_cols)))

    def gf_lowrank_init(self, lr: gf_lowrank, ws, ws_bytes, stream=None):
        self._check(self.lib.gf_lowrank_init(self.h, C.byref(lr), _ptr(ws), int(ws_bytes), _stream(stream)))

    def gf_lowrank_fom(self, lr: gf_lowrank, fom_out, stream=None):
        self._check(self.lib.gf_lowrank_fom(self.h, C.byref(lr), _ptr(fom_out), _stream(stream)))

    def gf_lowrank_eval(self, lr: gf_lowrank, state, spec, dfom, stream=None):
        s = spec_struct(spec)
        self._check(self.lib.gf_lowrank_eval(self.h, C.byref(lr), _ptr(state), C.byref(s), _ptr(dfom),
                                             _stream(stream)))

    def gf_lowrank_update(self, lr: gf_lowrank, state, spec, idx, status, fom_out, ws, ws_bytes, stream=None,
                          applied=None):
        s = spec_struct(spec)
        self._check(self.lib.gf_lowrank_update(self.h, C.byref(lr), _ptr(state), C.byref(s), _ptr(idx),
                                               _ptr(status), _ptr(fom_out), _ptr(applied), _ptr(ws), int(ws_bytes),
                                               _stream(stream)))

    def gf_lowrank_count(self, lr: gf_lowrank, ws, ws_bytes, stream=None):
        nt, nc = C.c_int32(), C.c_int32()
        self._check(self.lib.gf_lowrank_count(self.h, C.byref(lr), _ptr(ws), int(ws_bytes), C.byref(nt), C.byref(nc),
                                              _stream(stream)))
        return nt.value, nc.value

    def gf_lowrank_materialize(self, lr: gf_lowrank, G, ldg, ws, ws_bytes, stream=None):
        self._check(self.lib.gf_lowrank_materialize(self.h, C.byref(lr), _ptr(G), int(ldg), _ptr(ws), int(ws_bytes),
                                                    _stream(stream)))

    # ---- row-block shards
    def gf_shard_rows(self, sh: gf_shard) -> int:
        return int(self.lib.gf_shard_rows(C.byref(sh)))

    def gf_shard_fill_g0(self, sh: gf_shard, dtype, ws, ws_bytes, stream=None):
        self._check(self.lib.gf_shard_fill_g0(self.h, C.byref(sh), int(dtype), _ptr(ws), int(ws_bytes), _stream(stream)))

    def gf_shard_eval(self, sh: gf_shard, dtype, state, spec, dfom, stream=None):
        s = spec_struct(spec)
        self._check(self.lib.gf_shard_eval(self.h, C.byref(sh), int(dtype), _ptr(state), C.byref(s), _ptr(dfom),
                                           _stream(stream)))

    def gf_shard_gather_rows(self, sh: gf_shard, dtype, state, spec, idx, status, panel, ldp, stream=None):
        s = spec_struct(spec)
        self._check(self.lib.gf_shard_gather_rows(self.h, C.byref(sh), int(dtype), _ptr(state), C.byref(s), _ptr(idx),
                                                  _ptr(status), _ptr(panel), int(ldp), _stream(stream)))

    def gf_shard_apply_update(self, sh: gf_shard, dtype, state, spec, idx, panel, ldp, status, fom_out, ws, ws_bytes,
                              stream=None, applied=None):
        s = spec_struct(spec)
        self._check(self.lib.gf_shard_apply_update(self.h, C.byref(sh), int(dtype), _ptr(state), C.byref(s), _ptr(idx),
                                                   _ptr(panel), int(ldp), _ptr(status), _ptr(fom_out), _ptr(applied),
                                                   _ptr(ws), int(ws_bytes), _stream(stream)))

    def gf_shard_pack_halo(self, sh: gf_shard, out, stream=None):
        self._check(self.lib.gf_shard_pack_halo(self.h, C.byref(sh), _ptr(out), _stream(stream)))

    def gf_shard_unpack_halo(self, sh: gf_shard, inp, stream=None):
        self._check(self.lib.gf_shard_unpack_halo(self.h, C.byref(sh), _ptr(inp), _stream(stream)))

    # ---- batches
    def gf_batch_table_size(self, nitems: int) -> int:
        return int(self.lib.gf_batch_table_size(int(nitems)))

    def gf_batch_create(self, items, dtype, spec, table, table_bytes, stream=None):
        """items: list of gf_batch_item.  Returns the gf_batch pointer (a c_void_p)."""
        arr = (gf_batch_item * len(items))(*items)
        s = spec_struct(spec)
        out = C.c_void_p()
        self._check(self.lib.gf_batch_create(self.h, len(items), arr, int(dtype), C.byref(s), _ptr(table),
                                             int(table_bytes), _stream(stream), C.byref(out)))
        return out

    def gf_batch_step(self, batch, stream=None):
        self._check(self.lib.gf_batch_step(batch, _stream(stream)))

    def gf_batch_set_schedule(self, batch, update_ctas: int):
        self._check(self.lib.gf_batch_set_schedule(batch, int(update_ctas)))

    def gf_batch_set_form(self, batch, form: int, step_ctas: int = 0, scale: int = 1, tile_rows: int = 32):
        self._check(self.lib.gf_batch_set_form(batch, int(form), int(step_ctas), int(scale), int(tile_rows)))

    def gf_batch_selftest_timeout(self, batch, timeout_ns: int, stream=None):
        self._check(self.lib.gf_batch_selftest_timeout(batch, int(timeout_ns), _stream(stream)))

    def gf_batch_destroy(self, batch):
        self.lib.gf_batch_destroy(batch)

    def gf_profile_begin(self, max_records: int):
        self._check(self.lib.gf_profile_begin(self.h, int(max_records)))

    def gf_profile_end(self):
        """Returns (ms_total, launches, bytes_total, flops_total) of the timed G updates."""
        ms, n, b, f = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
        self._check(self.lib.gf_profile_end(self.h, C.byref(ms), C.byref(n), C.byref(b), C.byref(f)))
        return ms.value, n.value, b.value, f.value
