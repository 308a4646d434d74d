"""ctypes binding of libbf.so (include/bf.h).  Argument marshalling only.

Every step of the solver runs in the CUDA library; this module only converts numpy
arrays / torch tensors to pointers and the C structs to Python values.  If the
library is missing the import fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes
import pathlib

import numpy as np

_PKG = pathlib.Path(__file__).resolve().parent
LIB_PATH = _PKG / "libbf.so"

BF_OK = 0
BF_PTR_HOST, BF_PTR_DEVICE = 0, 1
BF_STORE_FP32, BF_STORE_BF16, BF_STORE_FP16 = 0, 1, 2
BF_PRECOND_BLOCK_JACOBI, BF_PRECOND_JACOBI = 0, 1
BF_PREC_MIXED, BF_PREC_FP32 = 0, 1
BF_FLAG_SINGULAR_BLOCK, BF_FLAG_EMPTY_FRAME, BF_FLAG_PCG_BREAKDOWN = 1, 2, 4
BF_PCG_AUTO, BF_PCG_CTA, BF_PCG_GRID, BF_PCG_CLUSTER = 0, 1, 2, 3
BF_SPARSE_BLOCKS, BF_SPARSE_MATFREE = 0, 1
BF_MAX_GN = 64
BF_MAX_PRUNE = 32
BF_TILE_AUTOTUNE = -1
BF_NPROF = 14
KERNEL_CLASSES = ["preprocess", "xform", "dense", "sparse", "merge", "assemble", "pcg", "update", "energy", "pack",
                  "verify", "keypoint", "tsdf", "batch"]

STATUS = {0: "BF_OK", 1: "BF_ERR_INVALID_ARG", 2: "BF_ERR_OUT_OF_MEMORY", 3: "BF_ERR_CUDA",
          4: "BF_ERR_NOT_FOUND", 5: "BF_ERR_SINGULAR", 6: "BF_ERR_TIMEOUT", 7: "BF_ERR_BUSY"}


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("depth_min", ctypes.c_float), ("depth_max", ctypes.c_float), ("storage", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("cuda_stream", ctypes.c_void_p),
                ("max_frames_hint", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("n_gn", ctypes.c_int), ("n_pcg", ctypes.c_int),
                ("w_sparse", ctypes.c_double), ("w_dense", ctypes.c_double), ("w_photo", ctypes.c_double),
                ("w_geo", ctypes.c_double), ("dense_ramp", ctypes.c_int), ("tau_dist", ctypes.c_double),
                ("tau_normal", ctypes.c_double), ("max_angle_deg", ctypes.c_double), ("precond", ctypes.c_int),
                ("dense_on", ctypes.c_int), ("warm_start", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("tile_px", ctypes.c_int), ("pcg_variant", ctypes.c_int),
                ("prune_rmax", ctypes.c_double), ("prune_rounds", ctypes.c_int),
                ("sparse_mode", ctypes.c_int), ("persistent", ctypes.c_int), ("compensated", ctypes.c_int),
                ("dense_tc", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("n_gn_done", ctypes.c_int),
                ("energy", ctypes.c_double * (BF_MAX_GN + 1)), ("e_sparse", ctypes.c_double * (BF_MAX_GN + 1)),
                ("e_photo", ctypes.c_double * (BF_MAX_GN + 1)), ("e_geo", ctypes.c_double * (BF_MAX_GN + 1)),
                ("n_dense_valid", ctypes.c_longlong * (BF_MAX_GN + 1)),
                ("r_max", ctypes.c_double), ("r_max_pair", ctypes.c_int * 2),
                ("n_frames", ctypes.c_int), ("n_pairs", ctypes.c_int), ("n_dense_pairs", ctypes.c_int),
                ("n_corr", ctypes.c_longlong), ("flags", ctypes.c_int), ("ms", ctypes.c_double),
                ("solves", ctypes.c_int), ("n_pruned", ctypes.c_int),
                ("pruned_pairs", ctypes.c_int * (2 * BF_MAX_PRUNE)), ("n_invalid", ctypes.c_int),
                ("invalid_frames", ctypes.c_int * BF_MAX_PRUNE)]

    def to_dict(self):
        k = self.n_gn_done + 1
        npr = min(self.n_pruned, BF_MAX_PRUNE)
        return dict(n_gn=self.n_gn_done, energy=list(self.energy[:k]), e_sparse=list(self.e_sparse[:k]),
                    e_photo=list(self.e_photo[:k]), e_geo=list(self.e_geo[:k]),
                    n_dense=list(self.n_dense_valid[:k]), r_max=self.r_max, r_max_pair=tuple(self.r_max_pair),
                    n_frames=self.n_frames, n_pairs=self.n_pairs, n_dense_pairs=self.n_dense_pairs,
                    n_corr=self.n_corr, flags=self.flags, ms=self.ms, solves=self.solves,
                    n_pruned=self.n_pruned,
                    pruned=[(self.pruned_pairs[2 * i], self.pruned_pairs[2 * i + 1]) for i in range(npr)],
                    n_invalid=self.n_invalid,
                    invalid=list(self.invalid_frames[:min(self.n_invalid, BF_MAX_PRUNE)]))


class VerifyParams(ctypes.Structure):
    _fields_ = [("tau_dist", ctypes.c_double), ("tau_normal", ctypes.c_double), ("tau_color", ctypes.c_double),
                ("max_err", ctypes.c_double), ("min_valid_frac", ctypes.c_double)]


class VerifyResult(ctypes.Structure):
    _fields_ = [("n_ij", ctypes.c_int), ("n_ji", ctypes.c_int), ("err_ij", ctypes.c_double),
                ("err_ji", ctypes.c_double), ("mean_err", ctypes.c_double), ("valid", ctypes.c_int)]

    def to_dict(self):
        return dict(n_ij=self.n_ij, n_ji=self.n_ji, err_ij=self.err_ij, err_ji=self.err_ji, mean_err=self.mean_err,
                    valid=bool(self.valid))


class KeypointParams(ctypes.Structure):
    _fields_ = [("max_residual", ctypes.c_double), ("max_cond", ctypes.c_double), ("min_area", ctypes.c_double),
                ("min_matches", ctypes.c_int)]


class TsdfConfig(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_double), ("trunc_voxels", ctypes.c_int), ("table_log2", ctypes.c_int),
                ("max_blocks", ctypes.c_int)]


BF_REQ_LOCAL, BF_REQ_GLOBAL = 0, 1


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("chunk_id", ctypes.c_int), ("frame_ids", ctypes.c_void_p),
                ("n", ctypes.c_int), ("params", SolveParams)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("count", ctypes.c_longlong * BF_NPROF),
                ("ms", ctypes.c_double * BF_NPROF)]

    def to_dict(self):
        return dict(launches=self.launches,
                    kernels={k: dict(count=self.count[i], ms=self.ms[i]) for i, k in enumerate(KERNEL_CLASSES)})


_lib = None


def lib():
    """Load libbf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1604_01093_b300.build.build()")
    L = ctypes.CDLL(str(LIB_PATH))
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "bf_default_config": (None, [ctypes.POINTER(Config)]),
        "bf_default_params": (None, [ctypes.POINTER(SolveParams)]),
        "bf_status_string": (ctypes.c_char_p, [I]),
        "bf_create": (I, [ctypes.POINTER(Config), ctypes.POINTER(P)]),
        "bf_destroy": (I, [P]),
        "bf_last_error": (ctypes.c_char_p, [P]),
        "bf_add_frames": (I, [P, I, I, P, P, I, P]),
        "bf_add_correspondences": (I, [P, I, I, I, P, P, P, I]),
        "bf_add_correspondences_batch": (I, [P, I, P, P, P, P, P, I]),
        "bf_remove_pair": (I, [P, I, I]),
        "bf_clear_correspondences": (I, [P]),
        "bf_solve_local": (I, [P, I, P, I, ctypes.POINTER(SolveParams), P]),
        "bf_solve_local_batch": (I, [P, I, P, P, P, ctypes.POINTER(SolveParams), P]),
        "bf_solve_global": (I, [P, P, I, ctypes.POINTER(SolveParams), P]),
        "bf_get_poses": (I, [P, P, I, P]),
        "bf_build_system": (I, [P, P, I, P, ctypes.POINTER(SolveParams), P, P, P, P]),
        "bf_get_frame_planes": (I, [P, I, P]),
        "bf_debug_association": (I, [P, I, I, P, P, ctypes.POINTER(SolveParams), P]),
        "bf_debug_record_association": (I, [P, I]),
        "bf_debug_recorded_association": (I, [P, I, I, I, P, P, P]),
        "bf_debug_tc_probe": (I, [I, I, P, P, P]),
        "bf_device_bytes": (ctypes.c_size_t, [P]),
        "bf_set_profiling": (I, [P, I]),
        "bf_get_profile": (I, [P, ctypes.POINTER(Profile)]),
        "bf_reset_profile": (I, [P]),
        "bf_serve_start": (I, [P, I, I, I]),
        "bf_serve_stop": (I, [P]),
        "bf_submit": (I, [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "bf_wait": (I, [P, ctypes.c_uint64, I, P]),
        "bf_dense_pair_noalloc": (I, [I, I, D, D, D, D, ctypes.c_float, ctypes.c_float, P, P, P, P, P, P,
                                      ctypes.POINTER(SolveParams), P, P]),
        "bf_default_verify_params": (None, [ctypes.POINTER(VerifyParams)]),
        "bf_selftest_wait_timeout": (I, [P, I, ctypes.c_longlong, P]),
        "bf_tuned_tile_px": (I, [P, P]),
        "bf_default_tsdf_config": (None, [ctypes.POINTER(TsdfConfig)]),
        "bf_tsdf_init": (I, [P, ctypes.POINTER(TsdfConfig)]),
        "bf_tsdf_integrate": (I, [P, I, P]),
        "bf_tsdf_deintegrate": (I, [P, I]),
        "bf_tsdf_reintegrate": (I, [P, I, P, P]),
        "bf_tsdf_export": (I, [P, ctypes.c_longlong, P, P, P]),
        "bf_default_keypoint_params": (None, [ctypes.POINTER(KeypointParams)]),
        "bf_filter_keypoints": (I, [P, I, P, P, P, ctypes.POINTER(KeypointParams), P, P, P]),
        "bf_verify_pairs": (I, [P, I, P, P, ctypes.POINTER(VerifyParams), P]),
        "bf_validate_chunk": (I, [P, I, D, ctypes.POINTER(VerifyParams), P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# symbols declared in include/bf.h (checked by the CPU tests)
EXPORTS = ["bf_default_config", "bf_default_params", "bf_status_string", "bf_create", "bf_destroy",
           "bf_last_error", "bf_add_frames", "bf_add_correspondences", "bf_add_correspondences_batch",
           "bf_remove_pair", "bf_set_profiling", "bf_get_profile", "bf_reset_profile",
           "bf_clear_correspondences", "bf_solve_local", "bf_solve_local_batch", "bf_solve_global",
           "bf_get_poses", "bf_build_system", "bf_get_frame_planes", "bf_debug_association",
           "bf_debug_record_association", "bf_debug_recorded_association", "bf_debug_tc_probe", "bf_device_bytes",
           "bf_dense_pair_noalloc", "bf_serve_start", "bf_serve_stop", "bf_submit", "bf_wait",
           "bf_default_verify_params", "bf_verify_pairs", "bf_validate_chunk", "bf_default_keypoint_params",
           "bf_filter_keypoints", "bf_selftest_wait_timeout", "bf_default_tsdf_config", "bf_tsdf_init",
           "bf_tsdf_integrate", "bf_tsdf_deintegrate", "bf_tsdf_reintegrate", "bf_tsdf_export", "bf_tuned_tile_px"]


class BFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a):
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _f32(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float32)
    import torch
    return a.to(torch.float32).contiguous()


def default_params(**kw) -> SolveParams:
    p = SolveParams()
    lib().bf_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"unknown solve parameter {k}")
        setattr(p, k, v)
    return p


def verify_params(**kw) -> VerifyParams:
    p = VerifyParams()
    lib().bf_default_verify_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"unknown verification parameter {k}")
        setattr(p, k, v)
    return p


class Context:
    """One library context (one frame size, one device, one stream)."""

    def __init__(self, width=80, height=60, fx=None, fy=None, cx=None, cy=None, device=0, depth_min=0.1,
                 depth_max=10.0, storage=BF_STORE_FP32, hbm_budget_bytes=0, stream=None, max_frames_hint=64):
        L = lib()
        cfg = Config()
        L.bf_default_config(ctypes.byref(cfg))
        s = width / 640.0
        cfg.device, cfg.width, cfg.height = device, width, height
        cfg.fx = 525.0 * s if fx is None else fx
        cfg.fy = 525.0 * s if fy is None else fy
        cfg.cx = (width - 1) / 2.0 if cx is None else cx
        cfg.cy = (height - 1) / 2.0 if cy is None else cy
        cfg.depth_min, cfg.depth_max, cfg.storage = depth_min, depth_max, storage
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.cuda_stream = stream
        cfg.max_frames_hint = max_frames_hint
        h = ctypes.c_void_p()
        st = L.bf_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != BF_OK:
            raise BFError(st, "bf_create failed")
        self.h = h
        self.cfg = cfg
        self.W, self.H = width, height

    def close(self):
        if self.h:
            lib().bf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != BF_OK:
            raise BFError(st, lib().bf_last_error(self.h).decode())

    # ---------------------------------------------------------------- inputs
    def add_frames(self, first_id, depth, lum, init_pose=None):
        depth, lum = _f32(depth), _f32(lum)
        n = depth.shape[0]
        kind = BF_PTR_DEVICE if _is_device(depth) else BF_PTR_HOST
        init = None if init_pose is None else np.ascontiguousarray(init_pose, dtype=np.float64).reshape(n, 16)
        self._check(lib().bf_add_frames(self.h, first_id, n, _ptr(depth), _ptr(lum), kind, _ptr(init)))

    def add_correspondences(self, i, j, p_i, p_j, weight=None):
        p_i, p_j = _f32(p_i), _f32(p_j)
        w = None if weight is None else _f32(weight)
        kind = BF_PTR_DEVICE if _is_device(p_i) else BF_PTR_HOST
        self._check(lib().bf_add_correspondences(self.h, i, j, p_i.shape[0], _ptr(p_i), _ptr(p_j), _ptr(w), kind))

    def add_correspondences_batch(self, pair_ids, offsets, p_i, p_j, weight=None):
        """All pairs at once: pair_ids (P,2), offsets (P+1,), p_i/p_j (C,3) host arrays or device tensors."""
        ids = np.ascontiguousarray(pair_ids, dtype=np.int32).reshape(-1, 2)
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        p_i, p_j = _f32(p_i), _f32(p_j)
        w = None if weight is None else _f32(weight)
        kind = BF_PTR_DEVICE if _is_device(p_i) else BF_PTR_HOST
        self._check(lib().bf_add_correspondences_batch(self.h, ids.shape[0], _ptr(ids), _ptr(off), _ptr(p_i),
                                                       _ptr(p_j), _ptr(w), kind))

    def set_profiling(self, on=True):
        self._check(lib().bf_set_profiling(self.h, 1 if on else 0))

    def reset_profile(self):
        self._check(lib().bf_reset_profile(self.h))

    def profile(self):
        p = Profile()
        self._check(lib().bf_get_profile(self.h, ctypes.byref(p)))
        return p.to_dict()

    def remove_pair(self, i, j):
        self._check(lib().bf_remove_pair(self.h, i, j))

    def clear_correspondences(self):
        self._check(lib().bf_clear_correspondences(self.h))

    # ---------------------------------------------------------------- solves
    def solve_local(self, chunk_id, frame_ids, params=None, **kw):
        p = params or default_params(**kw)
        ids = np.ascontiguousarray(frame_ids, dtype=np.int32)
        st = SolveStats()
        self._check(lib().bf_solve_local(self.h, chunk_id, _ptr(ids), len(ids), ctypes.byref(p), ctypes.byref(st)))
        return st.to_dict()

    def solve_local_batch(self, chunk_ids, frame_lists, params=None, **kw):
        p = params or default_params(**kw)
        cids = np.ascontiguousarray(chunk_ids, dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.int32) for f in frame_lists]))
        off = np.zeros(len(frame_lists) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(f) for f in frame_lists])
        stats = (SolveStats * len(frame_lists))()
        self._check(lib().bf_solve_local_batch(self.h, len(cids), _ptr(cids), _ptr(flat), _ptr(off), ctypes.byref(p),
                                               ctypes.cast(stats, ctypes.c_void_p)))
        return [s.to_dict() for s in stats]

    def solve_global(self, keyframe_ids, params=None, **kw):
        p = params or default_params(**kw)
        ids = np.ascontiguousarray(keyframe_ids, dtype=np.int32)
        st = SolveStats()
        self._check(lib().bf_solve_global(self.h, _ptr(ids), len(ids), ctypes.byref(p), ctypes.byref(st)))
        return st.to_dict()

    def get_poses(self, frame_ids):
        ids = np.ascontiguousarray(frame_ids, dtype=np.int32)
        out = np.zeros((len(ids), 4, 4), dtype=np.float64)
        self._check(lib().bf_get_poses(self.h, _ptr(ids), len(ids), _ptr(out)))
        return out

    # ------------------------------------------------------------------ TSDF
    def tsdf_init(self, **kw):
        cfg = TsdfConfig()
        lib().bf_default_tsdf_config(ctypes.byref(cfg))
        for k, v in kw.items():
            if not hasattr(cfg, k):
                raise AttributeError(f"unknown TSDF setting {k}")
            setattr(cfg, k, v)
        self._check(lib().bf_tsdf_init(self.h, ctypes.byref(cfg)))

    def tsdf_integrate(self, frame_id, pose=None):
        T = None if pose is None else np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        self._check(lib().bf_tsdf_integrate(self.h, frame_id, None if T is None else _ptr(T)))

    def tsdf_deintegrate(self, frame_id):
        self._check(lib().bf_tsdf_deintegrate(self.h, frame_id))

    def tsdf_reintegrate(self, n_fix=10):
        ids = np.zeros(max(n_fix, 1), dtype=np.int32)
        n = ctypes.c_int(0)
        self._check(lib().bf_tsdf_reintegrate(self.h, n_fix, _ptr(ids), ctypes.byref(n)))
        return ids[:n.value].tolist()

    def tsdf_export(self):
        """{(bx, by, bz): int64 array (3, 512) of S, W, SC}."""
        n = ctypes.c_longlong(0)
        self._check(lib().bf_tsdf_export(self.h, 0, None, None, ctypes.byref(n)))
        cap = n.value
        coords = np.zeros((max(cap, 1), 3), dtype=np.int32)
        sums = np.zeros((max(cap, 1), 3, 512), dtype=np.int32)
        self._check(lib().bf_tsdf_export(self.h, cap, _ptr(coords), _ptr(sums), ctypes.byref(n)))
        return {tuple(map(int, coords[k])): sums[k].astype(np.int64) for k in range(cap)}

    def tuned_tile_px(self):
        """The autotuner's choice for this context (0 = staged target frame), or None."""
        v = ctypes.c_int(0)
        st = lib().bf_tuned_tile_px(self.h, ctypes.byref(v))
        return v.value if st == 0 else None

    # ------------------------------------------------------ failure detection
    def selftest_wait_timeout(self, which, limit=1 << 16):
        """Make one bounded device wait run out (0: a word nothing changes, 1: an mbarrier nothing
        arrives on, 2: a work-queue slot nothing publishes); returns (status, gave_up)."""
        flag = ctypes.c_int(0)
        st = lib().bf_selftest_wait_timeout(self.h, which, limit, ctypes.byref(flag))
        return st, flag.value

    # ------------------------------------------------------ key-point filter
    def filter_keypoints(self, offsets, p_i, p_j, **kw):
        """Sec. 4.1.1 key-point and surface-area filters for a batch of pairs.  Returns
        (keep mask over all matches, per-pair 4x4 transforms, per-pair status)."""
        kp = KeypointParams()
        lib().bf_default_keypoint_params(ctypes.byref(kp))
        for k, v in kw.items():
            if not hasattr(kp, k):
                raise AttributeError(f"unknown key-point parameter {k}")
            setattr(kp, k, v)
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        n_pairs = len(off) - 1
        P = np.ascontiguousarray(p_i, dtype=np.float32).reshape(-1, 3)
        Q = np.ascontiguousarray(p_j, dtype=np.float32).reshape(-1, 3)
        keep = np.zeros(max(int(off[-1]), 1), dtype=np.uint8)
        T = np.zeros((max(n_pairs, 1), 4, 4))
        status = np.zeros(max(n_pairs, 1), dtype=np.int32)
        self._check(lib().bf_filter_keypoints(self.h, n_pairs, _ptr(off), _ptr(P), _ptr(Q), ctypes.byref(kp),
                                              _ptr(keep), _ptr(T), _ptr(status)))
        return keep[:int(off[-1])].astype(bool), T[:n_pairs], status[:n_pairs]

    # ---------------------------------------------------- dense verification
    def verify_pairs(self, frame_pairs, rel, **kw):
        """Sec. 4.1.1 two-sided check of frame pairs (k, 2) under relative transforms (k, 4, 4)."""
        vp = verify_params(**kw)
        fp = np.ascontiguousarray(frame_pairs, dtype=np.int32).reshape(-1, 2)
        T = np.ascontiguousarray(rel, dtype=np.float64).reshape(len(fp), 16)
        out = (VerifyResult * max(len(fp), 1))()
        self._check(lib().bf_verify_pairs(self.h, len(fp), _ptr(fp), _ptr(T), ctypes.byref(vp),
                                          ctypes.cast(out, ctypes.c_void_p)))
        return [out[k].to_dict() for k in range(len(fp))]

    def validate_chunk(self, chunk_id, max_err=0.05, **kw):
        """Sec. 4.2 chunk validation at the chunk's solved local poses."""
        vp = verify_params(**kw)
        valid = ctypes.c_int(0)
        worst = ctypes.c_double(0.0)
        pair = (ctypes.c_int * 2)()
        self._check(lib().bf_validate_chunk(self.h, chunk_id, max_err, ctypes.byref(vp), ctypes.byref(valid),
                                            ctypes.byref(worst), ctypes.cast(pair, ctypes.c_void_p)))
        return dict(valid=bool(valid.value), worst_err=worst.value, worst_pair=(pair[0], pair[1]))

    # ------------------------------------------------------------ inspection
    def build_system(self, frame_ids, poses, params=None, **kw):
        p = params or default_params(**kw)
        ids = np.ascontiguousarray(frame_ids, dtype=np.int32)
        n = len(ids)
        P = np.ascontiguousarray(poses, dtype=np.float64).reshape(n, 16)
        m = 6 * (n - 1)
        A = np.zeros((m, m))
        b = np.zeros(m)
        e4 = np.zeros(4)
        nd = ctypes.c_longlong()
        self._check(lib().bf_build_system(self.h, _ptr(ids), n, _ptr(P), ctypes.byref(p), _ptr(A), _ptr(b), _ptr(e4),
                                          ctypes.byref(nd)))
        return dict(A=A, b=b, energy=e4[0], e_sparse=e4[1], e_photo=e4[2], e_geo=e4[3], n_dense=nd.value)

    def frame_planes(self, frame_id):
        out = np.zeros((7, self.H, self.W), dtype=np.float32)
        self._check(lib().bf_get_frame_planes(self.h, frame_id, _ptr(out)))
        return out

    def association(self, i, j, pose_i, pose_j, params=None, **kw):
        p = params or default_params(**kw)
        out = np.zeros(self.W * self.H, dtype=np.int32)
        pi = np.ascontiguousarray(pose_i, dtype=np.float64).reshape(16)
        pj = np.ascontiguousarray(pose_j, dtype=np.float64).reshape(16)
        self._check(lib().bf_debug_association(self.h, i, j, _ptr(pi), _ptr(pj), ctypes.byref(p), _ptr(out)))
        return out

    def record_association(self, on=True):
        """Debug: record the association of every dense evaluation of the next single-problem solves."""
        self._check(lib().bf_debug_record_association(self.h, 1 if on else 0))

    def recorded_association(self, evaluation, i, j):
        """(targets (H*W int32), pose_i (4x4), pose_j (4x4)) of directed pair i -> j at a recorded
        dense evaluation of the last recorded solve."""
        out = np.zeros(self.W * self.H, dtype=np.int32)
        pi = np.zeros(16)
        pj = np.zeros(16)
        self._check(lib().bf_debug_recorded_association(self.h, evaluation, i, j, _ptr(out), _ptr(pi), _ptr(pj)))
        return out, pi.reshape(4, 4), pj.reshape(4, 4)

    # --------------------------------------------------------------- serving
    def serve_start(self, n_slots=2, max_batch=64, max_queue=1024):
        self._check(lib().bf_serve_start(self.h, n_slots, max_batch, max_queue))

    def serve_stop(self):
        self._check(lib().bf_serve_stop(self.h))

    def submit(self, frame_ids, kind=BF_REQ_LOCAL, chunk_id=0, params=None, **kw):
        """Queue a request; returns its ticket (raises BFError with BF_ERR_BUSY if the queue is full)."""
        ids = np.ascontiguousarray(frame_ids, dtype=np.int32)
        r = Request()
        r.kind, r.chunk_id, r.frame_ids, r.n = kind, chunk_id, ids.ctypes.data, len(ids)
        r.params = params or default_params(**kw)
        t = ctypes.c_uint64()
        st = lib().bf_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if st != BF_OK:
            raise BFError(st, "bf_submit failed")
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """(status, stats dict or None): status BF_ERR_TIMEOUT (6) if not done within timeout_ms."""
        st = SolveStats()
        code = lib().bf_wait(self.h, ticket, timeout_ms, ctypes.byref(st))
        return code, (st.to_dict() if code in (BF_OK,) else (st.to_dict() if code not in (4, 6) else None))

    def device_bytes(self):
        return lib().bf_device_bytes(self.h)


def dense_pair_noalloc(depth_i, lum_i, depth_j, lum_j, pose_i, pose_j, out, width, height, fx, fy, cx, cy,
                       depth_min=0.1, depth_max=10.0, stream=None, params=None, **kw):
    """bf_dense_pair_noalloc: device tensors in, 124 doubles into the device tensor out.

    For callers that cannot allocate device memory at the point of use; see include/bf.h."""
    p = params or default_params(**kw)
    pi = np.ascontiguousarray(pose_i, dtype=np.float64).reshape(16)
    pj = np.ascontiguousarray(pose_j, dtype=np.float64).reshape(16)
    st = lib().bf_dense_pair_noalloc(width, height, fx, fy, cx, cy, depth_min, depth_max, _ptr(depth_i), _ptr(lum_i),
                                     _ptr(depth_j), _ptr(lum_j), _ptr(pi), _ptr(pj), ctypes.byref(p), _ptr(out),
                                     stream)
    if st != BF_OK:
        raise BFError(st, "bf_dense_pair_noalloc failed")


def tc_probe(fa, fb, passes=3):
    """bf_debug_tc_probe: fa, fb host arrays (8, n_rows, 8); returns the (128, 64) accumulator."""
    fa = np.ascontiguousarray(fa, dtype=np.float32)
    fb = np.ascontiguousarray(fb, dtype=np.float32)
    if fa.shape != fb.shape or fa.ndim != 3 or fa.shape[0] != 8 or fa.shape[2] != 8:
        raise ValueError("fa and fb must both be (8, n_rows, 8)")
    out = np.zeros((128, 64), np.float32)
    st = lib().bf_debug_tc_probe(fa.shape[1], passes, _ptr(fa), _ptr(fb), _ptr(out))
    if st != BF_OK:
        raise BFError(st, "bf_debug_tc_probe failed")
    return out
