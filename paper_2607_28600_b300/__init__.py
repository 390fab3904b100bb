"""B300-native SymFT per-shot sampling engine: thin Python binding of libsymft.so.

Every step of the sampler runs in the library (C++ compile step, CUDA kernels);
this module only marshals arguments through ctypes.  Device buffers are passed
as raw pointers (``torch.Tensor.data_ptr()``), host buffers as numpy arrays.
There is no CPU fallback: if the shared library is missing the import of
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsymft.so")

SYMFT_OK = 0
SHOT_ALIGN = 512          # SYMFT_SHOT_ALIGN: shot offsets are multiples of this
POSTSELECT_NONE, POSTSELECT_ALL, POSTSELECT_LISTED = 0, 1, 2
FP32, FP64 = 0, 1
OUT_DEVICE, OUT_HOST = 0, 1
PLAIN_OFF, PLAIN_IN_KERNEL, PLAIN_PREPASS = 0, 1, 2
INSTR_NAMES = ("PromoteRot", "ActiveDiagRot", "ActivePairRot", "RandomMeas", "DetMeas",
               "ActiveDiagMeas", "ActivePairMeas")

EXPORTS = ("symft_compile", "symft_compile_ex", "symft_plan_info", "symft_plan_free",
           "symft_sample", "symft_sample_ex", "symft_last_error", "symft_last_launch_count",
           "symft_sample_noalloc", "symft_noalloc_last_error", "symft_autotune",
           "symft_sample_batch", "symft_plan_active_meas", "symft_measure_peaks")


class SymftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"symft error {code}: {msg}")
        self.code = code


class _Options(ctypes.Structure):
    _fields_ = [("postselect", ctypes.c_int), ("n_post_dets", ctypes.c_uint32),
                 ("post_dets", ctypes.POINTER(ctypes.c_uint32)), ("no_simplify", ctypes.c_int),
                ("no_product_components", ctypes.c_int), ("executor", ctypes.c_int),
                ("wide_tile_bits", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_uint32), ("n_meas_events", ctypes.c_uint32),
                ("n_records", ctypes.c_uint32), ("n_dets", ctypes.c_uint32),
                ("n_obs", ctypes.c_uint32), ("n_channels", ctypes.c_uint32),
                ("k_max", ctypes.c_uint32), ("n_instr", ctypes.c_uint32 * 7),
                ("max_expr_weight", ctypes.c_uint32), ("n_noise_components", ctypes.c_uint32),
                ("n_targets", ctypes.c_uint32), ("n_causal", ctypes.c_uint32),
                ("sign_xor_terms", ctypes.c_uint64), ("tuned_ns_per_shot", ctypes.c_float * 2),
                ("dense_amp_traffic", ctypes.c_uint64), ("dense_flops", ctypes.c_uint64),
                ("wide_amp_traffic", ctypes.c_uint64 * 2),
                ("dense_executor", ctypes.c_uint32 * 2), ("pc_capacity", ctypes.c_uint32),
                ("pc_selected", ctypes.c_uint32), ("pc_work", ctypes.c_uint64 * 2),
                ("sign_model", ctypes.c_double * 3),
                ("simplified", ctypes.c_uint32 * 3),
                ("wide_tile_bits", ctypes.c_uint32 * 2)]


class _SampleArgs(ctypes.Structure):
    _fields_ = [("shots", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("shot_offset", ctypes.c_uint64), ("meas_out", ctypes.c_void_p),
                ("det_out", ctypes.c_void_p), ("obs_out", ctypes.c_void_p),
                ("discard_out", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("out_location", ctypes.c_int), ("check", ctypes.c_int),
                ("plain", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("prob_out", ctypes.c_void_p), ("counts_out", ctypes.c_void_p)]


class _Peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int), ("sm_clock_mhz_attr", ctypes.c_double),
                ("int32_lop3_per_s", ctypes.c_double), ("int32_imad_wide_per_s", ctypes.c_double),
                ("philox_blocks_per_s", ctypes.c_double), ("fp32_fma_per_s", ctypes.c_double),
                ("fp64_fma_per_s", ctypes.c_double), ("smem_bytes_per_s", ctypes.c_double)]


class _Job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
                ("shots", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("shot_offset", ctypes.c_uint64), ("meas_out", ctypes.c_void_p),
                ("det_out", ctypes.c_void_p), ("obs_out", ctypes.c_void_p),
                ("discard_out", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("plain", ctypes.c_int), ("counts_out", ctypes.c_void_p)]


_LIB = None


def lib():
    """Load libsymft.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2607_28600_b300.build` "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    L.symft_compile.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    L.symft_compile.restype = ctypes.c_int
    L.symft_compile_ex.argtypes = [ctypes.c_char_p, ctypes.POINTER(_Options), ctypes.POINTER(ctypes.c_void_p)]
    L.symft_compile_ex.restype = ctypes.c_int
    L.symft_plan_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Info)]
    L.symft_plan_info.restype = ctypes.c_int
    L.symft_plan_active_meas.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32]
    L.symft_plan_active_meas.restype = ctypes.c_int
    L.symft_plan_free.argtypes = [ctypes.c_void_p]
    L.symft_plan_free.restype = None
    L.symft_sample.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.symft_sample.restype = ctypes.c_int
    L.symft_sample_ex.argtypes = [ctypes.c_void_p, ctypes.POINTER(_SampleArgs)]
    L.symft_sample_ex.restype = ctypes.c_int
    L.symft_last_error.argtypes = []
    L.symft_last_error.restype = ctypes.c_char_p
    L.symft_last_launch_count.argtypes = []
    L.symft_last_launch_count.restype = ctypes.c_int
    L.symft_sample_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p]
    L.symft_sample_noalloc.restype = ctypes.c_int
    L.symft_noalloc_last_error.argtypes = []
    L.symft_noalloc_last_error.restype = ctypes.c_char_p
    L.symft_autotune.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
    L.symft_autotune.restype = ctypes.c_int
    L.symft_sample_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                     ctypes.POINTER(_Job), ctypes.c_int, ctypes.c_void_p]
    L.symft_sample_batch.restype = ctypes.c_int
    L.symft_measure_peaks.argtypes = [ctypes.POINTER(_Peaks)]
    L.symft_measure_peaks.restype = ctypes.c_int
    _LIB = L
    return L


def _check(rc):
    if rc != SYMFT_OK:
        raise SymftError(rc, lib().symft_last_error().decode(errors="replace"))


def _ptr(x):
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


class Plan:
    """Owned handle of a compiled plan (frees it on garbage collection)."""

    def __init__(self, handle):
        self.handle = handle
        self._info = None

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _LIB is not None:
            _LIB.symft_plan_free(h)

    @property
    def info(self) -> dict:
        if self._info is None:
            self._info = symft_plan_info(self)
        return self._info

    def refresh_info(self) -> dict:
        self._info = symft_plan_info(self)
        return self._info

    def words(self, shots: int) -> int:
        return (shots + 63) // 64

    def active_meas(self) -> list:
        """Measurement ordinals of the active measurements (rows of prob_out)."""
        return symft_plan_active_meas(self)


EXECUTORS = {"auto": 0, "register": 1, "warp": 2, "cta": 3, "wide": 4, "components_warp": 5,
             "components_cta": 6}


def symft_compile(circuit_text: str, postselect: int = POSTSELECT_NONE, post_dets=None,
                  simplify: bool = True, product_components: bool = True, executor: str = "auto",
                  wide_tile_bits: int = 0) -> Plan:
    """Compile circuit text.  postselect=POSTSELECT_LISTED rejects a shot only at
    the detectors whose indices are listed in `post_dets`; simplify=False skips
    the commutation-aware simplification before planning."""
    h = ctypes.c_void_p()
    opt = _Options()
    opt.postselect = postselect
    opt.no_simplify = 0 if simplify else 1
    opt.no_product_components = 0 if product_components else 1
    opt.executor = EXECUTORS[executor]
    opt.wide_tile_bits = int(wide_tile_bits)
    if post_dets is not None:
        dets = [int(d) for d in post_dets]
        arr = (ctypes.c_uint32 * max(1, len(dets)))(*dets)
        opt.n_post_dets = len(dets)
        opt.post_dets = ctypes.cast(arr, ctypes.POINTER(ctypes.c_uint32))
    _check(lib().symft_compile_ex(circuit_text.encode(), ctypes.byref(opt), ctypes.byref(h)))
    return Plan(h.value)


def symft_plan_info(plan: Plan) -> dict:
    info = _Info()
    _check(lib().symft_plan_info(plan.handle, ctypes.byref(info)))
    d = {name: getattr(info, name) for name, _ in _Info._fields_
         if name not in ("n_instr", "tuned_ns_per_shot", "simplified", "wide_amp_traffic", "sign_model",
                         "dense_executor", "pc_work", "wide_tile_bits")}
    d["wide_tile_bits"] = [int(info.wide_tile_bits[0]), int(info.wide_tile_bits[1])]
    d["pc_work"] = [int(info.pc_work[0]), int(info.pc_work[1])]
    kinds = {0: "none", 1: "register", 2: "warp", 3: "cta", 4: "wide", 5: "components_warp",
             6: "components_cta"}
    d["dense_executor"] = [kinds.get(int(info.dense_executor[i]), "?") for i in range(2)]
    d["sign_model"] = {"philox_blocks_per_block": float(info.sign_model[0]),
                       "fires_per_block": float(info.sign_model[1]),
                       "xor_ops_per_block": float(info.sign_model[2])}
    d["wide_amp_traffic"] = [int(info.wide_amp_traffic[0]), int(info.wide_amp_traffic[1])]
    d["simplified"] = {"fused": int(info.simplified[0]), "cancelled": int(info.simplified[1]),
                       "branch_phase": int(info.simplified[2])}
    d["tuned_ns_per_shot"] = [float(info.tuned_ns_per_shot[0]), float(info.tuned_ns_per_shot[1])]
    d["n_instr"] = {INSTR_NAMES[i]: int(info.n_instr[i]) for i in range(7)}
    return d


def symft_plan_active_meas(plan: Plan) -> list:
    n = lib().symft_plan_active_meas(plan.handle, None, 0)
    if n < 0:
        _check(n)
    buf = (ctypes.c_uint32 * max(1, n))()
    _check(min(0, lib().symft_plan_active_meas(plan.handle, buf, n)))
    return [int(buf[j]) for j in range(n)]


def symft_sample(plan: Plan, shots: int, seed: int, meas_out=None, det_out=None, obs_out=None,
                 stream=None) -> None:
    _check(lib().symft_sample(plan.handle, shots, seed, _ptr(meas_out), _ptr(det_out),
                              _ptr(obs_out), _stream(stream)))


def symft_sample_ex(plan: Plan, shots: int, seed: int, shot_offset: int = 0, meas_out=None,
                    det_out=None, obs_out=None, discard_out=None, precision: int = FP32,
                    out_location: int = OUT_DEVICE, check: bool = False, stream=None,
                    plain: int = PLAIN_OFF, prob_out=None, counts_out=None) -> None:
    a = _SampleArgs()
    a.shots, a.seed, a.shot_offset = shots, seed, shot_offset
    a.meas_out, a.det_out = _ptr(meas_out), _ptr(det_out)
    a.obs_out, a.discard_out = _ptr(obs_out), _ptr(discard_out)
    a.precision, a.out_location, a.check = precision, out_location, int(bool(check))
    a.plain = int(plain)
    a.stream = _stream(stream)
    a.prob_out, a.counts_out = _ptr(prob_out), _ptr(counts_out)
    _check(lib().symft_sample_ex(plan.handle, ctypes.byref(a)))


def symft_sample_noalloc(plan: Plan, shots: int, seed: int, shot_offset: int = 0, meas_out=None,
                         det_out=None, obs_out=None, discard_out=None, precision: int = FP32,
                         stream=None) -> None:
    """Sample into caller-owned device buffers without any device allocation
    (scratch comes from the library's fixed 32 MiB device array)."""
    rc = lib().symft_sample_noalloc(plan.handle, shots, seed, shot_offset, _ptr(meas_out),
                                    _ptr(det_out), _ptr(obs_out), _ptr(discard_out), precision,
                                    _stream(stream))
    if rc != SYMFT_OK:
        raise SymftError(rc, lib().symft_noalloc_last_error().decode(errors="replace"))


def symft_autotune(plan: Plan, shots: int, precision: int = FP32, stream=None) -> None:
    """Time candidate launch shapes on `shots` shots and keep the fastest (synchronous)."""
    _check(lib().symft_autotune(plan.handle, shots, precision, _stream(stream)))


def symft_sample_batch(plans, jobs, stream=None) -> None:
    """Run jobs (dicts with plan index, shots, seed, outputs ...) as one CUDA graph launch.

    Each job: {"plan": i, "shots": n, "seed": s, "shot_offset": 0, "meas_out": t,
    "det_out": t, "obs_out": t, "discard_out": t, "precision": FP32, "plain": False,
    "counts_out": t}.
    """
    arr_p = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    arr_j = (_Job * len(jobs))()
    for k, j in enumerate(jobs):
        J = arr_j[k]
        J.plan = j["plan"]
        J.shots = j["shots"]
        J.seed = j.get("seed", 0)
        J.shot_offset = j.get("shot_offset", 0)
        J.meas_out = _ptr(j.get("meas_out"))
        J.det_out = _ptr(j.get("det_out"))
        J.obs_out = _ptr(j.get("obs_out"))
        J.discard_out = _ptr(j.get("discard_out"))
        J.precision = j.get("precision", FP32)
        J.plain = int(j.get("plain", PLAIN_OFF))
        J.counts_out = _ptr(j.get("counts_out"))
    _check(lib().symft_sample_batch(arr_p, len(plans), arr_j, len(jobs), _stream(stream)))


def symft_measure_peaks() -> dict:
    """Whole-GPU peak rates of the current device (integer LOP3 / IMAD.WIDE,
    Philox blocks, FP32 / FP64 FMA, shared-memory loads), measured by the
    library's microbenchmarks."""
    p = _Peaks()
    rc = lib().symft_measure_peaks(ctypes.byref(p))
    if rc != SYMFT_OK:
        raise SymftError(rc, "peak microbenchmarks failed")
    return {name: getattr(p, name) for name, _ in _Peaks._fields_}


def symft_last_launch_count() -> int:
    return lib().symft_last_launch_count()


def sample_to_tensors(plan: Plan, shots: int, seed: int, shot_offset: int = 0,
                      precision: int = FP32, stream=None, device="cuda", plain: bool = False):
    """Allocate device output columns (torch int64 holding the uint64 words) and sample."""
    import torch
    W = plan.words(shots)
    info = plan.info
    meas = torch.empty((info["n_records"], W), dtype=torch.int64, device=device)
    det = torch.empty((info["n_dets"], W), dtype=torch.int64, device=device)
    obs = torch.empty((info["n_obs"], W), dtype=torch.int64, device=device)
    disc = torch.empty((W,), dtype=torch.int64, device=device)
    symft_sample_ex(plan, shots, seed, shot_offset=shot_offset,
                    meas_out=meas if meas.numel() else None,
                    det_out=det if det.numel() else None,
                    obs_out=obs if obs.numel() else None,
                    discard_out=disc, precision=precision, stream=stream, plain=plain)
    return meas, det, obs, disc
