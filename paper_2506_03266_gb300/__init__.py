"""Python binding of libqca, the GB300 message-passing automaton decoder.

Thin ctypes marshalling over the C ABI declared in include/qca.h: every
computation runs in the library's CUDA kernels.  PyTorch only provides device
memory and the current CUDA stream.  There is no CPU fallback: if libqca.so is
missing or no CUDA device is present, the compute functions raise.

    import paper_2506_03266_gb300 as qca
    N = qca.sample_errors(L=256, shots=1000, p=0.05, seed=0)      # cuda uint8
    C, steps, fail = qca.decode_batch(N, max_steps=4096)
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqca.so")

QCA_OK = 0
QCA_ERR_ARG = -1
QCA_ERR_UNSUPPORTED = -2
QCA_ERR_CUDA = -3
QCA_ERR_WATCHDOG = -4
QCA_MAX_L = 1024
QCA_MAX_STEPS = 1 << 20

_lock = threading.Lock()
_lib = None


class QcaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libqca error {code}: {msg}")
        self.code = code


class QcaConfig(ctypes.Structure):
    """Mirror of struct qca_config (include/qca.h)."""
    _fields_ = [("v", ctypes.c_int32), ("m_max", ctypes.c_int32), ("p_move", ctypes.c_double),
                ("shot_offset", ctypes.c_int64), ("tie_order", ctypes.c_int32),
                ("balance_rule", ctypes.c_int32)]


# Readings of Eq. degbreak and of a balanced axis (qca_config.tie_order /
# balance_rule).
TIE_LEX, TIE_LITERAL = 0, 1
BALANCE_STAY, BALANCE_RANDOM = 0, 1


def build(force: bool = False) -> str:
    from . import builder
    return builder.build(force=force)


def lib():
    """Load libqca.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libqca.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        cfgp = ctypes.POINTER(QcaConfig)
        sig = {
            "qca_version": ([], i32),
            "qca_last_error": ([], ctypes.c_char_p),
            "qca_default_config": ([cfgp], i32),
            "qca_sample_errors": ([i32, i32, ctypes.c_double, u64, vp], i32),
            "qca_sample_errors_async": ([i32, i64, i64, ctypes.c_double, u64, vp, vp], i32),
            "qca_decode_batch": ([vp, i32, i32, i32, u64, vp, vp, vp], i32),
            "qca_decode_batch_async": ([vp, i32, i64, i32, u64, vp, vp, vp, cfgp, vp], i32),
            "qca_decode_syndrome_batch_async": ([vp, i32, i64, i32, u64, vp, vp, vp, vp, cfgp, vp],
                                                i32),
            "qca_decode_syndrome_batch": ([vp, i32, i32, i32, u64, vp, vp, vp], i32),
            "qca_decode_batch_host": ([vp, i32, i64, i32, u64, vp, vp, vp, cfgp], i32),
            "qca_decode_batch_noalloc": ([vp, i32, i64, i32, u64, vp, vp, vp, cfgp, vp], i32),
            "qca_uneven_draw": ([i64, u64, vp, vp], i32),
            "qca_set_tuning": ([i32, i32, i32], i32),
            "qca_set_cluster_ctas": ([i32, i32], i32),
            "qca_get_tuning": ([i32, vp, vp, vp], i32),
            "qca_autotune": ([i32, i64, ctypes.c_double, u64, i32, vp, vp, vp], i32),
            "qca_uneven_plan_create": ([vp, i64, vp, vp, ctypes.POINTER(vp)], i32),
            "qca_uneven_plan_destroy": ([vp], i32),
            "qca_uneven_plan_set_mode": ([vp, i32], i32),
            "qca_uneven_plan_offsets_device": ([vp, ctypes.POINTER(vp)], i32),
            "qca_sample_errors_uneven_async": ([vp, vp, vp, i64, u64, vp, vp], i32),
            "qca_decode_uneven_async": ([vp, vp, i32, u64, vp, vp, vp, cfgp, vp], i32),
            "qca_kernel_path": ([i32, cfgp], i32),
            "qca_set_kernel_path": ([i32, i32], i32),
            "qca_sample_errors_1d_async": ([i32, i64, i64, ctypes.c_double, u64, vp, vp], i32),
            "qca_decode_1d_batch_async": ([vp, i32, i64, i32, u64, cfgp, vp, vp, vp, vp, vp],
                                          i32),
            "qca_decode_open_batch_async": ([vp, i32, i64, i32, cfgp, vp, vp, vp, vp], i32),
            "qca_decode_desync_batch_async": ([vp, i32, i64, i32, ctypes.c_double, u64, cfgp,
                                               vp, vp, vp, vp], i32),
            "qca_net_param_count": ([], i64),
            "qca_net_create": ([u64, ctypes.POINTER(vp)], i32),
            "qca_net_destroy": ([vp], i32),
            "qca_net_get_params": ([vp, vp, i64], i32),
            "qca_net_set_params": ([vp, vp, i64], i32),
            "qca_net_train": ([vp, i32, i64, i32, ctypes.c_double, ctypes.c_double, u64,
                               ctypes.c_float, vp], i32),
            "qca_net_gradients": ([vp, vp, i32, i32, vp, i64, vp], i32),
            "qca_net_labels_async": ([vp, i32, i64, vp, vp, vp], i32),
            "qca_net_chunk_shots": ([i32], i64),
            "qca_net_calibrate_fp8": ([vp, vp, i32, i64, vp], i32),
            "qca_net_set_fp8_scales": ([vp, vp], i32),
            "qca_net_get_fp8_scales": ([vp, vp], i32),
            "qca_net_set_precision": ([vp, i32], i32),
            "qca_net_set_tensor_path": ([vp, i32], i32),
            "qca_net_status": ([vp], i32),
            "qca_watchdog_selftest": ([vp, vp, vp, vp], i32),
            "qca_probe_peaks": ([vp], i32),
            "qca_net_logits_async": ([vp, vp, i32, i64, vp, vp], i32),
            "qca_net_activations": ([vp, vp, i32, i64, i32, vp], i32),
            "qca_net_predecode_async": ([vp, vp, i32, i64, vp, vp, vp], i32),
            "qca_net_decode_batch_async": ([vp, vp, i32, i64, i32, u64, vp, vp, vp, cfgp, vp,
                                            vp], i32),
            "qca_free_workspace": ([], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _check(rc: int):
    if rc != QCA_OK:
        raise QcaError(rc, lib().qca_last_error().decode())


def last_error() -> str:
    return lib().qca_last_error().decode()


def make_config(v: int = 3, m_max: int = 255, p_move: float = 0.0,
                shot_offset: int = 0, tie_order: int = TIE_LEX,
                balance_rule: int = BALANCE_STAY) -> QcaConfig:
    c = QcaConfig()
    _check(lib().qca_default_config(ctypes.byref(c)))
    c.v, c.m_max, c.p_move, c.shot_offset = v, m_max, p_move, shot_offset
    c.tie_order, c.balance_rule = tie_order, balance_rule
    return c


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libqca needs a CUDA device; no CPU fallback exists")
    return torch


def _stream(torch, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_u8(torch, t, shape, name):
    if not (t.is_cuda and t.dtype == torch.uint8 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous cuda uint8 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _check_out(torch, out, specs, device):
    """Raise ValueError unless `out` holds one contiguous tensor per spec
    (dtype, shape, name), each on `device`: the kernels write those extents."""
    if not isinstance(out, (tuple, list)) or len(out) != len(specs):
        raise ValueError(f"out must be a tuple of {len(specs)} tensors")
    for t, (dtype, shape, name) in zip(out, specs):
        if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_contiguous() \
                or t.device != device:
            raise ValueError(f"{name} must be a contiguous {dtype} tensor on {device}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _decode_specs(torch, shots, L):
    return [(torch.uint8, (shots, 2, L, L), "correction"), (torch.int32, (shots,), "steps"),
            (torch.uint8, (shots,), "logical_fail")]


def kernel_path(L: int, v: int = 3) -> int:
    rc = lib().qca_kernel_path(L, ctypes.byref(make_config(v=v)))
    if rc < 0:
        _check(rc)
    return rc


def sample_errors_1d(L: int, shots: int, p: float, seed: int, shot0: int = 0, stream=None):
    """i.i.d. link flips of the ring (uint8 [shots][L] on the current cuda device)."""
    torch = _torch()
    out = torch.empty((shots, L), dtype=torch.uint8, device="cuda")
    _check(lib().qca_sample_errors_1d_async(L, shot0, shots, float(p), seed & (2**64 - 1),
                                            ctypes.c_void_p(out.data_ptr()),
                                            _stream(torch, stream)))
    return out


def decode_1d_batch(errors, max_steps: int = 4096, rng_seed: int = 0, *, v: int = 3,
                    m_max: int = 255, p_move: float = 0.0, shot_offset: int = 0, out=None,
                    stream=None):
    """1D decode of uint8 [shots][L] ring noise (cuda).  Returns (correction,
    steps, flag, majority_flag)."""
    torch = _torch()
    shots, L = errors.shape
    _dev_u8(torch, errors, (shots, L), "errors")
    if out is None:
        out = (torch.empty_like(errors), torch.empty(shots, dtype=torch.int32, device=errors.device),
               torch.empty(shots, dtype=torch.uint8, device=errors.device),
               torch.empty(shots, dtype=torch.uint8, device=errors.device))
    _check_out(torch, out, [(torch.uint8, (shots, L), "correction"),
                            (torch.int32, (shots,), "steps"), (torch.uint8, (shots,), "flag"),
                            (torch.uint8, (shots,), "majority_flag")], errors.device)
    C, steps, flag, maj = out
    cfg = make_config(v, m_max, p_move, shot_offset)
    _check(lib().qca_decode_1d_batch_async(
        ctypes.c_void_p(errors.data_ptr()), L, shots, max_steps, rng_seed & (2**64 - 1),
        ctypes.byref(cfg), ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(steps.data_ptr()),
        ctypes.c_void_p(flag.data_ptr()), ctypes.c_void_p(maj.data_ptr()),
        _stream(torch, stream)))
    return C, steps, flag, maj


def _variant_out(errors, out):
    torch = _torch()
    shots, L = errors.shape[0], errors.shape[-1]
    if out is None:
        out = (torch.empty_like(errors), torch.empty(shots, dtype=torch.int32, device=errors.device),
               torch.empty(shots, dtype=torch.uint8, device=errors.device))
    _check_out(torch, out, _decode_specs(torch, shots, L), errors.device)
    return out


def decode_open_batch(errors, max_steps: int = 4096, *, v: int = 3, m_max: int = 255, out=None,
                      stream=None):
    """Open-boundary decode of uint8 [shots][2][L][L] noise: (correction, steps, flag)."""
    torch = _torch()
    shots, L = errors.shape[0], errors.shape[-1]
    _dev_u8(torch, errors, (shots, 2, L, L), "errors")
    C, steps, fail = _variant_out(errors, out)
    cfg = make_config(v, m_max, 0.0, 0)
    _check(lib().qca_decode_open_batch_async(
        ctypes.c_void_p(errors.data_ptr()), L, shots, max_steps, ctypes.byref(cfg),
        ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(steps.data_ptr()),
        ctypes.c_void_p(fail.data_ptr()), _stream(torch, stream)))
    return C, steps, fail


def decode_desync_batch(errors, q: float, max_ticks: int = 100000, rng_seed: int = 0, *,
                        v: int = 3, m_max: int = 255, shot_offset: int = 0, out=None,
                        stream=None):
    """Uncoordinated (desynchronised) decode: (correction, ticks, flag)."""
    torch = _torch()
    shots, L = errors.shape[0], errors.shape[-1]
    _dev_u8(torch, errors, (shots, 2, L, L), "errors")
    C, ticks, fail = _variant_out(errors, out)
    cfg = make_config(v, m_max, 0.0, shot_offset)
    _check(lib().qca_decode_desync_batch_async(
        ctypes.c_void_p(errors.data_ptr()), L, shots, max_ticks, float(q),
        rng_seed & (2**64 - 1), ctypes.byref(cfg), ctypes.c_void_p(C.data_ptr()),
        ctypes.c_void_p(ticks.data_ptr()), ctypes.c_void_p(fail.data_ptr()),
        _stream(torch, stream)))
    return C, ticks, fail


def set_kernel_path(L: int, path: int = -1):
    """Override the kernel for size L: -1 automatic, 0 generic, 3 large-lattice."""
    _check(lib().qca_set_kernel_path(L, path))


def sample_errors(L: int, shots: int, p: float, seed: int, shot0: int = 0, out=None,
                  stream=None):
    """i.i.d. link flips (uint8 [shots][2][L][L] on the current cuda device)."""
    torch = _torch()
    if out is None:
        out = torch.empty((shots, 2, L, L), dtype=torch.uint8, device="cuda")
    _dev_u8(torch, out, (shots, 2, L, L), "out")
    _check(lib().qca_sample_errors_async(L, shot0, shots, float(p), seed & (2**64 - 1),
                                         ctypes.c_void_p(out.data_ptr()),
                                         _stream(torch, stream)))
    return out


def decode_batch(errors, max_steps: int = 4096, rng_seed: int = 0, *, v: int = 3,
                 m_max: int = 255, p_move: float = 0.0, shot_offset: int = 0, out=None,
                 stream=None, tie_order: int = TIE_LEX, balance_rule: int = BALANCE_STAY):
    """Decode noise realisations uint8 [shots][2][L][L] (cuda).

    Returns (correction uint8 [shots][2][L][L], steps int32 [shots],
    logical_fail uint8 [shots]); enqueued on the current stream.
    """
    torch = _torch()
    shots, L = errors.shape[0], errors.shape[-1]
    _dev_u8(torch, errors, (shots, 2, L, L), "errors")
    if out is None:
        C = torch.empty_like(errors)
        steps = torch.empty(shots, dtype=torch.int32, device=errors.device)
        fail = torch.empty(shots, dtype=torch.uint8, device=errors.device)
    else:
        _check_out(torch, out, _decode_specs(torch, shots, L), errors.device)
        C, steps, fail = out
    cfg = make_config(v, m_max, p_move, shot_offset, tie_order, balance_rule)
    _check(lib().qca_decode_batch_async(
        ctypes.c_void_p(errors.data_ptr()), L, shots, max_steps, rng_seed & (2**64 - 1),
        ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(steps.data_ptr()),
        ctypes.c_void_p(fail.data_ptr()), ctypes.byref(cfg), _stream(torch, stream)))
    return C, steps, fail


def decode_syndrome_batch(sigma, max_steps: int = 4096, rng_seed: int = 0, *, v: int = 3,
                          m_max: int = 255, p_move: float = 0.0, shot_offset: int = 0,
                          stream=None, tie_order: int = TIE_LEX,
                          balance_rule: int = BALANCE_STAY):
    """Decode anyon indicators uint8 [shots][L][L] (cuda, 1 = anyon).

    Returns (correction, steps, cut_parity uint8 [shots][2], exhausted uint8 [shots]).
    """
    torch = _torch()
    shots, L = sigma.shape[0], sigma.shape[-1]
    _dev_u8(torch, sigma, (shots, L, L), "sigma")
    C = torch.empty((shots, 2, L, L), dtype=torch.uint8, device=sigma.device)
    steps = torch.empty(shots, dtype=torch.int32, device=sigma.device)
    cut = torch.empty((shots, 2), dtype=torch.uint8, device=sigma.device)
    exh = torch.empty(shots, dtype=torch.uint8, device=sigma.device)
    cfg = make_config(v, m_max, p_move, shot_offset, tie_order, balance_rule)
    _check(lib().qca_decode_syndrome_batch_async(
        ctypes.c_void_p(sigma.data_ptr()), L, shots, max_steps, rng_seed & (2**64 - 1),
        ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(steps.data_ptr()),
        ctypes.c_void_p(cut.data_ptr()), ctypes.c_void_p(exh.data_ptr()), ctypes.byref(cfg),
        _stream(torch, stream)))
    return C, steps, cut, exh


def decode_syndrome_batch_sync(sigma, max_steps: int = 4096, rng_seed: int = 0):
    """The synchronous companion entry point qca_decode_syndrome_batch (default
    options, legacy default stream).  Returns (correction, steps, cut_parity)."""
    torch = _torch()
    shots, L = sigma.shape[0], sigma.shape[-1]
    _dev_u8(torch, sigma, (shots, L, L), "sigma")
    C = torch.empty((shots, 2, L, L), dtype=torch.uint8, device=sigma.device)
    steps = torch.empty(shots, dtype=torch.int32, device=sigma.device)
    cut = torch.empty((shots, 2), dtype=torch.uint8, device=sigma.device)
    torch.cuda.current_stream().synchronize()  # sigma is ready before the legacy stream reads it
    _check(lib().qca_decode_syndrome_batch(
        ctypes.c_void_p(sigma.data_ptr()), L, shots, max_steps, rng_seed & (2**64 - 1),
        ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(steps.data_ptr()),
        ctypes.c_void_p(cut.data_ptr())))
    return C, steps, cut


def decode_batch_host(errors, max_steps: int = 4096, rng_seed: int = 0, *, v: int = 3,
                      m_max: int = 255, p_move: float = 0.0, correction: bool = True,
                      out=None, tie_order: int = TIE_LEX, balance_rule: int = BALANCE_STAY):
    """End-to-end decode of HOST tensors (uint8 [shots][2][L][L], ideally pinned).

    Returns host tensors (correction or None, steps, logical_fail).
    """
    torch = _torch()
    if errors.is_cuda or errors.dtype != torch.uint8 or not errors.is_contiguous():
        raise ValueError("errors must be a contiguous host uint8 tensor")
    shots, L = errors.shape[0], errors.shape[-1]
    if tuple(errors.shape) != (shots, 2, L, L):
        raise ValueError(f"errors has shape {tuple(errors.shape)}, expected (shots, 2, L, L)")
    if out is None:
        pin = errors.is_pinned()
        C = torch.empty_like(errors, pin_memory=pin) if correction else None
        steps = torch.empty(shots, dtype=torch.int32, pin_memory=pin)
        fail = torch.empty(shots, dtype=torch.uint8, pin_memory=pin)
    else:
        specs = _decode_specs(torch, shots, L)
        if isinstance(out, (tuple, list)) and len(out) == 3 and out[0] is None:
            _check_out(torch, out[1:], specs[1:], errors.device)  # correction not copied back
        else:
            _check_out(torch, out, specs, errors.device)
        C, steps, fail = out
    cfg = make_config(v, m_max, p_move, 0, tie_order, balance_rule)
    _check(lib().qca_decode_batch_host(
        ctypes.c_void_p(errors.data_ptr()), L, shots, max_steps, rng_seed & (2**64 - 1),
        ctypes.c_void_p(C.data_ptr()) if C is not None else None,
        ctypes.c_void_p(steps.data_ptr()), ctypes.c_void_p(fail.data_ptr()), ctypes.byref(cfg)))
    return C, steps, fail


def decode_batch_noalloc(errors, out, max_steps: int = 4096, rng_seed: int = 0, *, v: int = 3,
                         m_max: int = 255, p_move: float = 0.0, shot_offset: int = 0,
                         stream=None, tie_order: int = TIE_LEX,
                         balance_rule: int = BALANCE_STAY):
    """Decode through qca_decode_batch_noalloc: the library allocates nothing.

    For callers that cannot allocate device memory while decoding (see the
    entry point's comment in include/qca.h): the caller provides the output
    tensors ``out = (correction, steps, logical_fail)``; the decoder state uses
    the library's fixed device array.  Calls that overlap on the GPU race on
    that array.
    """
    torch = _torch()
    shots, L = errors.shape[0], errors.shape[-1]
    _dev_u8(torch, errors, (shots, 2, L, L), "errors")
    _check_out(torch, out, _decode_specs(torch, shots, L), errors.device)
    C, steps, fail = out
    cfg = make_config(v, m_max, p_move, shot_offset, tie_order, balance_rule)
    _check(lib().qca_decode_batch_noalloc(
        ctypes.c_void_p(errors.data_ptr()), L, shots, max_steps, rng_seed & (2**64 - 1),
        ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(steps.data_ptr()),
        ctypes.c_void_p(fail.data_ptr()), ctypes.byref(cfg), _stream(torch, stream)))
    return C, steps, fail


def set_tuning(L: int, band_height: int = 0, sparse_divisor: int = 0):
    _check(lib().qca_set_tuning(L, band_height, sparse_divisor))


def set_cluster_ctas(L: int, ctas: int):
    """CTAs per cluster (2 or 4) of the on-chip sweep for 128 < L <= 256."""
    _check(lib().qca_set_cluster_ctas(L, ctas))


def get_tuning(L: int):
    """(band_height, sparse_divisor, threads_per_cta) in effect for L."""
    h, d, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().qca_get_tuning(L, ctypes.byref(h), ctypes.byref(d), ctypes.byref(t)))
    return h.value, d.value, t.value


def autotune(L: int, shots: int, p: float, seed: int = 1, max_steps: int = 4096):
    """Time the valid tunings for L and keep the fastest; returns
    (band_height, sparse_divisor, ms per decode of `shots` shots)."""
    _torch()
    h, d, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().qca_autotune(L, shots, float(p), seed & (2**64 - 1), max_steps, ctypes.byref(h),
                              ctypes.byref(d), ctypes.byref(ms)))
    return h.value, d.value, ms.value


def uneven_draw(shots: int, seed: int):
    """Per-shot L (int32) and flip threshold (uint64) of the mixed-size workload
    (host computation, numpy arrays)."""
    import numpy as np
    L = np.zeros(shots, dtype=np.int32)
    thr = np.zeros(shots, dtype=np.uint64)
    if shots:
        _check(lib().qca_uneven_draw(shots, seed & (2**64 - 1), L.ctypes.data_as(ctypes.c_void_p),
                                     thr.ctypes.data_as(ctypes.c_void_p)))
    return L, thr


class UnevenPlan:
    """Shots of mixed lattice sizes packed back to back (qca_uneven_plan_*)."""

    def __init__(self, L_host):
        import numpy as np
        self.L = np.ascontiguousarray(L_host, dtype=np.int32)
        self.shots = len(self.L)
        self.offsets = np.zeros(self.shots, dtype=np.int64)
        total = ctypes.c_int64()
        h = ctypes.c_void_p()
        _check(lib().qca_uneven_plan_create(self.L.ctypes.data_as(ctypes.c_void_p), self.shots,
                                            self.offsets.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(total), ctypes.byref(h)))
        self.handle = h
        self.total_bytes = total.value

    def set_mode(self, mode: str):
        """"mixed" (default): one persistent launch over every size the on-chip
        sweep takes; "per_size": one persistent launch per size."""
        _check(lib().qca_uneven_plan_set_mode(self.handle, {"mixed": 0, "per_size": 1}[mode]))

    def close(self):
        if self.handle:
            lib().qca_uneven_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def offsets_device_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check(lib().qca_uneven_plan_offsets_device(self.handle, ctypes.byref(p)))
        return p.value

    def sample(self, thr_host, seed: int, out=None, stream=None):
        """Packed noise on the device (uint8 [total_bytes])."""
        torch = _torch()
        import numpy as np
        if out is None:
            out = torch.empty(self.total_bytes, dtype=torch.uint8, device="cuda")
        _dev_u8(torch, out, (self.total_bytes,), "out")
        Ld = torch.from_numpy(self.L).cuda()
        td = torch.from_numpy(np.ascontiguousarray(thr_host, dtype=np.uint64).view(np.int64)).cuda()
        _check(lib().qca_sample_errors_uneven_async(
            ctypes.c_void_p(Ld.data_ptr()), ctypes.c_void_p(self.offsets_device_ptr()),
            ctypes.c_void_p(td.data_ptr()), self.shots, seed & (2**64 - 1),
            ctypes.c_void_p(out.data_ptr()), _stream(torch, stream)))
        torch.cuda.current_stream().synchronize()
        return out

    def decode(self, errors, max_steps: int = 4096, rng_seed: int = 0, out=None, v: int = 3,
               m_max: int = 255, p_move: float = 0.0, stream=None, tie_order: int = TIE_LEX,
               balance_rule: int = BALANCE_STAY):
        """Decode packed noise; returns (correction packed uint8, steps, logical_fail)."""
        torch = _torch()
        _dev_u8(torch, errors, (self.total_bytes,), "errors")
        if out is None:
            C = torch.empty_like(errors)
            steps = torch.empty(self.shots, dtype=torch.int32, device=errors.device)
            fail = torch.empty(self.shots, dtype=torch.uint8, device=errors.device)
        else:
            _check_out(torch, out, [(torch.uint8, (self.total_bytes,), "correction"),
                                    (torch.int32, (self.shots,), "steps"),
                                    (torch.uint8, (self.shots,), "logical_fail")], errors.device)
            C, steps, fail = out
        cfg = make_config(v, m_max, p_move, 0, tie_order, balance_rule)
        _check(lib().qca_decode_uneven_async(
            self.handle, ctypes.c_void_p(errors.data_ptr()), max_steps, rng_seed & (2**64 - 1),
            ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(steps.data_ptr()),
            ctypes.c_void_p(fail.data_ptr()), ctypes.byref(cfg), _stream(torch, stream)))
        return C, steps, fail


def net_labels(errors, stream=None):
    """First-step labels (uint8 [shots][L][L]: 0..3 direction, 4 none, 255 no anyon)."""
    torch = _torch()
    shots, L = errors.shape[0], errors.shape[-1]
    _dev_u8(torch, errors, (shots, 2, L, L), "errors")
    out = torch.empty((shots, L, L), dtype=torch.uint8, device=errors.device)
    scratch = torch.empty(2 * shots * L * L, dtype=torch.uint8, device=errors.device)
    _check(lib().qca_net_labels_async(ctypes.c_void_p(errors.data_ptr()), L, shots,
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(scratch.data_ptr()), _stream(torch, stream)))
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return out


def net_chunk_shots(L: int) -> int:
    n = int(lib().qca_net_chunk_shots(L))
    if n < 0:
        _check(n)
    return n


class Net:
    """Learned pre-decoder handle (qca_net_*): 3x3 circular conv net
    2 -> 32 -> 32 -> 32 -> 4 proposing moves that pair adjacent anyons."""

    def __init__(self, seed: int = 0):
        _torch()
        h = ctypes.c_void_p()
        _check(lib().qca_net_create(seed & (2**64 - 1), ctypes.byref(h)))
        self.handle = h

    @staticmethod
    def param_count() -> int:
        return int(lib().qca_net_param_count())

    def close(self):
        if self.handle:
            lib().qca_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        out = np.zeros(self.param_count(), dtype=np.float32)
        _check(lib().qca_net_get_params(self.handle, out.ctypes.data_as(ctypes.c_void_p),
                                        out.size))
        return out

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().qca_net_set_params(self.handle, a.ctypes.data_as(ctypes.c_void_p), a.size))

    def train(self, L: int, iterations: int, batch: int, p_lo: float, p_hi: float,
              seed: int = 1, lr: float = 1e-3):
        """Adam steps on fresh automaton-labelled syndromes; returns the losses."""
        import numpy as np
        losses = np.zeros(max(iterations, 1), dtype=np.float32)
        _check(lib().qca_net_train(self.handle, L, iterations, batch, float(p_lo), float(p_hi),
                                   seed & (2**64 - 1), float(lr),
                                   losses.ctypes.data_as(ctypes.c_void_p)))
        return losses[:iterations]

    def calibrate_fp8(self, errors, stream=None):
        """Per-layer activation scales of the FP8 form from these noise realisations."""
        torch = _torch()
        shots, L = errors.shape[0], errors.shape[-1]
        _dev_u8(torch, errors, (shots, 2, L, L), "errors")
        _check(lib().qca_net_calibrate_fp8(self.handle, ctypes.c_void_p(errors.data_ptr()), L,
                                           shots, _stream(torch, stream)))
        return self.fp8_scales()

    def fp8_scales(self):
        import numpy as np
        out = np.zeros(3, dtype=np.float32)
        _check(lib().qca_net_get_fp8_scales(self.handle, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_fp8_scales(self, scales):
        import numpy as np
        a = np.ascontiguousarray(scales, dtype=np.float32)
        _check(lib().qca_net_set_fp8_scales(self.handle, a.ctypes.data_as(ctypes.c_void_p)))

    def set_precision(self, precision: str):
        """"bf16" or "fp8" for every inference entry point."""
        _check(lib().qca_net_set_precision(self.handle, {"bf16": 0, "fp8": 1}[precision]))

    def set_tensor_path(self, path: str):
        """Layers 2-4 where L % 128 == 0: "tcgen05_ws" (default,
        warp-specialised; bf16 and FP8 forms), "tcgen05" (row-synchronous,
        bf16 form; FP8 then on mma.sync) or "mma" (mma.sync; also the path for
        other L)."""
        _check(lib().qca_net_set_tensor_path(
            self.handle, {"mma": 0, "tcgen05": 1, "tcgen05_ws": 2}[path]))

    def status(self):
        """Raises QcaError if a tensor-core wait timed out since the last call."""
        _check(lib().qca_net_status(self.handle))

    def gradients(self, errors):
        """(loss, flat fp32 gradient) of the training loss on these noise
        realisations (cuda uint8 [batch][2][L][L]); the weights are unchanged."""
        import numpy as np
        torch = _torch()
        batch, L = errors.shape[0], errors.shape[-1]
        _dev_u8(torch, errors, (batch, 2, L, L), "errors")
        g = np.zeros(self.param_count(), dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().qca_net_gradients(self.handle, ctypes.c_void_p(errors.data_ptr()), L, batch,
                                       g.ctypes.data_as(ctypes.c_void_p), g.size,
                                       ctypes.byref(loss)))
        return loss.value, g

    def logits(self, errors, stream=None):
        """fp32 [shots][4][L][L] logits of the noise realisations' syndromes."""
        torch = _torch()
        shots, L = errors.shape[0], errors.shape[-1]
        _dev_u8(torch, errors, (shots, 2, L, L), "errors")
        out = torch.empty((shots, 4, L, L), dtype=torch.float32, device=errors.device)
        _check(lib().qca_net_logits_async(self.handle, ctypes.c_void_p(errors.data_ptr()), L,
                                          shots, ctypes.c_void_p(out.data_ptr()),
                                          _stream(torch, stream)))
        return out

    def activations(self, errors, layer: int):
        """Layer `layer` (1..3) activations as the next layer reads them, fp32
        [shots][32][L][L]: bf16 values, or e4m3 values before the layer's
        scale in the FP8 form (qca_net_activations; synchronises)."""
        torch = _torch()
        shots, L = errors.shape[0], errors.shape[-1]
        _dev_u8(torch, errors, (shots, 2, L, L), "errors")
        out = torch.empty((shots, 32, L, L), dtype=torch.float32, device=errors.device)
        torch.cuda.synchronize()
        _check(lib().qca_net_activations(self.handle, ctypes.c_void_p(errors.data_ptr()), L,
                                         shots, layer, ctypes.c_void_p(out.data_ptr())))
        return out

    def predecode(self, errors, stream=None):
        """(residual N xor C0, C0), both uint8 [shots][2][L][L]."""
        torch = _torch()
        shots, L = errors.shape[0], errors.shape[-1]
        _dev_u8(torch, errors, (shots, 2, L, L), "errors")
        R = torch.empty_like(errors)
        C0 = torch.empty_like(errors)
        _check(lib().qca_net_predecode_async(self.handle, ctypes.c_void_p(errors.data_ptr()), L,
                                             shots, ctypes.c_void_p(R.data_ptr()),
                                             ctypes.c_void_p(C0.data_ptr()),
                                             _stream(torch, stream)))
        return R, C0

    def decode_batch(self, errors, max_steps: int = 4096, rng_seed: int = 0, *, v: int = 3,
                     m_max: int = 255, p_move: float = 0.0, shot_offset: int = 0, out=None,
                     scratch=None, stream=None, tie_order: int = TIE_LEX,
                     balance_rule: int = BALANCE_STAY):
        """Net + automaton: (correction, automaton steps, logical_fail)."""
        torch = _torch()
        shots, L = errors.shape[0], errors.shape[-1]
        _dev_u8(torch, errors, (shots, 2, L, L), "errors")
        if out is None:
            C = torch.empty_like(errors)
            steps = torch.empty(shots, dtype=torch.int32, device=errors.device)
            fail = torch.empty(shots, dtype=torch.uint8, device=errors.device)
        else:
            _check_out(torch, out, _decode_specs(torch, shots, L), errors.device)
            C, steps, fail = out
        if scratch is None:
            scratch = torch.empty_like(errors)
        _dev_u8(torch, scratch, (shots, 2, L, L), "scratch")
        cfg = make_config(v, m_max, p_move, shot_offset, tie_order, balance_rule)
        _check(lib().qca_net_decode_batch_async(
            self.handle, ctypes.c_void_p(errors.data_ptr()), L, shots, max_steps,
            rng_seed & (2**64 - 1), ctypes.c_void_p(C.data_ptr()),
            ctypes.c_void_p(steps.data_ptr()), ctypes.c_void_p(fail.data_ptr()),
            ctypes.byref(cfg), ctypes.c_void_p(scratch.data_ptr()), _stream(torch, stream)))
        return C, steps, fail


def watchdog_selftest():
    """(first wait gave up, second wait gave up, first wait in s, second
    waiter's lag in s) of the device watchdog self-test: a bounded wait on a
    barrier nothing completes gives up and stops a second waiter."""
    a, b = ctypes.c_int(), ctypes.c_int()
    t1, t2 = ctypes.c_double(), ctypes.c_double()
    _check(lib().qca_watchdog_selftest(ctypes.byref(a), ctypes.byref(b), ctypes.byref(t1),
                                       ctypes.byref(t2)))
    return bool(a.value), bool(b.value), t1.value, t2.value


class QcaPeaks(ctypes.Structure):
    """Mirror of struct qca_peaks (include/qca.h)."""
    _fields_ = [("sms", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("sm_clock_mhz", ctypes.c_double), ("min16x2_per_clk_sm", ctypes.c_double),
                ("lop3_per_clk_sm", ctypes.c_double), ("min_u32_per_clk_sm", ctypes.c_double),
                ("smem_bytes_per_clk_sm", ctypes.c_double),
                ("min16x2_lane_ops_per_s", ctypes.c_double), ("smem_bytes_per_s", ctypes.c_double)]


def probe_peaks():
    """Measured issue rates of min.u16x2, lop3.b32 and min.u32 and the
    shared-memory load bandwidth of the current device (per clock per SM and
    per second), with the SM clock seen during the probes: the denominators of
    the sweep's integer-ALU and shared-memory rooflines."""
    out = QcaPeaks()
    _check(lib().qca_probe_peaks(ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in QcaPeaks._fields_}


def free_workspace():
    _check(lib().qca_free_workspace())
