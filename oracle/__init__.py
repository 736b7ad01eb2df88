"""CPU oracle of the message-passing automaton decoder (arXiv 2506.03266).

TEST INFRASTRUCTURE ONLY.  This package wraps the plain single-threaded C
implementation in ``qca_oracle.c`` with ctypes + numpy.  Only the test-suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library's product path never does.  It shares no code with the CUDA
library: neither imports nor links the other.

Every function follows one definition of the paper (Sec. 3.2,
Def. "D-dimensional message passing automaton"; Def. "synchronous automaton
decoder"; Def. "logical failure rate and decoding time"; Sec. 7 numerics); see
the header comment of ``qca_oracle.c`` for the readings R1-R11 of points where
the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qca_oracle.c")
_SRC_1D = os.path.join(_HERE, "qca_oracle_1d.c")
_SRC_VAR = os.path.join(_HERE, "qca_oracle_variants.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libqca_oracle.so")
_lock = threading.Lock()
_lib = None

# Defaults fixed by the paper's numerics (Sec. 7: v = 3) and by the 8-bit
# message register (m_max = 255, reading R5).
V_DEFAULT = 3
M_MAX_DEFAULT = 255
# Readings of Eq. degbreak (R3) and of a balanced axis (R4): 0 / 0 are the
# defaults (lexicographic ties; a balanced anyon stays).
TIE_LEX, TIE_LITERAL = 0, 1
BALANCE_STAY, BALANCE_RANDOM = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "qca_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC_1D),
                                                   os.path.getmtime(_SRC_VAR),
                                                   os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_1D, _SRC_VAR,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        c_int, c_i64, c_u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        lib.qo_splitmix64.argtypes = [c_u64]
        lib.qo_splitmix64.restype = c_u64
        lib.qo_prob_threshold.argtypes = [ctypes.c_double]
        lib.qo_prob_threshold.restype = c_u64
        lib.qo_sample_errors.argtypes = [c_int, c_i64, c_i64, c_u64, c_u64, u8p]
        lib.qo_sample_errors.restype = None
        lib.qo_uneven_draw.argtypes = [c_i64, c_u64, i32p,
                                       np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")]
        lib.qo_uneven_draw.restype = None
        lib.qo_syndrome.argtypes = [c_int, u8p, i8p]
        lib.qo_syndrome.restype = None
        lib.qo_message_substep.argtypes = [c_int, c_int, i8p, i32p, i32p]
        lib.qo_message_substep.restype = None
        lib.qo_forces.argtypes = [c_int, i8p, i32p, i8p]
        lib.qo_forces.restype = None
        lib.qo_forces_rule.argtypes = [c_int, c_int, i8p, i32p, i8p, ctypes.c_void_p]
        lib.qo_forces_rule.restype = None
        lib.qo_feedback_links.argtypes = [c_int, i8p, i8p, u8p]
        lib.qo_feedback_links.restype = None
        lib.qo_step.argtypes = [c_int, c_int, c_int, c_int, c_int, c_u64, c_u64, c_i64,
                                ctypes.c_int32, i8p, i32p, u8p, ctypes.c_void_p]
        lib.qo_step.restype = c_int
        lib.qo_cut_parity.argtypes = [c_int, u8p, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
        lib.qo_cut_parity.restype = None
        lib.qo_decode_shot.argtypes = [u8p, c_int, c_int, c_int, c_int, c_int, c_int, c_u64,
                                       c_u64, c_i64, u8p, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.c_void_p, c_int]
        lib.qo_decode_shot.restype = c_int
        lib.qo_decode_syndrome_shot.argtypes = [u8p, c_int, c_int, c_int, c_int, c_int, c_int,
                                                c_u64, c_u64, c_i64, u8p,
                                                ctypes.POINTER(ctypes.c_int32), u8p]
        lib.qo_decode_syndrome_shot.restype = c_int
        lib.qo_decode_batch.argtypes = [u8p, c_int, c_i64, c_i64, c_int, c_int, c_int, c_int,
                                        c_int, c_u64, c_u64, u8p, i32p, u8p]
        lib.qo_decode_batch.restype = None
        lib.qo1_sample_errors.argtypes = [c_int, c_i64, c_i64, c_u64, c_u64, u8p]
        lib.qo1_sample_errors.restype = None
        lib.qo1_syndrome.argtypes = [c_int, u8p, i8p]
        lib.qo1_syndrome.restype = None
        lib.qo1_substep.argtypes = [c_int, c_int, i8p, i32p, i32p]
        lib.qo1_substep.restype = None
        lib.qo1_forces.argtypes = [c_int, i8p, i32p, i8p]
        lib.qo1_forces.restype = None
        lib.qo1_feedback.argtypes = [c_int, i8p, i8p, u8p]
        lib.qo1_feedback.restype = None
        lib.qo1_step.argtypes = [c_int, c_int, c_int, c_u64, c_u64, c_i64, ctypes.c_int32,
                                 i8p, i32p, u8p]
        lib.qo1_step.restype = c_int
        lib.qo1_decode_shot.argtypes = [u8p, c_int, c_int, c_int, c_int, c_u64, c_u64, c_i64,
                                        u8p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_uint8)]
        lib.qo1_decode_shot.restype = c_int
        lib.qo_open_link_exists.argtypes = [c_int, c_int, c_int, c_int]
        lib.qo_open_link_exists.restype = c_int
        lib.qo_open_syndrome.argtypes = [c_int, u8p, i8p]
        lib.qo_open_syndrome.restype = None
        lib.qo_open_substep.argtypes = [c_int, c_int, i8p, i32p, i32p]
        lib.qo_open_substep.restype = None
        lib.qo_open_decode_shot.argtypes = [u8p, c_int, c_int, c_int, c_int, u8p,
                                            ctypes.POINTER(ctypes.c_int32)]
        lib.qo_open_decode_shot.restype = c_int
        lib.qo_desync_decode_shot.argtypes = [u8p, c_int, c_int, c_int, c_int, c_u64, c_u64,
                                              c_u64, c_i64, u8p, ctypes.POINTER(ctypes.c_int32)]
        lib.qo_desync_decode_shot.restype = c_int
        _lib = lib
        return lib


# ----------------------------------------------------------------- helpers --

def splitmix64(z: int) -> int:
    return int(_load().qo_splitmix64(ctypes.c_uint64(z & (2**64 - 1))))


def prob_threshold(p: float) -> int:
    """Integer threshold floor(p * 2^64) used by both sides for an edge flip."""
    return int(_load().qo_prob_threshold(float(p)))


def sample_errors(L: int, shots: int, p: float, seed: int, shot0: int = 0,
                  thr: int = None) -> np.ndarray:
    """i.i.d. bit-flip noise (Sec. 7), uint8 [shots][2][L][L]; `thr` (the integer
    flip threshold) overrides p."""
    out = np.zeros((shots, 2, L, L), dtype=np.uint8)
    t = prob_threshold(p) if thr is None else int(thr)
    _load().qo_sample_errors(L, shot0, shots, t, seed, out)
    return out


def uneven_draw(shots: int, seed: int):
    """Per-shot (L, flip threshold) of the mixed-size workload."""
    L = np.zeros(shots, dtype=np.int32)
    thr = np.zeros(shots, dtype=np.uint64)
    if shots:
        _load().qo_uneven_draw(shots, seed, L, thr)
    return L, thr


def syndrome(edges: np.ndarray) -> np.ndarray:
    """sigma (int8, +1/-1) of a link set uint8 [2][L][L] (Def. synch_ccqs)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint8)
    L = edges.shape[-1]
    sig = np.zeros((L, L), dtype=np.int8)
    _load().qo_syndrome(L, edges, sig)
    return sig


def message_substep(sigma: np.ndarray, m: np.ndarray, m_max: int = M_MAX_DEFAULT) -> np.ndarray:
    """One application of A^(D) (Def. Dd_msg_passing); m is int32 [4][L][L]."""
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    m = np.ascontiguousarray(m, dtype=np.int32)
    L = sigma.shape[0]
    out = np.zeros_like(m)
    _load().qo_message_substep(L, m_max, sigma, m, out)
    return out


def forces(sigma: np.ndarray, m: np.ndarray, tie_order: int = TIE_LEX,
           with_balanced: bool = False):
    """f^a_r, int8 [2][L][L] (Eqs. blahdef / degbreak).  With with_balanced,
    returns (f, balanced) where balanced (uint8 [L][L]) holds the chosen axis
    (1 x, 2 y) of anyons whose chosen axis is balanced."""
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    m = np.ascontiguousarray(m, dtype=np.int32)
    L = sigma.shape[0]
    f = np.zeros((2, L, L), dtype=np.int8)
    if tie_order == TIE_LEX and not with_balanced:
        _load().qo_forces(L, sigma, m, f)
        return f
    bal = np.zeros((L, L), dtype=np.uint8)
    _load().qo_forces_rule(L, tie_order, sigma, m, f, bal.ctypes.data_as(ctypes.c_void_p))
    return (f, bal) if with_balanced else f


def feedback_links(sigma: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Links flipped by F^(D) (Eq. ddfeedback), uint8 [2][L][L]."""
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    f = np.ascontiguousarray(f, dtype=np.int8)
    L = sigma.shape[0]
    out = np.zeros((2, L, L), dtype=np.uint8)
    _load().qo_feedback_links(L, sigma, f, out)
    return out


def step(sigma: np.ndarray, m: np.ndarray, C: np.ndarray, *, v: int = V_DEFAULT,
         m_max: int = M_MAX_DEFAULT, tie_order: int = TIE_LEX, balance_rule: int = BALANCE_STAY,
         move_thr: int = 0, seed: int = 0, shot: int = 0, t: int = 0):
    """One decoder step, in place on (sigma, m, C).  Returns (anyons, flips)."""
    L = sigma.shape[0]
    flips = np.zeros((2, L, L), dtype=np.uint8)
    n = _load().qo_step(L, v, m_max, tie_order, balance_rule, move_thr, seed, shot, t, sigma, m,
                        C, flips.ctypes.data_as(ctypes.c_void_p))
    return n, flips


def cut_parity(R: np.ndarray):
    R = np.ascontiguousarray(R, dtype=np.uint8)
    L = R.shape[-1]
    wx, wy = ctypes.c_int(), ctypes.c_int()
    _load().qo_cut_parity(L, R, ctypes.byref(wx), ctypes.byref(wy))
    return wx.value, wy.value


def decode_shot(N: np.ndarray, *, v: int = V_DEFAULT, m_max: int = M_MAX_DEFAULT,
                max_steps: int = 4096, move_thr: int = 0, seed: int = 0, shot: int = 0,
                trace: bool = False, tie_order: int = TIE_LEX,
                balance_rule: int = BALANCE_STAY):
    """Decode one noise realisation N (uint8 [2][L][L]).

    Returns (C, steps, flag) or, with trace=True, (C, steps, flag, anyons_per_step).
    """
    N = np.ascontiguousarray(N, dtype=np.uint8)
    L = N.shape[-1]
    C = np.zeros_like(N)
    steps = ctypes.c_int32()
    tr = np.zeros(max(1, max_steps), dtype=np.int32) if trace else None
    flag = _load().qo_decode_shot(N, L, v, m_max, tie_order, balance_rule, max_steps, move_thr,
                                  seed, shot, C,
                                  ctypes.byref(steps),
                                  tr.ctypes.data_as(ctypes.c_void_p) if trace else None,
                                  len(tr) if trace else 0)
    if trace:
        return C, steps.value, flag, tr[: min(steps.value, len(tr))].copy()
    return C, steps.value, flag


def decode_syndrome_shot(anyon: np.ndarray, *, v: int = V_DEFAULT, m_max: int = M_MAX_DEFAULT,
                         max_steps: int = 4096, move_thr: int = 0, seed: int = 0, shot: int = 0,
                         tie_order: int = TIE_LEX, balance_rule: int = BALANCE_STAY):
    """Decode a pure syndrome (uint8 [L][L], 1 = anyon).  Returns (C, steps, flag, cut)."""
    anyon = np.ascontiguousarray(anyon, dtype=np.uint8)
    L = anyon.shape[-1]
    C = np.zeros((2, L, L), dtype=np.uint8)
    cut = np.zeros(2, dtype=np.uint8)
    steps = ctypes.c_int32()
    flag = _load().qo_decode_syndrome_shot(anyon, L, v, m_max, tie_order, balance_rule, max_steps,
                                           move_thr, seed, shot, C, ctypes.byref(steps), cut)
    return C, steps.value, flag, cut


def decode_batch(N: np.ndarray, *, v: int = V_DEFAULT, m_max: int = M_MAX_DEFAULT,
                 max_steps: int = 4096, move_thr: int = 0, seed: int = 0, shot0: int = 0,
                 tie_order: int = TIE_LEX, balance_rule: int = BALANCE_STAY):
    """Decode uint8 [shots][2][L][L].  Returns (C, steps int32[shots], flags uint8[shots])."""
    N = np.ascontiguousarray(N, dtype=np.uint8)
    shots, L = N.shape[0], N.shape[-1]
    C = np.zeros_like(N)
    steps = np.zeros(shots, dtype=np.int32)
    flags = np.zeros(shots, dtype=np.uint8)
    if shots:
        _load().qo_decode_batch(N, L, shot0, shots, v, m_max, tie_order, balance_rule, max_steps,
                                move_thr, seed, C, steps, flags)
    return C, steps, flags


# ------------------------------------------------------------- 1D variant
# Repetition code on a ring (Sec. 3.1, Def. "message passing automaton, 1D";
# Sec. 7.1 numerics); readings in qca_oracle_1d.c.

def sample_errors_1d(L: int, shots: int, p: float, seed: int, shot0: int = 0) -> np.ndarray:
    out = np.zeros((shots, L), dtype=np.uint8)
    _load().qo1_sample_errors(L, shot0, shots, prob_threshold(p), seed, out)
    return out


def syndrome_1d(links: np.ndarray) -> np.ndarray:
    links = np.ascontiguousarray(links, dtype=np.uint8)
    sigma = np.zeros(links.shape[-1], dtype=np.int8)
    _load().qo1_syndrome(links.shape[-1], links, sigma)
    return sigma


def substep_1d(sigma: np.ndarray, m: np.ndarray, m_max: int = M_MAX_DEFAULT) -> np.ndarray:
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    m = np.ascontiguousarray(m, dtype=np.int32)
    out = np.zeros_like(m)
    _load().qo1_substep(sigma.shape[0], m_max, sigma, m, out)
    return out


def forces_1d(sigma: np.ndarray, m: np.ndarray) -> np.ndarray:
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    m = np.ascontiguousarray(m, dtype=np.int32)
    f = np.zeros(sigma.shape[0], dtype=np.int8)
    _load().qo1_forces(sigma.shape[0], sigma, m, f)
    return f


def feedback_1d(sigma: np.ndarray, f: np.ndarray) -> np.ndarray:
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    f = np.ascontiguousarray(f, dtype=np.int8)
    out = np.zeros(sigma.shape[0], dtype=np.uint8)
    _load().qo1_feedback(sigma.shape[0], sigma, f, out)
    return out


def step_1d(sigma, m, C, *, v=V_DEFAULT, m_max=M_MAX_DEFAULT, move_thr=0, seed=0, shot=0, t=0):
    """One step in place on (sigma, m, C); returns the anyon count."""
    return _load().qo1_step(sigma.shape[0], v, m_max, move_thr, seed, shot, t, sigma, m, C)


def decode_shot_1d(N: np.ndarray, *, v: int = V_DEFAULT, m_max: int = M_MAX_DEFAULT,
                   max_steps: int = 4096, move_thr: int = 0, seed: int = 0, shot: int = 0):
    """Returns (C, steps, flag, majority_flag)."""
    N = np.ascontiguousarray(N, dtype=np.uint8)
    L = N.shape[-1]
    C = np.zeros_like(N)
    steps = ctypes.c_int32()
    maj = ctypes.c_uint8()
    flag = _load().qo1_decode_shot(N, L, v, m_max, max_steps, move_thr, seed, shot, C,
                                   ctypes.byref(steps), ctypes.byref(maj))
    return C, steps.value, flag, maj.value


# ---------------------------------------------------------- 2D variants
# Open boundaries (Appendix "Open boundary conditions") and uncoordinated
# desynchronisation (Sec. 7.3); readings R16 / R17 in qca_oracle_variants.c.

def open_link_mask(L: int) -> np.ndarray:
    """uint8 [2][L][L]: 1 where the open lattice has a qubit."""
    lib = _load()
    m = np.zeros((2, L, L), np.uint8)
    for a in range(2):
        for y in range(L):
            for x in range(L):
                m[a, y, x] = lib.qo_open_link_exists(L, a, x, y)
    return m


def open_syndrome(E: np.ndarray) -> np.ndarray:
    E = np.ascontiguousarray(E, dtype=np.uint8)
    L = E.shape[-1]
    s = np.zeros((L, L), np.int8)
    _load().qo_open_syndrome(L, E, s)
    return s


def open_substep(sigma, m, m_max: int = M_MAX_DEFAULT):
    sigma = np.ascontiguousarray(sigma, dtype=np.int8)
    m = np.ascontiguousarray(m, dtype=np.int32)
    out = np.zeros_like(m)
    _load().qo_open_substep(sigma.shape[0], m_max, sigma, m, out)
    return out


def open_decode_shot(N, *, v: int = V_DEFAULT, m_max: int = M_MAX_DEFAULT, max_steps: int = 4096):
    """Returns (C, steps, flag) on the open lattice."""
    N = np.ascontiguousarray(N, dtype=np.uint8)
    L = N.shape[-1]
    C = np.zeros_like(N)
    steps = ctypes.c_int32()
    flag = _load().qo_open_decode_shot(N, L, v, m_max, max_steps, C, ctypes.byref(steps))
    return C, steps.value, flag


def desync_thresholds(q: float, v: int = V_DEFAULT):
    """(message, move) firing thresholds of a tick of length q."""
    return prob_threshold(min(1.0, v * q)), prob_threshold(q)


def desync_decode_shot(N, q: float, *, v: int = V_DEFAULT, m_max: int = M_MAX_DEFAULT,
                       max_ticks: int = 100000, seed: int = 0, shot: int = 0):
    """Returns (C, ticks, flag) of the uncoordinated decoder."""
    N = np.ascontiguousarray(N, dtype=np.uint8)
    L = N.shape[-1]
    C = np.zeros_like(N)
    ticks = ctypes.c_int32()
    tm, tf = desync_thresholds(q, v)
    flag = _load().qo_desync_decode_shot(N, L, v, m_max, max_ticks, tm, tf, seed, shot, C,
                                         ctypes.byref(ticks))
    return C, ticks.value, flag
