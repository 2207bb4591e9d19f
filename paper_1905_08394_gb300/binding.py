"""ctypes binding of libpeps_gb300.so (C ABI in include/peps_gb300.h).

Argument marshalling only: every step of the amplitude path runs in the
library's CUDA kernels.  The functions keep the C names (peps_create,
peps_apply_1q, ...).  Device memory (the workspace) and the CUDA stream come
from PyTorch.  There is no CPU fallback: if the shared library is missing the
import fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes as ct
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = Path(os.environ.get("PEPS_GB300_LIB", _PKG / "libpeps_gb300.so"))

PEPS_OK = 0
PEPS_EINVAL = -1
PEPS_ENOTADJ = -2
PEPS_ENOMEM = -3
PEPS_ECUDA = -4
PEPS_ETIMEOUT = -5
PEPS_ESTATE = -6
PEPS_EUNSUPPORTED = -7

PEPS_FLAG_MARGINALS = 16

PEPS_SCHEME_COLUMNS = 0
PEPS_SCHEME_QUADRANTS = 1
SCHEMES = {"columns": PEPS_SCHEME_COLUMNS, "quadrants": PEPS_SCHEME_QUADRANTS}

PEPS_FP32_SIMT = 0
PEPS_TF32 = 1
PEPS_BF16 = 2
PEPS_BF16X3 = 3
PEPS_FP16 = 4
PEPS_FP16X3 = 5
PRECISIONS = {"fp32": PEPS_FP32_SIMT, "tf32": PEPS_TF32, "bf16": PEPS_BF16,
              "bf16x3": PEPS_BF16X3, "fp16": PEPS_FP16, "fp16x3": PEPS_FP16X3}

PEPS_FLAG_REBUILD = 1
PEPS_FLAG_TIMING = 2
PEPS_FLAG_NO_TC = 4
PEPS_FLAG_GRAPH = 8
PEPS_FLAG_ESTIMATE = 32
PEPS_FLAG_HOLD_TIES = 64
PEPS_FLAG_STEPWISE = 128

EXPORTED = ("peps_create", "peps_destroy", "peps_apply_1q", "peps_apply_cz", "peps_apply_2q",
            "peps_bond_dim",
            "peps_workspace_bytes", "peps_amplitudes", "peps_amplitudes_device",
            "peps_get_stats", "peps_cz_count", "peps_last_error", "peps_version",
            "peps_plan_info_get", "peps_amplitudes_noalloc", "peps_output_ties",
            "peps_plan_steps", "peps_launch_log")


class peps_c128(ct.Structure):
    _fields_ = [("re", ct.c_double), ("im", ct.c_double)]


class peps_opts(ct.Structure):
    _fields_ = [("precision", ct.c_int32), ("flags", ct.c_int32),
                ("prefix_cols", ct.c_int32), ("prefix_group", ct.c_int32),
                ("max_lanes", ct.c_int32), ("n_sliced", ct.c_int32),
                ("sliced_cz", ct.POINTER(ct.c_uint32)), ("slice_ids", ct.POINTER(ct.c_uint64)),
                ("n_slice_ids", ct.c_int64), ("watchdog_ns", ct.c_int64),
                ("n_fixed", ct.c_int32), ("tc_ksplit", ct.c_int32),
                ("fixed_cz", ct.POINTER(ct.c_uint32)), ("fixed_s", ct.POINTER(ct.c_uint8)),
                ("tc_kchunk", ct.c_int32), ("tc_cluster", ct.c_int32),
                ("fuse_rows", ct.c_int32), ("scheme", ct.c_int32),
                ("measured_mask", ct.c_uint64), ("tc_epi", ct.c_int32), ("pad_", ct.c_int32)]


class peps_stats(ct.Structure):
    _fields_ = [("launches_total", ct.c_int64), ("launches_evolve", ct.c_int64),
                ("launches_operand", ct.c_int64), ("launches_contract", ct.c_int64),
                ("launches_contract_tc", ct.c_int64), ("launches_finalize", ct.c_int64),
                ("contract_flops", ct.c_double), ("contract_bytes", ct.c_double),
                ("contract_ms", ct.c_double), ("contract_tc_ms", ct.c_double),
                ("contract_tc_flops", ct.c_double), ("contract_tc_bytes", ct.c_double),
                ("n_steps", ct.c_int64), ("n_lanes", ct.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class peps_plan_info(ct.Structure):
    _fields_ = [("n_steps", ct.c_int64), ("max_entries", ct.c_int64),
                ("flops_per_chain", ct.c_double), ("bytes_per_chain", ct.c_double),
                ("flops_call", ct.c_double), ("bytes_call", ct.c_double),
                ("n_launches", ct.c_int64), ("n_tc_launches", ct.c_int64),
                ("n_slices", ct.c_int64), ("lanes", ct.c_int64),
                ("flops_lower", ct.c_double), ("n_lower_bits", ct.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class peps_step_info(ct.Structure):
    _fields_ = [("M", ct.c_int64), ("K", ct.c_int32), ("N", ct.c_int32),
                ("sites", ct.c_int32), ("variants", ct.c_int32), ("tensor_cores", ct.c_int32),
                ("part", ct.c_int32), ("launches", ct.c_int64), ("flops", ct.c_double),
                ("P", ct.c_int64), ("Mr", ct.c_int64), ("dv", ct.c_int32), ("dh", ct.c_int32),
                ("open_leg", ct.c_int32), ("fused_dot", ct.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class peps_launch_info(ct.Structure):
    _fields_ = [("flops", ct.c_double), ("bytes", ct.c_double), ("ms", ct.c_float),
                ("tensor_cores", ct.c_int32), ("step", ct.c_int32), ("pad_", ct.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class PepsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"peps error {code}: {msg}")
        self.code = code


_lib = None


def load() -> ct.CDLL:
    """Load the shared library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ct.CDLL(str(LIB_PATH))
    P = ct.c_void_p
    lib.peps_create.argtypes = [ct.c_int, ct.c_int, ct.POINTER(P)]
    lib.peps_destroy.argtypes = [P]
    lib.peps_apply_1q.argtypes = [P, ct.c_int, ct.c_int, ct.POINTER(peps_c128)]
    lib.peps_apply_cz.argtypes = [P, ct.c_int, ct.c_int, ct.c_int, ct.c_int]
    lib.peps_apply_2q.argtypes = [P, ct.c_int, ct.c_int, ct.c_int, ct.c_int,
                                  ct.POINTER(peps_c128)]
    lib.peps_bond_dim.argtypes = [P, ct.c_int, ct.c_int, ct.c_int, ct.c_int,
                                  ct.POINTER(ct.c_int64)]
    lib.peps_workspace_bytes.argtypes = [P, ct.c_int64, ct.POINTER(peps_opts),
                                         ct.POINTER(ct.c_size_t)]
    lib.peps_amplitudes.argtypes = [P, P, ct.c_int64, P, ct.POINTER(peps_opts), P, ct.c_size_t, P]
    lib.peps_amplitudes_device.argtypes = [P, P, ct.c_int64, P, ct.POINTER(peps_opts), P,
                                           ct.c_size_t, P]
    lib.peps_amplitudes_noalloc.argtypes = [P, P, ct.c_int64, P, ct.POINTER(peps_opts), P]
    lib.peps_get_stats.argtypes = [P, ct.POINTER(peps_stats)]
    lib.peps_cz_count.argtypes = [P, ct.POINTER(ct.c_int64)]
    lib.peps_plan_info_get.argtypes = [P, ct.c_int64, ct.POINTER(peps_opts),
                                       ct.POINTER(peps_plan_info)]
    lib.peps_output_ties.argtypes = [P, P, P, P, P, ct.c_int64, ct.POINTER(ct.c_int64)]
    lib.peps_launch_log.argtypes = [P, ct.POINTER(peps_launch_info), ct.c_int64,
                                    ct.POINTER(ct.c_int64)]
    lib.peps_plan_steps.argtypes = [P, ct.c_int64, ct.POINTER(peps_opts),
                                    ct.POINTER(peps_step_info), ct.c_int64,
                                    ct.POINTER(ct.c_int64)]
    lib.peps_last_error.restype = ct.c_char_p
    lib.peps_version.restype = ct.c_char_p
    for name in EXPORTED:
        if name not in ("peps_last_error", "peps_version"):
            getattr(lib, name).restype = ct.c_int
    _lib = lib
    return lib


def _check(rc: int) -> None:
    if rc != PEPS_OK:
        raise PepsError(rc, load().peps_last_error().decode())


# ---------------------------------------------------------------------------
# The C functions, one to one
# ---------------------------------------------------------------------------

def peps_create(R: int, C: int) -> ct.c_void_p:
    h = ct.c_void_p()
    _check(load().peps_create(R, C, ct.byref(h)))
    return h


def peps_destroy(h) -> None:
    _check(load().peps_destroy(h))


def peps_apply_1q(h, r: int, c: int, U) -> None:
    U = np.asarray(U, dtype=np.complex128).reshape(4)
    arr = (peps_c128 * 4)(*[peps_c128(float(u.real), float(u.imag)) for u in U])
    _check(load().peps_apply_1q(h, r, c, arr))


def peps_apply_cz(h, r0: int, c0: int, r1: int, c1: int) -> None:
    _check(load().peps_apply_cz(h, r0, c0, r1, c1))


def peps_apply_2q(h, r0: int, c0: int, r1: int, c1: int, G) -> None:
    """A general two-qubit gate: G 4x4, rows 2*t0 + t1, columns 2*s0 + s1,
    qubit (r0, c0) first."""
    G = np.asarray(G, dtype=np.complex128).reshape(4, 4)
    arr = (peps_c128 * 16)(*[peps_c128(float(v.real), float(v.imag)) for v in G.reshape(-1)])
    _check(load().peps_apply_2q(h, r0, c0, r1, c1, arr))


def peps_bond_dim(h, r0: int, c0: int, r1: int, c1: int) -> int:
    d = ct.c_int64()
    _check(load().peps_bond_dim(h, r0, c0, r1, c1, ct.byref(d)))
    return d.value


def peps_cz_count(h) -> int:
    d = ct.c_int64()
    _check(load().peps_cz_count(h, ct.byref(d)))
    return d.value


def make_opts(precision="fp32", flags: int = 0, prefix_cols: int = 0, prefix_group: int = 0,
              max_lanes: int = 0, sliced_cz=None, slice_ids=None, watchdog_ns: int = 0,
              fixed_cz=None, fixed_s=None, tc_kchunk: int = 0, tc_cluster: int = 0,
              tc_epi: int = 0,
              fuse_rows: int = 0, scheme="columns", tc_ksplit: int = 0,
              measured_mask=None, hold_ties: bool = False):
    """peps_opts plus the arrays it points to (keep both alive).  With
    measured_mask (an int, bit q = qubit q measured) the call returns the
    marginal probabilities of the measured bits (PEPS_FLAG_MARGINALS); with
    hold_ties the CZ bits the output fixes are held (PEPS_FLAG_HOLD_TIES)."""
    o = peps_opts()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.flags = flags | (PEPS_FLAG_HOLD_TIES if hold_ties else 0)
    o.prefix_cols = prefix_cols
    o.prefix_group = prefix_group
    o.max_lanes = max_lanes
    keep = []
    if sliced_cz is not None and len(sliced_cz):
        a = np.ascontiguousarray(sliced_cz, dtype=np.uint32)
        keep.append(a)
        o.n_sliced = len(a)
        o.sliced_cz = a.ctypes.data_as(ct.POINTER(ct.c_uint32))
    if slice_ids is not None:
        b = np.ascontiguousarray(slice_ids, dtype=np.uint64)
        keep.append(b)
        o.n_slice_ids = len(b)
        o.slice_ids = b.ctypes.data_as(ct.POINTER(ct.c_uint64))
    o.watchdog_ns = watchdog_ns
    o.tc_kchunk = tc_kchunk
    o.tc_cluster = tc_cluster
    o.tc_epi = tc_epi
    o.fuse_rows = fuse_rows
    o.tc_ksplit = tc_ksplit
    if measured_mask is not None:
        o.flags |= PEPS_FLAG_MARGINALS
        o.measured_mask = int(measured_mask)
    o.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    if fixed_cz is not None and len(fixed_cz):
        f = np.ascontiguousarray(fixed_cz, dtype=np.uint32)
        v = np.ascontiguousarray(fixed_s, dtype=np.uint8)
        assert len(f) == len(v)
        keep += [f, v]
        o.n_fixed = len(f)
        o.fixed_cz = f.ctypes.data_as(ct.POINTER(ct.c_uint32))
        o.fixed_s = v.ctypes.data_as(ct.POINTER(ct.c_uint8))
    return o, keep


def peps_workspace_bytes(h, n: int, opts: peps_opts) -> int:
    b = ct.c_size_t()
    _check(load().peps_workspace_bytes(h, n, ct.byref(opts), ct.byref(b)))
    return b.value


def peps_amplitudes(h, bitstrings: np.ndarray, opts: peps_opts, ws_ptr: int, ws_bytes: int,
                    stream: int) -> np.ndarray:
    bits = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    out = np.zeros(len(bits), dtype=np.complex128)
    _check(load().peps_amplitudes(h, bits.ctypes.data, len(bits), out.ctypes.data,
                                  ct.byref(opts), ws_ptr, ws_bytes, stream))
    return out


def peps_amplitudes_device(h, d_bits_ptr: int, n: int, d_out_ptr: int, opts: peps_opts,
                           ws_ptr: int, ws_bytes: int, stream: int) -> None:
    _check(load().peps_amplitudes_device(h, d_bits_ptr, n, d_out_ptr, ct.byref(opts), ws_ptr,
                                         ws_bytes, stream))


def peps_amplitudes_noalloc(h, d_bits_ptr: int, n: int, d_out_ptr: int, opts: peps_opts,
                            stream: int) -> None:
    """Allocation-free variant (static device scratch inside the library)."""
    _check(load().peps_amplitudes_noalloc(h, d_bits_ptr, n, d_out_ptr, ct.byref(opts), stream))


def peps_get_stats(h) -> dict:
    s = peps_stats()
    _check(load().peps_get_stats(h, ct.byref(s)))
    return s.as_dict()


def peps_plan_info_get(h, n: int, opts: peps_opts) -> dict:
    i = peps_plan_info()
    _check(load().peps_plan_info_get(h, n, ct.byref(opts), ct.byref(i)))
    return i.as_dict()


def peps_output_ties(h, with_src: bool = False) -> list:
    """[(cz ordinal, kind, flip)] (with_src: a fourth item, the source CZ of a
    linked bit, else -1): kind 1 = the Schmidt bit is `flip`, kind 2 = it is
    x_q XOR flip for every output bitstring x (q = the CZ's lower-index qubit),
    kind 3 = it is the bit of CZ `src` (same edge) XOR flip."""
    n = ct.c_int64()
    _check(load().peps_output_ties(h, None, None, None, None, 0, ct.byref(n)))
    k = n.value
    cz = np.zeros(max(k, 1), dtype=np.uint32)
    kind = np.zeros(max(k, 1), dtype=np.uint8)
    flip = np.zeros(max(k, 1), dtype=np.uint8)
    src = np.zeros(max(k, 1), dtype=np.uint32)
    _check(load().peps_output_ties(h, cz.ctypes.data, kind.ctypes.data, flip.ctypes.data,
                                   src.ctypes.data, k, ct.byref(n)))
    if with_src:
        return [(int(cz[i]), int(kind[i]), int(flip[i]),
                 -1 if int(src[i]) == 0xFFFFFFFF else int(src[i])) for i in range(k)]
    return [(int(cz[i]), int(kind[i]), int(flip[i])) for i in range(k)]


def peps_plan_steps(h, n: int, opts: peps_opts) -> list:
    """The plan's contraction steps (peps_step_info as dicts), in sweep order."""
    k = ct.c_int64()
    _check(load().peps_plan_steps(h, n, ct.byref(opts), None, 0, ct.byref(k)))
    arr = (peps_step_info * max(k.value, 1))()
    _check(load().peps_plan_steps(h, n, ct.byref(opts), arr, k.value, ct.byref(k)))
    return [arr[i].as_dict() for i in range(k.value)]


def peps_launch_log(h) -> list:
    """Contraction launches of the last timed call (peps_launch_info as dicts)."""
    k = ct.c_int64()
    _check(load().peps_launch_log(h, None, 0, ct.byref(k)))
    arr = (peps_launch_info * max(k.value, 1))()
    _check(load().peps_launch_log(h, arr, k.value, ct.byref(k)))
    return [arr[i].as_dict() for i in range(k.value)]


def peps_last_error() -> str:
    return load().peps_last_error().decode()


def peps_version() -> str:
    return load().peps_version().decode()
