"""Python binding of libbpx (ctypes): argument marshalling only.

Every call forwards to the C ABI declared in ``include/bpx.h``; every step of
the hot path runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream.  The binding fails loudly when the library
has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbpx.so")

# enums of bpx.h
TABLE1, TABLE3, SYSTEMATIC, MOJETTE_A, MOJETTE_B, LITERAL, XCODE = 0, 1, 2, 3, 4, 5, 6
SEARCH_SYSTEMATIC = 1  # bpx_code_search_ex flag
FP32, BF16, BF16X3, MXFP8, EXACT, FP16X3 = 0, 1, 2, 3, 4, 5
OK, ERR_INVAL, ERR_UNSUPPORTED, ERR_UNDECODABLE, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM = range(7)
INFO_STATUS, INFO_RECOVERED, INFO_WAVES, INFO_SURVIVING, INFO_DIRECT, INFO_DEVICE_ERR = range(6)
INFO_LEN = 16

PRECISIONS = {"fp32": FP32, "bf16": BF16, "bf16x3": BF16X3, "mxfp8": MXFP8, "exact": EXACT, "fp16x3": FP16X3}


class BpxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bpx error {code}: {msg}")
        self.code = code


class _CodeInfo(ct.Structure):
    _fields_ = [
        ("variant", ct.c_int), ("n", ct.c_int), ("k", ct.c_int), ("e", ct.c_int),
        ("b", ct.c_int), ("q_e", ct.c_int), ("num_sources", ct.c_int),
        ("num_cells", ct.c_int), ("num_edges", ct.c_int), ("sigma", ct.c_int),
        ("eps", ct.c_double),
        ("col_ptr", ct.POINTER(ct.c_int32)), ("cell_ptr", ct.POINTER(ct.c_int32)),
        ("cell_src", ct.POINTER(ct.c_int32)), ("col_of_cell", ct.POINTER(ct.c_int32)),
        ("heights", ct.POINTER(ct.c_int32)), ("proj_p", ct.POINTER(ct.c_int32)),
        ("proj_q", ct.POINTER(ct.c_int32)),
    ]


class Opts(ct.Structure):
    _fields_ = [("direct_write", ct.c_int), ("compensate_depth", ct.c_int),
                ("peel_ctas", ct.c_int), ("gemm_config", ct.c_int),
                ("stage_events", ct.POINTER(ct.c_void_p)), ("mask_cells", ct.c_int),
                ("fused_encode", ct.c_int)]


STAGE_SCHEDULE, STAGE_B_PREP, STAGE_A_PREP, STAGE_GEMM, STAGE_PEEL = range(5)
NUM_STAGES = 5
STAGE_NAMES = ["schedule", "b_prep", "a_prep", "gemm", "peel"]


class Job(ct.Structure):
    _fields_ = [("code", ct.c_void_p), ("A", ct.c_void_p), ("B", ct.c_void_p), ("C", ct.c_void_p),
                ("erasure_mask", ct.c_void_p), ("info", ct.c_void_p),
                ("M", ct.c_int), ("N", ct.c_int), ("K", ct.c_int), ("h", ct.c_int)]


_lib = None


def lib():
    """Loads libbpx.so (built in-tree by ``build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "paper_1904_11563_gb300.build.build() (no CPU fallback exists)")
    L = ct.CDLL(LIB_PATH)
    vp, i, sz, f32p = ct.c_void_p, ct.c_int, ct.c_size_t, ct.c_void_p
    sig = {
        "bpx_code_build": (i, [i, i, i, i, i, i, ct.POINTER(vp)]),
        "bpx_code_info_get": (i, [vp, ct.POINTER(_CodeInfo)]),
        "bpx_code_free": (None, [vp]),
        "bpx_last_error": (ct.c_char_p, []),
        "bpx_workspace_bytes": (sz, [vp, i, i, i, i, i]),
        "bpx_workspace_init": (i, [vp, vp, sz, vp]),
        "bpx_workspace_info_offset": (sz, [vp]),
        "bpx_schedule": (i, [vp, vp, vp, sz, vp, vp, vp, vp]),
        "bpx_encode": (i, [vp, f32p, i, i, i, vp, f32p, vp]),
        "bpx_coded_products": (i, [vp, f32p, f32p, i, i, i, i, i, vp, sz, f32p, f32p,
                                   ct.POINTER(Opts), vp]),
        "bpx_peel_decode": (i, [vp, f32p, vp, i, i, f32p, i, ct.POINTER(Opts), vp, sz, vp, vp]),
        "bpx_exact_params": (i, [vp, i, ct.POINTER(ct.c_int32)]),
        "bpx_peel_decode_exact": (i, [vp, vp, vp, i, i, f32p, ct.POINTER(Opts), vp, sz, vp, vp]),
        "bpx_coded_matmul": (i, [vp, f32p, f32p, i, i, i, i, i, vp, f32p, ct.POINTER(Opts),
                                 vp, sz, vp, vp]),
        "bpx_coded_matmul_host": (i, [vp, f32p, f32p, i, i, i, i, i, vp, f32p, f32p, f32p, vp,
                                      f32p, ct.POINTER(Opts), vp, sz, vp, vp]),
        "bpx_coded_matmul_host_async": (i, [vp, f32p, f32p, i, i, i, i, i, vp, f32p, f32p, f32p, vp,
                                            f32p, ct.POINTER(Opts), vp, sz, vp, vp]),
        "bpx_schedule_noalloc": (i, [vp, vp, vp, vp, vp, vp]),
        "bpx_schedule_cells": (i, [vp, vp, vp, sz, vp, vp, vp, vp]),
        "bpx_first_decodable": (i, [vp, vp, i, vp, vp]),
        "bpx_bound_k_equals_sigma": (i, [i, i, ct.POINTER(ct.c_int)]),
        "bpx_bound_paterson": (i, [i, i, i, ct.POINTER(ct.c_int)]),
        "bpx_code_from_cells": (i, [i, i, i, i, vp, vp, vp, i, ct.POINTER(vp)]),
        "bpx_code_search": (i, [i, i, i, i, ct.c_longlong, ct.c_ulonglong, ct.POINTER(vp),
                                ct.POINTER(ct.c_longlong)]),
        "bpx_code_search_ex": (i, [i, i, i, i, ct.c_longlong, ct.c_ulonglong, i, i, ct.POINTER(vp),
                                   ct.POINTER(ct.c_longlong)]),
        "bpx_terms_2d": (i, [vp, vp, vp]),
        "bpx_workspace_bytes_2d": (sz, [vp, i, i, i, i, i]),
        "bpx_coded_matmul_2d": (i, [vp, f32p, f32p, i, i, i, i, i, vp, f32p, ct.POINTER(Opts), vp, sz, vp, vp]),
        "bpx_group_create": (i, [ct.POINTER(Job), i, i, ct.POINTER(vp)]),
        "bpx_group_workspace_bytes": (sz, [vp]),
        "bpx_group_init": (i, [vp, vp, sz, vp]),
        "bpx_grouped_run": (i, [vp, ct.POINTER(Opts), vp]),
        "bpx_group_graph_launch": (i, [vp, ct.POINTER(Opts), vp]),
        "bpx_group_set_config": (i, [vp, i, vp]),
        "bpx_group_autotune": (i, [vp, ct.POINTER(ct.c_int), i, vp, ct.POINTER(ct.c_int),
                                   ct.POINTER(ct.c_float)]),
        "bpx_autotune": (i, [vp, f32p, f32p, i, i, i, i, i, vp, f32p, vp, sz, ct.POINTER(ct.c_int), i, vp,
                             ct.POINTER(ct.c_int), ct.POINTER(ct.c_float)]),
        "bpx_group_autotune_peel": (i, [vp, ct.POINTER(ct.c_int), i, vp, ct.POINTER(ct.c_int),
                                        ct.POINTER(ct.c_float)]),
        "bpx_autotune_peel": (i, [vp, f32p, f32p, i, i, i, i, i, vp, f32p, vp, sz, ct.POINTER(ct.c_int), i, vp,
                                  ct.POINTER(ct.c_int), ct.POINTER(ct.c_float)]),
        "bpx_group_free": (None, [vp]),
        "bpx_selftest_wait_timeout": (i, [ct.c_longlong, vp, vp]),
        "bpx_default_opts": (Opts, []),
        "bpx_build_info": (ct.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise BpxError(rc, lib().bpx_last_error().decode())
    return rc


def default_opts(**kw) -> Opts:
    o = lib().bpx_default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Code:
    """A code graph built by the library (bpx_code_build)."""

    def __init__(self, variant, n, k, b, e=-1, q_e=0, handle=None):
        self._h = None
        h = ct.c_void_p()
        if handle is not None:
            h = handle
        else:
            _check(lib().bpx_code_build(variant, n, k, e, b, q_e, ct.byref(h)))
        self._h = h
        info = _CodeInfo()
        _check(lib().bpx_code_info_get(h, ct.byref(info)))
        self.variant, self.n, self.k, self.e, self.b, self.q_e = (
            info.variant, info.n, info.k, info.e, info.b, info.q_e)
        self.num_sources, self.num_cells, self.num_edges = info.num_sources, info.num_cells, info.num_edges
        self.sigma, self.eps = info.sigma, info.eps

        def arr(p, n):
            return np.ctypeslib.as_array(p, shape=(n,)).copy() if n > 0 else np.zeros(0, np.int32)

        self.col_ptr = arr(info.col_ptr, self.n + 1)
        self.cell_ptr = arr(info.cell_ptr, self.num_cells + 1)
        self.cell_src = arr(info.cell_src, self.num_edges)
        self.col_of_cell = arr(info.col_of_cell, self.num_cells)
        self.heights = arr(info.heights, self.n)
        self.proj_p = arr(info.proj_p, self.n)
        self.proj_q = arr(info.proj_q, self.n)

    @property
    def handle(self):
        return self._h

    @property
    def cells(self):
        return [tuple(int(x) for x in self.cell_src[self.cell_ptr[c]:self.cell_ptr[c + 1]])
                for c in range(self.num_cells)]

    def __del__(self):
        if self._h is not None and _lib is not None:
            _lib.bpx_code_free(self._h)
            self._h = None

    # factories
    @classmethod
    def table1(cls):
        return cls(TABLE1, 5, 2, 2)

    @classmethod
    def table3(cls):
        return cls(TABLE3, 5, 3, 3)

    @classmethod
    def systematic(cls, k, e, b):
        return cls(SYSTEMATIC, k + e, k, b)

    @classmethod
    def mojette_a(cls, n, k, b):
        return cls(MOJETTE_A, n, k, b)

    @classmethod
    def mojette_b(cls, n, k, b, q_e):
        return cls(MOJETTE_B, n, k, b, q_e=q_e)

    @classmethod
    def xcode(cls, p):
        """The X-code on p (prime) columns: k = p - 2, b = p, e = 2."""
        return cls(XCODE, p, p - 2, p)

    @classmethod
    def from_columns(cls, n, k, b, columns, e):
        """A code given by its columns, each a list of cells (source tuples)."""
        col_of, ptr, src = [], [0], []
        for j, col in enumerate(columns):
            for cell in col:
                col_of.append(j)
                src.extend(sorted(cell))
                ptr.append(len(src))
        a = [np.ascontiguousarray(x, dtype=np.int32) for x in (col_of, ptr, src)]
        h = ct.c_void_p()
        _check(lib().bpx_code_from_cells(n, k, b, len(col_of), *(x.ctypes.data_as(ct.c_void_p) for x in a), e,
                                         ct.byref(h)))
        return cls(LITERAL, n, k, b, handle=h)

    @classmethod
    def search(cls, n, k, b, sigma, iters=200000, seed=0, systematic=False, threads=1):
        """Equal-height array BP-XOR code search; (code or None, moves taken).
        systematic: the first k columns fixed to single sources; threads:
        independent chains (seeds seed .. seed + threads - 1, iters moves
        each; the lowest chain that found a code wins)."""
        h = ct.c_void_p()
        used = ct.c_longlong()
        rc = lib().bpx_code_search_ex(n, k, b, sigma, iters, seed, SEARCH_SYSTEMATIC if systematic else 0,
                                      threads, ct.byref(h), ct.byref(used))
        if rc == ERR_UNSUPPORTED:
            return None, used.value
        _check(rc)
        return cls(LITERAL, n, k, b, handle=h), used.value

    def columns(self):
        """Cells grouped by column (source tuples)."""
        cells = self.cells
        return [[cells[c] for c in range(self.col_ptr[j], self.col_ptr[j + 1])] for j in range(self.n)]


def workspace_bytes(code: Code, M, N, K, h, precision) -> int:
    return int(lib().bpx_workspace_bytes(code.handle, M, N, K, h, precision))


# ------------------------------------------------------------------ device calls

def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


class Workspace:
    """Device workspace bound to a code (bpx_workspace_init)."""

    def __init__(self, code: Code, M, N, K, h, precision, device="cuda"):
        torch = _torch()
        self.nbytes = workspace_bytes(code, M, N, K, h, precision)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.t = self.buf[off:off + self.nbytes]
        self.code = code
        _check(lib().bpx_workspace_init(code.handle, _ptr(self.t), self.nbytes, _stream()))

    @property
    def ptr(self):
        return _ptr(self.t)

    def info(self):
        """The plan's device info words (a view into the workspace)."""
        torch = _torch()
        off = lib().bpx_workspace_info_offset(self.code.handle)
        return self.t[off:off + 4 * INFO_LEN].view(torch.int32)


def schedule(code: Code, mask, ws: Workspace, cells=False):
    """a1: returns (peel_order int32[S,3], recovered uint8[S], info int32[16])
    on device; cells=True: the mask has one byte per cell."""
    torch = _torch()
    S = code.num_sources
    order = torch.empty((S, 3), dtype=torch.int32, device=mask.device)
    rec = torch.empty(S, dtype=torch.uint8, device=mask.device)
    info = torch.empty(INFO_LEN, dtype=torch.int32, device=mask.device)
    fn = lib().bpx_schedule_cells if cells else lib().bpx_schedule
    _check(fn(code.handle, _ptr(mask), ws.ptr, ws.nbytes, _ptr(order), _ptr(rec), _ptr(info), _stream()))
    return order, rec, info


def encode(code: Code, A, h, ws: Workspace):
    """a2 (materialized): coded rows of the surviving cells, FP32."""
    torch = _torch()
    out = torch.zeros((code.num_cells * h, A.shape[1]), dtype=torch.float32, device=A.device)
    _check(lib().bpx_encode(code.handle, _ptr(A), A.shape[0], A.shape[1], h, ws.ptr, _ptr(out),
                            _stream()))
    return out


def coded_products(code: Code, A, B, h, precision, ws: Workspace, products=None, C=None, opts=None):
    """a3: products[c] = A_c B for surviving cells (num_cells*h x N);
    depth-1 resolvers go to C when C is given."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[1]
    if products is None:
        products = torch.zeros((code.num_cells * h, N), dtype=torch.float32, device=A.device)
    _check(lib().bpx_coded_products(code.handle, _ptr(A), _ptr(B), M, N, K, h, precision, ws.ptr,
                                    ws.nbytes, _ptr(products), _ptr(C),
                                    ct.byref(opts) if opts is not None else None, _stream()))
    return products


def peel_decode(code: Code, products, N, h, C, ws: Workspace, direct_written=False, opts=None, mask=None,
                info=None):
    """a4: numeric peel into C (S*h x N) for the erasure mask `mask` (planned
    first, as bpx_schedule), or along the plan already in ws when mask is
    None."""
    _check(lib().bpx_peel_decode(code.handle, _ptr(products), _ptr(mask) if mask is not None else None, N, h,
                                 _ptr(C), int(direct_written), ct.byref(opts) if opts is not None else None,
                                 ws.ptr, ws.nbytes, _ptr(info) if info is not None else None, _stream()))
    return C


def bound(kind, k, b, sigma=None) -> int:
    """Bounds on n (host only): kind 'k_equals_sigma' or 'paterson'."""
    out = ct.c_int()
    if kind == "k_equals_sigma":
        _check(lib().bpx_bound_k_equals_sigma(k, b, ct.byref(out)))
    elif kind == "paterson":
        _check(lib().bpx_bound_paterson(k, b, sigma, ct.byref(out)))
    else:
        raise ValueError(kind)
    return out.value


def first_decodable(code: Code, order):
    """Online peel over cells arriving in `order` (host only): (number of
    arrivals after which every source is recovered, or -1; sources recovered
    after each arrival)."""
    order = np.ascontiguousarray(order, dtype=np.int32)
    rec = np.zeros(len(order), dtype=np.int32)
    first = ct.c_int32()
    _check(lib().bpx_first_decodable(code.handle, order.ctypes.data_as(ct.c_void_p), len(order),
                                     rec.ctypes.data_as(ct.c_void_p), ct.byref(first)))
    return int(first.value), rec


def exact_params(code: Code, K) -> dict:
    """Exact-slice representation for this code and K (host only):
    digit width w, digit planes S, fixed-point bits, K elements per exact
    FP32 segment, padded K."""
    out = (ct.c_int32 * 5)()
    _check(lib().bpx_exact_params(code.handle, K, out))
    return dict(zip(("w", "S", "bits", "seg", "Kp"), list(out)))


def exact_products(code: Code, A, B, h, ws: Workspace, planes=None, opts=None):
    """a3 with exact slices: the S int32 diagonal planes (S, num_cells*h, N)."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[1]
    S = exact_params(code, K)["S"]
    if planes is None:
        planes = torch.zeros((S, code.num_cells * h, N), dtype=torch.int32, device=A.device)
    _check(lib().bpx_coded_products(code.handle, _ptr(A), _ptr(B), M, N, K, h, EXACT, ws.ptr, ws.nbytes,
                                    _ptr(planes), None, ct.byref(opts) if opts is not None else None,
                                    _stream()))
    return planes


def peel_decode_exact(code: Code, planes, N, h, C, ws: Workspace, opts=None, mask=None, info=None):
    """a4 with exact slices: exact integer peel of the diagonal planes into C
    (mask as for peel_decode)."""
    _check(lib().bpx_peel_decode_exact(code.handle, _ptr(planes), _ptr(mask) if mask is not None else None, N, h,
                                       _ptr(C), ct.byref(opts) if opts is not None else None, ws.ptr, ws.nbytes,
                                       _ptr(info) if info is not None else None, _stream()))
    return C


def terms_2d(code: Code):
    """Two-dimensional scheme factoring (host only): (products per cell,
    {total, gray, a_operands, b_operands})."""
    per = np.zeros(code.num_cells, dtype=np.int32)
    summ = np.zeros(4, dtype=np.int32)
    _check(lib().bpx_terms_2d(code.handle, per.ctypes.data_as(ct.c_void_p), summ.ctypes.data_as(ct.c_void_p)))
    return per, dict(zip(("total", "gray", "a_operands", "b_operands"), (int(x) for x in summ)))


class Workspace2D:
    """Device workspace of the two-dimensional scheme (bound to a code)."""

    def __init__(self, code: Code, M, N, K, h, precision, device="cuda"):
        torch = _torch()
        self.nbytes = int(lib().bpx_workspace_bytes_2d(code.handle, M, N, K, h, precision))
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.base = self.buf[off:off + self.nbytes]
        self.code = code
        _check(lib().bpx_workspace_init(code.handle, ct.c_void_p(self.base.data_ptr()), self.nbytes, _stream()))

    @property
    def ptr(self):
        return ct.c_void_p(self.base.data_ptr())


def coded_matmul_2d(code: Code, A, B, h, precision, mask, ws: Workspace2D, C=None, opts=None, info=None):
    """Two-dimensional scheme: C ((b h) x N) with block (z, l) = A_z B_l."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[1]
    if C is None:
        C = torch.zeros((code.b * h, N), dtype=torch.float32, device=A.device)
    if info is None:
        info = torch.zeros(INFO_LEN, dtype=torch.int32, device=A.device)
    _check(lib().bpx_coded_matmul_2d(code.handle, _ptr(A), _ptr(B), M, N, K, h, precision, _ptr(mask), _ptr(C),
                                     ct.byref(opts) if opts is not None else None, ws.ptr, ws.nbytes, _ptr(info),
                                     _stream()))
    return C, info


def alloc_C(code: Code, h, N, device="cuda"):
    torch = _torch()
    return torch.zeros((code.num_sources * h, N), dtype=torch.float32, device=device)


def coded_matmul(code: Code, A, B, h, precision, mask, ws: Workspace, C=None, opts=None, info=None):
    """Whole path; returns (C [S*h x N], info int32[16] on device)."""
    torch = _torch()
    M, K = A.shape
    N = B.shape[1]
    if C is None:
        C = alloc_C(code, h, N, A.device)
    if info is None:
        info = torch.zeros(INFO_LEN, dtype=torch.int32, device=A.device)
    _check(lib().bpx_coded_matmul(code.handle, _ptr(A), _ptr(B), M, N, K, h, precision, _ptr(mask),
                                  _ptr(C), ct.byref(opts) if opts is not None else None, ws.ptr,
                                  ws.nbytes, _ptr(info), _stream()))
    return C, info


def coded_matmul_host(code: Code, hA, hB, h, precision, hmask, hC, dA, dB, dmask, dC,
                      ws: Workspace, opts=None):
    """End-to-end from host buffers (copies inside the call); returns
    (status, info numpy int32[16])."""
    M, K = hA.shape
    N = hB.shape[1]
    info = np.zeros(INFO_LEN, dtype=np.int32)
    rc = lib().bpx_coded_matmul_host(
        code.handle, _ptr(hA), _ptr(hB), M, N, K, h, precision, _ptr(hmask), _ptr(hC),
        _ptr(dA), _ptr(dB), _ptr(dmask), _ptr(dC), ct.byref(opts) if opts is not None else None,
        ws.ptr, ws.nbytes, info.ctypes.data_as(ct.c_void_p), _stream())
    if rc not in (OK, ERR_UNDECODABLE):
        raise BpxError(rc, lib().bpx_last_error().decode())
    return rc, info


def coded_matmul_host_async(code: Code, hA, hB, h, precision, hmask, hC, dA, dB, dmask, dC,
                            ws: Workspace, hinfo, opts=None, stream=None):
    """Enqueues copies in, the path and copies out on `stream` (default: the
    current torch stream) without synchronizing; hC and hinfo (a pinned
    int32[16] tensor) are valid once the stream has completed."""
    M, K = hA.shape
    N = hB.shape[1]
    st = _stream() if stream is None else ct.c_void_p(stream.cuda_stream)
    _check(lib().bpx_coded_matmul_host_async(
        code.handle, _ptr(hA), _ptr(hB), M, N, K, h, precision, _ptr(hmask), _ptr(hC),
        _ptr(dA), _ptr(dB), _ptr(dmask), _ptr(dC), ct.byref(opts) if opts is not None else None,
        ws.ptr, ws.nbytes, _ptr(hinfo), st))


def autotune(code: Code, A, B, h, precision, mask, ws: Workspace, C=None, configs=None):
    """Tile autotuner of the tensor-core GEMM for one job; returns (config, ms)."""
    M, K = A.shape
    N = B.shape[1]
    if C is None:
        C = alloc_C(code, h, N, A.device)
    best, ms = ct.c_int(), ct.c_float()
    arr = (ct.c_int * len(configs))(*configs) if configs else None
    _check(lib().bpx_autotune(code.handle, _ptr(A), _ptr(B), M, N, K, h, precision, _ptr(mask), _ptr(C),
                              ws.ptr, ws.nbytes, arr, len(configs) if configs else 0, _stream(),
                              ct.byref(best), ct.byref(ms)))
    return best.value, ms.value


def autotune_peel(code: Code, A, B, h, precision, mask, ws: Workspace, C=None, ctas=None):
    """Peel-schedule autotuner for one job: returns (peel_ctas, ms) for
    bpx_opts.peel_ctas."""
    M, K = A.shape
    N = B.shape[1]
    if C is None:
        C = alloc_C(code, h, N, A.device)
    best, ms = ct.c_int(), ct.c_float()
    arr = (ct.c_int * len(ctas))(*ctas) if ctas else None
    _check(lib().bpx_autotune_peel(code.handle, _ptr(A), _ptr(B), M, N, K, h, precision, _ptr(mask), _ptr(C),
                                   ws.ptr, ws.nbytes, arr, len(ctas) if ctas else 0, _stream(),
                                   ct.byref(best), ct.byref(ms)))
    return best.value, ms.value


class Group:
    """A batch of coded multiplications run together (bpx_group_*).

    jobs: list of dicts with keys code, A, B, C, mask, h (torch tensors on
    the device; C with S*h rows) and optionally info (int32[16] tensor)."""

    def __init__(self, jobs, precision=BF16X3, device="cuda"):
        torch = _torch()
        self._h = None
        self.jobs = jobs
        arr = (Job * len(jobs))()
        for i, j in enumerate(jobs):
            A, B = j["A"], j["B"]
            arr[i] = Job(j["code"].handle, A.data_ptr(), B.data_ptr(), j["C"].data_ptr(),
                         j["mask"].data_ptr(), j["info"].data_ptr() if j.get("info") is not None else None,
                         A.shape[0], B.shape[1], A.shape[1], j["h"])
        self._arr = arr
        h = ct.c_void_p()
        _check(lib().bpx_group_create(arr, len(jobs), precision, ct.byref(h)))
        self._h = h
        self.nbytes = int(lib().bpx_group_workspace_bytes(h))
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.ws = self.buf[off:off + self.nbytes]
        _check(lib().bpx_group_init(h, _ptr(self.ws), self.nbytes, _stream()))

    def run(self, opts=None):
        _check(lib().bpx_grouped_run(self._h, ct.byref(opts) if opts is not None else None, _stream()))

    def graph_launch(self, opts=None):
        _check(lib().bpx_group_graph_launch(self._h, ct.byref(opts) if opts is not None else None, _stream()))

    def set_config(self, config):
        _check(lib().bpx_group_set_config(self._h, config, _stream()))

    def autotune(self, configs=None):
        best, ms = ct.c_int(), ct.c_float()
        arr = (ct.c_int * len(configs))(*configs) if configs else None
        _check(lib().bpx_group_autotune(self._h, arr, len(configs) if configs else 0, _stream(),
                                        ct.byref(best), ct.byref(ms)))
        return best.value, ms.value

    def autotune_peel(self, targets=None):
        """Peel-schedule autotuner: (CTAs per job aimed at, ms of the grouped peel)."""
        best, ms = ct.c_int(), ct.c_float()
        arr = (ct.c_int * len(targets))(*targets) if targets else None
        _check(lib().bpx_group_autotune_peel(self._h, arr, len(targets) if targets else 0, _stream(),
                                             ct.byref(best), ct.byref(ms)))
        return best.value, ms.value

    def __del__(self):
        if self._h is not None and _lib is not None:
            _lib.bpx_group_free(self._h)
            self._h = None
