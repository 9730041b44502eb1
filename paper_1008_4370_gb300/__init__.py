"""GB300-native Log-Fourier sum-product decoder for (2,k)-regular non-binary LDPC codes.

Python binding of libnbfd (include/nbfd.h): the functions below carry the C names and only
marshal arguments -- every step of decoding runs in the library's CUDA kernels. Device buffers
are torch CUDA tensors (contiguous, of the dtype the header states) or raw device addresses.
The library is loaded on first use; if it has not been built the call raises instead of
falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "NbfdError", "lib", "FORM_FP32_DIRECT", "FORM_BF16_HGEMM", "FORM_FP16_HGEMM", "FORM_FP32_FWHT", "FORM_FP32_TC",
    "FORM_FP64_DIRECT",
    "nbfd_code_create", "nbfd_code_destroy", "nbfd_code_info", "nbfd_code_edge_order",
    "nbfd_code_index_map", "nbfd_field_index_map", "nbfd_decode_workspace_size", "nbfd_decode", "nbfd_decode_noalloc", "nbfd_init_messages",
    "nbfd_decode_batch_workspace_size", "nbfd_decode_batch", "nbfd_autotune", "nbfd_autotune_result", "BATCH_AUTOTUNE", "decode_batch",
    "STORE_F16", "UNFUSED", "TCGEN05", "MMA_SYNC", "KERNEL_FUSED", "nbfd_init_messages_f16", "nbfd_check_update_f16", "nbfd_diag_wait_expiry",
    "nbfd_diag_preset_status", "nbfd_diag_fp32_rate", "nbfd_logsp_init", "nbfd_logsp_check_update",
    "nbfd_logsp_var_update",
    "nbfd_last_decode_stats",
    "nbfd_check_update", "nbfd_var_update", "nbfd_syndrome", "nbfd_prof_enable", "nbfd_prof_get",
    "nbfd_last_error", "nbfd_status_string", "Code", "decode", "nbfd_srv_create", "nbfd_srv_submit",
    "nbfd_srv_poll", "nbfd_srv_stats", "nbfd_srv_destroy", "nbfd_srv_clock", "nbfd_srv_submit_many",
    "nbfd_srv_collect", "nbfd_srv_register", "nbfd_srv_worker_times",
]

FORM_FP32_DIRECT = 0
FORM_BF16_HGEMM = 1
FORM_FP16_HGEMM = 2
FORM_FP32_FWHT = 3
FORM_FP32_TC = 4
FORM_FP64_DIRECT = 5  # the direct form with the variable node's sums in FP64
DECIDE_SYMBOL = 0x100  # OR into a form: symbol-MAP tentative decisions
SUPPORTED_FORMS = (FORM_FP32_DIRECT, FORM_FP32_FWHT, FORM_BF16_HGEMM, FORM_FP16_HGEMM, FORM_FP32_TC, FORM_FP64_DIRECT)
TC_FORMS = (FORM_BF16_HGEMM, FORM_FP16_HGEMM, FORM_FP32_TC)  # need m = 8
KERNEL_INIT, KERNEL_CHECK, KERNEL_VAR, KERNEL_SYNDROME, KERNEL_TAIL, KERNEL_FUSED = 0, 1, 2, 3, 4, 5
NOALLOC_SCRATCH_BYTES = 64 << 20

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libnbfd.so")

# (name, restype, argtypes) of every exported symbol declared in include/nbfd.h
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = [
    ("nbfd_code_create", _I, [_I, _I, _I, _I, ctypes.c_uint32, _I, _P, _P, _P, ctypes.POINTER(_P)]),
    ("nbfd_code_destroy", None, [_P]),
    ("nbfd_code_info", _I, [_P, _P, _P, _P, _P]),
    ("nbfd_code_edge_order", _I, [_P, _P]),
    ("nbfd_code_index_map", _I, [_P, _P]),
    ("nbfd_field_index_map", _I, [_I, ctypes.c_uint32, _P]),
    ("nbfd_decode_workspace_size", ctypes.c_size_t, [_P, _I, _I, _I]),
    ("nbfd_decode", _I, [_P, _I, _P, _I, _I, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    ("nbfd_decode_noalloc", _I, [_P, _I, _P, _I, _I, _P, _P, _P, _P]),
    ("nbfd_decode_batch_workspace_size", ctypes.c_size_t, [_I, _P, _P, _I, _I]),
    ("nbfd_decode_batch", _I, [_I, _P, _P, _P, _I, _I, _I, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    ("nbfd_autotune", _I, [_P, _I, _I, _P]),
    ("nbfd_init_messages_f16", _I, [_P, _I, _P, _P, _P]),
    ("nbfd_diag_wait_expiry", _I, [ctypes.c_longlong, _P]),
    ("nbfd_diag_preset_status", _I, [ctypes.c_int32]),
    ("nbfd_diag_fp32_rate", _I, [_I, _I, ctypes.c_longlong, _P, _P, _P]),
    ("nbfd_logsp_init", _I, [_P, _I, _P, _P, _P]),
    ("nbfd_logsp_check_update", _I, [_P, _I, _P, _P, _P]),
    ("nbfd_logsp_var_update", _I, [_P, _I, _P, _P, _P, _P, _P]),
    ("nbfd_last_decode_stats", _I, [_P]),
    ("nbfd_check_update_f16", _I, [_P, _I, _P, _P, _P]),
    ("nbfd_autotune_result", _I, [_P, _I, _I, _P, _P, _P, _P, _P]),
    ("nbfd_init_messages", _I, [_P, _I, _P, _P, _P, _P]),
    ("nbfd_check_update", _I, [_P, _I, _P, _P, _P]),
    ("nbfd_var_update", _I, [_P, _I, _I, _P, _P, _P, _P, _P, _P]),
    ("nbfd_syndrome", _I, [_P, _I, _P, _P, _P, _P, _P]),
    ("nbfd_srv_create", _I, [ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    ("nbfd_srv_submit", _I, [_P, _P, _P, _I, ctypes.POINTER(ctypes.c_uint64)]),
    ("nbfd_srv_poll", _I, [_P, ctypes.c_uint64, _P, _P, _P, _P]),
    ("nbfd_srv_stats", _I, [_P, _P, _P, _P, _P]),
    ("nbfd_srv_clock", ctypes.c_double, []),
    ("nbfd_srv_submit_many", _I, [_P, _P, _I, _P, _I, _P, _P]),
    ("nbfd_srv_collect", _I, [_P, _I, _P, _P, _P, _P]),
    ("nbfd_srv_destroy", None, [_P]),
    ("nbfd_srv_register", _I, [_P, _P]),
    ("nbfd_srv_worker_times", _I, [_P, _P]),
    ("nbfd_prof_enable", _I, [_I]),
    ("nbfd_prof_get", _I, [_I, _P, _P, _P]),
    ("nbfd_last_error", ctypes.c_char_p, []),
    ("nbfd_status_string", ctypes.c_char_p, [_I]),
]

_lib = None


class NbfdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib() -> ctypes.CDLL:
    """The loaded libnbfd (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1008_4370_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise NbfdError(status, nbfd_last_error())


def _dptr(t, dtype=None):
    """Device address of a torch CUDA tensor (or pass an int / None through)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def nbfd_last_error() -> str:
    return lib().nbfd_last_error().decode()


def nbfd_status_string(status: int) -> str:
    return lib().nbfd_status_string(status).decode()


def nbfd_code_create(N, M, k, m, prim_poly, edge_check, edge_var, edge_h):
    ec = np.ascontiguousarray(edge_check, dtype=np.int32)
    ev = np.ascontiguousarray(edge_var, dtype=np.int32)
    eh = np.ascontiguousarray(edge_h, dtype=np.uint16)
    h = ctypes.c_void_p()
    _check(lib().nbfd_code_create(int(N), int(M), int(k), int(m), int(prim_poly), len(ec),
                                  ec.ctypes.data, ev.ctypes.data, eh.ctypes.data, ctypes.byref(h)))
    return h.value


def nbfd_code_destroy(handle):
    lib().nbfd_code_destroy(handle)


def nbfd_code_info(handle):
    vals = [ctypes.c_int() for _ in range(4)]
    _check(lib().nbfd_code_info(handle, *[ctypes.byref(v) for v in vals]))
    return tuple(v.value for v in vals)


def nbfd_code_edge_order(handle, n_edges):
    out = np.empty(n_edges, dtype=np.int32)
    _check(lib().nbfd_code_edge_order(handle, out.ctypes.data))
    return out


def nbfd_code_index_map(handle, q):
    out = np.empty((q, q), dtype=np.uint8)
    _check(lib().nbfd_code_index_map(handle, out.ctypes.data))
    return out


def nbfd_field_index_map(m, prim_poly):
    q = 1 << int(m)
    out = np.empty((q, q), dtype=np.uint8)
    _check(lib().nbfd_field_index_map(int(m), int(prim_poly), out.ctypes.data))
    return out


def nbfd_decode_workspace_size(handle, n_frames, max_iter, form):
    return int(lib().nbfd_decode_workspace_size(handle, int(n_frames), int(max_iter), int(form)))


def nbfd_decode(handle, n_frames, llr, max_iter, form, symbols, syndrome_ok, iters,
                workspace=None, workspace_bytes=0, stream=None):
    import torch
    _check(lib().nbfd_decode(handle, int(n_frames), _dptr(llr, torch.float32), int(max_iter), int(form),
                             _dptr(symbols),
                             _dptr(syndrome_ok, torch.uint8), _dptr(iters, torch.int32),
                             _dptr(workspace), int(workspace_bytes), _stream(stream)))


BATCH_AUTOTUNE = 1
STORE_F16 = 0x200  # form flag: messages stored as IEEE half (FWHT form, m = 8)
UNFUSED = 0x400  # form flag: per-iteration kernels even where the fused GF(16) kernel applies
TCGEN05 = 0x800  # form flag: tensor-core forms on tcgen05 (TMEM accumulators)
MMA_SYNC = 0x1000  # form flag: tensor-core forms on warp-level mma.sync


def nbfd_last_decode_stats():
    """(frame, iteration) pairs of this thread's last nbfd_decode where the Fourier-domain
    syndrome cleared while H x_hat != 0."""
    v = ctypes.c_longlong()
    _check(lib().nbfd_last_decode_stats(ctypes.byref(v)))
    return v.value


def nbfd_diag_wait_expiry(budget_cycles, stream=None):
    """Runs the bounded-wait expiry path on purpose; raises NbfdError(NBFD_ETIMEDOUT)."""
    _check(lib().nbfd_diag_wait_expiry(int(budget_cycles), _stream(stream)))


def nbfd_diag_fp32_rate(packed=0, blocks_per_sm=4, iters=1 << 20, stream=None):
    """Measured FP32 FMA rate: (TFLOP/s, ms of the timed launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().nbfd_diag_fp32_rate(int(packed), int(blocks_per_sm), int(iters), ctypes.byref(t),
                                     ctypes.byref(ms), _stream(stream)))
    return t.value, ms.value


def nbfd_logsp_init(handle, n_frames, llr, v2c, stream=None):
    """Conventional Log-SP INITIALIZATION (Section 2.2): lambda0 on both edges of every variable."""
    import torch
    _check(lib().nbfd_logsp_init(handle, int(n_frames), _dptr(llr, torch.float32), _dptr(v2c, torch.float32),
                                 _stream(stream)))


def nbfd_logsp_check_update(handle, n_frames, v2c, c2v, stream=None):
    """Conventional Log-SP CHECK TO VARIABLE: the log-convolution of the other k - 1 messages."""
    import torch
    _check(lib().nbfd_logsp_check_update(handle, int(n_frames), _dptr(v2c, torch.float32),
                                         _dptr(c2v, torch.float32), _stream(stream)))


def nbfd_logsp_var_update(handle, n_frames, llr, c2v, v2c, symbols=None, stream=None):
    """Conventional Log-SP VARIABLE TO CHECK + argmax TENTATIVE DECISION."""
    import torch
    _check(lib().nbfd_logsp_var_update(handle, int(n_frames), _dptr(llr, torch.float32), _dptr(c2v, torch.float32),
                                       _dptr(v2c, torch.float32), _dptr(symbols), _stream(stream)))


def nbfd_diag_preset_status(value):
    """The calling thread's next nbfd_decode / nbfd_decode_noalloc starts its device status word
    at `value` (one-shot); a nonzero value must come back as NbfdError(NBFD_ETIMEDOUT)."""
    _check(lib().nbfd_diag_preset_status(int(value)))


def nbfd_init_messages_f16(handle, n_frames, llr, v2c, stream=None):
    _check(lib().nbfd_init_messages_f16(handle, int(n_frames), _dptr(llr), _dptr(v2c), _stream(stream)))


def nbfd_check_update_f16(handle, n_frames, v2c, c2v, stream=None):
    _check(lib().nbfd_check_update_f16(handle, int(n_frames), _dptr(v2c), _dptr(c2v), _stream(stream)))


def _ptr_array(ptrs, ctype=ctypes.c_void_p):
    arr = (ctype * len(ptrs))(*[p if p is not None else 0 for p in ptrs])
    return arr


def nbfd_decode_batch_workspace_size(handles, n_frames, max_iter, form):
    n = len(handles)
    return lib().nbfd_decode_batch_workspace_size(n, ctypes.cast(_ptr_array(handles), _P),
                                                  ctypes.cast((ctypes.c_int * n)(*n_frames), _P),
                                                  int(max_iter), int(form))


def nbfd_decode_batch(handles, n_frames, llrs, max_iter, form, flags, symbols, syndrome_ok, iters,
                      workspace=None, workspace_bytes=0, stream=None):
    """One call over several codes: lists (one entry per code) of handles, frame counts, LLR
    tensors and output tensors."""
    import torch
    n = len(handles)
    _check(lib().nbfd_decode_batch(
        n, ctypes.cast(_ptr_array(handles), _P), ctypes.cast((ctypes.c_int * n)(*n_frames), _P),
        ctypes.cast(_ptr_array([_dptr(x, torch.float32) for x in llrs]), _P), int(max_iter), int(form),
        int(flags), ctypes.cast(_ptr_array([_dptr(x) for x in symbols]), _P),
        ctypes.cast(_ptr_array([_dptr(x, torch.uint8) for x in syndrome_ok]), _P),
        ctypes.cast(_ptr_array([_dptr(x, torch.int32) for x in iters]), _P),
        _dptr(workspace), int(workspace_bytes), _stream(stream)))


def nbfd_autotune(handle, n_frames, form, stream=None):
    _check(lib().nbfd_autotune(handle, int(n_frames), int(form), _stream(stream)))


def nbfd_autotune_result(handle, n_frames, form):
    """(check warps, check stages, check blocks per SM, variable-node blocks per SM, variable-node
    warps per block or 0)."""
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().nbfd_autotune_result(handle, int(n_frames), int(form), *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def nbfd_decode_noalloc(handle, n_frames, llr, max_iter, form, symbols, syndrome_ok, iters, stream=None):
    """nbfd_decode without any device allocation: scratch lives in a fixed array of
    NOALLOC_SCRATCH_BYTES inside the library (see include/nbfd.h for who needs this)."""
    import torch
    _check(lib().nbfd_decode_noalloc(handle, int(n_frames), _dptr(llr, torch.float32), int(max_iter), int(form),
                                     _dptr(symbols), _dptr(syndrome_ok, torch.uint8), _dptr(iters, torch.int32),
                                     _stream(stream)))


def nbfd_init_messages(handle, n_frames, llr, lambda0, v2c, stream=None):
    _check(lib().nbfd_init_messages(handle, int(n_frames), _dptr(llr), _dptr(lambda0), _dptr(v2c),
                                    _stream(stream)))


def nbfd_check_update(handle, n_frames, v2c, c2v, stream=None):
    _check(lib().nbfd_check_update(handle, int(n_frames), _dptr(v2c), _dptr(c2v), _stream(stream)))


def nbfd_var_update(handle, n_frames, form, llr, c2v, v2c, symbols=None, fsyn=None, stream=None):
    _check(lib().nbfd_var_update(handle, int(n_frames), int(form), _dptr(llr), _dptr(c2v), _dptr(v2c),
                                 _dptr(symbols), _dptr(fsyn), _stream(stream)))


def nbfd_syndrome(handle, n_frames, symbols, fsyn, fourier, exact, stream=None):
    _check(lib().nbfd_syndrome(handle, int(n_frames), _dptr(symbols), _dptr(fsyn), _dptr(fourier),
                               _dptr(exact), _stream(stream)))


def nbfd_srv_create(mem_budget_bytes, form):
    h = ctypes.c_void_p()
    _check(lib().nbfd_srv_create(int(mem_budget_bytes), int(form), ctypes.byref(h)))
    return h.value


def nbfd_srv_submit(srv, code_handle, llr_host, max_iter):
    x = np.ascontiguousarray(llr_host, dtype=np.float32)
    t = ctypes.c_uint64()
    _check(lib().nbfd_srv_submit(srv, code_handle, x.ctypes.data, int(max_iter), ctypes.byref(t)))
    return t.value


def nbfd_srv_poll(srv, ticket, n_symbols):
    """None while pending, else (symbols uint16 array, ok, iters, latency_s)."""
    sym = np.empty(n_symbols, dtype=np.uint16)
    ok = ctypes.c_uint8()
    it = ctypes.c_int32()
    lat = ctypes.c_double()
    r = lib().nbfd_srv_poll(srv, ctypes.c_uint64(ticket), sym.ctypes.data, ctypes.byref(ok), ctypes.byref(it),
                            ctypes.byref(lat))
    if r < 0:
        _check(r)
    if r == 0:
        return None
    return sym, ok.value, it.value, lat.value


def nbfd_srv_clock():
    return float(lib().nbfd_srv_clock())


def nbfd_srv_submit_many(srv, code_handle, llr_host, max_iter, arrival=None):
    x = np.ascontiguousarray(llr_host, dtype=np.float32)
    n = int(x.shape[0])
    t = np.empty(n, dtype=np.uint64)
    arr = None if arrival is None else np.ascontiguousarray(arrival, dtype=np.float64)
    _check(lib().nbfd_srv_submit_many(srv, code_handle, n, x.ctypes.data, int(max_iter),
                                      None if arr is None else arr.ctypes.data, t.ctypes.data))
    return t


def nbfd_srv_collect(srv, max_n=4096):
    """(tickets, ok, iters, latency_s) of up to max_n retired frames."""
    t = np.empty(max_n, dtype=np.uint64)
    ok = np.empty(max_n, dtype=np.uint8)
    it = np.empty(max_n, dtype=np.int32)
    lat = np.empty(max_n, dtype=np.float64)
    n = lib().nbfd_srv_collect(srv, int(max_n), t.ctypes.data, ok.ctypes.data, it.ctypes.data, lat.ctypes.data)
    if n < 0:
        _check(n)
    return t[:n], ok[:n], it[:n], lat[:n]


def nbfd_srv_stats(srv):
    vals = [ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_size_t()]
    _check(lib().nbfd_srv_stats(srv, *[ctypes.byref(v) for v in vals]))
    return tuple(v.value for v in vals)


def nbfd_srv_register(srv, code_handle):
    """Create the code's pool now (device memory, streams, pinned staging)."""
    _check(lib().nbfd_srv_register(srv, code_handle))


def nbfd_srv_worker_times(srv):
    """Cumulative worker seconds per phase: admission, issue, wait, retire, idle."""
    out = np.zeros(5, dtype=np.float64)
    _check(lib().nbfd_srv_worker_times(srv, out.ctypes.data))
    return dict(zip(("admission", "issue", "wait", "retire", "idle"), out.tolist()))


def nbfd_srv_destroy(srv):
    lib().nbfd_srv_destroy(srv)


def nbfd_prof_enable(kernel_mask: int):
    """Time the kernels whose bit (1 << KERNEL_*) is set; 0 disables, 0x3F times all."""
    _check(lib().nbfd_prof_enable(int(kernel_mask)))


def nbfd_prof_get(kernel: int):
    ms = ctypes.c_double()
    launches = ctypes.c_longlong()
    units = ctypes.c_longlong()
    _check(lib().nbfd_prof_get(int(kernel), ctypes.byref(ms), ctypes.byref(launches), ctypes.byref(units)))
    return ms.value, launches.value, units.value


class Code:
    """Owner of an nbfd_code handle built from a code dict (N, M, k, m, poly, edge arrays)."""

    def __init__(self, code: dict):
        self.N, self.M, self.k, self.m = int(code["N"]), int(code["M"]), int(code["k"]), int(code["m"])
        self.q = 1 << self.m
        self.E = 2 * self.N
        self.handle = nbfd_code_create(self.N, self.M, self.k, self.m, int(code["poly"]),
                                       code["edge_check"], code["edge_var"], code["edge_h"])

    def close(self):
        if self.handle:
            nbfd_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decode(code: Code, llr, max_iter: int, form: int = FORM_FP32_DIRECT, workspace=None, stream=None):
    """Allocate outputs (torch, on llr's device) and run nbfd_decode; returns (symbols, ok, iters)."""
    import torch
    F = int(llr.shape[0])
    dev = llr.device
    sym = torch.empty((F, code.N), dtype=torch.int16, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    it = torch.empty(F, dtype=torch.int32, device=dev)
    need = nbfd_decode_workspace_size(code.handle, F, max_iter, form)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    nbfd_decode(code.handle, F, llr, max_iter, form, sym.data_ptr(), ok, it, workspace, workspace.numel(),
                stream)
    return sym, ok, it


def decode_batch(codes, llrs, max_iter: int, form: int = FORM_FP32_FWHT, flags: int = 0, stream=None):
    """Allocate outputs and run nbfd_decode_batch over several codes; returns a list of
    (symbols, ok, iters) per code."""
    import torch
    dev = llrs[0].device
    ns = [int(x.shape[0]) for x in llrs]
    outs = [(torch.empty((n, c.N), dtype=torch.int16, device=dev), torch.empty(n, dtype=torch.uint8, device=dev),
             torch.empty(n, dtype=torch.int32, device=dev)) for c, n in zip(codes, ns)]
    handles = [c.handle for c in codes]
    need = nbfd_decode_batch_workspace_size(handles, ns, max_iter, form)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    nbfd_decode_batch(handles, ns, llrs, max_iter, form, flags, [o[0].data_ptr() for o in outs],
                      [o[1] for o in outs], [o[2] for o in outs], ws, ws.numel(), stream)
    return outs
