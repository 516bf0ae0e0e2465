"""Python binding of libdl (include/dl.h): argument marshalling only.

Every step of every path runs in the CUDA library; this module converts numpy arrays (host
memory, DL_MEM_HOST) or torch CUDA tensors (device memory, DL_MEM_DEVICE) into pointers and
sizes, calls the C ABI and raises :class:`DLError` on a non-zero status.  There is no CPU
fallback: if libdl.so is missing or the GPU is not an sm_103 part, calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdl.so")

DL_OK, DL_EINVAL, DL_ENOMEM, DL_EDEVICE, DL_ETIMEOUT, DL_EBUSY, DL_ENOTCONV, DL_ECANCELED, \
    DL_ENOTIMPL = range(9)
STATUS_NAMES = ["DL_OK", "DL_EINVAL", "DL_ENOMEM", "DL_EDEVICE", "DL_ETIMEOUT", "DL_EBUSY",
                "DL_ENOTCONV", "DL_ECANCELED", "DL_ENOTIMPL"]
PATHS = {"auto": 0, "fp64": 1, "mixed": 2, "bool_fp8": 3, "fp8": 3}
DL_MEM_HOST, DL_MEM_DEVICE = 0, 1

EXPORTED = ["dl_create", "dl_destroy", "dl_last_error", "dl_set_stream", "dl_tc_closure", "dl_tc_closure_bits",
            "dl_sg_least_model", "dl_sg_real", "dl_tail_recursive", "dl_tail_recursive_real", "dl_tail_system", "dl_transposed", "dl_compose",
            "dl_program_create", "dl_program_destroy", "dl_program_set", "dl_program_run", "dl_program_get",
            "dl_program_describe", "dl_autotune", "dl_tc_batch", "dl_submit", "dl_poll", "dl_cancel",
            "dl_tc_closure_noalloc", "dl_selftest_wait_timeout"]
NOALLOC_MAX_N = 2048


class DLError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status
        self.message = message


class Config(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_slots", ctypes.c_int32), ("refine_tol", ctypes.c_double),
                ("refine_max_iters", ctypes.c_int32), ("guard_tau", ctypes.c_double),
                ("wait_timeout_s", ctypes.c_double), ("autotune", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p)]


class Stats(ctypes.Structure):
    _fields_ = [("path_used", ctypes.c_int32), ("eps_used", ctypes.c_double),
                ("iters", ctypes.c_int32), ("final_resid", ctypes.c_double),
                ("guard_flagged", ctypes.c_int64), ("rows_rechecked", ctypes.c_int64),
                ("recheck_sweeps", ctypes.c_int32), ("model_ones", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("ms_refine", ctypes.c_double),
                ("ms_epilogue", ctypes.c_double), ("tflops_equiv", ctypes.c_double),
                ("gpu_launches", ctypes.c_int32), ("gemm_launches", ctypes.c_int32),
                ("ms_gemm", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("ms_queue", ctypes.c_double), ("ms_latency", ctypes.c_double),
                ("sweep_launches", ctypes.c_int32), ("ms_sweep", ctypes.c_double),
                ("sweep_bytes", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TailEq(ctypes.Structure):
    _fields_ = [("A1", ctypes.c_void_p), ("B0", ctypes.c_void_p), ("nterms", ctypes.c_int32),
                ("B", ctypes.POINTER(ctypes.c_void_p)), ("j", ctypes.POINTER(ctypes.c_int32)),
                ("eps", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("base", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("mem", ctypes.c_int), ("path", ctypes.c_int),
                ("out_bits", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load libdl.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1608_00139_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.dl_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(Config)]
            L.dl_destroy.argtypes = [vp]
            L.dl_last_error.argtypes = []
            L.dl_last_error.restype = ctypes.c_char_p
            L.dl_set_stream.argtypes = [vp, vp]
            L.dl_tc_closure.argtypes = [vp, i32, vp, ctypes.c_int, f64, f64, ctypes.c_int, vp, vp,
                                        ctypes.POINTER(Stats)]
            L.dl_tc_closure_bits.argtypes = [vp, i32, vp, ctypes.c_int, f64, f64, ctypes.c_int, vp, vp,
                                             ctypes.POINTER(Stats)]
            L.dl_sg_least_model.argtypes = [vp, i32, vp, vp, ctypes.c_int, f64, f64, ctypes.c_int,
                                            vp, ctypes.POINTER(Stats)]
            L.dl_tail_recursive.argtypes = [vp, i32, vp, vp, ctypes.c_int, f64, f64, ctypes.c_int, vp, vp,
                                            ctypes.POINTER(Stats)]
            L.dl_sg_real.argtypes = [vp, i32, vp, vp, ctypes.c_int, f64, ctypes.c_int, vp, vp,
                                     ctypes.POINTER(Stats)]
            L.dl_transposed.argtypes = [vp, i32, vp, ctypes.c_int, f64, f64, ctypes.c_int, vp, vp,
                                        ctypes.POINTER(Stats)]
            L.dl_tail_recursive_real.argtypes = [vp, i32, vp, vp, i32, vp, vp, ctypes.c_int, f64, ctypes.c_int, vp, vp,
                                                 ctypes.POINTER(Stats)]
            L.dl_tail_system.argtypes = [vp, i32, i32, vp, ctypes.c_int, ctypes.c_int, vp, vp,
                                         ctypes.POINTER(Stats)]
            L.dl_compose.argtypes = [vp, i32, vp, vp, ctypes.c_int, vp, ctypes.POINTER(Stats)]
            L.dl_autotune.argtypes = [vp, i32, i32, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
            L.dl_program_create.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(vp)]
            L.dl_program_destroy.argtypes = [vp]
            L.dl_program_set.argtypes = [vp, ctypes.c_char_p, i32, vp, ctypes.c_int]
            L.dl_program_run.argtypes = [vp, ctypes.POINTER(Stats)]
            L.dl_program_get.argtypes = [vp, ctypes.c_char_p, vp, ctypes.c_int]
            L.dl_program_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
            L.dl_tc_batch.argtypes = [vp, i32, vp, vp, ctypes.c_int, vp, ctypes.POINTER(Stats)]
            L.dl_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
            L.dl_poll.argtypes = [vp, ctypes.c_uint64, i64, ctypes.POINTER(Stats)]
            L.dl_cancel.argtypes = [vp, ctypes.c_uint64]
            L.dl_tc_closure_noalloc.argtypes = [i32, vp, vp, vp, ctypes.POINTER(i32)]
            L.dl_selftest_wait_timeout.argtypes = [vp, f64]
            for f in EXPORTED:
                if f != "dl_last_error":
                    getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != DL_OK:
        msg = lib().dl_last_error() or b""
        raise DLError(rc, msg.decode(errors="replace"))


def words(n: int) -> int:
    return (n + 63) // 64


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _square_u8(x, sync=True):
    """(pointer, n, mem, keepalive) of a square 0/1 uint8 matrix (numpy or torch CUDA).
    sync=False leaves the wait for torch's pending writes to the caller."""
    if _is_torch(x):
        import torch
        if not x.is_cuda:
            x = x.numpy()
        else:
            if x.dtype != torch.uint8 or x.dim() != 2 or x.shape[0] != x.shape[1]:
                raise ValueError("expected a square torch.uint8 CUDA tensor")
            x = x.contiguous()
            # the library reads on its own stream: finish torch's pending writes first
            if sync:
                torch.cuda.current_stream(x.device).synchronize()
            return x.data_ptr(), int(x.shape[0]), DL_MEM_DEVICE, x
    a = np.ascontiguousarray(x, dtype=np.uint8)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected a square matrix")
    return a.ctypes.data, int(a.shape[0]), DL_MEM_HOST, a


def _bits_u64(x, n: int, sync=True):
    """(pointer, mem, keepalive) of an n x ceil(n/64) array of 64-bit words (numpy or torch
    CUDA)."""
    shape = (int(n), words(int(n)))
    if _is_torch(x):
        import torch
        if not x.is_cuda:
            x = x.numpy()
        else:
            if x.dtype not in (torch.int64, torch.uint64) or tuple(x.shape) != shape:
                raise ValueError(f"expected a {shape} int64 CUDA tensor")
            x = x.contiguous()
            if sync:
                torch.cuda.current_stream(x.device).synchronize()
            return x.data_ptr(), DL_MEM_DEVICE, x
    a = np.ascontiguousarray(x)
    if a.dtype not in (np.uint64, np.int64) or a.shape != shape:
        raise ValueError(f"expected a {shape} array of 64-bit words")
    return a.ctypes.data, DL_MEM_HOST, a


def _alloc_bits(n: int, mem: int, like=None):
    if mem == DL_MEM_DEVICE:
        import torch
        # no fill kernel: the library writes every word, on its own stream
        t = torch.empty((n, words(n)), dtype=torch.int64, device=like.device)
        return t, t.data_ptr()
    a = np.zeros((n, words(n)), dtype=np.uint64)
    return a, a.ctypes.data


class Context:
    """A libdl context on one GPU.  ``stream``: a torch.cuda.Stream or raw cudaStream_t."""

    def __init__(self, device: int = 0, stream=None, **cfg):
        c = Config()
        for k, v in cfg.items():
            setattr(c, k, v.encode() if isinstance(v, str) else v)
        h = ctypes.c_void_p()
        _check(lib().dl_create(ctypes.byref(h), int(device), ctypes.byref(c)))
        self._h = h
        self._inflight = {}  # ticket -> buffers the library may still read or write
        self._programs = weakref.WeakSet()  # programs on this context: closed before it
        if stream is not None:
            self.set_stream(stream)

    def close(self) -> None:
        if getattr(self, "_h", None):
            for prog in list(getattr(self, "_programs", ())):
                prog.close()  # a program's destruction uses its context
            lib().dl_destroy(self._h)  # waits for running requests
            self._h = None
            self._inflight = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream) -> None:
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib().dl_set_stream(self._h, ctypes.c_void_p(raw or 0)))

    def tc_closure(self, E, eps: float = 0.0, thr: float = 0.0, path: str = "auto",
                   rtilde: bool = False, out=None):
        """Least model of the closure program; returns (bits, stats[, R~]).

        ``out``: optional preallocated output (same memory kind as E, n x ceil(n/64) 64-bit
        words, e.g. a pinned numpy array), written in place."""
        p, n, mem, keep = _square_u8(E)
        if out is None:
            bits, bp = _alloc_bits(n, mem, keep)
        else:
            if tuple(out.shape) != (n, words(n)):
                raise ValueError("out must have shape (n, ceil(n/64))")
            bits = out
            bp = out.data_ptr() if _is_torch(out) else out.ctypes.data
        rt, rp = None, None
        if rtilde:
            if mem == DL_MEM_DEVICE:
                import torch
                rt = torch.empty((n, n), dtype=torch.float64, device=keep.device)
                rp = rt.data_ptr()
            else:
                rt = np.zeros((n, n), dtype=np.float64)
                rp = rt.ctypes.data
        st = Stats()
        _check(lib().dl_tc_closure(self._h, n, p, mem, float(eps), float(thr), PATHS[path], bp, rp,
                                   ctypes.byref(st)))
        return (bits, st.as_dict(), rt) if rtilde else (bits, st.as_dict())

    def tc_closure_bits(self, Eb, n: int, eps: float = 0.0, thr: float = 0.0, path: str = "auto",
                        rtilde: bool = False, out=None):
        """The closure of a bit-packed E (n x ceil(n/64) words, LSB first: a numpy uint64/int64
        array or an int64 CUDA tensor); returns (bits, stats[, R~]) like tc_closure."""
        p, mem, keep = _bits_u64(Eb, n)
        if out is None:
            bits, bp = _alloc_bits(n, mem, keep)
        else:
            if tuple(out.shape) != (n, words(n)):
                raise ValueError("out must have shape (n, ceil(n/64))")
            bits = out
            bp = out.data_ptr() if _is_torch(out) else out.ctypes.data
        rt, rp = None, None
        if rtilde:
            if mem == DL_MEM_DEVICE:
                import torch
                rt = torch.empty((n, n), dtype=torch.float64, device=keep.device)
                rp = rt.data_ptr()
            else:
                rt = np.zeros((n, n), dtype=np.float64)
                rp = rt.ctypes.data
        st = Stats()
        _check(lib().dl_tc_closure_bits(self._h, int(n), p, mem, float(eps), float(thr), PATHS[path], bp, rp,
                                        ctypes.byref(st)))
        return (bits, st.as_dict(), rt) if rtilde else (bits, st.as_dict())

    def sg_least_model(self, P, B=None, eps: float = 0.0, thr: float = 0.0,
                       path: str = "auto"):
        """Least model of the same-generation program; returns (bits, stats)."""
        p, n, mem, keep = _square_u8(P)
        bptr, keepb = None, None
        if B is not None:
            bptr, nb, memb, keepb = _square_u8(B)
            if nb != n or memb != mem:
                raise ValueError("B must match P in size and memory kind")
        bits, bp = _alloc_bits(n, mem, keep)
        st = Stats()
        _check(lib().dl_sg_least_model(self._h, n, p, bptr, mem, float(eps), float(thr),
                                       PATHS[path], bp, ctypes.byref(st)))
        return bits, st.as_dict()

    def tail_recursive(self, B0, A, eps: float = 0.0, path: str = "auto", rtilde: bool = False):
        """One equation of the tail recursive class, R~ = eps (A + B0 R~) (Sec. 6.1); returns
        (bits of the model, stats[, R~])."""
        pb, n, mem, keep = _square_u8(B0)
        pa, na, mema, keepa = _square_u8(A)
        if na != n or mema != mem:
            raise ValueError("A must match B0 in size and memory kind")
        bits, bp = _alloc_bits(n, mem, keep)
        rt, rp = None, None
        if rtilde:
            if mem == DL_MEM_DEVICE:
                import torch
                rt = torch.empty((n, n), dtype=torch.float64, device=keep.device)
                rp = rt.data_ptr()
            else:
                rt = np.zeros((n, n), dtype=np.float64)
                rp = rt.ctypes.data
        st = Stats()
        _check(lib().dl_tail_recursive(self._h, n, pb, pa, mem, float(eps), 0.0, PATHS[path], bp, rp,
                                       ctypes.byref(st)))
        return (bits, st.as_dict(), rt) if rtilde else (bits, st.as_dict())

    def _real_out(self, n, mem, keep):
        if mem == DL_MEM_DEVICE:
            import torch
            rt = torch.empty((n, n), dtype=torch.float64, device=keep.device)
            return rt, rt.data_ptr()
        rt = np.zeros((n, n), dtype=np.float64)
        return rt, rt.ctypes.data

    def tail_recursive_real(self, B0, A1, terms, eps: float = 0.0, path: str = "mixed", rtilde: bool = True):
        """R~ = eps (A1 + B0 R~ + sum_k B_k R_k) with real lower solutions R_k (Sec. 6.1);
        terms = [(B_k, R_k)].  B0 / A1 may be None.  Returns (bits, stats[, R~])."""
        ref = next(x for x in [B0, A1] + [b for b, _ in terms] if x is not None)
        _, n, mem, keep = _square_u8(ref)
        keepalive, bps, rps = [], [], []
        sb0 = _square_u8(B0) if B0 is not None else (None, n, mem, None)
        sa1 = _square_u8(A1) if A1 is not None else (None, n, mem, None)
        for sx in (sb0, sa1):
            if sx[1] != n or sx[2] != mem:
                raise ValueError("B0 and A1 must match the terms in size and memory kind")
        keepalive += [sb0[3], sa1[3]]
        pb0, pa1 = sb0[0], sa1[0]
        for b, r in terms:
            pb, nb, memb, kb = _square_u8(b)
            if nb != n or memb != mem:
                raise ValueError("terms must match in size and memory kind")
            if mem == DL_MEM_DEVICE:
                if not (r.dtype == __import__("torch").float64 and r.is_cuda and r.is_contiguous()):
                    raise ValueError("R_k must be a contiguous float64 CUDA tensor")
                rp = r.data_ptr()
            else:
                r = np.ascontiguousarray(r, dtype=np.float64)
                rp = r.ctypes.data
            keepalive += [kb, r]
            bps.append(pb)
            rps.append(rp)
        bits, bp = _alloc_bits(n, mem, keep)
        rt, rp_out = self._real_out(n, mem, keep) if rtilde else (None, None)
        k = len(terms)
        barr = (ctypes.c_void_p * max(k, 1))(*bps)
        rarr = (ctypes.c_void_p * max(k, 1))(*rps)
        st = Stats()
        _check(lib().dl_tail_recursive_real(self._h, n, pb0, pa1, k, barr, rarr, mem, float(eps), PATHS[path],
                                            bp, rp_out, ctypes.byref(st)))
        return (bits, st.as_dict(), rt) if rtilde else (bits, st.as_dict())

    def tail_system(self, eqs, path: str = "mixed", rtilde: bool = True):
        """A layered tail recursive system (Sec. 6.1): eqs[h] = dict(A1=, B0=, terms=[(B, j)],
        eps=) with j < h.  Returns (bits per equation, stats[, R~ per equation])."""
        ref = next(x for eq in eqs for x in [eq.get("A1"), eq.get("B0")] + [b for b, _ in eq.get("terms", [])]
                   if x is not None)
        _, n, mem, keep = _square_u8(ref)
        keepalive, structs = [], []
        def held(x):
            if x is None:
                return None
            p_, n_, mem_, k_ = _square_u8(x)
            if n_ != n or mem_ != mem:
                raise ValueError("every matrix must match in size and memory kind")
            keepalive.append(k_)
            return p_

        for eq in eqs:
            pa = held(eq.get("A1"))
            pb = held(eq.get("B0"))
            terms = eq.get("terms", [])
            bptrs = (ctypes.c_void_p * max(len(terms), 1))(*[held(b) for b, _ in terms])
            js = (ctypes.c_int32 * max(len(terms), 1))(*[int(j) for _, j in terms])
            keepalive += [bptrs, js]
            structs.append(TailEq(pa, pb, len(terms), ctypes.cast(bptrs, ctypes.POINTER(ctypes.c_void_p)),
                                  ctypes.cast(js, ctypes.POINTER(ctypes.c_int32)), float(eq.get("eps", 0.0) or 0.0)))
        m = len(eqs)
        arr = (TailEq * m)(*structs)
        outs = [_alloc_bits(n, mem, keep) for _ in range(m)]
        obits = (ctypes.c_void_p * m)(*[p for _, p in outs])
        rts = [self._real_out(n, mem, keep) for _ in range(m)] if rtilde else []
        ort = (ctypes.c_void_p * m)(*[p for _, p in rts]) if rtilde else None
        st = Stats()
        _check(lib().dl_tail_system(self._h, n, m, arr, mem, PATHS[path], obits, ort, ctypes.byref(st)))
        bits = [b for b, _ in outs]
        return (bits, st.as_dict(), [r for r, _ in rts]) if rtilde else (bits, st.as_dict())

    def transposed(self, R1, eps: float = 0.0, path: str = "auto", rtilde: bool = False):
        """The transposed class, r2(x,z) <- r1(x,z); r2(x,z) <- r1(x,y), r2(z,y) (Sec. 6.2);
        returns (bits of the model, stats[, R~2 as float64 in R1's memory kind])."""
        p, n, mem, keep = _square_u8(R1)
        bits, bp = _alloc_bits(n, mem, keep)
        rt, rp = None, None
        if rtilde:
            if mem == DL_MEM_DEVICE:
                import torch
                rt = torch.empty((n, n), dtype=torch.float64, device=keep.device)
                rp = rt.data_ptr()
            else:
                rt = np.zeros((n, n), dtype=np.float64)
                rp = rt.ctypes.data
        st = Stats()
        _check(lib().dl_transposed(self._h, n, p, mem, float(eps), 0.0, PATHS[path], bp, rp, ctypes.byref(st)))
        return (bits, st.as_dict(), rt) if rtilde else (bits, st.as_dict())

    def sg_real(self, P, B=None, eps: float = 0.0, path: str = "auto", bits: bool = True):
        """Real S~ = eps (B + P S~ P^T) of same generation (Sec. 7.2); returns (S~, bits or
        None, stats), S~ as float64 in P's memory kind."""
        p, n, mem, keep = _square_u8(P)
        bptr, keepb = None, None
        if B is not None:
            bptr, nb, memb, keepb = _square_u8(B)
            if nb != n or memb != mem:
                raise ValueError("B must match P in size and memory kind")
        if mem == DL_MEM_DEVICE:
            import torch
            x = torch.empty((n, n), dtype=torch.float64, device=keep.device)
            xp = x.data_ptr()
        else:
            x = np.zeros((n, n), dtype=np.float64)
            xp = x.ctypes.data
        out, bp = (_alloc_bits(n, mem, keep) if bits else (None, None))
        st = Stats()
        _check(lib().dl_sg_real(self._h, n, p, bptr, mem, float(eps), PATHS[path], xp, bp, ctypes.byref(st)))
        return x, out, st.as_dict()

    def autotune(self, n: int, force: bool = False) -> dict:
        """Tuned choices for problems of size n (dl_autotune): measured now, or from this context's
        table or the cache; returns the report as a dict."""
        import json
        buf = ctypes.create_string_buffer(4096)
        need = ctypes.c_size_t()
        _check(lib().dl_autotune(self._h, int(n), 1 if force else 0, buf, len(buf), ctypes.byref(need)))
        if need.value >= len(buf):
            raise RuntimeError("dl_autotune report longer than expected")
        return json.loads(buf.value.decode())

    def program(self, text: str) -> "Program":
        """A linear Datalog program (the class C_lin of Sec. 5) bound to this context."""
        return Program(self, text)

    def compose(self, R1, R2):
        """Bits of min1(R1 R2), the join of Sec. 2; returns (bits, stats)."""
        p1, n, mem, k1 = _square_u8(R1)
        p2, n2, mem2, k2 = _square_u8(R2)
        if n2 != n or mem2 != mem:
            raise ValueError("R1 and R2 must match in size and memory kind")
        bits, bp = _alloc_bits(n, mem, k1)
        st = Stats()
        _check(lib().dl_compose(self._h, n, p1, p2, mem, bp, ctypes.byref(st)))
        return bits, st.as_dict()

    def tc_batch(self, Es):
        """Closure of each matrix in ``Es`` in one batched call; returns (bits list, stats)."""
        parts = [_square_u8(e, sync=False) for e in Es]
        if not parts:
            return [], Stats().as_dict()
        mems = {m for _, _, m, _ in parts}
        if len(mems) != 1:
            raise ValueError("all matrices must live in the same memory kind")
        mem = mems.pop()
        if mem == DL_MEM_DEVICE:
            import torch
            devs = {keep.device for _, _, _, keep in parts}
            for d in devs:
                torch.cuda.current_stream(d).synchronize()
            if len(devs) == 1:
                # one allocation, one view per model (the library writes every word)
                sizes = [n * words(n) for _, n, _, _ in parts]
                flat = torch.empty(sum(sizes), dtype=torch.int64, device=devs.pop())
                views = [v.view(n, words(n)) for v, (_, n, _, _) in zip(flat.split(sizes), parts)]
                outs = [(v, v.data_ptr()) for v in views]
            else:
                outs = [_alloc_bits(n, mem, keep) for _, n, _, keep in parts]
        else:
            outs = [_alloc_bits(n, mem, keep) for _, n, _, keep in parts]
        cnt = len(parts)
        ns = (ctypes.c_int32 * cnt)(*[n for _, n, _, _ in parts])
        ptrs = (ctypes.c_void_p * cnt)(*[p for p, _, _, _ in parts])
        optrs = (ctypes.c_void_p * cnt)(*[bp for _, bp in outs])
        st = Stats()
        _check(lib().dl_tc_batch(self._h, cnt, ns, ptrs, mem, optrs, ctypes.byref(st)))
        return [b for b, _ in outs], st.as_dict()

    def tc_batch_flat(self, buf, ns, offsets):
        """dl_tc_batch over instances stored back to back in one buffer: instance k is the
        ns[k] x ns[k] row-major matrix at byte offsets[k] of ``buf`` (a 1-D uint8 torch CUDA
        tensor or numpy array).  Returns (out, out_offsets, stats): ``out`` is one int64 buffer
        (same memory kind) holding model k as ns[k] rows of words(ns[k]) words from word
        out_offsets[k].  The pointer arrays are built with numpy, so the call costs no Python
        work per instance."""
        ns = np.ascontiguousarray(ns, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        cnt = int(ns.shape[0])
        if offsets.shape[0] != cnt:
            raise ValueError("ns and offsets differ in length")
        if cnt == 0:
            return None, np.zeros(0, np.int64), Stats().as_dict()
        wsz = ns.astype(np.int64) * ((ns.astype(np.int64) + 63) // 64)
        out_offsets = np.concatenate(([0], np.cumsum(wsz)[:-1])).astype(np.int64)
        total = int(wsz.sum())
        if _is_torch(buf) and buf.is_cuda:
            import torch
            if buf.dtype != torch.uint8 or buf.dim() != 1 or not buf.is_contiguous():
                raise ValueError("expected a contiguous 1-D torch.uint8 CUDA tensor")
            torch.cuda.current_stream(buf.device).synchronize()
            mem, base, size = DL_MEM_DEVICE, buf.data_ptr(), buf.numel()
            out = torch.empty(max(total, 1), dtype=torch.int64, device=buf.device)
            obase = out.data_ptr()
        else:
            a = buf.numpy() if _is_torch(buf) else buf
            a = np.ascontiguousarray(a, dtype=np.uint8).reshape(-1)
            mem, base, size, buf = DL_MEM_HOST, a.ctypes.data, a.size, a
            out = np.zeros(max(total, 1), dtype=np.uint64)
            obase = out.ctypes.data
        end = offsets + (ns.astype(np.uint64) * ns.astype(np.uint64))
        if cnt and int(end.max()) > size:
            raise ValueError("an instance extends past the end of the buffer")
        ptrs = (np.uint64(base) + offsets).astype(np.uint64)
        optrs = (np.uint64(obase) + out_offsets.astype(np.uint64) * np.uint64(8)).astype(np.uint64)
        c_ns = (ctypes.c_int32 * cnt).from_buffer(ns)
        c_ptrs = (ctypes.c_void_p * cnt).from_buffer(ptrs)
        c_optrs = (ctypes.c_void_p * cnt).from_buffer(optrs)
        st = Stats()
        _check(lib().dl_tc_batch(self._h, cnt, c_ns, c_ptrs, mem, c_optrs, ctypes.byref(st)))
        return out[:total], out_offsets, st.as_dict()

    # ---- serving -------------------------------------------------------------------
    def submit(self, kind: int, base, B=None, path: str = "auto", out=None):
        """Queue a request (0 = closure, 1 = same generation); returns (ticket, handle).

        Keep ``handle`` alive until :meth:`poll` has returned for the ticket: it owns the
        input and output buffers.  ``handle['bits']`` is the output: ``out`` if given (same
        memory kind as ``base``, n x ceil(n/64) 64-bit words with contiguous rows, e.g. a view of
        a pinned buffer), else a new array.
        """
        p, n, mem, keep = _square_u8(base)
        bptr, keepb = None, None
        if B is not None:
            bptr, _, _, keepb = _square_u8(B)
        if out is None:
            bits, bp = _alloc_bits(n, mem, keep)
        else:
            if tuple(out.shape) != (n, words(n)):
                raise ValueError("out must have shape (n, ceil(n/64))")
            bits = out
            bp = out.data_ptr() if _is_torch(out) else out.ctypes.data
        req = Request(int(kind), n, p, bptr, mem, PATHS[path], bp)
        t = ctypes.c_uint64(0)
        _check(lib().dl_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        handle = {"bits": bits, "keep": (keep, keepb), "n": n}
        self._inflight[t.value] = handle
        return t.value, handle

    def poll(self, ticket: int, timeout_us: int = 0):
        """(status, stats): status DL_OK when done, DL_EBUSY while running; raises on errors."""
        st = Stats()
        rc = lib().dl_poll(self._h, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(st))
        if rc == DL_EBUSY:
            return DL_EBUSY, None
        self._inflight.pop(ticket, None)
        _check(rc)
        return DL_OK, st.as_dict()

    def cancel(self, ticket: int) -> int:
        return lib().dl_cancel(self._h, ctypes.c_uint64(ticket))

    def selftest_wait_timeout(self, seconds: float) -> int:
        """Status of a deliberately unsatisfied bounded device wait (DL_ETIMEOUT expected)."""
        return lib().dl_selftest_wait_timeout(self._h, float(seconds))


class Program:
    """A program of dl_program_create: set its base relations, run it, read its models.

    ``set(pred, R)``: R a square 0/1 uint8 numpy array or torch CUDA tensor.  ``get(pred,
    device=False)``: the model's bits (n x ceil(n/64) words; a torch CUDA tensor with
    device=True).  ``base`` / ``defined`` / ``layers`` / ``plan`` come from dl_program_describe."""

    def __init__(self, ctx: Context, text: str):
        h = ctypes.c_void_p()
        _check(lib().dl_program_create(ctx._h, text.encode(), ctypes.byref(h)))
        self._h = h
        self._ctx = ctx  # the context must outlive the program
        ctx._programs.add(self)  # and closes it first when closed explicitly
        self.n = None

    def close(self) -> None:
        if getattr(self, "_h", None):
            if getattr(self._ctx, "_h", None):  # (a context closed first has closed it already)
                lib().dl_program_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, pred: str, R) -> None:
        p, n, mem, keep = _square_u8(R)
        _check(lib().dl_program_set(self._h, pred.encode(), n, p, mem))
        self.n = n

    def run(self) -> dict:
        st = Stats()
        _check(lib().dl_program_run(self._h, ctypes.byref(st)))
        return st.as_dict()

    def get(self, pred: str, device: bool = False):
        n = self.n or 0
        if device:
            import torch
            t = torch.empty((n, words(n)), dtype=torch.int64, device="cuda")
            _check(lib().dl_program_get(self._h, pred.encode(), t.data_ptr(), DL_MEM_DEVICE))
            return t
        a = np.zeros((n, words(n)), dtype=np.uint64)
        _check(lib().dl_program_get(self._h, pred.encode(), a.ctypes.data, DL_MEM_HOST))
        return a

    def describe(self) -> str:
        need = ctypes.c_size_t()
        _check(lib().dl_program_describe(self._h, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value + 1)
        _check(lib().dl_program_describe(self._h, buf, need.value + 1, None))
        return buf.value.decode()

    def _lines(self, key):
        return [ln[len(key) + 1:].split() for ln in self.describe().splitlines() if ln.startswith(key + ":")]

    @property
    def base(self) -> list:
        return self._lines("base")[0]

    @property
    def defined(self) -> list:
        return self._lines("defined")[0]

    @property
    def layers(self) -> list:
        return [ln.split(":", 1)[1].split() for ln in self.describe().splitlines()
                if ln.startswith("layer ") and ln.split(":", 1)[1].strip() and "{" not in ln]

    @property
    def plan(self) -> list:
        text = self.describe()
        return text.split("plan:\n", 1)[1].splitlines() if "plan:\n" in text else []


def tc_closure_noalloc(E, stream=None):
    """Closure of a square torch.uint8 CUDA tensor without any device allocation inside the
    library (n <= NOALLOC_MAX_N); returns (bits as an int64 CUDA tensor, squarings).  The
    output tensor is allocated here, by the caller's side (torch), not by the library."""
    import torch
    if not (_is_torch(E) and E.is_cuda):
        raise ValueError("expected a CUDA tensor")
    p, n, mem, keep = _square_u8(E)
    bits = torch.zeros((n, words(n)), dtype=torch.int64, device=keep.device)
    raw = getattr(stream, "cuda_stream", stream) if stream is not None else \
        torch.cuda.current_stream(keep.device).cuda_stream
    sq = ctypes.c_int32(0)
    _check(lib().dl_tc_closure_noalloc(n, p, bits.data_ptr(), ctypes.c_void_p(raw),
                                       ctypes.byref(sq)))
    return bits, sq.value
