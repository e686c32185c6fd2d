"""Python binding of ``librdm.so`` (argument marshalling only; every step of the
estimator runs in the library's CUDA kernels and host code).

PyTorch supplies the CUDA stream and, optionally, the device workspace; numpy holds
host arrays. The library must have been built (``python -m
paper_2204_08147_gb300.build``); importing this module fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librdm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2204_08147_gb300.build`")
_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, EBUSY, ENOTPD, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, FP32 = 0, 1
RADEMACHER, GAUSS, BASIS = 0, 1, 2
GRAM, QUADRATURE = 0, 1
BLOCK, SINGLE = 0, 1
PASSES_AUTO, PASSES_STORE, PASSES_RECOMPUTE = 0, 1, 2
FLAG_DEFLATED, FLAG_PADDED = 1, 2

_PREC = {"fp64": FP64, "fp32": FP32, FP64: FP64, FP32: FP32}
_DIST = {"rademacher": RADEMACHER, "gauss": GAUSS, "basis": BASIS,
         RADEMACHER: RADEMACHER, GAUSS: GAUSS, BASIS: BASIS}
_FORM = {"gram": GRAM, "quadrature": QUADRATURE, GRAM: GRAM, QUADRATURE: QUADRATURE}

_dp = C.POINTER(C.c_double)


class Model(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("n_sys", C.c_int), ("jx", _dp), ("jy", _dp), ("jz", _dp),
                ("hz", _dp), ("gx", _dp), ("lambda_sb", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("vec_dist", C.c_int), ("form", C.c_int),
                ("passes", C.c_int), ("first_vector", C.c_int64), ("recurrence", C.c_int)]


class Result(C.Structure):
    _fields_ = [("rho", _dp), ("ln_z", _dp), ("rho_other", _dp), ("gram_l", _dp), ("quad_l", _dp),
                ("t_a", _dp), ("t_b", _dp), ("e0", C.c_double), ("flags", C.c_uint32),
                ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64)]


class BatchItem(C.Structure):
    _fields_ = [("ham", C.c_void_p), ("betas", _dp), ("n_beta", C.c_int), ("n_v", C.c_int), ("k", C.c_int),
                ("seed", C.c_uint64), ("opts", Opts), ("out", C.POINTER(Result)), ("status", C.c_int)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("ms", C.c_double),
                ("bytes", C.c_double)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_vp = C.c_void_p
_sig("rdm_create", C.c_int, C.POINTER(_vp), C.c_int, _vp)
_sig("rdm_destroy", None, _vp)
_sig("rdm_set_workspace", C.c_int, _vp, _vp, C.c_size_t)
_sig("rdm_workspace_size", C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.POINTER(Opts),
     C.POINTER(C.c_size_t))
_sig("rdm_synchronize", C.c_int, _vp)
_sig("rdm_last_error", C.c_char_p)
_sig("rdm_build_hamiltonian", C.c_int, _vp, C.POINTER(Model), C.POINTER(_vp))
_sig("rdm_destroy_hamiltonian", None, _vp)
_sig("rdm_hamiltonian_info", C.c_int, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
     C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double))
_sig("rdm_estimate", C.c_int, _vp, _dp, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(Opts),
     C.POINTER(Result))
_sig("rdm_apply_hamiltonian", C.c_int, _vp, C.c_int, _vp, _vp, C.c_int)
_sig("rdm_starting_block", C.c_int, _vp, C.c_int, C.c_int, C.c_uint64, C.c_int, _vp)
_sig("rdm_starting_block_noalloc", C.c_int, _vp, C.c_int, C.c_int, C.c_uint64, C.c_int, _vp)
_sig("rdm_mean_force", C.c_int, _dp, C.c_int, C.c_double, _dp)
_sig("rdm_build_bath_hamiltonian", C.c_int, _vp, C.POINTER(Model), C.POINTER(_vp))
_sig("rdm_system_hamiltonian", C.c_int, C.POINTER(Model), _dp)
_sig("rdm_mean_force_abs", C.c_int, _dp, C.c_int, C.c_double, C.c_double, C.c_double, _dp)
_sig("rdm_energy_deviation", C.c_int, _dp, _dp, _dp, C.c_int, C.c_double, _dp)
_sig("rdm_entropy", C.c_int, _dp, C.c_int, _dp)
_sig("rdm_function_of_t", C.c_int, C.c_int, C.c_int, _dp, C.c_int, _dp, _dp, _dp)
_sig("rdm_function_of_t_batch", C.c_int, C.c_int, C.c_int, C.c_int, _dp, C.c_int, _dp, _dp, _dp)
_sig("rdm_symmetric_eig", C.c_int, C.c_int, _dp, _dp, _dp)
_sig("rdm_serve_start", C.c_int, _vp, C.c_size_t, C.c_int)
_sig("rdm_serve_stop", C.c_int, _vp)
_sig("rdm_submit", C.c_int, _vp, C.POINTER(Model), _dp, C.c_int, C.c_int, C.c_int, C.c_uint64,
     C.POINTER(Opts), C.POINTER(Result), C.POINTER(C.c_uint64))
_sig("rdm_poll", C.c_int, _vp, C.c_uint64, C.POINTER(C.c_int))
_sig("rdm_wait", C.c_int, _vp, C.c_uint64, C.c_int, C.POINTER(C.c_int))
_sig("rdm_request_times", C.c_int, _vp, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double))
_sig("rdm_profile", C.c_int, _vp, C.c_int)
_sig("rdm_set_graphs", C.c_int, _vp, C.c_int)
_sig("rdm_probe_copy_rate", C.c_int, _vp, C.c_size_t, C.c_int, C.POINTER(C.c_double))
_sig("rdm_profile_stats", C.c_int, _vp, C.POINTER(KernelStat), C.c_int, C.POINTER(C.c_int))
_sig("rdm_estimate_batch", C.c_int, _vp, C.POINTER(BatchItem), C.c_int)
_sig("rdm_set_bath_order", C.c_int, _vp, C.c_int)
_sig("rdm_set_device_dense", C.c_int, _vp, C.c_int)
_sig("rdm_set_packed_form", C.c_int, _vp, C.c_int)
_sig("rdm_set_spmm_form", C.c_int, _vp, C.c_int)
_sig("rdm_bath_order", C.c_int, C.POINTER(Model), C.POINTER(C.c_int), C.POINTER(C.c_double),
     C.POINTER(C.c_double))
_sig("rdm_packed_tuning", C.c_int, _vp, C.POINTER(C.c_int), C.POINTER(C.c_uint64))


class RdmError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.rdm_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _check(st: int, where: str):
    if st != OK:
        raise RdmError(st, where)


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def last_error() -> str:
    return _lib.rdm_last_error().decode(errors="replace")


# ---------------------------------------------------------------- model marshalling

class _ModelArrays:
    """Keeps the float64 arrays of an rdm_model alive."""

    def __init__(self, spec):
        n = int(spec.n_sites)
        self.jx = np.ascontiguousarray(spec.jx, dtype=np.float64).reshape(n, n)
        self.jy = np.ascontiguousarray(spec.jy, dtype=np.float64).reshape(n, n)
        self.jz = np.ascontiguousarray(spec.jz, dtype=np.float64).reshape(n, n)
        self.hz = np.ascontiguousarray(spec.hz, dtype=np.float64).reshape(n)
        self.gx = np.ascontiguousarray(spec.gx, dtype=np.float64).reshape(n)
        self.struct = Model(n, int(spec.n_sys), _ptr(self.jx), _ptr(self.jy), _ptr(self.jz),
                            _ptr(self.hz), _ptr(self.gx), float(spec.lambda_sb))


_PASSES = {"auto": PASSES_AUTO, "store": PASSES_STORE, "recompute": PASSES_RECOMPUTE,
           PASSES_AUTO: PASSES_AUTO, PASSES_STORE: PASSES_STORE, PASSES_RECOMPUTE: PASSES_RECOMPUTE}


_REC = {"block": BLOCK, "single": SINGLE, BLOCK: BLOCK, SINGLE: SINGLE}


def _opts(precision, dist, form, passes="auto", first_vector=0, recurrence="block") -> Opts:
    return Opts(_PREC[precision], _DIST[dist], _FORM[form], _PASSES[passes], int(first_vector),
                _REC[recurrence])


class _ResultArrays:
    def __init__(self, n_beta, n_v, k, d_s, full: bool):
        nv = d_s * d_s
        self.rho = np.zeros((n_beta, d_s, d_s))
        self.ln_z = np.zeros(n_beta)
        self.rho_other = np.zeros((n_beta, d_s, d_s))
        self.gram_l = np.zeros((n_beta, n_v, d_s, d_s)) if full else None
        self.quad_l = np.zeros((n_beta, n_v, d_s, d_s)) if full else None
        self.t_a = np.zeros((n_v, k, d_s, d_s)) if full else None
        self.t_b = np.zeros((n_v, k, d_s, d_s)) if full else None
        self.struct = Result(_ptr(self.rho), _ptr(self.ln_z), _ptr(self.rho_other),
                             _ptr(self.gram_l), _ptr(self.quad_l), _ptr(self.t_a), _ptr(self.t_b),
                             0.0, 0)
        del nv

    def as_dict(self, form):
        d = dict(rho=self.rho, lnZ=self.ln_z, e0=self.struct.e0, flags=int(self.struct.flags),
                 h2d_bytes=int(self.struct.h2d_bytes), d2h_bytes=int(self.struct.d2h_bytes))
        if form == GRAM:
            d["rho_quad"] = self.rho_other
        else:
            d["rho_gram"] = self.rho_other
        if self.gram_l is not None:
            d.update(gram_l=self.gram_l, quad_l=self.quad_l, t_a=self.t_a, t_b=self.t_b)
        return d


# ---------------------------------------------------------------- objects

class Context:
    """A library context bound to one CUDA device and one stream.

    By default the stream is PyTorch's current stream on that device, so library
    work is ordered with the caller's torch work.
    """

    def __init__(self, device: int = 0, stream: int | None = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
            if not stream:
                stream = 1  # cudaStreamLegacy: torch's default stream
        h = _vp()
        _check(_lib.rdm_create(C.byref(h), int(device), _vp(stream) if stream else None), "rdm_create")
        self.h = h
        self.device = int(device)
        self._ws = None
        self._serving = False

    def attach_workspace(self, nbytes: int):
        """Backs the estimator's scratch with a PyTorch-allocated device buffer."""
        import torch
        t = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        base = (t.data_ptr() + 255) // 256 * 256
        _check(_lib.rdm_set_workspace(self.h, _vp(base), int(nbytes)), "rdm_set_workspace")
        self._ws = t
        return t

    def detach_workspace(self):
        _check(_lib.rdm_set_workspace(self.h, None, 0), "rdm_set_workspace")
        self._ws = None

    def synchronize(self):
        _check(_lib.rdm_synchronize(self.h), "rdm_synchronize")

    def probe_copy_rate(self, buffer_bytes: int, stages: int = 6) -> float:
        """GB/s of 32 KB TMA bulk copies into shared memory (one block per SM, `stages`
        in flight) from a buffer of buffer_bytes: <= 64 MB measures L2, larger DRAM."""
        g = C.c_double()
        _check(_lib.rdm_probe_copy_rate(self.h, int(buffer_bytes), int(stages), C.byref(g)),
               "rdm_probe_copy_rate")
        return g.value

    def set_device_dense(self, mode=1):
        """Where the small dense step (f(T) E1 per bath vector and beta) runs: 0/False the
        host, 1/True the device for grids of >= 8 betas (default), 2 always the device."""
        _check(_lib.rdm_set_device_dense(self.h, int(mode)), "rdm_set_device_dense")

    def set_spmm_form(self, form: int = 0):
        """SpMM of the estimator: 0 tiled from 32 tiles on (default), 1 tiled whenever the
        layout allows, 2 the plain kernel."""
        _check(_lib.rdm_set_spmm_form(self.h, int(form)), "rdm_set_spmm_form")

    def set_packed_form(self, form: int = 0):
        """Launch forms of estimate_batch's packed first pass: 0 autotuned (default), 1 the
        cooperative grid only, 2 one block per slice only (same results in every form)."""
        _check(_lib.rdm_set_packed_form(self.h, int(form)), "rdm_set_packed_form")

    def set_bath_order(self, enable: bool = True):
        """Let rdm_build_hamiltonian reorder bath bits for the tiled SpMM (default on)."""
        _check(_lib.rdm_set_bath_order(self.h, 1 if enable else 0), "rdm_set_bath_order")

    def set_graphs(self, enable: bool = True):
        """Replay repeated first-pass launch sequences from CUDA graphs (default on)."""
        _check(_lib.rdm_set_graphs(self.h, 1 if enable else 0), "rdm_set_graphs")

    def profile(self, enable: bool = True):
        """Starts (and clears) or stops per-kernel launch counting and event timing."""
        _check(_lib.rdm_profile(self.h, 1 if enable else 0), "rdm_profile")

    def profile_stats(self) -> dict:
        """{kernel: {"launches", "ms", "bytes"}} recorded since profile(True)."""
        arr = (KernelStat * 32)()
        n = C.c_int()
        _check(_lib.rdm_profile_stats(self.h, arr, 32, C.byref(n)), "rdm_profile_stats")
        return {arr[i].name.decode(): dict(launches=int(arr[i].launches), ms=arr[i].ms, bytes=arr[i].bytes)
                for i in range(min(n.value, 32))}

    def estimate_batch(self, jobs, full: bool = False) -> list:
        """Runs several estimates at once (rdm_estimate_batch): `jobs` is a list of dicts
        with keys ham (a Hamiltonian of this context), betas, n_v, k, seed and optional
        precision, dist, form, passes, first_vector. Returns one result dict per job (as
        Hamiltonian.estimate) plus its "status"; raises RdmError if any job failed."""
        n = len(jobs)
        items = (BatchItem * n)()
        keep = []
        for i, jb in enumerate(jobs):
            ham = jb["ham"]
            b = np.ascontiguousarray(np.atleast_1d(jb["betas"]), dtype=np.float64)
            res = _ResultArrays(len(b), int(jb["n_v"]), int(jb["k"]), ham.d_s, full)
            o = _opts(jb.get("precision", "fp32"), jb.get("dist", "rademacher"), jb.get("form", "gram"),
                      jb.get("passes", "auto"), jb.get("first_vector", 0), jb.get("recurrence", "block"))
            items[i].ham = ham.h
            items[i].betas = _ptr(b)
            items[i].n_beta = len(b)
            items[i].n_v = int(jb["n_v"])
            items[i].k = int(jb["k"])
            items[i].seed = int(jb["seed"]) & (2 ** 64 - 1)
            items[i].opts = o
            items[i].out = C.pointer(res.struct)
            keep.append((b, res, o))
        st = _lib.rdm_estimate_batch(self.h, items, n)
        outs = []
        for i, (_, res, o) in enumerate(keep):
            d = res.as_dict(o.form)
            d["status"] = int(items[i].status)
            outs.append(d)
        _check(st, "rdm_estimate_batch")
        return outs

    def packed_tuning(self) -> tuple:
        """(size classes tuned, candidate launches timed) of the batch autotuner."""
        n, r = C.c_int(), C.c_uint64()
        _check(_lib.rdm_packed_tuning(self.h, C.byref(n), C.byref(r)), "rdm_packed_tuning")
        return int(n.value), int(r.value)

    def close(self):
        if getattr(self, "h", None):
            _lib.rdm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- serving
    def serve_start(self, budget_bytes: int, max_inflight: int = 4):
        _check(_lib.rdm_serve_start(self.h, int(budget_bytes), int(max_inflight)), "rdm_serve_start")
        self._serving = True
        self._tickets = {}

    def serve_stop(self):
        _check(_lib.rdm_serve_stop(self.h), "rdm_serve_stop")
        self._serving = False

    def submit(self, spec, betas, n_v, k, seed, precision="fp32", dist="rademacher", form="gram",
               full=False) -> int:
        m = _ModelArrays(spec)
        b = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
        res = _ResultArrays(len(b), n_v, k, 1 << int(spec.n_sys), full)
        o = _opts(precision, dist, form)
        t = C.c_uint64()
        _check(_lib.rdm_submit(self.h, C.byref(m.struct), _ptr(b), len(b), int(n_v), int(k),
                               int(seed) & (2 ** 64 - 1), C.byref(o), C.byref(res.struct), C.byref(t)),
               "rdm_submit")
        self._tickets[t.value] = (m, b, res, o)
        return t.value

    def poll(self, ticket: int):
        """None while pending, else the result dict (raises on a failed request)."""
        return self.wait(ticket, 0)

    def wait(self, ticket: int, timeout_ms: int = -1):
        st = C.c_int()
        r = _lib.rdm_wait(self.h, C.c_uint64(ticket), int(timeout_ms), C.byref(st))
        if r in (EBUSY, ETIMEOUT):
            return None
        _check(r, "rdm_wait")
        _check(st.value, f"request {ticket}")
        _, _, res, o = self._tickets[ticket]
        return res.as_dict(o.form)

    def request_times(self, ticket: int):
        lat, q = C.c_double(), C.c_double()
        _check(_lib.rdm_request_times(self.h, C.c_uint64(ticket), C.byref(lat), C.byref(q)),
               "rdm_request_times")
        return lat.value, q.value


class Hamiltonian:
    """A model compiled to term descriptors on the context's device."""

    def __init__(self, ctx: Context, spec, part: str = "total"):
        """part="total": the model; part="bath": its bare bath H_b (no system sites),
        whose estimate with the same seed, n_v and distribution gives ln Z_b."""
        self.ctx = ctx
        self.spec = spec
        m = _ModelArrays(spec)
        h = _vp()
        if part == "total":
            _check(_lib.rdm_build_hamiltonian(ctx.h, C.byref(m.struct), C.byref(h)), "rdm_build_hamiltonian")
            self.n_sites, self.n_sys = int(spec.n_sites), int(spec.n_sys)
        elif part == "bath":
            _check(_lib.rdm_build_bath_hamiltonian(ctx.h, C.byref(m.struct), C.byref(h)),
                   "rdm_build_bath_hamiltonian")
            self.n_sites, self.n_sys = int(spec.n_sites) - int(spec.n_sys), 0
        else:
            raise ValueError("part must be 'total' or 'bath'")
        self.h = h
        self.d_s = 1 << self.n_sys
        self.dim = 1 << self.n_sites

    def info(self):
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        nb = C.c_double()
        _check(_lib.rdm_hamiltonian_info(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d),
                                         C.byref(nb)), "rdm_hamiltonian_info")
        return dict(n_sites=a.value, n_sys=b.value, n_flip=c.value, n_diag=d.value, norm_bound=nb.value)

    def close(self):
        if getattr(self, "h", None):
            _lib.rdm_destroy_hamiltonian(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_size(self, n_beta, n_v, k, precision="fp32", dist="rademacher", form="gram",
                       passes="recompute") -> int:
        o = _opts(precision, dist, form, passes)
        n = C.c_size_t()
        _check(_lib.rdm_workspace_size(self.h, int(n_beta), int(n_v), int(k), C.byref(o), C.byref(n)),
               "rdm_workspace_size")
        return n.value

    def estimate(self, betas, n_v, k, seed, precision="fp32", dist="rademacher", form="gram",
                 full=False, passes="auto", first_vector=0, recurrence="block") -> dict:
        """recurrence="block": block Lanczos of block size d_s per bath vector (Algorithm 1);
        "single": one block-size-1 Lanczos per column e_i (x) v_l (Sec. 4.2)."""
        b = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
        res = _ResultArrays(len(b), n_v, k, self.d_s, full)
        o = _opts(precision, dist, form, passes, first_vector, recurrence)
        _check(_lib.rdm_estimate(self.h, _ptr(b), len(b), int(n_v), int(k), int(seed) & (2 ** 64 - 1),
                                 C.byref(o), C.byref(res.struct)), "rdm_estimate")
        return res.as_dict(o.form)

    def apply(self, x, y, precision=None):
        """y = H x for torch CUDA tensors of shape (2^N, n_cols), float32 or float64."""
        import torch
        prec = FP32 if x.dtype == torch.float32 else FP64
        if precision is not None:
            prec = _PREC[precision]
        assert x.is_contiguous() and y.is_contiguous() and x.shape == y.shape and x.dtype == y.dtype
        _check(_lib.rdm_apply_hamiltonian(self.h, prec, _vp(x.data_ptr()), _vp(y.data_ptr()),
                                          int(x.shape[1])), "rdm_apply_hamiltonian")

    def starting_block(self, x, n_v, seed, dist="rademacher"):
        import torch
        prec = FP32 if x.dtype == torch.float32 else FP64
        assert x.is_contiguous() and x.shape[1] == self.d_s * n_v
        _check(_lib.rdm_starting_block(self.h, prec, int(n_v), int(seed) & (2 ** 64 - 1),
                                       _DIST[dist], _vp(x.data_ptr())), "rdm_starting_block")

    def starting_block_noalloc(self, x, n_v, seed, dist="rademacher"):
        """As starting_block, with the library's fixed scratch instead of an allocation."""
        import torch
        prec = FP32 if x.dtype == torch.float32 else FP64
        assert x.is_contiguous() and x.shape[1] == self.d_s * n_v
        _check(_lib.rdm_starting_block_noalloc(self.h, prec, int(n_v), int(seed) & (2 ** 64 - 1),
                                               _DIST[dist], _vp(x.data_ptr())),
               "rdm_starting_block_noalloc")


# ---------------------------------------------------------------- host post-processing

def bath_order(spec) -> tuple:
    """The bath-site order rdm_build_hamiltonian stores for `spec` (host only):
    (order, partner tiles per tile in the caller's order, in the chosen order), where
    order[q] is the caller's site at internal site q."""
    m = _ModelArrays(spec)
    order = (C.c_int * int(spec.n_sites))()
    t0, t1 = C.c_double(), C.c_double()
    _check(_lib.rdm_bath_order(C.byref(m.struct), order, C.byref(t0), C.byref(t1)), "rdm_bath_order")
    return list(order), float(t0.value), float(t1.value)


def mean_force(rho: np.ndarray, beta: float) -> np.ndarray:
    r = np.ascontiguousarray(rho, dtype=np.float64)
    d = r.shape[0]
    out = np.zeros((d, d))
    _check(_lib.rdm_mean_force(_ptr(r), d, float(beta), _ptr(out)), "rdm_mean_force")
    return out


def mean_force_abs(rho: np.ndarray, beta: float, ln_z_t: float, ln_z_b: float) -> np.ndarray:
    """H* with its constant (eq. H_est): -(1/beta)(ln rho + (ln Z_t - ln Z_b) I)."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    d = r.shape[0]
    out = np.zeros((d, d))
    _check(_lib.rdm_mean_force_abs(_ptr(r), d, float(beta), float(ln_z_t), float(ln_z_b), _ptr(out)),
           "rdm_mean_force_abs")
    return out


def system_hamiltonian(spec) -> np.ndarray:
    """The bare system Hamiltonian H_s of a model, d_s x d_s (host)."""
    m = _ModelArrays(spec)
    d = 1 << int(spec.n_sys)
    out = np.zeros((d, d))
    _check(_lib.rdm_system_hamiltonian(C.byref(m.struct), _ptr(out)), "rdm_system_hamiltonian")
    return out


def energy_deviation(rho: np.ndarray, h_star: np.ndarray, h_s: np.ndarray, beta: float) -> float:
    """tr(H* rho*) - tr(H_s rho_s) (Sec. 5.3.2)."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    hst = np.ascontiguousarray(h_star, dtype=np.float64)
    hs = np.ascontiguousarray(h_s, dtype=np.float64)
    out = C.c_double()
    _check(_lib.rdm_energy_deviation(_ptr(r), _ptr(hst), _ptr(hs), r.shape[0], float(beta), C.byref(out)),
           "rdm_energy_deviation")
    return out.value


def entropy(rho: np.ndarray) -> float:
    r = np.ascontiguousarray(rho, dtype=np.float64)
    s = C.c_double()
    _check(_lib.rdm_entropy(_ptr(r), r.shape[0], C.byref(s)), "rdm_entropy")
    return s.value


def function_of_t(t: np.ndarray, p: int, betas) -> tuple:
    """(t_min, c) with c[b] = exp(-beta_b (T - t_min) / 2) E1 (n x p), the small dense
    step of the estimator for one recurrence (eq. fT)."""
    m = np.ascontiguousarray(t, dtype=np.float64)
    n = m.shape[0]
    b = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
    c = np.zeros((len(b), n, p))
    tmin = C.c_double()
    _check(_lib.rdm_function_of_t(n, int(p), _ptr(m), len(b), _ptr(b), C.byref(tmin), _ptr(c)),
           "rdm_function_of_t")
    return tmin.value, c


def function_of_t_batch(ts: np.ndarray, p: int, betas) -> tuple:
    """function_of_t for a stack of matrices ts (n_mat, n, n) on the host worker pool:
    (t_min (n_mat,), c (n_mat, n_beta, n, p))."""
    m = np.ascontiguousarray(ts, dtype=np.float64)
    n_mat, n = m.shape[0], m.shape[1]
    b = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
    c = np.zeros((n_mat, len(b), n, p))
    tmin = np.zeros(n_mat)
    _check(_lib.rdm_function_of_t_batch(n_mat, n, int(p), _ptr(m), len(b), _ptr(b), _ptr(tmin), _ptr(c)),
           "rdm_function_of_t_batch")
    return tmin, c


def symmetric_eig(a: np.ndarray, vectors: bool = True):
    m = np.ascontiguousarray(a, dtype=np.float64)
    n = m.shape[0]
    w = np.zeros(n)
    v = np.zeros((n, n)) if vectors else None
    _check(_lib.rdm_symmetric_eig(n, _ptr(m), _ptr(w), _ptr(v)), "rdm_symmetric_eig")
    return (w, v) if vectors else w
