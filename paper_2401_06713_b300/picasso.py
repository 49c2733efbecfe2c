"""Python binding of libpicasso (ctypes).  Argument marshalling only: every
step of the Picasso round runs in the library's CUDA kernels; torch supplies
device memory and the current stream.  There is no CPU fallback -- if the
library is missing this module raises."""
from __future__ import annotations

import ctypes
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpicasso.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "picasso.h")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_BUDGET, ERR_TIMEOUT, ERR_INTERNAL, ERR_UNSUPPORTED, ERR_STATE = range(9)
ALGOS = {"auto": 0, "allpairs": 1, "bucket": 2}
COLOR_ALGOS = {"auto": 0, "sweep": 1, "dynamic": 2}
CSR_FORMS = {"earlier": 0, "full": 1}
SMALL_ENGINE = {"auto": 0, "off": 1}
BUDGET_MODES = {"fail": 0, "chunk": 1, "host": 2}


class PicassoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().picasso_strerror(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class Schedule(ctypes.Structure):
    _fields_ = [
        ("engine_blocks_per_sm", ctypes.c_int32),
        ("cluster_max_n", ctypes.c_int32),
        ("cluster_blocks", ctypes.c_int32),
        ("bits_blocks_per_sm", ctypes.c_int32),
        ("color_blocks_per_sm", ctypes.c_int32),
        ("engine_max_n", ctypes.c_int32),
        ("block_max_n", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Config(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("palette_num", ctypes.c_int64),
        ("palette_den", ctypes.c_int64),
        ("alpha", ctypes.c_double),
        ("conflict_algo", ctypes.c_int32),
        ("max_rounds", ctypes.c_int32),
        ("byte_budget", ctypes.c_int64),
        ("color_algo", ctypes.c_int32),
        ("csr_form", ctypes.c_int32),
        ("small_engine", ctypes.c_int32),
        ("budget_mode", ctypes.c_int32),
        ("wait_polls", ctypes.c_int32),
        ("sched", Schedule),
    ]


class CSR(ctypes.Structure):
    _fields_ = [("d_off", ctypes.c_void_p), ("d_col", ctypes.c_void_p), ("n_rows", ctypes.c_int64),
                ("nnz", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("round", ctypes.c_int32),
        ("n_total", ctypes.c_int64),
        ("n_round", ctypes.c_int64),
        ("P", ctypes.c_int64),
        ("L", ctypes.c_int32),
        ("base", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("colored", ctypes.c_int64),
        ("colors_used", ctypes.c_int64),
        ("peak_bytes", ctypes.c_int64),
        ("conflict_algo_used", ctypes.c_int32),
        ("jp_sweeps", ctypes.c_int32),
        ("ordered_fallbacks", ctypes.c_int32),
        ("max_bucket", ctypes.c_int64),
        ("rounds_done", ctypes.c_int32),
        ("t_assign_ms", ctypes.c_double),
        ("t_build_ms", ctypes.c_double),
        ("t_color_ms", ctypes.c_double),
        ("t_carry_ms", ctypes.c_double),
        ("t_pairs_ms", ctypes.c_double),
        ("pairs_launches", ctypes.c_int64),
        ("logical_pairs", ctypes.c_int64),
        ("tested_pairs", ctypes.c_int64),
        ("t_emit_ms", ctypes.c_double),
        ("emit_launches", ctypes.c_int64),
        ("emit_bytes", ctypes.c_int64),
        ("nnz_total", ctypes.c_int64),
        ("sweep_pending", ctypes.c_int32 * 64),
        ("sweep_active", ctypes.c_int32 * 64),
        ("sweep_us", ctypes.c_float * 64),
        ("small_rounds", ctypes.c_int32),
        ("small_stops", ctypes.c_int32),
        ("t_small_ms", ctypes.c_double),
        ("round_chunks", ctypes.c_int32),
        ("host_csr_rounds", ctypes.c_int32),
        ("barrier_timeout", ctypes.c_int32 * 4),
    ]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


_LIB = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pi32 = ctypes.POINTER(ctypes.c_int32)

_SIGS = {
    "picasso_config_default": [ctypes.POINTER(Config)],
    "picasso_pack": [_vp, _i64, _i32, _vp, _vp],
    "picasso_init": [ctypes.POINTER(_vp), ctypes.POINTER(Config), _vp, _i64, _i32, _vp],
    "picasso_init_batch": [ctypes.POINTER(_vp), ctypes.POINTER(Config), _vp, _pi64, _i32,
                           ctypes.POINTER(ctypes.c_uint64), _i32, _vp],
    "picasso_round_params": [_vp, _pi64, _pi32, _pi64],
    "picasso_assign_lists": [_vp, _i64, _i32, _i64],
    "picasso_build_conflicts": [_vp, ctypes.POINTER(CSR)],
    "picasso_color": [_vp, _pi64],
    "picasso_carry": [_vp, _pi64],
    "picasso_round": [_vp, _pi64],
    "picasso_run": [_vp, _vp, _pi32],
    "picasso_color_host": [ctypes.POINTER(Config), _vp, _i64, _i32, _vp, _pi32, _vp],
    "picasso_autotune": [ctypes.POINTER(Config), _vp, _pi64, _i32, ctypes.POINTER(ctypes.c_uint64), _i32, _i32,
                         ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                         _vp],
    "picasso_get_colors": [_vp, _vp],
    "picasso_get_round": [_vp, _vp, _vp, _vp],
    "picasso_get_runs": [_vp, ctypes.POINTER(_vp)],
    "picasso_copy_csr": [_vp, _vp, _vp],
    "picasso_copy_runs": [_vp, _vp],
    "picasso_get_stats": [_vp, ctypes.POINTER(Stats)],
    "picasso_philox_draws": [ctypes.c_uint64, _i32, _i64, ctypes.c_uint32, ctypes.c_uint32, _i32, _vp, _vp],
    "picasso_kernel_launches": [_pi64],
    "picasso_memory_requests": [_pi64],
    "picasso_trim_memory": [_i64],
    "picasso_run_small_static": [_vp, _i64, _i32, ctypes.POINTER(Config), _vp, _pi32, _vp],
    "picasso_destroy": [_vp],
    "picasso_get_set_stats": [_vp, _pi64, _pi64, _pi64],
    "picasso_save_state": [_vp, _vp, _i64, _pi64],
    "picasso_load_state": [_vp, _vp, _i64],
    "picasso_features": [_vp, _i64, _i32, ctypes.c_uint64, _i64, ctypes.c_double, _vp, _vp, _vp],
    "picasso_features_beta": [_vp, _i64, _i32, ctypes.c_uint64, _i64, ctypes.c_double, _vp, _vp, _vp],
    "picasso_mlp_param_count": [],
    "picasso_mlp_forward": [_vp, _vp, _i32, _vp, _vp],
    "picasso_mlp_backward": [_vp, _vp, _vp, ctypes.c_float, ctypes.c_float, _i32, _vp, _vp, _vp],
    "picasso_mlp_adamw": [_vp, _vp, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, _i32, _vp],
    "picasso_mlp_to_bf16": [_vp, _vp, _i32, _vp],
}


def header_symbols(path: str = HEADER):
    """Names of the functions include/picasso.h declares."""
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|int32_t|const char\*)\s+(picasso_\w+)\s*\(", text, re.M)))


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpicasso.so not built ({LIB_PATH}); run paper_2401_06713_b300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.picasso_strerror.argtypes = [ctypes.c_int]
        L.picasso_strerror.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def lib():
    return _lib()


def _ck(status: int, where: str):
    if status != OK:
        raise PicassoError(status, where)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def words_per_part(q: int) -> int:
    """64-bit words per part (x or z) of a packed string of q qubits."""
    return (q + 63) // 64


def pack(codes: torch.Tensor, stream=None) -> torch.Tensor:
    """uint8 codes [n, q] (0=I 1=X 2=Y 3=Z) on the GPU -> symplectic words
    int64 [n, 2W] (bit patterns of uint64 x_0 .. x_{W-1}, z_0 .. z_{W-1};
    W = ceil(q / 64))."""
    assert codes.is_cuda and codes.dtype == torch.uint8 and codes.dim() == 2
    codes = codes.contiguous()
    n, q = codes.shape
    xz = torch.empty((n, 2 * words_per_part(q)), dtype=torch.int64, device=codes.device)
    _ck(_lib().picasso_pack(_ptr(codes), n, q, _ptr(xz), _stream(stream)), "picasso_pack")
    return xz


def kernel_launches() -> int:
    """Process-wide count of kernels libpicasso has launched."""
    k = ctypes.c_int64()
    _ck(_lib().picasso_kernel_launches(ctypes.byref(k)), "picasso_kernel_launches")
    return int(k.value)


def memory_requests() -> int:
    """Process-wide count of libpicasso's memory requests (pool creations,
    device allocations from its pool, pinned and mapped host allocations)."""
    k = ctypes.c_int64()
    _ck(_lib().picasso_memory_requests(ctypes.byref(k)), "picasso_memory_requests")
    return int(k.value)


def trim_memory(keep_bytes: int = 0):
    """Return the library's cached device memory (current device) to the driver."""
    _ck(_lib().picasso_trim_memory(keep_bytes), "picasso_trim_memory")


def philox_draws(seed: int, rnd: int, gid: int, tag: int, i0: int, count: int, device="cuda") -> torch.Tensor:
    out = torch.empty(count, dtype=torch.int32, device=device)
    _ck(_lib().picasso_philox_draws(seed, rnd, gid, tag, i0, count, _ptr(out), _stream()), "picasso_philox_draws")
    return out


def color_host(codes: torch.Tensor, q: int, colors: torch.Tensor | None = None, seed: int = 0, palette=(1, 8),
               alpha: float = 2.0, stream=None):
    """picasso_color_host: host codes (uint8 [n, q] on the CPU, pinned for
    full copy speed) in, host colors (int32 [n]) and rounds out."""
    assert not codes.is_cuda and codes.dtype == torch.uint8 and codes.dim() == 2 and codes.shape[1] == q
    codes = codes.contiguous()
    n = int(codes.shape[0])
    if colors is None:
        colors = torch.empty(n, dtype=torch.int32, pin_memory=codes.is_pinned())
    assert not colors.is_cuda and colors.dtype == torch.int32 and colors.numel() >= n
    stream = stream if stream is not None else torch.cuda.current_stream()
    cfg = Config()
    _ck(_lib().picasso_config_default(ctypes.byref(cfg)), "picasso_config_default")
    cfg.seed = seed
    cfg.palette_num, cfg.palette_den = palette
    cfg.alpha = alpha
    r = ctypes.c_int32()
    _ck(_lib().picasso_color_host(ctypes.byref(cfg), ctypes.c_void_p(codes.data_ptr()), n, q,
                                  ctypes.c_void_p(colors.data_ptr()), ctypes.byref(r),
                                  ctypes.c_void_p(stream.cuda_stream)), "picasso_color_host")
    return colors[:n], int(r.value)


def autotune(xz: torch.Tensor, q: int, set_offsets=None, seeds=None, reps: int = 3, seed: int = 0,
             palette=(1, 8), alpha: float = 2.0, schedule=None, stream=None):
    """picasso_autotune over the sets of ``xz`` (one set when set_offsets is
    None): returns (schedule dict, its median ms per run, the starting
    schedule's median ms)."""
    assert xz.is_cuda and xz.dtype == torch.int64 and xz.shape[1] == 2 * words_per_part(q)
    xz = xz.contiguous()
    stream = stream if stream is not None else torch.cuda.current_stream()
    cfg = Config()
    _ck(_lib().picasso_config_default(ctypes.byref(cfg)), "picasso_config_default")
    cfg.seed = seed
    cfg.palette_num, cfg.palette_den = palette
    cfg.alpha = alpha
    for k, v in (schedule or {}).items():
        setattr(cfg.sched, k, int(v))
    offs_l = [0, int(xz.shape[0])] if set_offsets is None else [int(x) for x in set_offsets]
    nsets = len(offs_l) - 1
    offs = (ctypes.c_int64 * len(offs_l))(*offs_l)
    sd = None
    if seeds is not None:
        sd = (ctypes.c_uint64 * nsets)(*[int(x) for x in seeds])
    elif set_offsets is None:
        sd = (ctypes.c_uint64 * 1)(seed)
    best = Schedule()
    bms, sms = ctypes.c_double(), ctypes.c_double()
    _ck(_lib().picasso_autotune(ctypes.byref(cfg), _ptr(xz), offs, nsets, sd, q, reps, ctypes.byref(best),
                                ctypes.byref(bms), ctypes.byref(sms), ctypes.c_void_p(stream.cuda_stream)),
        "picasso_autotune")
    return best.as_dict(), float(bms.value), float(sms.value)


class Picasso:
    """A context over packed strings ``xz`` (int64 [n, 2W] on the GPU, W =
    ceil(q / 64))."""

    def __init__(self, xz: torch.Tensor, q: int, seed: int = 0, palette=(1, 8), alpha: float = 2.0,
                 algo: str = "auto", max_rounds: int = 100000, byte_budget: int = 0, stream=None,
                 color: str = "auto", set_offsets=None, seeds=None, csr: str = "earlier", small: str = "auto",
                 budget_mode: str = "fail", wait_polls: int = 0, schedule=None):
        """One set, or with ``set_offsets`` (host, nsets + 1 ints) a batch of
        independent sets stored back to back in ``xz`` (seeds default to
        seed + k).  ``schedule``: a dict of picasso_schedule fields (launch
        shapes only; ``autotune`` returns one)."""
        assert xz.is_cuda and xz.dtype == torch.int64 and xz.dim() == 2 and xz.shape[1] == 2 * words_per_part(q)
        self.xz = xz.contiguous()
        self.n = int(xz.shape[0])
        self.q = q
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.set_offsets = None if set_offsets is None else [int(x) for x in set_offsets]
        cfg = Config()
        _ck(_lib().picasso_config_default(ctypes.byref(cfg)), "picasso_config_default")
        cfg.seed = seed
        cfg.palette_num, cfg.palette_den = palette
        cfg.alpha = alpha
        cfg.conflict_algo = ALGOS[algo]
        cfg.max_rounds = max_rounds
        cfg.byte_budget = byte_budget
        cfg.color_algo = COLOR_ALGOS[color]
        cfg.csr_form = CSR_FORMS[csr]
        cfg.small_engine = SMALL_ENGINE[small]
        cfg.budget_mode = BUDGET_MODES[budget_mode]
        cfg.wait_polls = wait_polls
        for k, v in (schedule or {}).items():
            setattr(cfg.sched, k, int(v))
        self.cfg = cfg
        h = ctypes.c_void_p()
        if set_offsets is None:
            _ck(_lib().picasso_init(ctypes.byref(h), ctypes.byref(cfg), _ptr(self.xz), self.n, q,
                                    ctypes.c_void_p(self.stream.cuda_stream)), "picasso_init")
        else:
            offs = (ctypes.c_int64 * len(set_offsets))(*[int(x) for x in set_offsets])
            nsets = len(set_offsets) - 1
            sd = None
            if seeds is not None:
                sd = (ctypes.c_uint64 * nsets)(*[int(x) for x in seeds])
            _ck(_lib().picasso_init_batch(ctypes.byref(h), ctypes.byref(cfg), _ptr(self.xz), offs, nsets, sd, q,
                                          ctypes.c_void_p(self.stream.cuda_stream)), "picasso_init_batch")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().picasso_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- Alg. 1 steps
    def round_params(self):
        P, L, b = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _ck(_lib().picasso_round_params(self.h, ctypes.byref(P), ctypes.byref(L), ctypes.byref(b)),
            "picasso_round_params")
        return int(P.value), int(L.value), int(b.value)

    def assign_lists(self, P: int, L: int, base: int):
        _ck(_lib().picasso_assign_lists(self.h, P, L, base), "picasso_assign_lists")

    def build_conflicts(self):
        csr = CSR()
        _ck(_lib().picasso_build_conflicts(self.h, ctypes.byref(csr)), "picasso_build_conflicts")
        return int(csr.n_rows), int(csr.nnz)

    def color(self) -> int:
        k = ctypes.c_int64()
        _ck(_lib().picasso_color(self.h, ctypes.byref(k)), "picasso_color")
        return int(k.value)

    def carry(self) -> int:
        k = ctypes.c_int64()
        _ck(_lib().picasso_carry(self.h, ctypes.byref(k)), "picasso_carry")
        return int(k.value)

    def round(self) -> int:
        k = ctypes.c_int64()
        _ck(_lib().picasso_round(self.h, ctypes.byref(k)), "picasso_round")
        return int(k.value)

    def run(self, out: torch.Tensor | None = None):
        """All rounds; returns (colors int32 [n] on the GPU, rounds)."""
        if out is None:
            out = torch.empty(self.n, dtype=torch.int32, device=self.xz.device)
        r = ctypes.c_int32()
        st = _lib().picasso_run(self.h, _ptr(out), ctypes.byref(r))
        if st == ERR_TIMEOUT:
            # a bounded grid barrier gave up: say where
            bt = self.stats()["barrier_timeout"]
            raise PicassoError(st, f"picasso_run (barrier timeout: kernel {bt[0]}, site {bt[1]}, "
                                   f"round {bt[2]}, arrivals {bt[3]})")
        _ck(st, "picasso_run")
        return out, int(r.value)

    # -- inspection
    def colors(self) -> torch.Tensor:
        out = torch.empty(self.n, dtype=torch.int32, device=self.xz.device)
        _ck(_lib().picasso_get_colors(self.h, _ptr(out)), "picasso_get_colors")
        return out

    def stats(self) -> dict:
        s = Stats()
        _ck(_lib().picasso_get_stats(self.h, ctypes.byref(s)), "picasso_get_stats")
        return s.as_dict()

    def vertices(self) -> torch.Tensor:
        """V_l of the current round: global ids, int32 [n_l] (ascending before
        the lists are assigned, in coloring order after)."""
        n = self.stats()["n_round"]
        gid = torch.empty(max(n, 1), dtype=torch.int32, device=self.xz.device)
        _ck(_lib().picasso_get_round(self.h, _ptr(gid), None, None), "picasso_get_round")
        return gid[:n]

    def round_state(self, L: int | None = None):
        """(gid int32 [n_l], lists int32 [n_l, L] round-local, prio int32 [n_l])."""
        st = self.stats()
        n = st["n_round"]
        L = st["L"] if L is None else L
        dev = self.xz.device
        gid = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        lists = torch.empty((max(n, 1), max(L, 1)), dtype=torch.int32, device=dev)
        prio = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        _ck(_lib().picasso_get_round(self.h, _ptr(gid), _ptr(lists), _ptr(prio)), "picasso_get_round")
        return gid[:n], lists[:n, :L], prio[:n]

    def csr(self):
        st = self.stats()
        n, nnz = st["n_round"], st["nnz"]
        dev = self.xz.device
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        _ck(_lib().picasso_copy_csr(self.h, _ptr(off), _ptr(col)), "picasso_copy_csr")
        return off, col[:nnz]

    def set_stats(self):
        """Per set: (colors used so far, peak conflict-structure bytes of one
        round, uncolored vertices), three lists of ints."""
        k = len(self.set_offsets) - 1 if self.set_offsets is not None else 1
        c, b, r = (ctypes.c_int64 * k)(), (ctypes.c_int64 * k)(), (ctypes.c_int64 * k)()
        _ck(_lib().picasso_get_set_stats(self.h, c, b, r), "picasso_get_set_stats")
        return list(c), list(b), list(r)

    def save_state(self) -> bytes:
        """Between-round checkpoint (host bytes)."""
        need = ctypes.c_int64()
        _ck(_lib().picasso_save_state(self.h, None, 0, ctypes.byref(need)), "picasso_save_state")
        buf = ctypes.create_string_buffer(int(need.value))
        _ck(_lib().picasso_save_state(self.h, buf, need.value, ctypes.byref(need)), "picasso_save_state")
        return buf.raw[:need.value]

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _ck(_lib().picasso_load_state(self.h, buf, len(blob)), "picasso_load_state")

    def runs(self):
        """Run offsets of the last build: int64 [E + 1] (run of list entry e is
        col[runoff[e]:runoff[e+1]])."""
        st = self.stats()
        n, L = st["n_round"], st["L"]
        runoff = torch.empty(n * L + 1, dtype=torch.int64, device=self.xz.device)
        _ck(_lib().picasso_copy_runs(self.h, _ptr(runoff)), "picasso_copy_runs")
        return runoff


def run_small_static(xz: torch.Tensor, q: int, seed: int = 0, palette=(1, 8), alpha: float = 2.0,
                     max_rounds: int = 100000, out: torch.Tensor | None = None, stream=None, color: str = "auto",
                     byte_budget: int = 0, csr: str = "earlier", wait_polls: int = 0):
    """Whole run for a small set (n <= 2048) that allocates no device memory
    inside the library; see picasso_run_small_static.  Returns (colors, rounds)."""
    assert xz.is_cuda and xz.dtype == torch.int64 and xz.dim() == 2 and xz.shape[1] == 2
    xz = xz.contiguous()
    n = int(xz.shape[0])
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=xz.device)
    cfg = Config()
    _ck(_lib().picasso_config_default(ctypes.byref(cfg)), "picasso_config_default")
    cfg.seed = seed
    cfg.palette_num, cfg.palette_den = palette
    cfg.alpha = alpha
    cfg.max_rounds = max_rounds
    cfg.color_algo = COLOR_ALGOS[color]
    cfg.byte_budget = byte_budget
    cfg.csr_form = CSR_FORMS[csr]
    cfg.wait_polls = wait_polls
    r = ctypes.c_int32()
    _ck(_lib().picasso_run_small_static(_ptr(xz), n, q, ctypes.byref(cfg), _ptr(out), ctypes.byref(r),
                                        _stream(stream)), "picasso_run_small_static")
    return out, int(r.value)


def color_strings(codes: torch.Tensor, seed: int = 0, palette=(1, 8), alpha: float = 2.0, algo: str = "auto"):
    """Convenience: pack + all rounds.  Returns (colors int32 [n], rounds, stats)."""
    xz = pack(codes)
    with Picasso(xz, codes.shape[1], seed=seed, palette=palette, alpha=alpha, algo=algo) as p:
        colors, rounds = p.run()
        return colors, rounds, p.stats()


def features(xz: torch.Tensor, q: int, seed: int, budget_bytes: float, samples: int = 1 << 16, stream=None):
    """Regressor inputs of one set (Sec. V): (counts int64 [2], feat float32 [5])
    on the GPU; see picasso_features."""
    assert xz.is_cuda and xz.dtype == torch.int64 and xz.dim() == 2 and xz.shape[1] == 2 * words_per_part(q)
    xz = xz.contiguous()
    counts = torch.empty(2, dtype=torch.int64, device=xz.device)
    feat = torch.empty(5, dtype=torch.float32, device=xz.device)
    _ck(_lib().picasso_features(_ptr(xz), int(xz.shape[0]), q, seed, samples, float(budget_bytes), _ptr(counts),
                                _ptr(feat), _stream(stream)), "picasso_features")
    return counts, feat


def features_beta(xz: torch.Tensor, q: int, seed: int, beta: float, samples: int = 1 << 16, stream=None):
    """Regressor inputs for the weighted objective of Eq. ml (feature 4 =
    4 beta - 2); see picasso_features_beta."""
    assert xz.is_cuda and xz.dtype == torch.int64 and xz.dim() == 2 and xz.shape[1] == 2 * words_per_part(q)
    xz = xz.contiguous()
    counts = torch.empty(2, dtype=torch.int64, device=xz.device)
    feat = torch.empty(5, dtype=torch.float32, device=xz.device)
    _ck(_lib().picasso_features_beta(_ptr(xz), int(xz.shape[0]), q, seed, samples, float(beta), _ptr(counts),
                                     _ptr(feat), _stream(stream)), "picasso_features_beta")
    return counts, feat


def mlp_param_count() -> int:
    return int(_lib().picasso_mlp_param_count())


def mlp_forward(w_bf16: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """y [B, 2] fp32 = MLP(bf16 weights, x [B, 5] fp32)."""
    assert w_bf16.dtype == torch.bfloat16 and x.dtype == torch.float32 and x.shape[-1] == 5
    x = x.contiguous()
    B = int(x.shape[0])
    if out is None:
        out = torch.empty((B, 2), dtype=torch.float32, device=x.device)
    _ck(_lib().picasso_mlp_forward(_ptr(w_bf16), _ptr(x), B, _ptr(out), _stream(stream)), "picasso_mlp_forward")
    return out


def mlp_backward(w_bf16: torch.Tensor, x: torch.Tensor, t: torch.Tensor, grad: torch.Tensor,
                 loss: torch.Tensor | None = None, weights=(1.0, 1.0), stream=None):
    """Gradient of the weighted half mean squared error into ``grad`` (fp32)."""
    assert grad.dtype == torch.float32 and grad.numel() == w_bf16.numel()
    x = x.contiguous()
    t = t.contiguous()
    _ck(_lib().picasso_mlp_backward(_ptr(w_bf16), _ptr(x), _ptr(t), float(weights[0]), float(weights[1]),
                                    int(x.shape[0]), _ptr(grad), _ptr(loss) if loss is not None else None,
                                    _stream(stream)), "picasso_mlp_backward")


def mlp_adamw(master: torch.Tensor, w_bf16: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor,
              step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              weight_decay: float = 0.0, stream=None):
    _ck(_lib().picasso_mlp_adamw(_ptr(master), _ptr(w_bf16), _ptr(grad), _ptr(m), _ptr(v), lr, beta1, beta2, eps,
                                 weight_decay, step, _stream(stream)), "picasso_mlp_adamw")


def mlp_to_bf16(src: torch.Tensor, dst: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    assert src.dtype == torch.float32
    if dst is None:
        dst = torch.empty(src.shape, dtype=torch.bfloat16, device=src.device)
    _ck(_lib().picasso_mlp_to_bf16(_ptr(src), _ptr(dst), src.numel(), _stream(stream)), "picasso_mlp_to_bf16")
    return dst
