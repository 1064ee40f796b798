"""Python binding of libnw (include/nw.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
(host buffers) or CUDA torch tensors (device buffers, passed with
NW_DEVICE_PTRS) into pointers and raises ``NwError`` for a failed status.
The library must have been built (``python -m paper_2509_01654_gb300.build``);
``load_library`` raises if it is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libnw.so")

NW_OK, NW_EINVAL, NW_ENOMEM, NW_ERANGE, NW_ECUDA, NW_ETIMEOUT, NW_EBUSY = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "NW_OK", -1: "NW_EINVAL", -2: "NW_ENOMEM", -3: "NW_ERANGE", -4: "NW_ECUDA",
                -5: "NW_ETIMEOUT", -6: "NW_EBUSY"}
NW_DEVICE_PTRS = 0x1
NW_ASYNC = 0x2
NW_RANK_NORMALISED = 0x4
MAX_WORD_LEN = 40
MAX_K = 128
MISSING_IDX = 0xFFFFFFFF
MISSING_SCORE = -32768

EXPORTED = [
    "nw_create", "nw_destroy", "nw_last_error", "nw_set_profiling", "nw_last_profile",
    "nw_load_dictionary", "nw_dict_info_get", "nw_dict_free", "nw_all_pairs_matrix",
    "nw_all_pairs_topk", "nw_all_pairs_topk_shard", "nw_topk_merge", "nw_topk_merge_device", "nw_score_pairs",
    "nw_query",
    "nw_measure_int_rates", "nw_debug_enumerate_pairs", "nw_debug_enumerate_query_pairs", "nw_debug_fail_alloc",
    "nw_debug_set_bounds",
    "nw_all_pairs_topk_noalloc",
    "nw_server_create", "nw_server_submit", "nw_server_wait", "nw_server_last_error", "nw_server_destroy",
    "nw_batch_create", "nw_batch_run", "nw_batch_run_queries", "nw_batch_info_get", "nw_batch_free", "nw_all_pairs_matrix_chunked",
    "nw_debug_norm_tables", "nw_load_dictionary_sim",
    # nw_proposal.h
    "nw_model_create", "nw_model_free", "nw_model_param_count", "nw_model_get_params", "nw_model_set_params",
    "nw_model_embed", "nw_model_loss_grad", "nw_model_train", "nw_quantize_embeddings", "nw_dot_topk",
    "nw_rescore_topk", "nw_proposal_topk", "nw_dot_topk_cross", "nw_proposal_query", "nw_server_create_proposal",
    "nw_proposal_set_exact_length",
    "nw_proposal_set_sweep_order",
]
EMBED_DIM = 64
MAX_CANDIDATES = 512
NW_BATCH_AUTOTUNE = 0x10
NW_LOCALITY_ORDER = 0x8
NOALLOC_SCRATCH_BYTES = 32 << 20


class TrainConfig(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("batch_pairs", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("nbr_fraction", ctypes.c_float), ("raw_scale", ctypes.c_float), ("lr_final", ctypes.c_float),
                ("clip_norm", ctypes.c_float), ("seed", ctypes.c_uint64), ("long_len", ctypes.c_uint32),
                ("long_fraction", ctypes.c_float)]


class ProposalProfile(ctypes.Structure):
    _fields_ = [("embed_ms", ctypes.c_double), ("quantize_ms", ctypes.c_double), ("candidates_ms", ctypes.c_double),
                ("rescore_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("exact_ms", ctypes.c_double)]


class NwError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap", ctypes.c_int32)]


class DictInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("alphabet", ctypes.c_uint32), ("min_len", ctypes.c_uint32),
                ("max_len", ctypes.c_uint32), ("score_lo", ctypes.c_int32), ("score_hi", ctypes.c_int32),
                ("nbins", ctypes.c_uint32), ("pad_", ctypes.c_uint32), ("pairs", ctypes.c_uint64),
                ("cells", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64)]


class Profile(ctypes.Structure):
    _fields_ = [("dp_ms", ctypes.c_double), ("finalize_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("dp_launches", ctypes.c_uint32), ("launches", ctypes.c_uint32), ("pairs", ctypes.c_uint64),
                ("cells", ctypes.c_uint64), ("list_inserts", ctypes.c_uint64)]


class IntRates(ctypes.Structure):
    _fields_ = [("viaddmax_s16x2", ctypes.c_double), ("vimax3_s16x2", ctypes.c_double),
                ("vimax_s16x2_relu", ctypes.c_double), ("iadd3", ctypes.c_double), ("lop3", ctypes.c_double),
                ("nw_cell_mix", ctypes.c_double), ("sm_clock_mhz", ctypes.c_double), ("sm_count", ctypes.c_uint32),
                ("pad_", ctypes.c_uint32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("max_batch_queries", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("pad_", ctypes.c_uint32), ("mem_budget_bytes", ctypes.c_size_t)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("nq", ctypes.c_uint32), ("batch_queries", ctypes.c_uint32), ("batch_requests", ctypes.c_uint32),
                ("inflight_at_start", ctypes.c_uint32)]


class BatchDict(ctypes.Structure):
    _fields_ = [("codes", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n", ctypes.c_uint32),
                ("alphabet", ctypes.c_uint32), ("scoring", Scoring), ("qcodes", ctypes.c_void_p),
                ("qoffsets", ctypes.c_void_p), ("nq", ctypes.c_uint32), ("queries_only", ctypes.c_uint32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("ndicts", ctypes.c_uint32), ("launches", ctypes.c_uint32), ("pairs", ctypes.c_uint64),
                ("cells", ctypes.c_uint64), ("tune_ms", ctypes.c_double),
                ("words_per_task", ctypes.c_uint32 * (MAX_WORD_LEN + 1)), ("query_words", ctypes.c_uint32),
                ("query_pairs", ctypes.c_uint64), ("query_cells", ctypes.c_uint64),
                ("blocks_per_sm", ctypes.c_uint32 * (MAX_WORD_LEN + 1)), ("tune_cached", ctypes.c_uint32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libnw.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libnw is not built ({path} missing); run paper_2509_01654_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, u32, i32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
    L.nw_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, sz, vp]
    L.nw_destroy.argtypes = [vp]
    L.nw_destroy.restype = None
    L.nw_last_error.argtypes = [vp]
    L.nw_last_error.restype = ctypes.c_char_p
    L.nw_set_profiling.argtypes = [vp, ctypes.c_int]
    L.nw_last_profile.argtypes = [vp, ctypes.POINTER(Profile)]
    L.nw_load_dictionary.argtypes = [vp, vp, vp, u32, u32, ctypes.POINTER(Scoring), u32, ctypes.POINTER(vp)]
    L.nw_dict_info_get.argtypes = [vp, ctypes.POINTER(DictInfo)]
    L.nw_load_dictionary_sim.argtypes = [vp, vp, vp, u32, u32, vp, i32, u32, ctypes.POINTER(vp)]
    L.nw_dict_free.argtypes = [vp]
    L.nw_dict_free.restype = None
    L.nw_all_pairs_matrix.argtypes = [vp, vp, u32]
    L.nw_all_pairs_matrix_chunked.argtypes = [vp, vp, u64, u32]
    L.nw_all_pairs_topk.argtypes = [vp, u32, vp, vp, vp, ctypes.POINTER(i32), u32, u32]
    L.nw_all_pairs_topk_shard.argtypes = [vp, u32, u32, u32, vp, vp, vp, ctypes.POINTER(i32), u32, u32]
    L.nw_topk_merge.argtypes = [u32, u32, u32, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]
    L.nw_topk_merge_device.argtypes = [vp, u32, u32, u32, vp, vp, vp, vp]
    L.nw_score_pairs.argtypes = [vp, vp, vp, sz, vp, u32]
    L.nw_query.argtypes = [vp, vp, vp, u32, u32, vp, vp, u32]
    L.nw_measure_int_rates.argtypes = [vp, ctypes.c_double, ctypes.POINTER(IntRates)]
    L.nw_debug_enumerate_pairs.argtypes = [vp, u32, u32, u32, vp, vp, u64, ctypes.POINTER(u64)]
    L.nw_debug_enumerate_query_pairs.argtypes = [vp, u32, vp, u32, u32, vp, vp, u64, ctypes.POINTER(u64)]
    L.nw_debug_fail_alloc.argtypes = [vp, u32]
    L.nw_debug_set_bounds.argtypes = [vp, i32, ctypes.c_int64, u32]
    L.nw_debug_norm_tables.argtypes = [ctypes.POINTER(Scoring), i32, i32, vp, vp, vp, u32, ctypes.POINTER(u32)]
    L.nw_model_create.argtypes = [vp, u32, u64, ctypes.POINTER(vp)]
    L.nw_model_free.argtypes = [vp]
    L.nw_model_free.restype = None
    L.nw_model_param_count.argtypes = [vp]
    L.nw_model_param_count.restype = u64
    L.nw_model_get_params.argtypes = [vp, vp, u32]
    L.nw_model_set_params.argtypes = [vp, vp, u32]
    L.nw_model_embed.argtypes = [vp, vp, vp, u32]
    L.nw_model_loss_grad.argtypes = [vp, vp, vp, vp, vp, u32, ctypes.POINTER(ctypes.c_float), vp, u32]
    L.nw_model_train.argtypes = [vp, vp, ctypes.POINTER(TrainConfig), vp, u32, vp, u32]
    L.nw_quantize_embeddings.argtypes = [vp, vp, u32, vp, vp, ctypes.POINTER(ctypes.c_float), u32]
    L.nw_dot_topk.argtypes = [vp, vp, vp, u32, u32, vp, vp, u32]
    L.nw_rescore_topk.argtypes = [vp, vp, u32, u32, vp, vp, u32]
    L.nw_proposal_topk.argtypes = [vp, vp, u32, u32, vp, vp, ctypes.POINTER(ProposalProfile), u32]
    L.nw_dot_topk_cross.argtypes = [vp, vp, u32, vp, vp, u32, u32, vp, vp, u32]
    L.nw_proposal_query.argtypes = [vp, vp, vp, vp, u32, u32, u32, vp, vp, u32]
    L.nw_proposal_set_exact_length.argtypes = [vp, u32]
    L.nw_proposal_set_sweep_order.argtypes = [vp, ctypes.c_int]
    L.nw_server_create_proposal.argtypes = [vp, vp, u32, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.nw_all_pairs_topk_noalloc.argtypes = [vp, u32, vp, vp, vp, ctypes.POINTER(i32), u32, u32]
    L.nw_server_create.argtypes = [vp, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.nw_server_submit.argtypes = [vp, vp, vp, u32, ctypes.POINTER(u64)]
    L.nw_server_wait.argtypes = [vp, u64, ctypes.c_int, vp, vp, ctypes.POINTER(RequestInfo)]
    L.nw_server_last_error.argtypes = [vp]
    L.nw_server_last_error.restype = ctypes.c_char_p
    L.nw_server_destroy.argtypes = [vp]
    L.nw_server_destroy.restype = None
    L.nw_batch_create.argtypes = [vp, ctypes.POINTER(BatchDict), u32, u32, u32, ctypes.POINTER(vp)]
    L.nw_batch_run.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), u32]
    L.nw_batch_run_queries.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), u32]
    L.nw_batch_info_get.argtypes = [vp, ctypes.POINTER(BatchInfo)]
    L.nw_batch_free.argtypes = [vp]
    L.nw_batch_free.restype = None
    _lib = L
    return L


# ---------------------------------------------------------------------------
# buffers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, is_device) of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, False
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), bool(x.is_cuda)
    if not isinstance(x, np.ndarray) or not x.flags.c_contiguous:
        raise ValueError("arrays must be C-contiguous numpy arrays or torch tensors")
    return ctypes.c_void_p(x.ctypes.data), False


def _flags(*bufs, async_: bool = False) -> int:
    kinds = {_ptr(b)[1] for b in bufs if b is not None}
    if len(kinds) > 1:
        raise ValueError("mixing host and device buffers in one call is not supported")
    dev = kinds == {True}
    return (NW_DEVICE_PTRS if dev else 0) | (NW_ASYNC if (async_ and dev) else 0)


def _check(ctx_handle, status):
    if status != NW_OK:
        msg = load_library().nw_last_error(ctx_handle)
        raise NwError(status, msg.decode() if msg else "")


def _empty_like_kind(ref, shape, np_dtype, torch_dtype):
    if ref is not None and _is_torch(ref):
        import torch
        return torch.empty(shape, dtype=torch_dtype, device=ref.device)
    return np.empty(shape, dtype=np_dtype)


# ---------------------------------------------------------------------------
# API

class Context:
    """nw_create / nw_destroy.  `stream`: a torch.cuda.Stream, a raw cudaStream_t int, or None."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream=None):
        L = load_library()
        h = ctypes.c_void_p()
        sp = None
        if stream is not None:
            sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        st = L.nw_create(ctypes.byref(h), device, mem_budget_bytes, sp)
        if st != NW_OK:
            raise NwError(st, (L.nw_last_error(None) or b"").decode())
        self.handle = h
        self.device = device
        self._stream = stream

    def close(self):
        if getattr(self, "handle", None):
            load_library().nw_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return (load_library().nw_last_error(self.handle) or b"").decode()

    def set_profiling(self, on: bool = True):
        _check(self.handle, load_library().nw_set_profiling(self.handle, int(on)))

    def last_profile(self) -> dict:
        p = Profile()
        _check(self.handle, load_library().nw_last_profile(self.handle, ctypes.byref(p)))
        return {f: getattr(p, f) for f, _ in Profile._fields_}

    def measure_int_rates(self, ms_target: float = 200.0) -> dict:
        r = IntRates()
        _check(self.handle, load_library().nw_measure_int_rates(self.handle, ms_target, ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in IntRates._fields_ if f != "pad_"}

    def debug_fail_alloc(self, countdown: int):
        _check(self.handle, load_library().nw_debug_fail_alloc(self.handle, countdown))

    def debug_set_bounds(self, insert_iters: int = -1, wait_cycles: int = -1, withhold_tile: int = 0xFFFFFFFF):
        """Device-side bounds for tests (nw_debug_set_bounds); no arguments restores the defaults."""
        _check(self.handle, load_library().nw_debug_set_bounds(self.handle, insert_iters, wait_cycles, withhold_tile))

    def load_dictionary(self, codes, offsets, alphabet: int, scoring) -> "Dictionary":
        return Dictionary(self, codes, offsets, alphabet, scoring)

    def load_dictionary_sim(self, codes, offsets, alphabet: int, sim, gap: int) -> "Dictionary":
        """A dictionary scored with a full similarity matrix (nw_load_dictionary_sim)."""
        return Dictionary(self, codes, offsets, alphabet, sim=sim, gap=gap)


class Dictionary:
    """nw_load_dictionary / nw_dict_free and the calls on a dictionary."""

    def __init__(self, ctx: Context, codes, offsets, alphabet: int, scoring=None, sim=None, gap=None):
        """scoring = (match, mismatch, gap), or sim (alphabet x alphabet matrix) and gap."""
        L = load_library()
        self.ctx = ctx
        if not _is_torch(codes):
            codes = np.ascontiguousarray(codes, dtype=np.uint8)
            if codes.size == 0:
                codes = np.zeros(1, np.uint8)
            offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
        n = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
        h = ctypes.c_void_p()
        if sim is not None:
            self.scoring = None
            self.sim = np.ascontiguousarray(sim, dtype=np.int32)
            self.gap = int(gap)
            st = L.nw_load_dictionary_sim(ctx.handle, _ptr(codes)[0], _ptr(offsets)[0], n, alphabet,
                                          ctypes.c_void_p(self.sim.ctypes.data), self.gap, _flags(codes, offsets),
                                          ctypes.byref(h))
        else:
            self.scoring = tuple(int(v) for v in scoring)
            sc = Scoring(*self.scoring)
            st = L.nw_load_dictionary(ctx.handle, _ptr(codes)[0], _ptr(offsets)[0], n, alphabet, ctypes.byref(sc),
                                      _flags(codes, offsets), ctypes.byref(h))
        _check(ctx.handle, st)
        self.handle = h
        self.n = n

    def free(self):
        if getattr(self, "handle", None) and getattr(self.ctx, "handle", None):
            load_library().nw_dict_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        i = DictInfo()
        _check(self.ctx.handle, load_library().nw_dict_info_get(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in DictInfo._fields_ if f != "pad_"}

    def all_pairs_matrix(self, out=None, async_: bool = False):
        """int8 scores of all pairs i < j, row-major upper triangle (n(n-1)/2 entries)."""
        E = self.n * (self.n - 1) // 2
        if out is None:
            out = np.empty(E, dtype=np.int8)
        _check(self.ctx.handle, load_library().nw_all_pairs_matrix(self.handle, _ptr(out)[0], _flags(out, async_=async_)))
        return out

    def all_pairs_matrix_chunked(self, chunk_bytes: int, out=None):
        """The int8 upper triangle through a device buffer of chunk_bytes (host output)."""
        E = self.n * (self.n - 1) // 2
        if out is None:
            out = np.empty(E, dtype=np.int8)
        _check(self.ctx.handle, load_library().nw_all_pairs_matrix_chunked(self.handle, _ptr(out)[0], chunk_bytes, 0))
        return out

    def all_pairs_topk(self, k: int, nbr_idx=None, nbr_score=None, hist=True, shard=None, async_: bool = False,
                       normalised: bool = False):
        """(idx[n, k] uint32, score[n, k] int16, hist int64 or None, hist_lo).

        normalised=True ranks neighbours by s / max(len_i, len_j) (Section 5);
        scores stay raw."""
        n = self.n
        if nbr_idx is None:
            nbr_idx = _empty_like_kind(None, (n, k), np.uint32, None)
        if nbr_score is None:
            nbr_score = _empty_like_kind(nbr_idx, (n, k), np.int16, _torch_dtype("int16"))
        h = None
        nbins = 0
        if hist is True:
            nbins = self.info()["nbins"]
            h = _empty_like_kind(nbr_idx, (nbins,), np.int64, _torch_dtype("int64"))
        elif hist is not None and hist is not False:
            h = hist
            nbins = int(h.shape[0])
        lo = ctypes.c_int32(0)
        L = load_library()
        flags = _flags(nbr_idx, nbr_score, h, async_=async_) | (NW_RANK_NORMALISED if normalised else 0)
        if shard is None:
            st = L.nw_all_pairs_topk(self.handle, k, _ptr(nbr_idx)[0], _ptr(nbr_score)[0], _ptr(h)[0],
                                     ctypes.byref(lo), nbins, flags)
        else:
            g, G = shard
            st = L.nw_all_pairs_topk_shard(self.handle, g, G, k, _ptr(nbr_idx)[0], _ptr(nbr_score)[0], _ptr(h)[0],
                                           ctypes.byref(lo), nbins, flags)
        _check(self.ctx.handle, st)
        return nbr_idx, nbr_score, h, int(lo.value)

    def all_pairs_topk_noalloc(self, k: int, nbr_idx, nbr_score, hist=None, async_: bool = False):
        """nw_all_pairs_topk_noalloc: the same lists and histogram as all_pairs_topk,
        computed with the library's fixed static scratch instead of any device
        allocation.  Outputs must be CUDA tensors; returns hist_lo."""
        lo = ctypes.c_int32(0)
        nbins = int(hist.shape[0]) if hist is not None else 0
        st = load_library().nw_all_pairs_topk_noalloc(self.handle, k, _ptr(nbr_idx)[0], _ptr(nbr_score)[0],
                                                      _ptr(hist)[0], ctypes.byref(lo), nbins,
                                                      _flags(nbr_idx, nbr_score, hist, async_=async_))
        _check(self.ctx.handle, st)
        return int(lo.value)

    def score_pairs(self, i, j, out=None, async_: bool = False):
        if not _is_torch(i):
            i = np.ascontiguousarray(i, dtype=np.uint32)
            j = np.ascontiguousarray(j, dtype=np.uint32)
        m = int(i.shape[0])
        if out is None:
            out = _empty_like_kind(i, (m,), np.int16, _torch_dtype("int16"))
        _check(self.ctx.handle, load_library().nw_score_pairs(self.handle, _ptr(i)[0], _ptr(j)[0], m, _ptr(out)[0],
                                                              _flags(i, j, out, async_=async_)))
        return out

    def query(self, qcodes, qoffsets, k: int, nbr_idx=None, nbr_score=None):
        if not _is_torch(qoffsets):
            qcodes = np.ascontiguousarray(qcodes, dtype=np.uint8)
            if qcodes.size == 0:
                qcodes = np.zeros(1, np.uint8)
            qoffsets = np.ascontiguousarray(qoffsets, dtype=np.uint32)
        nq = int(qoffsets.shape[0]) - 1
        if nbr_idx is None:
            nbr_idx = _empty_like_kind(qoffsets if _is_torch(qoffsets) else None, (nq, k), np.uint32,
                                       _torch_dtype("int32"))
        if nbr_score is None:
            nbr_score = _empty_like_kind(nbr_idx, (nq, k), np.int16, _torch_dtype("int16"))
        _check(self.ctx.handle, load_library().nw_query(self.handle, _ptr(qcodes)[0], _ptr(qoffsets)[0], nq, k,
                                                        _ptr(nbr_idx)[0], _ptr(nbr_score)[0],
                                                        _flags(qcodes, qoffsets, nbr_idx, nbr_score)))
        return nbr_idx, nbr_score


def _torch_dtype(name):
    try:
        import torch
        return getattr(torch, name)
    except ImportError:
        return None


def topk_merge(parts, k: int):
    """nw_topk_merge over host parts [(idx[n, k] uint32, score[n, k] int16), ...]."""
    L = load_library()
    idx_parts = [np.ascontiguousarray(p[0], dtype=np.uint32) for p in parts]
    sc_parts = [np.ascontiguousarray(p[1], dtype=np.int16) for p in parts]
    n = idx_parts[0].shape[0] if parts else 0
    ip = (ctypes.c_void_p * len(parts))(*[ctypes.c_void_p(a.ctypes.data) for a in idx_parts])
    sp = (ctypes.c_void_p * len(parts))(*[ctypes.c_void_p(a.ctypes.data) for a in sc_parts])
    oi = np.empty((n, k), dtype=np.uint32)
    os_ = np.empty((n, k), dtype=np.int16)
    st = L.nw_topk_merge(n, k, len(parts), ctypes.cast(ip, ctypes.POINTER(ctypes.c_void_p)),
                         ctypes.cast(sp, ctypes.POINTER(ctypes.c_void_p)), ctypes.c_void_p(oi.ctypes.data),
                         ctypes.c_void_p(os_.ctypes.data))
    if st != NW_OK:
        raise NwError(st, "nw_topk_merge failed")
    return oi, os_


def topk_merge_device(ctx: "Context", idx_parts, score_parts, k: int):
    """nw_topk_merge_device: idx_parts / score_parts are CUDA tensors of shape
    (nparts, n, k) (int32 / int16); returns the merged (n, k) CUDA tensors."""
    import torch
    nparts, n = int(idx_parts.shape[0]), int(idx_parts.shape[1])
    idx_parts = idx_parts.contiguous()
    score_parts = score_parts.contiguous()
    oi = torch.empty((n, k), dtype=torch.int32, device=idx_parts.device)
    os_ = torch.empty((n, k), dtype=torch.int16, device=idx_parts.device)
    _check(ctx.handle, load_library().nw_topk_merge_device(ctx.handle, n, k, nparts, idx_parts.data_ptr(),
                                                           score_parts.data_ptr(), oi.data_ptr(), os_.data_ptr()))
    return oi, os_


def debug_enumerate_query_pairs(q_lengths, d_lengths, ta: int = 0):
    """The (query, dictionary word) original-index pairs nw_query's kernels would score."""
    L = load_library()
    ql = np.ascontiguousarray(q_lengths, dtype=np.uint32)
    dl = np.ascontiguousarray(d_lengths, dtype=np.uint32)
    qp = ql if ql.size else np.zeros(1, np.uint32)
    dp = dl if dl.size else np.zeros(1, np.uint32)
    cnt = ctypes.c_uint64()
    st = L.nw_debug_enumerate_query_pairs(qp.ctypes.data, ql.size, dp.ctypes.data, dl.size, ta, None, None, 0,
                                          ctypes.byref(cnt))
    if st != NW_OK:
        raise NwError(st, "nw_debug_enumerate_query_pairs failed")
    q = np.empty(max(1, cnt.value), dtype=np.uint32)
    d = np.empty(max(1, cnt.value), dtype=np.uint32)
    st = L.nw_debug_enumerate_query_pairs(qp.ctypes.data, ql.size, dp.ctypes.data, dl.size, ta, q.ctypes.data,
                                          d.ctypes.data, cnt.value, ctypes.byref(cnt))
    if st != NW_OK:
        raise NwError(st, "nw_debug_enumerate_query_pairs failed")
    return q[:cnt.value], d[:cnt.value]


def debug_enumerate_pairs(lengths, shard: int = 0, nshards: int = 1):
    """The (a, b) original-index pairs the all-pairs kernels would score, in task order."""
    L = load_library()
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    n = lengths.size
    cnt = ctypes.c_uint64(0)
    st = L.nw_debug_enumerate_pairs(ctypes.c_void_p(lengths.ctypes.data), n, shard, nshards, None, None, 0,
                                    ctypes.byref(cnt))
    if st != NW_OK:
        raise NwError(st, "nw_debug_enumerate_pairs failed")
    a = np.empty(max(1, cnt.value), dtype=np.uint32)
    b = np.empty(max(1, cnt.value), dtype=np.uint32)
    st = L.nw_debug_enumerate_pairs(ctypes.c_void_p(lengths.ctypes.data), n, shard, nshards,
                                    ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data), cnt.value,
                                    ctypes.byref(cnt))
    if st != NW_OK:
        raise NwError(st, "nw_debug_enumerate_pairs failed")
    return a[:cnt.value], b[:cnt.value]


def debug_norm_tables(scoring, lo: int, hi: int):
    """(rank[hi-lo+1, 41] uint16, smin[R, 41] int16, frac[R, 2] int16) of NW_RANK_NORMALISED."""
    L = load_library()
    sc = Scoring(*scoring)
    nr = ctypes.c_uint32(0)
    nb = MAX_WORD_LEN + 1
    rank = np.zeros((hi - lo + 1, nb), dtype=np.uint16)
    z = np.zeros(1, dtype=np.int16)
    st = L.nw_debug_norm_tables(ctypes.byref(sc), lo, hi, ctypes.c_void_p(rank.ctypes.data),
                                ctypes.c_void_p(z.ctypes.data), ctypes.c_void_p(z.ctypes.data), 0, ctypes.byref(nr))
    if st not in (NW_OK, NW_ERANGE):
        raise NwError(st, "nw_debug_norm_tables failed")
    R = nr.value
    smin = np.zeros((max(R, 1), nb), dtype=np.int16)
    frac = np.zeros((max(R, 1), 2), dtype=np.int16)
    st = L.nw_debug_norm_tables(ctypes.byref(sc), lo, hi, ctypes.c_void_p(rank.ctypes.data),
                                ctypes.c_void_p(smin.ctypes.data), ctypes.c_void_p(frac.ctypes.data), R,
                                ctypes.byref(nr))
    if st != NW_OK:
        raise NwError(st, "nw_debug_norm_tables failed")
    return rank, smin[:R], frac[:R]


class Batch:
    """nw_batch_*: many dictionaries, each with an optional query set, reduced to top-k
    lists in one CUDA-graph launch.  `dicts`: [(codes, offsets, alphabet, (match, mismatch,
    gap)[, (qcodes, qoffsets)[, queries_only]]), ...] as host numpy arrays."""

    def __init__(self, ctx: Context, dicts, k: int = 10, autotune: bool = True):
        L = load_library()
        arrs, specs = [], []

        def csr(codes, offsets):
            codes = np.ascontiguousarray(codes, dtype=np.uint8)
            if codes.size == 0:
                codes = np.zeros(1, np.uint8)
            return codes, np.ascontiguousarray(offsets, dtype=np.uint32)

        self.sizes, self.qsizes, self.self_lists = [], [], []
        for entry in dicts:
            codes, offsets, alphabet, scoring = entry[:4]
            queries = entry[4] if len(entry) > 4 else None
            only = bool(entry[5]) if len(entry) > 5 else False
            codes, offsets = csr(codes, offsets)
            q = csr(*queries) if queries is not None else (None, None)
            arrs.append((codes, offsets, q))
            nq = q[1].size - 1 if q[1] is not None else 0
            specs.append(BatchDict(codes.ctypes.data, offsets.ctypes.data, offsets.size - 1, alphabet,
                                   Scoring(*scoring), q[0].ctypes.data if nq else None,
                                   q[1].ctypes.data if q[1] is not None else None, nq, int(only)))
            self.sizes.append(offsets.size - 1)
            self.qsizes.append(nq)
            self.self_lists.append(not only)
        arr = (BatchDict * max(1, len(specs)))(*specs)
        h = ctypes.c_void_p()
        st = L.nw_batch_create(ctx.handle, arr, len(specs), k, NW_BATCH_AUTOTUNE if autotune else 0,
                               ctypes.byref(h))
        _check(ctx.handle, st)
        self.handle = h
        self.ctx = ctx
        self.k = k

    def info(self) -> dict:
        i = BatchInfo()
        _check(self.ctx.handle, load_library().nw_batch_info_get(self.handle, ctypes.byref(i)))
        out = {f: getattr(i, f) for f, _ in BatchInfo._fields_ if f not in ("words_per_task", "blocks_per_sm")}
        out["words_per_task"] = list(i.words_per_task)
        out["blocks_per_sm"] = list(i.blocks_per_sm)
        return out

    def _host_lists(self, sizes):
        return [(np.empty((n, self.k), np.uint32), np.empty((n, self.k), np.int16)) for n in sizes]

    def run(self, outputs=None):
        """One graph launch; returns [(idx[n, k] uint32, score[n, k] int16), ...] (host) or fills
        `outputs` (same structure, numpy or CUDA torch tensors)."""
        if outputs is None:
            outputs = self._host_lists(self.sizes)
        ip = (ctypes.c_void_p * max(1, len(outputs)))(*[_ptr(o[0])[0] for o in outputs])
        sp = (ctypes.c_void_p * max(1, len(outputs)))(*[_ptr(o[1])[0] for o in outputs])
        flags = _flags(*[b for o in outputs for b in o])
        _check(self.ctx.handle, load_library().nw_batch_run(self.handle, ip, sp, flags))
        return outputs

    def run_queries(self, outputs=None, query_outputs=None):
        """One graph launch by nw_batch_run_queries; returns (outputs, query_outputs): each
        dictionary's lists and each query set's lists [(idx[nq, k] uint32, score[nq, k] int16), ...]
        (host arrays unless buffers are given; all buffers host or all CUDA tensors)."""
        if outputs is None:
            outputs = self._host_lists(self.sizes)
        if query_outputs is None:
            query_outputs = self._host_lists(self.qsizes)
        n = max(1, len(outputs))
        ip = (ctypes.c_void_p * n)(*[_ptr(o[0])[0] for o in outputs])
        sp = (ctypes.c_void_p * n)(*[_ptr(o[1])[0] for o in outputs])
        qip = (ctypes.c_void_p * n)(*[_ptr(o[0])[0] for o in query_outputs])
        qsp = (ctypes.c_void_p * n)(*[_ptr(o[1])[0] for o in query_outputs])
        flags = _flags(*[b for o in list(outputs) + list(query_outputs) for b in o])
        _check(self.ctx.handle, load_library().nw_batch_run_queries(self.handle, ip, sp, qip, qsp, flags))
        return outputs, query_outputs

    def free(self):
        if getattr(self, "handle", None) and getattr(self.ctx, "handle", None):
            load_library().nw_batch_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """nw_server_*: continuous-batching query service over a loaded dictionary."""

    def __init__(self, dictionary: "Dictionary", k: int = 10, max_batch_queries: int = 8192, max_inflight: int = 4,
                 mem_budget_bytes: int = 0, proposal=None):
        """proposal=(model, C): answer through the learned proposal
        (nw_server_create_proposal) instead of exhaustively."""
        L = load_library()
        cfg = ServerConfig(k, max_batch_queries, max_inflight, 0, mem_budget_bytes)
        h = ctypes.c_void_p()
        if proposal is None:
            st = L.nw_server_create(dictionary.handle, ctypes.byref(cfg), ctypes.byref(h))
        else:
            model, C = proposal
            st = L.nw_server_create_proposal(dictionary.handle, model.handle, C, ctypes.byref(cfg), ctypes.byref(h))
            self.model = model  # keeps the model alive
        if st != NW_OK:
            raise NwError(st, (L.nw_server_last_error(None) or b"").decode())
        self.handle = h
        self.k = k
        self.dictionary = dictionary  # keeps the dictionary alive

    def _err(self, st):
        raise NwError(st, (load_library().nw_server_last_error(self.handle) or b"").decode())

    def submit(self, qcodes, qoffsets) -> int:
        qcodes = np.ascontiguousarray(qcodes, dtype=np.uint8)
        if qcodes.size == 0:
            qcodes = np.zeros(1, np.uint8)
        qoffsets = np.ascontiguousarray(qoffsets, dtype=np.uint32)
        rid = ctypes.c_uint64(0)
        st = load_library().nw_server_submit(self.handle, ctypes.c_void_p(qcodes.ctypes.data),
                                             ctypes.c_void_p(qoffsets.ctypes.data), qoffsets.size - 1,
                                             ctypes.byref(rid))
        if st != NW_OK:
            self._err(st)
        self._pending_nq = getattr(self, "_pending_nq", {})
        self._pending_nq[rid.value] = qoffsets.size - 1
        return rid.value

    def wait(self, request_id: int, timeout_ms: int = -1):
        """(idx[nq, k] uint32, score[nq, k] int16, info dict) or None if still pending."""
        nq = self._pending_nq[request_id]
        idx = np.empty((nq, self.k), dtype=np.uint32)
        sc = np.empty((nq, self.k), dtype=np.int16)
        info = RequestInfo()
        st = load_library().nw_server_wait(self.handle, request_id, timeout_ms, ctypes.c_void_p(idx.ctypes.data),
                                           ctypes.c_void_p(sc.ctypes.data), ctypes.byref(info))
        if st == NW_EBUSY:
            return None
        del self._pending_nq[request_id]
        if st != NW_OK:
            self._err(st)
        return idx, sc, {f: getattr(info, f) for f, _ in RequestInfo._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load_library().nw_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned candidate proposal (nw_proposal.h)

class Model:
    """nw_model_*: the character CNN whose embeddings' dot products propose
    neighbour candidates for exact rescoring."""

    def __init__(self, ctx: Context, alphabet: int, seed: int = 0):
        L = load_library()
        h = ctypes.c_void_p()
        _check(ctx.handle, L.nw_model_create(ctx.handle, alphabet, seed, ctypes.byref(h)))
        self.ctx = ctx
        self.handle = h
        self.alphabet = alphabet

    def free(self):
        if getattr(self, "handle", None) and getattr(self.ctx, "handle", None):
            load_library().nw_model_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def param_count(self) -> int:
        return int(load_library().nw_model_param_count(self.handle))

    def set_exact_length(self, min_len: int):
        """nw_proposal_set_exact_length: words and queries of at least min_len symbols take the exhaustive path (0: none)."""
        _check(self.ctx.handle, load_library().nw_proposal_set_exact_length(self.handle, min_len))

    def set_sweep_order(self, locality: bool):
        """nw_proposal_set_sweep_order: sweep the candidate product in a locality order (default) or in
        dictionary order; the results are the same."""
        _check(self.ctx.handle, load_library().nw_proposal_set_sweep_order(self.handle, 1 if locality else 0))

    def get_params(self, out=None):
        if out is None:
            out = np.empty(self.param_count, dtype=np.float32)
        _check(self.ctx.handle, load_library().nw_model_get_params(self.handle, _ptr(out)[0], _flags(out)))
        return out

    def set_params(self, params):
        if not _is_torch(params):
            params = np.ascontiguousarray(params, dtype=np.float32)
        assert int(params.shape[0]) == self.param_count
        _check(self.ctx.handle, load_library().nw_model_set_params(self.handle, _ptr(params)[0], _flags(params)))

    def embed(self, d: "Dictionary", out=None):
        if out is None:
            out = np.empty((d.n, EMBED_DIM), dtype=np.float32)
        _check(self.ctx.handle, load_library().nw_model_embed(self.handle, d.handle, _ptr(out)[0], _flags(out)))
        return out

    def loss_grad(self, d: "Dictionary", pi, pj, target, grad=True):
        pi = np.ascontiguousarray(pi, dtype=np.uint32)
        pj = np.ascontiguousarray(pj, dtype=np.uint32)
        target = np.ascontiguousarray(target, dtype=np.float32)
        g = np.empty(self.param_count, dtype=np.float32) if grad else None
        loss = ctypes.c_float(0)
        _check(self.ctx.handle, load_library().nw_model_loss_grad(
            self.handle, d.handle, _ptr(pi)[0], _ptr(pj)[0], _ptr(target)[0], int(pi.shape[0]),
            ctypes.byref(loss), _ptr(g)[0], 0))
        return float(loss.value), g

    def train(self, d: "Dictionary", steps: int, batch_pairs: int = 8192, lr: float = 1e-3, seed: int = 1,
              nbr=None, nbr_fraction: float = 0.5, raw_scale: float = 0.0, lr_final: float = 0.0,
              clip_norm: float = 0.0, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              long_len: int = 0, long_fraction: float = 0.0):
        """Adam on device-drawn pairs labelled by Algorithm 1; returns the per-step losses.
        raw_scale > 0 trains on s * raw_scale, else on s / max(len); lr_final > 0 decays
        the rate linearly to it; clip_norm > 0 clips the gradient norm; long_fraction > 0
        draws that share of the pairs' first words among the words of >= long_len symbols."""
        cfg = TrainConfig(steps, batch_pairs, lr, beta1, beta2, eps, nbr_fraction if nbr is not None else 0.0,
                          raw_scale, lr_final, clip_norm, seed, long_len, long_fraction)
        losses = np.zeros(max(steps, 1), dtype=np.float32)
        knb = 0
        if nbr is not None:
            nbr = np.ascontiguousarray(nbr, dtype=np.uint32)
            knb = int(nbr.shape[1])
        _check(self.ctx.handle, load_library().nw_model_train(
            self.handle, d.handle, ctypes.byref(cfg), _ptr(nbr)[0], knb, _ptr(losses)[0], 0))
        return losses[:steps]

    def query(self, d: "Dictionary", qcodes, qoffsets, C: int, k: int, nbr_idx=None, nbr_score=None):
        """(idx[nq, k], score[nq, k]) by nw_proposal_query: the query words' k best
        dictionary words among C proposed candidates, scored exactly."""
        if not _is_torch(qoffsets):
            qcodes = np.ascontiguousarray(qcodes, dtype=np.uint8)
            if qcodes.size == 0:
                qcodes = np.zeros(1, np.uint8)
            qoffsets = np.ascontiguousarray(qoffsets, dtype=np.uint32)
        nq = int(qoffsets.shape[0]) - 1
        if nbr_idx is None:
            nbr_idx = _empty_like_kind(qoffsets if _is_torch(qoffsets) else None, (nq, k), np.uint32,
                                       _torch_dtype("int32"))
        if nbr_score is None:
            nbr_score = _empty_like_kind(nbr_idx, (nq, k), np.int16, _torch_dtype("int16"))
        _check(self.ctx.handle, load_library().nw_proposal_query(
            self.handle, d.handle, _ptr(qcodes)[0], _ptr(qoffsets)[0], nq, C, k, _ptr(nbr_idx)[0],
            _ptr(nbr_score)[0], _flags(qcodes, qoffsets, nbr_idx, nbr_score)))
        return nbr_idx, nbr_score

    def proposal_topk(self, d: "Dictionary", C: int, k: int, nbr_idx=None, nbr_score=None):
        """(idx[n, k], score[n, k], profile dict): embed, quantise, C candidates, exact rescoring."""
        n = d.n
        if nbr_idx is None:
            nbr_idx = _empty_like_kind(None, (n, k), np.uint32, None)
        if nbr_score is None:
            nbr_score = _empty_like_kind(nbr_idx, (n, k), np.int16, _torch_dtype("int16"))
        prof = ProposalProfile()
        _check(self.ctx.handle, load_library().nw_proposal_topk(
            self.handle, d.handle, C, k, _ptr(nbr_idx)[0], _ptr(nbr_score)[0], ctypes.byref(prof),
            _flags(nbr_idx, nbr_score)))
        return nbr_idx, nbr_score, {f: getattr(prof, f) for f, _ in ProposalProfile._fields_}


def quantize_embeddings(ctx: Context, E):
    """(q int8 [n, 64], bias int32 [n], scale) by nw_quantize_embeddings (host arrays)."""
    E = np.ascontiguousarray(E, dtype=np.float32)
    n = int(E.shape[0])
    q = np.empty((n, EMBED_DIM), dtype=np.int8)
    b = np.empty(max(n, 1), dtype=np.int32)
    sc = ctypes.c_float(0)
    _check(ctx.handle, load_library().nw_quantize_embeddings(ctx.handle, _ptr(E)[0], n, _ptr(q)[0], _ptr(b)[0],
                                                             ctypes.byref(sc), 0))
    return q, b[:n], np.float32(sc.value)


def dot_topk(ctx: Context, q, C: int, bias=None, locality: bool = False):
    """(idx uint32 [n, C], val int32 [n, C]) by nw_dot_topk (host or CUDA buffers);
    locality sets NW_LOCALITY_ORDER (same result, another sweep order)."""
    if not _is_torch(q):
        q = np.ascontiguousarray(q, dtype=np.int8)
        if bias is not None:
            bias = np.ascontiguousarray(bias, dtype=np.int32)
    n = int(q.shape[0])
    idx = _empty_like_kind(q, (n, C), np.uint32, _torch_dtype("int32"))
    val = _empty_like_kind(q, (n, C), np.int32, _torch_dtype("int32"))
    _check(ctx.handle, load_library().nw_dot_topk(ctx.handle, _ptr(q)[0], _ptr(bias)[0], n, C, _ptr(idx)[0],
                                                  _ptr(val)[0], _flags(q, bias, idx, val) |
                                                  (NW_LOCALITY_ORDER if locality else 0)))
    return idx, val


def dot_topk_cross(ctx: Context, qa, qb, C: int, bias=None):
    """(idx uint32 [na, C], val int32 [na, C]) by nw_dot_topk_cross (host or CUDA buffers)."""
    if not _is_torch(qa):
        qa = np.ascontiguousarray(qa, dtype=np.int8)
        qb = np.ascontiguousarray(qb, dtype=np.int8)
        if bias is not None:
            bias = np.ascontiguousarray(bias, dtype=np.int32)
    na, nb = int(qa.shape[0]), int(qb.shape[0])
    idx = _empty_like_kind(qa, (na, C), np.uint32, _torch_dtype("int32"))
    val = _empty_like_kind(qa, (na, C), np.int32, _torch_dtype("int32"))
    _check(ctx.handle, load_library().nw_dot_topk_cross(ctx.handle, _ptr(qa)[0], na, _ptr(qb)[0], _ptr(bias)[0], nb,
                                                        C, _ptr(idx)[0], _ptr(val)[0], _flags(qa, qb, bias, idx, val)))
    return idx, val


def rescore_topk(d: "Dictionary", cand, k: int):
    """(idx uint32 [n, k], score int16 [n, k]) by nw_rescore_topk (host arrays)."""
    cand = np.ascontiguousarray(cand, dtype=np.uint32)
    n, C = cand.shape
    idx = np.empty((n, k), dtype=np.uint32)
    sc = np.empty((n, k), dtype=np.int16)
    _check(d.ctx.handle, load_library().nw_rescore_topk(d.handle, _ptr(cand)[0], C, k, _ptr(idx)[0], _ptr(sc)[0], 0))
    return idx, sc
