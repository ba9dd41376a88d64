"""ctypes binding of libspegg_gb300 (include/spegg.h).

Argument marshalling only: every step of a generation runs in the library's
CUDA kernels.  PyTorch supplies device memory (through the library's allocator
hooks, backed by the caching allocator) and the CUDA stream.  There is no CPU
fallback: if the library or a GPU is missing, these calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libspegg_gb300.so")

OK, EXTINCT = 0, 1
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_RANGE, ERR_BUDGET = -1, -2, -3, -4, -5, -6
CERTAIN = 0xFFFFFFFF
N_BINS = 4096

STATS_DTYPE = np.dtype([
    ("gen", "<u4"), ("n", "<u4"), ("s", "<u4"), ("status", "<u4"),
    ("sum_raw", "<i8"), ("sum_raw2", "<u8"), ("sum_raw_surv", "<i8"),
    ("min_raw", "<i4"), ("max_raw", "<i4"),
    ("het", "<u8"), ("allele", "<u8"), ("consumption", "<u8"),
    ("R", "<f8"), ("f", "<u4"), ("pad", "<u4"),
])

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class spg_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class spg_pop_desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32), ("n_loci", ctypes.c_uint32), ("seed", ctypes.c_uint64),
        ("replicate", ctypes.c_uint32), ("effects", ctypes.c_void_p), ("init_genotypes", ctypes.c_void_p),
        ("p0_q32", ctypes.c_uint32), ("surv_table", ctypes.c_void_p), ("bin_bias", ctypes.c_int32),
        ("bin_shift", ctypes.c_uint32), ("mu", ctypes.c_double), ("stats_capacity", ctypes.c_uint32),
        ("map_morgans", ctypes.c_void_p), ("mother_weights", ctypes.c_void_p), ("father_weights", ctypes.c_void_p),
        ("dominance", ctypes.c_void_p), ("allele_model", ctypes.c_uint32), ("mut_sd", ctypes.c_double),
        ("env_sd", ctypes.c_double), ("init_values", ctypes.c_void_p),
    ]


class spg_ecology(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double), ("K", ctypes.c_double), ("R0", ctypes.c_double),
                ("R_half", ctypes.c_double), ("attack", ctypes.c_void_p), ("model", ctypes.c_uint32),
                ("r_sd", ctypes.c_double)]


class spg_noalloc_generation(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32), ("n_loci", ctypes.c_uint32), ("seed", ctypes.c_uint64),
        ("replicate", ctypes.c_uint32), ("generation", ctypes.c_uint32), ("S", ctypes.c_uint32),
        ("f", ctypes.c_uint32), ("effects", ctypes.c_void_p), ("surv_table", ctypes.c_void_p),
        ("bin_bias", ctypes.c_int32), ("bin_shift", ctypes.c_uint32), ("mu", ctypes.c_double),
        ("parents", ctypes.c_void_p), ("survivors", ctypes.c_void_p), ("children", ctypes.c_void_p),
        ("survivors_out", ctypes.c_void_p), ("stats", ctypes.c_void_p),
    ]


class spg_launch_shape(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_uint32), ("items_per_thread", ctypes.c_uint32),
                ("lanes_per_offspring", ctypes.c_uint32)]


class spg_autotune_report(ctypes.Structure):
    _fields_ = [("groups", spg_launch_shape * 4), ("best_ms", ctypes.c_float * 4), ("worst_ms", ctypes.c_float * 4),
                ("gens_run", ctypes.c_uint32)]


def _shape_tuple(sh: spg_launch_shape):
    return (int(sh.threads_per_block), int(sh.items_per_thread), int(sh.lanes_per_offspring))


class spg_server_config(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_size_t), ("max_resident", ctypes.c_uint32),
                ("gens_per_tick", ctypes.c_uint32)]


class spg_job_info(ctypes.Structure):
    _fields_ = [("job", ctypes.c_uint64), ("state", ctypes.c_uint32), ("gen", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("n_gen", ctypes.c_uint32), ("t_arrival", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_finish", ctypes.c_double), ("footprint", ctypes.c_size_t)]


class spg_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("resident", ctypes.c_uint64),
                ("peak_resident", ctypes.c_uint64), ("memory_budget", ctypes.c_size_t),
                ("memory_used", ctypes.c_size_t), ("peak_memory_used", ctypes.c_size_t)]


class spg_species(ctypes.Structure):
    _fields_ = [("effects", ctypes.c_void_p), ("tables", ctypes.c_void_p), ("bin_bias", ctypes.c_int32),
                ("bin_shift", ctypes.c_uint32), ("mu", ctypes.c_double), ("n0", ctypes.c_uint32),
                ("p0_q32", ctypes.c_uint32), ("D", ctypes.c_uint32), ("A", ctypes.c_uint32 * 4),
                ("G", ctypes.c_uint32), ("P", ctypes.c_uint32 * 4), ("E", ctypes.c_uint32),
                ("C", ctypes.c_uint32 * 4), ("beta_q16", ctypes.c_uint32), ("bmax", ctypes.c_uint32)]


class spg_space_desc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_uint32), ("Y", ctypes.c_uint32), ("n_species", ctypes.c_uint32),
                ("n_loci", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("disp_q32", ctypes.c_uint32),
                ("capacity", ctypes.c_uint32), ("staging_capacity", ctypes.c_uint32),
                ("stats_capacity", ctypes.c_uint32), ("species", ctypes.c_void_p)]


SPACE_STATS_DTYPE = np.dtype([
    ("t", "<u4"), ("species", "<u4"), ("n_before", "<u4"), ("adults_before", "<u4"), ("births", "<u4"),
    ("survivors", "<u4"), ("movers", "<u4"), ("n_after", "<u4"), ("adults_after", "<u4"), ("pad", "<u4"),
    ("sum_raw_surv", "<i8"), ("het_newborn", "<u8"), ("allele_newborn", "<u8"),
])


class spg_state(ctypes.Structure):
    _fields_ = [("gen", ctypes.c_uint32), ("S", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("f", ctypes.c_uint32), ("R", ctypes.c_double)]


class SpeggError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


_lib = None
_lock = threading.Lock()

_SIGNATURES = {
    "spg_abi_version": ([], ctypes.c_uint32),
    "spg_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "spg_last_error": ([], ctypes.c_char_p),
    "spg_create_population": ([ctypes.POINTER(spg_pop_desc), ctypes.POINTER(spg_allocator), ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "spg_set_ecology": ([ctypes.c_void_p, ctypes.POINTER(spg_ecology)], ctypes.c_int),
    "spg_step_generations": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "spg_read_stats": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "spg_set_locus_counts": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "spg_read_locus_counts": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "spg_read_genotypes": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "spg_read_survivors": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint32)],
                           ctypes.c_int),
    "spg_get_state": ([ctypes.c_void_p, ctypes.POINTER(spg_state)], ctypes.c_int),
    "spg_checkpoint_size": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "spg_checkpoint": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "spg_restore": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "spg_synchronize": ([ctypes.c_void_p], ctypes.c_int),
    "spg_destroy": ([ctypes.c_void_p], None),
    "spg_summarize": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p], None),
    "spg_mutation_cdf": ([ctypes.c_double, ctypes.c_uint32, ctypes.c_void_p], ctypes.c_uint32),
    "spg_set_tiling": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "spg_generation_noalloc": ([ctypes.POINTER(spg_noalloc_generation), ctypes.c_void_p], ctypes.c_int),
    "spg_batch_create": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(spg_allocator), ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "spg_batch_set_ecology": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(spg_ecology)], ctypes.c_int),
    "spg_batch_step": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "spg_batch_set_tiling": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32], ctypes.c_int),
    "spg_batch_get_tiling": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "spg_batch_autotune": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(spg_autotune_report)], ctypes.c_int),
    "spg_batch_set_launch_shape": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(spg_launch_shape)],
                                   ctypes.c_int),
    "spg_batch_get_launch_shape": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(spg_launch_shape)],
                                   ctypes.c_int),
    "spg_set_launch_shape": ([ctypes.c_void_p, ctypes.POINTER(spg_launch_shape)], ctypes.c_int),
    "spg_get_launch_shape": ([ctypes.c_void_p, ctypes.POINTER(spg_launch_shape)], ctypes.c_int),
    "spg_batch_set_locus_counts": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "spg_batch_read_locus_counts": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_void_p], ctypes.c_int),
    "spg_batch_read_stats": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p],
                             ctypes.c_int),
    "spg_batch_read_genotypes": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "spg_batch_read_survivors": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "spg_batch_get_state": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(spg_state)], ctypes.c_int),
    "spg_batch_synchronize": ([ctypes.c_void_p], ctypes.c_int),
    "spg_batch_size": ([ctypes.c_void_p], ctypes.c_uint32),
    "spg_batch_destroy": ([ctypes.c_void_p], None),
    "spg_server_create": ([ctypes.POINTER(spg_server_config), ctypes.POINTER(spg_allocator), ctypes.c_void_p,
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "spg_server_submit": ([ctypes.c_void_p, ctypes.POINTER(spg_pop_desc), ctypes.POINTER(spg_ecology), ctypes.c_uint32,
                           ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "spg_server_tick": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)],
                        ctypes.c_int),
    "spg_server_drain": ([ctypes.c_void_p], ctypes.c_int),
    "spg_server_run_trace": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "spg_server_job_info": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(spg_job_info)], ctypes.c_int),
    "spg_server_job_stats": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p],
                             ctypes.c_int),
    "spg_server_stats": ([ctypes.c_void_p, ctypes.POINTER(spg_server_counters)], ctypes.c_int),
    "spg_server_clock": ([ctypes.c_void_p], ctypes.c_double),
    "spg_server_destroy": ([ctypes.c_void_p], None),
    "spg_space_create": ([ctypes.POINTER(spg_space_desc), ctypes.POINTER(spg_allocator), ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "spg_space_step": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "spg_space_read_stats": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "spg_space_sizes": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "spg_space_read_deme": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "spg_space_get_state": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "spg_space_synchronize": ([ctypes.c_void_p], ctypes.c_int),
    "spg_space_destroy": ([ctypes.c_void_p], None),
    "spg_get_tiling": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
}


def lib():
    """Load libspegg_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1603_09255_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGNATURES)


def check(code: int, where: str) -> int:
    if code < 0:
        msg = lib().spg_last_error().decode(errors="replace")
        raise SpeggError(code, where, msg or lib().spg_status_string(code).decode())
    return code


def status_string(code: int) -> str:
    return lib().spg_status_string(code).decode()


# ------------------------------------------------------------ torch memory
class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device: Optional[int] = None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._live = {}
        self._alloc = _ALLOC_FN(self._do_alloc)
        self._free = _FREE_FN(self._do_free)
        self.struct = spg_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes) + 256, dtype=self._torch.uint8, device=self.device)
        except Exception:
            return None
        ptr = t.data_ptr()
        aligned = (ptr + 255) & ~255
        self._live[aligned] = t
        return aligned

    def _do_free(self, ptr, ctx):
        self._live.pop(ptr, None)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


class Population:
    """A population advanced on the GPU (spg_create_population ...)."""

    def __init__(self, n: int, n_loci: int, seed: int, replicate: int, effects, surv_table, bin_bias: int,
                 bin_shift: int, mu: float, init_genotypes=None, p0_q32: int = 0x80000000,
                 stats_capacity: int = 0, stream=None, allocator: Optional[TorchAllocator] = None,
                 map_morgans=None, mother_weights=None, father_weights=None, dominance=None,
                 allele_model: int = 0, mut_sd: float = 0.0, env_sd: float = 0.0, init_values=None):
        L = lib()
        self.n, self.n_loci = int(n), int(n_loci)
        self.continuous = int(allele_model) == 1
        # a record is 2 * words uint32: bit-packed haplotypes or 2L int16 values
        self.words = self.n_loci // 2 if self.continuous else self.n_loci // 32
        e = np.ascontiguousarray(effects, dtype=np.int16)
        t = _u32(surv_table)
        if t.shape != (N_BINS,) or e.shape != (self.n_loci,):
            raise ValueError("surv_table must have 4096 entries and effects n_loci entries")
        g = None if init_genotypes is None else _u32(init_genotypes).reshape(-1)
        m = None if map_morgans is None else np.ascontiguousarray(map_morgans, dtype=np.float64)
        if m is not None and m.shape != (self.n_loci,):
            raise ValueError("map_morgans must have n_loci entries")
        mw = None if mother_weights is None else _u32(mother_weights)
        fw = None if father_weights is None else _u32(father_weights)
        for x in (mw, fw):
            if x is not None and x.shape != (N_BINS,):
                raise ValueError("weight tables must have 4096 entries")
        dm = None if dominance is None else np.ascontiguousarray(dominance, dtype=np.int16)
        if dm is not None and dm.shape != (self.n_loci,):
            raise ValueError("dominance must have n_loci entries")
        iv = None if init_values is None else np.ascontiguousarray(init_values, dtype=np.int16).reshape(-1)
        if iv is not None and iv.size != self.n * 2 * self.n_loci:
            raise ValueError("init_values must have n * 2 * n_loci entries")
        self._keep = (e, t, g, m, mw, fw, dm, iv)
        d = spg_pop_desc(self.n, self.n_loci, int(seed), int(replicate), e.ctypes.data,
                         None if g is None else g.ctypes.data, int(p0_q32), t.ctypes.data, int(bin_bias),
                         int(bin_shift), float(mu), int(stats_capacity), None if m is None else m.ctypes.data,
                         None if mw is None else mw.ctypes.data, None if fw is None else fw.ctypes.data,
                         None if dm is None else dm.ctypes.data, int(allele_model), float(mut_sd), float(env_sd),
                         None if iv is None else iv.ctypes.data)
        self.allocator = allocator if allocator is not None else TorchAllocator()
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        check(L.spg_create_population(ctypes.byref(d), ctypes.byref(self.allocator.struct), self._stream,
                                      ctypes.byref(h)), "spg_create_population")
        self._h = h

    @classmethod
    def from_workload(cls, w, **kw) -> "Population":
        kw.setdefault("map_morgans", getattr(w, "map_morgans", None))
        kw.setdefault("mother_weights", getattr(w, "mother_weights", None))
        kw.setdefault("father_weights", getattr(w, "father_weights", None))
        kw.setdefault("dominance", getattr(w, "dominance", None))
        kw.setdefault("allele_model", getattr(w, "allele_model", 0))
        kw.setdefault("mut_sd", getattr(w, "mut_sd", 0.0))
        kw.setdefault("env_sd", getattr(w, "env_sd", 0.0))
        kw.setdefault("init_values", getattr(w, "init_values", None))
        p = cls(w.n, w.n_loci, w.seed, w.replicate, w.effects, w.surv_table, w.bias, w.shift, w.mu,
                w.init_genotypes, w.p0_q32, **kw)
        if w.has_ecology:
            p.set_ecology(w.eco_r, w.eco_K, w.eco_R0, w.eco_R_half, w.attack, getattr(w, "eco_model", 0),
                          getattr(w, "eco_r_sd", 0.0))
        return p

    @property
    def handle(self):
        return self._h

    def set_ecology(self, r, K, R0, R_half, attack, model: int = 0, r_sd: float = 0.0):
        """Resource: model 0 logistic, 1 Beverton-Holt with growth rate r + r_sd z."""
        a = _u32(attack)
        eco = spg_ecology(float(r), float(K), float(R0), float(R_half), a.ctypes.data, int(model), float(r_sd))
        check(lib().spg_set_ecology(self._h, ctypes.byref(eco)), "spg_set_ecology")

    def step(self, n_gen: int) -> None:
        check(lib().spg_step_generations(self._h, int(n_gen)), "spg_step_generations")

    def read_stats(self, first_gen: int, count: int) -> np.ndarray:
        out = np.zeros(max(int(count), 1), STATS_DTYPE)
        check(lib().spg_read_stats(self._h, int(first_gen), int(count), out.ctypes.data), "spg_read_stats")
        return out[:count]

    def state(self) -> dict:
        s = spg_state()
        check(lib().spg_get_state(self._h, ctypes.byref(s)), "spg_get_state")
        return {"gen": s.gen, "S": s.S, "status": s.status, "R": s.R, "f": s.f}

    def genotypes(self) -> np.ndarray:
        out = np.zeros((self.n, 2 * self.words), np.uint32)
        check(lib().spg_read_genotypes(self._h, out.ctypes.data, out.size), "spg_read_genotypes")
        return out

    def set_locus_counts(self, enable: bool = True) -> None:
        """Count the allele-1 copies of every locus in each generation formed
        from now on (spg_set_locus_counts)."""
        check(lib().spg_set_locus_counts(self._h, 1 if enable else 0), "spg_set_locus_counts")

    def locus_counts(self, first_gen: int, count: int) -> np.ndarray:
        """Per-locus allele counts [count, L] of generations first_gen ..
        first_gen + count - 1 (spg_read_locus_counts)."""
        out = np.zeros((max(int(count), 0), self.n_loci), np.uint32)
        check(lib().spg_read_locus_counts(self._h, int(first_gen), int(count), out.ctypes.data if count else None),
              "spg_read_locus_counts")
        return out

    def values(self) -> np.ndarray:
        """Allelic values [n, 2, L] (int16 Q8) of a continuous population."""
        if not self.continuous:
            raise ValueError("not a continuous-allele population")
        return self.genotypes().view(np.int16).reshape(self.n, 2, self.n_loci)

    def survivors(self) -> np.ndarray:
        S = ctypes.c_uint32(0)
        check(lib().spg_read_survivors(self._h, None, 0, ctypes.byref(S)), "spg_read_survivors")
        out = np.zeros(max(S.value, 1), np.uint32)
        check(lib().spg_read_survivors(self._h, out.ctypes.data, out.size, ctypes.byref(S)), "spg_read_survivors")
        return out[:S.value]

    def checkpoint(self) -> bytes:
        size = ctypes.c_size_t()
        check(lib().spg_checkpoint_size(self._h, ctypes.byref(size)), "spg_checkpoint_size")
        buf = ctypes.create_string_buffer(size.value)
        check(lib().spg_checkpoint(self._h, buf, size.value), "spg_checkpoint")
        return buf.raw

    def restore(self, blob) -> None:
        buf = (ctypes.c_char * len(blob)).from_buffer_copy(blob) if isinstance(blob, (bytes, bytearray)) else blob
        check(lib().spg_restore(self._h, buf, len(blob)), "spg_restore")

    def restore_from(self, ptr: int, nbytes: int) -> None:
        """Restore from a raw host pointer (e.g. pinned memory)."""
        check(lib().spg_restore(self._h, ctypes.c_void_p(ptr), int(nbytes)), "spg_restore")

    def set_tiling(self, items_per_thread: int) -> None:
        check(lib().spg_set_tiling(self._h, int(items_per_thread)), "spg_set_tiling")

    def tiling(self) -> int:
        v = ctypes.c_uint32()
        check(lib().spg_get_tiling(self._h, ctypes.byref(v)), "spg_get_tiling")
        return v.value

    def set_launch_shape(self, threads_per_block: int = 0, items_per_thread: int = 0,
                         lanes_per_offspring: int = 0) -> None:
        sh = spg_launch_shape(int(threads_per_block), int(items_per_thread), int(lanes_per_offspring))
        check(lib().spg_set_launch_shape(self._h, ctypes.byref(sh)), "spg_set_launch_shape")

    def launch_shape(self):
        """(threads per block, offspring per thread, lanes per offspring) in use."""
        sh = spg_launch_shape()
        check(lib().spg_get_launch_shape(self._h, ctypes.byref(sh)), "spg_get_launch_shape")
        return _shape_tuple(sh)

    def synchronize(self) -> None:
        check(lib().spg_synchronize(self._h), "spg_synchronize")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().spg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc_for(w, keep: list, stats_capacity: int = 0) -> spg_pop_desc:
    e = np.ascontiguousarray(w.effects, dtype=np.int16)
    t = _u32(w.surv_table)
    g = None if w.init_genotypes is None else _u32(w.init_genotypes).reshape(-1)
    mm = getattr(w, "map_morgans", None)
    m = None if mm is None else np.ascontiguousarray(mm, dtype=np.float64)
    mw = None if getattr(w, "mother_weights", None) is None else _u32(w.mother_weights)
    fw = None if getattr(w, "father_weights", None) is None else _u32(w.father_weights)
    dm = None if getattr(w, "dominance", None) is None else np.ascontiguousarray(w.dominance, dtype=np.int16)
    iv = getattr(w, "init_values", None)
    if iv is not None:
        iv = np.ascontiguousarray(iv, dtype=np.int16).reshape(-1)
        if iv.size != int(w.n) * 2 * int(w.n_loci):
            raise ValueError("init_values must have n * 2 * n_loci entries")
    keep.extend([e, t, g, m, mw, fw, dm, iv])
    return spg_pop_desc(int(w.n), int(w.n_loci), int(w.seed), int(w.replicate), e.ctypes.data,
                        None if g is None else g.ctypes.data, int(w.p0_q32), t.ctypes.data, int(w.bias),
                        int(w.shift), float(w.mu), int(stats_capacity), None if m is None else m.ctypes.data,
                        None if mw is None else mw.ctypes.data, None if fw is None else fw.ctypes.data,
                        None if dm is None else dm.ctypes.data, int(getattr(w, "allele_model", 0)),
                        float(getattr(w, "mut_sd", 0.0)), float(getattr(w, "env_sd", 0.0)),
                        None if iv is None else iv.ctypes.data)


class Batch:
    """Independent populations advanced by shared launches (spg_batch_*)."""

    def __init__(self, workloads, stats_capacity: int = 0, stream=None, allocator: Optional[TorchAllocator] = None):
        L = lib()
        keep = []
        descs = (spg_pop_desc * len(workloads))(*[_desc_for(w, keep, stats_capacity) for w in workloads])
        self.workloads = list(workloads)
        self.allocator = allocator if allocator is not None else TorchAllocator()
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        check(L.spg_batch_create(descs, len(workloads), ctypes.byref(self.allocator.struct), self._stream,
                                 ctypes.byref(h)), "spg_batch_create")
        self._h = h
        for i, w in enumerate(workloads):
            if w.has_ecology:
                a = _u32(w.attack)
                eco = spg_ecology(float(w.eco_r), float(w.eco_K), float(w.eco_R0), float(w.eco_R_half),
                                  a.ctypes.data, int(getattr(w, "eco_model", 0)), float(getattr(w, "eco_r_sd", 0.0)))
                check(L.spg_batch_set_ecology(self._h, i, ctypes.byref(eco)), "spg_batch_set_ecology")

    def __len__(self):
        return int(lib().spg_batch_size(self._h))

    def step(self, n_gen: int) -> None:
        check(lib().spg_batch_step(self._h, int(n_gen)), "spg_batch_step")

    def set_tiling(self, n_loci: int, items: int) -> None:
        check(lib().spg_batch_set_tiling(self._h, int(n_loci), int(items)), "spg_batch_set_tiling")

    def tiling(self, n_loci: int) -> int:
        v = ctypes.c_uint32()
        check(lib().spg_batch_get_tiling(self._h, int(n_loci), ctypes.byref(v)), "spg_batch_get_tiling")
        return v.value

    def set_launch_shape(self, n_loci: int, threads_per_block: int = 0, items_per_thread: int = 0,
                         lanes_per_offspring: int = 0) -> None:
        sh = spg_launch_shape(int(threads_per_block), int(items_per_thread), int(lanes_per_offspring))
        check(lib().spg_batch_set_launch_shape(self._h, int(n_loci), ctypes.byref(sh)), "spg_batch_set_launch_shape")

    def launch_shape(self, n_loci: int):
        """(threads per block, offspring per thread, lanes per offspring) of
        the members with n_loci loci."""
        sh = spg_launch_shape()
        check(lib().spg_batch_get_launch_shape(self._h, int(n_loci), ctypes.byref(sh)), "spg_batch_get_launch_shape")
        return _shape_tuple(sh)

    def autotune(self, gens_per_trial: int) -> int:
        """Time every candidate launch shape per locus-count group and keep the
        fastest; returns the generations every member advanced.  The report
        of the last call is kept in self.autotune_report (by L: chosen shape,
        best and worst ms per generation)."""
        rep = spg_autotune_report()
        check(lib().spg_batch_autotune(self._h, int(gens_per_trial), ctypes.byref(rep)), "spg_batch_autotune")
        self.autotune_report = {
            32 << gi: {"shape": _shape_tuple(rep.groups[gi]), "best_ms": float(rep.best_ms[gi]),
                       "worst_ms": float(rep.worst_ms[gi])}
            for gi in range(4) if rep.groups[gi].threads_per_block}
        return int(rep.gens_run)

    def read_stats(self, member: int, first_gen: int, count: int) -> np.ndarray:
        out = np.zeros(max(int(count), 1), STATS_DTYPE)
        check(lib().spg_batch_read_stats(self._h, int(member), int(first_gen), int(count), out.ctypes.data),
              "spg_batch_read_stats")
        return out[:count]

    def set_locus_counts(self, enable: bool = True) -> None:
        """Per-locus allele counts of every biallelic member from now on
        (spg_batch_set_locus_counts)."""
        check(lib().spg_batch_set_locus_counts(self._h, 1 if enable else 0), "spg_batch_set_locus_counts")

    def locus_counts(self, member: int, first_gen: int, count: int) -> np.ndarray:
        """Per-locus allele counts [count, L] of one member's generations
        first_gen .. first_gen + count - 1 (spg_batch_read_locus_counts)."""
        n_loci = self.workloads[member].n_loci
        out = np.zeros((max(int(count), 0), n_loci), np.uint32)
        check(lib().spg_batch_read_locus_counts(self._h, int(member), int(first_gen), int(count),
                                                out.ctypes.data if count else None), "spg_batch_read_locus_counts")
        return out

    def genotypes(self, member: int) -> np.ndarray:
        w = self.workloads[member]
        words = w.n_loci // 2 if int(getattr(w, "allele_model", 0)) == 1 else w.n_loci // 32
        out = np.zeros((w.n, 2 * words), np.uint32)
        check(lib().spg_batch_read_genotypes(self._h, int(member), out.ctypes.data, out.size),
              "spg_batch_read_genotypes")
        return out

    def values(self, member: int) -> np.ndarray:
        """Allelic values [n, 2, L] (int16 Q8) of a continuous-allele member."""
        w = self.workloads[member]
        if int(getattr(w, "allele_model", 0)) != 1:
            raise ValueError("not a continuous-allele member")
        return self.genotypes(member).view(np.int16).reshape(w.n, 2, w.n_loci)

    def survivors(self, member: int) -> np.ndarray:
        S = ctypes.c_uint32(0)
        w = self.workloads[member]
        out = np.zeros(max(w.n, 1), np.uint32)
        check(lib().spg_batch_read_survivors(self._h, int(member), out.ctypes.data, out.size, ctypes.byref(S)),
              "spg_batch_read_survivors")
        return out[:S.value]

    def state(self, member: int) -> dict:
        s = spg_state()
        check(lib().spg_batch_get_state(self._h, int(member), ctypes.byref(s)), "spg_batch_get_state")
        return {"gen": s.gen, "S": s.S, "status": s.status, "R": s.R, "f": s.f}

    def synchronize(self) -> None:
        check(lib().spg_batch_synchronize(self._h), "spg_batch_synchronize")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().spg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _eco_for(w, keep: list):
    if not w.has_ecology:
        return None
    a = _u32(w.attack)
    keep.append(a)
    return spg_ecology(float(w.eco_r), float(w.eco_K), float(w.eco_R0), float(w.eco_R_half), a.ctypes.data,
                       int(getattr(w, "eco_model", 0)), float(getattr(w, "eco_r_sd", 0.0)))


class Server:
    """Continuous batching of jobs (spg_server_*): jobs are admitted by device
    footprint as they arrive and advanced together in shared launches."""

    def __init__(self, memory_budget: int = 0, max_resident: int = 0, gens_per_tick: int = 0, stream=None,
                 allocator: Optional[TorchAllocator] = None):
        cfg = spg_server_config(int(memory_budget), int(max_resident), int(gens_per_tick))
        self.allocator = allocator if allocator is not None else TorchAllocator()
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        check(lib().spg_server_create(ctypes.byref(cfg), ctypes.byref(self.allocator.struct), self._stream,
                                      ctypes.byref(h)), "spg_server_create")
        self._h = h

    def submit(self, w, n_gen: int, t_arrival: Optional[float] = None) -> int:
        keep = []
        d = _desc_for(w, keep)
        eco = _eco_for(w, keep)
        job = ctypes.c_uint64()
        t = self.clock() if t_arrival is None else float(t_arrival)
        check(lib().spg_server_submit(self._h, ctypes.byref(d), ctypes.byref(eco) if eco is not None else None,
                                      int(n_gen), t, ctypes.byref(job)), "spg_server_submit")
        return job.value

    def tick(self):
        r, q = ctypes.c_uint32(), ctypes.c_uint32()
        check(lib().spg_server_tick(self._h, ctypes.byref(r), ctypes.byref(q)), "spg_server_tick")
        return r.value, q.value

    def drain(self) -> None:
        check(lib().spg_server_drain(self._h), "spg_server_drain")

    def run_trace(self, workloads, n_gens, arrivals):
        keep = []
        count = len(workloads)
        descs = (spg_pop_desc * count)(*[_desc_for(w, keep) for w in workloads])
        ecos = (spg_ecology * count)()
        has = np.zeros(count, np.uint8)
        for i, w in enumerate(workloads):
            e = _eco_for(w, keep)
            if e is not None:
                ecos[i] = e
                has[i] = 1
        ng = _u32(n_gens)
        arr = np.ascontiguousarray(arrivals, dtype=np.float64)
        jobs = np.zeros(count, np.uint64)
        check(lib().spg_server_run_trace(self._h, descs, ecos, has.ctypes.data, ng.ctypes.data, arr.ctypes.data,
                                         count, jobs.ctypes.data), "spg_server_run_trace")
        return jobs

    def job_info(self, job: int) -> dict:
        i = spg_job_info()
        check(lib().spg_server_job_info(self._h, int(job), ctypes.byref(i)), "spg_server_job_info")
        return {k: getattr(i, k) for k, _ in spg_job_info._fields_}

    def job_stats(self, job: int, first_gen: int, count: int) -> np.ndarray:
        out = np.zeros(max(int(count), 1), STATS_DTYPE)
        check(lib().spg_server_job_stats(self._h, int(job), int(first_gen), int(count), out.ctypes.data),
              "spg_server_job_stats")
        return out[:count]

    def counters(self) -> dict:
        c = spg_server_counters()
        check(lib().spg_server_stats(self._h, ctypes.byref(c)), "spg_server_stats")
        return {k: getattr(c, k) for k, _ in spg_server_counters._fields_}

    def clock(self) -> float:
        return float(lib().spg_server_clock(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().spg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Space:
    """Spatial, age-structured multi-species community (spg_space_*)."""

    def __init__(self, community, capacity: int = 0, staging_capacity: int = 0, stats_capacity: int = 0,
                 stream=None, allocator: Optional[TorchAllocator] = None):
        L = lib()
        self.c = community
        self.ns = len(community.species)
        self.words = community.n_loci // 32
        keep = []
        arr = (spg_species * self.ns)()
        for i, sp in enumerate(community.species):
            e = np.ascontiguousarray(sp.effects, dtype=np.int16)
            t = np.ascontiguousarray(sp.tables, dtype=np.uint32).reshape(3, 4096)
            keep += [e, t]
            pad = lambda v: (ctypes.c_uint32 * 4)(*(list(v) + [0] * (4 - len(v))))
            arr[i] = spg_species(e.ctypes.data, t.ctypes.data, int(sp.bias), int(sp.shift), float(sp.mu), int(sp.n0),
                                 int(sp.p0_q32), int(sp.D), pad(sp.A), int(sp.G), pad(sp.P), int(sp.E), pad(sp.C),
                                 int(sp.beta_q16), int(sp.bmax))
        d = spg_space_desc(community.X, community.Y, self.ns, community.n_loci, community.seed, community.disp_q32,
                           int(capacity), int(staging_capacity), int(stats_capacity),
                           ctypes.cast(arr, ctypes.c_void_p))
        self.allocator = allocator if allocator is not None else TorchAllocator()
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        check(L.spg_space_create(ctypes.byref(d), ctypes.byref(self.allocator.struct), self._stream,
                                 ctypes.byref(h)), "spg_space_create")
        self._h = h

    def step(self, n: int = 1) -> None:
        check(lib().spg_space_step(self._h, int(n)), "spg_space_step")

    def read_stats(self, first: int, count: int) -> np.ndarray:
        out = np.zeros((max(count, 1), self.ns), SPACE_STATS_DTYPE)
        check(lib().spg_space_read_stats(self._h, int(first), int(count), out.ctypes.data), "spg_space_read_stats")
        return out[:count]

    def sizes(self) -> np.ndarray:
        out = np.zeros(self.ns * self.c.patches, np.uint32)
        check(lib().spg_space_sizes(self._h, out.ctypes.data, out.size), "spg_space_sizes")
        return out.reshape(self.ns, self.c.patches).astype(np.int64)

    def deme(self, species: int, patch: int):
        n = ctypes.c_uint32()
        check(lib().spg_space_read_deme(self._h, int(species), int(patch), None, None, 0, ctypes.byref(n)),
              "spg_space_read_deme")
        rec = np.zeros((max(n.value, 1), 2 * self.words), np.uint32)
        age = np.zeros(max(n.value, 1), np.uint8)
        check(lib().spg_space_read_deme(self._h, int(species), int(patch), rec.ctypes.data, age.ctypes.data,
                                        max(n.value, 1), ctypes.byref(n)), "spg_space_read_deme")
        return rec[:n.value], age[:n.value]

    def state(self) -> dict:
        t, st, tot = ctypes.c_uint32(), ctypes.c_int32(), ctypes.c_uint32()
        check(lib().spg_space_get_state(self._h, ctypes.byref(t), ctypes.byref(st), ctypes.byref(tot)),
              "spg_space_get_state")
        return {"t": t.value, "status": st.value, "total": tot.value}

    def synchronize(self) -> None:
        check(lib().spg_space_synchronize(self._h), "spg_space_synchronize")

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().spg_space_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def summarize(stats: np.ndarray, n_loci: int) -> np.ndarray:
    stats = np.ascontiguousarray(stats, dtype=STATS_DTYPE)
    out = np.zeros((len(stats), 5), np.float32)
    for i in range(len(stats)):
        lib().spg_summarize(stats[i:i + 1].ctypes.data, int(n_loci), out[i].ctypes.data)
    return out


def mutation_cdf(mu: float, n_copies: int) -> np.ndarray:
    out = np.zeros(32, np.uint32)
    k = lib().spg_mutation_cdf(float(mu), int(n_copies), out.ctypes.data)
    return out[:k].copy()


def generation_noalloc(args: spg_noalloc_generation, stream: int = 0) -> None:
    """One generation on caller-owned device buffers, without any device
    allocation (spg_generation_noalloc); enqueued on `stream`."""
    check(lib().spg_generation_noalloc(ctypes.byref(args), ctypes.c_void_p(stream)), "spg_generation_noalloc")
