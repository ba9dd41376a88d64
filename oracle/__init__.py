"""CPU oracle for the sPEGG per-generation update -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  It wraps ``spegg_oracle.c`` (a plain,
per-locus C statement of the model) through ctypes and shares no code with the
CUDA library.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import build as _build

STATS_DTYPE = np.dtype([
    ("gen", "<u4"), ("n", "<u4"), ("s", "<u4"), ("status", "<u4"),
    ("sum_raw", "<i8"), ("sum_raw2", "<u8"), ("sum_raw_surv", "<i8"),
    ("min_raw", "<i4"), ("max_raw", "<i4"),
    ("het", "<u8"), ("allele", "<u8"), ("consumption", "<u8"),
    ("R", "<f8"), ("f", "<u4"), ("pad", "<u4"),
])
OK, EXTINCT = 0, 1
CERTAIN = 0xFFFFFFFF

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_mutation_cdf.argtypes = [ctypes.c_double, ctypes.c_uint32, u32p]
        L.orc_mutation_cdf.restype = ctypes.c_uint32
        L.orc_phenotype_packed.argtypes = [ctypes.c_void_p, ctypes.c_uint32, u32p]
        L.orc_phenotype_packed.restype = ctypes.c_int32
        L.orc_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                 ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_destroy.restype = None
        L.orc_set_ecology.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        L.orc_set_ecology.restype = ctypes.c_int
        L.orc_set_linkage.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_set_linkage.restype = ctypes.c_int
        L.orc_set_weights.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_set_weights.restype = ctypes.c_int
        L.orc_set_resource_model.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        L.orc_set_resource_model.restype = ctypes.c_int
        L.orc_set_continuous.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        L.orc_set_continuous.restype = ctypes.c_int
        L.orc_set_dominance.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_set_dominance.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
        L.orc_step.restype = ctypes.c_int
        L.orc_read_genotypes.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_read_genotypes.restype = ctypes.c_int
        L.orc_locus_counts.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_locus_counts.restype = ctypes.c_int
        L.orc_read_survivors.argtypes = [ctypes.c_void_p, ctypes.c_void_p, u32p]
        L.orc_read_survivors.restype = ctypes.c_int
        L.orc_get_state.argtypes = [ctypes.c_void_p, u32p, u32p, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_double), u32p]
        L.orc_get_state.restype = None
        L.orc_stats_size.argtypes = []
        L.orc_stats_size.restype = ctypes.c_uint32
        L.orc_summarize.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
        L.orc_summarize.restype = None
        assert L.orc_stats_size() == STATS_DTYPE.itemsize
        _lib = L
    return _lib


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = _u32(ctr); k = _u32(key); out = np.zeros(4, np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def mutation_cdf(mu: float, n_copies: int) -> np.ndarray:
    buf = np.zeros(32, np.uint32)
    k = lib().orc_mutation_cdf(float(mu), int(n_copies), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return buf[:k].copy()


def phenotype(effects: np.ndarray, record: np.ndarray) -> int:
    e = np.ascontiguousarray(effects, dtype=np.int16)
    r = _u32(record)
    return int(lib().orc_phenotype_packed(e.ctypes.data, len(e), r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))


def summarize(stats: np.ndarray, n_loci: int) -> np.ndarray:
    """FP32 summaries (mean z, var z, survival fraction, heterozygosity,
    allele-1 frequency) of each statistics record."""
    stats = np.ascontiguousarray(stats, dtype=STATS_DTYPE)
    out = np.zeros((len(stats), 5), np.float32)
    for i in range(len(stats)):
        lib().orc_summarize(stats[i:i + 1].ctypes.data, n_loci, out[i].ctypes.data)
    return out


class OraclePopulation:
    """One population advanced generation by generation on the CPU."""

    def __init__(self, n: int, n_loci: int, seed: int, replicate: int, effects, surv_table,
                 bin_bias: int, bin_shift: int, mu: float, init_genotypes=None,
                 p0_q32: int = 0x80000000):
        self.n, self.n_loci = int(n), int(n_loci)
        self.words = self.n_loci // 32
        self.continuous = False
        e = np.ascontiguousarray(effects, dtype=np.int16)
        t = _u32(surv_table)
        assert t.shape == (4096,) and e.shape == (self.n_loci,)
        g = None
        if init_genotypes is not None:
            g = _u32(init_genotypes).reshape(self.n, 2 * self.words)
        self._h = lib().orc_create(self.n, self.n_loci, int(seed), int(replicate), e.ctypes.data,
                                   None if g is None else g.ctypes.data, int(p0_q32),
                                   t.ctypes.data, int(bin_bias), int(bin_shift), float(mu))
        if not self._h:
            raise ValueError("oracle rejected the population description")

    @classmethod
    def from_workload(cls, w) -> "OraclePopulation":
        p = cls(w.n, w.n_loci, w.seed, w.replicate, w.effects, w.surv_table, w.bias, w.shift, w.mu,
                w.init_genotypes, w.p0_q32)
        if w.has_ecology:
            p.set_ecology(w.eco_r, w.eco_K, w.eco_R0, w.eco_R_half, w.attack,
                          getattr(w, "eco_model", 0), getattr(w, "eco_r_sd", 0.0))
        if getattr(w, "allele_model", 0) == 1:
            p.set_continuous(w.mut_sd, w.env_sd, getattr(w, "init_values", None))
        if getattr(w, "dominance", None) is not None:
            p.set_dominance(w.dominance)
        if getattr(w, "map_morgans", None) is not None:
            p.set_linkage(w.map_morgans)
        if getattr(w, "mother_weights", None) is not None or getattr(w, "father_weights", None) is not None:
            p.set_weights(w.mother_weights, w.father_weights)
        return p

    def set_ecology(self, r, K, R0, R_half, attack, model: int = 0, r_sd: float = 0.0):
        """Resource: model 0 logistic, 1 Beverton-Holt with growth rate r +
        r_sd z per generation."""
        a = _u32(attack)
        rc = lib().orc_set_ecology(self._h, float(r), float(K), float(R0), float(R_half), a.ctypes.data)
        if rc == 0 and (model or r_sd):
            rc = lib().orc_set_resource_model(self._h, int(model), float(r_sd))
        if rc != 0:
            raise ValueError("oracle rejected the ecology description")

    def set_linkage(self, map_morgans):
        """Linkage map: map_morgans[l] = distance (Morgans) between loci l-1
        and l, negative where locus l starts a new chromosome."""
        m = np.ascontiguousarray(map_morgans, dtype=np.float64)
        assert m.shape == (self.n_loci,)
        if lib().orc_set_linkage(self._h, m.ctypes.data) != 0:
            raise ValueError("oracle rejected the linkage map")

    def set_continuous(self, mut_sd: float, env_sd: float, init_values=None):
        """Continuous allelic values (int16 Q8 per allele copy): Gaussian
        (Irwin-Hall) mutation steps of sd mut_sd and environmental phenotype
        deviations of sd env_sd, both in trait units."""
        v = None if init_values is None else np.ascontiguousarray(init_values, dtype=np.int16)
        assert v is None or v.size == self.n * 2 * self.n_loci
        rc = lib().orc_set_continuous(self._h, float(mut_sd), float(env_sd), None if v is None else v.ctypes.data)
        if rc != 0:
            raise ValueError("oracle rejected the continuous-allele description")
        self.continuous = True

    def values(self) -> np.ndarray:
        """Allelic values [n, 2, L] (int16 Q8) of a continuous population."""
        assert self.continuous
        return self.genotypes().view(np.int16).reshape(self.n, 2, self.n_loci)

    def set_dominance(self, dominance):
        """Dominance deviations (int16 Q8, one per locus) of heterozygous loci."""
        d = np.ascontiguousarray(dominance, dtype=np.int16)
        assert d.shape == (self.n_loci,)
        if lib().orc_set_dominance(self._h, d.ctypes.data) != 0:
            raise ValueError("oracle rejected the dominance deviations")

    def set_weights(self, mother_weights, father_weights):
        """Weighted parents: uint32 weights over the 4096 phenotype bins for
        mothers and for fathers (None: uniform for that role)."""
        m = None if mother_weights is None else _u32(mother_weights)
        f = None if father_weights is None else _u32(father_weights)
        for t in (m, f):
            assert t is None or t.shape == (4096,)
        rc = lib().orc_set_weights(self._h, None if m is None else m.ctypes.data,
                                   None if f is None else f.ctypes.data)
        if rc != 0:
            raise ValueError("oracle rejected the weight tables")

    def step(self, n_gen: int) -> np.ndarray:
        out = np.zeros(max(int(n_gen), 1), STATS_DTYPE)
        done = lib().orc_step(self._h, int(n_gen), out.ctypes.data)
        if done < 0:
            raise RuntimeError(f"oracle step failed ({done})")
        return out[:done]

    def genotypes(self) -> np.ndarray:
        out = np.zeros((self.n, self.n_loci if self.continuous else 2 * self.words), np.uint32)
        lib().orc_read_genotypes(self._h, out.ctypes.data)
        return out

    def locus_counts(self) -> np.ndarray:
        """Allele-1 copies per locus over both haplotypes of the current
        generation's N individuals (biallelic populations)."""
        if self.continuous:
            raise ValueError("per-locus allele counts are for biallelic populations")
        out = np.zeros(self.n_loci, np.uint32)
        if lib().orc_locus_counts(self._h, out.ctypes.data) != 0:
            raise RuntimeError("oracle per-locus counts failed")
        return out

    def survivors(self) -> np.ndarray:
        S = ctypes.c_uint32(0)
        lib().orc_read_survivors(self._h, None, ctypes.byref(S))
        out = np.zeros(S.value, np.uint32)
        if S.value:
            lib().orc_read_survivors(self._h, out.ctypes.data, ctypes.byref(S))
        return out

    def state(self) -> dict:
        g, S, f = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        st, R = ctypes.c_int32(), ctypes.c_double()
        lib().orc_get_state(self._h, ctypes.byref(g), ctypes.byref(S), ctypes.byref(st), ctypes.byref(R),
                            ctypes.byref(f))
        return {"gen": g.value, "S": S.value, "status": st.value, "R": R.value, "f": f.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- spatial
SP_STATS_DTYPE = np.dtype([
    ("t", "<u4"), ("species", "<u4"), ("n_before", "<u4"), ("adults_before", "<u4"), ("births", "<u4"),
    ("survivors", "<u4"), ("movers", "<u4"), ("n_after", "<u4"), ("adults_after", "<u4"), ("pad", "<u4"),
    ("sum_raw_surv", "<i8"), ("het_newborn", "<u8"), ("allele_newborn", "<u8"),
])


class _SpeciesDesc(ctypes.Structure):
    _fields_ = [("effects", ctypes.c_void_p), ("tables", ctypes.c_void_p), ("bin_bias", ctypes.c_int32),
                ("bin_shift", ctypes.c_uint32), ("mu", ctypes.c_double), ("n0", ctypes.c_uint32),
                ("p0_q32", ctypes.c_uint32), ("D", ctypes.c_uint32), ("A", ctypes.c_uint32 * 4),
                ("G", ctypes.c_uint32), ("P", ctypes.c_uint32 * 4), ("E", ctypes.c_uint32),
                ("C", ctypes.c_uint32 * 4), ("beta_q16", ctypes.c_uint32), ("bmax", ctypes.c_uint32)]


def _splib():
    L = lib()
    if not getattr(L, "_sp_ready", False):
        L.orc_space_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
        L.orc_space_create.restype = ctypes.c_void_p
        L.orc_space_destroy.argtypes = [ctypes.c_void_p]
        L.orc_space_destroy.restype = None
        L.orc_space_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_space_step.restype = ctypes.c_int
        L.orc_space_deme_size.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_space_deme_size.restype = ctypes.c_uint32
        L.orc_space_read_deme.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                          ctypes.c_void_p]
        L.orc_space_read_deme.restype = ctypes.c_int
        L.orc_space_set_deme.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_uint32]
        L.orc_space_set_deme.restype = ctypes.c_int
        L.orc_sp_stats_size.restype = ctypes.c_uint32
        L.orc_species_desc_size.restype = ctypes.c_uint32
        assert L.orc_sp_stats_size() == SP_STATS_DTYPE.itemsize
        assert L.orc_species_desc_size() == ctypes.sizeof(_SpeciesDesc)
        L._sp_ready = True
    return L


class OracleSpace:
    """The spatial community advanced step by step on the CPU."""

    def __init__(self, community):
        L = _splib()
        self.c = community
        self.ns = len(community.species)
        self.words = community.n_loci // 32
        self._keep = []
        descs = (_SpeciesDesc * self.ns)()
        for i, sp in enumerate(community.species):
            e = np.ascontiguousarray(sp.effects, dtype=np.int16)
            t = np.ascontiguousarray(sp.tables, dtype=np.uint32).reshape(3, 4096)
            self._keep += [e, t]
            pad = lambda v: (ctypes.c_uint32 * 4)(*(list(v) + [0] * (4 - len(v))))
            descs[i] = _SpeciesDesc(e.ctypes.data, t.ctypes.data, int(sp.bias), int(sp.shift), float(sp.mu),
                                    int(sp.n0), int(sp.p0_q32), int(sp.D), pad(sp.A), int(sp.G), pad(sp.P),
                                    int(sp.E), pad(sp.C), int(sp.beta_q16), int(sp.bmax))
        self._h = L.orc_space_create(community.X, community.Y, self.ns, community.n_loci, community.seed,
                                     community.disp_q32, ctypes.cast(descs, ctypes.c_void_p))
        if not self._h:
            raise ValueError("oracle rejected the community description")

    def step(self, n: int = 1) -> np.ndarray:
        out = np.zeros((n, self.ns), SP_STATS_DTYPE)
        for i in range(n):
            if _splib().orc_space_step(self._h, out[i].ctypes.data) != 0:
                raise RuntimeError("oracle step failed")
        return out

    def deme(self, species: int, patch: int):
        k = _splib().orc_space_deme_size(self._h, species, patch)
        rec = np.zeros((max(k, 1), 2 * self.words), np.uint32)
        age = np.zeros(max(k, 1), np.uint8)
        _splib().orc_space_read_deme(self._h, species, patch, rec.ctypes.data, age.ctypes.data)
        return rec[:k], age[:k]

    def set_deme(self, species: int, patch: int, rec, age) -> None:
        r = np.ascontiguousarray(rec, dtype=np.uint32).reshape(-1, 2 * self.words)
        a = np.ascontiguousarray(age, dtype=np.uint8)
        if _splib().orc_space_set_deme(self._h, species, patch, r.ctypes.data, a.ctypes.data, len(a)) != 0:
            raise ValueError("invalid deme contents")

    def sizes(self) -> np.ndarray:
        return np.array([[_splib().orc_space_deme_size(self._h, s, p) for p in range(self.c.patches)]
                         for s in range(self.ns)], dtype=np.int64)

    def close(self):
        if getattr(self, "_h", None):
            _splib().orc_space_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
