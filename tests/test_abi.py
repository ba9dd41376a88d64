"""C ABI checks that need no GPU: the library builds, loads, exports every
entry point include/spegg.h declares, rejects bad descriptions before touching
the device, and its host-side helpers agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import spegg_synth as S
from paper_1603_09255_gb300 import build as pkg_build
from paper_1603_09255_gb300 import spegg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg_build.build()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(spg_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = spegg.lib()
    decl = declared_symbols()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert set(spegg.exported_symbols()) == decl


def test_abi_version_and_status_strings():
    assert spegg.lib().spg_abi_version() == 3
    assert spegg.status_string(0) == "ok"
    assert "extinct" in spegg.status_string(1)
    assert "timed out" in spegg.status_string(-4)


def test_invalid_descriptions_are_rejected_before_any_device_work():
    e = np.zeros(32, np.int16)
    t = S.constant_table(S.CERTAIN)
    L = spegg.lib()

    def create(**kw):
        d = dict(n=10, n_loci=32, seed=0, replicate=0, effects=e.ctypes.data, init_genotypes=None,
                 p0_q32=0, surv_table=t.ctypes.data, bin_bias=0, bin_shift=0, mu=0.0, stats_capacity=0)
        d.update(kw)
        desc = spegg.spg_pop_desc(**d)
        h = ctypes.c_void_p()
        rc = L.spg_create_population(ctypes.byref(desc), None, None, ctypes.byref(h))
        return rc, L.spg_last_error().decode()

    for kw, frag in [(dict(n=0), "n must"), (dict(n_loci=48), "n_loci"), (dict(n_loci=512), "n_loci"),
                     (dict(effects=None), "effects"), (dict(surv_table=None), "surv_table"),
                     (dict(bin_shift=32), "bin_shift"), (dict(mu=1.0), "mu"), (dict(mu=-0.1), "mu"),
                     (dict(stats_capacity=1 << 25), "stats_capacity")]:
        rc, msg = create(**kw)
        assert rc == spegg.ERR_INVALID and frag in msg, (kw, rc, msg)
    assert L.spg_create_population(None, None, None, None) == spegg.ERR_INVALID


@pytest.mark.parametrize("mu,n", [(0.0, 64), (1e-4, 64), (1e-5, 256), (1e-5, 512), (0.05, 64), (0.3, 128)])
def test_mutation_table_matches_oracle(mu, n):
    """The library and the oracle build the Binomial CDF independently from
    the same stated arithmetic; the tables must be identical."""
    assert np.array_equal(spegg.mutation_cdf(mu, n), oracle.mutation_cdf(mu, n))


def test_fp32_summaries_match_oracle():
    w = S.consumer_resource(n=2000, n_loci=64, n_gen=4, mu=1e-3, K=1e5)
    st = oracle.OraclePopulation.from_workload(w).step(4)
    a = spegg.summarize(st.astype(spegg.STATS_DTYPE), 64)
    b = oracle.summarize(st, 64)
    assert np.allclose(a, b, rtol=1e-6, atol=0)
