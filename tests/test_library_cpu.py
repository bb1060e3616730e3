"""CPU checks of the C ABI: the library loads, exports every declared symbol,
its host-side builders match the oracle's, and argument checks reject bad
input before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2507_00254_gb300 import bpsf as B
from paper_2507_00254_gb300 import build as libbuild
from paper_2507_00254_gb300 import codes, harness

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    libbuild.build()
    return B.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bpsf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bpsf_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 20
    L = B.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(B.EXPORTS) == names


def test_status_strings():
    L = B.lib()
    assert L.bpsf_status_str(0) == b"ok"
    assert L.bpsf_status_str(4) == b"timeout"


@pytest.mark.parametrize("name", ["bb72", "bb90", "bb108", "bb144", "bb288", "gb254", "cbb126", "cbb154"])
def test_bb_builder_matches_oracle(name):
    hx_o, hz_o = oracle.named_code(name)
    assert (codes.bb(name, 0).dense() == hx_o).all()
    assert (codes.bb(name, 1).dense() == hz_o).all()


def test_phenom_builder_matches_oracle():
    hx_o, _ = oracle.named_code("bb144")
    H_o = oracle.phenom_code(hx_o, 12)
    c = codes.phenom("bb144", 12)
    assert (c.M, c.N, int(c.ptr[-1])) == (864, 2592, 6840)
    assert (c.dense() == H_o).all()


def test_bb_builder_cancels_repeated_terms():
    ptr, idx = B.bpsf_bb_code(3, 3, [(1, 0), (1, 0), (0, 1)], [(0, 0)])
    assert (np.diff(ptr) == 2).all()


def test_pack_roundtrip():
    rng = np.random.default_rng(0)
    for nb in (1, 31, 32, 33, 72, 144, 2592):
        bits = rng.integers(0, 2, size=(7, nb), dtype=np.uint8)
        assert (harness.unpack_rows(harness.pack_rows(bits), nb) == bits).all()


def test_harness_logicals_agree_with_oracle_rank():
    hx, hz = codes.bb("bb72", 0).dense(), codes.bb("bb72", 1).dense()
    lx = harness.x_logicals(hx, hz)
    assert lx.shape[0] == 12
    assert not ((hz.astype(int) @ lx.T.astype(int)) % 2).any()
    assert oracle.gf2_rank(np.vstack([hx, lx])) == oracle.gf2_rank(hx) + 12


def _create(M, N, ptr, idx, priors, **kw):
    p = B.Params(**kw).c()
    return B.bpsf_create(M, N, B.BPSF_CSR, ptr, idx, priors, p)


def test_create_rejects_bad_arguments_before_device_work():
    c = codes.bb("bb72")
    good = dict(max_iter=50, w=4, short_iter=10)
    cases = [
        (dict(priors=0.6), "prior"),
        (dict(priors=0.0), "prior"),
        (dict(max_iter=0), "max_iter"),
        (dict(w=65), "w must"),
        (dict(w=17), "w_max must be at most 16"),
        (dict(w=4, w_max=5), "w_max"),
        (dict(short_iter=60), "short_iter"),
        (dict(alpha=-0.5), "alpha"),
        (dict(alpha=float("inf")), "alpha"),
        (dict(select=3), "select"),
    ]
    for over, msg in cases:
        kw = dict(good)
        priors = over.pop("priors", 0.05)
        kw.update(over)
        with pytest.raises(B.BpsfError) as ei:
            _create(c.M, c.N, c.ptr, c.idx, priors, **kw)
        assert ei.value.status == B.BPSF_EINVAL and msg in str(ei.value), (over, str(ei.value))
    # Only the layered-schedule bit of params.flags is defined.
    p = B.Params(**good).c()
    p.flags = 2
    with pytest.raises(B.BpsfError) as ei:
        B.bpsf_create(c.M, c.N, B.BPSF_CSR, c.ptr, c.idx, 0.05, p)
    assert ei.value.status == B.BPSF_EINVAL and "flags" in str(ei.value)


def test_create_rejects_bad_graphs():
    ptr = np.array([0, 2, 3], dtype=np.int32)
    idx = np.array([0, 1, 2], dtype=np.int32)
    with pytest.raises(B.BpsfError, match="degree"):
        _create(2, 3, ptr, idx, 0.1, w=0)
    with pytest.raises(B.BpsfError, match="duplicate"):
        _create(1, 3, np.array([0, 2], dtype=np.int32), np.array([1, 1], dtype=np.int32), 0.1, w=0)
    with pytest.raises(B.BpsfError, match="out of range"):
        _create(1, 3, np.array([0, 2], dtype=np.int32), np.array([1, 5], dtype=np.int32), 0.1, w=0)
    with pytest.raises(B.BpsfError, match="nnz"):
        _create(1, 3, np.array([0, 0], dtype=np.int32), np.array([], dtype=np.int32), 0.1, w=0)


def test_null_context_is_rejected():
    L = B.lib()
    assert L.bpsf_decode(None, 1, None, 1, None, 1, None, None, None, None) == B.BPSF_EINVAL
    assert L.bpsf_sync(None, None) == B.BPSF_EINVAL
    assert L.bpsf_num_trials(None) == -1


def test_multi_job_calls_reject_bad_job_lists():
    """bpsf_decode_multi and bpsf_decode_multi_host check the job list before any device work."""
    L = B.lib()
    for fn in (L.bpsf_decode_multi, L.bpsf_decode_multi_host):
        assert fn(0, None, None) == B.BPSF_EINVAL
        one = (B.bpsf_job * 1)(B.bpsf_job(None, 1, None, 1, None, 1, None, None, None))
        assert fn(1, one, None) == B.BPSF_EINVAL  # NULL context
        many = (B.bpsf_job * 17)()
        assert fn(17, many, None) == B.BPSF_EINVAL  # more than 16 jobs
