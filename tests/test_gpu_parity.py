"""GPU parity: the CUDA BP-SF path (through the C ABI) against the CPU oracle.

Same seeded inputs on both sides.  Integer work (syndromes, Phi, trial
syndromes, flip counts, parity checks) must match bit for bit; posterior
LLRs within |d| <= 1e-4 * max(1, |L|); corrections identical on >= 99.99% of
shots; the logical error rate within the binomial 1-sigma of the FP64 oracle.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import Code, Params as OParams  # noqa: E402
from paper_2507_00254_gb300 import bpsf as B  # noqa: E402
from paper_2507_00254_gb300 import build as libbuild  # noqa: E402
from paper_2507_00254_gb300 import codes  # noqa: E402

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
CORR_MATCH = 0.9999
LLR_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    libbuild.build()
    return B.lib()


def pack(bits):
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    n, nb = bits.shape
    w = (nb + 31) // 32
    pad = np.zeros((n, 32 * w), dtype=np.uint8)
    pad[:, :nb] = bits
    return np.packbits(pad.reshape(n, w * 4, 8), axis=-1, bitorder="little").reshape(n, w * 4).view(np.uint32)


def unpack(words, nb):
    words = np.ascontiguousarray(words).view(np.uint8)
    return np.unpackbits(words.reshape(words.shape[0], -1), axis=-1, bitorder="little")[:, :nb]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def oracle_code(name):
    if name.endswith("_phenom"):
        hx, _ = oracle.named_code(name[: -len("_phenom")])
        return Code(oracle.phenom_code(hx, 12))
    hx, _ = oracle.named_code(name)
    return Code(hx)


def product_code(name):
    return codes.phenom(name[: -len("_phenom")]) if name.endswith("_phenom") else codes.bb(name)


def make_inputs(name, p, n, seed, stream=0):
    oc = oracle_code(name)
    if name.endswith("_phenom"):
        e = synth.phenom_error_bits(seed, stream, 0, n, 144, 72, 12, p, p)
    else:
        e = synth.bernoulli_bits(seed, stream, 0, n, oc.N, p)
    s = oc.syndrome(e)
    return oc, e, s


def decoder(name, p, params):
    c = product_code(name)
    return B.Decoder(c.ptr, c.idx, c.M, c.N, np.full(c.N, p), params)


def oparams(P):
    return OParams(P.max_iter, P.alpha, P.w, P.w_max, P.short_iter, P.select, layered=P.layered)


def gpu_decode(dec, s_bits, **kw):
    out = dec.decode(dev(pack(s_bits)), **kw)
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare(oc, dec, s, p, P, e_bits=None, fp32=True):
    eo, co, io, so = oc.bpsf_batch(s, p, oparams(P), fp32=fp32, threads=THREADS)
    g = gpu_decode(dec, s)
    eg = unpack(g["corr"], oc.N)
    same = (eg == eo).all(axis=1)
    frac = same.mean()
    assert frac >= CORR_MATCH, "corrections match on %.6f of shots" % frac
    assert ((g["conv"] != 0) == co)[same].all()
    assert (g["iters"] == io)[same].all()
    assert (g["stage"] == so)[same].all()
    # Every converged correction satisfies the syndrome (checked by the oracle).
    conv = g["conv"] != 0
    if conv.any():
        assert (oc.syndrome(eg[conv]) == s[conv]).all()
    return g, (eo, co, io, so)


# --------------------------------------------------------------------------
# Workload parity
# --------------------------------------------------------------------------

def test_bb72_workload_matches_oracle():
    """[[72,12,6]], p = 0.05, 10^4 shots, max_iter 50, w 4, short_iter 10."""
    P = B.Params(max_iter=50, alpha=0.625, w=4, short_iter=10)
    oc, e, s = make_inputs("bb72", 0.05, 10000, synth.SEEDS["bb72_cc"])
    dec = decoder("bb72", 0.05, P)
    g, (eo, co, io, so) = compare(oc, dec, s, 0.05, P)
    assert (so == 2).sum() < (so == 1).sum() + (so == 0).sum()
    assert (g["stage"] == 1).sum() > 0  # the trial path ran


# The paper's code-capacity settings for its other code families (Section V,
# Fig. capacity and the [[154]] study): adaptive damping alpha_t = 1 - 2^-t,
# weight-1 trial vectors, |Phi| = 6 ([[126]]), 13 ([[254]]) and 8 ([[154]]),
# 50 iterations per run.
FAMILY_CASES = [("cbb126", 6, 0), ("gb254", 13, 1), ("cbb154", 8, 2)]


@pytest.mark.parametrize("name,w,k", FAMILY_CASES)
def test_code_families_match_oracle(name, w, k):
    p = 0.06
    P = B.Params(max_iter=50, alpha=0.0, w=w, w_max=1, short_iter=50)
    oc, e, s = make_inputs(name, p, 3000, synth.SEEDS["families"][k])
    dec = decoder(name, p, P)
    g, (eo, co, io, so) = compare(oc, dec, s, p, P)
    assert (g["stage"] == 1).sum() > 0  # the trial path ran
    assert B.bpsf_num_trials(dec.handle) == w


# The sampled variant (Section V): n_s random trial vectors per weight
# 1..w_max over |Phi| = 50, the setting of the paper's complexity study
# (w_max = 6, n_s = 5, 100 iterations per BP instance, adaptive damping).
@pytest.mark.parametrize("name,p,n", [("bb144", 0.06, 2000), ("bb144_phenom", 0.008, 1500)])
def test_sampled_trial_list_matches_oracle(name, p, n):
    masks = synth.sample_trial_masks(7001, 50, 6, 5)
    P = B.Params(max_iter=100, alpha=0.0, w=50, w_max=6, short_iter=100)
    oc, e, s = make_inputs(name, p, n, 7002)
    dec = decoder(name, p, P)
    dec.set_trials(masks)
    assert B.bpsf_num_trials(dec.handle) == 30
    OP = oparams(P)
    OP = OParams(OP.max_iter, OP.alpha, OP.w, OP.w_max, OP.short_iter, OP.select, tuple(int(m) for m in masks))
    eo, co, io, so = oc.bpsf_batch(s, p, OP, fp32=True, threads=THREADS)
    g = gpu_decode(dec, s)
    eg = unpack(g["corr"], oc.N)
    same = (eg == eo).all(axis=1)
    assert same.mean() >= CORR_MATCH, same.mean()
    for k, ref in (("conv", co), ("iters", io), ("stage", so)):
        assert ((g[k] != 0) == ref if k == "conv" else g[k] == ref)[same].all(), k
    assert (g["stage"] == 1).sum() > 0
    # Weight <= 6 over 50 bits is far beyond 4096 trials: the create-time set is
    # empty, and decoding without a list is refused.
    dec.set_trials([])
    assert B.bpsf_num_trials(dec.handle) == 0
    with pytest.raises(B.BpsfError) as ei:
        gpu_decode(dec, s[:4])
    assert ei.value.status == B.BPSF_EINVAL


def test_set_trials_rejects_bad_masks():
    P = B.Params(max_iter=50, alpha=0.625, w=4, short_iter=10)
    dec = decoder("bb72", 0.05, P)
    n0 = B.bpsf_num_trials(dec.handle)
    assert n0 == 15
    for bad in ([0], [1 << 4], [(1 << 17) - 1]):
        with pytest.raises(B.BpsfError) as ei:
            dec.set_trials(np.array(bad, dtype=np.uint64))
        assert ei.value.status == B.BPSF_EINVAL
    dec.set_trials([3, 1])
    assert B.bpsf_num_trials(dec.handle) == 2
    dec.set_trials([])
    assert B.bpsf_num_trials(dec.handle) == n0


def test_first_success_cancels_trials_that_cannot_win():
    """Under the first-success rule trials after the earliest converged one are not run
    (or are stopped); the results still equal the oracle's, which runs every trial."""
    p = 0.06
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20, select=B.BPSF_SELECT_FIRST)
    oc, e, s = make_inputs("bb144", p, 3000, synth.SEEDS["bb144_cc"][2], stream=2)
    dec = decoder("bb144", p, P)
    compare(oc, dec, s, p, P)
    wf = dec.last_work()
    assert wf["trials_cancelled"] > 0
    assert wf["trial_runs"] + wf["trials_cancelled"] == 63 * wf["failed_shots"]
    Pm = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    decm = decoder("bb144", p, Pm)
    gpu_decode(decm, s)
    wm = decm.last_work()
    assert wm["trials_cancelled"] == 0 and wm["failed_shots"] == wf["failed_shots"]
    assert wf["iterations"] < wm["iterations"]


def test_adaptive_damping_matches_oracle():
    """[[144,12,12]] at p = 0.06 with alpha_t = 1 - 2^-t instead of 0.625."""
    p = 0.06
    P = B.Params(max_iter=100, alpha=0.0, w=6, short_iter=20)
    oc, e, s = make_inputs("bb144", p, 3000, synth.SEEDS["bb144_cc"][2], stream=1)
    dec = decoder("bb144", p, P)
    compare(oc, dec, s, p, P)


@pytest.mark.parametrize("p_idx", range(4))
def test_bb144_workload_matches_oracle(p_idx):
    """[[144,12,12]] at p in {0.02, 0.04, 0.06, 0.08}: max_iter 100, w 6, short_iter 20."""
    p = (0.02, 0.04, 0.06, 0.08)[p_idx]
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    oc, e, s = make_inputs("bb144", p, 3000, synth.SEEDS["bb144_cc"][p_idx])
    dec = decoder("bb144", p, P)
    compare(oc, dec, s, p, P)


@pytest.mark.parametrize("p,n,seed_idx,min_sf,min_fail", [(0.002, 20000, 0, 1, 0), (0.004, 30000, 1, 50, 10),
                                                        (0.010, 3000, 1, 50, 10)])
def test_phenomenological_matches_oracle(p, n, seed_idx, min_sf, min_fail):
    """12-round phenomenological [[144]] (864 x 2592), p = q: max_iter 200, w 5 (31 trials), short_iter 30.

    Enough shots that the trial path (stage 1) and the total-failure output
    (stage 2, 31 failed trials) are both compared many times."""
    P = B.Params(max_iter=200, alpha=0.625, w=5, short_iter=30)
    oc, e, s = make_inputs("bb144_phenom", p, n, synth.SEEDS["bb144_phenom"][seed_idx])
    dec = decoder("bb144_phenom", p, P)
    g, (eo, co, io, so) = compare(oc, dec, s, p, P)
    assert (so == 1).sum() >= min_sf and (so == 2).sum() >= min_fail
    assert (g["stage"] == so).all() and (g["iters"] == io).all()


def test_mixed_codes_one_launch_match_oracle():
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    names = ["bb72", "bb90", "bb108", "bb144", "bb288"]
    decs, synds, cases = [], [], []
    for k, name in enumerate(names):
        n = 300 + 97 * k
        oc, e, s = make_inputs(name, 0.05, n, synth.SEEDS["mixed"][k])
        decs.append(decoder(name, 0.05, P))
        synds.append(dev(pack(s)))
        cases.append((oc, s))
    outs = B.decode_multi(decs, synds)
    for (oc, s), o in zip(cases, outs):
        eo, co, io, so = oc.bpsf_batch(s, 0.05, oparams(P), threads=THREADS)
        eg = unpack(o["corr"].cpu().numpy(), oc.N)
        same = (eg == eo).all(axis=1)
        assert same.mean() >= CORR_MATCH
        assert ((o["conv"].cpu().numpy() != 0) == co)[same].all()
        assert (o["iters"].cpu().numpy() == io)[same].all()
        assert (o["stage"].cpu().numpy() == so)[same].all()


# --------------------------------------------------------------------------
# Layered schedule (the paper's variant for [[288]])
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,p,n,alpha", [("bb144", 0.06, 2000, 0.625), ("bb288", 0.06, 1500, 0.0),
                                            ("bb144_phenom", 0.006, 800, 0.625)])
def test_layered_schedule_matches_oracle(name, p, n, alpha):
    P = B.Params(max_iter=100, alpha=alpha, w=6, short_iter=20, layered=True)
    oc, e, s = make_inputs(name, p, n, 7301)
    dec = decoder(name, p, P)
    g, (eo, co, io, so) = compare(oc, dec, s, p, P)
    assert (g["stage"] != 0).sum() > 0


def test_layered_and_flooding_codes_in_one_launch():
    Pl = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20, layered=True)
    Pf = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    decs, synds, cases = [], [], []
    for k, (name, P) in enumerate((("bb144", Pl), ("bb72", Pf), ("bb288", Pl))):
        oc, e, s = make_inputs(name, 0.05, 500 + 100 * k, 7400 + k)
        decs.append(decoder(name, 0.05, P))
        synds.append(dev(pack(s)))
        cases.append((oc, s, P))
    outs = B.decode_multi(decs, synds)
    for (oc, s, P), o in zip(cases, outs):
        eo, co, io, so = oc.bpsf_batch(s, 0.05, oparams(P), threads=THREADS)
        eg = unpack(o["corr"].cpu().numpy(), oc.N)
        assert (eg == eo).all(axis=1).mean() >= CORR_MATCH
        assert (o["iters"].cpu().numpy() == io).mean() >= CORR_MATCH


# --------------------------------------------------------------------------
# Step-level parity through the debug dump
# --------------------------------------------------------------------------

# (code, p, shots, params, least failed shots): the [[72]] workload's settings,
# the [[144]] benchmark settings at its highest p, and the phenomenological
# settings on the row-weight-8 kernel variant.
DUMP_CASES = [("bb72", 0.09, 1500, (50, 4, 10), 20), ("bb144", 0.08, 800, (100, 6, 20), 100),
              ("bb144_phenom", 0.010, 1500, (200, 5, 30), 15)]


@pytest.mark.parametrize("name,p,n,prm,min_failed", DUMP_CASES)
def test_internal_values_match_oracle_bit_for_bit(name, p, n, prm, min_failed):
    """LLRs, flip counts, Phi, trial syndromes and trial outcomes on a failure-heavy batch."""
    max_iter, w, short_iter = prm
    P = B.Params(max_iter=max_iter, alpha=0.625, w=w, short_iter=short_iter)
    oc, e, s = make_inputs(name, p, n, 77)
    dec = decoder(name, p, P)
    g = dec.decode_debug(dev(pack(s)))
    g = {k: v.cpu().numpy() for k, v in g.items()}
    n_failed = n_trial_conv = 0
    for k in range(s.shape[0]):
        r = oc.bp(s[k], p, P.max_iter, P.alpha, fp32=True, track=True)
        L = r["lout"].astype(np.float64)
        d = np.abs(g["lout"][k].astype(np.float64) - L)
        assert (d <= LLR_TOL * np.maximum(1.0, np.abs(L))).all()
        assert (g["flips"][k].astype(np.uint16) == r["flips"]).all()
        if r["converged"]:
            continue
        n_failed += 1
        phi = oracle.top(r["flips"], P.w)
        assert (g["phi"][k] == phi).all()
        synd, conv, iters, es = oc.trials(s[k], p, phi, oparams(P))
        tsyn = unpack(g["trial_synd"][k].reshape(len(synd), -1), oc.M)
        assert (tsyn == synd).all()
        assert (g["trial_conv"][k] == conv).all()
        assert (g["trial_iters"][k] == iters).all()
        n_trial_conv += int(conv.sum())
    assert n_failed >= min_failed and n_trial_conv > 0


# --------------------------------------------------------------------------
# Forms and launch shapes give identical results
# --------------------------------------------------------------------------

def test_launch_shape_does_not_change_results():
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    oc, e, s = make_inputs("bb144", 0.07, 4000, 5)
    dec = decoder("bb144", 0.07, P)
    ref = gpu_decode(dec, s)
    # (W, S, B, blocks per SM, iteration chunk): the chunk delays refills only.
    for t in [(1, 1, 4, 0), (1, 16, 4, 0), (2, 2, 8, 0), (4, 1, 8, 1), (1, 8, 4, 0), (1, 2, 15, 0), (8, 1, 8, 0),
              (1, 32, 2, 0), (8, 32, 8, 0), (4, 16, 12, 0), (1, 4, 12, 0), (2, 4, 8, 0), (1, 8, 12, 0, 4),
              (1, 4, 15, 0, 8), (2, 8, 8, 0, 2), (4, 1, 12, 0, 3), (1, 32, 3, 0, 64)]:
        dec.tuning = t
        got = gpu_decode(dec, s)
        for key in ("corr", "conv", "iters", "stage"):
            assert (got[key] == ref[key]).all(), (t, key)
    with pytest.raises(B.BpsfError):
        dec.tuning = (1, 8, 12, 0, 65)


def test_autotune_result_is_accepted_cached_and_decodes_like_the_oracle():
    """bpsf_autotune picks a shape (threads per shot, shots per block,
    iteration chunk) that bpsf_set_tuning accepts; a second context of the
    same code and parameters starts with it from the cache; decoding under it
    equals the oracle."""
    P = B.Params(max_iter=50, alpha=0.625, w=4, short_iter=10)
    dec = decoder("bb72", 0.06, P)
    chosen = dec.autotune(p_sample=0.06, n_sample=1 << 13)
    assert dec.tuning == chosen
    W, S, Bw, bps, chunk = chosen
    assert W in (1, 2, 4, 8) and S in (1, 2, 4, 8, 16, 32) and Bw % W == 0 and 1 <= max(chunk, 1) <= 8
    fresh = decoder("bb72", 0.06, P)
    assert fresh.tuning == chosen  # from the cache: same code shape and parameters
    fresh.tuning = (1, 1, 1, 0)
    fresh.tuning = chosen  # accepted by bpsf_set_tuning
    oc, e, s = make_inputs("bb72", 0.06, 3000, 41)
    compare(oc, fresh, s, 0.06, P)


def test_one_byte_flip_words():
    """Thirteen teams of 8 slots fit on an SM only with one-byte flip words
    (max_iter <= 127): results, flip counts, Phi and posteriors equal those of
    the two-byte shape; with max_iter > 127 the shape is refused."""
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    oc, e, s = make_inputs("bb144", 0.07, 3000, 31)
    dec = decoder("bb144", 0.07, P)
    dec.tuning = (1, 8, 12, 0)
    ref = gpu_decode(dec, s)
    ref_dbg = {k: v.cpu().numpy() for k, v in dec.decode_debug(dev(pack(s[:400]))).items()}
    dec.tuning = (1, 8, 13, 0)
    got = gpu_decode(dec, s)
    for key in ("corr", "conv", "iters", "stage"):
        assert (got[key] == ref[key]).all(), key
    dbg = {k: v.cpu().numpy() for k, v in dec.decode_debug(dev(pack(s[:400]))).items()}
    for key in ("flips", "phi", "lout", "trial_conv", "trial_iters", "corr"):
        assert (dbg[key] == ref_dbg[key]).all(), key
    eo, co, io, so = oc.bpsf_batch(s, 0.07, oparams(P), threads=THREADS)
    assert (unpack(got["corr"], oc.N) == eo).all(axis=1).mean() >= CORR_MATCH
    long_runs = decoder("bb144", 0.07, B.Params(max_iter=200, alpha=0.625, w=6, short_iter=20))
    with pytest.raises(B.BpsfError) as ei:
        long_runs.tuning = (1, 8, 13, 0)
    assert ei.value.status == B.BPSF_EINVAL


def test_sharded_batch_equals_its_pieces_decoded_alone():
    """A batch large enough to be decoded as four shards (streams of one launch
    with their own counters and record-ring slices) gives exactly the outputs
    and work of its four quarters decoded one by one (too small to shard)."""
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    q = 9000
    oc, e, s = make_inputs("bb144", 0.07, 4 * q, 21)
    dec = decoder("bb144", 0.07, P)
    whole = gpu_decode(dec, s)
    ww = dec.last_work()
    parts, works = [], []
    for k in range(4):
        parts.append(gpu_decode(dec, s[k * q:(k + 1) * q]))
        works.append(dec.last_work())
    for key in ("corr", "conv", "iters", "stage"):
        assert (whole[key] == np.concatenate([p_[key] for p_ in parts])).all(), key
    for key in ("initial_runs", "failed_shots", "trial_runs", "iterations", "edge_updates"):
        assert ww[key] == sum(w_[key] for w_ in works), key
    assert ww["initial_runs"] == 4 * q and (whole["stage"] == 1).sum() > 0
    # And the oracle on a sample of each quarter.
    idx = np.concatenate([k * q + np.arange(0, q, 37) for k in range(4)])
    eo, co, io, so = oc.bpsf_batch(s[idx], 0.07, oparams(P), threads=THREADS)
    assert (unpack(whole["corr"][idx], oc.N) == eo).all(axis=1).mean() >= CORR_MATCH
    assert (whole["stage"][idx] == so).all()


def test_launch_shape_irregular_code():
    """Every slot count has its own message layout (rank stride and edge order);
    for the irregular-row [[254,28]] code the strides differ from M at some slot
    counts.  Results equal the oracle at each of them."""
    P = B.Params(max_iter=60, alpha=0.625, w=5, short_iter=15)
    oc, e, s = make_inputs("gb254", 0.03, 600, 6)
    dec = decoder("gb254", 0.03, P)
    eo, co, io, so = oc.bpsf_batch(s, 0.03, oparams(P), threads=THREADS)
    for t in [(1, 1, 8, 0), (1, 2, 8, 0), (1, 4, 8, 0), (1, 8, 4, 0), (2, 16, 2, 0)]:
        dec.tuning = t
        got = gpu_decode(dec, s)
        assert (unpack(got["corr"], oc.N) == eo).all(axis=1).mean() >= CORR_MATCH, t
        assert (got["stage"] == so).mean() >= CORR_MATCH, t
        assert (got["iters"] == io).mean() >= CORR_MATCH, t


def test_cuda_graph_replay_equals_eager():
    """A decode recorded into a CUDA graph after a warm-up call (counter and
    queue resets plus the persistent launch) replays to the eager results,
    also after new syndromes are written into the recorded input buffer; the
    same for a mixed-code launch."""
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    n = 3000
    _, _, s1 = make_inputs("bb144", 0.07, n, 21)
    _, _, s2 = make_inputs("bb144", 0.07, n, 22)
    dec = decoder("bb144", 0.07, P)
    refs = [gpu_decode(dec, s) for s in (s1, s2)]
    synd = dev(pack(s1))
    out = dec.outputs(n)
    dec.decode(synd, out=out)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dec.decode(synd, out=out, sync=False)
    for s, ref in zip((s1, s2), refs):
        synd.copy_(dev(pack(s)))
        for v in out.values():
            v.zero_()
        g.replay()
        torch.cuda.synchronize()
        for key in ("corr", "conv", "iters", "stage"):
            assert (out[key].cpu().numpy() == ref[key]).all(), key
    # Two codes in one recorded launch.
    _, _, s3 = make_inputs("bb72", 0.06, 1500, 23)
    dec72 = decoder("bb72", 0.06, P)
    synds = [dev(pack(s1)), dev(pack(s3))]
    ref = B.decode_multi([dec, dec72], synds)
    ref = [{k: v.clone() for k, v in o.items()} for o in ref]
    outs = B.decode_multi([dec, dec72], synds)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2):
        B.decode_multi([dec, dec72], synds, outs=outs, sync=False)
    for o in outs:
        for v in o.values():
            v.zero_()
    g2.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        for key in r:
            assert torch.equal(o[key], r[key]), key


def test_plain_form_equals_batched_form():
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    oc, e, s = make_inputs("bb144", 0.07, 300, 6)
    dec = decoder("bb144", 0.07, P)
    a = gpu_decode(dec, s)
    b = gpu_decode(dec, s, plain=True)
    for key in ("corr", "conv", "iters", "stage"):
        assert (a[key] == b[key]).all(), key
    assert (a["stage"] == 1).any()


def test_host_buffer_form_equals_device_form():
    P = B.Params(max_iter=50, alpha=0.625, w=4, short_iter=10)
    oc, e, s = make_inputs("bb72", 0.06, 2000, 8)
    dec = decoder("bb72", 0.06, P)
    a = gpu_decode(dec, s)
    h = dec.decode_host(pack(s))
    assert (h["corr"].view(np.int32) == a["corr"]).all()
    assert (h["conv"] == a["conv"]).all() and (h["iters"] == a["iters"]).all() and (h["stage"] == a["stage"]).all()


def test_multi_host_form_equals_device_multi_and_oracle():
    """bpsf_decode_multi_host: one launch over host buffers of several codes,
    including an empty job; results equal the device-buffer multi launch and
    the oracle."""
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    names = ["bb72", "bb144", "bb288", "bb90"]
    sizes = [700, 1200, 400, 0]
    decs, host_synds, cases = [], [], []
    for k, (name, n) in enumerate(zip(names, sizes)):
        oc, e, s = make_inputs(name, 0.06, max(n, 1), synth.SEEDS["mixed"][k])
        s = s[:n]
        decs.append(decoder(name, 0.06, P))
        host_synds.append(pack(s))
        cases.append((oc, s))
    h = B.decode_multi_host(decs, host_synds)
    live = [k for k, n in enumerate(sizes) if n > 0]
    d = B.decode_multi([decs[k] for k in live], [dev(host_synds[k]) for k in live])
    for k, o in zip(live, d):
        assert (h[k]["corr"].view(np.int32) == o["corr"].cpu().numpy()).all()
        for f in ("conv", "iters", "stage"):
            assert (h[k][f] == o[f].cpu().numpy()).all()
        oc, s = cases[k]
        eo, co, io, so = oc.bpsf_batch(s, 0.06, oparams(P), threads=THREADS)
        assert (unpack(h[k]["corr"].view(np.int32), oc.N) == eo).all(axis=1).mean() >= CORR_MATCH
        assert (h[k]["stage"] == so).mean() >= CORR_MATCH
    assert h[3]["corr"].shape == (0, decs[3].Wn)


# --------------------------------------------------------------------------
# Variants and edge cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["bp_only", "select_first", "w_max2", "ragged_bb90"])
def test_variants_match_oracle(variant):
    name, p = "bb72", 0.08
    P = B.Params(max_iter=50, alpha=0.625, w=4, short_iter=10)
    if variant == "bp_only":
        P = B.Params(max_iter=50, alpha=0.625, w=0)
    elif variant == "select_first":
        P.select = B.BPSF_SELECT_FIRST
    elif variant == "w_max2":
        P = B.Params(max_iter=50, alpha=0.625, w=5, w_max=2, short_iter=10)
    elif variant == "ragged_bb90":
        name, p = "bb90", 0.06
    oc, e, s = make_inputs(name, p, 2000, 9)
    compare(oc, decoder(name, p, P), s, p, P)


def test_edge_cases():
    P = B.Params(max_iter=50, alpha=0.625, w=4, short_iter=10)
    dec = decoder("bb90", 0.05, P)  # M = 45, N = 90: ragged words on both sides
    oc = oracle_code("bb90")
    # Empty batch.
    out = dec.outputs(1)
    B.bpsf_decode(dec.handle, 0, 0, 2, 0, 3, 0, 0, 0, 0)
    # Zero syndromes converge at iteration 1 with e = 0.
    g = gpu_decode(dec, np.zeros((5, 45), dtype=np.uint8))
    assert (g["conv"] == 1).all() and (g["iters"] == 1).all() and (g["corr"] == 0).all() and (g["stage"] == 0).all()
    # One shot; all-ones syndrome (maximum weight).
    s1 = np.ones((1, 45), dtype=np.uint8)
    compare(oc, dec, s1, 0.05, P)
    # Padding bits beyond M are ignored; wide strides are honoured.
    oc2, e, s = make_inputs("bb90", 0.06, 700, 10)
    packed = pack(s)
    wide = np.zeros((packed.shape[0], 4), dtype=np.uint32)
    wide[:, :2] = packed
    wide[:, 1] |= np.uint32(0xFFFFE000)  # bits 45..63 set
    wide[:, 2:] = np.uint32(0xDEADBEEF)
    o = dec.outputs(len(s))
    o["corr"] = torch.zeros((len(s), 6), dtype=torch.int32, device="cuda")
    dec.decode(dev(wide), out=o)
    ref = gpu_decode(dec, s)
    got = o["corr"].cpu().numpy()
    assert (got[:, :3] == ref["corr"]).all() and (got[:, 3:] == 0).all()
    assert (o["stage"].cpu().numpy() == ref["stage"]).all()
    # Strides below the word count are rejected.
    with pytest.raises(B.BpsfError) as ei:
        B.bpsf_decode(dec.handle, 1, out["corr"].data_ptr(), 1, out["corr"].data_ptr(), 3,
                      out["conv"].data_ptr(), out["iters"].data_ptr(), 0, 0)
    assert ei.value.status == B.BPSF_EINVAL


def test_work_counters_are_consistent():
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    oc, e, s = make_inputs("bb144", 0.08, 2000, 11)
    dec = decoder("bb144", 0.08, P)
    g = gpu_decode(dec, s)
    w = dec.last_work()
    assert w["initial_runs"] == 2000
    assert w["failed_shots"] == int((g["stage"] != 0).sum())
    assert w["trial_runs"] == w["failed_shots"] * 63
    assert w["edge_updates"] == w["iterations"] * 432
    assert w["iterations"] >= int(g["iters"][g["stage"] == 0].sum()) + 100 * w["failed_shots"]
    # Slots offered while teams worked: at least the iterations run, at most all of them busy.
    S = dec.tuning[1]
    assert w["iterations"] <= w["slot_capacity"] and w["slot_capacity"] % S == 0


# --------------------------------------------------------------------------
# Full-size configuration: sampled parity plus properties of every shot
# --------------------------------------------------------------------------

def test_full_size_bb144_p008_sampled_parity_and_ler():
    """10^6 shots at p = 0.08 in the benchmark's launch shape; oracle on a random sample."""
    p, n = 0.08, 1_000_000
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    c = product_code("bb144")
    e = synth.bernoulli_bits(synth.SEEDS["bb144_cc"][3], 0, 0, n, c.N, p)
    dec = decoder("bb144", p, P)
    err = dev(pack(e))
    synd = dec.syndrome(err)
    torch.cuda.synchronize()
    out = dec.decode(synd)
    corr = out["corr"]
    conv = out["conv"].bool()
    # Property on every shot: converged corrections satisfy their syndrome.
    resid = dec.syndrome(corr)
    assert bool(((resid == synd).all(dim=1) | ~conv).all())
    stage = out["stage"].cpu().numpy()
    assert set(np.unique(stage)).issubset({0, 1, 2})
    assert ((stage < 2) == conv.cpu().numpy()).all()
    # Oracle on a random sample of shots.
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(n, size=1500, replace=False))
    oc = oracle_code("bb144")
    s_np = unpack(synd.cpu().numpy()[idx], 72)
    assert (s_np == oc.syndrome(e[idx])).all()
    eo, co, io, so = oc.bpsf_batch(s_np, p, oparams(P), threads=THREADS)
    eg = unpack(corr.cpu().numpy()[idx], 144)
    assert (eg == eo).all(axis=1).mean() >= CORR_MATCH
    # Logical error rate within the binomial 1-sigma of the FP64 oracle on the same shots.
    hx, hz = oracle.named_code("bb144")
    lx = oracle.logicals(hx, hz)
    e64, c64, _, _ = oc.bpsf_batch(s_np, p, oparams(P), fp32=False, threads=THREADS)
    f64 = oracle.logical_failures(hx, lx, e[idx], e64, c64).mean()
    fg = oracle.logical_failures(hx, lx, e[idx], eg, conv.cpu().numpy()[idx]).mean()
    sigma = np.sqrt(max(f64 * (1 - f64), 1e-12) / len(idx))
    assert abs(fg - f64) <= sigma + 1e-12


@pytest.mark.parametrize("p_idx", range(4))
def test_ler_within_one_sigma_of_fp64_oracle(p_idx):
    """[[144,12,12]] benchmark settings, 10^5 shots per p: the GPU's logical error
    rate lies within the binomial 1-sigma of the FP64 oracle on the same shots."""
    p = (0.02, 0.04, 0.06, 0.08)[p_idx]
    n = 100_000
    P = B.Params(max_iter=100, alpha=0.625, w=6, short_iter=20)
    oc, e, s = make_inputs("bb144", p, n, synth.SEEDS["bb144_cc"][p_idx])
    dec = decoder("bb144", p, P)
    g = gpu_decode(dec, s)
    eg = unpack(g["corr"], oc.N)
    e64, c64, _, _ = oc.bpsf_batch(s, p, oparams(P), fp32=False, threads=THREADS)
    hx, hz = oracle.named_code("bb144")
    lx = oracle.logicals(hx, hz)
    f64 = oracle.logical_failures(hx, lx, e, e64, c64).mean()
    fg = oracle.logical_failures(hx, lx, e, eg, g["conv"] != 0).mean()
    sigma = np.sqrt(max(f64 * (1 - f64), 1e-12) / n)
    assert abs(fg - f64) <= sigma + 1e-12, (fg, f64, sigma)
    assert (eg == e64).all(axis=1).mean() >= CORR_MATCH


def test_c2v_clamp_where_it_fires_matches_oracle():
    """H = [[1,1],[1,1],[1,1]], s = (1,0,0) never converges; with alpha_t -> 1 the
    messages grow by half a bit per iteration until the 2^100 clamp holds them.
    The kernel's posteriors equal the FP32 oracle's bit for bit before, at and
    after saturation."""
    H = np.array([[1, 1], [1, 1], [1, 1]], dtype=np.uint8)
    ptr = np.array([0, 2, 4, 6], dtype=np.int32)
    idx = np.array([0, 1, 0, 1, 0, 1], dtype=np.int32)
    oc = Code(H)
    s = np.array([[1, 0, 0]] * 4, dtype=np.uint8)
    for T in (100, 260, 401):
        P = B.Params(max_iter=T, alpha=0.0, w=2, short_iter=10)
        dec = B.Decoder(ptr, idx, 3, 2, np.full(2, 0.1), P)
        g = dec.decode_debug(dev(pack(s)))
        r = oc.bp(s[0], 0.1, T, 0.0, fp32=True, track=True)
        lg = g["lout"].cpu().numpy()
        assert (lg == r["lout"][None, :]).all()
        assert np.isfinite(lg).all()
        if T >= 260:
            assert (np.abs(lg) >= 2.0 ** 100).all()
        assert (g["stage"].cpu().numpy() == 2).all() and (g["iters"].cpu().numpy() == T).all()
        eo, co, io, so = oc.bpsf_batch(s, 0.1, oparams(P), threads=1)
        assert (unpack(g["corr"].cpu().numpy(), 2) == eo).all()
        dec.close()
