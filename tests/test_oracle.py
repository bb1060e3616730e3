"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked
example and the code parameters the paper prints, closed forms, brute force on
tiny inputs, and invariants of Algorithm 1.  A plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed operand) fails one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import Code, Params


def parse_terms(s):
    return [tuple(int(x) for x in t.split(",")) for t in s.split(";")]


def np_rank(a):
    """GF(2) rank written independently of the oracle (row reduction on a copy)."""
    a = (np.array(a, dtype=np.uint8) & 1).copy()
    r = 0
    for c in range(a.shape[1]):
        piv = np.nonzero(a[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        a[[r, p]] = a[[p, r]]
        hit = np.nonzero(a[:, c])[0]
        hit = hit[hit != r]
        a[hit] ^= a[r]
        r += 1
        if r == a.shape[0]:
            break
    return r


def np_nullspace(a):
    """Basis of ker(a) over GF(2), independent of the oracle."""
    a = (np.array(a, dtype=np.uint8) & 1).copy()
    rows, cols = a.shape
    piv_cols, r = [], 0
    for c in range(cols):
        if r == rows:
            break
        piv = np.nonzero(a[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        a[[r, p]] = a[[p, r]]
        hit = np.nonzero(a[:, c])[0]
        hit = hit[hit != r]
        a[hit] ^= a[r]
        piv_cols.append(c)
        r += 1
    free = [c for c in range(cols) if c not in piv_cols]
    basis = []
    for f in free:
        v = np.zeros(cols, dtype=np.uint8)
        v[f] = 1
        for i, pc in enumerate(piv_cols):
            v[pc] = a[i, f]
        basis.append(v)
    return np.array(basis, dtype=np.uint8)


# --------------------------------------------------------------------------
# Code builder (Appendix "Code Construction")
# --------------------------------------------------------------------------

def test_shift_matrix_worked_example(golden):
    expect = np.array(golden("shift_S3.txt"), dtype=np.uint8)
    assert (oracle.shift_matrix(3) == expect).all()


def _fixture_codes(golden):
    return [(r[0], int(r[1]), int(r[2]), parse_terms(r[3]), parse_terms(r[4]), int(r[5]), int(r[6]))
            for r in golden("code_params.txt")]


def test_code_parameters_match_the_paper(golden):
    for name, l, m, a, b, n, k in _fixture_codes(golden):
        hx, hz = oracle.bb_code(l, m, a, b)
        assert hx.shape == (n // 2, n), name
        # CSS condition H_X H_Z^T = 0 (Section II-A).
        assert not ((hx.astype(np.int64) @ hz.T.astype(np.int64)) % 2).any(), name
        # k = n - rank H_X - rank H_Z, against the [[n, k]] the tables print.
        assert n - np_rank(hx) - np_rank(hz) == k, name
        assert n - oracle.gf2_rank(hx) - oracle.gf2_rank(hz) == k, name
        w = len(a) + len(b)
        assert (hx.sum(axis=1) == w).all() and (hx.sum(axis=0) == w // 2).all(), name


def test_bb_matrices_commute():
    # x and y commute, so A = a(x,y) and B = b(x,y) commute; H_X = [A|B].
    hx, hz = oracle.named_code("bb144")
    A, B = hx[:, :72].astype(np.int64), hx[:, 72:].astype(np.int64)
    assert ((A @ B - B @ A) % 2 == 0).all()
    assert (hz[:, :72] == B.T).all() and (hz[:, 72:] == A.T).all()


@pytest.mark.parametrize("name,k", [("bb72", 12), ("bb90", 8), ("bb108", 8), ("bb144", 12)])
def test_logicals(name, k):
    hx, hz = oracle.named_code(name)
    lx = oracle.logicals(hx, hz)
    assert lx.shape[0] == k
    # X logicals commute with every Z stabiliser: H_Z L_X^T = 0.
    assert not ((hz.astype(np.int64) @ lx.T.astype(np.int64)) % 2).any()
    # Independent of H_X: rank([H_X; L_X]) = rank H_X + k.
    assert np_rank(np.vstack([hx, lx])) == np_rank(hx) + k
    # Non-degenerate on Z-type candidates ker(H_X): the pairing has rank k,
    # so exactly the residuals outside rowspace(H_Z) are flagged.
    K = np_nullspace(hx)
    assert np_rank((lx.astype(np.int64) @ K.T.astype(np.int64)) % 2) == k


def test_phenomenological_matrix():
    hx, _ = oracle.named_code("bb144")
    R, m0, n0 = 12, 72, 144
    H = oracle.phenom_code(hx, R)
    assert H.shape == (864, 2592)
    assert int(H.sum()) == 6840
    rw = H.sum(axis=1)
    assert (rw[:m0] == 7).all() and (rw[m0:] == 8).all()
    cw = H.sum(axis=0)
    assert (cw[: R * n0] == 3).all()
    assert (cw[R * n0: R * n0 + (R - 1) * m0] == 2).all()
    assert (cw[R * n0 + (R - 1) * m0:] == 1).all()
    # Closed form of the model: measured syndromes m_t = H_X (e_1 ^ ... ^ e_t) ^ f_t,
    # detectors D_t = m_t ^ m_{t-1} (m_0 = 0) must equal H [e; f].
    rng = np.random.default_rng(7)
    for _ in range(20):
        e = rng.integers(0, 2, size=(R, n0), dtype=np.uint8)
        f = rng.integers(0, 2, size=(R, m0), dtype=np.uint8)
        acc = np.zeros(n0, dtype=np.int64)
        prev = np.zeros(m0, dtype=np.int64)
        det = []
        for t in range(R):
            acc = (acc + e[t]) % 2
            mt = ((hx.astype(np.int64) @ acc) + f[t]) % 2
            det.append((mt + prev) % 2)
            prev = mt
        det = np.concatenate(det)
        x = np.concatenate([e.reshape(-1), f.reshape(-1)]).astype(np.int64)
        assert ((H.astype(np.int64) @ x) % 2 == det).all()


# --------------------------------------------------------------------------
# BP framework (Section II-B) on cycle-free graphs, where BP is exact
# --------------------------------------------------------------------------

def random_tree_H(rng, n_var, n_chk):
    """Random Tanner graph that is a tree; every check has degree >= 2."""
    while True:
        H = np.zeros((n_chk, n_var), dtype=np.uint8)
        nodes = [("v", i) for i in range(n_var)] + [("c", j) for j in range(n_chk)]
        order = [nodes[i] for i in rng.permutation(len(nodes))]
        placed = {"v": [], "c": []}
        first = order.pop(0)
        placed[first[0]].append(first[1])
        pending = order
        while pending:
            for idx, (t, k) in enumerate(pending):
                other = "c" if t == "v" else "v"
                if placed[other]:
                    o = placed[other][rng.integers(len(placed[other]))]
                    if t == "v":
                        H[o, k] = 1
                    else:
                        H[k, o] = 1
                    placed[t].append(k)
                    pending.pop(idx)
                    break
        if (H.sum(axis=1) >= 2).all():
            return H


def brute_marginals(H, p, s):
    n = H.shape[1]
    E = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
    ok = (((E.astype(np.int64) @ H.T.astype(np.int64)) % 2) == s).all(axis=1)
    E = E[ok]
    logw = (E * np.log(p) + (1 - E) * np.log(1 - p)).sum(axis=1)
    out = np.zeros(n)
    for i in range(n):
        a = np.logaddexp.reduce(logw[E[:, i] == 0])
        b = np.logaddexp.reduce(logw[E[:, i] == 1])
        out[i] = a - b
    return out


def brute_min_cost(H, lch, s):
    n = H.shape[1]
    E = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
    ok = (((E.astype(np.int64) @ H.T.astype(np.int64)) % 2) == s).all(axis=1)
    E = E[ok]
    cost = E.astype(np.float64) @ lch
    return np.array([cost[E[:, i] == 1].min() - cost[E[:, i] == 0].min() for i in range(n)])


@pytest.mark.parametrize("seed", range(6))
def test_sum_product_is_exact_on_trees(seed):
    rng = np.random.default_rng(100 + seed)
    n_var, n_chk = 9 + seed % 4, 3 + seed % 3
    H = random_tree_H(rng, n_var, n_chk)
    p = rng.uniform(0.05, 0.3, size=n_var)
    e = (rng.random(n_var) < 0.3).astype(np.uint8)
    s = ((H.astype(np.int64) @ e) % 2).astype(np.uint8)
    code = Code(H)
    got = code.sumproduct(s, p, iters=n_var + n_chk + 2)
    want = brute_marginals(H, p, s)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_min_sum_alpha_one_is_min_cost_on_trees(seed):
    rng = np.random.default_rng(200 + seed)
    n_var, n_chk = 10 + seed % 3, 4 + seed % 2
    H = random_tree_H(rng, n_var, n_chk)
    p = rng.uniform(0.02, 0.3, size=n_var)
    e = (rng.random(n_var) < 0.3).astype(np.uint8)
    s = ((H.astype(np.int64) @ e) % 2).astype(np.uint8)
    code = Code(H)
    lch = np.log((1 - p) / p)
    want = brute_min_cost(H, lch, s)
    r64 = code.bp(s, p, max_iter=n_var + n_chk + 2, alpha=1.0, fp32=False, stop_on_converge=False)
    assert np.allclose(r64["lout"], want, rtol=1e-12, atol=1e-9)
    r32 = code.bp(s, p, max_iter=n_var + n_chk + 2, alpha=1.0, fp32=True, stop_on_converge=False)
    assert np.allclose(r32["lout"], want, rtol=1e-5, atol=1e-4)


# --------------------------------------------------------------------------
# Layered schedule: rows by greedy layer, running posterior
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_layered_min_sum_alpha_one_is_min_cost_on_trees(seed):
    # On a cycle-free graph the layered schedule reaches the same fixed point as
    # flooding: min-sum with alpha = 1 gives the exact min-cost differences.
    rng = np.random.default_rng(200 + seed)
    n_var, n_chk = 10 + seed % 3, 4 + seed % 2
    H = random_tree_H(rng, n_var, n_chk)
    p = rng.uniform(0.02, 0.3, size=n_var)
    e = (rng.random(n_var) < 0.3).astype(np.uint8)
    s = ((H.astype(np.int64) @ e) % 2).astype(np.uint8)
    code = Code(H)
    lch = np.log((1 - p) / p)
    want = brute_min_cost(H, lch, s)
    r64 = code.bp(s, p, max_iter=n_var + n_chk + 2, alpha=1.0, fp32=False, stop_on_converge=False, layered=True)
    assert np.allclose(r64["lout"], want, rtol=1e-9, atol=1e-9)


def test_layers_are_the_greedy_colouring():
    hx, _ = oracle.named_code("bb72")
    code = Code(hx)
    lay = code.layers()
    share = (hx.astype(np.int64) @ hx.T.astype(np.int64)) > 0
    for j in range(hx.shape[0]):
        earlier = {int(lay[k]) for k in range(j) if share[j, k]}
        mex = 0
        while mex in earlier:
            mex += 1
        assert lay[j] == mex
    for a in range(hx.shape[0]):  # rows of one layer share no variable
        for b in range(a + 1, hx.shape[0]):
            if lay[a] == lay[b]:
                assert not share[a, b]


@pytest.mark.parametrize("fp32", [False, True])
def test_layered_single_check_equals_flooding(fp32):
    H = np.ones((1, 4), dtype=np.uint8)
    p = np.array([0.05, 0.05, 0.2, 0.05])
    code = Code(H)
    f = code.bp(np.array([1], dtype=np.uint8), p, max_iter=1, alpha=0.625, fp32=fp32, stop_on_converge=False)
    g = code.bp(np.array([1], dtype=np.uint8), p, max_iter=1, alpha=0.625, fp32=fp32, stop_on_converge=False,
                layered=True)
    assert (f["lout"] == g["lout"]).all()


def test_layered_chain_closed_form():
    # v0 - c0 - v1 - c1 - v2, s = (1, 0), alpha = 1, one iteration.  c0 is layer 0 and
    # c1 layer 1 (they share v1), so c1 already sees c0's new message through L1:
    #   c0: q = (l0, l1); r00 = -l1, r01 = -l0; L0 = l0 - l1, L1 = l1 - l0
    #   c1: q1 = L1 - 0, q2 = l2; r11 = +|l2|, r12 = sign(q1) |q1|; L1 += r11, L2 = l2 + r12
    # Under flooding c1 would see q1 = l1 instead (and L2 = l2 + l1).
    H = np.array([[1, 1, 0], [0, 1, 1]], dtype=np.uint8)
    p = np.array([0.1, 0.2, 0.1])
    code = Code(H)
    assert code.layers().tolist() == [0, 1]
    r = code.bp(np.array([1, 0], dtype=np.uint8), p, max_iter=1, alpha=1.0, fp32=False, stop_on_converge=False,
                layered=True)
    l0, l1, l2 = (float(np.log((1 - x) / x)) for x in p)
    L0 = l0 + (-(1.0 * l1))
    q1 = (l1 + (-(1.0 * l0))) - 0.0
    L1 = q1 + (1.0 * abs(l2))
    L2 = l2 + ((1.0 if q1 >= 0 else -1.0) * (1.0 * abs(q1)))
    assert r["lout"].tolist() == [L0, L1, L2]
    f = code.bp(np.array([1, 0], dtype=np.uint8), p, max_iter=1, alpha=1.0, fp32=False, stop_on_converge=False)
    assert f["lout"][2] != r["lout"][2]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("s_bit", [0, 1])
def test_single_check_closed_form(fp32, s_bit):
    # One check over four variables; one variable has the smaller prior LLR.
    # After one iteration every message is (-1)^s * alpha * (min of the others)
    # (all V2C messages are positive), so l_out is known in closed form.
    H = np.ones((1, 4), dtype=np.uint8)
    p = np.array([0.05, 0.05, 0.2, 0.05])
    alpha = 0.625
    code = Code(H)
    r = code.bp(np.array([s_bit], dtype=np.uint8), p, max_iter=1, alpha=alpha, fp32=fp32, stop_on_converge=False)
    ty = np.float32 if fp32 else np.float64
    L = ty(np.log(0.95 / 0.05))
    L2 = ty(np.log(0.8 / 0.2))
    sgn = ty(-1.0 if s_bit else 1.0)
    a = ty(alpha)
    want = np.array([L + sgn * (a * L2), L + sgn * (a * L2), L2 + sgn * (a * L), L + sgn * (a * L2)], dtype=ty)
    assert (r["lout"] == want).all()
    # Hard decision: e_i = 1 iff l_out <= 0 (with s = 1 the low-prior bit flips).
    assert (r["e"] == (want <= 0)).all()
    assert r["e"].tolist() == ([0, 0, 1, 0] if s_bit else [0, 0, 0, 0])


@pytest.mark.parametrize("fp32", [False, True])
def test_adaptive_damping_schedule_closed_form(fp32):
    # alpha = 0 selects alpha_t = 1 - 2^-t (0.5, 0.75, 0.875, ...).  One check over
    # two bits with s = 1: every iteration's V2C messages are the channel LLRs
    # (each bit has no other check), so r_t = -alpha_t * (the other bit's LLR) and
    # l_out_2(t) = L2 - alpha_t * L1.  With L2 / L1 = 0.8 the run converges at the
    # first t with alpha_t >= 0.8, i.e. t = 3; a schedule shifted by one step, or
    # 2^-t, or a fixed alpha would stop elsewhere or never.
    H = np.ones((1, 2), dtype=np.uint8)
    L1 = 4.0
    L2 = 0.8 * L1
    p = 1.0 / (1.0 + np.exp(np.array([L1, L2])))  # priors with these channel LLRs
    code = Code(H)
    r = code.bp(np.array([1], dtype=np.uint8), p, max_iter=10, alpha=0.0, fp32=fp32)
    assert r["converged"] and r["iters"] == 3
    assert r["e"].tolist() == [0, 1]
    ty = np.float32 if fp32 else np.float64
    l1, l2 = ty(np.log((1 - p[0]) / p[0])), ty(np.log((1 - p[1]) / p[1]))
    a3 = ty(1.0 - 2.0 ** -3)
    assert r["lout"][1] == l2 + (-(a3 * l1))
    assert r["lout"][0] == l1 + (-(a3 * l2))
    # Stopped one iteration early, alpha_2 = 0.75 leaves bit 2 positive.
    r2 = code.bp(np.array([1], dtype=np.uint8), p, max_iter=2, alpha=0.0, fp32=fp32)
    assert not r2["converged"] and r2["e"].tolist() == [0, 0]


def test_two_check_chain_signs():
    # v0 - c0 - v1 - c1 - v2 with s = (1, 0): the unique lowest-cost solution flips v0 or v1.
    # Min-sum with alpha = 1 on this tree equals the min-cost difference (checked above); here
    # the signs of l_out are checked directly: v2 is 0 and exactly one of v0, v1 is chosen.
    H = np.array([[1, 1, 0], [0, 1, 1]], dtype=np.uint8)
    p = np.array([0.1, 0.2, 0.1])  # v1 is the cheaper bit, but flipping it breaks c1
    code = Code(H)
    r = code.bp(np.array([1, 0], dtype=np.uint8), p, max_iter=5, alpha=1.0, fp32=False, stop_on_converge=False)
    assert r["e"].tolist() == [1, 0, 0]
    assert r["converged"]


def _clamp_toy_reduced(T, p, clamp=2.0 ** 100):
    """Posterior after T iterations on H = [[1,1],[1,1],[1,1]], s = (1,0,0),
    alpha_t = 1 - 2^-t, reduced by symmetry to two numbers: both variables
    carry the same V2C message a to check 0 and b to checks 1 and 2 (which
    stay equal), a check of degree two passes the other variable's message
    scaled and signed, so a' = l + 2 r_b, b' = l + r_a + r_b with
    r_a = -sign(a) min(alpha |a|, clamp), r_b = sign(b) min(alpha |b|, clamp)."""
    l = math.log((1 - p) / p)
    a = b = l
    lout = l
    for t in range(1, T + 1):
        al = 1.0 - math.ldexp(1.0, -t)
        ra = min(al * abs(a), clamp) if a < 0 else -min(al * abs(a), clamp)
        rb = -min(al * abs(b), clamp) if b < 0 else min(al * abs(b), clamp)
        lout = ((l + ra) + rb) + rb
        a, b = (l + rb) + rb, (l + ra) + rb
    return lout


def test_c2v_clamp_where_it_fires():
    """Messages that grow without bound, and the 2^100 clamp that keeps them finite.

    On H = [[1,1],[1,1],[1,1]] with s = (1,0,0) no e satisfies the syndrome
    (every check sees the same parity), so BP never stops.  With alpha_t -> 1
    the reduced map (a, b) -> (2b, b - a) has eigenvalues (1 +- i sqrt 7) / 2 of
    modulus sqrt 2: magnitudes grow by half a bit per iteration until the
    clamp at 2^100 holds them, after which every posterior is a small multiple
    of 2^100 (the channel LLR is far below its last place)."""
    H = np.array([[1, 1], [1, 1], [1, 1]], dtype=np.uint8)
    code = Code(H)
    s = np.array([1, 0, 0], dtype=np.uint8)
    p = 0.1
    growth = []
    for T in (20, 60, 100, 140, 180, 220, 260, 300, 333, 400, 401, 402):
        r64 = code.bp(s, p, T, 0.0, fp32=False)
        r32 = code.bp(s, p, T, 0.0, fp32=True)
        assert not r64["converged"] and r64["iters"] == T and r32["iters"] == T
        assert r64["lout"][0] == r64["lout"][1] and np.isfinite(r32["lout"]).all()
        # FP64 equals the hand-reduced two-number recursion at every length.
        assert r64["lout"][0] == _clamp_toy_reduced(T, p)
        growth.append((T, math.log2(abs(r64["lout"][0]))))
        if T >= 260:
            # Saturated: |r| = 2^100 on every edge, posteriors are +-2^100 or 2^101.
            for v in (r64["lout"][0], float(r32["lout"][0])):
                assert abs(v) in (2.0 ** 100, 2.0 ** 101)
            assert float(r32["lout"][0]) == r64["lout"][0]
    # Before the clamp: half a bit per iteration (|lambda| = sqrt 2).
    slope = (growth[4][1] - growth[1][1]) / (growth[4][0] - growth[1][0])
    assert abs(slope - 0.5) < 0.03
    # Without the clamp the same recursion leaves FP32's range long before 400.
    assert abs(_clamp_toy_reduced(400, p, clamp=float("inf"))) > 2.0 ** 128


def test_batch_syndrome_equals_the_matvec_and_the_columns():
    for H in (oracle.named_code("bb144")[0], oracle.phenom_code(oracle.named_code("bb72")[0], 3)):
        code = Code(H)
        rng = np.random.default_rng(5)
        e = (rng.random((40, code.N)) < 0.1).astype(np.uint8)
        assert (code.syndrome(e) == code.syndrome_matvec(e)).all()
        # Unit errors give the columns of H.
        eye = np.eye(code.N, dtype=np.uint8)[:50]
        assert (code.syndrome(eye) == H[:, :50].T).all()


def test_zero_syndrome_is_trivial():
    hx, _ = oracle.named_code("bb72")
    code = Code(hx)
    for fp32 in (False, True):
        out = code.bpsf(np.zeros(36, dtype=np.uint8), 0.05, Params(max_iter=50, w=4, short_iter=10), fp32=fp32)
        assert out["converged"] and out["iters"] == 1 and out["stage"] == 0
        assert not out["e"].any()


# --------------------------------------------------------------------------
# Algorithm 1 pieces on the [[72,12,6]] workload
# --------------------------------------------------------------------------

def _bb72_shots(n, p, seed=1001):
    hx, hz = oracle.named_code("bb72")
    e = synth.bernoulli_bits(seed, 0, 0, n, 72, p)
    code = Code(hx)
    return code, hx, hz, e, code.syndrome(e)


def test_oscillation_counter_invariants():
    code, hx, hz, e, s = _bb72_shots(300, 0.1)
    for k in range(300):
        r = code.bp(s[k], 0.1, max_iter=50, alpha=0.625, fp32=True, track=True)
        f = r["flips"].astype(np.int64)
        assert (f <= r["iters"]).all()
        # e_prev starts at 0, so the parity of the flip count is the final bit.
        assert ((f % 2) == r["e"]).all()


def test_top_matches_full_sort():
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = int(rng.integers(5, 300))
        f = rng.integers(0, 6, size=n).astype(np.uint16)  # many ties
        w = int(rng.integers(1, min(n, 16) + 1))
        want = sorted(range(n), key=lambda i: (-int(f[i]), i))[:w]
        assert oracle.top(f, w).tolist() == want


def test_trials_and_winner_by_brute_force():
    code, hx, hz, e, s = _bb72_shots(600, 0.1)
    P = Params(max_iter=50, alpha=0.625, w=4, short_iter=10)
    failed = 0
    for k in range(600):
        out = code.bpsf(s[k], 0.1, P, fp32=True)
        if out["stage"] == 0:
            continue
        failed += 1
        phi = out["phi"]
        synd, conv, iters, es = code.trials(s[k], 0.1, phi, P, fp32=True)
        assert len(synd) == 2 ** P.w - 1
        masks = [m for m in range(1, 2 ** P.w)]
        best = None
        for idx, m in enumerate(masks):
            t = np.zeros(72, dtype=np.uint8)
            for j in range(P.w):
                if (m >> j) & 1:
                    t[phi[j]] = 1
            # s' = s xor t H^T by dense GF(2) arithmetic.
            want = (s[k].astype(np.int64) + hx.astype(np.int64) @ t) % 2
            assert (synd[idx] == want).all()
            if conv[idx]:
                # H (e' xor t) = s for every converged trial.
                assert (((hx.astype(np.int64) @ es[idx]) % 2) == s[k]).all()
                wt = int(es[idx].sum())
                if best is None or wt < best[0]:
                    best = (wt, idx)
        if best is None:
            assert out["stage"] == 2 and not out["converged"] and out["iters"] == 50
            init = code.bp(s[k], 0.1, max_iter=50, alpha=0.625, fp32=True)
            assert (out["e"] == init["e"]).all()
        else:
            assert out["stage"] == 1 and out["converged"]
            assert (out["e"] == es[best[1]]).all() and out["iters"] == iters[best[1]]
        # The empty trial vector is BP(s) truncated, so it always fails.
        assert not code.bp(s[k], 0.1, max_iter=10, alpha=0.625, fp32=True)["converged"]
    assert failed > 10


@pytest.mark.parametrize("select", [0, 1])
def test_explicit_trial_list_by_brute_force(select):
    # The sampled variant (Section V): an explicit list of trial masks over a
    # larger Phi, decoded and selected in list order.
    code, hx, hz, e, s = _bb72_shots(400, 0.1)
    masks = synth.sample_trial_masks(11, 10, 3, 4)[::-1].copy()  # reversed: list order != mask order
    P = Params(max_iter=50, alpha=0.625, w=10, w_max=3, short_iter=10, select=select, trials=tuple(int(m) for m in masks))
    failed = 0
    for k in range(400):
        out = code.bpsf(s[k], 0.1, P, fp32=True)
        if out["stage"] == 0:
            continue
        failed += 1
        phi = out["phi"]
        assert len(phi) == 10 and len(set(phi.tolist())) == 10
        synd, conv, iters, es = code.trials(s[k], 0.1, phi, P, fp32=True)
        assert len(synd) == len(masks)
        best = None
        for idx, m in enumerate(masks):
            t = np.zeros(72, dtype=np.uint8)
            for j in range(10):
                if (int(m) >> j) & 1:
                    t[phi[j]] = 1
            assert (synd[idx] == (s[k].astype(np.int64) + hx.astype(np.int64) @ t) % 2).all()
            if conv[idx]:
                assert (((hx.astype(np.int64) @ es[idx]) % 2) == s[k]).all()
                key = (int(es[idx].sum()), idx) if select == 0 else (0, idx)
                if best is None or key < best:
                    best = key
        if best is None:
            assert out["stage"] == 2
        else:
            assert out["stage"] == 1 and (out["e"] == es[best[1]]).all() and out["iters"] == iters[best[1]]
    assert failed > 10


def test_sampled_trial_masks():
    m = synth.sample_trial_masks(5, 50, 6, 5)
    assert m.dtype == np.uint64 and len(m) == 30
    wts = [bin(int(x)).count("1") for x in m]
    assert wts == [k for k in range(1, 7) for _ in range(5)]  # n_s per weight, weight by weight
    assert len(set(int(x) for x in m)) == 30 and int(m.max()) < (1 << 50)
    assert (synth.sample_trial_masks(5, 50, 6, 5) == m).all()  # counter-based: reproducible
    assert not (synth.sample_trial_masks(6, 50, 6, 5) == m).all()
    # A weight with at most n_s subsets contributes all of them.
    assert synth.sample_trial_masks(1, 4, 2, 10).tolist() == [1, 2, 4, 8, 3, 5, 6, 9, 10, 12]
    # Exactly n_s subsets of a weight: all of them.
    big = synth.sample_trial_masks(9, 8, 1, 8)
    assert sorted(int(x) for x in big) == [1 << b for b in range(8)]


def test_select_first_and_w_max():
    code, hx, hz, e, s = _bb72_shots(400, 0.1)
    P1 = Params(max_iter=50, alpha=0.625, w=4, short_iter=10, select=1)
    P2 = Params(max_iter=50, alpha=0.625, w=4, w_max=1, short_iter=10)
    for k in range(400):
        o1 = code.bpsf(s[k], 0.1, P1)
        if o1["stage"] == 0:
            continue
        synd, conv, iters, es = code.trials(s[k], 0.1, o1["phi"], P1)
        idx = np.nonzero(conv)[0]
        if idx.size:
            assert (o1["e"] == es[idx[0]]).all()
        o2 = code.bpsf(s[k], 0.1, P2)
        synd2, conv2, _, es2 = code.trials(s[k], 0.1, o2["phi"], P2)
        assert len(synd2) == 4  # weight-1 trials only
        if conv2.any():
            wts = [int(es2[i].sum()) if conv2[i] else 10 ** 9 for i in range(4)]
            assert (o2["e"] == es2[int(np.argmin(wts))]).all()


@pytest.mark.parametrize("fp32", [False, True])
def test_converged_corrections_satisfy_the_syndrome(fp32):
    code, hx, hz, e, s = _bb72_shots(2000, 0.05)
    eh, conv, iters, stage = code.bpsf_batch(s, 0.05, Params(max_iter=50, w=4, short_iter=10), fp32=fp32, threads=4)
    synd = (eh.astype(np.int64) @ hx.T.astype(np.int64)) % 2
    assert (synd[conv] == s[conv]).all()
    assert ((stage == 0) | (stage == 1) | (stage == 2)).all()
    assert (conv == (stage < 2)).all()


def test_bpsf_never_worse_than_bp_shot_by_shot():
    code, hx, hz, e, s = _bb72_shots(2000, 0.06)
    lx = oracle.logicals(hx, hz)
    e_bp, c_bp, _, _ = code.bpsf_batch(s, 0.06, Params(max_iter=50, w=0), threads=4)
    e_sf, c_sf, _, st = code.bpsf_batch(s, 0.06, Params(max_iter=50, w=4, short_iter=10), threads=4)
    f_bp = oracle.logical_failures(hx, lx, e, e_bp, c_bp)
    f_sf = oracle.logical_failures(hx, lx, e, e_sf, c_sf)
    assert not (f_sf & ~f_bp).any()
    assert (e_sf[st == 0] == e_bp[st == 0]).all()
    assert f_sf.sum() < f_bp.sum()


def test_fp32_and_fp64_modes_agree():
    code, hx, hz, e, s = _bb72_shots(2000, 0.05)
    P = Params(max_iter=50, w=4, short_iter=10)
    e32, c32, i32, _ = code.bpsf_batch(s, 0.05, P, fp32=True, threads=4)
    e64, c64, i64, _ = code.bpsf_batch(s, 0.05, P, fp32=False, threads=4)
    same = (e32 == e64).all(axis=1)
    assert same.mean() >= 0.995


def test_exhaustive_min_weight_on_a_small_cyclic_code():
    # [[18, ...]] member of the BB family (l = m = 3); every syndrome in the image of H.
    hx, _ = oracle.bb_code(3, 3, [(1, 0), (0, 1), (0, 2)], [(0, 1), (1, 0), (2, 0)])
    M, N = hx.shape
    E = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)
    S = (E.astype(np.int64) @ hx.T.astype(np.int64)) % 2
    key = S @ (1 << np.arange(M))
    wt = E.sum(axis=1)
    minw = {}
    for kk, ww in zip(key.tolist(), wt.tolist()):
        if kk not in minw or ww < minw[kk]:
            minw[kk] = ww
    code = Code(hx)
    P = Params(max_iter=20, w=3, short_iter=10)
    equal = total = 0
    for kk, ww in minw.items():
        s = ((kk >> np.arange(M)) & 1).astype(np.uint8)
        out = code.bpsf(s, 0.1, P)
        if out["converged"]:
            assert (((hx.astype(np.int64) @ out["e"]) % 2) == s).all()
            assert int(out["e"].sum()) >= ww
            total += 1
            equal += int(out["e"].sum()) == ww
    assert total > 0 and equal / total > 0.5


def test_min_sum_finds_the_unique_min_weight_error_on_trees():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(10):
        H = random_tree_H(rng, 10, 4)
        M, N = H.shape
        E = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)
        S = (E.astype(np.int64) @ H.T.astype(np.int64)) % 2
        code = Code(H)
        for sbits in itertools.product([0, 1], repeat=M):
            s = np.array(sbits, dtype=np.uint8)
            sel = (S == s).all(axis=1)
            if not sel.any():
                continue
            wts = E[sel].sum(axis=1)
            if (wts == wts.min()).sum() != 1:
                continue
            out = code.bp(s, 0.1, max_iter=20, alpha=1.0, fp32=False, stop_on_converge=False)
            assert out["converged"]
            assert (out["e"] == E[sel][np.argmin(wts)]).all()
            checked += 1
    assert checked > 20
