"""Split-precision (Ozaki, BF16 slices on tcgen05) Gram product vs exact references.

* Bit-exactness: when every column of J has entries that are integers of at
  most 8 significant bits (|J_ij| <= 200 here), one slice represents J exactly
  and every partial sum is an integer below 2^24, so G_split must equal the
  exact Gram matrix (computed in FP64, exact for these integers) bit for bit.
  This pins the whole path: TMA tiles and swizzle, instruction and shared
  memory descriptors, the tensor-memory accumulators and the epilogue.
* Accuracy: for a real Jacobian the error of each entry obeys the bound of
  the split (scaled columns x = J 2^{-e}, |x| < 1, K rows, S slices):
      |dG_ij| 2^{-(e_i+e_j)} <= 2^{-8S-1} (|x_:i|_1 + |x_:j|_1)        (digits)
                               + K 2^{-16S-2} + K S(S-1)/2 2^{-8S-2}  (dropped pairs)
                               + [S >= 4] (K_pad/16) 2^{-48} K S      (FP32 tail)
  checked against the oracle's Jacobian and an FP64 product on the CPU.
"""
import numpy as np
import pytest
import torch

from tests.gpu_cases import dev, gpu_problem, host, oracle_problem, small
from oracle import gn as ogn

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

SPLIT = 1


def split_bound(J, S):
    """Entrywise bound of the split Gram error (see the module docstring)."""
    K = J.shape[0]
    M = np.max(np.abs(J), axis=0)
    e = np.where(M > 0, np.frexp(M)[1], 0).astype(np.float64)
    X = J * 2.0 ** (-e)
    n1 = np.sum(np.abs(X), axis=0)
    per = 2.0 ** (-8 * S - 1) * (n1[:, None] + n1[None, :]) + K * 2.0 ** (-16 * S - 2) \
        + K * S * (S - 1) / 2 * 2.0 ** (-8 * S - 2)
    if S >= 4:
        kpad = -(-K // 128) * 128
        per = per + (kpad / 16) * 2.0 ** -48 * K * S
    return per * 2.0 ** (e[:, None] + e[None, :])


def _split_gram(prob, J, slices, accumulate=False, G=None):
    Pp = prob.P + 1
    prob.gn_set_precision(SPLIT, slices)
    if G is None:
        G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    prob.gn_gram(J, J.shape[0], None, G, None, precision=SPLIT, accumulate=accumulate)
    torch.cuda.synchronize()
    return G


@pytest.mark.parametrize("nrows", [128, 300])
def test_split_gram_bit_exact_on_8bit_integers(nrows):
    w = small("ccf")                     # P' = 1762: 14 column tiles, ragged last tile
    prob = gpu_problem(w)
    Pp = prob.P + 1
    rng = np.random.default_rng(7)
    Jh = rng.integers(-200, 201, size=(nrows, Pp)).astype(np.float64)
    Jh[:, 5] = 0.0                       # an all-zero column
    Jh[:, 7] *= 2.0 ** -20               # a column at a different power-of-two scale
    G = host(_split_gram(prob, dev(Jh), 1))
    Gx = Jh.T @ Jh                       # exact: integers below 2^53
    assert np.array_equal(np.tril(G), np.tril(Gx))


def test_split_gram_one_slice_rounds_ties_to_even():
    """The digits are round(x 2^(8S - e)) to the nearest integer with ties to even, formed from
    the double's bits.  With one slice and every entry an odd multiple of 1/2 below 200 (each
    column's largest entry in [128, 256), so x 2^(8S - e) = x), every entry is a tie: the split
    Gram must equal A^T A bit for bit with A = J rounded half to even (numpy's rule), not
    half away from zero.  Columns rescaled by powers of two, negative ties and a zero column
    take the same path."""
    w = small("ccf")
    prob = gpu_problem(w)
    Pp = prob.P + 1
    rng = np.random.default_rng(23)
    nrows = 700
    Jh = rng.integers(-200, 200, size=(nrows, Pp)).astype(np.float64) + 0.5
    Jh[0, :] = 199.5                     # each column's maximum in [128, 256): exponent 8
    Jh[:, 3] = 0.0
    scale = np.ones(Pp)
    scale[9::97] = 2.0 ** -30
    scale[10::97] = 2.0 ** 12
    A = np.round(Jh)                     # half to even
    assert np.any(A != np.trunc(Jh + np.copysign(0.5, Jh)))   # the ties are really ties
    G = host(_split_gram(prob, dev(Jh * scale), 1))
    Gx = (A * scale).T @ (A * scale)     # exact: integers times powers of two, below 2^53
    assert np.array_equal(np.tril(G), np.tril(Gx))


@pytest.mark.parametrize("slices", [1, 2, 3, 4, 5, 6])
def test_split_gram_error_bound(slices):
    w = small("ccf")
    p = oracle_problem(w)
    J = ogn.jacobian(p, w.theta, w.lam)
    prob = gpu_problem(w)
    G = np.tril(host(_split_gram(prob, dev(J), slices)))
    Gx = np.tril(J.T @ J)
    bound = np.tril(split_bound(J, slices))
    err = np.abs(G - Gx)
    assert np.all(err <= 2.0 * bound + 1e-300), float(np.max(err / (bound + 1e-300)))


def test_split_gram_accumulate_two_row_blocks():
    w = small("boussinesq")
    p = oracle_problem(w)
    J = ogn.jacobian(p, w.theta, w.lam)
    prob = gpu_problem(w)
    h = J.shape[0] // 2
    G = _split_gram(prob, dev(J[:h]), 4)
    G = _split_gram(prob, dev(J[h:]), 4, accumulate=True, G=G)
    Gx = J.T @ J
    bound = split_bound(J[:h], 4) + split_bound(J[h:], 4)
    assert np.all(np.tril(np.abs(host(G) - Gx)) <= 2.0 * np.tril(bound) + 1e-300)


SPLIT_ALL = 2


def test_split_all_jacobian_hilbert_contraction():
    """CCF Jacobian with the Hilbert contraction J_U = K J_g on the tensor cores (S = 6)."""
    from tests.gpu_cases import TOL, rel
    w = small("ccf")
    p = oracle_problem(w)
    J_o = ogn.jacobian(p, w.theta, w.lam)
    prob = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    J = host(prob.jacobian(dev(w.theta), w.lam))
    assert rel(J, J_o) <= TOL


def test_split_all_damped_solve():
    """Blocked Cholesky with split trailing updates: backward error and agreement with the oracle."""
    w = small("ccf")
    p = oracle_problem(w)
    J_o = ogn.jacobian(p, w.theta, w.lam)
    r_o = p.rows(w.theta, w.lam)
    Go, go = J_o.T @ J_o, J_o.T @ r_o
    prob = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    delta = prob.new_vec(prob.P + 1)
    rc, gam, retries = prob.gn_damped_solve(dev(Go), dev(go), 1e-6, delta)
    assert rc == 0 and retries == 0
    A = Go + 1e-6 * np.eye(len(go))
    d = host(delta)
    assert np.max(np.abs(A @ d - go)) / (np.max(np.abs(A)) * np.max(np.abs(d))) <= 1e-12
    d_o, _, _, _ = ogn.damped_solve(Go, go, 1e-6)
    # trailing updates accumulate in double-FP32 (~2^-48 per panel): the factor's
    # backward error is ~1e-13 |A|, so the forward error scales with cond(A)
    assert np.max(np.abs(d - d_o)) / np.max(np.abs(d_o)) <= max(1e-12, 5e-13 * np.linalg.cond(A))


def test_split_all_gn_step_ill_conditioned_is_valid():
    """IPM's first step has G + gamma I close to singular in floating point: the split
    factorisation may need a damping escalation the FP64 oracle does not.  The outcome
    must still be a valid damped GN step: accepted with a decrease, or rejected cleanly."""
    w = small("ipm")
    p = oracle_problem(w)
    prob = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc in (0, 1)
    assert gam >= w.gamma * (2.0 / 3.0) * 10.0 ** info["chol_retries"] - 1e-300
    if rc == 0:
        assert info["loss_after"] < info["loss_before"]
        assert abs(p.loss(host(theta), lam) - info["loss_after"]) <= 1e-12 * info["loss_before"]
    else:
        assert np.array_equal(host(theta), w.theta) and lam == w.lam


@pytest.mark.parametrize("name", ["ccf"])
def test_split_all_gn_step_matches_oracle(name):
    w = small(name)
    p = oracle_problem(w)
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, w.gamma)
    prob = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc == info_o["status"] and info["alpha"] == info_o["alpha"]
    assert gam == pytest.approx(gam_o, rel=1e-15)
    if rc != 0:     # both rejected the step: theta and lambda are unchanged
        assert np.array_equal(host(theta), w.theta) and lam == w.lam
        return
    cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(p.P + 1))
    d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
    d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
    # G, J_U and the factorisation each carry ~1e-13 relative error at S = 6
    # (FP32 tail accumulator); the step amplifies it by cond(G + gamma I)
    assert np.max(np.abs(d_gpu - d_o)) / np.max(np.abs(d_o)) <= max(1e-12, 2e-13 * cond)


# --- split-K (the contraction over rows cut into parts summed by a second launch) ---------

@pytest.mark.parametrize("ksplit", [2, 3, 5, 8])
def test_split_gram_splitk_bit_exact_on_8bit_integers(ksplit):
    """Integer J (8-bit entries): every partial tile is an exact integer sum and the final
    FP64 sum of the parts is exact too, so any split must give the exact Gram bit for bit
    (this pins the partial-tile layout, the chunk ranges of each part and the reduction)."""
    w = small("ccf")
    prob = gpu_problem(w)
    Pp = prob.P + 1
    rng = np.random.default_rng(11)
    Jh = rng.integers(-200, 201, size=(2000, Pp)).astype(np.float64)
    Jh[:, 3] = 0.0
    Jh[:, 9] *= 2.0 ** -30
    prob.gn_set_gram_split(ksplit)
    G = host(_split_gram(prob, dev(Jh), 1))
    assert np.array_equal(np.tril(G), np.tril(Jh.T @ Jh))


@pytest.mark.parametrize("ksplit", [1, 2, 4, 7])
def test_split_gram_splitk_error_bound(ksplit):
    w = small("ccf")
    p = oracle_problem(w)
    J1 = ogn.jacobian(p, w.theta, w.lam)
    J = np.concatenate([J1] * 7)          # 2114 rows: 17 flush chunks, ragged
    prob = gpu_problem(w)
    prob.gn_set_gram_split(ksplit)
    G = np.tril(host(_split_gram(prob, dev(J), 6)))
    Gx = np.tril(J.T @ J)
    bound = np.tril(split_bound(J, 6))
    err = np.abs(G - Gx)
    assert np.all(err <= 2.0 * bound + 1e-300), float(np.max(err / (bound + 1e-300)))
    # accumulate (mode 1) through the split path as well
    G2 = _split_gram(prob, dev(J), 6)
    G2 = host(_split_gram(prob, dev(J), 6, accumulate=True, G=G2))
    assert np.all(np.tril(np.abs(G2 - 2 * (J.T @ J))) <= 4.0 * bound + 1e-300)


def test_gram_autotuner_records_a_choice_per_shape():
    """The first split Gram of a shape times the candidates and records the fastest; a second
    handle of the same shape reuses it; forcing a factor overrides the table."""
    w = small("ccf")
    prob = gpu_problem(w)
    Pp = prob.P + 1
    rng = np.random.default_rng(3)
    J = dev(rng.standard_normal((4000, Pp)))
    _split_gram(prob, J, 6)
    k = prob.gn_gram_split_choice(4000)
    assert 1 <= k <= 8
    prob2 = gpu_problem(w)
    prob2.gn_set_precision(SPLIT, 6)          # the table is keyed by the slice count too
    assert prob2.gn_gram_split_choice(4000) == k
    prob2.gn_set_gram_split(3)
    assert prob2.gn_gram_split_choice(4000) == 3
    with pytest.raises(Exception):
        prob2.gn_set_gram_split(9)


# --- 128 x 64 output tiles (the autotuner's second tile shape) ----------------------------

@pytest.mark.parametrize("ksplit", [1, 3])
def test_split_gram_half_tiles_bit_exact_on_8bit_integers(ksplit):
    """128 x 64 tiles: the lower part of G is covered by 2 ti + 2 column tiles per row tile
    (the last one ragged here, P' = 1762), B tiles of 64 rows, 256 tensor-memory columns and a
    32-column epilogue per thread; on 8-bit integer J the Gram is exact bit for bit, with or
    without split-K."""
    w = small("ccf")
    prob = gpu_problem(w)
    Pp = prob.P + 1
    rng = np.random.default_rng(17)
    Jh = rng.integers(-200, 201, size=(1500, Pp)).astype(np.float64)
    Jh[:, 4] = 0.0
    Jh[:, 11] *= 2.0 ** -25
    prob.gn_set_gram_tile(64)
    prob.gn_set_gram_split(ksplit)
    assert prob.gn_gram_tile_choice(1500) == 64
    G = host(_split_gram(prob, dev(Jh), 1))
    assert np.array_equal(np.tril(G), np.tril(Jh.T @ Jh))


@pytest.mark.parametrize("slices", [2, 6])
def test_split_gram_half_tiles_equal_square_tiles(slices):
    """The tile shape changes which CTA computes an entry, not its arithmetic: a real Jacobian's
    Gram on 128 x 64 tiles equals the one on 128 x 128 tiles bit for bit (and both obey the
    bound), in overwrite and accumulate modes."""
    w = small("ccf")
    p = oracle_problem(w)
    J = ogn.jacobian(p, w.theta, w.lam)
    prob = gpu_problem(w)
    prob.gn_set_gram_split(1)
    prob.gn_set_gram_tile(128)
    G128 = host(_split_gram(prob, dev(J), slices))
    prob.gn_set_gram_tile(64)
    G64 = host(_split_gram(prob, dev(J), slices))
    np.testing.assert_array_equal(np.tril(G64), np.tril(G128))
    bound = np.tril(split_bound(J, slices))
    assert np.all(np.abs(np.tril(G64) - np.tril(J.T @ J)) <= 2.0 * bound + 1e-300)
    G2 = _split_gram(prob, dev(J), slices)
    G2 = host(_split_gram(prob, dev(J), slices, accumulate=True, G=G2))
    assert np.all(np.tril(np.abs(G2 - 2 * (J.T @ J))) <= 4.0 * bound + 1e-300)


def test_gram_autotuner_chooses_a_tile_shape():
    """The autotuner times both tile widths (with their split-K candidates) and records one; a
    second handle of the shape reuses it; forcing a width overrides the table; bad widths are
    refused."""
    w = small("burgers")                       # P' = 674: 6 row tiles, 21 or 42 tiles
    prob = gpu_problem(w)
    Pp = prob.P + 1
    rng = np.random.default_rng(5)
    J = dev(rng.standard_normal((3000, Pp)))
    assert prob.gn_gram_tile_choice(3000) == 0          # not tuned yet
    _split_gram(prob, J, 5)
    t = prob.gn_gram_tile_choice(3000)
    assert t in (64, 128)
    prob2 = gpu_problem(w)
    prob2.gn_set_precision(SPLIT, 5)
    assert prob2.gn_gram_tile_choice(3000) == t
    prob2.gn_set_gram_tile(64)
    assert prob2.gn_gram_tile_choice(3000) == 64
    with pytest.raises(Exception):
        prob2.gn_set_gram_tile(96)
