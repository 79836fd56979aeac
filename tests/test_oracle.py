"""Pins for the CPU oracle: closed forms, brute force, identities (no GPU).

Each test ties an oracle function to something other than itself: a value
worked by hand, a textbook routine on a special case (np.convolve, a recursion,
an explicit DFT sum), the dense matrix, or an identity the mathematics fixes.
"""
import numpy as np
import pytest

import oracle
import synth
from golden_io import hand_examples

RNG = np.random.default_rng(1234)


def rand_case(Nt, Nd, Nm, K=None, seed=0):
    Fcol = synth.block_column(Nt, Nd, Nm, seed=seed)
    k = 1 if K is None else K
    m = synth.vectors(synth.TAG_M, Nt, Nm, k=k, seed=seed)
    d = synth.vectors(synth.TAG_D, Nt, Nd, k=k, seed=seed)
    if K is None:
        m, d = m[0], d[0]
    return Fcol, m, d


ALL_MATVECS = [
    ("direct", oracle.matvec_direct, oracle.rmatvec_direct),
    ("fft", oracle.matvec_fft, oracle.rmatvec_fft),
    ("mixed_d", lambda F, m: oracle.matvec_mixed(oracle.spectrum(F), m, F.shape[0], "ddddd"),
     lambda F, d: oracle.rmatvec_mixed(oracle.spectrum(F), d, F.shape[0], "ddddd")),
]


# --- hand-worked values (tests/golden) ---------------------------------------

@pytest.mark.parametrize("name,mv,rmv", ALL_MATVECS)
def test_hand_examples(name, mv, rmv):
    for ex in hand_examples():
        d = mv(ex["Fcol"], ex["m"])
        ms = rmv(ex["Fcol"], ex["d_in"])
        tol = 0 if name == "direct" else 1e-13
        np.testing.assert_allclose(d, ex["d"], rtol=0, atol=tol * 20)
        np.testing.assert_allclose(ms, ex["mstar"], rtol=0, atol=tol * 20)


def test_hand_examples_entries():
    for ex in hand_examples():
        Nt, Nd, Nm = ex["Nt"], ex["Nd"], ex["Nm"]
        idx = [(i, r) for i in range(Nt) for r in range(Nd)]
        np.testing.assert_array_equal(oracle.matvec_entries(ex["Fcol"], ex["m"], idx), ex["d"].ravel())
        idx = [(j, n) for j in range(Nt) for n in range(Nm)]
        np.testing.assert_array_equal(oracle.rmatvec_entries(ex["Fcol"], ex["d_in"], idx), ex["mstar"].ravel())


# --- P1: brute force dense matrix -------------------------------------------

@pytest.mark.parametrize("Nt,Nd,Nm", [(1, 1, 1), (2, 3, 2), (3, 2, 5), (5, 3, 4), (8, 2, 3), (7, 4, 1)])
def test_brute_force_dense(Nt, Nd, Nm):
    Fcol, m, d = rand_case(Nt, Nd, Nm, seed=Nt * 100 + Nd * 10 + Nm)
    A = oracle.dense_matrix(Fcol)
    d_ref = (A @ m.ravel()).reshape(Nt, Nd)
    ms_ref = (A.T @ d.ravel()).reshape(Nt, Nm)
    for name, mv, rmv in ALL_MATVECS:
        assert oracle.rel_l2(mv(Fcol, m), d_ref) <= 1e-13, name
        assert oracle.rel_l2(rmv(Fcol, d), ms_ref) <= 1e-13, name


def test_direct_fft_agree_c1_size():
    # Nt=64, Nd=8, Nm=32, seed 0: the plain FP64 workload
    Fcol, m, d = rand_case(64, 8, 32, seed=0)
    assert oracle.rel_l2(oracle.matvec_fft(Fcol, m), oracle.matvec_direct(Fcol, m)) <= 1e-13
    assert oracle.rel_l2(oracle.rmatvec_fft(Fcol, d), oracle.rmatvec_direct(Fcol, d)) <= 1e-13


def test_multi_rhs_is_columnwise():
    Fcol, m, d = rand_case(6, 3, 4, K=3, seed=5)
    for name, mv, rmv in ALL_MATVECS:
        D = mv(Fcol, m)
        MS = rmv(Fcol, d)
        for b in range(3):
            np.testing.assert_allclose(D[b], oracle.matvec_direct(Fcol, m[b]), rtol=0, atol=1e-12)
            np.testing.assert_allclose(MS[b], oracle.rmatvec_direct(Fcol, d[b]), rtol=0, atol=1e-12)


# --- P2: closed forms --------------------------------------------------------

def test_identity_operator():
    Nt, N = 9, 4
    Fcol = np.zeros((Nt, N, N))
    Fcol[0] = np.eye(N)
    m = RNG.standard_normal((Nt, N))
    for name, mv, rmv in ALL_MATVECS:
        tol = 0 if name == "direct" else 1e-14
        np.testing.assert_allclose(mv(Fcol, m), m, rtol=0, atol=tol * 10)
        np.testing.assert_allclose(rmv(Fcol, m), m, rtol=0, atol=tol * 10)


@pytest.mark.parametrize("s", [0, 1, 3, 6])
def test_time_shift(s):
    Nt, N = 7, 3
    Fcol = np.zeros((Nt, N, N))
    Fcol[s] = np.eye(N)
    m = RNG.standard_normal((Nt, N))
    want = np.zeros_like(m)
    want[s:] = m[: Nt - s]            # F shifts forward in time
    want_adj = np.zeros_like(m)
    want_adj[: Nt - s] = m[s:]        # F* shifts backward
    for name, mv, rmv in ALL_MATVECS:
        tol = 0 if name == "direct" else 1e-14
        np.testing.assert_allclose(mv(Fcol, m), want, rtol=0, atol=tol * 10)
        np.testing.assert_allclose(rmv(Fcol, m), want_adj, rtol=0, atol=tol * 10)


@pytest.mark.parametrize("s", [0, 2, 4])
def test_single_nonzero_block(s):
    Nt, Nd, Nm = 5, 2, 3
    A = np.array([[1.0, -2.0, 0.5], [3.0, 0.0, -1.0]])   # not symmetric, not square
    Fcol = np.zeros((Nt, Nd, Nm))
    Fcol[s] = A
    m = RNG.standard_normal((Nt, Nm))
    d = RNG.standard_normal((Nt, Nd))
    want = np.zeros((Nt, Nd))
    want_adj = np.zeros((Nt, Nm))
    for t in range(s, Nt):
        want[t] = A @ m[t - s]
        want_adj[t - s] = A.T @ d[t]
    for name, mv, rmv in ALL_MATVECS:
        np.testing.assert_allclose(mv(Fcol, m), want, rtol=0, atol=1e-13)
        np.testing.assert_allclose(rmv(Fcol, d), want_adj, rtol=0, atol=1e-13)


def test_constant_blocks_prefix_sum():
    Nt, Nd, Nm = 10, 3, 4
    A = RNG.standard_normal((Nd, Nm))
    Fcol = np.broadcast_to(A, (Nt, Nd, Nm)).copy()
    m = RNG.standard_normal((Nt, Nm))
    want = np.cumsum(m, axis=0) @ A.T
    for name, mv, rmv in ALL_MATVECS:
        assert oracle.rel_l2(mv(Fcol, m), want) <= 1e-13, name


def test_geometric_blocks_recursion():
    # F_k = a^k A, the impulse response of the LTI recursion d_t = a d_{t-1} + A m_t
    Nt, Nd, Nm, a = 12, 2, 3, -0.7
    A = RNG.standard_normal((Nd, Nm))
    Fcol = np.stack([a ** k * A for k in range(Nt)])
    m = RNG.standard_normal((Nt, Nm))
    want = np.zeros((Nt, Nd))
    prev = np.zeros(Nd)
    for t in range(Nt):
        prev = a * prev + A @ m[t]
        want[t] = prev
    for name, mv, rmv in ALL_MATVECS:
        assert oracle.rel_l2(mv(Fcol, m), want) <= 1e-13, name


@pytest.mark.parametrize("Nt", [1, 2, 5, 16, 33])
def test_scalar_blocks_are_polynomial_product(Nt):
    f = RNG.standard_normal(Nt)
    mv_ = RNG.standard_normal(Nt)
    Fcol = f.reshape(Nt, 1, 1)
    want = np.convolve(f, mv_)[:Nt]
    want_adj = np.correlate(mv_, f, mode="full")[Nt - 1:]    # sum_i f_{i-j} x_i
    for name, mv, rmv in ALL_MATVECS:
        assert oracle.rel_l2(mv(Fcol, mv_.reshape(Nt, 1)).ravel(), want) <= 1e-13, name
        assert oracle.rel_l2(rmv(Fcol, mv_.reshape(Nt, 1)).ravel(), want_adj) <= 1e-13, name


# --- P3: adjoint identity ---------------------------------------------------

@pytest.mark.parametrize("Nt,Nd,Nm", [(4, 3, 5), (17, 2, 9), (64, 8, 32)])
def test_adjoint_identity(Nt, Nd, Nm):
    Fcol, m, d = rand_case(Nt, Nd, Nm, seed=7)
    for name, mv, rmv in ALL_MATVECS:
        lhs = np.vdot(mv(Fcol, m), d)
        rhs = np.vdot(m, rmv(Fcol, d))
        scale = np.linalg.norm(mv(Fcol, m)) * np.linalg.norm(d)
        assert abs(lhs - rhs) <= 1e-13 * scale, name


# --- P4: causality and time invariance --------------------------------------

def test_causality_and_time_invariance():
    Nt, Nd, Nm, j, s = 12, 3, 4, 5, 3
    Fcol, m, _ = rand_case(Nt, Nd, Nm, seed=11)
    d0 = oracle.matvec_direct(Fcol, m)
    m2 = m.copy()
    m2[j] += 1.0
    d2 = oracle.matvec_direct(Fcol, m2)
    np.testing.assert_array_equal(d2[:j], d0[:j])          # exactly unchanged before j
    assert np.all(np.abs(d2[j:] - d0[j:]).sum(axis=1) > 0)
    df = oracle.matvec_fft(Fcol, m2)
    np.testing.assert_allclose(df[:j], d0[:j], rtol=0, atol=1e-12)
    # shift m later by s blocks: d shifts by s
    ms = np.zeros_like(m)
    ms[s:] = m[: Nt - s]
    for name, mv, rmv in ALL_MATVECS:
        ds = mv(Fcol, ms)
        np.testing.assert_allclose(ds[s:], d0[: Nt - s], rtol=0, atol=1e-12)
        np.testing.assert_allclose(ds[:s], 0, rtol=0, atol=1e-12)


# --- P5: spectrum facts -----------------------------------------------------

def test_spectrum_against_explicit_dft_sum():
    Nt, Nd, Nm = 6, 2, 3
    Fcol, _, _ = rand_case(Nt, Nd, Nm, seed=3)
    L = 2 * Nt
    Fh = oracle.spectrum(Fcol)
    assert Fh.shape == (Nt + 1, Nd, Nm)
    for w in range(Nt + 1):
        acc = np.zeros((Nd, Nm), dtype=complex)
        for k in range(Nt):
            acc += Fcol[k] * complex(np.cos(2 * np.pi * w * k / L), -np.sin(2 * np.pi * w * k / L))
        np.testing.assert_allclose(Fh[w], acc, rtol=0, atol=1e-13)


def test_spectrum_endpoints_and_parseval():
    Nt, Nd, Nm = 20, 3, 4
    Fcol, _, _ = rand_case(Nt, Nd, Nm, seed=4)
    Fh = oracle.spectrum(Fcol)
    np.testing.assert_allclose(Fh[0].real, Fcol.sum(axis=0), rtol=0, atol=1e-13)
    np.testing.assert_allclose(Fh[Nt].real, (Fcol * ((-1.0) ** np.arange(Nt))[:, None, None]).sum(axis=0),
                               rtol=0, atol=1e-13)
    assert np.all(Fh[0].imag == 0) and np.all(np.abs(Fh[Nt].imag) <= 1e-13)
    L = 2 * Nt
    energy_t = (Fcol ** 2).sum(axis=0)
    wts = np.full(Nt + 1, 2.0)
    wts[0] = wts[Nt] = 1.0
    energy_f = (wts[:, None, None] * np.abs(Fh) ** 2).sum(axis=0) / L
    np.testing.assert_allclose(energy_f, energy_t, rtol=1e-13)


# --- Section 3.2 mixed precision --------------------------------------------

def test_mixed_all_double_is_fft_path():
    Fcol, m, d = rand_case(32, 4, 16, seed=2)
    Fh = oracle.spectrum(Fcol)
    assert oracle.rel_l2(oracle.matvec_mixed(Fh, m, 32, "ddddd"), oracle.matvec_fft(Fcol, m)) <= 1e-15
    assert oracle.rel_l2(oracle.rmatvec_mixed(Fh, d, 32, "ddddd"), oracle.rmatvec_fft(Fcol, d)) <= 1e-15


def test_mixed_pad_only_costs_nothing_on_fp32_exact_inputs():
    # Section 4.2.1: without perturbed mantissas an FP32 pad is free
    Fcol, m, _ = rand_case(16, 3, 8, seed=9)
    m32 = m.astype(np.float32).astype(np.float64)
    Fh = oracle.spectrum(Fcol)
    a = oracle.matvec_mixed(Fh, m32, 16, "sdddd")
    b = oracle.matvec_mixed(Fh, m32, 16, "ddddd")
    np.testing.assert_array_equal(a, b)
    # With the perturbation (every fraction bit past the 23rd set to one) the
    # inputs are no longer FP32-exact, so the FP32 pad now rounds.  Each value
    # sits (1 - 2^-29) FP32 ulps above an FP32 number and rounds up to the next
    # one, a relative change of about 2^-52: nonzero, but one FP64 ulp.
    mp = synth.perturb_mantissa(m32.copy())
    a = oracle.matvec_mixed(Fh, mp, 16, "sdddd")
    b = oracle.matvec_mixed(Fh, mp, 16, "ddddd")
    assert 0 < oracle.rel_l2(a, b) < 1e-14
    cast = mp.astype(np.float32).astype(np.float64)
    assert np.all(cast != mp)
    assert np.all(np.abs(cast - mp) <= 2.0 ** -51 * np.abs(mp))


def test_mixed_pad_rounds_generic_fp64_inputs():
    # plain FP64 draws are not FP32-exact: an FP32 pad rounds at 2^-24 level
    Fcol, m, _ = rand_case(16, 3, 8, seed=9)
    Fh = oracle.spectrum(Fcol)
    e = oracle.rel_l2(oracle.matvec_mixed(Fh, m, 16, "sdddd"), oracle.matvec_mixed(Fh, m, 16, "ddddd"))
    assert 1e-10 < e < 1e-6


@pytest.mark.parametrize("prec", ["sdddd", "dsddd", "ddsdd", "dddsd", "dddds", "dssdd", "sssss"])
def test_mixed_single_phases_have_fp32_error_level(prec):
    Nt, Nd, Nm = 32, 4, 64
    Fcol = synth.block_column(Nt, Nd, Nm, seed=1)
    m = synth.vectors(synth.TAG_M, Nt, Nm, seed=1)[0]
    d = synth.vectors(synth.TAG_D, Nt, Nd, seed=1)[0]
    Fh = oracle.spectrum(Fcol)
    ref = oracle.matvec_direct(Fcol, m)
    refa = oracle.rmatvec_direct(Fcol, d)
    e = oracle.rel_l2(oracle.matvec_mixed(Fh, m, Nt, prec), ref)
    ea = oracle.rel_l2(oracle.rmatvec_mixed(Fh, d, Nt, prec), refa)
    # at least one FP32 rounding happened, and the error stays at FP32 level
    assert 1e-10 < e < 1e-5
    assert 1e-10 < ea < 1e-5
    # Eq. (error): within the first-order bound times a modest constant
    sv = np.linalg.svd(Fh, compute_uv=False)
    kappa = sv.max() / sv.min()
    assert e <= 10 * oracle.relative_error_bound(prec, Nt, Nm, kappa)
    assert ea <= 10 * oracle.relative_error_bound(prec, Nt, Nd, kappa)


# --- Eq. (error), Section 3.2.1: values worked by hand -------------------------
#
# The bound is kappa [c1 e1 + (cF ed + c2 e2 + c4 e4) log2(Nt) + c3 e3 n + c5 e5 log2(p)]
# with every c_i = 1, c1 = 0 for an FP64 pad, n = n_m = ceil(Nm / p_c) and p = p_c
# for F, n = n_d = ceil(Nd / p_r) and p = p_r for F*, plus e5 outside kappa when
# the unpad phase is FP32 (reading R10).  e_i is the unit roundoff of phase i:
# us = 2^-24 (FP32), ud = 2^-53 (FP64).  The case below has Nt = 1024
# (log2 Nt = 10 exactly), Nd = 100, Nm = 5000, kappa = 4.  Each expected value
# is written as (a, b) for a ud + b us:
#   ddddd F : 4 [(ud+ud+ud) 10 + ud 5000]            = 4 * 5030 ud        -> (20120, 0)
#   ddddd F*: 4 [30 ud + 100 ud]                      = 4 * 130 ud         -> (520, 0)
#   dssdd F : 4 [(ud+us+ud) 10 + us 5000]             = 4 (20 ud + 5010 us) -> (80, 20040)
#   dssdd F*: 4 [(ud+us+ud) 10 + us 100]              = 4 (20 ud + 110 us)  -> (80, 440)
#   ddsdd F : 4 [30 ud + us 5000]                     -> (120, 20000)
#   ddsdd F*: 4 [30 ud + us 100]                      -> (120, 400)
#   ddssd F*: 4 [(ud+ud+us) 10 + us 100]              = 4 (20 ud + 110 us)  -> (80, 440)
#   sdddd F : 4 [us + 30 ud + 5000 ud]                -> (20120, 4)
#   dddds F : 4 [30 ud + 5000 ud] + us                -> (20120, 1)
# On a 2 x 4 grid (p_r = 2, p_c = 4): n_m = 1250, log2 p_c = 2; n_d = 50, log2 p_r = 1:
#   ddddd F : 4 [30 ud + 1250 ud + 2 ud]              = 4 * 1282 ud        -> (5128, 0)
#   ddddd F*: 4 [30 ud + 50 ud + 1 ud]                = 4 * 81 ud          -> (324, 0)
#   dddds F : 4 [30 ud + 1250 ud + 2 us] + us         -> (5120, 9)
#   dssdd F*: 4 [(ud+us+ud) 10 + 50 us + 1 ud]        = 4 (21 ud + 60 us)  -> (84, 240)
BOUND_CASES = [
    # prec, which, p_r, p_c, (a, b)
    ("ddddd", "F", 1, 1, (20120, 0)),
    ("ddddd", "F*", 1, 1, (520, 0)),
    ("dssdd", "F", 1, 1, (80, 20040)),
    ("dssdd", "F*", 1, 1, (80, 440)),
    ("ddsdd", "F", 1, 1, (120, 20000)),
    ("ddsdd", "F*", 1, 1, (120, 400)),
    ("ddssd", "F*", 1, 1, (80, 440)),
    ("sdddd", "F", 1, 1, (20120, 4)),
    ("dddds", "F", 1, 1, (20120, 1)),
    ("ddddd", "F", 2, 4, (5128, 0)),
    ("ddddd", "F*", 2, 4, (324, 0)),
    ("dddds", "F", 2, 4, (5120, 9)),
    ("dssdd", "F*", 2, 4, (84, 240)),
]
US, UD = 2.0 ** -24, 2.0 ** -53


def _bound_pin_failures(fn):
    """The hand-worked cases that ``fn`` (signature of oracle.error_bound) misses."""
    bad = []
    for prec, which, pr, pc, (a, b) in BOUND_CASES:
        want = a * UD + b * US
        got = fn(prec, which, 1024, 100, 5000, 4.0, pr=pr, pc=pc)
        if not abs(got - want) <= 1e-15 * want:
            bad.append((prec, which, pr, pc, got, want))
    return bad


def test_error_bound_hand_values():
    assert _bound_pin_failures(oracle.error_bound) == []


def test_relative_error_bound_hand_values():
    # the same cases through the lower-level entry point, n and p given directly
    for prec, which, pr, pc, (a, b) in BOUND_CASES:
        n, p = (-(-5000 // pc), pc) if which == "F" else (-(-100 // pr), pr)
        got = oracle.relative_error_bound(prec, 1024, n, 4.0, p)
        assert abs(got - (a * UD + b * US)) <= 1e-15 * (a * UD + b * US), (prec, which, pr, pc)


def test_error_bound_rejects_planted_mistakes():
    # plausible slips in restating Eq. (error); each must fail a hand-worked case
    def base(prec, Nt, n, kappa, p, c1_d=0.0, lg=True, unpad=True, pterm=True):
        eps = {"s": US, "d": UD}
        e = [eps[c] for c in prec]
        c1 = c1_d if prec[0] == "d" else 1.0
        b = c1 * e[0] + (UD + e[1] + e[3]) * (np.log2(Nt) if lg else 1.0) + e[2] * n
        if pterm and p > 1:
            b += e[4] * np.log2(p)
        return kappa * b + ((0.0 if prec[4] == "d" else 1.0) * e[4] if unpad else 0.0)

    def with_grid(inner, swap=False, ceil=True):
        def fn(prec, which, Nt, Nd, Nm, kappa, pr=1, pc=1):
            fwd = (which == "F") != swap
            num, q = (Nm, pc) if fwd else (Nd, pr)
            n = -(-num // q) if ceil else num
            return inner(prec, Nt, n, kappa, pc if which == "F" else pr)
        return fn

    assert _bound_pin_failures(with_grid(base)) == []          # the restatement itself passes
    mutants = {
        "n_d and n_m swapped": with_grid(base, swap=True),
        "grid ignored in n": with_grid(base, ceil=False),
        "log2 Nt dropped": with_grid(lambda *a: base(*a, lg=False)),
        "c1 e1 charged for an FP64 pad": with_grid(lambda *a: base(*a, c1_d=1.0)),
        "FP32 unpad term omitted": with_grid(lambda *a: base(*a, unpad=False)),
        "reduction term dropped": with_grid(lambda *a: base(*a, pterm=False)),
    }
    for name, fn in mutants.items():
        assert _bound_pin_failures(fn), name


def test_parse_precision():
    assert oracle.parse_precision("dssdd")[1] == np.float32
    with pytest.raises(ValueError):
        oracle.parse_precision("dsx")
    with pytest.raises(ValueError):
        oracle.parse_precision("dsdsdd")


# --- one-by-one entries -----------------------------------------------------

def test_entries_match_direct():
    Fcol, m, d = rand_case(9, 3, 5, seed=21)
    D = oracle.matvec_direct(Fcol, m)
    MS = oracle.rmatvec_direct(Fcol, d)
    idx = [(0, 0), (8, 2), (4, 1), (7, 0)]
    np.testing.assert_allclose(oracle.matvec_entries(Fcol, m, idx), [D[i, r] for i, r in idx], rtol=1e-14, atol=1e-14)
    idx = [(0, 0), (8, 4), (3, 2), (5, 1)]
    np.testing.assert_allclose(oracle.rmatvec_entries(Fcol, d, idx), [MS[j, n] for j, n in idx], rtol=1e-14, atol=1e-14)


# --- the input generators ---------------------------------------------------

def test_synth_is_blockwise_and_thread_independent():
    F = synth.block_column(5, 3, 4, seed=3, decay=200.0)
    g = synth.block_generator(3, synth.TAG_BLOCK, 4)
    np.testing.assert_array_equal(F[4], g.standard_normal((3, 4)) * np.exp(-4 / 200.0))
    v = synth.vectors(synth.TAG_M, 4, 6, k=2, seed=3)
    g = synth.block_generator(3, synth.TAG_M, 1, 2)
    np.testing.assert_array_equal(v[1, 2], g.standard_normal(6))


def test_perturb_mantissa():
    x = np.array([1.0, -2.5, 0.0, 3.0e-5, np.inf])
    y = synth.perturb_mantissa(x.copy())
    assert y[2] == 0.0 and np.isinf(y[4])
    for a, b in zip(x[[0, 1, 3]], y[[0, 1, 3]]):
        assert a != b and abs(a - b) <= 2.0 ** -23 * abs(a)
        assert np.float64(np.float32(b)) != b          # not FP32-exact any more
        assert (np.float64(b).view(np.uint64) & np.uint64((1 << 29) - 1)) == (1 << 29) - 1


# --- data-space Hessian entries (Section 2, Remark 1) ------------------------

def test_hessian_entries_match_dense_gram():
    # H_d = prior F F^T + noise I: rows of the dense matrix, entry by entry
    Nt, Nd, Nm = 7, 3, 5
    Fcol = synth.block_column(Nt, Nd, Nm, seed=8)
    A = oracle.dense_matrix(Fcol)
    H = 0.7 * A @ A.T + 0.05 * np.eye(Nt * Nd)
    rng = np.random.default_rng(0)
    pairs = [((int(a), int(b)), (int(c), int(e))) for a, b, c, e in
             zip(rng.integers(Nt, size=40), rng.integers(Nd, size=40), rng.integers(Nt, size=40), rng.integers(Nd, size=40))]
    pairs += [((3, 1), (3, 1)), ((0, 0), (6, 2))]
    got = oracle.hessian_entries(Fcol, pairs, prior_var=0.7, noise_var=0.05)
    ref = np.array([H[t1 * Nd + r1, t2 * Nd + r2] for (t1, r1), (t2, r2) in pairs])
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(H).max())


def test_hessian_entries_identity_operator():
    # F_0 = I, F_k = 0: F F^T = I, so H_d = (prior + noise) I exactly
    Nt, N = 5, 4
    Fcol = np.zeros((Nt, N, N))
    Fcol[0] = np.eye(N)
    pairs = [((t, r), (t2, r2)) for t in range(Nt) for r in range(N) for t2 in (0, t) for r2 in (0, r)]
    got = oracle.hessian_entries(Fcol, pairs, prior_var=2.0, noise_var=0.25)
    ref = np.array([2.25 if (a == b) else 0.0 for a, b in pairs])
    np.testing.assert_array_equal(got, ref)
