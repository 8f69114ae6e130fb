"""Pins of the strip-expansion oracle (Sec. IV.C) against closed forms, literal
spin sums, the formulas the paper prints, and Onsager's free energy."""
import itertools
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I
from oracle import exact as X
from oracle import strips as S


def _bethe_ln_z(beta):
    # paramagnetic BP fixed point of the square-lattice Ising model: per spin
    # 2 (states) x cosh(beta) per bond, two bonds per spin
    return math.log(2.0) + 2.0 * math.log(math.cosh(beta))


@pytest.mark.parametrize("beta", [0.1, 0.25, 0.34])
def test_uniform_bp_is_the_paramagnetic_bethe_value(beta):
    mR, mL, mD, mU, lz, _ = S.uniform_bp(I.uniform_ising(beta, 1))
    assert abs(lz - _bethe_ln_z(beta)) < 1e-13
    for m in (mR, mL, mD, mU):
        np.testing.assert_allclose(m, [2 ** -0.5, 2 ** -0.5], atol=1e-13)


def _open_strip_spin_transfer(k, beta):
    """Row-to-row transfer matrix of an open chain of k Ising spins, written
    from the Boltzmann weights: the vertical bonds between the rows in full,
    each row's own horizontal bonds split half and half between the two
    matrices that share the row."""
    states = list(itertools.product((1, -1), repeat=k))
    T = np.zeros((len(states), len(states)))
    for i, s in enumerate(states):
        for j, t in enumerate(states):
            e = sum(a * b for a, b in zip(s, t))
            e += 0.5 * sum(s[x] * s[x + 1] for x in range(k - 1))
            e += 0.5 * sum(t[x] * t[x + 1] for x in range(k - 1))
            T[i, j] = math.exp(beta * e)
    return T


@pytest.mark.parametrize("beta", [0.2, 0.3])
def test_strip_eigenvalues_are_open_ising_strips(beta):
    # in the paramagnetic phase each capped leg gives sqrt(cosh beta) for
    # either spin value: a width-k strip has two capped legs per row
    A = I.uniform_ising(beta, 1)
    mR, mL, mD, mU, lz, _ = S.uniform_bp(A)
    for k in range(1, 5):
        lead = max(np.linalg.eigvalsh(_open_strip_spin_transfer(k, beta)))
        assert abs(S.leading_log_eig(A, k, mR, mL) - (math.log(math.cosh(beta)) + math.log(lead))) < 1e-12


@pytest.mark.parametrize("w,h", [(1, 1), (1, 3), (2, 2), (3, 2), (2, 4), (3, 3)])
def test_patches_are_open_ising_spin_sums(w, h):
    beta = 0.3
    A = I.uniform_ising(beta, 1)
    msgs = S.uniform_bp(A)[:4]
    spin = X.ising_spin_sum(I.square_lattice(w, h, 2), beta)
    want = (w + h) * math.log(math.cosh(beta)) + math.log(spin)
    sign, lz = S.patch_log_z(A, w, h, msgs)
    assert sign == 1 and abs(lz - want) < 1e-12
    assert abs(S.patch_log_z_rows(A, w, h, msgs)[h - 1] - want) < 1e-12


def test_row_apply_matches_the_dense_transfer_matrix():
    A = I.uniform_random(3, 11)
    mR, mL = S.uniform_bp(A)[:2]
    rng = np.random.default_rng(0)
    for k in range(1, 5):
        v = rng.standard_normal(3 ** k)
        T = S.row_transfer_matrix(A, k, mR, mL)
        np.testing.assert_allclose(S.row_apply(A, k, mR, mL, v), T @ v, rtol=0, atol=1e-12 * np.abs(T @ v).max())


def _column_transfer(A, k, mD, mU):
    """Horizontal strip of k rows (a column of k tensors, top u leg capped by
    mD, bottom d leg by mU), as the matrix from the l legs to the r legs,
    built directly from A."""
    chi = A.shape[0]
    ops, lab = [], {}

    def L(name):
        return lab.setdefault(name, len(lab))
    for y in range(k):
        ops += [A, [L(("l", y)), L(("v", y - 1)), L(("r", y)), L(("v", y))]]
    ops += [mD, [L(("v", -1))], mU, [L(("v", k - 1))]]
    out = [L(("r", y)) for y in range(k)] + [L(("l", y)) for y in range(k)]
    return np.einsum(*ops, out).reshape(chi ** k, chi ** k)


def test_transposed_lattice_gives_the_horizontal_strips():
    A = I.uniform_random(3, 5)
    msgs = S.uniform_bp(A)[:4]
    At, mt = S.transpose_lattice(A, msgs)
    for k in range(1, 4):
        ev = np.linalg.eigvals(_column_transfer(A, k, msgs[2], msgs[3]))
        assert abs(S.leading_log_eig(At, k, mt[0], mt[1]) - math.log(max(abs(ev)))) < 1e-12
    for w, h in ((1, 2), (2, 3)):
        assert abs(S.patch_log_z(At, h, w, mt)[1] - S.patch_log_z(A, w, h, msgs)[1]) < 1e-12


@pytest.mark.parametrize("tensor", ["random", "ising"])
def test_width_one_strips_are_bp(tensor):
    # at a BP fixed point mD is the Perron vector of the one-site transfer
    # matrix, with eigenvalue z_BP: the L = 1 expansion is BP
    A = I.uniform_random(3, 2) if tensor == "random" else I.uniform_ising(0.44, 2)
    r = S.strip_expansion(A, 1)
    assert abs(r["log_lam"][1] + r["f_bp"]) < 1e-12
    assert abs(r["f"] - r["f_bp"]) < 1e-12
    assert abs(S.expansion_1d(r["log_lam"], 1) - r["f_bp"]) < 1e-12


def test_the_printed_width_two_and_three_formulas():
    A = I.uniform_ising(0.42, 2)
    r = S.strip_expansion(A, 3)
    lam = [None] + [math.exp(x) for x in r["log_lam"][1:]]
    gam = [None] + [math.exp(x) for x in r["log_gam"][1:]]
    Z = [[None] * 4] + [[None] + [math.exp(x) for x in row[1:]] for row in r["log_z"][1:]]
    assert abs(S.expansion_1d(r["log_lam"], 2) + math.log(2 * lam[2] - lam[1] ** 2) / 2) < 1e-13
    assert abs(S.expansion_1d(r["log_lam"], 3)
               + math.log(3 * lam[3] - 3 * lam[2] * lam[1] + lam[1] ** 3) / 3) < 1e-13
    R1 = 2 * lam[2] ** 2 + 2 * gam[2] ** 2
    R2 = 4 * Z[2][2] + lam[1] ** 4 + gam[1] ** 4
    R3 = 2 * Z[2][1] ** 2 + 2 * Z[1][2] ** 2
    R4 = Z[1][1] ** 4
    assert abs(S.expansion_2d(r["log_lam"], r["log_gam"], r["log_z"], 2) + math.log(R1 - R2 + R3 - R4) / 4) < 1e-13


def test_product_network_is_exact_at_every_width():
    rng = np.random.default_rng(3)
    a, b, c, e = (rng.uniform(0.2, 1.0, 3) for _ in range(4))
    A = I.uniform_product(a, b, c, e)
    exact = -math.log(float(a @ c) * float(b @ e))
    r = S.strip_expansion(A, 4)
    for L in range(1, 5):
        assert abs(S.expansion_1d(r["log_lam"], L) - exact) < 1e-12
        assert abs(S.expansion_2d(r["log_lam"], r["log_gam"], r["log_z"], L) - exact) < 1e-12
    # the width-3 formula with every sign positive is not exact here
    lam = [math.exp(x) for x in r["log_lam"][1:4]]
    assert abs(-math.log(3 * lam[2] + 3 * lam[1] * lam[0] + lam[0] ** 3) / 3 - exact) > 0.1


def test_patch_ratios_converge_to_the_strip_eigenvalue():
    A = I.uniform_ising(0.3, 2)
    msgs = S.uniform_bp(A)[:4]
    for w in (1, 2, 3):
        z = S.patch_log_z_rows(A, w, 40, msgs)
        assert abs((z[39] - z[38]) - S.leading_log_eig(A, w, msgs[0], msgs[1])) < 1e-12


@pytest.mark.parametrize("beta,bound4", [(0.3, 5e-8), (0.6, 1e-9)])
def test_blocked_ising_approaches_onsager(beta, bound4):
    # 2 x 2 blocked tensor: four spins per site
    exact = -4.0 * X.onsager_minus_beta_f(beta)
    r = S.strip_expansion(I.uniform_ising(beta, 2), 4)
    errs = [abs(S.expansion_2d(r["log_lam"], r["log_gam"], r["log_z"], L) - exact) / abs(exact) for L in range(1, 5)]
    bp_err = abs(r["f_bp"] - exact) / abs(exact)
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[1] < bp_err / 10
    assert errs[3] < bound4, errs
