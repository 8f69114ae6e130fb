"""The infinite-lattice strip expansion (Sec. IV.C) on the GPU, through the C
ABI, against the FP64 oracle: BP messages, strip eigenvalues, capped patches
and the free energy, for blocked Ising tensors across the transition and for
random tensors; exactness on product networks; convergence to Onsager's free
energy at widths beyond the oracle's reach; argument checks.

Tolerances: messages and ln z_BP within 1e-12; ln lambda_k, ln gamma_k and
ln Z_wh within 1e-11 absolute (values up to ~100; both sides converge the
eigenvalue to ~1e-15 relative); f within 1e-10 relative (the FP64 bound:
the subset sum amplifies input rounding by its cancellation factor, below
4e3 at the widths compared here).
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402
from oracle import exact as X  # noqa: E402
from oracle import strips as S  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build
    build.build()
    c = pne.Context(0)
    yield c
    c.close()


def _tensors():
    return [("ising_b0.30", I.uniform_ising(0.30, 2)), ("ising_b0.4407", I.uniform_ising(0.4407, 2)),
            ("ising_b0.47", I.uniform_ising(0.47, 2)), ("random_chi3", I.uniform_random(3, 7)),
            ("random_chi2_n", I.uniform_random(2, 9, "n1,0.3"))]


def _check(res, ref, L, two_d=True):
    for a, b in zip(res["msgs"], ref["msgs"]):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    assert abs(res["f_bp"] - ref["f_bp"]) < 1e-12
    for k in range(1, L + 1):
        assert abs(res["log_lam"][k] - ref["log_lam"][k]) < 1e-11, (k, res["log_lam"][k], ref["log_lam"][k])
        if two_d:
            assert abs(res["log_gam"][k] - ref["log_gam"][k]) < 1e-11, k
            for h in range(1, L + 1):
                assert res["sign_z"][k][h] == 1
                assert abs(res["log_z"][k][h] - ref["log_z"][k][h]) < 1e-11, (k, h)
    assert abs(res["f"] - ref["f"]) <= 1e-10 * abs(ref["f"]), (res["f"], ref["f"])


@pytest.mark.parametrize("arith", [0, 1], ids=["fp64", "ff"])
@pytest.mark.parametrize("L", [1, 2, 4])
def test_strip_expansion_matches_oracle_2d(ctx, L, arith):
    # every tensor of one chi in one call (data-parallel over the tensors)
    groups = {}
    for name, A in _tensors():
        groups.setdefault(A.shape[0], []).append((name, A))
    for chi, items in groups.items():
        res = pne.pne_strip_expansion(ctx.h, np.stack([A for _, A in items]), L, arithmetic=arith)
        for (name, A), r in zip(items, res):
            assert r["status"] == pne.PNE_OK, name
            _check(r, S.strip_expansion(A, L), L)


@pytest.mark.parametrize("arith", [0, 1], ids=["fp64", "ff"])
def test_strip_expansion_matches_oracle_width5(ctx, arith):
    A = I.uniform_ising(0.42, 2)
    (r,) = pne.pne_strip_expansion(ctx.h, A, 5, arithmetic=arith)
    _check(r, S.strip_expansion(A, 5), 5)


def test_float_float_rows_agree_with_fp64_at_width8(ctx):
    # the two arithmetics of the row products, beyond the oracle's widths
    A = np.stack([I.uniform_ising(b, 2) for b in (0.35, 0.44)] + [I.uniform_random(4, 3)])
    r64 = pne.pne_strip_expansion(ctx.h, A, 8, arithmetic=0)
    rff = pne.pne_strip_expansion(ctx.h, A, 8, arithmetic=1)
    for a, b in zip(r64, rff):
        for k in range(1, 9):
            assert abs(a["log_lam"][k] - b["log_lam"][k]) < 1e-11
            assert abs(a["log_gam"][k] - b["log_gam"][k]) < 1e-11
            for h in range(1, 9):
                assert abs(a["log_z"][k][h] - b["log_z"][k][h]) < 1e-11
        assert abs(a["f"] - b["f"]) <= 1e-11 * abs(a["f"])
        assert all(x >= 8 for x in a["iters"][0][1:]) and all(x >= 8 for x in b["iters"][1][1:])


def test_one_dimensional_form_matches_oracle(ctx):
    for name, A in _tensors()[:4]:
        (r,) = pne.pne_strip_expansion(ctx.h, A, 6, two_d=False)
        ref = S.strip_expansion(A, 6, two_d=False)
        _check(r, ref, 6, two_d=False)


def test_device_input_gives_the_same_results(ctx):
    A = np.stack([I.uniform_ising(b, 2) for b in (0.35, 0.45)])
    host = pne.pne_strip_expansion(ctx.h, A, 3)
    dev = pne.pne_strip_expansion(ctx.h, torch.from_numpy(A).cuda(), 3)
    for a, b in zip(host, dev):
        assert a["f"] == b["f"] and a["log_lam"] == b["log_lam"] and a["log_z"] == b["log_z"]


def test_product_network_is_exact(ctx):
    rng = np.random.default_rng(4)
    a, b, c, e = (rng.uniform(0.2, 1.0, 4) for _ in range(4))
    exact = -math.log(float(a @ c) * float(b @ e))
    for L in (1, 3, 6):
        (r,) = pne.pne_strip_expansion(ctx.h, I.uniform_product(a, b, c, e), L)
        assert abs(r["f"] - exact) < 1e-12 * abs(exact) + 1e-13, (L, r["f"], exact)


def test_wide_strips_approach_onsager(ctx):
    # beyond the oracle's widths: at L = 10 (chi^11 = 4M entries per running
    # tensor) the lambda_k and Z_wh of the narrow strips still equal the
    # oracle's, and the error against Onsager keeps falling with L
    betas = (0.30, 0.42, 0.60)
    A = np.stack([I.uniform_ising(b, 2) for b in betas])
    res10 = pne.pne_strip_expansion(ctx.h, A, 10, arithmetic=1)
    for beta, r in zip(betas, res10):
        exact = -4.0 * X.onsager_minus_beta_f(beta)
        ref = S.strip_expansion(I.uniform_ising(beta, 2), 4)
        for k in range(1, 5):
            assert abs(r["log_lam"][k] - ref["log_lam"][k]) < 1e-11
            for h in range(1, 5):
                assert abs(r["log_z"][k][h] - ref["log_z"][k][h]) < 1e-11
        errs = []
        for L in range(2, 11):
            f = S.expansion_2d(r["log_lam"], r["log_gam"], r["log_z"], L)
            errs.append(abs(f - exact) / abs(exact))
        assert abs(errs[-1] - abs(r["f"] - exact) / abs(exact)) <= 1e-10
        # monotone down to the FP64 floor of the sum (cancellation x rounding)
        floor = 1e-12
        assert all(errs[i + 1] < errs[i] or errs[i + 1] < floor for i in range(len(errs) - 1)), (beta, errs)
        assert errs[-1] < errs[2] / 3 or errs[-1] < floor, (beta, errs)


@pytest.mark.parametrize("chi,L", [(1, 2), (9, 2), (4, 0), (4, 13), (8, 9)])
def test_bad_arguments_are_rejected_before_any_launch(ctx, chi, L):
    A = np.ones((1,) + (max(chi, 1),) * 4)
    with pytest.raises(pne.PneError) as e:
        pne.pne_strip_expansion(ctx.h, A, L)
    assert e.value.status == pne.PNE_EINVAL
