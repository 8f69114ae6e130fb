"""Dense contractions on the tensor cores (tcgen05) and the exact contraction
of 2D grid networks built on them, through the C ABI.

* pne_dense_gemm: the TF32 / BF16 products equal the FP64 product of the
  inputs rounded the way the call states (TF32 nearest with ties away, BF16
  nearest-even; rounding emulated here on the bits), within the FP32
  accumulation bound K 2^-24 sum |a b| per entry; FP64 equals numpy's FP64
  product to 1e-13 relative.  Shapes cover one tile, ragged M, N and K tails,
  several N tiles and several K stages, and a batch.
* pne_grid_contract: FP64 equals the oracle's exact contraction within 1e-12
  relative (random, AKLT-like signed and Ising blocked tensors, bond
  dimensions 2 .. 16, uneven dimensions); TF32 / BF16 within the stated
  err_bound (non-negative networks, where the bound is relative to Z), and the
  bound itself below 0.1 (TF32) / 0.5 (BF16).
"""
import math

import numpy as np
import pytest

from paper_2512_10910_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2512_10910_gb300 import pne  # noqa: E402
from oracle import exact as X  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_10910_gb300 import build
    build.build()
    c = pne.Context(0)
    yield c
    c.close()


def _round_tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)       # nearest, ties away (on the magnitude bits)
    return b.view(np.float32).astype(np.float64)


def _round_bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16          # nearest, ties to even
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


SHAPES = [(1, 16, 1), (128, 16, 32), (100, 40, 7), (300, 256, 33), (257, 300, 200), (64, 1, 70), (513, 96, 129)]


@pytest.mark.parametrize("dtype", [pne.PNE_TF32, pne.PNE_BF16, pne.PNE_F64], ids=["tf32", "bf16", "f64"])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_dense_gemm_matches_rounded_fp64_product(ctx, dtype, M, N, K):
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    batch = 2
    A = rng.standard_normal((batch, M, K))
    B = rng.standard_normal((batch, N, K))
    tdt = torch.float64 if dtype == pne.PNE_F64 else torch.float32
    At = torch.from_numpy(A).to(tdt).cuda()
    Bt = torch.from_numpy(B).to(tdt).cuda()
    Ct = torch.full((batch, M, N), float("nan"), dtype=tdt, device="cuda")
    pne.pne_dense_gemm(ctx.h, dtype, At, Bt, Ct)
    C = Ct.cpu().numpy().astype(np.float64)
    if dtype == pne.PNE_F64:
        ref = np.einsum("bmk,bnk->bmn", A, B)
        np.testing.assert_allclose(C, ref, rtol=0, atol=1e-13 * np.einsum("bmk,bnk->bmn", abs(A), abs(B)).max())
        return
    rnd = _round_tf32 if dtype == pne.PNE_TF32 else _round_bf16
    a32, b32 = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    ra, rb = rnd(a32), rnd(b32)
    ref = np.einsum("bmk,bnk->bmn", ra, rb)
    absref = np.einsum("bmk,bnk->bmn", abs(ra), abs(rb))
    err = np.abs(C - ref)
    assert np.all(err <= (K + 2) * 2.0 ** -24 * absref + 1e-30), float((err / (absref + 1e-300)).max())


def _grid_cases():
    out = []
    for lx, ly, d, seed in ((3, 3, 4, 1), (4, 3, 5, 2), (2, 5, 3, 3), (1, 4, 6, 4), (5, 1, 7, 5)):
        out.append((f"random{lx}x{ly}_D{d}", I.random_tensors(I.square_lattice(lx, ly, d), seed), lx, ly, True))
    out.append(("ising3x3_blocked4_b0.44", I.ising_blocked(3, 3, 4, 0.44), 3, 3, True))   # chi = 16
    out.append(("signed3x3_D3", I.random_tensors(I.square_lattice(3, 3, 3), 9, "bias:0.2"), 3, 3, False))
    # uneven bond dimensions on one grid
    g = I.square_lattice(3, 2, 2)
    g.bond_dim[:] = np.array([2, 3, 4, 5, 6, 3, 2], dtype=np.int32)[:g.n_bonds]
    out.append(("uneven3x2", I.random_tensors(g, 11), 3, 2, True))
    return out


@pytest.mark.parametrize("case", _grid_cases(), ids=lambda c: c[0])
def test_grid_contract_matches_oracle(ctx, case):
    name, net, lx, ly, nonneg = case
    t, ls = X.contract_sweep(net)
    exact = float(t) * math.exp(ls) if abs(ls) < 600 else None
    ln_exact = math.log(abs(float(t))) + ls
    sign = 1 if float(t) > 0 else -1
    (r64,) = pne.pne_grid_contract(ctx.h, net, lx, ly, pne.PNE_F64)
    assert r64["sign"] == sign
    assert abs(r64["log_abs"] - ln_exact) < 1e-12 * max(1.0, abs(ln_exact)), (r64["log_abs"], ln_exact)
    for dt, cap in ((pne.PNE_TF32, 0.1), (pne.PNE_BF16, 0.5)):
        (r,) = pne.pne_grid_contract(ctx.h, net, lx, ly, dt)
        assert r["err_bound"] < cap
        if nonneg:
            assert r["sign"] == sign
            assert abs(math.expm1(r["log_abs"] - ln_exact)) <= r["err_bound"], (name, dt, r["log_abs"], ln_exact)
    del exact


def test_grid_contract_batches_tensor_sets_and_device_data(ctx):
    g = I.square_lattice(4, 4, 8)
    nets = [I.random_tensors(g, 100 + i) for i in range(3)]
    flat = np.concatenate([n.flat_data()[0] for n in nets])
    ref = []
    for n in nets:
        t, ls = X.contract_sweep(n)
        ref.append(math.log(abs(float(t))) + ls)
    host = pne.pne_grid_contract(ctx.h, g, 4, 4, pne.PNE_F64, data=flat, n_batch=3)
    dev = pne.pne_grid_contract(ctx.h, g, 4, 4, pne.PNE_F64, data=torch.from_numpy(flat).cuda(), n_batch=3)
    tf = pne.pne_grid_contract(ctx.h, g, 4, 4, pne.PNE_TF32, data=torch.from_numpy(flat).cuda(), n_batch=3)
    for a, b, c, e in zip(host, dev, tf, ref):
        assert a["log_abs"] == b["log_abs"]
        assert abs(a["log_abs"] - e) < 1e-12 * abs(e)
        assert abs(math.expm1(c["log_abs"] - e)) <= c["err_bound"]


def test_grid_contract_rejects_non_grids(ctx):
    net = I.random_tensors(I.cubic_lattice(2, 2, 2, 2), 1)
    with pytest.raises(pne.PneError) as e:
        pne.pne_grid_contract(ctx.h, net, 4, 2, pne.PNE_F64)
    assert e.value.status == pne.PNE_EINVAL
    net = I.random_tensors(I.square_lattice(3, 3, 2), 1)
    with pytest.raises(pne.PneError):
        pne.pne_grid_contract(ctx.h, net, 3, 3, pne.PNE_F32)


def test_grid_contract_large_batch(ctx):
    # enough row tiles (5 x 4 grid of bond dimension 8, 16 tensor sets: up to
    # 8^4 rows per set) for the persistent tensor-core form; FP64 against the
    # oracle on two sets, TF32 / BF16 within their stated bounds of FP64 on all
    g = I.square_lattice(5, 4, 8)
    nets = [I.random_tensors(g, 300 + i) for i in range(16)]
    flat = np.concatenate([n.flat_data()[0] for n in nets])
    data = torch.from_numpy(flat).cuda()
    r64 = pne.pne_grid_contract(ctx.h, g, 5, 4, pne.PNE_F64, data=data, n_batch=16)
    for i in (0, 7):
        t, ls = X.contract_sweep(nets[i])
        e = math.log(abs(float(t))) + ls
        assert abs(r64[i]["log_abs"] - e) < 1e-12 * abs(e)
    for dt in (pne.PNE_TF32, pne.PNE_BF16):
        r = pne.pne_grid_contract(ctx.h, g, 5, 4, dt, data=data, n_batch=16)
        for a, b in zip(r, r64):
            assert a["sign"] == b["sign"]
            assert abs(math.expm1(a["log_abs"] - b["log_abs"])) <= a["err_bound"]
