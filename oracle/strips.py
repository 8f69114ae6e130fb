"""Infinite-lattice strip expansion of the PNE (oracle; FP64).

Test infrastructure only (see ``oracle/__init__.py``).

The network is an infinite square lattice with one tensor A on every site,
axes [l, u, r, d] (the leg towards x - 1, y - 1, x + 1, y + 1).  Sec. IV.C:

* A partition is the set of horizontal bonds crossing one family of vertical
  lines, every L-th column boundary at a fixed offset (or, for horizontal
  strips, the vertical bonds crossing every L-th row boundary).  Its projector
  factorises over those bonds into the rank-1 BP projectors (Eq. A7, A8), so
  inserting it cuts the lattice into independent strips whose cut legs are
  capped by the BP messages; with messages scaled to unit overlap on every
  bond the cut bonds contribute no further factor.
* A vertical strip of width k, infinite in y, contributes lambda_k per row:
  the leading eigenvalue of its row transfer matrix, the row of k tensors with
  the outer l and r legs capped.  gamma_k is the same for horizontal strips.
  Where vertical and horizontal partitions are both inserted the lattice falls
  into finite w x h patches with every boundary leg capped; Z_wh is the value
  of one (w columns, h rows).
* The expansion is the combinatorial form (Eq. A6) over the 2L partitions of
  one L x L unit cell (L vertical offsets, L horizontal offsets), written per
  cell as the paper does for its width-2 and width-3 formulas: every non-empty
  subset x of the partitions contributes (-1)^{|x|+1} times the product of its
  pieces over one cell, and f = -ln(sum) / L^2 per site (-ln(sum) / L for the
  vertical strips alone, the 1D form).  For x with vertical offsets V and
  horizontal offsets H the pieces are the strips or patches between the
  consecutive offsets (cyclically, so the gaps of V sum to L):
      H empty:   prod_{w in gaps(V)} lambda_w^L
      V empty:   prod_{h in gaps(H)} gamma_h^L
      otherwise: prod_{w in gaps(V)} prod_{h in gaps(H)} Z_wh.
  For L = 2 this is the paper's R1 - R2 + R3 - R4 and, for vertical strips
  alone, 2 lambda_2 - lambda_1^2.  Reading: the width-3 formula is taken with
  the alternating signs of Eq. A6 (3 lambda_3 - 3 lambda_2 lambda_1 +
  lambda_1^3); with every sign positive the expansion would not be exact for
  a product network, where lambda_k = lambda_1^k.

Free energies are per site of the lattice of A: f = -lim ln Z / N.
"""
from __future__ import annotations

import math
from itertools import combinations

import numpy as np

__all__ = ["uniform_bp", "transpose_lattice", "row_transfer_matrix", "row_apply", "leading_log_eig",
           "patch_log_z", "patch_log_z_rows", "gaps", "expansion_1d", "expansion_2d", "strip_expansion"]


def uniform_bp(A, tol=1e-14, max_iter=200000):
    """BP fixed point of the infinite uniform lattice (Eq. A7 with every site
    alike): four messages mR (flowing +x, arriving on an l leg), mL (-x, on an
    r leg), mD (+y, on a u leg), mU (-y, on a d leg), each the tensor contracted
    with the three messages arriving on its other legs.  Parallel updates,
    each message scaled to unit 2-norm with its largest entry positive.  At
    the end mR, mL (and mD, mU) are rescaled to unit overlap <mR, mL> = 1
    (<mD, mU> = 1).  Returns (mR, mL, mD, mU, ln z_BP, sweeps), z_BP the site
    value sum A mR mD mL mU: the BP value per site."""
    A = np.asarray(A, dtype=np.float64)
    chi = A.shape[0]
    m = [np.ones(chi) / math.sqrt(chi) for _ in range(4)]

    def norm(x):
        x = x / np.linalg.norm(x)
        return x if x[np.argmax(np.abs(x))] > 0 else -x
    for it in range(1, max_iter + 1):
        mR, mL, mD, mU = m
        new = [norm(np.einsum("lurd,l,u,d->r", A, mR, mD, mU)),
               norm(np.einsum("lurd,r,u,d->l", A, mL, mD, mU)),
               norm(np.einsum("lurd,l,r,u->d", A, mR, mL, mD)),
               norm(np.einsum("lurd,l,r,d->u", A, mR, mL, mU))]
        diff = max(float(np.max(np.abs(a - b))) for a, b in zip(new, m))
        m = new
        if diff < tol:
            break
    else:
        raise RuntimeError("uniform BP did not converge")
    mR, mL, mD, mU = m
    sh = float(mR @ mL)
    sv = float(mD @ mU)
    mR, mL = mR / math.sqrt(abs(sh)), mL * (math.copysign(1.0, sh) / math.sqrt(abs(sh)))
    mD, mU = mD / math.sqrt(abs(sv)), mU * (math.copysign(1.0, sv) / math.sqrt(abs(sv)))
    z = float(np.einsum("lurd,l,u,r,d->", A, mR, mD, mL, mU))
    return mR, mL, mD, mU, math.log(z), it


def transpose_lattice(A, msgs):
    """The lattice reflected across its diagonal (x <-> y): horizontal strips
    of A are the vertical strips of the result, and a w x h patch of A is an
    h x w patch of the result.  ``msgs`` = (mR, mL, mD, mU)."""
    mR, mL, mD, mU = msgs
    return np.ascontiguousarray(np.transpose(A, (1, 0, 3, 2))), (mD, mU, mR, mL)


def row_transfer_matrix(A, k, mR, mL):
    """T_k[d_1..d_k, u_1..u_k]: one row of k tensors, the l leg of the first
    capped by mR and the r leg of the last by mL (the messages a cut bond's
    projector leaves on the strip), as a chi^k x chi^k matrix."""
    chi = A.shape[0]
    # running tensor R[h, d_1..d_j, u_1..u_j]
    R = np.einsum("l,lurd->rdu", mR, A)
    for j in range(1, k):
        R = np.einsum("h...,hurd->r...du", R, A)
        # axes now [r, d_1..d_j, u_1..u_j, d_{j+1}, u_{j+1}]: move d_{j+1} after d_j
        nd = j
        perm = [0] + list(range(1, 1 + nd)) + [1 + 2 * nd] + list(range(1 + nd, 1 + 2 * nd)) + [2 + 2 * nd]
        R = np.transpose(R, perm)
    T = np.tensordot(mL, R, axes=([0], [0]))
    return T.reshape(chi ** k, chi ** k)


def row_apply(A, k, mR, mL, v):
    """T_k v without forming T_k: the tensors applied one site at a time
    (for widths whose matrix would not fit).  The running tensor has axes
    [h, d_1..d_j, u_{j+1}..u_k], h the open r leg of site j."""
    chi = A.shape[0]
    W = np.multiply.outer(mR, np.asarray(v, dtype=np.float64).reshape(-1))      # [h, u_1..u_k]
    for j in range(k):
        W = W.reshape(chi, chi ** j, chi, chi ** (k - j - 1))                    # [h, P, u, S]
        W = np.einsum("hpus,hurd->rpds", W, A)
    return np.tensordot(mL, W.reshape(chi, -1), axes=([0], [0]))


def leading_log_eig(A, k, mR, mL, dense_limit=4096):
    """ln lambda_k: the leading eigenvalue of T_k (largest modulus; real and
    positive for a non-negative network).  Dense eigenvalues (LAPACK) up to
    chi^k = dense_limit, ARPACK on ``row_apply`` above."""
    chi = A.shape[0]
    n = chi ** k
    if n <= dense_limit:
        ev = np.linalg.eigvals(row_transfer_matrix(A, k, mR, mL))
    else:
        from scipy.sparse.linalg import LinearOperator, eigs
        op = LinearOperator((n, n), matvec=lambda x: row_apply(A, k, mR, mL, np.asarray(x, dtype=np.float64)),
                            dtype=np.float64)
        ev = eigs(op, k=2, which="LM", tol=1e-15, return_eigenvectors=False)
    lead = ev[np.argmax(np.abs(ev))]
    if abs(lead.imag) > 1e-12 * abs(lead) or lead.real <= 0:
        raise ValueError(f"leading eigenvalue {lead} is not real and positive")
    return math.log(lead.real)


def patch_log_z(A, w, h, msgs):
    """(sign, ln|Z_wh|) of the w x h patch (w columns, h rows) with every
    boundary leg capped by the message arriving there, contracted as one
    einsum over the whole patch."""
    mR, mL, mD, mU = msgs
    lab = {}

    def hb(x, y):
        return lab.setdefault(("h", x, y), len(lab))

    def vb(x, y):
        return lab.setdefault(("v", x, y), len(lab))
    ops = []
    for y in range(h):
        for x in range(w):
            ops += [A, [hb(x - 1, y), vb(x, y - 1), hb(x, y), vb(x, y)]]
    for y in range(h):
        ops += [mR, [hb(-1, y)], mL, [hb(w - 1, y)]]
    for x in range(w):
        ops += [mD, [vb(x, -1)], mU, [vb(x, h - 1)]]
    z = float(np.einsum(*ops, [], optimize="greedy"))
    return (1 if z > 0 else -1 if z < 0 else 0), (math.log(abs(z)) if z != 0 else -math.inf)


def patch_log_z_rows(A, w, h_max, msgs):
    """ln Z_wh for h = 1..h_max by a row sweep: the top caps mD^{(x)w}, then
    T_w applied row after row, each height closed with mU^{(x)w}."""
    mR, mL, mD, mU = msgs
    top = np.ones(())
    bot = np.ones(())
    for _ in range(w):
        top = np.multiply.outer(top, mD)
        bot = np.multiply.outer(bot, mU)
    v = top.reshape(-1)
    bot = bot.reshape(-1)
    out, scale = [], 0.0
    for _ in range(h_max):
        v = row_apply(A, w, mR, mL, v)
        nv = float(np.max(np.abs(v)))
        v = v / nv
        scale += math.log(nv)
        z = float(v @ bot)
        out.append(scale + math.log(abs(z)))
    return out


def gaps(offsets, L):
    """Widths of the pieces between consecutive cut offsets of one period."""
    o = sorted(offsets)
    return [o[i + 1] - o[i] for i in range(len(o) - 1)] + [L - o[-1] + o[0]]


def _log_sum_signed(terms):
    """ln of sum s_i exp(t_i) for signs s_i = +-1 (math.fsum: correctly
    rounded), referred to the largest t_i."""
    ref = max(t for _, t in terms)
    s = math.fsum(sg * math.exp(t - ref) for sg, t in terms)
    if s <= 0:
        raise ValueError("the expansion's sum is not positive")
    return ref + math.log(s)


def expansion_1d(log_lam, L):
    """f of the L-strip expansion with vertical strips only: the L offsets'
    non-empty subsets, each the product of lambda_w over its strips per row
    of one L-column cell; f = -ln(sum) / L.  ``log_lam[w]`` = ln lambda_w."""
    terms = []
    for m in range(1, L + 1):
        for V in combinations(range(L), m):
            terms.append((1 if m % 2 == 1 else -1, sum(log_lam[w] for w in gaps(V, L))))
    return -_log_sum_signed(terms) / L


def expansion_2d(log_lam, log_gam, log_z, L):
    """f of the 2D L-strip expansion: vertical offsets V and horizontal
    offsets H of one L x L cell, not both empty, sign (-1)^{|V|+|H|+1}; see
    the module notes for the pieces.  ``log_z[w][h]`` = ln Z_wh (w columns,
    h rows); f = -ln(sum) / L^2."""
    subsets = [()] + [V for m in range(1, L + 1) for V in combinations(range(L), m)]
    terms = []
    for V in subsets:
        for H in subsets:
            if not V and not H:
                continue
            if not H:
                t = L * sum(log_lam[w] for w in gaps(V, L))
            elif not V:
                t = L * sum(log_gam[h] for h in gaps(H, L))
            else:
                t = sum(log_z[w][h] for w in gaps(V, L) for h in gaps(H, L))
            terms.append((1 if (len(V) + len(H)) % 2 == 1 else -1, t))
    return -_log_sum_signed(terms) / (L * L)


def strip_expansion(A, L, two_d=True, tol=1e-14):
    """The whole strip expansion of the uniform tensor A at width L: BP
    messages, ln lambda_k and ln gamma_k (k = 1..L), ln Z_wh (w, h = 1..L) and
    f.  Returns a dict (f, f_bp, log_lam, log_gam, log_z, msgs); log lists are
    indexed from 1 (index 0 unused)."""
    A = np.asarray(A, dtype=np.float64)
    mR, mL, mD, mU, lz_bp, _ = uniform_bp(A, tol=tol)
    msgs = (mR, mL, mD, mU)
    log_lam = [None] + [leading_log_eig(A, k, mR, mL) for k in range(1, L + 1)]
    out = {"f_bp": -lz_bp, "log_lam": log_lam, "msgs": msgs}
    if not two_d:
        out["f"] = expansion_1d(log_lam, L)
        return out
    At, mt = transpose_lattice(A, msgs)
    log_gam = [None] + [leading_log_eig(At, k, mt[0], mt[1]) for k in range(1, L + 1)]
    log_z = [None] + [[None] + patch_log_z_rows(A, w, L, msgs) for w in range(1, L + 1)]
    out.update(log_gam=log_gam, log_z=log_z, f=expansion_2d(log_lam, log_gam, log_z, L))
    return out
