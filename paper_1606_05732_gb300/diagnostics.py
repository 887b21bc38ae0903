"""Numerical checks of Theorem 1's distance bound and of its tightness (Lemma 5), run on
the device's own sketches.

Theorem 1's proof goes through the covariance M = U^T S^T S U of one row of G.S.U given
S (U: n x d with orthonormal columns).  Given S, a row of G.S.U is N(0, M), a row of
G~.U is N(0, I), and

    KL(N(0, I) || N(0, M)) = 1/2 tr(M^-1 - I) + 1/2 ln det M          (Claim 3)

so, by additivity over the m independent rows and Pinsker's inequality, the total
variation distance between the m rows of G~.U and those of G.S.U given S is at most
sqrt(m KL / 2).  E_S ||M - I||_F^2 = O(d^2 / B) (Lemma 4) makes that small once
B >> d^2 m.  Lemma 5 shows the bound is tight: for the block matrix U whose column i
holds L = ceil(sqrt(B) / d) entries 1/sqrt(L) in its own block of rows, a bucket
collision between two blocks moves ||T.U (e_i + e_j)||^2 / m away from 2 by 2/L, which
max over pairs of | ||Y (e_i + e_j)||^2 / m - 2 | detects when B <= d^2 m / (C log d).

Device work: the sketch S.U (cg_sketch_csr), T.U (cg_apply_csr), G~.U
(cg_plain_gaussian_apply) and the FP64 Gram matrices (cg_moments_f64).  Host work: the
eigenvalues of d x d matrices and the bookkeeping of the sweep.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import countgauss, synth


# ------------------------------------------------------------------------------
# Closed forms (host, FP64, d x d).
# ------------------------------------------------------------------------------
def gaussian_kl(M: np.ndarray) -> float:
    """KL(N(0, I) || N(0, M)) = 1/2 tr(M^-1 - I) + 1/2 ln det M (Claim 3), from the
    eigenvalues of the symmetric matrix M; inf when M is singular."""
    M = np.asarray(M, np.float64)
    lam = np.linalg.eigvalsh(0.5 * (M + M.T))
    if lam.min() <= 0.0:
        return math.inf
    return float(0.5 * np.sum(1.0 / lam - 1.0 + np.log(lam)))


def tv_upper_bound(kl: float, m: int) -> float:
    """Pinsker's inequality over m independent rows: TV <= sqrt(m KL / 2), capped at 1."""
    if not math.isfinite(kl):
        return 1.0
    return min(1.0, math.sqrt(0.5 * m * kl))


def frobenius_closed_form(U_row_norms_sq: np.ndarray, d: int, B: int) -> float:
    """E_S ||U^T S^T S U - I||_F^2 = (d^2 + d - 2 sum_k ||u_k||^4) / B for U with
    orthonormal columns and rows u_k (the exact form of Lemma 4's O(d^2 / B) for a
    CountSketch with independent buckets and signs)."""
    return float((d * d + d - 2.0 * np.sum(np.asarray(U_row_norms_sq, np.float64) ** 2)) / B)


# ------------------------------------------------------------------------------
# Test matrices with orthonormal columns (CSR, one nonzero per row).
# ------------------------------------------------------------------------------
def spread_orthonormal_csr(n: int, d: int) -> synth.CSR:
    """n x d, row k's one nonzero in column k mod d, value 1/sqrt(rows of that column):
    orthonormal columns with every row norm small (the easy case of Theorem 1)."""
    cols = (np.arange(n) % d).astype(np.int32)
    counts = np.bincount(cols, minlength=d).astype(np.float64)
    vals = (1.0 / np.sqrt(counts[cols])).astype(np.float32)
    return synth.CSR(n, d, np.arange(n + 1, dtype=np.int64), cols, vals)


def lemma5_block_csr(d: int, B: int) -> synth.CSR:
    """Lemma 5's matrix: column i holds L = ceil(sqrt(B) / d) entries 1/sqrt(L) in rows
    L i .. L (i + 1) - 1 (n = L d rows, orthonormal columns)."""
    L = max(1, math.ceil(math.sqrt(B) / d))
    n = L * d
    cols = (np.arange(n) // L).astype(np.int32)
    vals = np.full(n, 1.0 / math.sqrt(L), np.float32)
    return synth.CSR(n, d, np.arange(n + 1, dtype=np.int64), cols, vals)


def _dev_csr(U: synth.CSR, device):
    return (torch.from_numpy(U.row_ptr.astype(np.int32)).to(device), torch.from_numpy(U.col_idx).to(device),
            torch.from_numpy(U.vals.astype(np.float32)).to(device))


# ------------------------------------------------------------------------------
# Device-side quantities.
# ------------------------------------------------------------------------------
def sketch_gram(plan: countgauss.CountGauss, row_ptr, col_idx, vals) -> np.ndarray:
    """M = (S U)^T (S U), d x d FP64: the sketch on the device, then its FP64 Gram."""
    SX = plan.sketch_csr(row_ptr, col_idx, vals)
    gram, _ = countgauss.moments_f64(SX)
    plan.check()
    return gram.cpu().numpy()


def pair_norm_statistic(Y: torch.Tensor) -> float:
    """max over column pairs i < j of | ||Y (e_i + e_j)||^2 / m - 2 | for Y (m x d, on the
    device), from its FP64 Gram: ||Y (e_i + e_j)||^2 = G_ii + G_jj + 2 G_ij."""
    m = Y.shape[0]
    G = countgauss.moments_f64(Y)[0].cpu().numpy()
    diag = np.diag(G)
    P = diag[:, None] + diag[None, :] + 2.0 * G
    iu = np.triu_indices(G.shape[0], 1)
    return float(np.max(np.abs(P[iu] / m - 2.0))) if iu[0].size else 0.0


def kl_sweep(U: synth.CSR, m: int, Bs, seeds, device="cuda") -> list[dict]:
    """For each B: over the seeds (one CountSketch each), the FP64 M = U^T S^T S U from
    the device, its KL divergence from the identity (Claim 3), ||M - I||_F^2 against
    the closed form, and Pinsker's bound on the distance of m rows."""
    d = U.d
    rp, ci, v = _dev_csr(U, device)
    row_norms_sq = np.bincount(np.repeat(np.arange(U.n), np.diff(U.row_ptr)),
                               weights=U.vals.astype(np.float64) ** 2, minlength=U.n)
    out = []
    for B in Bs:
        kls, frob = [], []
        for s in seeds:
            plan = countgauss.CountGauss(U.n, d, m, B, s)
            M = sketch_gram(plan, rp, ci, v)
            kls.append(gaussian_kl(M))
            frob.append(float(np.sum((M - np.eye(d)) ** 2)))
        kls = np.array(kls)
        frob = np.array(frob)
        med = float(np.median(kls))
        out.append({"B": int(B), "B_over_d2m": B / (d * d * m), "samples": len(seeds),
                    "kl_mean": float(np.mean(kls)), "kl_median": med,
                    "frob2_mean": float(np.mean(frob)), "frob2_sd": float(np.std(frob)),
                    "frob2_closed_form": frobenius_closed_form(row_norms_sq, d, B),
                    "tv_bound_at_median_kl": tv_upper_bound(med, m)})
    return out


def lemma5_experiment(d: int, m: int, B: int, seeds, device="cuda") -> dict:
    """Lemma 5's distinguisher on the block matrix for B buckets: the pair-norm statistic
    of T.U (CountGauss) and of G~.U (the plain product) for every seed."""
    U = lemma5_block_csr(d, B)
    rp, ci, v = _dev_csr(U, device)
    cg, plain = [], []
    for s in seeds:
        plan = countgauss.CountGauss(U.n, d, m, B, s)
        cg.append(pair_norm_statistic(plan.apply_csr(rp, ci, v)))
        plain.append(pair_norm_statistic(plan.plain_csr(rp, ci, v)))
        plan.check()
    return {"d": d, "m": m, "B": B, "L": math.ceil(math.sqrt(B) / d), "countgauss": np.array(cg),
            "plain": np.array(plain)}
