"""The truncated sweep with every truncation held fixed, and its gradient (oracle; a
REJECTED reading, kept to show why).

The library's gradient is su.su_grad_total_logprob: the exact affine identity of the rates
evaluated by the decoder.  This module holds the other candidate reading, the "frozen
projector" gradient, and tests/test_oracle_grad.py shows that it is not the gradient of
P(m) even when nothing is truncated: the simple update also cuts each bond to the rank of
its two-site core, and under a change of rates the kept row spaces rotate, which a fixed
projector drops.

The rates enter the layered network of Sec. 3.4 multilinearly: every mechanism is one
weighted node (an equality node between (1 - p) and p), so with every truncation of the
sweep (Sec. 4) replaced by the fixed linear map it applied at the given rates, the
contracted P(m) is a smooth function of the rates whose derivative is the "frozen
projector" gradient of the approximate decoder.  The paper has no gradient; this module
defines it by replaying the recorded maps and takes d log P / d p_j by central differences
(step 1e-4 p_j), which is exact up to O(h^2) and rounding.

What is frozen, per step of su._one_shot:
  * local operators: the normalising divisor of each site;
  * gate on bond b between sites A < B (A is the left or lower site): with the doubled
    bond index (d, k) and the R factors and truncated SVD theta = U S V^T of the forward
    step, the site maps T_A = R_A^+ U_k, T_B = R_B^+ V_k and the bond map
        L_new = U_k^T R_A (L (x) diag(1 - p, p)) R_B^T V_k / s_1,
    where L is the bond's weight as a full matrix (diag(lambda) on the forward path);
    the site tensors become G_X <- G_X^doubled T_X (the environment weights that the
    simple update multiplies in and divides out act on other legs and cancel);
  * final contraction: the principal square root X of each bond matrix (X X = L) is
    absorbed on both sides (A side: sum_i G_A[.., i] X[i, k]; B side: sum_j X[k, j]
    G_B[.., j]), which is sqrt(lambda) on both sides on the forward path; every zip-up
    cut keeps its recorded isometry U_k and divisor, every last column its divisor.
The total P(m) = sum_L p_{m,L} is unaffected by mechanisms without detectors (they only
mix the classes), so they get gradient 0.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .su import SUPlan, PEPS, ZeroProbability, keep_count, plan_det


def _local_matrix(plan, m, s, t):
    """X^m pre[t][s] post[t-1][s]: the site-local operator of layer t (as in su._one_shot)."""
    M = plan.pre[t][s]
    if m[plan_det(plan, s, t)]:
        Pm = plan.P[s]
        M = np.eye(Pm)[np.arange(Pm) ^ 1] @ M
    if t > 0:
        M = M @ plan.post[t - 1][s]
    return M


def _range_pinv(R, rtol=1e-12):
    """Pseudo-inverse of R restricted to its singular values above rtol * the largest."""
    P, s, Wt = np.linalg.svd(R, full_matrices=False)
    keep = s > rtol * (s[0] if s.size else 0.0)
    return (Wt[keep].T / s[keep]) @ P[:, keep].T


def _double(G, ax, mask):
    """Doubled tensor along axis ax: index d * 2 + k, k = whether the gate fired."""
    G1 = G[np.arange(G.shape[0]) ^ mask]
    D2 = np.stack([G, G1], axis=ax + 1)
    shp = list(G.shape)
    shp[ax] *= 2
    return D2.reshape(shp)


def _apply_leg(G, ax, M):
    """sum_i G[.., i, ..] M[i, k] on axis ax."""
    return np.moveaxis(np.tensordot(G, M, axes=(ax, 0)), -1, ax)


class Recording:
    def __init__(self):
        self.local = []      # per layer: [S] divisors
        self.gates = []      # per layer: list of (T_A, T_B, W_A, W_B, s1)
        self.cuts = {}       # (y, x) -> (U_k, s1) or ('col', mx) or ('row',)
        self.logP = None     # forward log P(m) (total over classes)


def record(plan: SUPlan, m, chi, chi_mps, cutoff=1e-12, mrtol=1e-8) -> Recording:
    """The forward sweep of su._one_shot, recording every truncation it applies."""
    rec = Recording()
    peps = PEPS(plan)
    for t in range(plan.T):
        divs = []
        for s in range(plan.S):
            M = _local_matrix(plan, m, s, t)
            peps.G[s] = np.tensordot(M, peps.G[s], axes=(1, 0))
            mx = np.abs(peps.G[s]).max()
            if mx == 0:
                raise ZeroProbability
            peps.G[s] /= mx
            peps.logscale += np.log(mx)
            divs.append(mx)
        rec.local.append(divs)
        gl = []
        for bond, p, maskA, maskB in plan.gates[t]:
            A, B = plan.bonds[bond]
            mats, axes = [], []
            for s, mask in ((A, maskA), (B, maskB)):
                ax = 1 + plan.site_bonds[s].index(bond)
                M2 = _double(peps._env(s, bond), ax, mask)
                Mm = np.moveaxis(M2, ax, -1)
                axes.append((ax, Mm.shape[:-1]))
                mats.append(Mm.reshape(-1, Mm.shape[-1]))
            lam2 = np.kron(peps.lam[bond], np.array([1.0 - p, p]))
            QA, RA = np.linalg.qr(mats[0])
            QB, RB = np.linalg.qr(mats[1])
            theta = (RA * lam2[None, :]) @ RB.T
            U, sv, Vt = np.linalg.svd(theta)
            if sv[0] <= 0:
                raise ZeroProbability
            k = keep_count(sv, chi, cutoff, mrtol)
            Uk, Vk = U[:, :k], Vt[:k].T
            gl.append((_range_pinv(RA) @ Uk, _range_pinv(RB) @ Vk, Uk.T @ RA, Vk.T @ RB, sv[0]))
            newM = (QA @ Uk, QB @ Vk)
            peps.lam[bond] = sv[:k] / sv[0]
            peps.logscale += np.log(sv[0])
            for (s, (ax, rest)), Mx in zip(((A, axes[0]), (B, axes[1])), newM):
                peps.G[s] = np.moveaxis(Mx.reshape(rest + (k,)), -1, ax)
                peps.G[s] = peps._env(s, bond, inv=True)
        rec.gates.append(gl)
    F = peps.final_tensors()
    Z, ls = _zipup(plan, F, chi_mps, cutoff, mrtol, rec.cuts, record=True)
    rec.logP = np.log(Z.sum()) + ls + peps.logscale
    return rec


def _zipup(plan, F, chi_mps, cutoff, mrtol, cuts, record):
    """The boundary-MPS contraction of su.boundary_mps; with record=False every cut applies
    its recorded isometry and divisor instead of a new SVD."""
    nx, ny = plan.nx, plan.ny
    logscale = 0.0
    empty = np.zeros((2, 1, 1, 1, 1))
    empty[0] = 1.0
    grid = [[empty] * nx for _ in range(ny)]
    for s, (x, y) in enumerate(plan.sites):
        grid[y][x] = F[s]
    mps = [np.ones((1, 1, 1)) for _ in range(nx)]
    last = np.zeros((1, 1, 2))
    last[0, 0, 0] = 1.0
    mps[-1] = last
    for y in range(ny):
        C = np.zeros((1, 1, 1, 2))
        C[0, 0, 0, 0] = 1.0
        new = []
        for x in range(nx):
            Fx = grid[y][x]
            Ft = np.zeros((Fx.shape[1], 2, Fx.shape[2], 2, Fx.shape[3], Fx.shape[4]))
            for pl in range(2):
                for pr in range(2):
                    Ft[:, pl, :, pr] = Fx[pl ^ pr]
            T = np.einsum("jalp,adb,lprqdu->jubrq", C, mps[x], Ft, optimize=True)
            J, U, Bd, R, Q = T.shape
            if x < nx - 1 and y < ny - 1:
                Tm = T.reshape(J * U, Bd * R * Q)
                if record:
                    Um, sv, Vt = np.linalg.svd(Tm, full_matrices=False)
                    if sv[0] <= 0:
                        raise ZeroProbability
                    k = keep_count(sv, chi_mps, cutoff, mrtol)
                    cuts[(y, x)] = (Um[:, :k], sv[0])
                Uk, s1 = cuts[(y, x)]
                k = Uk.shape[1]
                new.append(Uk.reshape(J, U, k))
                C = (Uk.T @ Tm / s1).reshape(k, Bd, R, Q)
                logscale += np.log(s1)
            elif x < nx - 1:
                new.append(np.eye(J * U).reshape(J, U, J * U))
                C = T.reshape(J * U, Bd, R, Q)
            else:
                out = np.zeros((J, U, 2))
                for cb in range(Bd):
                    for q in range(2):
                        out[:, :, cb ^ q] += T[:, :, cb, 0, q]
                if record:
                    mx = np.abs(out).max()
                    if mx == 0:
                        raise ZeroProbability
                    cuts[(y, "col")] = mx
                mx = cuts[(y, "col")]
                new.append(out / mx)
                logscale += np.log(mx)
        mps = new
    v = np.ones(1)
    for x in range(nx):
        v = np.einsum("a,ab->b", v, mps[x][:, 0, :])
    return v, logscale


def _sqrtm(L):
    """Principal square root of a bond matrix (diagonal with positive entries on the
    forward path, a small perturbation of one in the replay)."""
    if L.size == 1:
        return np.sqrt(L)
    if np.count_nonzero(L - np.diag(np.diagonal(L))) == 0:
        return np.diag(np.sqrt(np.diagonal(L)))
    return np.real(scipy.linalg.sqrtm(L))


def replay(plan: SUPlan, m, rec: Recording) -> float:
    """log P(m) of the frozen program at the rates of `plan` (same structure as recorded)."""
    G = []
    for s in range(plan.S):
        g = np.zeros((plan.P[s],) + (1,) * len(plan.site_bonds[s]))
        g.flat[0] = 1.0
        G.append(g)
    L = [np.ones((1, 1)) for _ in plan.bonds]
    logscale = 0.0
    for t in range(plan.T):
        for s in range(plan.S):
            G[s] = np.tensordot(_local_matrix(plan, m, s, t), G[s], axes=(1, 0)) / rec.local[t][s]
            logscale += np.log(rec.local[t][s])
        for (bond, p, maskA, maskB), (TA, TB, WA, WB, s1) in zip(plan.gates[t], rec.gates[t]):
            A, B = plan.bonds[bond]
            for s, mask, Tx in ((A, maskA, TA), (B, maskB, TB)):
                ax = 1 + plan.site_bonds[s].index(bond)
                G[s] = _apply_leg(_double(G[s], ax, mask), ax, Tx)
            L[bond] = WA @ np.kron(L[bond], np.diag([1.0 - p, p])) @ WB.T / s1
            logscale += np.log(s1)
    # final tensors: readout, then the square root of each bond matrix on both sides
    X = [_sqrtm(Lb) for Lb in L]
    F = []
    for s in range(plan.S):
        g = G[s]
        for pos, b in enumerate(plan.site_bonds[s]):
            ax = 1 + pos
            g = _apply_leg(g, ax, X[b] if plan.bonds[b][0] == s else X[b].T)
        F.append(g)
    F = _final_layout(plan, F)
    Z, ls = _zipup(plan, F, 0, 0.0, 0.0, rec.cuts, record=False)
    return float(np.log(Z.sum()) + ls + logscale)


def _final_layout(plan, Gw):
    """Readout and (c, left, right, down, up) axes of already-weighted site tensors (the
    layout step of su.PEPS.final_tensors with the weights applied by the caller)."""
    out = []
    for s in range(plan.S):
        F = np.tensordot(plan.readout[s], Gw[s], axes=(0, 0))
        x, y = plan.sites[s]
        src = {}
        for pos, b in enumerate(plan.site_bonds[s]):
            a2, b2 = plan.bonds[b]
            other = b2 if a2 == s else a2
            ox, oy = plan.sites[other]
            d = {(x - 1, y): 0, (x + 1, y): 1, (x, y - 1): 2, (x, y + 1): 3}[(ox, oy)]
            src[d] = pos
        perm = [0] + [1 + src[d] for d in range(4) if d in src]
        F = np.transpose(F, perm)
        shape = [2] + [F.shape[1 + sorted(src).index(d)] if d in src else 1 for d in range(4)]
        out.append(F.reshape(shape))
    return out


def frozen_grad(dem, det_bits: np.ndarray, chi: int, chi_mps: int, cutoff: float = 1e-12,
                mrtol: float = 1e-8, rel_step: float = 1e-4):
    """(log P [B], d log P / d p [B, n_mech]) of the truncated sweep with frozen truncations,
    by central differences of the replay.  Tiny problems only (2 n_mech replays per shot)."""
    plan0 = SUPlan(dem)
    p0 = np.array(dem.p, dtype=np.float64)
    B = det_bits.shape[0]
    logP = np.full(B, -np.inf)
    grad = np.zeros((B, dem.n_mech))
    plans = []
    for j in range(dem.n_mech):
        h = rel_step * max(p0[j], 1e-6)
        pp, pm = p0.copy(), p0.copy()
        pp[j] += h
        pm[j] -= h
        plans.append((SUPlan(dem.with_rates(pp)), SUPlan(dem.with_rates(pm)), h))
    for b in range(B):
        try:
            rec = record(plan0, det_bits[b], chi, chi_mps, cutoff, mrtol)
        except ZeroProbability:
            continue
        logP[b] = rec.logP
        for j, (pl_p, pl_m, h) in enumerate(plans):
            grad[b, j] = (replay(pl_p, det_bits[b], rec) - replay(pl_m, det_bits[b], rec)) / (2 * h)
    return logP, grad
