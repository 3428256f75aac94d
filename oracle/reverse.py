"""Gradient of the truncated sweep by reverse-mode differentiation (oracle, FP64 numpy).

The sweep of su.py (Sec. 4) is run forward with every intermediate kept, then differentiated
backwards through every step, truncations included, so the result is the derivative of
su.su_logprob's total log P(m) = log sum_L p_{m,L} (Sec. 2.4) with respect to the rates.
Each step is an ordinary matrix function with a textbook adjoint:
  * a site-local operator G <- M G / mx: M-bar = G-bar G^T / mx, G-bar <- M^T G-bar / mx;
  * a gate: with M_A, M_B the doubled side matrices (other bonds' lambda absorbed) the
    simple update is the truncated SVD Theta = M_A diag(lambda (x) (1-p, p)) M_B^T = X S Y^T,
    new tensors X_k, Y_k (divided by the environment again) and lambda = S_k / s_1; the
    adjoint of a truncated SVD over the nonzero singular values s is
        A-bar = U [diag(S-bar) + (F o (U^T U-bar - U-bar^T U)) S + S (F o (V^T V-bar - V-bar^T V))] V^T
                + (I - U U^T) U-bar S^-1 V^T + U S^-1 V-bar^T (I - V V^T),  F_ij = 1 / (s_j^2 - s_i^2);
  * the zip-up cut of the final contraction keeps U_k and passes U_k^T M / s_1 on (same adjoint);
  * sqrt(lambda) absorbed on both sides of every bond in the final tensors.
Every normalising divisor (mx, s_1, the zip-up divisors) is held fixed: log P does not
depend on them (each is a gauge of the representation).  The object adjoints are mapped to
the rates through the objects' exact dependence on each rate (an object is affine in each
rate: d object / d p_j = object(p_j = 1) - object(p_j = 0), plans rebuilt).
Pins (tests/test_oracle_grad.py): the exact gradient without truncation, central
differences of su.su_logprob with truncation.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np

from .su import SUPlan, PEPS, keep_count, plan_det


def _local_matrix(plan, m, s, t):
    M = plan.pre[t][s]
    if m[plan_det(plan, s, t)]:
        Pm = plan.P[s]
        M = np.eye(Pm)[np.arange(Pm) ^ 1] @ M
    if t > 0:
        M = M @ plan.post[t - 1][s]
    return M


def _svd_adjoint(U, s, V, k, Ubar, Vbar, Sbar, rel=1e-13):
    """Adjoint of A = U diag(s) V^T w.r.t. A, for outputs U[:, :k], V[:, :k], s[:k]."""
    r = int(np.count_nonzero(s > rel * s[0]))
    Uf, Vf, sf = U[:, :r], V[:, :r], s[:r]
    m, n = U.shape[0], V.shape[0]
    Ub = np.zeros((m, r)); Vb = np.zeros((n, r)); Sb = np.zeros(r)
    if Ubar is not None: Ub[:, :k] = Ubar
    if Vbar is not None: Vb[:, :k] = Vbar
    if Sbar is not None: Sb[:k] = Sbar
    d = sf[None, :] ** 2 - sf[:, None] ** 2          # d[i, j] = s_j^2 - s_i^2
    F = np.zeros_like(d)
    nz = np.abs(d) > 1e-300
    F[nz] = 1.0 / d[nz]
    np.fill_diagonal(F, 0.0)
    J = Uf.T @ Ub
    K = Vf.T @ Vb
    inner = np.diag(Sb) + (F * (J - J.T)) * sf[None, :] + sf[:, None] * (F * (K - K.T))
    Ab = Uf @ inner @ Vf.T
    Ab += (Ub - Uf @ (Uf.T @ Ub)) @ np.diag(1 / sf) @ Vf.T
    Ab += Uf @ np.diag(1 / sf) @ (Vb - Vf @ (Vf.T @ Vb)).T
    return Ab


def _scale_axis(A, ax, w):
    shape = [1] * A.ndim
    shape[ax] = -1
    return A * w.reshape(shape)


def _sum_but(A, ax):
    return np.moveaxis(A, ax, 0).reshape(A.shape[ax], -1).sum(axis=1)


def grad_shot(plan, m, chi, chi_mps, cutoff=1e-12, mrtol=1e-8):
    """(log P, K-bar[t][s], p-bar[t][gate], R-bar[s]) of one shot: the adjoints of the site-local
    matrices K = pre[t][s] post[t-1][s], of the gates' rates and of the readouts."""
    S, T = plan.S, plan.T
    peps = PEPS(plan)
    tape_local, tape_gate = [], []
    for t in range(T):
        tl = []
        for s in range(S):
            M = _local_matrix(plan, m, s, t)
            Gin = peps.G[s]
            Gn = np.tensordot(M, Gin, axes=(1, 0))
            mx = np.abs(Gn).max()
            peps.G[s] = Gn / mx
            peps.logscale += np.log(mx)
            tl.append((M, Gin, mx))
        tape_local.append(tl)
        tg = []
        for bond, p, maskA, maskB in plan.gates[t]:
            A, B = plan.bonds[bond]
            lam_snap = [l.copy() for l in peps.lam]
            rec = {"bond": bond, "p": p, "lam": lam_snap, "sides": []}
            mats = []
            for s, mask in ((A, maskA), (B, maskB)):
                ax = 1 + plan.site_bonds[s].index(bond)
                G = peps.G[s]
                Mw = peps._env(s, bond)
                M1 = Mw[np.arange(Mw.shape[0]) ^ mask]
                M2 = np.stack([Mw, M1], axis=ax + 1)
                shp = list(Mw.shape); shp[ax] *= 2
                M2 = M2.reshape(shp)
                Mm = np.moveaxis(M2, ax, -1)
                rest = Mm.shape[:-1]
                mats.append(Mm.reshape(-1, Mm.shape[-1]))
                rec["sides"].append({"s": s, "mask": mask, "ax": ax, "G": G, "rest": rest, "shp": shp})
            lam2 = np.kron(peps.lam[bond], np.array([1.0 - p, p]))
            Th = mats[0] @ np.diag(lam2) @ mats[1].T
            U, sv, Vt = np.linalg.svd(Th)
            k = keep_count(sv, chi, cutoff, mrtol)
            rec.update({"MA": mats[0], "MB": mats[1], "lam2": lam2, "U": U, "sv": sv, "V": Vt.T, "k": k, "s1": sv[0]})
            new = (U[:, :k], Vt[:k].T)
            peps.lam[bond] = sv[:k] / sv[0]
            peps.logscale += np.log(sv[0])
            for sd, X in zip(rec["sides"], new):
                g = np.moveaxis(X.reshape(sd["rest"] + (k,)), -1, sd["ax"])
                peps.G[sd["s"]] = g
                peps.G[sd["s"]] = peps._env(sd["s"], bond, inv=True)
                sd["Gnew"] = peps.G[sd["s"]]
            tg.append(rec)
        tape_gate.append(tg)
    # final tensors
    Gfin = [g.copy() for g in peps.G]
    lamfin = [l.copy() for l in peps.lam]
    F = peps.final_tensors()
    nx, ny = plan.nx, plan.ny
    empty = np.zeros((2, 1, 1, 1, 1)); empty[0] = 1.0
    grid = [[None] * nx for _ in range(ny)]
    for s, (x, y) in enumerate(plan.sites):
        grid[y][x] = s
    def Fof(y, x):
        return F[grid[y][x]] if grid[y][x] is not None else empty
    mps = [np.ones((1, 1, 1)) for _ in range(nx)]
    last = np.zeros((1, 1, 2)); last[0, 0, 0] = 1.0
    mps[-1] = last
    rows = []
    logscale = 0.0
    for y in range(ny):
        C = np.zeros((1, 1, 1, 2)); C[0, 0, 0, 0] = 1.0
        new = []
        cols = []
        for x in range(nx):
            Fx = Fof(y, x)
            Ft = np.zeros((Fx.shape[1], 2, Fx.shape[2], 2, Fx.shape[3], Fx.shape[4]))
            for pl in range(2):
                for pr in range(2):
                    Ft[:, pl, :, pr] = Fx[pl ^ pr]
            Tt = np.einsum("jalp,adb,lprqdu->jubrq", C, mps[x], Ft, optimize=True)
            J, Uu, Bd, R, Q = Tt.shape
            col = {"C": C, "A": mps[x], "Ft": Ft, "T": Tt}
            if x < nx - 1 and y < ny - 1:
                Tm = Tt.reshape(J * Uu, Bd * R * Q)
                Um, sv, Vt = np.linalg.svd(Tm, full_matrices=False)
                k = keep_count(sv, chi_mps, cutoff, mrtol)
                col.update({"kind": "cut", "Um": Um, "sv": sv, "V": Vt.T, "k": k, "s0": sv[0]})
                new.append(Um[:, :k].reshape(J, Uu, k))
                C = (Um[:, :k].T @ Tm / sv[0]).reshape(k, Bd, R, Q)
                logscale += np.log(sv[0])
            elif x < nx - 1:
                col["kind"] = "row"
                new.append(np.eye(J * Uu).reshape(J, Uu, J * Uu))
                C = Tt.reshape(J * Uu, Bd, R, Q)
            else:
                out = np.zeros((J, Uu, 2))
                for cb in range(Bd):
                    for q in range(2):
                        out[:, :, cb ^ q] += Tt[:, :, cb, 0, q]
                mx = np.abs(out).max()
                col.update({"kind": "col", "mx": mx})
                new.append(out / mx)
                logscale += np.log(mx)
            cols.append(col)
        rows.append(cols)
        mps = new
    v = np.ones(1)
    vs = [v]
    for x in range(nx):
        v = np.einsum("a,ab->b", v, mps[x][:, 0, :])
        vs.append(v)
    Z = v
    logP = np.log(Z.sum()) + logscale + peps.logscale

    # ---------------- backward ----------------
    vbar = np.ones(2) / Z.sum()
    mpsbar = [None] * nx
    for x in range(nx - 1, -1, -1):
        Ax = mps[x][:, 0, :]
        mpsbar[x] = np.zeros_like(mps[x])
        mpsbar[x][:, 0, :] = np.outer(vs[x], vbar)
        vbar = Ax @ vbar
    Fbar = [np.zeros_like(f) for f in F]
    for y in range(ny - 1, -1, -1):
        cols = rows[y]
        Cbar = None
        inbar = [None] * nx
        for x in range(nx - 1, -1, -1):
            col = cols[x]
            Tt = col["T"]
            J, Uu, Bd, R, Q = Tt.shape
            if col["kind"] == "col":
                ob = mpsbar[x] / col["mx"]
                Tb = np.zeros_like(Tt)
                for cb in range(Bd):
                    for q in range(2):
                        Tb[:, :, cb, 0, q] += ob[:, :, cb ^ q]
            elif col["kind"] == "row":
                Tb = Cbar.reshape(Tt.shape)
            else:
                k = col["k"]
                Tm = Tt.reshape(J * Uu, -1)
                Cb = Cbar.reshape(k, -1)
                Abar = mpsbar[x].reshape(J * Uu, k) if mpsbar[x] is not None else np.zeros((J * Uu, k))
                Ubar = Abar + Tm @ Cb.T / col["s0"]
                Tmb = col["Um"][:, :k] @ Cb / col["s0"]
                Tmb = Tmb + _svd_adjoint(col["Um"], col["sv"], col["V"], k, Ubar, None, None)
                Tb = Tmb.reshape(Tt.shape)
            Cb_in = np.einsum("jubrq,adb,lprqdu->jalp", Tb, col["A"], col["Ft"], optimize=True)
            Ab_in = np.einsum("jubrq,jalp,lprqdu->adb", Tb, col["C"], col["Ft"], optimize=True)
            Ftb = np.einsum("jubrq,jalp,adb->lprqdu", Tb, col["C"], col["A"], optimize=True)
            Fxb = np.zeros((2,) + (Ftb.shape[0], Ftb.shape[2], Ftb.shape[4], Ftb.shape[5]))
            for pl in range(2):
                for pr in range(2):
                    Fxb[pl ^ pr] += Ftb[:, pl, :, pr]
            if grid[y][x] is not None:
                Fbar[grid[y][x]] += Fxb
            Cbar = Cb_in
            inbar[x] = Ab_in
        mpsbar = inbar
    # F -> G, lambda, readout
    Mbar = [[None] * S for _ in range(T)]
    Rbar = [None] * S
    lambar = [np.zeros_like(l) for l in lamfin]
    Gbar = [None] * S
    for s in range(S):
        g = Gfin[s]
        gw = g
        for pos, b in enumerate(plan.site_bonds[s]):
            gw = _scale_axis(gw, 1 + pos, np.sqrt(lamfin[b]))
        # undo the layout of final_tensors: F = transpose(tensordot(R, gw)) reshaped
        x, y = plan.sites[s]
        src = {}
        for pos, b in enumerate(plan.site_bonds[s]):
            a2, b2 = plan.bonds[b]
            other = b2 if a2 == s else a2
            ox, oy = plan.sites[other]
            d = {(x - 1, y): 0, (x + 1, y): 1, (x, y - 1): 2, (x, y + 1): 3}[(ox, oy)]
            src[d] = pos
        perm = [0] + [1 + src[d] for d in range(4) if d in src]
        Fr = np.tensordot(plan.readout[s], gw, axes=(0, 0))
        Fp = np.transpose(Fr, perm)
        Fpb = Fbar[s].reshape(Fp.shape)
        Frb = np.transpose(Fpb, np.argsort(perm))
        Rbar[s] = np.tensordot(gw, Frb, axes=(list(range(1, gw.ndim)), list(range(1, Frb.ndim))))
        gwb = np.tensordot(plan.readout[s], Frb, axes=(1, 0))
        gb = gwb
        for pos, b in enumerate(plan.site_bonds[s]):
            w = np.sqrt(lamfin[b])
            lambar[b] += _sum_but(gwb * gw, 1 + pos) / np.where(w > 0, 2 * lamfin[b], 1.0)
            gb = _scale_axis(gb, 1 + pos, w)
        Gbar[s] = gb
    pbar = [[0.0] * len(plan.gates[t]) for t in range(T)]
    for t in range(T - 1, -1, -1):
        for gi in range(len(tape_gate[t]) - 1, -1, -1):
            rec = tape_gate[t][gi]
            bond, p, k, s1 = rec["bond"], rec["p"], rec["k"], rec["s1"]
            lam_old = rec["lam"]
            Sbar = lambar[bond] / s1
            Xbars = []
            for sd in rec["sides"]:
                s = sd["s"]
                gnb = Gbar[s]
                xb = gnb
                # G_new = env^-1(X): X-bar = env^-1(G-bar); lambda-bar of env legs
                for pos, b in enumerate(plan.site_bonds[s]):
                    if b == bond:
                        continue
                    w = lam_old[b]
                    winv = np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0)
                    lambar[b] += -_sum_but(gnb * sd["Gnew"], 1 + pos) * winv
                    xb = _scale_axis(xb, 1 + pos, winv)
                Xbars.append(np.moveaxis(xb, sd["ax"], -1).reshape(-1, k))
            Thb = _svd_adjoint(rec["U"], rec["sv"], rec["V"], k, Xbars[0], Xbars[1], Sbar)
            MA, MB, lam2 = rec["MA"], rec["MB"], rec["lam2"]
            MAb = Thb @ MB @ np.diag(lam2)
            MBb = Thb.T @ MA @ np.diag(lam2)
            l2b = np.einsum("ia,ij,ja->a", MA, Thb, MB)
            D = len(lam_old[bond])
            l2b = l2b.reshape(D, 2)
            lambar[bond] = l2b[:, 0] * (1 - p) + l2b[:, 1] * p
            pbar[t][gi] = float(np.sum(lam_old[bond] * (l2b[:, 1] - l2b[:, 0])))
            for sd, Mb in zip(rec["sides"], (MAb, MBb)):
                s, ax, mask = sd["s"], sd["ax"], sd["mask"]
                M2b = np.moveaxis(Mb.reshape(sd["rest"] + (2 * D,)), -1, ax)
                shp2 = list(M2b.shape); shp2[ax] = D; shp2.insert(ax + 1, 2)
                M2b = M2b.reshape(shp2)
                Mwb0 = np.take(M2b, 0, axis=ax + 1)
                Mwb1 = np.take(M2b, 1, axis=ax + 1)
                Mwb = Mwb0 + Mwb1[np.arange(Mwb1.shape[0]) ^ mask]
                G = sd["G"]
                # Mw = env(G): lambda-bar of env legs and G-bar
                Gw = G
                for pos, b in enumerate(plan.site_bonds[s]):
                    if b == bond:
                        continue
                    Gw = _scale_axis(Gw, 1 + pos, lam_old[b])
                gb = Mwb
                for pos, b in enumerate(plan.site_bonds[s]):
                    if b == bond:
                        continue
                    w = lam_old[b]
                    lambar[b] += _sum_but(Mwb * Gw, 1 + pos) / np.where(w > 0, w, 1.0)
                    gb = _scale_axis(gb, 1 + pos, w)
                Gbar[s] = gb
        for s in range(S):
            M, Gin, mx = tape_local[t][s]
            gnb = Gbar[s]
            Mb = np.tensordot(gnb, Gin, axes=(list(range(1, Gin.ndim)), list(range(1, Gin.ndim)))) / mx
            # M = X^m K with K = pre[t][s] post[t-1][s]: K-bar = (X^m)^T M-bar
            Mbar[t][s] = Mb[np.arange(Mb.shape[0]) ^ 1] if m[plan_det(plan, s, t)] else Mb
            Gbar[s] = np.tensordot(M, gnb, axes=(0, 0)) / mx
    return logP, Mbar, pbar, Rbar


def object_jacobian(dem):
    """Per mechanism j: [(kind, index, d object)] with kind "K" (index (t, s)), "p" (index
    (t, gate)) or "R" (index s), from plans rebuilt with p_j = 0 and p_j = 1."""
    p0 = np.array(dem.p, dtype=np.float64)
    base = SUPlan(dem)
    out = []
    for j in range(dem.n_mech):
        plans = []
        for x in (0.0, 1.0):
            pj = p0.copy()
            pj[j] = x
            plans.append(SUPlan(dem.with_rates(pj)))
        a, b = plans
        ent = []
        for t in range(base.T):
            for s in range(base.S):
                Ka = a.pre[t][s] @ a.post[t - 1][s] if t > 0 else a.pre[t][s]
                Kb = b.pre[t][s] @ b.post[t - 1][s] if t > 0 else b.pre[t][s]
                if not np.array_equal(Ka, Kb):
                    ent.append(("K", (t, s), Kb - Ka))
            for gi, (ga, gb) in enumerate(zip(a.gates[t], b.gates[t])):
                if ga[1] != gb[1]:
                    ent.append(("p", (t, gi), gb[1] - ga[1]))
        for s in range(base.S):
            if not np.array_equal(a.readout[s], b.readout[s]):
                ent.append(("R", s, b.readout[s] - a.readout[s]))
        out.append(ent)
    return out


def reverse_grad_total_logprob(dem, det_bits: np.ndarray, chi: int, chi_mps: int, cutoff: float = 1e-12,
                               mrtol: float = 1e-8, jac=None):
    """(log P [B], d log P / d p [B, n_mech]) of su's truncated sweep by the reverse sweep."""
    plan = SUPlan(dem)
    jac = jac if jac is not None else object_jacobian(dem)
    B = det_bits.shape[0]
    lp = np.full(B, -np.inf)
    g = np.zeros((B, dem.n_mech))
    for b in range(B):
        logP, Kbar, pbar, Rbar = grad_shot(plan, det_bits[b], chi, chi_mps, cutoff, mrtol)
        lp[b] = logP
        for j, ent in enumerate(jac):
            acc = 0.0
            for kind, idx, d in ent:
                if kind == "K":
                    acc += np.sum(Kbar[idx[0]][idx[1]] * d)
                elif kind == "p":
                    acc += pbar[idx[0]][idx[1]] * d
                else:
                    acc += np.sum(Rbar[idx] * d)
            g[b, j] = acc
    return lp, g
