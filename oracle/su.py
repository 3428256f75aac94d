"""Approximate coset probabilities by the boundary sweep of Sec. 4 (plain numpy, FP64).

The layered detector network (Sec. 3.1 for a DEM, Sec. 3.4) is contracted by sweeping a
2D tensor network (a PEPS over the sites of one layer) from the first layer to the last
(Sec. 4), absorbing one layer at a time as a sequence of two-site gates and truncating
each gate's bond to chi with the simple update: the environment of the two sites is
approximated by the diagonal bond weights lambda of their other bonds, and the bond is
cut by a truncated SVD (Sec. 4; simple-update steps as in the reference the paper cites
for it).  The remaining 2D network is contracted by an MPS sweep with bond chi_mps
(Sec. 4, and chi_MPS of Sec. 5).

Readings taken where the paper is silent:
  * Boundary state: PEPS amplitude psi(sigma) over sigma_s = the bit of the vertical
    (inter-layer) mechanism entering site s of the current layer; starts at sigma = 0.
  * A layer: detector flips and single-detector mechanisms act on one site; vertical
    mechanisms weight the outgoing bit after the layer's gates; a two-detector mechanism
    inside the layer is the gate (1-p) I x I + p X x X on a grid bond (the natural split
    of Sec. 5.1, where the =_p node between two + nodes becomes a two-site gate).
  * Gate = exact bond doubling (new bond index (b, k), k = whether the mechanism fired),
    then truncation of that bond.  The SVD of the doubled bond's two-site matrix is the
    SVD of the gate-applied two-site tensor, so this is the simple-update step.
  * Class tracking without signed tensors: instead of the Hadamard trick of Sec. 3.1.2
    (whose minority class is a difference of two nearly equal contractions), each site
    hosting a class-flipping mechanism carries a class counter bit on its physical leg.
    Single-detector mechanisms of the last layer are read out at the end; their class
    flip is the readout bit itself and needs no counter.  The observable may be replaced
    by l + (sum of all rows of H) -- the single-detector mechanisms -- with the class
    offset by the parity of all detector bits, when that needs fewer counters.
  * Gate order in a layer: bonds (x,y)-(x+1,y) with x even, then x odd, then bonds
    (x,y)-(x,y+1) with y even, then y odd; row-major inside a colour (bonds of one colour
    are disjoint, so their order does not matter).
  * Truncation: keep s_i > cutoff * s_1, at most chi; if the cut falls inside a
    multiplet (s_k - s_{k+1} <= mrtol * s_1), drop the whole multiplet.  lambda = s / s_1
    and ln s_1 goes to the log-scale.
  * A class whose truncated weight comes out <= 0 gets log p = -inf.
  * Final contraction: every site's physical leg is read out into (class bit c_s), sqrt
    of each lambda is absorbed on both sides, rows are absorbed into a boundary MPS by
    zip-up (SVD truncation to chi_mps column by column), the class parity flows along
    each row into a two-valued output leg on the last MPS tensor; the last row is
    contracted exactly.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from .exact import _parity_weights


class SUPlan:
    """The layered network of a graph-like DEM, built from the detector coordinates."""

    def __init__(self, dem, merge: bool = True, deform: bool | None = None):
        assert dem.n_obs == 1, "the sweep reference handles one observable"
        xyt = dem.det_xyt
        self.nx = int(xyt[:, 0].max()) + 1
        self.ny = int(xyt[:, 1].max()) + 1
        self.T = int(xyt[:, 2].max()) + 1
        sites = sorted({(int(x), int(y)) for x, y, _ in xyt}, key=lambda s: (s[1], s[0]))
        self.sites = sites
        self.site_of_xy = {s: k for k, s in enumerate(sites)}
        self.S = len(sites)
        self.det_site = np.array([self.site_of_xy[(int(x), int(y))] for x, y, _ in xyt])
        self.det_layer = xyt[:, 2].astype(int)
        if len(set(zip(self.det_site.tolist(), self.det_layer.tolist()))) != self.S * self.T \
                or dem.n_det != self.S * self.T:
            raise ValueError("every site needs exactly one detector per layer")

        # merge mechanisms with identical detectors and identical class effect (Sec. 2.4)
        mechs = {}
        order = []
        for j in range(dem.n_mech):
            key = (tuple(sorted(dem.mech_dets[j])), tuple(sorted(dem.mech_obs[j])))
            if merge and key in mechs:
                q = mechs[key]
                mechs[key] = q + dem.p[j] - 2 * q * dem.p[j]
            else:
                mechs[key] = float(dem.p[j])
                order.append(key)
        self.mechs = [(k[0], 1 if k[1] else 0, mechs[k]) for k in order]   # (dets, l, p)

        # classify
        kinds = []
        for dets, l, p in self.mechs:
            if len(dets) == 0:
                kinds.append(("global",))
                continue
            ts = [int(self.det_layer[i]) for i in dets]
            ss = [int(self.det_site[i]) for i in dets]
            if len(dets) == 1:
                kinds.append(("single", ss[0], ts[0]))
            elif len(dets) == 2 and ts[0] == ts[1]:
                (x0, y0), (x1, y1) = sites[ss[0]], sites[ss[1]]
                if abs(x0 - x1) + abs(y0 - y1) != 1:
                    raise ValueError("two-detector mechanism between non-adjacent sites")
                kinds.append(("pair", min(ss), max(ss), ts[0]))
            elif len(dets) == 2 and ss[0] == ss[1] and abs(ts[0] - ts[1]) == 1:
                kinds.append(("vert", ss[0], min(ts)))
            else:
                raise ValueError("mechanism is neither in-layer nor vertical")
        self.kinds = kinds

        # choose the observable representative with fewer counters
        single_ind = [k[0] == "single" for k in kinds]
        l0 = [l for _, l, _ in self.mechs]
        l1 = [l ^ int(si) for l, si in zip(l0, single_ind)]
        c0, c1 = self._counters(l0), self._counters(l1)
        if deform if deform is not None else len(c1) < len(c0):
            self.lvec, self.counter_sites, self.offset_all = l1, c1, True
        else:
            self.lvec, self.counter_sites, self.offset_all = l0, c0, False
        self.P = [4 if s in self.counter_sites else 2 for s in range(self.S)]

        # bonds: grid-adjacent site pairs that host at least one gate
        bonds = sorted({(k[1], k[2]) for k in kinds if k[0] == "pair"})
        self.bonds = bonds
        self.bond_of = {b: i for i, b in enumerate(bonds)}
        self.site_bonds = [[] for _ in range(self.S)]     # ordered left, right, down, up
        for s in range(self.S):
            x, y = sites[s]
            for nb in ((x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)):
                t = self.site_of_xy.get(nb)
                if t is None:
                    continue
                key = (min(s, t), max(s, t))
                if key in self.bond_of:
                    self.site_bonds[s].append(self.bond_of[key])

        # per-layer operations
        T, S = self.T, self.S
        self.pre = [[np.eye(self.P[s]) for s in range(S)] for _ in range(T)]
        self.post = [[None] * S for _ in range(T)]
        self.gates = [[] for _ in range(T)]
        vert_groups = [[[] for _ in range(S)] for _ in range(T)]
        read_groups = [[] for _ in range(S)]
        gl = []
        for idx, ((dets, _, p), kind) in enumerate(zip(self.mechs, kinds)):
            l = self.lvec[idx]
            if kind[0] == "global":
                gl.append((l, p))
            elif kind[0] == "single":
                s, t = kind[1], kind[2]
                if t == T - 1:
                    read_groups[s].append((l, idx))
                else:
                    mask = 1 | (2 if l else 0)
                    Pm = self.P[s]
                    X = np.eye(Pm)[np.arange(Pm) ^ mask]
                    self.pre[t][s] = ((1 - p) * np.eye(Pm) + p * X) @ self.pre[t][s]
            elif kind[0] == "pair":
                a, b, t = kind[1], kind[2], kind[3]
                self.gates[t].append((self._colour(a, b), sites[a][1], sites[a][0], idx,
                                      self.bond_of[(a, b)], p, 1 | (2 if l else 0), 1))
            else:
                s, t = kind[1], kind[2]
                vert_groups[t][s].append((l, idx))
        for t in range(T):
            self.gates[t] = [g[4:] for g in sorted(self.gates[t])]
        pvec = np.array([m[2] for m in self.mechs])
        for t in range(T - 1):
            for s in range(S):
                W = _parity_weights(vert_groups[t][s], pvec, 2)   # W[tau, dc]
                self.post[t][s] = self._phys_from_W(W, s)
        self.readout = []
        for s in range(S):
            W = _parity_weights(read_groups[s], pvec, 2)
            Pm = self.P[s]
            R = np.zeros((Pm, 2))
            for ph in range(Pm):
                tau, cl = ph & 1, ph >> 1
                for c in range(2):
                    R[ph, c] = W[tau, c ^ cl]
            self.readout.append(R)
        self.glob = gl

    def _counters(self, lvec):
        cs = set()
        for l, kind in zip(lvec, self.kinds):
            if not l:
                continue
            if kind[0] == "pair":
                cs.add(kind[1])
            elif kind[0] == "single" and kind[2] != self.T - 1:
                cs.add(kind[1])
            elif kind[0] == "vert":
                cs.add(kind[1])
        return cs

    def _phys_from_W(self, W, s):
        Pm = self.P[s]
        M = np.zeros((Pm, Pm))
        for ph in range(Pm):
            tau, cl = ph & 1, ph >> 1
            for dc in range(2):
                if W[tau, dc] == 0:
                    continue
                if Pm == 2 and dc:
                    raise ValueError("class-flipping vertical mechanism on a site without counter")
                M[tau | ((cl ^ dc) << 1), ph] += W[tau, dc]
        return M

    def _colour(self, a, b):
        (x0, y0), (x1, y1) = self.sites[a], self.sites[b]
        if y0 == y1:
            return 0 if min(x0, x1) % 2 == 0 else 1
        return 2 if min(y0, y1) % 2 == 0 else 3


def keep_count(s: np.ndarray, chi: int, cutoff: float, mrtol: float) -> int:
    """Number of singular values kept (s sorted descending, s[0] > 0)."""
    r = int(np.count_nonzero(s > cutoff * s[0]))
    k = min(chi, r)
    if k < r:
        kk = k
        while kk > 0 and s[kk - 1] - s[kk] <= mrtol * s[0]:
            kk -= 1
        if kk > 0:
            k = kk
    return k


class ZeroProbability(Exception):
    pass


def discarded_fraction(sv: np.ndarray, k: int) -> float:
    """Weight a truncation to k singular values drops: sum_{i >= k} s_i^2 / sum_i s_i^2 (the
    squared Frobenius error of the truncated matrix relative to its squared norm)."""
    s2 = np.asarray(sv, dtype=np.float64) ** 2
    tot = s2.sum()
    return float(s2[k:].sum() / tot) if tot > 0 else 0.0


def _scale_axis(A, ax, w):
    shape = [1] * A.ndim
    shape[ax] = -1
    return A * w.reshape(shape)


class PEPS:
    def __init__(self, plan: SUPlan):
        self.plan = plan
        self.G = []
        for s in range(plan.S):
            g = np.zeros((plan.P[s],) + (1,) * len(plan.site_bonds[s]))
            g.flat[0] = 1.0
            self.G.append(g)
        self.lam = [np.ones(1) for _ in plan.bonds]
        self.logscale = 0.0
        self.trunc = []          # discarded fraction of every simple-update truncation

    def apply_local(self, s, M):
        self.G[s] = np.tensordot(M, self.G[s], axes=(1, 0))
        mx = np.abs(self.G[s]).max()
        if mx == 0:
            raise ZeroProbability
        self.G[s] /= mx
        self.logscale += np.log(mx)

    def _env(self, s, skip, inv=False):
        g = self.G[s]
        for pos, b in enumerate(self.plan.site_bonds[s]):
            if b == skip:
                continue
            w = self.lam[b]
            if inv:
                w = np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0)
            g = _scale_axis(g, 1 + pos, w)
        return g

    def gate(self, bond, p, maskA, maskB, chi, cutoff, mrtol):
        plan = self.plan
        A, B = plan.bonds[bond]
        axes = []
        mats = []
        for s, mask in ((A, maskA), (B, maskB)):
            ax = 1 + plan.site_bonds[s].index(bond)
            M = self._env(s, bond)
            M1 = M[np.arange(M.shape[0]) ^ mask]
            M2 = np.stack([M, M1], axis=ax + 1)                # (..., D, 2, ...)
            shp = list(M.shape)
            shp[ax] *= 2
            M2 = M2.reshape(shp)                                # doubled bond, index b*2+k
            Mm = np.moveaxis(M2, ax, -1)
            rest = Mm.shape[:-1]
            axes.append((ax, rest))
            mats.append(Mm.reshape(-1, Mm.shape[-1]))
        lam2 = np.kron(self.lam[bond], np.array([1.0 - p, p]))
        QA, RA = np.linalg.qr(mats[0])
        QB, RB = np.linalg.qr(mats[1])
        theta = (RA * lam2[None, :]) @ RB.T
        U, sv, Vt = np.linalg.svd(theta)
        if sv[0] <= 0:
            raise ZeroProbability
        k = keep_count(sv, chi, cutoff, mrtol)
        self.trunc.append(discarded_fraction(sv, k))
        newM = (QA @ U[:, :k], QB @ Vt[:k].T)
        self.lam[bond] = sv[:k] / sv[0]
        self.logscale += np.log(sv[0])
        for (s, (ax, rest)), M in zip(((A, axes[0]), (B, axes[1])), newM):
            g = np.moveaxis(M.reshape(rest + (k,)), -1, ax)
            self.G[s] = g
            self.G[s] = self._env(s, bond, inv=True)

    def final_tensors(self):
        """F[s] with axes (c, left, right, down, up) (absent bonds have dimension 1)."""
        plan = self.plan
        out = []
        for s in range(plan.S):
            g = self.G[s]
            for pos, b in enumerate(plan.site_bonds[s]):
                g = _scale_axis(g, 1 + pos, np.sqrt(self.lam[b]))
            F = np.tensordot(plan.readout[s], g, axes=(0, 0))    # (c, bonds...)
            x, y = plan.sites[s]
            dims = []
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


def boundary_mps(plan: SUPlan, F, chi_mps: int, cutoff: float, mrtol: float, trunc: list | None = None):
    """Zip-up boundary-MPS contraction of the final 2D network with a class-parity leg.

    Returns (Z[2], logscale): Z[c] * exp(logscale) = sum over readouts with total class c.
    """
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
            Fx = grid[y][x]                                     # (c, l, r, d, u)
            Ft = np.zeros((Fx.shape[1], 2, Fx.shape[2], 2, Fx.shape[3], Fx.shape[4]))
            for pl in range(2):
                for pr in range(2):
                    Ft[:, pl, :, pr] = Fx[pl ^ pr]
            T = np.einsum("jalp,adb,lprqdu->jubrq", C, mps[x], Ft, optimize=True)
            J, U, Bd, R, Q = T.shape
            if x < nx - 1:
                if y < ny - 1:
                    Um, sv, Vt = np.linalg.svd(T.reshape(J * U, Bd * R * Q), full_matrices=False)
                    if sv[0] <= 0:
                        raise ZeroProbability
                    k = keep_count(sv, chi_mps, cutoff, mrtol)
                    if trunc is not None:
                        trunc.append(discarded_fraction(sv, k))
                    new.append(Um[:, :k].reshape(J, U, k))
                    C = ((sv[:k] / sv[0])[:, None] * Vt[:k]).reshape(k, Bd, R, Q)
                    logscale += np.log(sv[0])
                else:
                    # last row: contract exactly (vertical legs are trivial)
                    new.append(np.eye(J * U).reshape(J, U, J * U))
                    C = T.reshape(J * U, Bd, R, Q)
            else:
                out = np.zeros((J, U, 2))
                for cb in range(Bd):
                    for q in range(2):
                        out[:, :, cb ^ q] += T[:, :, cb, 0, q]
                mx = np.abs(out).max()
                if mx == 0:
                    raise ZeroProbability
                new.append(out / mx)
                logscale += np.log(mx)
        mps = new
    v = np.ones(1)
    for x in range(nx):
        v = np.einsum("a,ab->b", v, mps[x][:, 0, :])
    return v, logscale


def su_logprob(dem, det_bits: np.ndarray, chi: int, chi_mps: int, cutoff: float = 1e-12,
               mrtol: float = 1e-8, plan: SUPlan | None = None) -> np.ndarray:
    """log p_{m,L} [B, 2] by the truncated sweep (see module docstring)."""
    plan = plan or SUPlan(dem)
    out = np.full((det_bits.shape[0], 2), -np.inf)
    for b in range(det_bits.shape[0]):
        try:
            out[b] = _one_shot(plan, det_bits[b], chi, chi_mps, cutoff, mrtol)
        except ZeroProbability:
            pass
    return out


def _one_shot(plan, m, chi, chi_mps, cutoff, mrtol, stats=None):
    peps = PEPS(plan)
    for t in range(plan.T):
        for s in range(plan.S):
            # post-layer weights of layer t-1, then this layer's single-site mechanisms and
            # the detector flip of site s (all act on the physical leg only)
            M = plan.pre[t][s]
            if m[plan_det(plan, s, t)]:
                Pm = plan.P[s]
                M = np.eye(Pm)[np.arange(Pm) ^ 1] @ M
            if t > 0:
                M = M @ plan.post[t - 1][s]
            peps.apply_local(s, M)
        for bond, p, ma, mb in plan.gates[t]:
            peps.gate(bond, p, ma, mb, chi, cutoff, mrtol)
    F = peps.final_tensors()
    cuts = []
    Z, ls = boundary_mps(plan, F, chi_mps, cutoff, mrtol, cuts)
    if stats is not None:
        su_t = peps.trunc or [0.0]
        mps_t = cuts or [0.0]
        stats[:] = [max(su_t), sum(su_t), max(mps_t), sum(mps_t)]
    for l, p in plan.glob:
        if l:
            Z = np.array([(1 - p) * Z[0] + p * Z[1], (1 - p) * Z[1] + p * Z[0]])
    off = int(np.bitwise_xor.reduce(m.astype(np.int64))) if plan.offset_all else 0
    # a class whose contracted weight is not positive (possible only through truncation
    # error, the exact weight is a sum of probabilities) is reported as log 0 = -inf
    with np.errstate(divide="ignore"):
        logZ = np.log(np.where(Z > 0, Z, 0.0)) + ls + peps.logscale
    return np.array([logZ[0 ^ off], logZ[1 ^ off]])


def su_truncation_stats(dem, det_bits: np.ndarray, chi: int, chi_mps: int, cutoff: float = 1e-12,
                        mrtol: float = 1e-8, plan: SUPlan | None = None) -> np.ndarray:
    """Per shot [B, 4]: the largest and the summed discarded fraction (discarded_fraction) of
    the simple-update truncations, then of the zip-up cuts, of the sweep of su_logprob.  Shots
    whose sweep meets a zero probability before its end keep what was recorded (zeros)."""
    plan = plan or SUPlan(dem)
    out = np.zeros((det_bits.shape[0], 4))
    for b in range(det_bits.shape[0]):
        st = [0.0] * 4
        try:
            _one_shot(plan, det_bits[b], chi, chi_mps, cutoff, mrtol, st)
        except ZeroProbability:
            pass
        out[b] = st
    return out


def plan_det(plan, s, t):
    if not hasattr(plan, "_det_at"):
        d = {}
        for i, (ss, tt) in enumerate(zip(plan.det_site.tolist(), plan.det_layer.tolist())):
            d[(ss, tt)] = i
        plan._det_at = d
    return plan._det_at[(s, t)]


def su_grad_total_logprob(dem, det_bits: np.ndarray, chi: int, chi_mps: int, cutoff: float = 1e-12,
                          mrtol: float = 1e-8):
    """(log P [B], d log P / d p [B, n_mech]) of the truncated sweep, P(m) = sum_L p_{m,L}.

    The contraction of Sec. 2.4 / Sec. 3.4 is affine in every rate p_j (mechanism j is one
    weighted node): P = (1 - p_j) P_{x_j=0} + p_j P_{x_j=1}, so
        d log P / d p_j = (P_{x_j=1} - P_{x_j=0}) / P,
    with P_{x_j=b} the network with mechanism j forced to b (rate set to b).  Each of the
    three values is the truncated sweep of this module at the same chi; without truncation
    this is the exact gradient of exact.grad_total_logprob.  Mechanisms without detectors
    only mix the classes and get 0.
    """
    def total(d):
        lp = su_logprob(d, det_bits, chi, chi_mps, cutoff, mrtol)
        with np.errstate(invalid="ignore"):
            return np.logaddexp(lp[:, 0], lp[:, 1])
    base = total(dem)
    grad = np.zeros((det_bits.shape[0], dem.n_mech))
    p0 = np.array(dem.p, dtype=np.float64)
    for j in range(dem.n_mech):
        pj = p0.copy()
        pj[j] = 1.0
        l1 = total(dem.with_rates(pj))
        pj[j] = 0.0
        l0 = total(dem.with_rates(pj))
        with np.errstate(invalid="ignore"):
            grad[:, j] = np.exp(l1 - base) - np.exp(l0 - base)
    return base, grad
