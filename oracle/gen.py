"""Coset probabilities in the generator picture (Sec. 3.2), as used for the loop sector
of the 3D surface code (Sec. 5.2).  Plain numpy, FP64.

Problem.  A CSS code is decoded against one error type: qubit j flips independently with
rate p_j, the checks H (here the plaquettes) see the flips, and the stabilizer generators
of the other type (here the vertices, each flipping the qubits on its edges) span the
errors that are equivalent to no error.  The coset of an error r is r + span(generators);
with w_j(0) = 1 - p_j, w_j(1) = p_j,
    p(coset of r) = sum over s in {0,1}^{n_gen} of prod_j w_j(r_j + sum_{v at j} s_v)
(each coset element counted 2^(n_gen - rank) times when the generators are dependent; that
factor is divided out).  The two classes of a syndrome m are the cosets of r and of
r + xbar (xbar a logical of the flipped type); the class of r is its parity on the
conjugate logical zbar.

Network (Sec. 3.2, Sec. 5.2).  One copy tensor per generator (its variable s_v) and one
weight per qubit joining the generators it touches: on the generator lattice this is a
network of 2x2 weight matrices W[s, s'] = w(r + s + s') on the edges and weight vectors
w(r + s) on edges with one generator.  It is contracted like the detector network of the
point sector (Sec. 4): a PEPS over the generators of one layer t, physical leg = s_v,
swept along t.  Readings taken where the paper is silent (the same as for the detector
network in su.py where they apply):
  * Layer t: the vertical edge entering each generator (t = 0: its dangling edge below)
    acts on the physical leg as the transfer matrix above (the old variable summed);
    then the layer's in-layer edges are two-site gates diag(w(r + s_a + s_b)), in the
    colour order of su.py (horizontal bonds x even, x odd, vertical bonds y even, y odd;
    row-major inside a colour), each followed by a simple-update truncation to chi.
  * Gate = exact bond doubling with the new index k = s_a: the A side keeps only k = s_a,
    the B side takes the weight w(r + k + s_b); the SVD of the doubled bond's two-site
    matrix is the SVD of the gate-applied two-site tensor (the simple-update step).
  * After the last layer the dangling edges above weight the physical legs, which are
    summed; the 2D network is contracted by su.boundary_mps.
  * Representative: the error supported on the greedy column basis of H (columns taken in
    qubit order, a column kept when it is independent of the kept ones): the unique
    solution of H r = m with zeros off that basis.  A truncated contraction depends on
    the representative, so this fixes it.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from . import gf2
from .su import PEPS, ZeroProbability, boundary_mps, keep_count


def _weights(p):
    return np.array([1.0 - p, p])


def check_matrix(gp) -> np.ndarray:
    """H [checks x qubits] of the problem's detector picture."""
    return gp.face_dem.H_dense()


def generator_matrix(gp) -> np.ndarray:
    """[generators x qubits]: row v flips the qubits of v's edges."""
    G = np.zeros((gp.n_gen, gp.n_qubits), dtype=np.uint8)
    for j, vs in enumerate(gp.edges):
        for v in vs:
            G[v, j] ^= 1
    return G


def representative(gp, m: np.ndarray):
    """The error r supported on the greedy column basis of H with H r = m, or None if m is
    not a syndrome."""
    return gf2.solve(check_matrix(gp), np.asarray(m, dtype=np.uint8))


def class_of(gp, r: np.ndarray) -> int:
    return int(np.asarray(r, dtype=np.int64)[list(gp.zbar)].sum() % 2)


def _dependency_offset(gp) -> float:
    """ln of the factor by which the sum over s counts every coset element."""
    return (gp.n_gen - gf2.rank(generator_matrix(gp))) * np.log(2.0)


def enumerate_coset_logprob(gp, syndromes: np.ndarray) -> np.ndarray:
    """log p_{m,L} [B, 2] by summing the generator-picture formula over all 2^n_gen s."""
    assert gp.n_gen <= 20, "enumeration is for tiny problems"
    G = generator_matrix(gp)
    combos = np.zeros((1 << gp.n_gen, gp.n_qubits), dtype=np.uint8)
    for k in range(gp.n_gen):
        blk = 1 << k
        combos[blk:2 * blk] = combos[:blk] ^ G[k]
    lp1, lp0 = np.log(gp.p), np.log1p(-gp.p)
    off = _dependency_offset(gp)
    xb = np.zeros(gp.n_qubits, dtype=np.uint8)
    xb[list(gp.xbar)] = 1
    out = np.full((syndromes.shape[0], 2), -np.inf)
    for b in range(syndromes.shape[0]):
        r = representative(gp, syndromes[b])
        if r is None:
            continue
        L = class_of(gp, r)
        for c in range(2):
            xs = combos ^ (r ^ (xb if c else 0))[None, :]
            lw = np.where(xs == 1, lp1[None, :], lp0[None, :]).sum(axis=1)
            mx = lw.max()
            out[b, L ^ c] = mx + np.log(np.exp(lw - mx).sum()) - off
    return out


class GenPlan:
    """The generator lattice as layers of a PEPS (attributes as su.SUPlan's, for PEPS and
    boundary_mps)."""

    def __init__(self, gp):
        xyt = np.asarray(gp.gen_xyt)
        self.nx = int(xyt[:, 0].max()) + 1
        self.ny = int(xyt[:, 1].max()) + 1
        self.T = int(xyt[:, 2].max()) + 1
        sites = sorted({(int(x), int(y)) for x, y, _ in xyt}, key=lambda s: (s[1], s[0]))
        self.sites = sites
        self.site_of_xy = {s: k for k, s in enumerate(sites)}
        self.S = len(sites)
        self.P = [2] * self.S
        gsite = [self.site_of_xy[(int(x), int(y))] for x, y, _ in xyt]
        glayer = [int(t) for _, _, t in xyt]
        if len(set(zip(gsite, glayer))) != self.S * self.T or gp.n_gen != self.S * self.T:
            raise ValueError("every site needs exactly one generator per layer")
        T, S = self.T, self.S
        # below[t][s]: the qubit entering generator (s, t) from below (t = 0: dangling);
        # above[s]: the dangling qubit above the last layer; inlayer[t]: (site a, site b, j)
        self.below = [[None] * S for _ in range(T)]
        self.above = [None] * S
        inlayer = [[] for _ in range(T)]
        for j, vs in enumerate(gp.edges):
            if len(vs) == 1:
                s, t = gsite[vs[0]], glayer[vs[0]]
                if t == 0 and self.below[0][s] is None:
                    self.below[0][s] = j
                elif t == T - 1 and self.above[s] is None:
                    self.above[s] = j
                else:
                    raise ValueError("dangling edge inside the lattice")
                continue
            (sa, ta), (sb, tb) = (gsite[vs[0]], glayer[vs[0]]), (gsite[vs[1]], glayer[vs[1]])
            if ta == tb:
                (xa, ya), (xb, yb) = sites[sa], sites[sb]
                if abs(xa - xb) + abs(ya - yb) != 1:
                    raise ValueError("in-layer edge between non-adjacent generators")
                inlayer[ta].append((min(sa, sb), max(sa, sb), j))
            elif sa == sb and abs(ta - tb) == 1:
                t = max(ta, tb)
                if self.below[t][sa] is not None:
                    raise ValueError("two vertical edges into one generator")
                self.below[t][sa] = j
            else:
                raise ValueError("edge that is neither in-layer nor vertical")
        if any(q is None for row in self.below for q in row) or any(q is None for q in self.above):
            raise ValueError("every generator needs one edge below and the last layer one above")
        bonds = sorted({(a, b) for lay in inlayer for a, b, _ in lay})
        self.bonds = bonds
        self.bond_of = {b: i for i, b in enumerate(bonds)}
        self.site_bonds = [[] for _ in range(S)]     # ordered left, right, down, up
        for s in range(S):
            x, y = sites[s]
            for nb in ((x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)):
                o = self.site_of_xy.get(nb)
                if o is None:
                    continue
                key = (min(s, o), max(s, o))
                if key in self.bond_of:
                    self.site_bonds[s].append(self.bond_of[key])

        def colour(a, b):
            (x0, y0), (x1, y1) = sites[a], sites[b]
            if y0 == y1:
                return 0 if min(x0, x1) % 2 == 0 else 1
            return 2 if min(y0, y1) % 2 == 0 else 3
        self.gates = []
        for t in range(T):
            key = sorted((colour(a, b), sites[a][1], sites[a][0], j, self.bond_of[(a, b)]) for a, b, j in inlayer[t])
            self.gates.append([(k[4], k[3]) for k in key])    # (bond, qubit)
        self.readout = None


def _diag_gate(peps, bond, p, r, chi, cutoff, mrtol):
    """Two-site gate diag(w(r + s_a + s_b)) on `bond`, then its simple-update truncation."""
    plan = peps.plan
    A, B = plan.bonds[bond]
    w = _weights(p)
    mats, axes = [], []
    for side, s in enumerate((A, B)):
        ax = 1 + plan.site_bonds[s].index(bond)
        M = peps._env(s, bond)                             # (s_phys, ..., D, ...)
        D = M.shape[ax]
        M2 = np.zeros(M.shape[:ax + 1] + (2,) + M.shape[ax + 1:])
        for k in range(2):
            for sp in range(2):
                # A side: k = s_a (a copy); B side: weight w(r + k + s_b)
                f = (1.0 if k == sp else 0.0) if side == 0 else w[r ^ k ^ sp]
                idx = (sp,) + (slice(None),) * (ax - 1) + (slice(None), k)
                M2[idx] = f * M[sp]
        shp = list(M.shape)
        shp[ax] = 2 * D
        M2 = M2.reshape(shp)                               # doubled bond, index b*2+k
        Mm = np.moveaxis(M2, ax, -1)
        axes.append((ax, Mm.shape[:-1]))
        mats.append(Mm.reshape(-1, Mm.shape[-1]))
    lam2 = np.kron(peps.lam[bond], np.ones(2))
    QA, RA = np.linalg.qr(mats[0])
    QB, RB = np.linalg.qr(mats[1])
    theta = (RA * lam2[None, :]) @ RB.T
    U, sv, Vt = np.linalg.svd(theta)
    if sv[0] <= 0:
        raise ZeroProbability
    k = keep_count(sv, chi, cutoff, mrtol)
    newM = (QA @ U[:, :k], QB @ Vt[:k].T)
    peps.lam[bond] = sv[:k] / sv[0]
    peps.logscale += np.log(sv[0])
    for (s, (ax, rest)), M in zip(((A, axes[0]), (B, axes[1])), newM):
        peps.G[s] = np.moveaxis(M.reshape(tuple(rest) + (k,)), -1, ax)
        peps.G[s] = peps._env(s, bond, inv=True)


def _sweep_logweight(plan, gp, r, chi, chi_mps, cutoff, mrtol):
    """ln of the (truncated) contraction of the network of representative r."""
    peps = PEPS(plan)
    for t in range(plan.T):
        for s in range(plan.S):
            j = plan.below[t][s]
            w = _weights(gp.p[j])
            # V[s', s] = w(r_j + s + s'): the old variable s is summed (t = 0: s = 0,
            # the weight of the dangling edge below)
            V = np.array([[w[r[j] ^ a ^ b] for a in range(2)] for b in range(2)])
            peps.apply_local(s, V)
        for bond, j in plan.gates[t]:
            _diag_gate(peps, bond, gp.p[j], int(r[j]), chi, cutoff, mrtol)
    plan.readout = []
    for s in range(plan.S):
        j = plan.above[s]
        w = _weights(gp.p[j])
        plan.readout.append(np.array([[w[r[j] ^ ph], 0.0] for ph in range(2)]))
    F = peps.final_tensors()
    Z, ls = boundary_mps(plan, F, chi_mps, cutoff, mrtol)
    if not Z[0] > 0:
        raise ZeroProbability
    return np.log(Z[0]) + ls + peps.logscale


def gen_su_logprob(gp, syndromes: np.ndarray, chi: int, chi_mps: int, cutoff: float = 1e-12,
                   mrtol: float = 1e-8, plan: GenPlan | None = None) -> np.ndarray:
    """log p_{m,L} [B, 2] by the truncated generator-picture sweep (module docstring)."""
    plan = plan or GenPlan(gp)
    H = check_matrix(gp)
    off = _dependency_offset(gp)
    xb = np.zeros(gp.n_qubits, dtype=np.uint8)
    xb[list(gp.xbar)] = 1
    out = np.full((syndromes.shape[0], 2), -np.inf)
    for b in range(syndromes.shape[0]):
        r = gf2.solve(H, np.asarray(syndromes[b], dtype=np.uint8))
        if r is None:
            continue
        L = class_of(gp, r)
        for c in range(2):
            try:
                out[b, L ^ c] = _sweep_logweight(plan, gp, r ^ (xb if c else 0), chi, chi_mps, cutoff, mrtol) - off
            except ZeroProbability:
                pass
    return out
