"""Exact coset probabilities p_{m,L} of a detector error model (Sec. 2.4).

p_{m,L} = sum over x in F_2^n with H x = m and l . x = L of prod_j p_j^{x_j} (1-p_j)^{1-x_j}.
Three independent evaluations, used to pin one another:
  brute_force_table -- the definition, summed over all 2^n patterns (n <= ~22);
  generator_sum     -- Sec. 3.2: fix one representative r with H r = m, l . r = L and sum
                       P over r + span(g_i), g_i a basis of {x : H x = 0, l . x = 0};
  transfer_matrix   -- untruncated layer-by-layer contraction of the detector network
                       (the sweep of Sec. 4 with no truncation): the state is indexed by
                       the bits of the inter-layer mechanisms entering the next layer and
                       the running class.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from . import gf2


def _masks(dem):
    dm = np.zeros(dem.n_mech, dtype=np.uint64)
    om = np.zeros(dem.n_mech, dtype=np.uint64)
    for j in range(dem.n_mech):
        for i in dem.mech_dets[j]:
            dm[j] ^= np.uint64(1) << np.uint64(i)
        for o in dem.mech_obs[j]:
            om[j] ^= np.uint64(1) << np.uint64(o)
    return dm, om


def brute_force_table(dem) -> np.ndarray:
    """Table P[m, L] over every detector outcome m (bit i of the index = detector i) and
    class L, by summing the probability of every error pattern (Sec. 2.4 definition)."""
    n = dem.n_mech
    assert n <= 24 and dem.n_det <= 22, "brute force is for tiny problems"
    dm, om = _masks(dem)
    logp1 = np.log(np.asarray(dem.p))
    logp0 = np.log1p(-np.asarray(dem.p))
    table = np.zeros((1 << dem.n_det, 1 << dem.n_obs), dtype=np.float64)
    chunk = 1 << min(n, 20)
    for start in range(0, 1 << n, chunk):
        X = np.arange(start, start + chunk, dtype=np.uint64)
        synd = np.zeros(chunk, dtype=np.uint64)
        cls = np.zeros(chunk, dtype=np.uint64)
        lw = np.zeros(chunk, dtype=np.float64)
        for j in range(n):
            bit = (X >> np.uint64(j)) & np.uint64(1)
            synd ^= bit * dm[j]
            cls ^= bit * om[j]
            lw += np.where(bit == 1, logp1[j], logp0[j])
        np.add.at(table, (synd.astype(np.int64), cls.astype(np.int64)), np.exp(lw))
    return table


def det_index(det_bits: np.ndarray) -> np.ndarray:
    """Pack detector bits [B, n_det] into the integer index used by brute_force_table."""
    w = (np.uint64(1) << np.arange(det_bits.shape[1], dtype=np.uint64))
    return (det_bits.astype(np.uint64) * w[None, :]).sum(axis=1).astype(np.int64)


def generator_sum(dem, det_bits: np.ndarray) -> np.ndarray:
    """log p_{m,L} [B, 2^n_obs] by the generator picture of Sec. 3.2.

    The trivial errors {x : H x = 0, l . x = 0} play the role of the stabilizer group;
    the coset of class L is r_{m,L} + span of their basis.
    """
    H = dem.H_dense()
    L = dem.L_dense()
    HL = np.concatenate([H, L], axis=0)
    G = gf2.kernel(HL)                     # trivial-error basis, rows
    r = G.shape[0]
    assert r <= 22, "generator sum is for tiny problems"
    logp1 = np.log(np.asarray(dem.p))
    logp0 = np.log1p(-np.asarray(dem.p))
    # all 2^r combinations of the basis
    combos = np.zeros((1 << r, dem.n_mech), dtype=np.uint8)
    for k in range(r):
        blk = 1 << k
        combos[blk:2 * blk] = combos[:blk] ^ G[k]
    C = 1 << dem.n_obs
    out = np.full((det_bits.shape[0], C), -np.inf)
    for b in range(det_bits.shape[0]):
        for c in range(C):
            target = np.concatenate([det_bits[b].astype(np.uint8),
                                     np.array([(c >> o) & 1 for o in range(dem.n_obs)], dtype=np.uint8)])
            rep = gf2.solve(HL, target)
            if rep is None:
                continue
            xs = combos ^ rep[None, :]
            lw = np.where(xs == 1, logp1[None, :], logp0[None, :]).sum(axis=1)
            mx = lw.max()
            out[b, c] = mx + np.log(np.exp(lw - mx).sum())
    return out


class Layering:
    """Classification of mechanisms by the detector layout, for the exact sweep.

    Sites are the distinct (x, y) of the detectors; every site must hold one detector in
    every layer t.  A mechanism is 'in-layer' when all its detectors share a layer (it
    flips the bits of their sites), 'vertical' when it joins the same site in layers t and
    t+1, and 'global' when it flips no detector.
    """

    def __init__(self, dem):
        xyt = dem.det_xyt
        nt = int(xyt[:, 2].max()) + 1
        sites = sorted({(int(x), int(y)) for x, y, _ in xyt})
        self.sites = sites
        sidx = {s: k for k, s in enumerate(sites)}
        self.S, self.T = len(sites), nt
        self.det_site = np.array([sidx[(int(x), int(y))] for x, y, _ in xyt])
        self.det_layer = xyt[:, 2].astype(int)
        seen = set(zip(self.det_site.tolist(), self.det_layer.tolist()))
        if len(seen) != dem.n_det or len(seen) != self.S * self.T:
            raise ValueError("every site needs exactly one detector per layer")
        self.inlayer = [[] for _ in range(nt)]     # (site mask, obs mask, j)
        self.vertical = [[] for _ in range(nt)]    # (site, obs mask, j): between t and t+1
        self.glob = []                             # (obs mask, j)
        for j, ds in enumerate(dem.mech_dets):
            om = 0
            for o in dem.mech_obs[j]:
                om ^= 1 << o
            if len(ds) == 0:
                self.glob.append((om, j))
                continue
            ts = {int(self.det_layer[i]) for i in ds}
            ss = [int(self.det_site[i]) for i in ds]
            if len(ts) == 1:
                m = 0
                for s in ss:
                    m ^= 1 << s
                self.inlayer[ts.pop()].append((m, om, j))
            elif len(ds) == 2 and ss[0] == ss[1] and abs(int(self.det_layer[ds[0]]) - int(self.det_layer[ds[1]])) == 1:
                t = min(int(self.det_layer[i]) for i in ds)
                self.vertical[t].append((ss[0], om, j))
            else:
                raise ValueError(f"mechanism {j} is not in-layer or vertical")


def _flip_perm(S, mask):
    return np.arange(1 << S, dtype=np.int64) ^ mask


def transfer_matrix(dem, det_bits: np.ndarray, layering: Layering | None = None,
                    return_states: bool = False):
    """log p_{m,L} [B, 2^n_obs] by exact layer-by-layer contraction.

    State psi[b, sigma, c]: sigma = bits of the vertical mechanisms entering the current
    layer (bit s = site s), c = class so far.  Layer t: flip sigma by the detector bits
    m(., t); apply every in-layer mechanism as psi <- (1-p) psi + p psi(sigma ^ mask,
    c ^ obs); the bits now required of the vertical mechanisms above are sigma (detector
    (s, t) has even total parity with m folded in); weight them by the probability that the
    vertical mechanisms at s have parity sigma_s (projection on sigma_s = 0 where there are
    none, in particular above the last layer).  p_{m,L} = psi[0, L] at the end.
    """
    lay = layering or Layering(dem)
    S, T = lay.S, lay.T
    assert S <= 26
    B = det_bits.shape[0]
    C = 1 << dem.n_obs
    N = 1 << S
    p = np.asarray(dem.p, dtype=np.float64)
    psi = np.zeros((B, N, C))
    psi[:, 0, 0] = 1.0
    logscale = np.zeros(B)
    ar = np.arange(N, dtype=np.int64)
    carr = np.arange(C, dtype=np.int64)
    states = []
    for t in range(T):
        # detector flips of layer t
        f = np.zeros(B, dtype=np.int64)
        for i in np.nonzero(lay.det_layer == t)[0]:
            f ^= det_bits[:, i].astype(np.int64) << int(lay.det_site[i])
        psi = np.take_along_axis(psi, (ar[None, :] ^ f[:, None])[:, :, None].repeat(C, axis=2), axis=1)
        for m, om, j in lay.inlayer[t]:
            psi = (1 - p[j]) * psi + p[j] * psi[:, ar ^ m][:, :, carr ^ om]
        # vertical mechanisms above layer t, grouped by site
        by_site = {}
        for s, om, j in lay.vertical[t]:
            by_site.setdefault(s, []).append((om, j))
        for s in range(S):
            group = by_site.get(s, [])
            W = _parity_weights(group, p, C)          # W[tau, dc]
            bit = (ar >> s) & 1
            new = np.zeros_like(psi)
            for dc in range(C):
                w = W[bit, dc]                         # [N]
                if not np.any(w):
                    continue
                new += w[None, :, None] * psi[:, :, carr ^ dc]
            psi = new
        if return_states:
            states.append(psi.copy())
        mx = np.abs(psi).reshape(B, -1).max(axis=1)
        mx = np.where(mx > 0, mx, 1.0)
        psi /= mx[:, None, None]
        logscale += np.log(mx)
    for om, j in lay.glob:
        psi = (1 - p[j]) * psi + p[j] * psi[:, :, carr ^ om]
    with np.errstate(divide="ignore"):
        out = np.log(psi[:, 0, :]) + logscale[:, None]
    return (out, states) if return_states else out


def _parity_weights(group, p, C):
    """W[tau, dc] = P(parity of the group's bits = tau and their class flips = dc)."""
    W = np.zeros((2, C))
    W[0, 0] = 1.0
    for om, j in group:
        nw = np.zeros_like(W)
        for tau in range(2):
            for dc in range(C):
                nw[tau, dc] += (1 - p[j]) * W[tau, dc]
                nw[tau ^ 1, dc ^ om] += p[j] * W[tau, dc]
        W = nw
    return W


def total_logprob(logp_cls: np.ndarray) -> np.ndarray:
    """log P(m) = log sum_L p_{m,L}  (-inf when every class has probability 0)."""
    mx = np.max(logp_cls, axis=1)
    fin = np.isfinite(mx)
    safe = np.where(fin, mx, 0.0)
    with np.errstate(divide="ignore"):
        return np.where(fin, safe + np.log(np.exp(logp_cls - safe[:, None]).sum(axis=1)), mx)


def grad_total_logprob(dem, det_bits: np.ndarray) -> np.ndarray:
    """d log P(m) / d p_j for every shot [B, n_mech], exact.

    P(m) is affine in each p_j: P = (1 - p_j) A_j + p_j B_j, where A_j (B_j) is P(m) with
    mechanism j forced off (on).  So d log P / d p_j = (B_j - A_j) / P, each term by the
    exact transfer matrix with p_j set to 0 and 1.  Plain and slow: tiny problems only.
    """
    lay = Layering(dem)
    base = total_logprob(transfer_matrix(dem, det_bits, lay))
    g = np.zeros((det_bits.shape[0], dem.n_mech))
    for j in range(dem.n_mech):
        pj = np.array(dem.p, dtype=np.float64)
        pj[j] = 1.0
        lb = total_logprob(transfer_matrix(dem.with_rates(pj), det_bits, lay))
        pj[j] = 0.0
        la = total_logprob(transfer_matrix(dem.with_rates(pj), det_bits, lay))
        g[:, j] = np.exp(lb - base) - np.exp(la - base)
    return g
