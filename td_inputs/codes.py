"""Decoding problems as detector error models (Sec. 2.4) with space-time layouts.

A DEM is the triple (H, p, l) of Sec. 2.4: mechanism j flips the detectors listed in
``mech_dets[j]`` and the logical observables listed in ``mech_obs[j]`` and occurs
independently with probability ``p[j]``.  Every detector also carries integer
coordinates (x, y, t): (x, y) is its site in a layer, t its layer.  The layered
3D form of Sec. 4 (identical layers, inter-layer bonds only between equal sites)
is read off these coordinates.

Generators:
  * point_sector_3d -- the point sector of the 3D surface code with open boundaries,
    as drawn for d=3 in the point-sector detector network figure of Sec. 5.1: checks on
    a d x d x (d-1) grid, one mechanism per edge (qubit), z edges dangling at the two
    rough boundaries.  n = d^3 + 2d(d-1)^2 mechanisms, d^2(d-1) detectors.
  * rotated_phenomenological -- the rotated 2D surface code under bit flips with noisy
    syndrome rounds stacked in time (Sec. 1 and Sec. 2.4: the noisy-measurement problem
    is a 3D decoding problem).  Z checks become sites on a rotated (u, v) grid.
  * repetition_phenomenological -- a 1D chain stacked in time (tiny test problems).
  * five_qubit_code -- the [[5,1,3]] code of the detector/generator figures of Sec. 3,
    as Pauli strings, for the general-stabilizer definition of Sec. 2.3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class DEM:
    n_det: int
    n_obs: int
    mech_dets: list            # list[tuple[int, ...]]: detectors flipped by mechanism j
    mech_obs: list             # list[tuple[int, ...]]: observables flipped by mechanism j
    p: np.ndarray              # float64 [n_mech]
    det_xyt: np.ndarray        # int32 [n_det, 3]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_mech(self) -> int:
        return len(self.mech_dets)

    @property
    def dims(self):
        """(nx, ny, nt): extent of the coordinate grid."""
        return tuple(int(v) + 1 for v in self.det_xyt.max(axis=0))

    def H_dense(self) -> np.ndarray:
        H = np.zeros((self.n_det, self.n_mech), dtype=np.uint8)
        for j, ds in enumerate(self.mech_dets):
            for i in ds:
                H[i, j] ^= 1
        return H

    def L_dense(self) -> np.ndarray:
        L = np.zeros((self.n_obs, self.n_mech), dtype=np.uint8)
        for j, os_ in enumerate(self.mech_obs):
            for o in os_:
                L[o, j] ^= 1
        return L

    def H_csr(self):
        """CSR of H (detectors x mechanisms): (indptr int32 [n_det+1], indices int32)."""
        return _csr(self.n_det, self.mech_dets)

    def L_csr(self):
        """CSR of l (observables x mechanisms)."""
        return _csr(self.n_obs, self.mech_obs)

    def with_rates(self, p) -> "DEM":
        p = np.asarray(p, dtype=np.float64)
        assert p.shape == (self.n_mech,)
        return DEM(self.n_det, self.n_obs, list(self.mech_dets), list(self.mech_obs), p.copy(),
                   self.det_xyt.copy(), self.name, dict(self.meta))


def _csr(n_rows, cols_of_mech):
    rows = [[] for _ in range(n_rows)]
    for j, rs in enumerate(cols_of_mech):
        for r in rs:
            rows[r].append(j)
    indptr = np.zeros(n_rows + 1, dtype=np.int32)
    for r in range(n_rows):
        indptr[r + 1] = indptr[r] + len(rows[r])
    indices = np.array([j for r in rows for j in sorted(r)], dtype=np.int32)
    return indptr, indices


def point_sector_3d(d: int, p: float = 0.05) -> DEM:
    """Point sector of the 3D surface code (phase flips on edges, vertex checks).

    Detector (x, y, t), x, y in [0, d), t in [0, d-1), index t*d*d + y*d + x.
    Mechanisms: x edges and y edges inside each layer, z edges between consecutive
    layers, and d^2 z edges dangling below layer 0 and above layer d-2 (the rough
    boundaries).  The logical observable is flipped by the bottom dangling edges: every
    error string joining the two rough boundaries crosses that plane once.
    """
    assert d >= 2
    nt = d - 1

    def det(x, y, t):
        return t * d * d + y * d + x

    dets, obs = [], []
    for t in range(nt):
        if t == 0:
            for y in range(d):
                for x in range(d):
                    dets.append((det(x, y, 0),)); obs.append((0,))
        for y in range(d):
            for x in range(d - 1):
                dets.append((det(x, y, t), det(x + 1, y, t))); obs.append(())
        for y in range(d - 1):
            for x in range(d):
                dets.append((det(x, y, t), det(x, y + 1, t))); obs.append(())
        if t + 1 < nt:
            for y in range(d):
                for x in range(d):
                    dets.append((det(x, y, t), det(x, y, t + 1))); obs.append(())
        if t == nt - 1:
            for y in range(d):
                for x in range(d):
                    dets.append((det(x, y, t),)); obs.append(())
    xyt = np.array([(x, y, t) for t in range(nt) for y in range(d) for x in range(d)], dtype=np.int32)
    n = len(dets)
    assert n == d ** 3 + 2 * d * (d - 1) ** 2
    return DEM(d * d * nt, 1, dets, obs, np.full(n, float(p)), xyt, name=f"point3d_d{d}",
               meta=dict(kind="point3d", d=d))


def rotated_z_checks(d: int):
    """Z plaquettes of the rotated distance-d code (d odd) and the qubits they act on.

    Data qubit (i, j), i, j in [0, d).  Plaquette (i, j) has corners (i, j), (i+1, j),
    (i, j+1), (i+1, j+1); interior plaquettes are Z type when i + j is even; weight-2
    Z plaquettes sit on the top (i = -1, j odd) and bottom (i = d-1, j even) edges.
    Returns a list of ((i, j), [qubits]) and the rotated site coordinate of each check.
    """
    assert d % 2 == 1 and d >= 3
    checks = []
    for i in range(-1, d):
        for j in range(0, d - 1):
            if 0 <= i <= d - 2:
                if (i + j) % 2:
                    continue
            elif i == -1:
                if j % 2 == 0:
                    continue
            else:  # i == d - 1
                if (i + j) % 2:
                    continue
            qs = [(a, b) for a in (i, i + 1) for b in (j, j + 1) if 0 <= a < d and 0 <= b < d]
            checks.append(((i, j), qs))
    # (i + j) is even for every Z plaquette: u = (i + j) / 2, v = (i - j) / 2 is a grid on
    # which checks sharing a qubit are nearest neighbours.
    coords = []
    for (i, j), _ in checks:
        assert (i + j) % 2 == 0
        coords.append(((i + j) // 2, (i - j + (d - 1)) // 2))
    return checks, coords


def rotated_phenomenological(d: int, rounds: int, p: float = 0.03, q: float = 0.03) -> DEM:
    """Rotated surface code, bit flips, `rounds` noisy syndrome rounds + 1 perfect round.

    Layer t in [0, rounds]: every data qubit flips with probability p, then the Z checks
    are measured; the measurement of layer t < rounds is wrong with probability q, the
    last round is perfect.  Detector (s, t) = M(s, t) xor M(s, t-1) with M(s, -1) = 0.
    A data flip at layer t flips detector t of its one or two checks; a measurement error
    at layer t flips detectors t and t+1 of its check.  The logical observable is the
    parity of flips on the qubit column j = 0 (a Z-logical representative); each of these
    qubits touches exactly one Z check, so they are single-detector mechanisms.
    """
    checks, coords = rotated_z_checks(d)
    S = len(checks)
    nt = rounds + 1
    q_of = {}
    for s, (_, qs) in enumerate(checks):
        for qq in qs:
            q_of.setdefault(qq, []).append(s)

    def det(s, t):
        return t * S + s

    dets, obs, pr = [], [], []
    for t in range(nt):
        for i in range(d):
            for j in range(d):
                ss = q_of.get((i, j), [])
                assert 1 <= len(ss) <= 2
                dets.append(tuple(det(s, t) for s in ss))
                obs.append((0,) if j == 0 else ())
                pr.append(p)
        if t < nt - 1:
            for s in range(S):
                dets.append((det(s, t), det(s, t + 1))); obs.append(()); pr.append(q)
    xyt = np.array([(coords[s][0], coords[s][1], t) for t in range(nt) for s in range(S)], dtype=np.int32)
    return DEM(S * nt, 1, dets, obs, np.array(pr, dtype=np.float64), xyt,
               name=f"rotated_d{d}_r{rounds}", meta=dict(kind="rotated", d=d, rounds=rounds))


def repetition_phenomenological(n: int, rounds: int, p: float = 0.05, q: float = 0.05) -> DEM:
    """Distance-n repetition code (n-1 checks on a line), `rounds` noisy rounds + 1 perfect.

    Bit j flips checks j-1 and j (bits 0 and n-1 touch one check); the observable is bit 0.
    """
    S = n - 1
    nt = rounds + 1
    dets, obs, pr = [], [], []
    for t in range(nt):
        for j in range(n):
            ds = tuple(t * S + s for s in (j - 1, j) if 0 <= s < S)
            dets.append(ds); obs.append((0,) if j == 0 else ()); pr.append(p)
        if t < nt - 1:
            for s in range(S):
                dets.append((t * S + s, (t + 1) * S + s)); obs.append(()); pr.append(q)
    xyt = np.array([(s, 0, t) for t in range(nt) for s in range(S)], dtype=np.int32)
    return DEM(S * nt, 1, dets, obs, np.array(pr, dtype=np.float64), xyt,
               name=f"rep_n{n}_r{rounds}", meta=dict(kind="repetition", n=n, rounds=rounds))


@dataclass
class GenProblem:
    """A CSS sector in the generator picture (Sec. 3.2): the coset of an error r is
    r + span of the stabilizer generators, each a vertex flipping the qubits of its edges.

    Qubit j is an edge of the generator graph joining one or two generators
    (``edges[j]``, indices into the generators) and flips with probability ``p[j]``.
    ``gen_xyt`` holds the (x, y, t) of every generator (the layered form of Sec. 4: t the
    layer, (x, y) the site).  ``xbar`` lists the qubits of a logical operator of the flipped
    type (the class shift: the other coset is r + xbar + span) and ``zbar`` those of the
    conjugate logical (the class of an error is its parity on zbar).  ``face_dem`` is the same
    problem in the detector picture (Sec. 2.4): its detectors are the checks that detect the
    errors, its observable is zbar -- used to sample syndromes and by the exact oracles.
    """
    n_gen: int
    edges: list                # list[tuple[int, ...]] generators of each qubit (1 or 2)
    p: np.ndarray              # float64 [n_qubits]
    gen_xyt: np.ndarray        # int32 [n_gen, 3]
    xbar: list
    zbar: list
    face_dem: "DEM"
    name: str = ""

    @property
    def n_qubits(self) -> int:
        return len(self.edges)


def loop_sector_3d(d: int, p: float = 0.1) -> GenProblem:
    """Loop sector of the 3D surface code with open boundaries (Sec. 5.2): bit flips on the
    qubits of point_sector_3d(d), detected by the plaquettes (loop-like syndromes), decoded
    in the generator picture of the vertex stabilizers -- the point sector's lattice with the
    roles of the + and = nodes swapped.

    Generators: the d x d x (d-1) vertices (x, y, t), index t*d*d + y*d + x; qubits in the
    order of point_sector_3d (x edges, y edges, z edges, dangling z edges at the two rough
    boundaries).  Plaquettes: every elementary square of the lattice, those crossing a
    rough boundary truncated to their three edges.  The logical membrane xbar is the d*d
    dangling edges below layer 0, the conjugate string zbar the z column at (0, 0)."""
    pt = point_sector_3d(d, p)
    edges = [tuple(ds) for ds in pt.mech_dets]
    nt = d - 1
    # qubit index of every edge, by kind
    idx = {}
    for j, ds in enumerate(edges):
        if len(ds) == 1:
            v = ds[0]
            t = v // (d * d)
            key = ("dn", v) if (t == 0 and ("dn", v) not in idx) else ("up", v)
            if t == 0 and t == nt - 1 and ("dn", v) in idx:
                key = ("up", v)
            idx[key] = j
        else:
            a, b = sorted(ds)
            idx[("e", a, b)] = j

    def vid(x, y, t):
        return t * d * d + y * d + x

    def edge(a, b):
        return idx[("e", min(a, b), max(a, b))]

    def zedge(x, y, t):
        """z edge from layer t to t+1 at (x, y); t = -1 / nt - 1: the dangling edges."""
        if t == -1:
            return idx[("dn", vid(x, y, 0))]
        if t == nt - 1:
            return idx[("up", vid(x, y, nt - 1))]
        return edge(vid(x, y, t), vid(x, y, t + 1))

    faces = []
    for t in range(nt):
        for y in range(d - 1):
            for x in range(d - 1):
                faces.append((edge(vid(x, y, t), vid(x + 1, y, t)), edge(vid(x, y + 1, t), vid(x + 1, y + 1, t)),
                              edge(vid(x, y, t), vid(x, y + 1, t)), edge(vid(x + 1, y, t), vid(x + 1, y + 1, t))))
    for t in range(-1, nt):          # squares between layers t and t+1 (t = -1, nt-1: the rough boundaries)
        for y in range(d):
            for x in range(d - 1):
                f = [zedge(x, y, t), zedge(x + 1, y, t)]
                if t >= 0:
                    f.append(edge(vid(x, y, t), vid(x + 1, y, t)))
                if t + 1 <= nt - 1:
                    f.append(edge(vid(x, y, t + 1), vid(x + 1, y, t + 1)))
                faces.append(tuple(f))
        for y in range(d - 1):
            for x in range(d):
                f = [zedge(x, y, t), zedge(x, y + 1, t)]
                if t >= 0:
                    f.append(edge(vid(x, y, t), vid(x, y + 1, t)))
                if t + 1 <= nt - 1:
                    f.append(edge(vid(x, y, t + 1), vid(x, y + 1, t + 1)))
                faces.append(tuple(f))
    n = len(edges)
    mech_dets = [[] for _ in range(n)]
    for fi, f in enumerate(faces):
        for q in f:
            mech_dets[q].append(fi)
    xbar = [idx[("dn", vid(x, y, 0))] for y in range(d) for x in range(d)]
    zbar = [zedge(0, 0, t) for t in range(-1, nt)]
    mech_obs = [(0,) if j in set(zbar) else () for j in range(n)]
    # face coordinates are not used by any sweep of this problem (the detector picture of the
    # loop sector is not graph-like); each face gets a distinct dummy coordinate
    fxyt = np.array([(fi, 0, 0) for fi in range(len(faces))], dtype=np.int32)
    face_dem = DEM(len(faces), 1, [tuple(m) for m in mech_dets], mech_obs, np.full(n, float(p)), fxyt,
                   name=f"loop3d_faces_d{d}", meta=dict(kind="loop3d_faces", d=d))
    gen_xyt = np.array([(x, y, t) for t in range(nt) for y in range(d) for x in range(d)], dtype=np.int32)
    return GenProblem(d * d * nt, edges, np.full(n, float(p)), gen_xyt, xbar, zbar, face_dem,
                      name=f"loop3d_d{d}")


def log_uniform_rates(dem: DEM, seed: int, lo: float = 1e-3, hi: float = 1e-2) -> DEM:
    """Replace every rate by exp(U(ln lo, ln hi)) drawn from the counter-based stream."""
    from .sampler import uniform53
    u = uniform53(seed, np.arange(dem.n_mech, dtype=np.uint64))
    return dem.with_rates(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))))


def five_qubit_code():
    """[[5,1,3]] code with the stabilizer generators named in Sec. 3.1.

    Returns (stabilizers, (x_logical, z_logical)) as Pauli strings over {I, X, Y, Z}.
    Sec. 3.1 names z1 = IZIXX, which commutes with every generator, and x1 = XZIZI, which
    anticommutes with s1, s2 and s4, so it is not a logical operator of this code; the
    transversal XXXXX (commutes with every generator, anticommutes with z1) is used.
    """
    stabs = ["XZZXI", "IXZZX", "XIXZZ", "ZXIXZ"]
    return stabs, ("XXXXX", "IZIXX")
