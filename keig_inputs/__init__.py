"""Seeded synthetic inputs for the k-eigenvalue transport problem.

This module holds data only: quadrature tables, cross-section tables,
material maps and random initial guesses.  It contains none of the solution
method's arithmetic, so both the CPU oracle (``oracle/``) and the GPU library
binding (``paper_2309_03347_gb300``) import it without sharing any solver code.

Problem statement followed (arXiv 2309.03347):

* unknowns live on the vertices of a Cartesian grid with ``n = 2**l`` points
  per axis, ``n - 1`` cells per axis, cell-constant cross sections
  (Sec. 2.1.3, Appendix A.3);
* multigroup energy with ``G`` groups (Appendix A.1);
* discrete ordinates with weights normalised to sum to one and directions
  ordered octant-major in the order of Eq. (hat-mu) of Appendix A.2:
  octant ``o`` has sign bits ``x = o & 1``, ``y = o & 2``, ``z = o & 4``
  (bit set means a positive cosine), so the first octant is (-,-,-) and the
  last (+,+,+).

The quadrature is the level-symmetric LQ_N family (the paper uses a square
set, Appendix A.2; a level-symmetric set is an equally valid octant-symmetric
set and is what the synthetic workloads ask for).  Levels follow the standard
recursion ``mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (N - 2)`` with the
published base cosines; the weight of each permutation class is fixed by
exact integration of even moments of one direction cosine over an octant
(S16, where those moments leave one degree of freedom, takes the tabulated
point weights).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

# Base cosines of the LQ_N level-symmetric sets (Lewis & Miller, Computational
# Methods of Neutron Transport, Table 4-1; Carlson).
_LQN_MU1 = {
    2: 0.5773503,
    4: 0.3500212,
    6: 0.2666355,
    8: 0.2182179,
    10: 0.1893213,
    12: 0.1672126,
    16: 0.1389568,
}

# Point weights of the orders whose even-moment system of one cosine does not
# fix them (S16: eight point classes, seven independent conditions), as
# tabulated with the base cosines above (Lewis & Miller, Table 4-1; weights of
# one octant summing to 1), keyed by the sorted level-index triple of the
# class.  The tabulated set also satisfies the mixed moments
# <mu^2 eta^2> = 1/15 and <mu^2 eta^2 xi^2> = 1/105.
_LQN_POINT_WEIGHTS = {
    16: {(0, 0, 7): 0.0489872, (0, 1, 6): 0.0413296, (0, 2, 5): 0.0212326, (0, 3, 4): 0.0256207,
         (1, 1, 5): 0.0360486, (1, 2, 4): 0.0144589, (1, 3, 3): 0.0344958, (2, 2, 3): 0.0085179},
}


@dataclasses.dataclass
class Quadrature:
    """Octant-symmetric quadrature.

    ``amu, aeta, axi, w8`` have length ``L/8``: the absolute direction cosines
    and the weight of one octant's directions (``8 * sum(w8) == 1``).  The full
    ``L``-direction arrays (signed, octant-major) are ``mu, eta, xi, w``.
    """

    order: int
    amu: np.ndarray
    aeta: np.ndarray
    axi: np.ndarray
    w8: np.ndarray

    @property
    def n_per_octant(self) -> int:
        return int(self.amu.size)

    @property
    def L(self) -> int:
        return 8 * self.n_per_octant

    def _signed(self, a: np.ndarray, bit: int) -> np.ndarray:
        out = np.empty(self.L)
        m = self.n_per_octant
        for o in range(8):
            s = 1.0 if (o & bit) else -1.0
            out[o * m:(o + 1) * m] = s * a
        return out

    @property
    def mu(self) -> np.ndarray:
        return self._signed(self.amu, 1)

    @property
    def eta(self) -> np.ndarray:
        return self._signed(self.aeta, 2)

    @property
    def xi(self) -> np.ndarray:
        return self._signed(self.axi, 4)

    @property
    def w(self) -> np.ndarray:
        return np.tile(self.w8, 8)


def level_symmetric(order: int) -> Quadrature:
    """Level-symmetric LQ_N set with ``N(N+2)`` directions (``N`` even)."""
    if order not in _LQN_MU1:
        raise ValueError(f"no LQ_N table for S{order}")
    h = order // 2
    m1 = _LQN_MU1[order]
    if order > 2:
        step = 2.0 * (1.0 - 3.0 * m1 * m1) / (order - 2)
    else:
        step = 0.0
    levels = np.sqrt(m1 * m1 + np.arange(h) * step)
    # points of one octant: level triples with i + j + k = h - 1 (0-based)
    pts = [(i, j, k) for k in range(h) for j in range(h) for i in range(h)
           if i + j + k == h - 1]
    classes = sorted(set(tuple(sorted(p)) for p in pts))
    c = len(classes)
    # even-moment conditions on one cosine; mu^2 is implied by symmetry and
    # the unit-sphere constraint, so use powers 0, 4, 6, ...
    powers = [0] + list(range(2, c + 1))
    a = np.zeros((c, c))
    rhs = np.zeros(c)
    for r, p in enumerate(powers):
        rhs[r] = 1.0 / (2 * p + 1)
        for ci, cl in enumerate(classes):
            a[r, ci] = sum(levels[q[0]] ** (2 * p) for q in pts
                           if tuple(sorted(q)) == cl)
    if order in _LQN_POINT_WEIGHTS:
        wc = np.array([_LQN_POINT_WEIGHTS[order][cl] for cl in classes])
        count = np.array([sum(1 for q in pts if tuple(sorted(q)) == cl) for cl in classes])
        wc = wc / float(count @ wc)  # the 7-digit table sums to 1 within 1e-6
        tol = 1e-6
    else:
        wc, *_ = np.linalg.lstsq(a, rhs, rcond=1e-12)
        tol = 1e-9
    if np.max(np.abs(a @ wc - rhs)) > tol or np.min(wc) <= 0:
        raise ValueError(f"S{order}: moment system has no positive solution")
    cls_w = {cl: wc[i] for i, cl in enumerate(classes)}
    amu = np.array([levels[p[0]] for p in pts])
    aeta = np.array([levels[p[1]] for p in pts])
    axi = np.array([levels[p[2]] for p in pts])
    w_oct = np.array([cls_w[tuple(sorted(p))] for p in pts])
    return Quadrature(order, amu, aeta, axi, w_oct / 8.0)


@dataclasses.dataclass
class Problem:
    """One k-eigenvalue problem in the layout the C-ABI ``tt_problem`` takes.

    Cross sections are per material ``m`` and group ``g``:
    ``sig_t[m, g]``, ``sig_s[m, g_to, g_from]``, ``nu_sig_f[m, g]``,
    ``chi[m, g]``.  ``mat[cz, cy, cx]`` gives the material of each cell
    (``n - 1`` cells per axis, x fastest).  ``bc`` lists the faces
    x-, x+, y-, y+, z-, z+ with 0 = vacuum, 1 = reflective.
    """

    name: str
    l: int
    side: tuple
    G: int
    sig_t: np.ndarray
    sig_s: np.ndarray
    nu_sig_f: np.ndarray
    chi: np.ndarray
    mat: np.ndarray
    quad: Quadrature
    bc: tuple = (0, 0, 0, 0, 0, 0)
    seed: int = 0
    eps: float = 1e-10
    rmax: int = 64
    inv_v: Optional[np.ndarray] = None
    sig_s1: Optional[np.ndarray] = None  # [m, g_to, g_from] P1 scattering moments (linear anisotropy)
    sig_s2: Optional[np.ndarray] = None  # [m, g_to, g_from] P2 moments
    sig_s3: Optional[np.ndarray] = None  # [m, g_to, g_from] P3 moments

    @property
    def n(self) -> int:
        return 1 << self.l

    @property
    def n_mat(self) -> int:
        return int(self.sig_t.shape[0])

    @property
    def L(self) -> int:
        return self.quad.L

    @property
    def delta(self) -> tuple:
        return tuple(float(s) / (self.n - 1) for s in self.side)

    @property
    def psi_shape(self) -> tuple:
        n = self.n
        return (self.G, self.L, n, n, n)

    @property
    def tt_modes(self) -> List[int]:
        """TT core mode sizes: [G, 8, L/8, z bits (MSB first), y bits, x bits]."""
        return [self.G, 8, self.quad.n_per_octant] + [2] * (3 * self.l)

    def with_bc(self, bc) -> "Problem":
        return dataclasses.replace(self, bc=tuple(bc))


def _downscatter(rng, sig_t_row, c_ratio, G, upscatter=()):
    """Scattering matrix [g_to, g_from]: the outscatter c*sig_t of each source
    group is split over destinations g >= g_from by Dirichlet(1) fractions;
    ``upscatter`` lists extra (g_to, g_from) pairs that share that split."""
    s = np.zeros((G, G))
    for gf in range(G):
        dests = list(range(gf, G)) + [gt for (gt, gsrc) in upscatter if gsrc == gf]
        frac = rng.dirichlet(np.ones(len(dests)))
        tot = c_ratio[gf] * sig_t_row[gf]
        for d, f in zip(dests, frac):
            s[d, gf] += tot * f
    return s


def _material(rng, G, fissile=True, c_fixed=None, upscatter=()):
    sig_t = rng.uniform(0.5, 1.5, G)
    if c_fixed is None:
        c = rng.uniform(0.3, 0.9, G)
    else:
        c = np.full(G, float(c_fixed))
    sig_s = _downscatter(rng, sig_t, c, G, upscatter)
    nsf = rng.uniform(0.05, 0.3, G) if fissile else np.zeros(G)
    return sig_t, sig_s, nsf


def _pack(mats, chi_rows):
    sig_t = np.stack([m[0] for m in mats])
    sig_s = np.stack([m[1] for m in mats])
    nsf = np.stack([m[2] for m in mats])
    chi = np.stack(chi_rows)
    return sig_t, sig_s, nsf, chi


def homogeneous(l=3, G=2, order=4, side=20.0, seed=1000, bc=(0,) * 6,
                name="homogeneous") -> Problem:
    """Homogeneous cube: one material, lower-triangular downscatter with
    scattering ratio U[0.3, 0.9], chi = e_1."""
    rng = np.random.default_rng(seed)
    m = _material(rng, G, fissile=True)
    chi = np.zeros(G)
    chi[0] = 1.0
    sig_t, sig_s, nsf, chi = _pack([m], [chi])
    n = 1 << l
    mat = np.zeros((n - 1,) * 3, dtype=np.uint8)
    return Problem(name, l, (side,) * 3, G, sig_t, sig_s, nsf, chi, mat,
                   level_symmetric(order), tuple(bc), seed)


def fissile_box(l=5, G=4, order=8, side=20.0, seed=1001, half_width=None,
                name="fissile_box") -> Problem:
    """Central fissile cube (cells [n/2 - h, n/2 + h) on each axis) inside a
    non-fissile reflector with scattering ratio 0.9; chi = e_1."""
    rng = np.random.default_rng(seed)
    n = 1 << l
    h = half_width if half_width is not None else max(1, n // 4)
    fuel = _material(rng, G, fissile=True)
    refl = _material(rng, G, fissile=False, c_fixed=0.9)
    chi = np.zeros(G)
    chi[0] = 1.0
    sig_t, sig_s, nsf, chi = _pack([fuel, refl], [chi, chi])
    mat = np.ones((n - 1,) * 3, dtype=np.uint8)
    lo, hi = max(0, n // 2 - h), min(n - 1, n // 2 + h)
    mat[lo:hi, lo:hi, lo:hi] = 0
    return Problem(name, l, (side,) * 3, G, sig_t, sig_s, nsf, chi, mat,
                   level_symmetric(order), (0,) * 6, seed)


def three_boxes(l=6, G=8, order=16, side=20.0, seed=1002,
                name="three_boxes") -> Problem:
    """Three materials in seeded axis-aligned boxes; upscatter only from the
    last group into the one before it; chi geometric (ratio 1/2) over the
    first three groups."""
    rng = np.random.default_rng(seed)
    n = 1 << l
    ups = ((G - 2, G - 1),) if G >= 2 else ()
    mats = [_material(rng, G, fissile=(i < 2), upscatter=ups) for i in range(3)]
    chi = np.zeros(G)
    k = min(3, G)
    chi[:k] = 0.5 ** np.arange(k)
    chi /= chi.sum()
    sig_t, sig_s, nsf, chi = _pack(mats, [chi] * 3)
    mat = np.full((n - 1,) * 3, 2, dtype=np.uint8)
    c = n - 1
    for m in (1, 0):
        lo = rng.integers(0, c // 3, size=3)
        hi = lo + rng.integers(c // 3, 2 * c // 3, size=3)
        hi = np.minimum(hi, c)
        mat[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = m
    return Problem(name, l, (side,) * 3, G, sig_t, sig_s, nsf, chi, mat,
                   level_symmetric(order), (0,) * 6, seed)


def config(idx: int, bc: str = "vacuum") -> Problem:
    """The seeded synthetic workloads.

    0: 8^3 points, 2 groups, S4, homogeneous (vacuum or all-reflective);
    1: 32^3 points, 4 groups, S8, fissile box in a c = 0.9 reflector, side
       2.5 cm: about 2.5 mean free paths across, the optical size of the
       paper's 10 cm Jezebel cube (Sec. 4.2), so that cells are thin
       (<= 0.12 mfp) as at the paper's 128-512 points per axis;
    2: 64^3 points, 8 groups, S16, three materials in boxes.
    """
    if idx == 0:
        p = homogeneous(l=3, G=2, order=4, seed=1000, name="cube8_g2_s4")
        p.eps, p.rmax = 1e-10, 64
        if bc == "reflective":
            p = p.with_bc((1,) * 6)
        return p
    if idx == 1:
        p = fissile_box(l=5, G=4, order=8, seed=1001, half_width=8, side=2.5,
                        name="box32_g4_s8")
        p.eps, p.rmax = 1e-7, 64
        return p
    if idx == 2:
        p = three_boxes(l=6, G=8, order=16, seed=1002, name="boxes64_g8_s16")
        p.eps, p.rmax = 1e-6, 128
        return p
    raise ValueError(idx)


def bare_cube(l: int, G: int = 2, order: int = 4, side: float = 10.0, seed: int = 1000) -> Problem:
    """Bare homogeneous cube with vacuum faces, the geometry of the paper's
    3-D benchmark (Sec. 4.2: a 10 cm cube at 128-512 grid points per axis),
    with the seeded synthetic cross sections of config 0 (the benchmark's
    256-group nuclear data is not available)."""
    p = homogeneous(l=l, G=G, order=order, side=side, seed=seed,
                    name=f"cube{1 << l}_g{G}_s{order}_{side:g}cm")
    return p


def random_rank1_cores(modes, seed: int, lo=0.5, hi=1.5) -> List[np.ndarray]:
    """Seeded positive rank-1 TT cores (shape (1, n_k, 1)) used as the random
    initial guess of the fixed-point iteration."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(lo, hi, (1, m, 1)) for m in modes]


def random_cores(modes, ranks, seed: int) -> List[np.ndarray]:
    """Seeded Gaussian TT cores with the given bond ranks (len(modes)+1)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((ranks[k], modes[k], ranks[k + 1]))
            for k in range(len(modes))]


def fissile_response(prob: Problem, group: int = 0):
    """Weights of the flux functional J = sum over fissile cells of
    vol * (8-corner average of the group-``group`` scalar flux), written as
    J = sum_g sum_v resp_g[g] resp_v[v] phi[g, v] on the vertices.

    resp_g is the unit vector of ``group``; resp_v[v] adds vol / 8 for every
    fissile cell (nu_sig_f > 0 in some group) that has v as a corner, in the
    vertex order of the scalar flux (z, y, x; x fastest)."""
    n = prob.n
    fissile = (prob.nu_sig_f.max(axis=1) > 0)[prob.mat]  # (cz, cy, cx)
    vol = float(np.prod(prob.delta))
    resp_v = np.zeros((n, n, n))
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                resp_v[a:a + n - 1, b:b + n - 1, c:c + n - 1] += fissile * (vol / 8.0)
    resp_g = np.zeros(prob.G)
    resp_g[group] = 1.0
    return resp_g, resp_v


# ---------------------------------------------------------------- 1-D slab
@dataclasses.dataclass
class Slab:
    """A 1-D slab k-eigenvalue problem (vacuum on both faces) in the layout
    the C-ABI ``tt_slab`` takes: 2^l points across ``width``, materials per
    cell (``mat[c]``, 2^l - 1 cells), tables as in ``Problem``, and a
    half-range quadrature: ``amu[d] > 0`` with weights ``w[d]`` used for both
    signs of mu (2 * sum(w) = 1)."""

    name: str
    l: int
    width: float
    G: int
    sig_t: np.ndarray
    sig_s: np.ndarray
    nu_sig_f: np.ndarray
    chi: np.ndarray
    mat: np.ndarray
    amu: np.ndarray
    w: np.ndarray

    @property
    def n(self) -> int:
        return 1 << self.l

    @property
    def n_mat(self) -> int:
        return int(self.sig_t.shape[0])

    @property
    def n_dir(self) -> int:
        return int(self.amu.size)

    @property
    def delta(self) -> float:
        return float(self.width) / (self.n - 1)

    @property
    def psi_shape(self) -> tuple:
        """(G, 2, n_dir, n): hemisphere 0 is mu < 0, 1 is mu > 0."""
        return (self.G, 2, self.n_dir, self.n)

    @property
    def tt_modes(self) -> List[int]:
        return [self.G, 2, self.n_dir] + [2] * self.l


def gauss_legendre_half(L: int):
    """Half-range Gauss-Legendre set of an S_L quadrature: the L/2 positive
    nodes of the L-point Gauss-Legendre rule and their weights halved (so
    that the weights of all L directions sum to 1)."""
    if L < 2 or L % 2:
        raise ValueError("L must be even and >= 2")
    x, wt = np.polynomial.legendre.leggauss(L)
    pos = x > 0
    order = np.argsort(x[pos])
    return x[pos][order].copy(), 0.5 * wt[pos][order].copy()


def pu239_slab(l: int = 10, L: int = 8) -> Slab:
    """The one-group bare Pu-239 slab of the paper's 1-D case study (Sec. 4.1,
    cross sections as printed in its table): nu = 3.24, sigma_f = 0.081600,
    sigma_s = 0.225216, sigma_t = 0.32640 (1/cm), width 3.707444 cm, vacuum
    faces; exactly critical (k = 1) for the exact transport solution."""
    amu, w = gauss_legendre_half(L)
    nu, sf, ss, st = 3.24, 0.081600, 0.225216, 0.32640
    return Slab(name=f"pu239_slab_l{l}_S{L}", l=l, width=3.707444, G=1,
                sig_t=np.array([[st]]), sig_s=np.array([[[ss]]]), nu_sig_f=np.array([[nu * sf]]),
                chi=np.array([[1.0]]), mat=np.zeros(2 ** l - 1, np.uint8), amu=amu, w=w)


def with_linear_anisotropy(prob: Problem, mu_bar: float) -> Problem:
    """The same problem with linearly anisotropic scattering: P1 moments
    sig_s1 = mu_bar * sig_s (mu_bar: mean scattering cosine, |mu_bar| < 1/3
    keeps the P1 kernel 1 + 3 mu_bar cos non-negative)."""
    return dataclasses.replace(prob, sig_s1=mu_bar * np.asarray(prob.sig_s, dtype=np.float64),
                               name=prob.name + f"_p1_{mu_bar:g}")


def with_anisotropy(prob: Problem, f1: float, f2: float = 0.0, f3: float = 0.0) -> Problem:
    """The same problem with Legendre scattering moments sig_sn = f_n * sig_s
    for n = 1..3 (f_n = 0 leaves the order out)."""
    s0 = np.asarray(prob.sig_s, dtype=np.float64)
    return dataclasses.replace(prob, sig_s1=f1 * s0 if f1 else None, sig_s2=f2 * s0 if f2 else None,
                               sig_s3=f3 * s0 if f3 else None,
                               name=prob.name + f"_aniso_{f1:g}_{f2:g}_{f3:g}")
