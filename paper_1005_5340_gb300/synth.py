"""Seeded synthetic molecules for the iterative polarizability solve.

This module only draws inputs; it contains none of the method's arithmetic
(no response function, no kernel application, no solver).  Both the CPU
oracle and the CUDA path receive the arrays it returns.

The inputs mirror what Sec. 2 (eq. lcao) and Sec. 3 (eq. vertex-ansatz,
eq. matrix_self_energy) of the paper assume to be available from a prior DFT
run: Kohn-Sham eigenvalues E and occupations n, LCAO coefficients X_a^E,
dominant-product vertex blocks V_mu^{ab} that live on one atom (local) or on
one pair of atoms (bilocal), the interaction kernel f_Hxc^{mu nu} and the
dipole moments d_i^mu.  The paper's molecules came from SIESTA runs that are
not available, so every quantity is synthetic:

* atoms: uniform in a cube at number density ``density`` (bohr^-3),
  rejection-sampled so that no two atoms are closer than ``min_spacing``;
* 13 orbitals per atom, orbitals of an atom contiguous;
* eigenvalues: n_orb uniform draws in [e_lo, e_hi] Ha, sorted ascending;
* occupations: 2 on the n_occ lowest states, 0 elsewhere (closed shell);
* X: Haar-random orthogonal n_orb x n_orb (QR of a Gaussian matrix with the
  sign of diag(R) fixed); column E holds state E;
* products: ``n_local`` per atom (block on A x A, symmetrised
  (G + G^T)/sqrt(2)), ``n_bilocal`` per atom pair closer than ``pair_cutoff``
  (block on A x B, the B x A mirror implied), entries Gaussian times
  ``vertex_scale * exp(-R_AB / 2)``;
* centres: the atom for a local product, the pair midpoint for a bilocal one;
* K^{mu nu} = 1 / sqrt(|c_mu - c_nu|^2 + 1) + 0.05 delta_{mu nu}
  (an inverse multiquadric, symmetric positive definite);
* d_i^mu = (c_mu - centroid)_i * ||V_mu||_F.

Random numbers come from one counter-based generator, the SplitMix64 output
function of Steele, Lea and Flood (OOPSLA 2014) applied to a counter, so a
given (seed, stream) pair yields the same integers on every machine.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Global scale of the vertex entries.  With unit-variance entries the
# spectral radius of chi0(omega) K is 1e4 (4 atoms) to 5e4 (64 atoms) and
# restarted GMRES needs thousands of products to reach 1e-6; at 0.05 the
# Krylov dimension at 1e-6 is 9-11 (4 atoms) and 26-33 (64 atoms), the same
# order as the paper's 7-12 at a 1% tolerance (Sec. 7.1).  One value for
# every workload and every precision.
VERTEX_SCALE = 0.05

# Stream tags: one independent counter stream per kind of draw.
_S_POS, _S_ENERGY, _S_X, _S_VERTEX, _S_SIZES = 1, 2, 3, 4, 5


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (bijective 64-bit finaliser)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class CounterRNG:
    """Counter-based SplitMix64: output i of stream (seed, tag) is
    mix64(key + (i + 1) * gamma), key = mix64(mix64(seed) ^ tag)."""

    def __init__(self, seed: int, tag: int):
        s = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
        self.key = _mix64(s ^ np.uint64(tag))[0]
        self.pos = 0

    def bits(self, n: int) -> np.ndarray:
        i = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix64(self.key + i * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by the Box-Muller transform."""
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]


@dataclasses.dataclass
class System:
    """One molecule in the layout of the C boundary (tddft_system).

    X is indexed X[a, E] (orbital a, state E).  vertex holds the blocks of all
    products back to back: product mu on atoms (A, B), A <= B, owns
    vertex[vertex_offset[mu]:vertex_offset[mu+1]] = an n_A x n_B row-major block.
    K is dense n_prod x n_prod, dipole is 3 x n_prod.
    """
    n_atoms: int
    atom_orb_offset: np.ndarray   # int32 [n_atoms + 1]
    eigenvalues: np.ndarray       # f64 [n_orb], ascending
    occupations: np.ndarray       # f64 [n_orb]
    X: np.ndarray                 # f64 [n_orb, n_orb], X[a, E]
    prod_atoms: np.ndarray        # int32 [n_prod, 2]
    vertex_offset: np.ndarray     # int64 [n_prod + 1]
    vertex: np.ndarray            # f64 [vertex_offset[-1]]
    K: np.ndarray                 # f64 [n_prod, n_prod]
    dipole: np.ndarray            # f64 [3, n_prod]
    positions: np.ndarray | None = None   # f64 [n_atoms, 3] (bohr), informative
    centres: np.ndarray | None = None     # f64 [n_prod, 3], informative

    @property
    def n_orb(self) -> int:
        return int(self.atom_orb_offset[-1])

    @property
    def n_prod(self) -> int:
        return int(self.prod_atoms.shape[0])

    @property
    def n_occ(self) -> int:
        return int(np.count_nonzero(self.occupations > 0))

    def vertex_block(self, mu: int) -> np.ndarray:
        A, B = self.prod_atoms[mu]
        nA = self.atom_orb_offset[A + 1] - self.atom_orb_offset[A]
        nB = self.atom_orb_offset[B + 1] - self.atom_orb_offset[B]
        return self.vertex[self.vertex_offset[mu]:self.vertex_offset[mu + 1]].reshape(nA, nB)


def atom_positions(n_atoms: int, seed: int, density: float, min_spacing: float) -> np.ndarray:
    rng = CounterRNG(seed, _S_POS)
    side = (n_atoms / density) ** (1.0 / 3.0)
    pos = np.zeros((0, 3))
    tries = 0
    while pos.shape[0] < n_atoms:
        c = rng.uniform(3) * side
        tries += 1
        if tries > 10000 * n_atoms:
            raise RuntimeError("cannot place atoms at this density and spacing")
        if pos.shape[0] and np.min(np.linalg.norm(pos - c, axis=1)) < min_spacing:
            continue
        pos = np.vstack([pos, c])
    return pos


def haar_orthogonal(n: int, rng: CounterRNG) -> np.ndarray:
    g = rng.normal(n * n).reshape(n, n)
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def make_system(n_atoms: int, seed: int, *, orb_per_atom: int = 13, occ_per_atom: int = 2,
                n_local: int = 40, n_bilocal: int = 20, pair_cutoff: float = 8.0,
                density: float = 0.0055, min_spacing: float = 2.5,
                e_lo: float = -1.0, e_hi: float = 0.5, vertex_scale: float = VERTEX_SCALE,
                with_K: bool = True) -> System:
    """Draw one synthetic molecule (see the module docstring for the recipe)."""
    pos = atom_positions(n_atoms, seed, density, min_spacing)
    n_orb = orb_per_atom * n_atoms
    n_occ = occ_per_atom * n_atoms
    aoff = np.arange(n_atoms + 1, dtype=np.int32) * orb_per_atom

    erng = CounterRNG(seed, _S_ENERGY)
    E = np.sort(e_lo + (e_hi - e_lo) * erng.uniform(n_orb))
    occ = np.zeros(n_orb)
    occ[:n_occ] = 2.0

    X = haar_orthogonal(n_orb, CounterRNG(seed, _S_X))

    vrng = CounterRNG(seed, _S_VERTEX)
    pairs, centres, blocks = [], [], []
    for A in range(n_atoms):
        for _ in range(n_local):
            g = vrng.normal(orb_per_atom * orb_per_atom).reshape(orb_per_atom, orb_per_atom)
            blocks.append(vertex_scale * (g + g.T) / math.sqrt(2.0))
            pairs.append((A, A))
            centres.append(pos[A])
    for A in range(n_atoms):
        for B in range(A + 1, n_atoms):
            R = float(np.linalg.norm(pos[A] - pos[B]))
            if R >= pair_cutoff:
                continue
            for _ in range(n_bilocal):
                g = vrng.normal(orb_per_atom * orb_per_atom).reshape(orb_per_atom, orb_per_atom)
                blocks.append(vertex_scale * math.exp(-R / 2.0) * g)
                pairs.append((A, B))
                centres.append(0.5 * (pos[A] + pos[B]))
    n_prod = len(pairs)
    prod_atoms = np.asarray(pairs, dtype=np.int32).reshape(n_prod, 2)
    centres = np.asarray(centres).reshape(n_prod, 3)
    sizes = np.array([b.size for b in blocks], dtype=np.int64)
    voff = np.zeros(n_prod + 1, dtype=np.int64)
    voff[1:] = np.cumsum(sizes)
    vertex = np.concatenate([b.ravel() for b in blocks])

    if with_K:
        # row blocks keep the temporaries small for tens of thousands of products
        K = np.empty((n_prod, n_prod))
        for r0 in range(0, n_prod, 2048):
            r1 = min(n_prod, r0 + 2048)
            d2 = np.zeros((r1 - r0, n_prod))
            for ax in range(3):
                d2 += (centres[r0:r1, ax, None] - centres[None, :, ax]) ** 2
            K[r0:r1] = 1.0 / np.sqrt(d2 + 1.0)
        K[np.diag_indices(n_prod)] += 0.05
    else:
        K = np.zeros((0, 0))
    norms = np.array([np.linalg.norm(b) for b in blocks])
    dip = ((centres - pos.mean(axis=0)) * norms[:, None]).T.copy()
    return System(n_atoms=n_atoms, atom_orb_offset=aoff, eigenvalues=E, occupations=occ,
                  X=X, prod_atoms=prod_atoms, vertex_offset=voff, vertex=vertex, K=K,
                  dipole=dip, positions=pos, centres=centres)


def tiny_system(seed: int, n_atoms: int = 2, orb_per_atom: int = 3, occ_per_atom: int = 1,
                n_local: int = 2, n_bilocal: int = 2, **kw) -> System:
    """A small molecule for brute-force checks (same recipe, fewer of everything)."""
    kw.setdefault("density", 0.01)
    return make_system(n_atoms, seed, orb_per_atom=orb_per_atom, occ_per_atom=occ_per_atom,
                       n_local=n_local, n_bilocal=n_bilocal, **kw)


# Workloads.  Frequencies are inclusive uniform grids (omega = 0 included).
WORKLOADS = {
    # density (bohr^-3) is calibrated per size so that the product count lands
    # near 280 / 9k / 35k (surface atoms of a small cube have fewer pairs).
    "tiny4": dict(n_atoms=4, seed=1, density=0.012, n_omega=64, w_hi=1.0, eps=0.01,
                  restart=30, tol=1e-8),
    "medium64": dict(n_atoms=64, seed=2, density=0.0094, n_omega=256, w_hi=1.5, eps=0.005,
                     restart=40, tol=1e-6),
    "large256": dict(n_atoms=256, seed=3, density=0.0064, n_omega=512, w_hi=1.5, eps=0.005,
                     restart=40, tol=1e-6),
}


def omega_grid(n_omega: int, w_hi: float, w_lo: float = 0.0) -> np.ndarray:
    return np.linspace(w_lo, w_hi, n_omega)


def workload(name: str, with_K: bool = True) -> tuple[System, dict]:
    w = dict(WORKLOADS[name])
    sysm = make_system(w["n_atoms"], w["seed"], density=w["density"], with_K=with_K)
    w["omega"] = omega_grid(w["n_omega"], w["w_hi"])
    return sysm, w


def random_complex_vectors(n_rhs: int, n: int, seed: int) -> np.ndarray:
    """n_rhs x n complex test vectors (independent stream per seed)."""
    rng = CounterRNG(seed, 77)
    z = rng.normal(2 * n_rhs * n).reshape(n_rhs, n, 2)
    return z[..., 0] + 1j * z[..., 1]


def batch_sizes(n_mol: int = 32, lo: int = 8, hi: int = 128, seed: int = 4999) -> list[int]:
    """Atom counts of the uneven batch: round(exp(U(ln lo, ln hi))) per molecule."""
    u = CounterRNG(seed, _S_SIZES).uniform(n_mol)
    return [int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * x))) for x in u]


def batch_molecules(n_mol: int = 32, lo: int = 8, hi: int = 128) -> list[System]:
    """The uneven batch: molecule i has seed 4000 + i, atom count from batch_sizes."""
    return [make_system(n, 4000 + i, density=0.0094)
            for i, n in enumerate(batch_sizes(n_mol, lo, hi))]


def workload_system(name: str) -> System:
    """The molecule of a named workload (picklable factory for worker processes)."""
    return workload(name)[0]
