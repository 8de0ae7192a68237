"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the potential itself: only lattices, random displacements,
species, strains, velocities and random parameters.  Both the CUDA path and the FP64 oracle take
their inputs from here, so the two sides see bit-identical data.

The paper trains and runs on DFT datasets (Sec. 4-6: bcc Mo, fcc Al, Ag-Pd alloys in small fcc,
bcc and hcp cells) that are not available; the recipes below reproduce their shapes: periodic
cells of 8-256 atoms (and large supercells for MD), 1-3 species, R_cut = 5 Angstrom.
All randomness comes from numpy.random.default_rng(seed); "N(0, s)" means standard deviation s.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# conventional / primitive cells: (fractional basis, lattice rows for lattice parameter a)
def _fcc(a):
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
    return basis, np.eye(3) * a


def _bcc(a):
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0.5]], dtype=np.float64)
    return basis, np.eye(3) * a


def _hcp(a, c_over_a=1.633):
    basis = np.array([[0, 0, 0], [1.0 / 3.0, 2.0 / 3.0, 0.5]], dtype=np.float64)
    cell = np.array([[a, 0, 0], [-0.5 * a, 0.5 * math.sqrt(3.0) * a, 0], [0, 0, c_over_a * a]])
    return basis, cell


LATTICES = {"fcc": lambda: _fcc(3.6), "bcc": lambda: _bcc(3.2), "hcp": lambda: _hcp(2.55)}


def supercell(kind_or_cell, reps):
    """Positions [n,3] and cell rows [3,3] of an n1 x n2 x n3 supercell."""
    basis, cell = kind_or_cell
    n1, n2, n3 = reps
    grid = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    frac = (grid[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = frac @ cell
    big = cell * np.array([[n1], [n2], [n3]], dtype=np.float64)
    return pos, big


@dataclass
class Config:
    """One periodic configuration: positions [n,3] (Angstrom), types [n] int32, cell rows [3,3]."""

    pos: np.ndarray
    types: np.ndarray
    cell: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class Batch:
    """Many configurations packed atom-wise (CSR over configurations)."""

    pos: np.ndarray  # [N,3] float64
    types: np.ndarray  # [N] int32
    cells: np.ndarray  # [K,3,3] float64
    cfg_off: np.ndarray  # [K+1] int32

    @property
    def n_cfg(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    def config(self, k: int) -> Config:
        a, b = int(self.cfg_off[k]), int(self.cfg_off[k + 1])
        return Config(self.pos[a:b], self.types[a:b], self.cells[k])


def pack(configs) -> Batch:
    off = np.zeros(len(configs) + 1, dtype=np.int32)
    off[1:] = np.cumsum([c.n for c in configs])
    return Batch(np.concatenate([c.pos for c in configs]).astype(np.float64),
                 np.concatenate([c.types for c in configs]).astype(np.int32),
                 np.stack([c.cell for c in configs]).astype(np.float64), off)


@dataclass
class Params:
    """Hyper-parameters and parameters theta = {xi, c} of one potential."""

    lev_max: int
    n_species: int
    n_radial: int  # N_Q
    r_min: float
    r_cut: float
    xi: np.ndarray  # [m]
    c: np.ndarray  # [S, S, N_mu, N_Q]


def n_mu(lev_max: int) -> int:
    """Number of radial functions f_mu: M_{mu,0} has level 2 + 4 mu <= lev_max."""
    return (lev_max - 2) // 4 + 1


def random_params(lev_max, n_species, n_radial, r_min, r_cut, m, seed, xi_std=1e-2, c_std=0.1):
    """xi ~ N(0, xi_std), c ~ N(0, c_std); m is the basis size of lev_max."""
    rng = np.random.default_rng(seed)
    xi = rng.normal(0.0, xi_std, size=m)
    c = rng.normal(0.0, c_std, size=(n_species, n_species, n_mu(lev_max), n_radial))
    return Params(lev_max, n_species, n_radial, r_min, r_cut, xi, c)


def labels_from_level_table(table):
    """Moment labels [(mu, nu), ...] of every basis function, read from a canonical level table
    (format of mtp_level_table: [m, then per function: level, n_components, then per component:
    n, mu_0, nu_0, ..., then the upper triangle of its adjacency])."""
    t = list(table)
    m = t[0]
    pos = 1
    out = []
    for _ in range(m):
        pos += 1  # level
        ncomp = t[pos]
        pos += 1
        labs = []
        for _ in range(ncomp):
            n = t[pos]
            for u in range(n):
                labs.append((t[pos + 1 + 2 * u], t[pos + 2 + 2 * u]))
            pos += 1 + 2 * n + n * (n - 1) // 2
        out.append(labs)
    return out


def scaled_params(lev_max, n_species, n_radial, r_min, r_cut, labels, seed, xi_std=1e-2, c_std=0.1,
                  n_bar=40.0, f_bar=0.5, r_bar=2.6, radial_decay=1.0):
    """Random parameters whose terms xi_alpha B_alpha are of order xi_std at neighbourhoods like the
    workloads' (about n_bar neighbours at distance r_bar, radial functions of size f_bar): each
    basis function's coefficient is divided by prod over its moments of n_bar f_bar r_bar^nu.
    Used for the lev_max-20 workloads, where the plain recipe gives energies of 1e25 eV.
    radial_decay < 1 damps the Chebyshev coefficient of order b by radial_decay^b: smooth radial
    functions, for molecular dynamics (with undamped random coefficients the fcc lattice collapses
    within ~100 fs at lev_max 16-20 and 1 fs steps no longer resolve the collisions)."""
    rng = np.random.default_rng(seed)
    scale = np.array([np.prod([n_bar * f_bar * r_bar ** nu for _, nu in labs]) for labs in labels])
    xi = rng.normal(0.0, xi_std, size=len(labels)) / scale
    c = rng.normal(0.0, c_std, size=(n_species, n_species, n_mu(lev_max), n_radial))
    c = c * radial_decay ** np.arange(n_radial)
    return Params(lev_max, n_species, n_radial, r_min, r_cut, xi, c)


def perturbed(kind, reps, sigma, rng, n_species=1, species_frac=None):
    base = LATTICES[kind]() if isinstance(kind, str) else kind
    pos, cell = supercell(base, reps)
    pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    n = pos.shape[0]
    if n_species == 1:
        types = np.zeros(n, dtype=np.int32)
    else:
        types = rng.choice(n_species, size=n, p=species_frac).astype(np.int32)
    return Config(pos, types, cell)


# ---------------------------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------------------------
def bcc_128(seed=1):
    """bcc 4x4x4 conventional cells, a = 3.2, 128 atoms, Gaussian displacements sigma = 0.1."""
    rng = np.random.default_rng(seed)
    return perturbed("bcc", (4, 4, 4), 0.1, rng)


def fcc_binary(reps=16, seed=2, sigma=0.15):
    """fcc reps^3 conventional cells (a = 3.6; 16^3 -> 16,384 atoms), 2 species 50/50, sigma 0.15."""
    rng = np.random.default_rng(seed)
    return perturbed("fcc", (reps, reps, reps), sigma, rng, n_species=2)


def fcc_ternary(reps=64, seed=5, sigma=0.0):
    """fcc reps^3 (64^3 -> 1,048,576 atoms), 3 species, random 1/3 occupancy."""
    rng = np.random.default_rng(seed)
    return perturbed("fcc", (reps, reps, reps), sigma, rng, n_species=3)


def _reps_for(n_target, atoms_per_cell, cell):
    """Smallest near-isotropic repetition n1 x n2 x n3 with atoms_per_cell * n1 n2 n3 >= n_target."""
    lens = np.linalg.norm(cell, axis=1)
    best = None
    for n1 in range(1, 12):
        for n2 in range(1, 12):
            for n3 in range(1, 12):
                k = atoms_per_cell * n1 * n2 * n3
                if k < n_target:
                    continue
                ext = np.array([n1, n2, n3]) * lens
                key = (k, ext.max() / ext.min())
                if best is None or key < best[0]:
                    best = (key, (n1, n2, n3))
    return best[1]


def random_small_config(rng, n_lo, n_hi, species_pool=(0, 1, 2), max_species=3):
    """One cell: N log-uniform in [n_lo, n_hi]; lattice fcc/bcc/hcp; strain (I + eps),
    eps symmetric with entries U(-0.05, 0.05); displacements sigma ~ U(0.1, 0.3);
    1..max_species species drawn from species_pool with uniform occupancy."""
    n_target = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    kind = ["fcc", "bcc", "hcp"][rng.integers(3)]
    basis, cell = LATTICES[kind]()
    reps = _reps_for(n_target, basis.shape[0], cell)
    pos, big = supercell((basis, cell), reps)
    if pos.shape[0] > n_target:  # random vacancies down to the target size
        keep = np.sort(rng.choice(pos.shape[0], size=n_target, replace=False))
        pos = pos[keep]
    e = rng.uniform(-0.05, 0.05, size=(3, 3))
    eps = 0.5 * (e + e.T)
    strain = np.eye(3) + eps
    pos = pos @ strain.T
    big = big @ strain.T
    sigma = rng.uniform(0.1, 0.3)
    pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    k = int(rng.integers(1, max_species + 1))
    species = np.sort(rng.choice(species_pool, size=k, replace=False))
    types = species[rng.integers(k, size=pos.shape[0])].astype(np.int32)
    return Config(pos, types, big, {"kind": kind, "sigma": sigma, "reps": reps})


def small_cells(n_cfg=4096, n_lo=8, n_hi=256, seed=3, max_species=3):
    """Batched workload: n_cfg random small cells (defaults: 4096 cells of 8-256 atoms, 1-3 species)."""
    rng = np.random.default_rng(seed)
    return pack([random_small_config(rng, n_lo, n_hi, max_species=max_species) for _ in range(n_cfg)])


def training_cells(n_cfg=2048, n_lo=32, n_hi=128, seed=4):
    """Training-loss workload: n_cfg cells of 32-128 atoms, 3 species present in the batch."""
    rng = np.random.default_rng(seed)
    return pack([random_small_config(rng, n_lo, n_hi) for _ in range(n_cfg)])


def maxwell_velocities(types, masses, temperature_k, seed):
    """Velocities (Angstrom/fs) drawn from the Maxwell distribution, centre-of-mass motion removed.
    masses in amu; k_B T / m converted with 1 amu Angstrom^2 / fs^2 = 103.6427 eV."""
    rng = np.random.default_rng(seed)
    kT = 8.617333262e-5 * temperature_k
    m = np.asarray(masses, dtype=np.float64)[types]
    v = rng.normal(size=(types.shape[0], 3)) * np.sqrt(kT / (m * 103.6427))[:, None]
    p = (m[:, None] * v).sum(0)
    v -= p / m.sum()
    return v


def rotation(seed, reflect=False):
    """A random orthogonal matrix (a proper rotation, or an improper one when reflect)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    if reflect:
        q[:, 2] = -q[:, 2]
    return q
