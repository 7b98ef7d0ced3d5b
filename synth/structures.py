"""Seeded random periodic structures that stand in for the paper's datasets.

The paper benchmarks on bulk Si, liquid methane, CH3SO3H in phenol, CSD-1000r and QM9 (Sec. 'Datasets'). None of
those are available here, so every workload is drawn from a named generator: numpy's PCG64 bit generator with a
fixed seed. Positions come from sequential random insertion, uniform in the cell, rejecting any trial closer than
d_min (minimum image) to an atom already accepted. Species are drawn uniformly or as an exact-ratio shuffle.

Nothing in this module computes any part of the method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class System:
    """A batch of structures in the flat layout both the oracle and the C-ABI take.

    positions      [N][3] float64, Å, as given (not wrapped)
    species        [N] int32 atomic labels (e.g. atomic numbers)
    cells          [n_structures][3][3] float64, rows are the cell vectors h1, h2, h3
    pbc            [n_structures][3] int32, 1 = periodic along that cell vector
    struct_offsets [n_structures + 1] int32, atoms of structure s are struct_offsets[s]:struct_offsets[s+1]
    hypers         the expansion parameters of the workload
    """

    positions: np.ndarray
    species: np.ndarray
    cells: np.ndarray
    pbc: np.ndarray
    struct_offsets: np.ndarray
    hypers: dict = field(default_factory=dict)
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])

    @property
    def n_structures(self) -> int:
        return int(self.cells.shape[0])

    def structure_of_atom(self) -> np.ndarray:
        out = np.empty(self.n_atoms, dtype=np.int32)
        for s in range(self.n_structures):
            out[self.struct_offsets[s]:self.struct_offsets[s + 1]] = s
        return out

    def subset(self, structures) -> "System":
        """A new System holding only the listed structures, in that order."""
        pos, spe, cel, pb, offs = [], [], [], [], [0]
        for s in structures:
            a, b = self.struct_offsets[s], self.struct_offsets[s + 1]
            pos.append(self.positions[a:b])
            spe.append(self.species[a:b])
            cel.append(self.cells[s])
            pb.append(self.pbc[s])
            offs.append(offs[-1] + (b - a))
        return System(np.concatenate(pos), np.concatenate(spe).astype(np.int32), np.stack(cel), np.stack(pb).astype(np.int32),
                      np.asarray(offs, dtype=np.int32), dict(self.hypers), self.name + "-subset")


def _min_image_frac(df: np.ndarray) -> np.ndarray:
    return df - np.round(df)


def random_cell_atoms(n_atoms: int, cell: np.ndarray, d_min: float, rng: np.random.Generator,
                      max_trials_per_atom: int = 20000) -> np.ndarray:
    """Sequential random insertion in a periodic cell with minimum-image rejection closer than d_min.

    A grid of bins at least d_min wide (in fractional units along each axis) restricts each check to the
    27 surrounding bins. The minimum image is taken in fractional coordinates, which is exact for the
    orthogonal cells the workloads use and a conservative approximation for skewed ones.
    """
    cell = np.asarray(cell, dtype=np.float64)
    inv = np.linalg.inv(cell)
    vol = abs(np.linalg.det(cell))
    widths = np.array([vol / np.linalg.norm(np.cross(cell[(k + 1) % 3], cell[(k + 2) % 3])) for k in range(3)])
    nb = np.maximum(1, np.floor(widths / max(d_min, 1e-9)).astype(int))
    nb = np.minimum(nb, 64)
    grid: dict = {}
    frac = np.empty((n_atoms, 3))
    pos = np.empty((n_atoms, 3))
    count = 0
    trials = 0
    d2min = d_min * d_min
    while count < n_atoms:
        trials += 1
        if trials > max_trials_per_atom * n_atoms:
            raise RuntimeError("random insertion did not converge; density too high for d_min")
        s = rng.random(3)
        b = np.floor(s * nb).astype(int) % nb
        cand = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((b[0] + dx) % nb[0], (b[1] + dy) % nb[1], (b[2] + dz) % nb[2])
                    lst = grid.get(key)
                    if lst:
                        cand.extend(lst)
        if cand:
            cand = np.unique(np.asarray(cand))
            df = _min_image_frac(frac[cand] - s)
            d = df @ cell
            if np.min(np.einsum("ij,ij->i", d, d)) < d2min:
                continue
        frac[count] = s
        pos[count] = s @ cell
        grid.setdefault((b[0], b[1], b[2]), []).append(count)
        count += 1
    _ = inv
    return pos


def _species_uniform(n: int, labels, rng) -> np.ndarray:
    return np.asarray(labels, dtype=np.int32)[rng.integers(0, len(labels), size=n)]


def _species_ratio(n: int, labels, ratio, rng) -> np.ndarray:
    ratio = np.asarray(ratio, dtype=np.float64)
    counts = np.floor(n * ratio / ratio.sum()).astype(int)
    counts[0] += n - counts.sum()
    arr = np.concatenate([np.full(c, lab, dtype=np.int32) for c, lab in zip(counts, labels)])
    rng.shuffle(arr)
    return arr


def _single(positions, species, L, hypers, name) -> System:
    return System(np.ascontiguousarray(positions, dtype=np.float64), np.ascontiguousarray(species, dtype=np.int32),
                  (np.eye(3) * L)[None].copy(), np.ones((1, 3), dtype=np.int32),
                  np.array([0, len(positions)], dtype=np.int32), hypers, name)


# Workload hypers. smooth_width is the cosine cutoff width; ps_norm keeps the (2l+1)^-1/2 factor of the
# nu=2 invariant (Eq. nu2-basis-coupled).
HYPERS_TINY = dict(r_cut=5.0, sigma=0.5, n_max=8, l_max=6, smooth_width=0.5, species=[14])
HYPERS_BATCH = dict(r_cut=5.0, sigma=0.5, n_max=12, l_max=9, smooth_width=0.5, species=[1, 6, 7, 8])
HYPERS_DIFF = dict(r_cut=5.5, sigma=0.4, n_max=8, l_max=6, smooth_width=0.5, species=[1, 6])
HYPERS_LARGE = dict(r_cut=6.0, sigma=0.5, n_max=10, l_max=8, smooth_width=0.5, species=[1, 6, 8])
HYPERS_MLP = dict(r_cut=6.0, sigma=0.5, n_max=16, l_max=12, smooth_width=0.5, species=[1, 5, 6, 7, 8, 9, 15, 16])


def config_tiny(seed: int = 1) -> System:
    """1 cubic cell, L = 10 Å, 64 atoms of one species, d_min 2.0 Å."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = 10.0
    pos = random_cell_atoms(64, np.eye(3) * L, 2.0, rng)
    return _single(pos, np.full(64, 14, dtype=np.int32), L, dict(HYPERS_TINY), "tiny")


def config_batch(seed: int = 2, n_structures: int = 512) -> System:
    """n_structures cubic cells with N_s ~ U{64..216} atoms at 0.05 atoms/Å^3, 4 species uniform, d_min 1.8 Å."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos, spe, cells, offs = [], [], [], [0]
    for _ in range(n_structures):
        n = int(rng.integers(64, 217))
        L = (n / 0.05) ** (1.0 / 3.0)
        pos.append(random_cell_atoms(n, np.eye(3) * L, 1.8, rng))
        spe.append(_species_uniform(n, HYPERS_BATCH["species"], rng))
        cells.append(np.eye(3) * L)
        offs.append(offs[-1] + n)
    return System(np.concatenate(pos), np.concatenate(spe).astype(np.int32), np.stack(cells),
                  np.ones((n_structures, 3), dtype=np.int32), np.asarray(offs, dtype=np.int32),
                  dict(HYPERS_BATCH), "batch")


def config_diff(seed: int = 3) -> System:
    """1 cubic cell, 4096 atoms at 0.05 atoms/Å^3, 2 species 1:1, d_min 1.8 Å."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 4096
    L = (n / 0.05) ** (1.0 / 3.0)
    pos = random_cell_atoms(n, np.eye(3) * L, 1.8, rng)
    spe = _species_ratio(n, HYPERS_DIFF["species"], [1, 1], rng)
    return _single(pos, spe, L, dict(HYPERS_DIFF), "diff")


def config_large(seed: int = 5) -> System:
    """1 cubic cell, 32768 atoms at 0.1 atoms/Å^3, 3 species 2:1:1, d_min 1.0 Å."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 32768
    L = (n / 0.1) ** (1.0 / 3.0)
    pos = random_cell_atoms(n, np.eye(3) * L, 1.0, rng)
    spe = _species_ratio(n, HYPERS_LARGE["species"], [2, 1, 1], rng)
    return _single(pos, spe, L, dict(HYPERS_LARGE), "large")


def config_mlp(seed: int = 6) -> System:
    """1 cubic cell, 8192 atoms at 0.06 atoms/Å^3, 8 species uniform, d_min 1.6 Å."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 8192
    L = (n / 0.06) ** (1.0 / 3.0)
    pos = random_cell_atoms(n, np.eye(3) * L, 1.6, rng)
    spe = _species_uniform(n, HYPERS_MLP["species"], rng)
    return _single(pos, spe, L, dict(HYPERS_MLP), "mlp")


CONFIGS = {
    "tiny": config_tiny,
    "batch": config_batch,
    "diff": config_diff,
    "large": config_large,
    "mlp": config_mlp,
}


def small_cell_system(seed: int = 11, n_atoms: int = 6, L: float = 4.0, skew: float = 0.3, d_min: float = 1.2,
                      hypers: dict | None = None) -> System:
    """A triclinic cell narrower than r_cut, so that atoms see several of their own periodic images.

    Positions are drawn and then displaced by whole cell vectors, so they are not wrapped into the cell.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cell = np.array([[L, 0.0, 0.0], [skew * L, L * 1.1, 0.0], [0.2 * L, -skew * L, L * 0.95]])
    pos = random_cell_atoms(n_atoms, cell, d_min, rng)
    pos = pos + rng.integers(-2, 3, size=(n_atoms, 3)) @ cell
    hyp = dict(HYPERS_TINY) if hypers is None else dict(hypers)
    labels = hyp["species"]
    spe = _species_uniform(n_atoms, labels, rng)
    return System(pos, spe, cell[None].copy(), np.ones((1, 3), dtype=np.int32), np.array([0, n_atoms], dtype=np.int32),
                  hyp, "small-cell")


def mlp_initial_params(hidden: int, n_out: int, seed: int = 21) -> np.ndarray:
    """Seeded initial parameters of the 1 -> H -> H -> F network, flattened as [W1 | b1 | W2 | b2 | W3 | b3].

    W1 ~ N(0, 4) spreads the first-layer kinks over t in [0, 1]; b1 ~ U(-2, 2); W2, W3 ~ N(0, 1/H); biases 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.standard_normal(hidden) * 2.0
    b1 = rng.uniform(-2.0, 2.0, hidden)
    W2 = rng.standard_normal((hidden, hidden)) / np.sqrt(hidden)
    W3 = rng.standard_normal((n_out, hidden)) / np.sqrt(hidden)
    return np.concatenate([W1, b1, W2.ravel(), np.zeros(hidden), W3.ravel(), np.zeros(n_out)]).astype(np.float32)


def mlp_training_draws(n_samples: int, r_max: float, batch: int, steps: int, seed: int = 22):
    """Seeded training distances r ~ U[0, r_max] (both end points included) and the minibatch order: a fresh
    permutation of the samples per epoch, concatenated to cover `steps` batches."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(0.0, r_max, n_samples)
    r[0], r[1] = 0.0, r_max
    need = batch * steps
    order = np.concatenate([rng.permutation(n_samples) for _ in range(max(1, -(-need // n_samples)))])[:max(need, batch)]
    return r, order.astype(np.int64)


def linear_weights(n_species: int, n_features: int, seed: int = 4) -> np.ndarray:
    """Gaussian N(0,1) weights of the additive linear energy model, one row per centre species."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n_species, n_features))


def gpr_sparse_draws(species: np.ndarray, labels, n_per_species: int, seed: int = 31):
    """Seeded choice of sparse points for a GPR model: `n_per_species` atoms of each label (all of them if fewer),
    whose environments serve as the active set, and regression weights x_I ~ N(0, 1). Returns (atom indices, x)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = []
    for lab in labels:
        cand = np.flatnonzero(species == lab)
        idx.append(rng.choice(cand, size=min(n_per_species, cand.size), replace=False) if cand.size else cand)
    idx = np.sort(np.concatenate(idx)).astype(np.int64)
    return idx, rng.standard_normal(idx.size)
