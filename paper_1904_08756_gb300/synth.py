"""Seeded synthetic inputs for the EPSR hot path (water and amorphous-silica boxes).

This module only *makes inputs*: force-field and grid parameters of the test systems
and initial coordinates on the fixed-point grid. It holds none of the method's
arithmetic (no minimum image, no bins, no energies, no sine transform); both the
CUDA library and the CPU oracle consume what it returns.

Box coordinates use only +, -, *, / and sqrt on IEEE doubles, elementwise (no BLAS,
no transcendental calls), and every random draw comes from a NumPy PCG64 stream, so
the same seed gives bit-identical boxes on x86 and Arm. The one libm call is the
power in `replica_sizes`, whose last-ulp differences vanish in the floor to a
multiple of 3.

Test systems follow the paper's correctness samples (Sec. 3.1): liquid water as a
3-site rigid molecule and amorphous SiO2 as single-atom "molecules". The ISIS
neutron data the paper fits are not available, so these synthetic boxes stand in
for their shapes (density, composition, potentials, bins, Q range).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SCALE_LOG2 = 20                      # fixed-point grid: 2^-20 Angstrom per unit
SCALE = float(1 << SCALE_LOG2)

# Water geometry: O-H 1.0 A, H-O-H 109.47 deg. sin/cos of the half angle, as literals
# (so that no libm call enters the generator).
_SIN_HALF_HOH = 0.8164904309201172
_COS_HALF_HOH = 0.5773589665155304


@dataclass
class System:
    """One periodic box: force field, grids and initial fixed-point coordinates."""
    name: str
    L_fx: int                        # box side in fixed-point units
    xyz: np.ndarray                  # int32 [N, 3], each in [0, L_fx)
    type: np.ndarray                 # int32 [N]
    mol_start: np.ndarray            # int64 [n_mol + 1], molecules are contiguous atom ranges
    type_names: list
    q: list                          # charge per type (e)
    sigma: list                      # LJ sigma per type (A)
    eps: list                        # LJ epsilon per type (kJ/mol)
    b: list                          # coherent scattering length per type (fm)
    r_coul: float = 9.0              # Coulomb cutoff (A)
    bin_p: int = 3                   # bin width = bin_p / bin_q Angstrom
    bin_q: int = 100
    n_bins: int = 333
    temperature: float = 298.0       # K
    rigid_molecules: bool = True     # True: rotate+translate molecules; False: atom moves
    max_translation: float = 0.1     # A
    max_rotation_deg: float = 5.0
    Q: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    seed: int = 0
    flexible: bool = False           # springs between every two atoms of a molecule (bond_k, bond_d)
    bond_k: list | None = None       # [n_types][n_types] spring constant (kJ/mol/A^2)
    bond_d: list | None = None       # [n_types][n_types] reference distance (A)
    r_lj: float = 0.0                # Lennard-Jones cutoff (A); 0: every pair

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_mol(self) -> int:
        return int(self.mol_start.shape[0] - 1)

    @property
    def n_types(self) -> int:
        return len(self.q)

    @property
    def L(self) -> float:
        return self.L_fx / SCALE

    @property
    def dr(self) -> float:
        return self.bin_p / self.bin_q


def box_side_fx(n_atoms: int, density: float) -> int:
    """Cubic side for a number density (atoms / A^3), rounded to the grid."""
    L = (n_atoms / density) ** (1.0 / 3.0)
    return int(round(L * SCALE))


def _rand_quat(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions by rejection from the 4-cube (no libm)."""
    out = np.empty((0, 4))
    while out.shape[0] < n:
        c = rng.random((2 * n + 16, 4)) * 2.0 - 1.0
        s = c[:, 0] * c[:, 0] + c[:, 1] * c[:, 1] + c[:, 2] * c[:, 2] + c[:, 3] * c[:, 3]
        keep = (s > 1e-2) & (s <= 1.0)
        c = c[keep] / np.sqrt(s[keep])[:, None]
        out = np.concatenate([out, c])
    return out[:n]


def _rotate(qt: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Rotate vectors v [B, m, 3] by unit quaternions qt [B, 4] (elementwise only)."""
    w, x, y, z = (qt[:, i][:, None] for i in range(4))
    vx, vy, vz = v[..., 0], v[..., 1], v[..., 2]
    r00 = 1 - 2 * (y * y + z * z); r01 = 2 * (x * y - w * z); r02 = 2 * (x * z + w * y)
    r10 = 2 * (x * y + w * z); r11 = 1 - 2 * (x * x + z * z); r12 = 2 * (y * z - w * x)
    r20 = 2 * (x * z - w * y); r21 = 2 * (y * z + w * x); r22 = 1 - 2 * (x * x + y * y)
    return np.stack([r00 * vx + r01 * vy + r02 * vz,
                     r10 * vx + r11 * vy + r12 * vz,
                     r20 * vx + r21 * vy + r22 * vz], axis=-1)


class _Grid:
    """Cell grid of placed atoms used only to reject overlapping placements."""

    def __init__(self, L_fx: int, cell_A: float, capacity: int, cap: int = 12):
        self.L = L_fx
        self.nc = max(3, int(L_fx // int(cell_A * SCALE)))
        self.cap = cap
        self.cells = np.full((self.nc ** 3, cap), -1, np.int64)
        self.count = np.zeros(self.nc ** 3, np.int64)
        self.pos = np.zeros((capacity, 3), np.int64)
        self.typ = np.zeros(capacity, np.int64)
        self.n = 0
        self.offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1)
                              for c in (-1, 0, 1)])

    def flat_cell(self, p: np.ndarray) -> np.ndarray:
        c = np.minimum((p * self.nc) // self.L, self.nc - 1)
        return (c[..., 0] * self.nc + c[..., 1]) * self.nc + c[..., 2]

    def neighbours(self, p: np.ndarray) -> np.ndarray:
        """Indices of placed atoms in the 27 cells around each position p [K, 3] -> [K, 27*cap]."""
        c = np.minimum((p * self.nc) // self.L, self.nc - 1)
        nb = (c[:, None, :] + self.offs[None]) % self.nc
        flat = (nb[..., 0] * self.nc + nb[..., 1]) * self.nc + nb[..., 2]
        return self.cells[flat].reshape(p.shape[0], -1)

    def insert(self, p: np.ndarray, t: np.ndarray):
        """Insert atoms p [K, 3] with types t [K] (in order)."""
        k0 = self.n
        self.pos[k0:k0 + len(p)] = p
        self.typ[k0:k0 + len(p)] = t
        self.n += len(p)
        for i, f in enumerate(self.flat_cell(p)):
            k = self.count[f]
            if k >= self.cap:
                raise RuntimeError("cell capacity exceeded while placing atoms")
            self.cells[f, k] = k0 + i
            self.count[f] = k + 1


def _wrapped_sep2(a: np.ndarray, b: np.ndarray, L: int) -> np.ndarray:
    """Squared separation on the periodic grid, used only for the placement test."""
    d = np.abs(a - b)                # both in [0, L), so |a - b| < L
    d = np.minimum(d, L - d)
    return (d * d).sum(axis=-1)


def _rsa(L_fx: int, n_units: int, unit_types: list, unit_offsets_A: np.ndarray | None,
         min_sep_A, rng: np.random.Generator, cell_A: float) -> np.ndarray:
    """Random sequential addition of rigid units (reading c8: no overlaps below min_sep).

    min_sep_A(ta, tb) -> minimum intermolecular separation in A for a type pair.
    Returns int64 [n_units * m, 3] positions in [0, L_fx), units in placement order.
    """
    m = len(unit_types)
    grid = _Grid(L_fx, cell_A, n_units * m)
    thr = np.zeros((8, 8), np.int64)
    for ta in set(unit_types):
        for tb in set(unit_types):
            thr[ta, tb] = int(math.ceil((min_sep_A(ta, tb) * SCALE) ** 2))
    ut = np.asarray(unit_types, np.int64)
    lim_uu = thr[ut[:, None], ut[None, :]]
    reach = 0.0 if unit_offsets_A is None else float(np.sqrt((unit_offsets_A ** 2).sum(1)).max())
    reach_A = max(min_sep_A(a, b) for a in ut for b in ut) + 2 * reach
    n_placed = 0
    attempts = 0
    batch = 1024
    while n_placed < n_units:
        attempts += batch
        if attempts > 200 * n_units + 100000:
            raise RuntimeError("random sequential addition did not converge")
        centre = rng.integers(0, L_fx, size=(batch, 3), dtype=np.int64)
        if unit_offsets_A is None:
            atoms = centre[:, None, :]
        else:
            qt = _rand_quat(rng, batch)
            off = _rotate(qt, np.broadcast_to(unit_offsets_A, (batch,) + unit_offsets_A.shape))
            atoms = (centre[:, None, :] + np.rint(off * SCALE).astype(np.int64)) % L_fx
        flat = atoms.reshape(-1, 3)
        ok = np.ones(batch, bool)
        if grid.n:
            nb = grid.neighbours(flat)                      # [batch*m, 27*cap]
            ri, ci = np.nonzero(nb >= 0)                    # compress to occupied slots
            other = nb[ri, ci]
            d2 = _wrapped_sep2(flat[ri], grid.pos[other], L_fx)
            lim = thr[np.tile(ut, batch)[ri], grid.typ[other]]
            bad_atom = np.zeros(batch * m, bool)
            bad_atom[ri[d2 < lim]] = True
            ok &= ~bad_atom.reshape(batch, m).any(axis=1)
        cand = np.nonzero(ok)[0]
        # conflicts among this batch's surviving candidates: only centres within `reach`
        # of each other can clash, found through a throw-away grid of the candidates.
        blocked_by = {}
        if len(cand) > 1:
            cc = centre[cand]
            cg = _Grid(L_fx, max(reach_A, L_fx / SCALE / 12.0), len(cand), cap=256)
            cg.insert(cc, np.zeros(len(cand), np.int64))
            nb = cg.neighbours(cc)
            rows = np.broadcast_to(np.arange(len(cand))[:, None], nb.shape)
            sel = (nb >= 0) & (nb < rows)
            bi, ai = rows[sel], nb[sel]
            if len(bi):
                d2 = _wrapped_sep2(atoms[cand[ai]][:, :, None, :], atoms[cand[bi]][:, None, :, :],
                                   L_fx)
                clash = (d2 < lim_uu[None]).any(axis=(1, 2))
                for a, b in zip(ai[clash], bi[clash]):
                    blocked_by.setdefault(int(b), []).append(int(a))
        accepted = []
        acc_set = set()
        for k in range(len(cand)):
            if any(a in acc_set for a in blocked_by.get(k, ())):
                continue
            acc_set.add(k)
            accepted.append(cand[k])
            if n_placed + len(accepted) == n_units:
                break
        if accepted:
            A = atoms[np.asarray(accepted)].reshape(-1, 3)
            grid.insert(A, np.tile(ut, len(accepted)))
            n_placed += len(accepted)
    return grid.pos[:n_units * m].copy()


def water_geometry_A() -> np.ndarray:
    """O at the origin, two H at 1.0 A with an H-O-H angle of 109.47 degrees."""
    return np.array([[0.0, 0.0, 0.0],
                     [_SIN_HALF_HOH, _COS_HALF_HOH, 0.0],
                     [-_SIN_HALF_HOH, _COS_HALF_HOH, 0.0]])


def water_box(n_mol: int, seed: int, L_A: float | None = None, density: float = 0.1,
              n_bins: int = 333, bin_p: int = 3, bin_q: int = 100,
              Q: np.ndarray | None = None) -> System:
    """Rigid 3-site water (O, H, H) at random positions and orientations.

    Potentials: LJ O-O eps 0.65 kJ/mol sigma 3.166 A (H has eps 0), charges O -0.8476 e,
    H +0.4238 e, Coulomb cut at 9 A; b_O 5.803 fm, b_H -3.739 fm; T = 298 K; moves of at
    most 0.1 A and 5 degrees. Placement keeps intermolecular O-O >= 2.3 A and any
    intermolecular atom pair >= 1.0 A.
    """
    n_atoms = 3 * n_mol
    L_fx = int(round(L_A * SCALE)) if L_A is not None else box_side_fx(n_atoms, density)
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = _rsa(L_fx, n_mol, [0, 1, 1], water_geometry_A(),
               lambda a, b: 2.3 if (a == 0 and b == 0) else 1.0, rng, cell_A=2.3)
    typ = np.tile(np.array([0, 1, 1], np.int32), n_mol)
    if Q is None:
        Q = 0.1 + np.arange(1000) * (29.9 / 999.0)
    return System(name="water", L_fx=L_fx, xyz=pos.astype(np.int32), type=typ,
                  mol_start=np.arange(0, n_atoms + 1, 3, dtype=np.int64),
                  type_names=["O", "H"], q=[-0.8476, 0.4238], sigma=[3.166, 0.0],
                  eps=[0.65, 0.0], b=[5.803, -3.739], r_coul=9.0, bin_p=bin_p, bin_q=bin_q,
                  n_bins=n_bins, temperature=298.0, rigid_molecules=True,
                  max_translation=0.1, max_rotation_deg=5.0, Q=np.asarray(Q, np.float64),
                  seed=seed)


def water_lattice(n_mol: int, seed: int, density: float = 0.1) -> System:
    """Rigid 3-site water for large boxes: O atoms on the first n_mol sites of a simple cubic
    lattice of side k = ceil(n_mol^(1/3)) in the box of the given density, each molecule in
    a random orientation. Same potentials, moves and bins as water_box.

    With O on the sites, two molecules' atoms are at least (spacing - 2 A) apart, so the
    intermolecular bounds of water_box (O-O >= 2.3 A, any pair >= 1.0 A) hold whenever the
    spacing is at least 3 A, without rejection; the generator refuses smaller spacings. It
    builds 10^7 molecules in seconds, where random sequential addition would take hours.
    """
    n_atoms = 3 * n_mol
    L_fx = box_side_fx(n_atoms, density)
    k = 1
    while k * k * k < n_mol:
        k += 1
    spacing_fx = L_fx // k
    if spacing_fx < 3 * SCALE:
        raise ValueError(f"lattice spacing {spacing_fx / SCALE:.3f} A below 3 A for {n_mol} molecules")
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.arange(n_mol, dtype=np.int64)
    sites = np.stack([idx % k, (idx // k) % k, idx // (k * k)], axis=1) * spacing_fx
    xyz = np.empty((n_atoms, 3), np.int64)
    geom = water_geometry_A()
    chunk = 1 << 20
    for c0 in range(0, n_mol, chunk):
        c1 = min(n_mol, c0 + chunk)
        qt = _rand_quat(rng, c1 - c0)
        off = np.rint(_rotate(qt, np.broadcast_to(geom, (c1 - c0,) + geom.shape)) * SCALE).astype(np.int64)
        xyz[3 * c0:3 * c1] = ((sites[c0:c1, None, :] + off) % L_fx).reshape(-1, 3)
    base = water_box(1, seed=0, L_A=L_fx / SCALE)
    return System(**{**base.__dict__, "L_fx": L_fx, "xyz": xyz.astype(np.int32),
                     "type": np.tile(np.array([0, 1, 1], np.int32), n_mol),
                     "mol_start": np.arange(0, n_atoms + 1, 3, dtype=np.int64), "seed": seed})


def flexible_water_box(n_mol: int, seed: int, L_A: float | None = None, k_spring: float = 2000.0,
                       density: float = 0.1) -> System:
    """Flexible 3-site water: the placement, potentials and bins of water_box, with the
    molecule held together by springs k (r - d)^2 between every two of its atoms (O-H with
    d = 1.0 A, H-H with d = the reference H-H distance) instead of being rigid; moves are
    molecule translations, molecule rotations and single-atom translations."""
    base = water_box(n_mol, seed=seed, L_A=L_A, density=density)
    d_hh = 2.0 * _SIN_HALF_HOH
    return System(**{**base.__dict__, "name": "flexible water", "rigid_molecules": False, "flexible": True,
                     "bond_k": [[0.0, k_spring], [k_spring, k_spring]],
                     "bond_d": [[0.0, 1.0], [1.0, d_hh]]})


def silica_box(n_si: int, seed: int, density: float = 0.0662, n_bins: int = 600,
               bin_p: int = 2, bin_q: int = 100, Q: np.ndarray | None = None) -> System:
    """Amorphous SiO2 as single atoms: RSA with 1.5 A minimum separation.

    Potentials: LJ Si eps 0.175 sigma 0.42, O eps 0.65 sigma 3.6 (kJ/mol, A); charges
    Si +2 e, O -1 e, Coulomb cut at 9 A; b_Si 4.149 fm, b_O 5.803 fm; T = 300 K; single
    atom moves of at most 0.1 A. Atoms are ordered Si first, then O.
    """
    n_o = 2 * n_si
    n_atoms = n_si + n_o
    L_fx = box_side_fx(n_atoms, density)
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = _rsa(L_fx, n_atoms, [0], None, lambda a, b: 1.5, rng, cell_A=1.5)
    typ = np.concatenate([np.zeros(n_si, np.int32), np.ones(n_o, np.int32)])
    if Q is None:
        Q = 0.3 + np.arange(2000) * (39.7 / 1999.0)
    return System(name="silica", L_fx=L_fx, xyz=pos.astype(np.int32), type=typ,
                  mol_start=np.arange(0, n_atoms + 1, dtype=np.int64),
                  type_names=["Si", "O"], q=[2.0, -1.0], sigma=[0.42, 3.6],
                  eps=[0.175, 0.65], b=[4.149, 5.803], r_coul=9.0, bin_p=bin_p, bin_q=bin_q,
                  n_bins=n_bins, temperature=300.0, rigid_molecules=False,
                  max_translation=0.1, max_rotation_deg=0.0, Q=np.asarray(Q, np.float64),
                  seed=seed)


def uniform_gas(n_atoms: int, L_A: float, seed: int, n_types: int = 2) -> System:
    """Uncorrelated uniform atoms (ideal gas) with zero potentials, types alternating."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L_fx = int(round(L_A * SCALE))
    xyz = rng.integers(0, L_fx, size=(n_atoms, 3), dtype=np.int64).astype(np.int32)
    typ = (np.arange(n_atoms) % n_types).astype(np.int32)
    z = [0.0] * n_types
    return System(name="gas", L_fx=L_fx, xyz=xyz, type=typ,
                  mol_start=np.arange(0, n_atoms + 1, dtype=np.int64),
                  type_names=[f"T{i}" for i in range(n_types)], q=list(z), sigma=list(z),
                  eps=list(z), b=[5.0 + i for i in range(n_types)], r_coul=9.0,
                  bin_p=1, bin_q=10, n_bins=min(100, int(L_A * 5)), temperature=300.0,
                  rigid_molecules=False, max_translation=0.1, max_rotation_deg=0.0,
                  Q=0.5 + np.arange(200) * 0.1, seed=seed)


def lj_fluid(n_side: int, seed: int, density: float = 0.021, sigma: float = 3.4, eps: float = 1.0,
             temperature: float = 120.0, max_translation: float = 0.3, n_bins: int = 333) -> System:
    """A one-type Lennard-Jones liquid (argon-like by default): n_side^3 atoms on a simple cubic
    lattice of the given density, each displaced uniformly by up to 1/4 of the spacing, no
    charges; single-atom moves; 0.03 A bins and Q on 0.3-20 1/A. The refinement loop's test
    system: it equilibrates in a few sweeps, and one pair means one dataset fixes it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_side ** 3
    L_fx = box_side_fx(n, density)
    a = L_fx / n_side
    g = np.stack(np.meshgrid(np.arange(n_side), np.arange(n_side), np.arange(n_side), indexing="ij"),
                 axis=-1).reshape(-1, 3).astype(np.float64)
    jit = rng.uniform(-0.25, 0.25, size=(n, 3))
    xyz = (np.floor((g + 0.5 + jit) * a).astype(np.int64) % L_fx).astype(np.int32)
    return System(name="lj-fluid", L_fx=L_fx, xyz=xyz, type=np.zeros(n, np.int32),
                  mol_start=np.arange(0, n + 1, dtype=np.int64), type_names=["Ar"], q=[0.0],
                  sigma=[sigma], eps=[eps], b=[1.909], r_coul=9.0, bin_p=3, bin_q=100, n_bins=n_bins,
                  temperature=temperature, rigid_molecules=False, max_translation=max_translation,
                  max_rotation_deg=0.0, Q=0.3 + np.arange(400) * (19.7 / 399.0), seed=seed)


# ----------------------------------------------------------------------------------------
# Named workloads (the paper-shaped test systems)
# ----------------------------------------------------------------------------------------

def small_water() -> System:
    """900-atom water box, side 20.8 A, seed 0 (runs through the oracle in seconds)."""
    return water_box(300, seed=0, L_A=20.8)


def paper_water(seed: int = 1) -> System:
    """33,333-molecule (99,999-atom) water box at 0.1 atoms/A^3, seed 1."""
    return water_box(33333, seed=seed)


def paper_silica(seed: int = 2) -> System:
    """33,000 Si + 66,000 O at 0.0662 atoms/A^3, 0-12 A in 0.02 A bins, seed 2."""
    return silica_box(33000, seed=seed)


def replica_sizes(n_boxes: int = 64, seed: int = 3, lo: int = 2000, hi: int = 60000) -> list:
    """Atom counts log-uniform on [lo, hi], rounded down to a multiple of 3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(n_boxes)
    # log-uniform via exp of a uniform in log space would need libm; draw the exponent
    # instead as lo * (hi/lo)^u evaluated with np.power on fixed inputs (same on all
    # platforms within 1 ulp; the floor to a multiple of 3 absorbs it except on exact ties).
    sizes = np.floor(lo * np.power(hi / lo, u))
    return [int(s) // 3 * 3 for s in sizes]


def replica_batch(n_boxes: int = 64, seed: int = 3, sizes: list | None = None) -> list:
    """Uneven replica boxes: first half water, second half silica, 600 x 0.02 A bins and
    the 2000-point Q grid 0.3-40 1/A for all."""
    if sizes is None:
        sizes = replica_sizes(n_boxes, seed)
    Q = 0.3 + np.arange(2000) * (39.7 / 1999.0)
    out = []
    for i, n in enumerate(sizes):
        s = seed * 1000 + i
        if i < n_boxes // 2:
            out.append(water_box(n // 3, seed=s, n_bins=600, bin_p=2, bin_q=100, Q=Q))
        else:
            out.append(silica_box(n // 3, seed=s, n_bins=600, bin_p=2, bin_q=100, Q=Q))
    return out


def lattice_box(n_side: int, a_fx: int, n_bins: int, bin_p: int, bin_q: int) -> System:
    """Simple-cubic lattice with spacing a_fx grid units (one type, no potentials)."""
    g = np.arange(n_side, dtype=np.int64) * a_fx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.int32)
    n = xyz.shape[0]
    return System(name="lattice", L_fx=n_side * a_fx, xyz=xyz, type=np.zeros(n, np.int32),
                  mol_start=np.arange(0, n + 1, dtype=np.int64), type_names=["X"], q=[0.0],
                  sigma=[0.0], eps=[0.0], b=[5.0], r_coul=9.0, bin_p=bin_p, bin_q=bin_q,
                  n_bins=n_bins, temperature=300.0, rigid_molecules=False,
                  max_translation=0.1, max_rotation_deg=0.0, Q=np.array([1.0]), seed=0)
