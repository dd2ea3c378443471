"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *describes* molecules, wavefunction parameters and walker
positions as plain numpy arrays.  It holds none of the arithmetic of the
variational Monte Carlo method (no orbital, determinant, Jastrow, energy or
sampling formula): both the CPU oracle and the CUDA library receive these
arrays and compute everything themselves.

Workloads (shapes follow the four molecules of the QMCTorch paper, Sec. 3 and
App. B; the paper's ADF/DZP basis data and Hartree-Fock orbitals are not
available, so seeded synthetic stand-ins of the same shape are generated):

* ``h2``   - H2, 1 up + 1 down, two 1s STOs (zeta 1.24), one bonding MO,
             Pade e-e Jastrow 0.5 r / (1 + r).
* ``lih``  - LiH, 2 + 2 electrons, 12 double-zeta STOs, random orthonormal
             12x6 MO block, Pade Jastrow b = 1.
* ``li2``  - Li2, 3 + 3 electrons, 20 STOs, inverse backflow w = 0.1.
* ``co``   - CO, 7 + 7 electrons, 58 contracted Cartesian GTOs (5s4p2d per
             atom, 3 primitives), 14 MOs, 100 determinants drawn from the
             (10e, 12o) active space of single and double excitations.

Seeds: walker positions 1, AO exponents 2, MO coefficients 3, CI weights 4,
determinant selection 5.

Conventions shared by both sides (they are data layout, not arithmetic):

* electrons are ordered up first (0 .. n_up-1), then down;
* an AO is (atom, kind, kx, ky, kz, kn) with a list of primitives
  (exponent, contraction coefficient); kind 0 = Slater (one primitive,
  coefficient 1), kind 1 = contracted Cartesian Gaussian;
* determinant n is described per spin by an excitation record
  ``(rank, h1, h2, p1, p2)``: occupied columns h1 (< h2) of the ground-state
  matrix (orbitals 0 .. n_s-1) are replaced in place by virtual orbitals p1
  (< p2); rank 0 is the ground state, unused slots are -1.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

STO = 0
GTO = 1

SEED_WALKERS = 1
SEED_EXPONENTS = 2
SEED_MO = 3
SEED_CI = 4
SEED_DETS = 5


@dataclasses.dataclass
class Molecule:
    """A Slater-Jastrow(-backflow) wavefunction specification (plain arrays)."""

    name: str
    atom_xyz: np.ndarray  # [n_atom, 3] float64, bohr
    atom_z: np.ndarray  # [n_atom] float64, nuclear charges
    n_up: int
    n_down: int
    ao_atom: np.ndarray  # [n_ao] int32
    ao_kind: np.ndarray  # [n_ao] int32, STO or GTO
    ao_pow: np.ndarray  # [n_ao, 4] int32: kx, ky, kz, kn
    ao_prim_start: np.ndarray  # [n_ao + 1] int32 offsets into prim_*
    prim_exp: np.ndarray  # [n_prim] float64 (zeta for STO, alpha for GTO)
    prim_coef: np.ndarray  # [n_prim] float64 contraction coefficients
    mo_coeff: np.ndarray  # [n_ao, n_mo] float64
    det_weight: np.ndarray  # [n_det] float64
    det_exc: np.ndarray  # [n_det, 2, 5] int32 (rank, h1, h2, p1, p2) per spin
    jastrow_w0_par: float = 0.25
    jastrow_w0_anti: float = 0.5
    jastrow_b: float = 1.0
    backflow_w: float = 0.0
    # many-body Jastrow (App. D): electron-nucleus kernel (w0, w1, w2) and
    # electron-electron-nucleus terms [n_terms, 7] = (c, a1, b1, a2, b2, a3, b3);
    # None = absent
    jastrow_en: np.ndarray | None = None
    jastrow_een: np.ndarray | None = None
    # electron -> home atom used to draw initial walker positions
    electron_home: np.ndarray | None = None

    @property
    def n_atom(self) -> int:
        return int(self.atom_xyz.shape[0])

    @property
    def n_elec(self) -> int:
        return self.n_up + self.n_down

    @property
    def n_ao(self) -> int:
        return int(self.ao_atom.shape[0])

    @property
    def n_mo(self) -> int:
        return int(self.mo_coeff.shape[1])

    @property
    def n_det(self) -> int:
        return int(self.det_weight.shape[0])

    @property
    def n_prim(self) -> int:
        return int(self.prim_exp.shape[0])

    def with_geometry(self, atom_xyz: np.ndarray) -> "Molecule":
        return dataclasses.replace(self, atom_xyz=np.ascontiguousarray(atom_xyz, dtype=np.float64))

    def with_bond_scale(self, scale: float) -> "Molecule":
        """Diatomic: stretch the bond about its midpoint by ``scale``."""
        xyz = self.atom_xyz.copy()
        mid = xyz.mean(axis=0)
        return self.with_geometry(mid + (xyz - mid) * scale)


# --------------------------------------------------------------------------
# basis builders (shapes only; normalisation is part of the method)


class _BasisBuilder:
    def __init__(self):
        self.atom, self.kind, self.pow, self.start = [], [], [], [0]
        self.exp, self.coef = [], []

    def add(self, atom, kind, kx, ky, kz, kn, exps, coefs):
        self.atom.append(atom)
        self.kind.append(kind)
        self.pow.append((kx, ky, kz, kn))
        self.exp.extend(float(e) for e in exps)
        self.coef.extend(float(c) for c in coefs)
        self.start.append(len(self.exp))

    def arrays(self):
        return dict(
            ao_atom=np.asarray(self.atom, dtype=np.int32),
            ao_kind=np.asarray(self.kind, dtype=np.int32),
            ao_pow=np.asarray(self.pow, dtype=np.int32).reshape(-1, 4),
            ao_prim_start=np.asarray(self.start, dtype=np.int32),
            prim_exp=np.asarray(self.exp, dtype=np.float64),
            prim_coef=np.asarray(self.coef, dtype=np.float64),
        )


P_SHELL = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
D_SHELL = ((2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1))


def _sto_dz_li_like(bb: _BasisBuilder, atom: int, rng: np.random.Generator, lo=0.5, hi=3.0):
    """Li double-zeta STO set: 1s x2, 2s x2, 2p x2 shells (10 AOs)."""
    z = np.exp(rng.uniform(np.log(lo), np.log(hi), size=6))
    for k in range(2):  # 1s, 1s'
        bb.add(atom, STO, 0, 0, 0, 0, [z[k]], [1.0])
    for k in range(2):  # 2s, 2s'  (r e^{-zeta r})
        bb.add(atom, STO, 0, 0, 0, 1, [z[2 + k]], [1.0])
    for k in range(2):  # 2p, 2p' shells
        for (a, b, c) in P_SHELL:
            bb.add(atom, STO, a, b, c, 0, [z[4 + k]], [1.0])


def _sto_dz_h_like(bb: _BasisBuilder, atom: int, rng: np.random.Generator, lo=0.5, hi=3.0):
    z = np.exp(rng.uniform(np.log(lo), np.log(hi), size=2))
    for k in range(2):
        bb.add(atom, STO, 0, 0, 0, 0, [z[k]], [1.0])


def _gto_5s4p2d(bb: _BasisBuilder, atom: int, rng: np.random.Generator, n_prim=3, lo=0.1, hi=50.0):
    def prims():
        a = np.sort(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_prim)))[::-1]
        c = rng.uniform(0.2, 1.0, size=n_prim)
        return a, c

    for _ in range(5):
        a, c = prims()
        bb.add(atom, GTO, 0, 0, 0, 0, a, c)
    for _ in range(4):
        a, c = prims()
        for (x, y, z) in P_SHELL:
            bb.add(atom, GTO, x, y, z, 0, a, c)
    for _ in range(2):
        a, c = prims()
        for (x, y, z) in D_SHELL:
            bb.add(atom, GTO, x, y, z, 0, a, c)


def random_orthonormal(n_rows: int, n_cols: int, rng: np.random.Generator) -> np.ndarray:
    """First n_cols columns of a Haar-random orthogonal n_rows x n_rows matrix."""
    g = rng.standard_normal((n_rows, n_rows))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q[:, :n_cols])


def electron_homes(atom_z: np.ndarray, n_up: int, n_down: int) -> np.ndarray:
    """Assign electrons to atoms in proportion to Z, alternating spins.

    Electrons are dealt atom by atom with a global up/down alternation; the
    up electrons (in dealing order) become electrons 0..n_up-1 and the down
    electrons n_up..N-1.  Returns the home atom of each electron (ions are
    padded round-robin over the atoms).
    """
    ups, downs = [], []
    c = 0
    for a, z in enumerate(atom_z):
        for _ in range(int(round(z))):
            (ups if c % 2 == 0 else downs).append(a)
            c += 1
    n_atom = len(atom_z)
    ups = (ups + [k % n_atom for k in range(n_up)])[:n_up]
    downs = (downs + [k % n_atom for k in range(n_down)])[:n_down]
    return np.asarray(ups + downs, dtype=np.int32)


# --------------------------------------------------------------------------
# determinant expansions


def ground_exc() -> tuple:
    return (0, -1, -1, -1, -1)


def spin_excitations(n_occ: int, n_orb: int, n_frozen: int = 0):
    """Single and double excitations of one spin channel.

    Occupied orbitals n_frozen .. n_occ-1 may be emptied (holes), virtual
    orbitals n_occ .. n_orb-1 may be filled (particles).  Returns
    (singles, doubles) as lists of excitation records.
    """
    holes = list(range(n_frozen, n_occ))
    parts = list(range(n_occ, n_orb))
    singles = [(1, h, -1, p, -1) for h in holes for p in parts]
    doubles = [
        (2, h1, h2, p1, p2)
        for (h1, h2) in itertools.combinations(holes, 2)
        for (p1, p2) in itertools.combinations(parts, 2)
    ]
    return singles, doubles


def sd_expansion(n_up: int, n_down: int, n_orb: int, n_frozen: int = 0):
    """All determinants of SD(n_e, n_o): ground, singles (either spin),
    same-spin doubles and opposite-spin doubles (an up single times a down
    single).  Returns a list of (up_record, down_record)."""
    su, du = spin_excitations(n_up, n_orb, n_frozen)
    sd, dd = spin_excitations(n_down, n_orb, n_frozen)
    g = ground_exc()
    dets = [(g, g)]
    dets += [(e, g) for e in su] + [(g, e) for e in sd]
    dets += [(e, g) for e in du] + [(g, e) for e in dd]
    dets += [(a, b) for a in su for b in sd]
    return dets


def sd_count(n_elec: int, n_orb: int) -> int:
    """Number of determinants in SD(n_e, n_o) with n_e/2 electrons per spin."""
    return len(sd_expansion(n_elec // 2, n_elec - n_elec // 2, n_orb))


def _select_dets(all_dets, n_keep: int, rng: np.random.Generator):
    """Ground state plus n_keep-1 excitations drawn without replacement."""
    idx = rng.choice(np.arange(1, len(all_dets)), size=n_keep - 1, replace=False)
    idx = np.sort(idx)
    return [all_dets[0]] + [all_dets[i] for i in idx]


def _ci_weights(n_det: int, rng: np.random.Generator, lead: float = 0.95) -> np.ndarray:
    if n_det == 1:
        return np.ones(1)
    d = rng.standard_normal(n_det - 1)
    d *= math.sqrt(1.0 - lead * lead) / np.linalg.norm(d)
    return np.concatenate([[lead], d])


def _dets_array(dets) -> np.ndarray:
    return np.asarray(dets, dtype=np.int32).reshape(len(dets), 2, 5)


# --------------------------------------------------------------------------
# the four molecules


def make_h2(bond: float = 1.4) -> Molecule:
    bb = _BasisBuilder()
    for a in range(2):
        bb.add(a, STO, 0, 0, 0, 0, [1.24], [1.0])
    xyz = np.array([[0.0, 0.0, -bond / 2], [0.0, 0.0, bond / 2]])
    z = np.array([1.0, 1.0])
    mo = np.array([[1.0], [1.0]]) / math.sqrt(2.0)
    return Molecule(
        name="h2", atom_xyz=xyz, atom_z=z, n_up=1, n_down=1, **bb.arrays(), mo_coeff=mo,
        det_weight=np.ones(1), det_exc=_dets_array([(ground_exc(), ground_exc())]),
        jastrow_w0_par=0.25, jastrow_w0_anti=0.5, jastrow_b=1.0, backflow_w=0.0,
        electron_home=electron_homes(z, 1, 1),
    )


def make_lih(bond: float = 3.015) -> Molecule:
    rng = np.random.default_rng(SEED_EXPONENTS)
    bb = _BasisBuilder()
    _sto_dz_li_like(bb, 0, rng)
    _sto_dz_h_like(bb, 1, rng)
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, bond]])
    z = np.array([3.0, 1.0])
    mo = random_orthonormal(12, 6, np.random.default_rng(SEED_MO))
    return Molecule(
        name="lih", atom_xyz=xyz, atom_z=z, n_up=2, n_down=2, **bb.arrays(), mo_coeff=mo,
        det_weight=np.ones(1), det_exc=_dets_array([(ground_exc(), ground_exc())]),
        jastrow_b=1.0, electron_home=electron_homes(z, 2, 2),
    )


def make_li2(bond: float = 5.05, backflow_w: float = 0.1, n_mo: int = 3, n_det: int = 1) -> Molecule:
    """Li2 with backflow; n_det > 1 draws the ground state plus n_det - 1
    excitations of SD(6, n_mo) (all orbitals active)."""
    rng = np.random.default_rng(SEED_EXPONENTS)
    bb = _BasisBuilder()
    _sto_dz_li_like(bb, 0, rng)
    _sto_dz_li_like(bb, 1, rng)
    xyz = np.array([[0.0, 0.0, -bond / 2], [0.0, 0.0, bond / 2]])
    z = np.array([3.0, 3.0])
    mo = random_orthonormal(20, n_mo, np.random.default_rng(SEED_MO))
    if n_det == 1:
        dets = [(ground_exc(), ground_exc())]
    else:
        all_dets = sd_expansion(3, 3, n_mo)
        dets = _select_dets(all_dets, n_det, np.random.default_rng(SEED_DETS)) if n_det < len(all_dets) else all_dets
    return Molecule(
        name="li2" if n_det == 1 else "li2_md", atom_xyz=xyz, atom_z=z, n_up=3, n_down=3, **bb.arrays(),
        mo_coeff=mo, det_weight=_ci_weights(len(dets), np.random.default_rng(SEED_CI)), det_exc=_dets_array(dets),
        jastrow_b=1.0, backflow_w=backflow_w, electron_home=electron_homes(z, 3, 3),
    )


def make_co(bond: float = 2.13, n_det: int = 100) -> Molecule:
    rng = np.random.default_rng(SEED_EXPONENTS)
    bb = _BasisBuilder()
    _gto_5s4p2d(bb, 0, rng)
    _gto_5s4p2d(bb, 1, rng)
    xyz = np.array([[0.0, 0.0, -bond / 2], [0.0, 0.0, bond / 2]])
    z = np.array([6.0, 8.0])
    n_frozen, n_orb = 2, 14  # (10e, 12o) active space above 2 frozen core orbitals per spin
    mo = random_orthonormal(58, n_orb, np.random.default_rng(SEED_MO))
    all_dets = sd_expansion(7, 7, n_orb, n_frozen)
    dets = _select_dets(all_dets, n_det, np.random.default_rng(SEED_DETS)) if n_det < len(all_dets) else all_dets
    w = _ci_weights(len(dets), np.random.default_rng(SEED_CI))
    return Molecule(
        name="co", atom_xyz=xyz, atom_z=z, n_up=7, n_down=7, **bb.arrays(), mo_coeff=mo,
        det_weight=w, det_exc=_dets_array(dets), jastrow_b=1.0,
        electron_home=electron_homes(z, 7, 7),
    )


def make_hydrogenic(zeta: float = 1.0, Z: float = 1.0) -> Molecule:
    """One electron, one nucleus, one 1s STO: a closed-form test system."""
    bb = _BasisBuilder()
    bb.add(0, STO, 0, 0, 0, 0, [zeta], [1.0])
    return Molecule(
        name="h_atom", atom_xyz=np.zeros((1, 3)), atom_z=np.array([Z]), n_up=1, n_down=0,
        **bb.arrays(), mo_coeff=np.ones((1, 1)), det_weight=np.ones(1),
        det_exc=_dets_array([(ground_exc(), ground_exc())]), jastrow_b=1.0,
        electron_home=np.zeros(1, dtype=np.int32),
    )


def make_helium(zeta: float = 27.0 / 16.0, jastrow: bool = False) -> Molecule:
    """He 1s^2 as a product of two 1s(zeta) orbitals; no Jastrow by default
    (both Pade prefactors zero), which has a closed-form local energy."""
    bb = _BasisBuilder()
    bb.add(0, STO, 0, 0, 0, 0, [zeta], [1.0])
    return Molecule(
        name="he", atom_xyz=np.zeros((1, 3)), atom_z=np.array([2.0]), n_up=1, n_down=1,
        **bb.arrays(), mo_coeff=np.ones((1, 1)), det_weight=np.ones(1),
        det_exc=_dets_array([(ground_exc(), ground_exc())]),
        jastrow_w0_par=0.25 if jastrow else 0.0, jastrow_w0_anti=0.5 if jastrow else 0.0,
        jastrow_b=1.0, electron_home=np.zeros(2, dtype=np.int32),
    )


MOLECULES = {"h2": make_h2, "lih": make_lih, "li2": make_li2, "co": make_co}

# walker counts of the four workloads
WORKLOAD_WALKERS = {"h2": 1024, "lih": 65536, "li2": 131072, "co": 262144}


def with_manybody_jastrow(mol: Molecule, n_terms: int = 5, seed: int = 9, en: bool = True) -> Molecule:
    """The molecule with seeded many-body Jastrow parameters (App. D: K_en and
    n_terms electron-electron-nucleus terms).  w0 ~ U(-0.3, -0.1), w1 ~ U(0,
    0.05), w2 ~ U(0.5, 1.5); c ~ N(0, 0.1), a ~ U(0.2, 1), b ~ U(0.5, 2)."""
    rng = np.random.default_rng(seed)
    jen = np.array([rng.uniform(-0.3, -0.1), rng.uniform(0.0, 0.05), rng.uniform(0.5, 1.5)]) if en else None
    een = None
    if n_terms > 0:
        een = np.empty((n_terms, 7))
        een[:, 0] = 0.1 * rng.standard_normal(n_terms)
        een[:, 1::2] = rng.uniform(0.2, 1.0, size=(n_terms, 3))
        een[:, 2::2] = rng.uniform(0.5, 2.0, size=(n_terms, 3))
    return dataclasses.replace(mol, name=mol.name + "_mbj", jastrow_en=jen, jastrow_een=een)


def make_molecule(name: str, **kw) -> Molecule:
    return MOLECULES[name](**kw)


# --------------------------------------------------------------------------
# walkers


def walkers(mol: Molecule, n_walkers: int, seed: int = SEED_WALKERS, sigma: float = 1.0) -> np.ndarray:
    """Initial walker positions [W, N, 3]: electron i ~ N(R_home(i), sigma^2 I)."""
    rng = np.random.default_rng(seed)
    homes = mol.electron_home if mol.electron_home is not None else np.zeros(mol.n_elec, dtype=np.int32)
    centre = mol.atom_xyz[homes]  # [N, 3]
    return centre[None, :, :] + sigma * rng.standard_normal((n_walkers, mol.n_elec, 3))


def to_soa(r: np.ndarray, ldw: int | None = None) -> np.ndarray:
    """[W, N, 3] -> coordinate-major [3N, ldw] (row k = electron k//3, axis k%3)."""
    W, N, _ = r.shape
    ldw = W if ldw is None else ldw
    out = np.zeros((3 * N, ldw), dtype=np.float64)
    out[:, :W] = r.reshape(W, 3 * N).T
    return out


def from_soa(x: np.ndarray, n_walkers: int, n_elec: int) -> np.ndarray:
    """Coordinate-major [3N, ldw] -> [W, N, 3]."""
    return np.ascontiguousarray(x[:, :n_walkers].T.reshape(n_walkers, n_elec, 3))


def serving_requests(n_requests: int, rate_hz: float, seed: int = 7,
                     walker_choices=(4096, 16384, 65536, 262144), n_bonds: int = 20):
    """A seeded request stream: (arrival_s, molecule, bond_scale, n_walkers, seed).

    Molecules are H2, LiH, Li2 and CO, each at 20 bond lengths from 0.6x to
    2.5x equilibrium; walker counts are uniform over ``walker_choices`` and
    arrivals are a Poisson process of the given rate.
    """
    rng = np.random.default_rng(seed)
    scales = np.linspace(0.6, 2.5, n_bonds)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests)) if rate_hz > 0 else np.zeros(n_requests)
    names = list(MOLECULES)
    out = []
    for k in range(n_requests):
        out.append(dict(
            arrival_s=float(t[k]), molecule=names[int(rng.integers(len(names)))],
            bond_scale=float(scales[int(rng.integers(n_bonds))]),
            n_walkers=int(walker_choices[int(rng.integers(len(walker_choices)))]),
            seed=int(rng.integers(1 << 31)),
        ))
    return out
