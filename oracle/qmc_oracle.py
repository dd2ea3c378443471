"""Plain FP64 CPU oracle for the variational Monte Carlo local energy.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm) may
import or run this module.  The CUDA library never calls it and shares no
code with it: the two sides only share the seeded input arrays produced by
``qmc_inputs``.

Everything is written with plain PyTorch CPU float64 tensor operations,
vectorised over walkers only; autograd (a library primitive) is used for the
brute-force definitions (Laplacian of Psi, parameter and nuclear
derivatives).  Citations are to the QMCTorch paper (arXiv:2506.09743):

* Eq. (Hmol), Sec. 1 ............ molecular Hamiltonian
* Eq. (psimol), Sec. 2.1 ........ Slater-Jastrow(-backflow) ansatz, backflow map
* Eq. (jastrow), Sec. 2.1 ....... Jastrow factor on the original coordinates
* Eq. (pade_kernel), App. D ..... Pade e-e kernel
* Eq. (nabla_loss), Sec. 2.2 .... low-variance gradient estimator
* Eq. (force), Sec. 2.3 ......... force estimator
* App. F ........................ kinetic decomposition, eqs. (nabla_sigma),
                                  (delta_sigma), Jacobi formula, (nabla_d),
                                  (table), (table_squared)
* App. G ........................ eq. (claudia_trace)
* App. H ........................ eqs. (AX), (BX), (inv_ax)

Readings of points the paper leaves open (listed with their reasons in the
design notes of the repository):

* AO normalisation.  STO: radial factor (2 zeta)^(n+1/2) / sqrt((2n)!) with
  n = kn + l + 1, times the Cartesian angular factor
  sqrt((2l+1)!! / (4 pi (2a-1)!!(2b-1)!!(2c-1)!!)).  GTO primitive:
  (2 alpha/pi)^(3/4) (4 alpha)^(l/2) / sqrt((2a-1)!!(2b-1)!!(2c-1)!!);
  a contracted GTO is sum_p c_p N_p x^a y^b z^c exp(-alpha_p r^2) (no
  renormalisation of the contraction).
* Matrices have electrons as rows and orbitals as columns; excited
  determinants replace hole columns in place by particle columns (eq. AX).
* The det ratio D_X / D_0 equals det(P A0^-1 A_X P) on the k x k hole block.
* An empty spin channel contributes a determinant equal to 1.
* J enters Psi as exp(J) (Eq. psimol); App. F's script-J is exp(J).

Parity status: every function here is pinned by tests in ``tests/`` against
closed forms, finite differences, brute-force differentiation, explicit
matrix inversion or the determinant counts printed in the paper; none is
"parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64


def dfact(n: int) -> int:
    """Double factorial with (-1)!! = 0!! = 1."""
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


class Wavefunction:
    """Torch view of a ``qmc_inputs.Molecule``; parameters may require grad."""

    def __init__(self, mol, requires_grad: bool = False):
        self.mol = mol
        self.n_up, self.n_down = int(mol.n_up), int(mol.n_down)
        self.n_elec = self.n_up + self.n_down
        self.atom_xyz = torch.tensor(mol.atom_xyz, dtype=DT)
        self.atom_z = torch.tensor(mol.atom_z, dtype=DT)
        self.ao_atom = [int(a) for a in mol.ao_atom]
        self.ao_kind = [int(k) for k in mol.ao_kind]
        self.ao_pow = [tuple(int(v) for v in p) for p in mol.ao_pow]
        self.prim_start = [int(s) for s in mol.ao_prim_start]
        self.prim_exp = torch.tensor(mol.prim_exp, dtype=DT)
        self.prim_coef = torch.tensor(mol.prim_coef, dtype=DT)
        self.mo = torch.tensor(mol.mo_coeff, dtype=DT)
        self.det_weight = torch.tensor(mol.det_weight, dtype=DT)
        self.det_exc = np.asarray(mol.det_exc).tolist()
        self.w0_par = float(mol.jastrow_w0_par)
        self.w0_anti = float(mol.jastrow_w0_anti)
        self.jastrow_b = torch.tensor(float(mol.jastrow_b), dtype=DT)
        # many-body Jastrow (App. D); None when absent
        jen = getattr(mol, "jastrow_en", None)
        jeen = getattr(mol, "jastrow_een", None)
        self.jastrow_en = None if jen is None else torch.tensor(np.asarray(jen, dtype=np.float64))
        self.jastrow_een = None if jeen is None else torch.tensor(np.asarray(jeen, dtype=np.float64))
        self.backflow_w = torch.tensor(float(mol.backflow_w), dtype=DT)
        if requires_grad:
            for t in self.params().values():
                t.requires_grad_(True)
            self.atom_xyz.requires_grad_(True)

    def params(self) -> dict:
        """Variational parameters in the library's gradient layout order; the
        many-body Jastrow's (App. D), when present, after the backflow weight:
        K_en (w0, w1, w2), then the K_een terms row by row."""
        p = {
            "exponents": self.prim_exp,
            "mo_coeff": self.mo,
            "det_weight": self.det_weight,
            "jastrow_b": self.jastrow_b,
            "backflow_w": self.backflow_w,
        }
        if self.jastrow_en is not None:
            p["jastrow_en"] = self.jastrow_en
        if self.jastrow_een is not None:
            p["jastrow_een"] = self.jastrow_een
        return p

    @property
    def n_ao(self):
        return len(self.ao_atom)

    @property
    def has_backflow(self) -> bool:
        return float(self.backflow_w.detach()) != 0.0

    def spin_of(self, i: int) -> int:
        return 0 if i < self.n_up else 1

    def occupation(self, n: int, s: int) -> list:
        """Orbital columns of determinant n, spin s: ground orbitals
        0..n_s-1 with holes replaced in place by particles (eq. AX)."""
        n_s = self.n_up if s == 0 else self.n_down
        occ = list(range(n_s))
        rank, h1, h2, p1, p2 = self.det_exc[n][s]
        if rank >= 1:
            occ[h1] = p1
        if rank >= 2:
            occ[h2] = p2
        return occ


# ---------------------------------------------------------------------------
# atomic orbitals (Sec. 2.1: STO N x^kx y^ky z^kz r^kn exp(-zeta r); GTOs)


def ao_norm_sto(zeta, a, b, c, kn):
    l = a + b + c
    n = kn + l + 1
    ang = math.sqrt(dfact(2 * l + 1) / (4.0 * math.pi * dfact(2 * a - 1) * dfact(2 * b - 1) * dfact(2 * c - 1)))
    return (2.0 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n)) * ang


def ao_norm_gto(alpha, a, b, c):
    l = a + b + c
    return (2.0 * alpha / math.pi) ** 0.75 * (4.0 * alpha) ** (l / 2.0) / math.sqrt(
        dfact(2 * a - 1) * dfact(2 * b - 1) * dfact(2 * c - 1))


def _mono(d, p):
    """d_x^p0 d_y^p1 d_z^p2 (zero if any power is negative)."""
    if min(p) < 0:
        return torch.zeros_like(d[..., 0])
    return d[..., 0] ** p[0] * d[..., 1] ** p[1] * d[..., 2] ** p[2]


def _radial(wf, beta, rho):
    """Radial factor f(rho) with normalisation and its derivatives f', f''."""
    a, b, c, kn = wf.ao_pow[beta]
    s, e = wf.prim_start[beta], wf.prim_start[beta + 1]
    if wf.ao_kind[beta] == 0:  # Slater
        zeta = wf.prim_exp[s]
        N = ao_norm_sto(zeta, a, b, c, kn) * wf.prim_coef[s]
        f = N * rho ** kn * torch.exp(-zeta * rho)
        q = kn / rho - zeta
        return f, q * f, (q * q - kn / rho ** 2) * f
    f = f1 = f2 = 0.0
    for p in range(s, e):
        al = wf.prim_exp[p]
        g = wf.prim_coef[p] * ao_norm_gto(al, a, b, c) * torch.exp(-al * rho * rho)
        f = f + g
        f1 = f1 - 2.0 * al * rho * g
        f2 = f2 + (4.0 * al * al * rho * rho - 2.0 * al) * g
    return f, f1, f2


def ao_eval(wf, r, order: int = 0):
    """Atomic orbitals at positions r [W, N, 3].

    order 0 -> values [W, N, n_ao]
    order 1 -> (values, gradients [W, N, n_ao, 3], Laplacians [W, N, n_ao])
    order 2 -> (values, gradients, Laplacians, Hessians [W, N, n_ao, 3, 3])

    phi = P(d) f(|d|) with d = r - R_atom and P = dx^a dy^b dz^c; the
    derivatives are the product and chain rules written out.
    """
    vals, grads, laps, hess = [], [], [], []
    eye = torch.eye(3, dtype=DT)
    for beta in range(wf.n_ao):
        d = r - wf.atom_xyz[wf.ao_atom[beta]]
        rho = torch.sqrt((d * d).sum(-1))
        pw = wf.ao_pow[beta][:3]
        f, f1, f2 = _radial(wf, beta, rho)
        P = _mono(d, pw)
        vals.append(P * f)
        if order == 0:
            continue
        unit = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
        dP = torch.stack([pw[e] * _mono(d, [pw[k] - unit[e][k] for k in range(3)]) for e in range(3)], -1)
        d2P = torch.stack([
            torch.stack([
                pw[e] * (pw[g] - (1 if e == g else 0))
                * _mono(d, [pw[k] - unit[e][k] - unit[g][k] for k in range(3)])
                for g in range(3)], -1)
            for e in range(3)], -2)
        n = d / rho[..., None]
        grads.append(f[..., None] * dP + (P * f1)[..., None] * n)
        dd = n[..., :, None] * n[..., None, :]
        H = (f[..., None, None] * d2P
             + (f1 / rho)[..., None, None] * (dP[..., :, None] * d[..., None, :] + d[..., :, None] * dP[..., None, :])
             + P[..., None, None] * (f2[..., None, None] * dd + (f1 / rho)[..., None, None] * (eye - dd)))
        hess.append(H)
        laps.append(H.diagonal(dim1=-2, dim2=-1).sum(-1))
    v = torch.stack(vals, -1)
    if order == 0:
        return v
    g = torch.stack(grads, -2)
    lp = torch.stack(laps, -1)
    if order == 1:
        return v, g, lp
    return v, g, lp, torch.stack(hess, -3)


# ---------------------------------------------------------------------------
# backflow (Sec. 2.1 and Sec. 3: r~_i = r_i + sum_{j!=i} K(r_ij)(r_i - r_j),
# inverse kernel K = w / r)


def backflow(wf, r):
    """Backflow-transformed positions r~ [W, N, 3]."""
    if wf.n_elec < 2:
        return r
    rij = r[:, :, None, :] - r[:, None, :, :]
    dist = torch.sqrt((rij * rij).sum(-1) + torch.eye(wf.n_elec, dtype=DT))  # unit diagonal, masked below
    eta = wf.backflow_w / dist * (1.0 - torch.eye(wf.n_elec, dtype=DT))
    return r + (eta[..., None] * rij).sum(2)


def backflow_derivs(wf, r):
    """First and diagonal second derivatives of the backflow map.

    Returns (rt, J1, J2) with
      J1[w, i, d, k, e] = d rt_{i,d} / d r_{k,e}
      J2[w, i, d, k, e] = d^2 rt_{i,d} / d r_{k,e}^2
    For g(v) = eta(|v|) v with eta = w/rho:
      dg_d/dv_e     = eta delta_de + eta' v_d v_e / rho
      d2g_d/dv_e^2  = 2 delta_de eta' v_e / rho + eta' v_d / rho
                      + (eta''/rho^2 - eta'/rho^3) v_d v_e^2
    and rt_i = r_i + sum_j g(r_i - r_j).
    """
    W, N, _ = r.shape
    w = wf.backflow_w
    rt = backflow(wf, r)
    eye3 = torch.eye(3, dtype=DT)
    J1 = torch.zeros(W, N, 3, N, 3, dtype=DT)
    J2 = torch.zeros(W, N, 3, N, 3, dtype=DT)
    for i in range(N):
        J1[:, i, :, i, :] = eye3
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            v = r[:, i] - r[:, j]
            rho = torch.sqrt((v * v).sum(-1))
            eta = w / rho
            e1 = -w / rho ** 2
            e2 = 2.0 * w / rho ** 3
            dg = eta[:, None, None] * eye3 + (e1 / rho)[:, None, None] * v[:, :, None] * v[:, None, :]
            d2g = (2.0 * eye3[None] * (e1 / rho)[:, None, None] * v[:, None, :]
                   + (e1 / rho)[:, None, None] * v[:, :, None].expand(W, 3, 3)
                   + (e2 / rho ** 2 - e1 / rho ** 3)[:, None, None] * v[:, :, None] * (v * v)[:, None, :])
            J1[:, i, :, i, :] = J1[:, i, :, i, :] + dg
            J1[:, i, :, j, :] = J1[:, i, :, j, :] - dg
            J2[:, i, :, i, :] = J2[:, i, :, i, :] + d2g
            J2[:, i, :, j, :] = J2[:, i, :, j, :] + d2g
    return rt, J1, J2


# ---------------------------------------------------------------------------
# Jastrow (Eq. jastrow with the Pade e-e kernel, Eq. pade_kernel, App. D)


def _pair_w0(wf):
    N = wf.n_elec
    w0 = torch.empty(N, N, dtype=DT)
    for i in range(N):
        for j in range(N):
            w0[i, j] = wf.w0_par if wf.spin_of(i) == wf.spin_of(j) else wf.w0_anti
    return w0


def jastrow(wf, r):
    """J, grad_i J [W, N, 3] and lap_i J [W, N] for u(r) = w0 r / (1 + b r).

    u' = w0/(1+br)^2,  u'' = -2 w0 b/(1+br)^3,
    grad_i J = sum_j u'(r_ij) r_ij_vec / r_ij,  lap_i J = sum_j u'' + 2u'/r_ij.
    """
    W, N, _ = r.shape
    manybody = wf.jastrow_en is not None or wf.jastrow_een is not None
    if N < 2:
        if manybody:
            return jastrow_manybody(wf, r)
        z = torch.zeros(W, dtype=DT)
        return z, torch.zeros(W, N, 3, dtype=DT), torch.zeros(W, N, dtype=DT)
    b = wf.jastrow_b
    off = 1.0 - torch.eye(N, dtype=DT)
    w0 = _pair_w0(wf) * off
    rij = r[:, :, None, :] - r[:, None, :, :]
    dist = torch.sqrt((rij * rij).sum(-1) + torch.eye(N, dtype=DT))
    den = 1.0 + b * dist
    u = w0 * dist / den
    u1 = w0 / den ** 2
    u2 = -2.0 * w0 * b / den ** 3
    J = 0.5 * u.sum((1, 2))
    gJ = ((u1 / dist)[..., None] * rij).sum(2)
    lJ = (u2 + 2.0 * u1 / dist).sum(2)
    if manybody:
        Jm, gm, lm = jastrow_manybody(wf, r)
        J, gJ, lJ = J + Jm, gJ + gm, lJ + lm
    return J, gJ, lJ


def _rational(a, b, x):
    """f = a x / (1 + b x), f' = a / (1 + b x)^2, f'' = -2 a b / (1 + b x)^3."""
    d = 1.0 + b * x
    return a * x / d, a / d ** 2, -2.0 * a * b / d ** 3


def jastrow_manybody(wf, r):
    """Many-body Jastrow terms of App. D with their electron derivatives.

    Electron-nucleus: K_en(r) = (w0 r + w1 r^2) / (1 + w2 r) summed over atoms
    alpha and electrons i, with r = r_alpha_i;
      K' = (w0 + 2 w1 r + w1 w2 r^2) / (1 + w2 r)^2,  K'' = 2 (w1 - w0 w2) / (1 + w2 r)^3.
    Electron-electron-nucleus: K_een(x, y, z) = sum_mu c_mu f(a1, b1; x)
    f(a2, b2; y) f(a3, b3; z), f(a, b; r) = a r / (1 + b r), with x = r_alpha_i,
    y = r_alpha_j, z = r_ij, summed over atoms and ordered pairs i != j with
    a factor 1/2 (the kernel symmetrised in i and j, so that J is symmetric
    under electron exchange).  Per electron i the gradient and Laplacian
    follow from the chain rule through x, y, z:
      grad_i = sum K_x u_ai + K_z u_ij,
      lap_i  = sum K_xx + 2 K_x / x + K_zz + 2 K_z / z + 2 K_xz (u_ai . u_ij)
    (and the mirror terms for i in the second slot).  Returns J [W],
    grad J [W, N, 3], lap_i J [W, N].
    """
    W, N, _ = r.shape
    J = torch.zeros(W, dtype=DT)
    g = torch.zeros(W, N, 3, dtype=DT)
    lap = torch.zeros(W, N, dtype=DT)
    n_atom = wf.atom_xyz.shape[0]
    ria = r[:, :, None, :] - wf.atom_xyz[None, None, :, :]  # [W, N, A, 3]
    dia = torch.sqrt((ria * ria).sum(-1))  # [W, N, A]
    uia = ria / dia[..., None]
    if wf.jastrow_en is not None:
        w0, w1, w2 = wf.jastrow_en[0], wf.jastrow_en[1], wf.jastrow_en[2]
        d = 1.0 + w2 * dia
        K = (w0 * dia + w1 * dia * dia) / d
        K1 = (w0 + 2.0 * w1 * dia + w1 * w2 * dia * dia) / d ** 2
        K2 = 2.0 * (w1 - w0 * w2) / d ** 3
        J = J + K.sum((1, 2))
        g = g + (K1[..., None] * uia).sum(2)
        lap = lap + (K2 + 2.0 * K1 / dia).sum(2)
    if wf.jastrow_een is not None and N >= 2:
        rij = r[:, :, None, :] - r[:, None, :, :]
        dij = torch.sqrt((rij * rij).sum(-1) + torch.eye(N, dtype=DT))
        uij = rij / dij[..., None]
        for a in range(n_atom):
            for i in range(N):
                for j in range(N):
                    if i == j:
                        continue
                    x, y, z = dia[:, i, a], dia[:, j, a], dij[:, i, j]
                    K = Kx = Ky = Kz = Kxx = Kyy = Kzz = Kxz = Kyz = 0.0
                    for c, a1, b1, a2, b2, a3, b3 in wf.jastrow_een:
                        f1, f1p, f1pp = _rational(a1, b1, x)
                        f2, f2p, f2pp = _rational(a2, b2, y)
                        f3, f3p, f3pp = _rational(a3, b3, z)
                        K = K + c * f1 * f2 * f3
                        Kx = Kx + c * f1p * f2 * f3
                        Ky = Ky + c * f1 * f2p * f3
                        Kz = Kz + c * f1 * f2 * f3p
                        Kxx = Kxx + c * f1pp * f2 * f3
                        Kyy = Kyy + c * f1 * f2pp * f3
                        Kzz = Kzz + c * f1 * f2 * f3pp
                        Kxz = Kxz + c * f1p * f2 * f3p
                        Kyz = Kyz + c * f1 * f2p * f3p
                    ui, uj, u = uia[:, i, a], uia[:, j, a], uij[:, i, j]
                    J = J + 0.5 * K
                    g[:, i] = g[:, i] + 0.5 * (Kx[:, None] * ui + Kz[:, None] * u)
                    g[:, j] = g[:, j] + 0.5 * (Ky[:, None] * uj - Kz[:, None] * u)
                    lap[:, i] = lap[:, i] + 0.5 * (Kxx + 2.0 * Kx / x + Kzz + 2.0 * Kz / z
                                                   + 2.0 * Kxz * (ui * u).sum(-1))
                    lap[:, j] = lap[:, j] + 0.5 * (Kyy + 2.0 * Ky / y + Kzz + 2.0 * Kz / z
                                                   - 2.0 * Kyz * (uj * u).sum(-1))
    return J, g, lap


# ---------------------------------------------------------------------------
# Coulomb potential (Eq. Hmol, Sec. 1)


def potential(wf, r):
    """V_ee + V_en + V_nn per walker [W]."""
    W, N, _ = r.shape
    V = torch.zeros(W, dtype=DT)
    for i in range(N):
        for j in range(i + 1, N):
            V = V + 1.0 / torch.sqrt(((r[:, i] - r[:, j]) ** 2).sum(-1))
    for i in range(N):
        for a in range(wf.atom_z.shape[0]):
            V = V - wf.atom_z[a] / torch.sqrt(((r[:, i] - wf.atom_xyz[a]) ** 2).sum(-1))
    return V + nuclear_repulsion(wf)


def nuclear_repulsion(wf):
    n = wf.atom_z.shape[0]
    v = torch.zeros((), dtype=DT)
    for a in range(n):
        for b in range(a + 1, n):
            v = v + wf.atom_z[a] * wf.atom_z[b] / torch.sqrt(((wf.atom_xyz[a] - wf.atom_xyz[b]) ** 2).sum())
    return v


# ---------------------------------------------------------------------------
# wavefunction value (Eq. psimol)


def _spin_rows(wf, s):
    return list(range(wf.n_up)) if s == 0 else list(range(wf.n_up, wf.n_elec))


def slater_dets(wf, Phi):
    """det A_n^s for every determinant [W, n_det, 2] from the MO matrix
    Phi [W, N, n_mo] (rows electrons, columns orbitals)."""
    W = Phi.shape[0]
    out = torch.ones(W, len(wf.det_exc), 2, dtype=DT)
    for s in range(2):
        rows = _spin_rows(wf, s)
        if not rows:
            continue
        for n in range(len(wf.det_exc)):
            A = Phi[:, rows][:, :, wf.occupation(n, s)]
            out[:, n, s] = torch.linalg.det(A)
    return out


def log_psi(wf, r):
    """(log|Psi|, sign Psi) with Psi = exp(J) sum_n d_n D_n^up D_n^dn.

    The backflow map is always applied (it is the identity at w = 0), so that
    log|Psi| stays differentiable in w there too."""
    rt = backflow(wf, r)
    Phi = ao_eval(wf, rt) @ wf.mo
    D = slater_dets(wf, Phi)
    Sigma = (wf.det_weight * D[..., 0] * D[..., 1]).sum(-1)
    J = jastrow(wf, r)[0]
    return J + torch.log(torch.abs(Sigma)), torch.sign(Sigma)


# ---------------------------------------------------------------------------
# local energy, three ways


def local_energy_ad(wf, r):
    """E_L = -1/2 lap(Psi)/Psi + V by automatic differentiation (brute-force
    definition, Eq. Hmol): lap Psi / Psi = sum_k d_k^2 log|Psi| + (d_k log|Psi|)^2."""
    r = r.detach().clone().requires_grad_(True)
    lp, _ = log_psi(wf, r)
    g = torch.autograd.grad(lp.sum(), r, create_graph=True)[0]
    W, N, _ = r.shape
    lap = torch.zeros(W, dtype=DT)
    for i in range(N):
        for d in range(3):
            h = torch.autograd.grad(g[:, i, d].sum(), r, retain_graph=True)[0][:, i, d]
            lap = lap + h
    kin = lap + (g * g).sum((1, 2))
    return (-0.5 * kin + potential(wf, r)).detach()


def _mo_channels(wf, r):
    """MO values, gradients, Laplacians at r (no backflow): Phi [W,N,M],
    dPhi [W,N,M,3], lPhi [W,N,M]."""
    v, g, lp = ao_eval(wf, r, order=1)
    C = wf.mo
    return v @ C, torch.einsum("wnbd,bm->wnmd", g, C), lp @ C


def slater_derivs_explicit(wf, r):
    """grad_i Sigma / Sigma [W, N, 3] and lap Sigma / Sigma [W] without
    backflow, every determinant inverted explicitly.

    Jacobi formula (App. F): grad_i D / D = sum_m (A^-1)_{m i} grad Phi_{i, m};
    eq. (claudia_trace), App. G: lap D / D = sum_i sum_m (A^-1)_{m i} lap Phi_{i, m};
    eqs. (nabla_sigma), (delta_sigma), App. F, whose up-down cross term
    vanishes because each coordinate belongs to one spin.
    Returns (Sigma, gS, lS).
    """
    Phi, dPhi, lPhi = _mo_channels(wf, r)
    W, N = Phi.shape[:2]
    n_det = len(wf.det_exc)
    D = torch.ones(W, n_det, 2, dtype=DT)
    g = torch.zeros(W, n_det, N, 3, dtype=DT)
    lap = torch.zeros(W, n_det, 2, dtype=DT)
    for s in range(2):
        rows = _spin_rows(wf, s)
        if not rows:
            continue
        for n in range(n_det):
            occ = wf.occupation(n, s)
            A = Phi[:, rows][:, :, occ]
            Ainv = torch.linalg.inv(A)  # [W, m, i]
            D[:, n, s] = torch.linalg.det(A)
            dA = dPhi[:, rows][:, :, occ]  # [W, i, m, 3]
            lA = lPhi[:, rows][:, :, occ]  # [W, i, m]
            g[:, n, rows, :] = torch.einsum("wmi,wimd->wid", Ainv, dA)
            lap[:, n, s] = torch.einsum("wmi,wim->w", Ainv, lA)
    prod = wf.det_weight * D[..., 0] * D[..., 1]  # [W, n_det]
    Sigma = prod.sum(-1)
    wn = prod / Sigma[:, None]
    gS = torch.einsum("wn,wnid->wid", wn, g)
    lS = (wn * (lap[..., 0] + lap[..., 1])).sum(-1)
    return Sigma, gS, lS


def slater_derivs_backflow(wf, r):
    """Per-coordinate first/second derivatives of Sigma with backflow.

    For each electron coordinate x_k: d_k A_{i,m} = sum_d d_d phi_m(rt_i) J1[i,d,k],
    d_k^2 A_{i,m} = sum_{d,e} H_de phi_m(rt_i) J1[i,d,k] J1[i,e,k]
                    + sum_d d_d phi_m(rt_i) J2[i,d,k];
    eq. (nabla_d), App. F:
      d_k^2 D / D = Tr(A^-1 d_k^2 A) + Tr(A^-1 d_k A)^2 - Tr(A^-1 d_k A A^-1 d_k A);
    eqs. (nabla_sigma), (delta_sigma) per coordinate, including the up-down
    cross term.  Returns (Sigma, dS [W, 3N], d2S [W, 3N]) (ratios to Sigma).
    """
    W, N, _ = r.shape
    rt, J1, J2 = backflow_derivs(wf, r)
    v, g, _, H = ao_eval(wf, rt, order=2)
    C = wf.mo
    Phi = v @ C
    dPhi = torch.einsum("wnbd,bm->wnmd", g, C)
    HPhi = torch.einsum("wnbde,bm->wnmde", H, C)
    J1f = J1.reshape(W, N, 3, 3 * N)
    J2f = J2.reshape(W, N, 3, 3 * N)
    dA = torch.einsum("wimd,widk->wkim", dPhi, J1f)  # [W, 3N, N, M]
    d2A = (torch.einsum("wimde,widk,wiek->wkim", HPhi, J1f, J1f)
           + torch.einsum("wimd,widk->wkim", dPhi, J2f))
    n_det = len(wf.det_exc)
    K = 3 * N
    D = torch.ones(W, n_det, 2, dtype=DT)
    a = torch.zeros(W, n_det, 2, K, dtype=DT)
    bterm = torch.zeros(W, n_det, 2, K, dtype=DT)
    for s in range(2):
        rows = _spin_rows(wf, s)
        if not rows:
            continue
        for n in range(n_det):
            occ = wf.occupation(n, s)
            A = Phi[:, rows][:, :, occ]
            Ainv = torch.linalg.inv(A)
            D[:, n, s] = torch.linalg.det(A)
            X1 = torch.einsum("wmi,wkin->wkmn", Ainv, dA[:, :, rows][:, :, :, occ])
            X2 = torch.einsum("wmi,wkin->wkmn", Ainv, d2A[:, :, rows][:, :, :, occ])
            tr1 = X1.diagonal(dim1=-2, dim2=-1).sum(-1)
            tr2 = X2.diagonal(dim1=-2, dim2=-1).sum(-1)
            trsq = torch.einsum("wkmn,wknm->wk", X1, X1)
            a[:, n, s] = tr1
            bterm[:, n, s] = tr2 + tr1 * tr1 - trsq
    prod = wf.det_weight * D[..., 0] * D[..., 1]
    Sigma = prod.sum(-1)
    wn = prod / Sigma[:, None]
    dS = torch.einsum("wn,wnk->wk", wn, a[:, :, 0] + a[:, :, 1])
    d2S = torch.einsum("wn,wnk->wk", wn, bterm[:, :, 0] + 2.0 * a[:, :, 0] * a[:, :, 1] + bterm[:, :, 1])
    return Sigma, dS, d2S


def local_energy(wf, r, return_parts: bool = False):
    """E_L = -1/2 [lap J/J + 2 grad J/J . grad Sigma/Sigma + lap Sigma/Sigma] + V
    (kinetic decomposition, App. F; J-script = exp(J) so
    lap exp(J)/exp(J) = sum_k d_k^2 J + (d_k J)^2), every determinant
    evaluated explicitly.  Returns E_L [W] (and log|Psi|, sign if requested).
    """
    W, N, _ = r.shape
    J, gJ, lJ = jastrow(wf, r)
    if wf.has_backflow:
        Sigma, dS, d2S = slater_derivs_backflow(wf, r)
        gJf = gJ.reshape(W, 3 * N)
        kin = lJ.sum(-1) + (gJf * gJf).sum(-1) + 2.0 * (gJf * dS).sum(-1) + d2S.sum(-1)
    else:
        Sigma, gS, lS = slater_derivs_explicit(wf, r)
        kin = lJ.sum(-1) + (gJ * gJ).sum((1, 2)) + 2.0 * (gJ * gS).sum((1, 2)) + lS
    E = -0.5 * kin + potential(wf, r)
    if return_parts:
        return E, J + torch.log(torch.abs(Sigma)), torch.sign(Sigma)
    return E


# ---------------------------------------------------------------------------
# excited-determinant table method (eqs. table, table_squared, App. F; App. H)


def excited_matrix(A0_full, rank_rec, n_s):
    """Columns of the excited matrix A_X built from the full MO matrix rows
    [.., n_s, n_mo] by in-place column replacement (eq. AX)."""
    occ = list(range(n_s))
    rank, h1, h2, p1, p2 = rank_rec
    if rank >= 1:
        occ[h1] = p1
    if rank >= 2:
        occ[h2] = p2
    return A0_full[..., occ]


def hole_projector_indices(rank_rec):
    rank, h1, h2, _, _ = rank_rec
    return [h1, h2][:rank]


def table_trace(Phi_s, B_s, rec):
    """Tr(A_X^-1 B_X) and D_X/D_0 for one spin channel via eq. (table).

    Phi_s, B_s: [W, n_s, n_mo] MO values and one-body operator applied to
    them.  Tr(A_X^-1 B_X) = Tr(A0^-1 B0) + Tr((P A0^-1 A_X P)^-1 P M P),
    M = A0^-1 B_X - A0^-1 B0 A0^-1 A_X, and D_X/D_0 = det(P A0^-1 A_X P).
    """
    n_s = Phi_s.shape[1]
    A0 = Phi_s[..., :n_s]
    B0 = B_s[..., :n_s]
    A0inv = torch.linalg.inv(A0)
    t0 = torch.einsum("wmi,wim->w", A0inv, B0)
    if rec[0] == 0:
        return t0, torch.ones_like(t0)
    AX = excited_matrix(Phi_s, rec, n_s)
    BX = excited_matrix(B_s, rec, n_s)
    M = A0inv @ BX - A0inv @ B0 @ A0inv @ AX
    idx = hole_projector_indices(rec)
    S = (A0inv @ AX)[:, idx][:, :, idx]
    Mp = M[:, idx][:, :, idx]
    return t0 + torch.einsum("wab,wba->w", torch.linalg.inv(S), Mp), torch.linalg.det(S)


def table_trace_squared(Phi_s, B_s, rec):
    """Tr((A_X^-1 B_X)^2) via eq. (table_squared), App. F / App. H:
    Tr((A0^-1 B0)^2) + Tr((T M)^2) + 2 Tr(A0^-1 B0 M T), T = P (A0^-1 A_X)^-1 P."""
    n_s = Phi_s.shape[1]
    A0 = Phi_s[..., :n_s]
    B0 = B_s[..., :n_s]
    A0inv = torch.linalg.inv(A0)
    X0 = A0inv @ B0
    base = torch.einsum("wab,wba->w", X0, X0)
    if rec[0] == 0:
        return base
    AX = excited_matrix(Phi_s, rec, n_s)
    BX = excited_matrix(B_s, rec, n_s)
    M = A0inv @ BX - X0 @ A0inv @ AX
    idx = hole_projector_indices(rec)
    T = torch.zeros_like(A0inv)
    Tk = torch.linalg.inv((A0inv @ AX)[:, idx][:, :, idx])
    for a, ia in enumerate(idx):
        for b, ib in enumerate(idx):
            T[:, ia, ib] = Tk[:, a, b]
    TM = T @ M
    return base + torch.einsum("wab,wba->w", TM, TM) + 2.0 * torch.einsum("wab,wbc,wca->w", X0, M, T)


def woodbury_inverse(Phi_s, rec):
    """A_X^-1 = A0^-1 - (A0^-1 A_X - I) T A0^-1 (eq. inv_ax, App. H)."""
    n_s = Phi_s.shape[1]
    A0inv = torch.linalg.inv(Phi_s[..., :n_s])
    AX = excited_matrix(Phi_s, rec, n_s)
    idx = hole_projector_indices(rec)
    T = torch.zeros_like(A0inv)
    Tk = torch.linalg.inv((A0inv @ AX)[:, idx][:, :, idx])
    for a, ia in enumerate(idx):
        for b, ib in enumerate(idx):
            T[:, ia, ib] = Tk[:, a, b]
    I = torch.eye(n_s, dtype=DT)
    return A0inv - (A0inv @ AX - I) @ T @ A0inv


def local_energy_table(wf, r):
    """E_L without backflow with every excited determinant handled by
    eq. (table) from the single reference inverse A0^-1 (App. F).

    The operator is applied per coordinate (d_k for the gradient in eq.
    nabla_sigma) and as the Laplacian (eq. delta_sigma with claudia_trace)."""
    W, N, _ = r.shape
    J, gJ, lJ = jastrow(wf, r)
    Phi, dPhi, lPhi = _mo_channels(wf, r)
    n_det = len(wf.det_exc)
    ratio = torch.ones(W, n_det, 2, dtype=DT)
    lap = torch.zeros(W, n_det, 2, dtype=DT)
    grad = torch.zeros(W, n_det, N, 3, dtype=DT)
    D0 = torch.ones(W, 2, dtype=DT)
    for s in range(2):
        rows = _spin_rows(wf, s)
        if not rows:
            continue
        P_s = Phi[:, rows]
        D0[:, s] = torch.linalg.det(P_s[..., :len(rows)])
        for n in range(n_det):
            rec = wf.det_exc[n][s]
            t, R = table_trace(P_s, lPhi[:, rows], rec)
            lap[:, n, s] = t
            ratio[:, n, s] = R
            for li, i in enumerate(rows):
                for d in range(3):
                    Bk = torch.zeros_like(P_s)
                    Bk[:, li] = dPhi[:, i, :, d]
                    grad[:, n, i, d] = table_trace(P_s, Bk, rec)[0]
    prod = wf.det_weight * ratio[..., 0] * ratio[..., 1]
    Sr = prod.sum(-1)
    wn = prod / Sr[:, None]
    gS = torch.einsum("wn,wnid->wid", wn, grad)
    lS = (wn * (lap[..., 0] + lap[..., 1])).sum(-1)
    kin = lJ.sum(-1) + (gJ * gJ).sum((1, 2)) + 2.0 * (gJ * gS).sum((1, 2)) + lS
    return -0.5 * kin + potential(wf, r)


# ---------------------------------------------------------------------------
# conditioning diagnostics (used by tests to separate near-node walkers)


def sensitivity(wf, r):
    """Per-walker amplification of rounding: max over spins of the 1-norm
    condition number of the reference matrix, times the CI cancellation
    factor sum_n |d_n D_n| / |sum_n d_n D_n|."""
    rt = backflow(wf, r) if wf.has_backflow else r
    Phi = ao_eval(wf, rt) @ wf.mo
    W = r.shape[0]
    kappa = torch.ones(W, dtype=DT)
    for s in range(2):
        rows = _spin_rows(wf, s)
        if not rows:
            continue
        A = Phi[:, rows][:, :, : len(rows)]
        k = torch.linalg.cond(A, p=1)
        kappa = torch.maximum(kappa, k)
    D = slater_dets(wf, Phi)
    prod = wf.det_weight * D[..., 0] * D[..., 1]
    cancel = prod.abs().sum(-1) / prod.sum(-1).abs()
    return kappa * cancel


# ---------------------------------------------------------------------------
# gradient and force estimators (Eqs. nabla_loss, force)


def grad_log_psi(wf, r):
    """Per-walker d log|Psi| / d theta for every parameter (autograd),
    returned as a [W, n_param] matrix in ``Wavefunction.params`` order."""
    params = list(wf.params().values())
    for p in params:
        if not p.requires_grad:
            raise ValueError("build the Wavefunction with requires_grad=True")
    W = r.shape[0]
    rows = []
    for w in range(W):
        lp, _ = log_psi(wf, r[w:w + 1])
        gs = torch.autograd.grad(lp.sum(), params, allow_unused=True)
        rows.append(torch.cat([(g if g is not None else torch.zeros_like(p)).reshape(-1)
                               for g, p in zip(gs, params)]))
    return torch.stack(rows)


def energy_grad(wf, r):
    """Mean/variance of E_L, the low-variance gradient (Eq. nabla_loss) and
    the forces (Eq. force) with E_v the batch mean and ln rho = 2 log|Psi|.

    grad = (1/M) sum_m 2 d_theta log|Psi_m| (E_L,m - E_v)
    F_alpha = -(1/M) sum_m [d_alpha E_L,m + (E_L,m - E_v) d_alpha ln rho_m]
    """
    params = list(wf.params().values())
    M = r.shape[0]
    E = local_energy(wf, r)
    lp, _ = log_psi(wf, r)
    Ev = E.mean().detach()
    dE = (E - Ev).detach()
    g = torch.autograd.grad((2.0 * lp * dE).sum() / M, params, allow_unused=True, retain_graph=True)
    grad = torch.cat([(gi if gi is not None else torch.zeros_like(p)).reshape(-1) for gi, p in zip(g, params)])
    fE = torch.autograd.grad(E.sum(), wf.atom_xyz, retain_graph=True)[0]
    flp = torch.autograd.grad((dE * 2.0 * lp).sum(), wf.atom_xyz)[0]
    forces = -(fE + flp) / M
    var = ((E.detach() - Ev) ** 2).mean()
    return Ev, var, grad.detach(), forces.detach()


def energy_grad_sums(wf, r):
    """Raw per-batch sums from which Eq. nabla_loss and Eq. force are
    assembled after the batches of a sharded sample are added together:
    [M, sum E, sum E^2, sum d_theta log|Psi| (n_param), sum E d_theta log|Psi|
    (n_param), sum d_R E (3 n_atom), sum d_R ln rho, sum E d_R ln rho],
    ln rho = 2 log|Psi|, every derivative by autograd."""
    params = list(wf.params().values())
    E = local_energy(wf, r)
    lp, _ = log_psi(wf, r)
    Ed = E.detach()

    def pgrad(y):
        g = torch.autograd.grad(y, params, allow_unused=True, retain_graph=True)
        return torch.cat([(gi if gi is not None else torch.zeros_like(p)).reshape(-1) for gi, p in zip(g, params)])

    s_dlp = pgrad(lp.sum())
    s_edlp = pgrad((Ed * lp).sum())
    s_de = torch.autograd.grad(E.sum(), wf.atom_xyz, retain_graph=True)[0].reshape(-1)
    s_dr = torch.autograd.grad((2.0 * lp).sum(), wf.atom_xyz, retain_graph=True)[0].reshape(-1)
    s_edr = torch.autograd.grad((Ed * 2.0 * lp).sum(), wf.atom_xyz)[0].reshape(-1)
    head = torch.tensor([float(r.shape[0]), float(Ed.sum()), float((Ed * Ed).sum())], dtype=DT)
    return torch.cat([head, s_dlp.detach(), s_edlp.detach(), s_de.detach(), s_dr.detach(), s_edr.detach()])


def assemble_energy_grad(sums, n_param, n_atom):
    """(E_v, variance, gradient, forces) from the sums of energy_grad_sums:
    E_v = S_E / M, var = S_EE / M - E_v^2, grad = 2 (S_E,dlp - E_v S_dlp) / M,
    forces = -(S_dE + S_E,dlnrho - E_v S_dlnrho) / M (Eqs. nabla_loss, force)."""
    M = sums[0]
    ev = sums[1] / M
    var = sums[2] / M - ev * ev
    P, A3 = n_param, 3 * n_atom
    s_dlp, s_edlp = sums[3:3 + P], sums[3 + P:3 + 2 * P]
    s_de, s_dr, s_edr = (sums[3 + 2 * P + k * A3:3 + 2 * P + (k + 1) * A3] for k in range(3))
    grad = 2.0 * (s_edlp - ev * s_dlp) / M
    forces = -(s_de + s_edr - ev * s_dr) / M
    return ev, var, grad, forces.reshape(n_atom, 3)


# ---------------------------------------------------------------------------
# Metropolis-Hastings sampler (App. B: Gaussian proposal, all electrons moved
# at once, accept with probability min(1, |Psi'/Psi|^2))


def metropolis(wf, r, n_steps: int, step: float, seed: int, step_offset: int = 0, first_walker: int = 0):
    """Run n_steps Metropolis steps; returns (r_final, log|Psi| final, n_accept [W]).

    Random numbers come from Philox4x32-10 (oracle.philox) with key = seed
    and counter (block, walker, step_lo, step_hi); Gaussians by Box-Muller in
    FP64; proposal r' = r + step * z; accept iff log u < 2 (log|Psi'| - log|Psi|).
    """
    from .philox import walker_normals_and_uniform

    r = r.detach().clone()
    W, N, _ = r.shape
    widx = np.arange(first_walker, first_walker + W, dtype=np.uint64)
    with torch.no_grad():
        lp, _ = log_psi(wf, r)
        nacc = torch.zeros(W, dtype=torch.int64)
        for t in range(n_steps):
            z, u = walker_normals_and_uniform(seed, widx, step_offset + t, 3 * N)
            prop = r + step * torch.from_numpy(z).reshape(W, N, 3)
            lp_new, _ = log_psi(wf, prop)
            acc = torch.from_numpy(np.log(u)) < 2.0 * (lp_new - lp)
            r = torch.where(acc[:, None, None], prop, r)
            lp = torch.where(acc, lp_new, lp)
            nacc += acc.to(torch.int64)
    return r, lp, nacc
