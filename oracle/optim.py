"""Plain FP64 CPU oracle of the wavefunction optimisation loop and of the
batched, axis-symmetrised force estimate.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU baseline and reference arm) may import or run this
module; the CUDA library shares no code with it.

* ADAM (the optimiser of App. B), written from its published definition
  (Kingma and Ba, "Adam: a method for stochastic optimization", ICLR 2015,
  Algorithm 1): with gradient g_t at step t = 1, 2, ...
      m_t = beta1 m_{t-1} + (1 - beta1) g_t
      v_t = beta2 v_{t-1} + (1 - beta2) g_t^2
      mhat = m_t / (1 - beta1^t),  vhat = v_t / (1 - beta2^t)
      theta_t = theta_{t-1} - lr mhat / (sqrt(vhat) + eps)
  Every operation is one IEEE operation in this order (beta^t by repeated
  multiplication), so a device implementation that rounds each operation
  the same way agrees bit for bit.
* The loop of App. B: walkers equilibrated by Metropolis, then per
  optimisation step the energy gradient (Eq. nabla_loss) at the current
  samples, one ADAM update of the parameters, and a resampling of the
  walkers with the updated wavefunction (App. B: 500 Metropolis steps).
* Forces along a dissociation curve (Sec. 3.3): the samples are split into
  batches, each batch is symmetrised about the molecular (z) axis, and the
  force of Eq. force is evaluated per batch; the spread over batches gives
  the error bar.  Symmetrisation reading: every sample is joined by its
  images under the two reflections through planes containing the axis
  (x -> -x, y -> -y) and their product (a rotation by pi), all electrons
  together, i.e. the C2v subgroup of the axis' symmetry group.
"""
import numpy as np
import torch

from . import qmc_oracle as O


def adam_step(theta, m, v, g, t: int, lr: float, beta1: float, beta2: float, eps: float):
    """One ADAM update (Kingma and Ba, Algorithm 1); float64 numpy arrays in,
    new (theta, m, v) out.  t counts from 1."""
    theta, m, v, g = (np.asarray(a, dtype=np.float64) for a in (theta, m, v, g))
    b1t = 1.0
    b2t = 1.0
    for _ in range(t):
        b1t *= beta1
        b2t *= beta2
    c1 = 1.0 - b1t
    c2 = 1.0 - b2t
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * (g * g)
    mhat = m / c1
    vhat = v / c2
    theta = theta - (lr * mhat) / (np.sqrt(vhat) + eps)
    return theta, m, v


def params_vector(wf) -> np.ndarray:
    """The variational parameters in the library's gradient layout."""
    return torch.cat([p.detach().reshape(-1) for p in wf.params().values()]).numpy().copy()


def molecule_with_params(mol, theta):
    """A copy of the molecule whose variational parameters are theta
    (exponents, MO coefficients, CI weights, Jastrow b, backflow w)."""
    import dataclasses

    k = 0
    n = mol.prim_exp.shape[0]
    prim_exp = theta[k:k + n].copy(); k += n
    n = mol.mo_coeff.size
    mo = theta[k:k + n].reshape(mol.mo_coeff.shape).copy(); k += n
    n = mol.det_weight.shape[0]
    det_w = theta[k:k + n].copy(); k += n
    b = float(theta[k]); k += 1
    w = float(theta[k]); k += 1
    return dataclasses.replace(mol, prim_exp=prim_exp, mo_coeff=mo, det_weight=det_w, jastrow_b=b, backflow_w=w)


def optimize(mol, r0, n_iter: int, n_equil: int, n_resample: int, step: float, seed: int, lr: float = 1e-2,
             beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, mask=None):
    """The optimisation loop of App. B.  Returns (history [n_iter][3] =
    (E mean, E variance, acceptance of the resampling), final theta, final
    walkers).  Metropolis steps are counted globally: equilibration uses
    steps 0 .. n_equil-1, the resampling after update t the next n_resample."""
    r = torch.as_tensor(r0, dtype=torch.float64)
    wf = O.Wavefunction(mol)
    W = r.shape[0]
    r, _, _ = O.metropolis(wf, r, n_equil, step, seed, step_offset=0)
    theta = params_vector(wf)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    msk = np.ones_like(theta) if mask is None else np.asarray(mask, dtype=np.float64)
    hist = []
    offset = n_equil
    for t in range(1, n_iter + 1):
        wfg = O.Wavefunction(molecule_with_params(mol, theta), requires_grad=True)
        Ev, var, g, _ = O.energy_grad(wfg, r)
        g = g.numpy() * msk
        new, m_new, v_new = adam_step(theta, m, v, g, t, lr, beta1, beta2, eps)
        theta = np.where(msk > 0, new, theta)
        m = np.where(msk > 0, m_new, m)
        v = np.where(msk > 0, v_new, v)
        wf = O.Wavefunction(molecule_with_params(mol, theta))
        r, _, nacc = O.metropolis(wf, r, n_resample, step, seed, step_offset=offset)
        offset += n_resample
        acc = float(nacc.sum()) / (W * n_resample) if n_resample > 0 else 0.0
        hist.append((float(Ev), float(var), acc))
    return np.asarray(hist), theta, r


def axis_images(r):
    """The sample and its images under x -> -x, y -> -y and both (all
    electrons together): [4W, N, 3] in the order identity, x, y, xy."""
    r = torch.as_tensor(r, dtype=torch.float64)
    out = []
    for sx, sy in ((1.0, 1.0), (-1.0, 1.0), (1.0, -1.0), (-1.0, -1.0)):
        s = torch.tensor([sx, sy, 1.0], dtype=torch.float64)
        out.append(r * s)
    return torch.cat(out, dim=0)


def force_batches(mol, r, n_batches: int, symmetrize: bool):
    """Per-batch (E mean, forces [n_atom, 3]) of Eq. force, batches being
    consecutive equal slices of the walkers (the last one takes the rest),
    each optionally symmetrised about the z axis (axis_images)."""
    r = torch.as_tensor(r, dtype=torch.float64)
    W = r.shape[0]
    per = W // n_batches
    out_e, out_f = [], []
    for b in range(n_batches):
        lo = b * per
        hi = W if b == n_batches - 1 else lo + per
        rb = r[lo:hi]
        if symmetrize:
            rb = axis_images(rb)
        wf = O.Wavefunction(mol, requires_grad=True)
        Ev, _, _, F = O.energy_grad(wf, rb)
        out_e.append(float(Ev))
        out_f.append(F.numpy())
    return np.asarray(out_e), np.asarray(out_f)
