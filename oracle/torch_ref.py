"""Independent FP64 restatement of the GMNN model in plain PyTorch CPU ops.

TEST INFRASTRUCTURE.  Written separately from ``gm_oracle.c``: the moments are built with
einsum over all neighbours, the features with einsum over explicit index lists, and every
derivative (forces, virial, the force-matching parameter gradient) comes from autograd
instead of a hand-derived chain rule.  It cross-checks the C oracle on small systems.

Model (section "Machine Learning Interatomic Potentials"; readings as in gm_oracle.c):
    Psi_{i,L,s} = sum_j R_s(r_ij) rhat^{(x)L}        (Eq. basis_fn)
    G_i         = 8 contraction families              (Eq. contraction)
    E_i         = sigma_Z NN(G_i) + mu_Z              (Eq. scale_shift)
    E           = sum_i E_i                           (Eq. energy_sum)
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch

NAMES = ("beta", "W1", "b1", "W2", "b2", "w3", "b3", "sigma", "mu")


def feature_index_lists(nr=5):
    """(family, s-tuple) in feature order: family-major, lexicographic within."""
    out = [(1, (s,)) for s in range(nr)]
    for fam in (2, 3, 4):
        out += [(fam, t) for t in itertools.combinations_with_replacement(range(nr), 2)]
    out += [(5, t) for t in itertools.combinations_with_replacement(range(nr), 3)]
    out += [(6, t) for t in itertools.product(range(nr), repeat=3) if t[0] <= t[2]]
    out += [(7, t) for t in itertools.product(range(nr), repeat=3) if t[0] <= t[1]]
    out += [(8, t) for t in itertools.product(range(nr), repeat=3)]
    return out


def _features(P0, P1, P2, P3, nr):
    """Stack the invariants of Eq. contraction for every atom: [N, n_features]."""
    cols = []
    for fam, s in feature_index_lists(nr):
        if fam == 1:
            cols.append(P0[:, s[0]])
        elif fam == 2:
            cols.append(torch.einsum("na,na->n", P1[:, s[0]], P1[:, s[1]]))
        elif fam == 3:
            cols.append(torch.einsum("nab,nab->n", P2[:, s[0]], P2[:, s[1]]))
        elif fam == 4:
            cols.append(torch.einsum("nabc,nabc->n", P3[:, s[0]], P3[:, s[1]]))
        elif fam == 5:
            cols.append(torch.einsum("nab,nbc,nca->n", P2[:, s[0]], P2[:, s[1]], P2[:, s[2]]))
        elif fam == 6:
            cols.append(torch.einsum("na,nab,nb->n", P1[:, s[0]], P2[:, s[1]], P1[:, s[2]]))
        elif fam == 7:
            cols.append(torch.einsum("nabc,nabd,ncd->n", P3[:, s[0]], P3[:, s[1]], P2[:, s[2]]))
        else:
            cols.append(torch.einsum("na,nabc,nbc->n", P1[:, s[0]], P3[:, s[1]], P2[:, s[2]]))
    return torch.stack(cols, dim=1)


def model_energy(pos, strain, params, desc, species, atom_ptr, cell, pairs):
    """Per-structure energies, per-atom energies, moments and features.

    pos [N,3], strain [B,3,3] (applied as x -> x (I + strain_b)), params: dict of tensors,
    pairs: (i, j, shift[P,3]) int64 tensors.  All FP64.
    """
    i, j, sh = pairs
    N = pos.shape[0]
    B = cell.shape[0]
    counts = atom_ptr[1:] - atom_ptr[:-1]
    sid = torch.repeat_interleave(torch.arange(B), counts)
    eye = torch.eye(3, dtype=torch.float64)
    defo = eye + strain                                    # [B,3,3]
    x = torch.einsum("na,nab->nb", pos, defo[sid])
    cl = torch.einsum("bka,bac->bkc", cell, defo)          # strained lattice vectors
    d = x[j] - x[i] + torch.einsum("pk,pkc->pc", sh.to(torch.float64), cl[sid[i]])
    r = torch.sqrt((d * d).sum(1))
    u = d / r[:, None]
    nb, nr, rc, rmin = desc["n_basis"], desc["n_radial"], desc["r_cut"], desc["r_min"]
    if desc.get("basis", "gaussian") == "bessel":
        # Kocer et al.: a_k [j0((k+1) pi r / r_c) + j0((k+2) pi r / r_c)], j0(x) = sin x / x
        k = torch.arange(nb, dtype=torch.float64)
        a = (-1.0) ** k * math.sqrt(2.0) * math.pi / rc ** 1.5 * (k + 1) * (k + 2) / torch.sqrt((k + 1) ** 2 + (k + 2) ** 2)
        x1 = (k[None, :] + 1) * math.pi * r[:, None] / rc
        x2 = (k[None, :] + 2) * math.pi * r[:, None] / rc
        phi = a[None, :] * (torch.sin(x1) / x1 + torch.sin(x2) / x2)
    else:
        mu_k = torch.tensor([rmin + k * (rc - rmin) / (nb - 1) for k in range(nb)], dtype=torch.float64)
        gamma = nb * nb / (rc * rc)
        phi = torch.exp(-gamma * (r[:, None] - mu_k[None, :]) ** 2)
    fc = torch.where(r < rc, 0.5 * (torch.cos(math.pi * r / rc) + 1.0), torch.zeros_like(r))
    beta = params["beta"][species[i], species[j]]          # [P, nr, nb]
    R = fc[:, None] * torch.einsum("psk,pk->ps", beta, phi) / math.sqrt(nb)
    P0 = torch.zeros(N, nr, dtype=torch.float64).index_add(0, i, R)
    P1 = torch.zeros(N, nr, 3, dtype=torch.float64).index_add(0, i, torch.einsum("ps,pa->psa", R, u))
    P2 = torch.zeros(N, nr, 3, 3, dtype=torch.float64).index_add(
        0, i, torch.einsum("ps,pa,pb->psab", R, u, u))
    P3 = torch.zeros(N, nr, 3, 3, 3, dtype=torch.float64).index_add(
        0, i, torch.einsum("ps,pa,pb,pc->psabc", R, u, u, u))
    G = _features(P0, P1, P2, P3, nr)
    phi_act = torch.tanh if desc["activation"] == "tanh" else torch.nn.functional.silu
    a1 = phi_act(G @ params["W1"] + params["b1"])
    a2 = phi_act(a1 @ params["W2"] + params["b2"])
    nn = a2 @ params["w3"] + params["b3"][0]
    Ea = params["sigma"][species] * nn + params["mu"][species]
    E = torch.zeros(B, dtype=torch.float64).index_add(0, sid, Ea)
    return E, Ea, (P0, P1, P2, P3), G


def _tensors(batch, nl, params):
    n = batch.n_atoms
    i = torch.from_numpy(np.repeat(np.arange(n), np.diff(nl.row_ptr))).long()
    j = torch.from_numpy(nl.col.astype(np.int64))
    sh = torch.from_numpy(nl.shift.astype(np.int64))
    pt = {k: torch.tensor(np.asarray(params[k]), dtype=torch.float64) for k in NAMES}
    return (i, j, sh), pt


def energy_forces(batch, desc, params, nl):
    """E [B], E_atom [N], F [N,3], virial [B,3,3] (= -dE/dstrain) via autograd."""
    pairs, pt = _tensors(batch, nl, params)
    pos = torch.tensor(batch.pos, dtype=torch.float64, requires_grad=True)
    strain = torch.zeros(batch.n_structures, 3, 3, dtype=torch.float64, requires_grad=True)
    cell = torch.tensor(batch.cell, dtype=torch.float64)
    E, Ea, _, G = model_energy(pos, strain, pt, desc, torch.from_numpy(batch.species.astype(np.int64)),
                               torch.from_numpy(batch.atom_ptr.astype(np.int64)), cell, pairs)
    gpos, gstr = torch.autograd.grad(E.sum(), (pos, strain))
    return {"E": E.detach().numpy(), "E_atom": Ea.detach().numpy(), "F": -gpos.numpy(),
            "virial": -gstr.numpy(), "G": G.detach().numpy()}


def loss_param_grad(batch, desc, params, nl, E_ref, F_ref, wE=1.0, wF=1.0):
    """Force-matching loss and its gradient with respect to every parameter (autograd
    double backward through F = -dE/dr)."""
    pairs, pt = _tensors(batch, nl, params)
    for v in pt.values():
        v.requires_grad_(True)
    pos = torch.tensor(batch.pos, dtype=torch.float64, requires_grad=True)
    strain = torch.zeros(batch.n_structures, 3, 3, dtype=torch.float64)
    cell = torch.tensor(batch.cell, dtype=torch.float64)
    ap = torch.from_numpy(batch.atom_ptr.astype(np.int64))
    E, _, _, _ = model_energy(pos, strain, pt, desc, torch.from_numpy(batch.species.astype(np.int64)),
                              ap, cell, pairs)
    (gpos,) = torch.autograd.grad(E.sum(), pos, create_graph=True)
    F = -gpos
    nat = (ap[1:] - ap[:-1]).to(torch.float64)
    Eref = torch.tensor(E_ref, dtype=torch.float64)
    Fref = torch.tensor(F_ref, dtype=torch.float64)
    L = wE * (((E - Eref) / nat) ** 2).mean() + wF * ((F - Fref) ** 2).sum() / (3 * batch.n_atoms)
    grads = torch.autograd.grad(L, [pt[k] for k in NAMES])
    return float(L.detach()), {k: g.numpy() for k, g in zip(NAMES, grads)}
