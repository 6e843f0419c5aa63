"""Seeded synthetic Stokes systems (input generation only).

This module builds the matrices and right-hand sides that both the FP64
oracle and the CUDA library are fed.  It contains no part of the solver:
no SpMV kernel, no AMG, no Krylov step.  It is the finite-difference
stand-in for the weak-Galerkin systems of the paper's Section 5, whose
meshes and matrices are not available.

Discretisation (the Stokes equations of Section 3, Eq. StokesPDE, on the
unit cube, collocated 7-point finite differences):

* N^3 nodes at ((i+1)h, (j+1)h, (k+1)h), h = 1/(N+1), node index
  m = i + N*(j + N*k); every node carries 4 unknowns [u, v, w, p]
  (interleaved, node-major).
* Ghost layer at index -1 and N: velocity Dirichlet 0 (no slip) and
  pressure 0 (keeps the system nonsingular).
* Viscosity mu per node; the value on the face between two nodes is the
  harmonic mean; a face to a ghost uses the interior node's mu.
* Momentum, component c at node m:
      sum_faces mu_f/h^2 (u_c,m - u_c,nb) + (p_{m+e_c} - p_{m-e_c})/(2h)
* Continuity at node m:
      sum_c (u_c,{m+e_c} - u_c,{m-e_c})/(2h) + 0.1 * sum_nb (p_m - p_nb)
  i.e. div u - 0.1 h^2 Lap_h p.
* Hence K = [A G; -G^T C] with A, C symmetric positive definite, so the
  symmetric part of K is blkdiag(A, C) and K is positive definite.

Random draws use numpy.random.Generator(PCG64(seed)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

__all__ = [
    "StokesSystem",
    "viscosity",
    "assemble_bsr",
    "bsr_nonzero_csr",
    "manufactured_x",
    "gaussian_rhs",
    "make_system",
    "CONFIGS",
]

PRESSURE_STAB = 0.1  # coefficient of the -0.1 h^2 Lap_h p stabilisation


def node_index(N: int, i, j, k):
    return i + N * (j + N * k)


def viscosity(N: int, sigma: float, seed: int | None) -> np.ndarray:
    """Per-node viscosity: 1 when sigma == 0, else exp(sigma*z), z ~ N(0,1)."""
    if sigma == 0.0 or seed is None:
        return np.ones(N ** 3)
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(N ** 3)
    return np.exp(sigma * z)


# Neighbour offsets in ascending column order: (-k), (-j), (-i), self, (+i), (+j), (+k)
# Each entry: (direction d in 0..2 or None for self, sign s).
_STENCIL = [(2, -1), (1, -1), (0, -1), (None, 0), (0, 1), (1, 1), (2, 1)]


def assemble_bsr(N: int, mu: np.ndarray):
    """Assemble K as 4x4 BSR: (indptr int32, indices int32, data f64[nnzb,4,4]).

    Columns are sorted within each block row (the stencil order above is
    ascending in node index).
    """
    n = N ** 3
    h = 1.0 / (N + 1)
    m = np.arange(n, dtype=np.int64)
    ii = m % N
    jj = (m // N) % N
    kk = m // (N * N)
    coord = [ii, jj, kk]
    stride = [1, N, N * N]

    # face viscosities for the 6 faces (d, s); ghost faces use the node's mu
    mu_face = {}
    valid = {}
    for d in range(3):
        for s in (-1, 1):
            c = coord[d] + s
            ok = (c >= 0) & (c < N)
            nb = np.where(ok, m + s * stride[d], m)
            mf = np.where(ok, 2.0 * mu * mu[nb] / (mu + mu[nb]), mu)
            mu_face[(d, s)] = mf
            valid[(d, s)] = ok

    counts = np.ones(n, dtype=np.int64)
    for (d, s), ok in valid.items():
        counts += ok
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    nnzb = int(indptr[-1])
    indices = np.empty(nnzb, dtype=np.int64)
    data = np.zeros((nnzb, 4, 4), dtype=np.float64)

    pos = indptr[:-1].copy()
    inv_h2 = 1.0 / (h * h)
    inv_2h = 1.0 / (2.0 * h)
    for d, s in _STENCIL:
        if d is None:
            diag = np.zeros(n)
            for key in mu_face:
                diag += mu_face[key] * inv_h2
            sel = m
            p = pos[sel]
            indices[p] = sel
            data[p, 0, 0] = diag
            data[p, 1, 1] = diag
            data[p, 2, 2] = diag
            data[p, 3, 3] = 6.0 * PRESSURE_STAB
            pos[sel] += 1
            continue
        ok = valid[(d, s)]
        sel = m[ok]
        p = pos[sel]
        indices[p] = sel + s * stride[d]
        off = -mu_face[(d, s)][ok] * inv_h2
        data[p, 0, 0] = off
        data[p, 1, 1] = off
        data[p, 2, 2] = off
        data[p, 3, 3] = -PRESSURE_STAB
        data[p, d, 3] = s * inv_2h
        data[p, 3, d] = s * inv_2h
        pos[sel] += 1
    assert np.array_equal(pos, indptr[1:])
    return indptr.astype(np.int32), indices.astype(np.int32), data


def bsr_nonzero_csr(indptr, indices, data):
    """Scalar CSR (int32 indptr/indices, f64 values) holding only the
    nonzero entries of a BSR matrix, columns sorted per row."""
    B = data.shape[1]
    nb = len(indptr) - 1
    A = sp.bsr_matrix((data, indices, indptr), shape=(nb * B, nb * B)).tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy()


def manufactured_x(N: int) -> np.ndarray:
    """Sampled manufactured field, interleaved [u,v,w,p] per node:
    u = (sin(pi x) cos(pi y) z, sin(pi y) cos(pi z) x, sin(pi z) cos(pi x) y),
    p = x y z (the cyclic reading of the unit-cube benchmark's field)."""
    h = 1.0 / (N + 1)
    m = np.arange(N ** 3)
    x = (m % N + 1) * h
    y = ((m // N) % N + 1) * h
    z = (m // (N * N) + 1) * h
    pi = math.pi
    out = np.empty((N ** 3, 4))
    out[:, 0] = np.sin(pi * x) * np.cos(pi * y) * z
    out[:, 1] = np.sin(pi * y) * np.cos(pi * z) * x
    out[:, 2] = np.sin(pi * z) * np.cos(pi * x) * y
    out[:, 3] = x * y * z
    return out.reshape(-1)


def gaussian_rhs(N: int, seed: int) -> np.ndarray:
    """N(0,1) per velocity unknown (node-major u,v,w), 0 for pressure."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(3 * N ** 3).reshape(N ** 3, 3)
    out = np.zeros((N ** 3, 4))
    out[:, :3] = g
    return out.reshape(-1)


def gaussian_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n)


@dataclass
class StokesSystem:
    name: str
    N: int
    bdim: int                      # 1 = scalar CSR, 4 = 4x4 BSR
    indptr: np.ndarray             # int32
    indices: np.ndarray            # int32
    data: np.ndarray               # f64, [nnz] (bdim 1) or [nnzb, 4, 4]
    b: np.ndarray                  # f64 [4 N^3]
    x_exact: np.ndarray | None     # f64 [4 N^3] when b = K x_exact
    mu: np.ndarray
    method: str                    # "amg_bicgstab" | "schur_gmres"
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return 4 * self.N ** 3

    def scipy(self):
        if self.bdim == 1:
            return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n))
        return sp.bsr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n))


# name -> (N, sigma, mu seed, rhs kind, rhs seed, storage bdim, method, extra seeds)
CONFIGS = {
    "c1": dict(N=16, sigma=0.0, mu_seed=None, rhs="manufactured", rhs_seed=None, bdim=1,
               method="amg_bicgstab"),
    "c2": dict(N=64, sigma=0.5, mu_seed=1001, rhs="gaussian", rhs_seed=1002, bdim=4,
               method="amg_bicgstab"),
    "c3": dict(N=128, sigma=1.0, mu_seed=3001, rhs="gaussian", rhs_seed=3002, bdim=4,
               method="schur_gmres"),
    "c4": dict(N=64, sigma=0.5, mu_seed=1001, rhs="gaussian", rhs_seed=1002, bdim=4,
               method="amg_bicgstab", xt_seed=4001, fd_seed=4002),
    "c5": dict(N=128, sigma=1.0, mu_seed=3001, rhs="gaussian", rhs_seed=3002, bdim=4,
               method="schur_gmres", xt_seed=5001),
}


def make_system(name: str, N: int | None = None) -> StokesSystem:
    """Build a named configuration; N overrides the grid size (same recipe)."""
    cfg = dict(CONFIGS[name])
    if N is not None:
        cfg["N"] = N
    N = cfg["N"]
    mu = viscosity(N, cfg["sigma"], cfg["mu_seed"])
    indptr, indices, data = assemble_bsr(N, mu)
    x_exact = None
    if cfg["rhs"] == "manufactured":
        x_exact = manufactured_x(N)
        K = sp.bsr_matrix((data, indices, indptr), shape=(4 * N ** 3, 4 * N ** 3))
        b = K @ x_exact
    else:
        b = gaussian_rhs(N, cfg["rhs_seed"])
    if cfg["bdim"] == 1:
        indptr, indices, data = bsr_nonzero_csr(indptr, indices, data)
    extra = {k: cfg[k] for k in ("xt_seed", "fd_seed") if k in cfg}
    return StokesSystem(name=name, N=N, bdim=cfg["bdim"], indptr=indptr, indices=indices,
                        data=data, b=b, x_exact=x_exact, mu=mu, method=cfg["method"],
                        extra=extra)
