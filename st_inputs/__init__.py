"""Seeded synthetic inputs shared by the CUDA library's tests/benchmark and the oracle.

This module only draws random numbers and applies index rules; it contains none
of the solver's arithmetic.  The workloads follow the paper's problem statement
(Section 3, eq. EddyCurrent: materials sigma, nu = mu^{-1} per element and a source
J on the unit cube); the concrete recipe is ours:

  * materials(n, kind, seed): per Kuhn tet (tet index 6*cube + permutation, cube
    index ci + n*(cj + n*ck)):
      kind "unit"      : nu = sigma = 1
      kind "two_material": nu = 1e-3 for tets of cubes whose centre lies in
                         [0.25, 0.75]^3, else 1; sigma = 10**U(-1, 1) per tet.
  * excitation(seed): the source J(x, t) = g(t) curl psi(x) with
      psi(x) = sum_{m<4} a_m sin(pi k_m . x + phi_m),  a_m ~ N(0, I_3),
      k_m uniform in {1,2,3}^3, phi_m ~ U(0, 2 pi),  g(t) = sin(pi t / T) + 1,
    returned as its parameters (a, k, phase); each side evaluates J itself.

  * request_stream(n, rate, seed, meshes, nt_range, degrees): a Poisson stream of
    solve requests (the serving workload): exponential inter-arrival gaps of mean
    1/rate; per request a mesh uniform over `meshes`, N_t uniform over the powers of
    two in nt_range, a DG degree uniform over `degrees`, a conductivity scale s drawn
    log-uniform in [0.1, 10] and rounded to the nearest power of two (so that tau / s
    stays on one power-of-two ladder per mesh and degree), and an excitation seed.

  * start_mesh(kind, seed): a coarse conforming tetrahedral mesh (xyz, tets) for the
    general-mesh path (refined uniformly by each side):
      "two_tet"  : two tets sharing the face (0,0,0), (1,0,0), (0,1,0), apexes
                   (0.3, 0.3, +-0.8) moved by U(-0.1, 0.1) per coordinate;
      "cube5"    : the unit cube cut into four corner tets and one central tet, then
                   mapped by x -> A x, A = I + U(-0.15, 0.15) per entry;
      "kuhn2_jitter": the 2x2x2 Kuhn mesh of the unit cube (vertex and tet numbering of
                   the Kuhn conventions) with its centre vertex moved by U(-0.12, 0.12)
                   per coordinate.
  * materials_tets(nt, kind, seed): per tet of a general mesh: "unit", or
    "two_material": nu = 1e-3 with probability 1/4 else 1, sigma = 10**U(-1, 1).

Random streams: numpy Generator(PCG64(seed)).
"""
from __future__ import annotations

import numpy as np

N_MODES = 4


def materials(n: int, kind: str = "two_material", seed: int = 0):
    nt = 6 * n ** 3
    if kind == "unit":
        return np.ones(nt), np.ones(nt)
    if kind != "two_material":
        raise ValueError(kind)
    c = np.arange(n ** 3)
    ci, cj, ck = c % n, (c // n) % n, c // (n * n)
    centre = (np.stack([ci, cj, ck], axis=1) + 0.5) / n
    inside = np.all((centre >= 0.25) & (centre <= 0.75), axis=1)
    nu = np.repeat(np.where(inside, 1e-3, 1.0), 6)
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma = 10.0 ** rng.uniform(-1.0, 1.0, size=nt)
    return nu, sigma


def excitation(seed: int = 0):
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    a = rng.normal(size=(N_MODES, 3))
    k = rng.integers(1, 4, size=(N_MODES, 3)).astype(np.float64)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=N_MODES)
    return {"a": a, "k": k, "phase": phase}


def random_iterate(shape, seed: int = 0):
    """Uniform [0, 1) values, e.g. the random start of the power iteration (Section 5.1)."""
    rng = np.random.Generator(np.random.PCG64(20_000 + seed))
    return rng.uniform(0.0, 1.0, size=shape)


def request_stream(n: int, rate: float, seed: int = 0, meshes=(8, 16, 24), nt_range=(64, 2048), degrees=(0, 1)):
    rng = np.random.Generator(np.random.PCG64(30_000 + seed))
    nts = [1 << k for k in range(int(np.log2(nt_range[0])), int(np.log2(nt_range[1])) + 1)]
    gaps = rng.exponential(1.0 / rate, size=n)
    out = []
    t = 0.0
    for i in range(n):
        t += gaps[i]
        s = 2.0 ** np.round(np.log2(10.0 ** rng.uniform(-1.0, 1.0)))
        out.append({"t": float(t), "n_cube": int(rng.choice(meshes)), "N_t": int(rng.choice(nts)),
                    "degree": int(rng.choice(degrees)), "sigma_scale": float(s), "seed": int(rng.integers(0, 1 << 30))})
    return out


def start_mesh(kind: str = "two_tet", seed: int = 0):
    rng = np.random.Generator(np.random.PCG64(30_000 + seed))
    if kind == "two_tet":
        xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.3, 0.3, 0.8], [0.3, 0.3, -0.8]])
        xyz[3:] += rng.uniform(-0.1, 0.1, size=(2, 3))
        return xyz, np.array([[0, 1, 2, 3], [0, 1, 2, 4]], dtype=np.int64)
    if kind == "cube5":
        c = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=np.float64)
        A = np.eye(3) + rng.uniform(-0.15, 0.15, size=(3, 3))
        tets = np.array([[0, 1, 2, 4], [3, 1, 2, 7], [5, 1, 4, 7], [6, 2, 4, 7], [1, 2, 4, 7]], dtype=np.int64)
        return c @ A.T, tets
    if kind == "kuhn2_jitter":
        n = 2
        ijk = np.array([[i, j, k] for k in range(n + 1) for j in range(n + 1) for i in range(n + 1)])
        xyz = ijk.astype(np.float64) / n
        centre = 1 + 3 * (1 + 3 * 1)
        xyz[centre] += rng.uniform(-0.12, 0.12, size=3)
        perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
        tets = []
        for ck in range(n):
            for cj in range(n):
                for ci in range(n):
                    for perm in perms:
                        p = [ci, cj, ck]
                        chain = [p[0] + 3 * (p[1] + 3 * p[2])]
                        for ax in perm:
                            p = list(p)
                            p[ax] += 1
                            chain.append(p[0] + 3 * (p[1] + 3 * p[2]))
                        tets.append(chain)
        return xyz, np.array(tets, dtype=np.int64)
    raise ValueError(kind)


def materials_tets(nt: int, kind: str = "two_material", seed: int = 0):
    if kind == "unit":
        return np.ones(nt), np.ones(nt)
    if kind != "two_material":
        raise ValueError(kind)
    rng = np.random.Generator(np.random.PCG64(40_000 + seed))
    nu = np.where(rng.uniform(size=nt) < 0.25, 1e-3, 1.0)
    sigma = 10.0 ** rng.uniform(-1.0, 1.0, size=nt)
    return nu, sigma
