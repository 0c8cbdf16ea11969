"""Seeded synthetic inputs for the synapse search.

This module only draws random inputs; it holds none of the method's
arithmetic.  It is the one piece shared by the CUDA path's tests/benchmark
and the oracle.  The paper's own networks are not public: these generators
stand in for them with the sizes and structure of the workloads the paper and
the benchmark describe (a Poisson-like uniform cube at the paper's density,
and clustered networks), with sigma = 750 um (Table 1) and vacant element
counts small integers as in the model of structural plasticity (Section 3.1).
All generators use numpy's PCG64 with the given seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SIGMA_UM = 750.0


def default_params(side: float, **kw) -> dict:
    """Search parameters: kernel width, expansion order, octree and pair rule."""
    p = dict(sigma=SIGMA_UM, p=4, leaf_capacity=32, max_depth=21,
             origin=(0.0, 0.0, 0.0), side=float(side), seed=0,
             rho_max=0.25, cutoff=4.0, m2l_min_pairs=0, boundary_tol=1e-5)
    p.update(kw)
    return p


@dataclass
class Workload:
    name: str
    pos: np.ndarray          # (3, n) float32, SoA x/y/z in um
    type: np.ndarray         # (n,) uint8, 0 = excitatory, 1 = inhibitory
    vac_axon: np.ndarray     # (n,) uint8 vacant axonal elements
    vac_dend_e: np.ndarray   # (n,) uint8 vacant excitatory dendritic elements
    vac_dend_i: np.ndarray   # (n,) uint8 vacant inhibitory dendritic elements
    params: dict = field(default_factory=dict)
    frames: tuple | None = None   # (offsets, level): networks in their own frames

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])

    def arrays(self):
        return self.pos, self.type, self.vac_axon, self.vac_dend_e, self.vac_dend_i


def _counts(rng, n, frac_exc=0.8, vmax=3):
    type_ = (rng.random(n) >= frac_exc).astype(np.uint8)
    va = rng.integers(0, vmax + 1, n, dtype=np.uint8)
    ve = rng.integers(0, vmax + 1, n, dtype=np.uint8)
    vi = rng.integers(0, vmax + 1, n, dtype=np.uint8)
    return type_, va, ve, vi


def _clamp_cube(pos, side):
    hi = np.nextafter(np.float32(side), np.float32(0))
    return np.clip(pos, np.float32(0), hi).astype(np.float32)


def uniform_cube(n: int, side: float, seed: int, name: str = "uniform", **kw) -> Workload:
    rng = np.random.default_rng(seed)
    pos = _clamp_cube(rng.random((3, n), dtype=np.float64).astype(np.float32) *
                      np.float32(side), side)
    t, a, e, i = _counts(rng, n)
    return Workload(name, pos, t, a, e, i, default_params(side, **kw))


def clustered(n_clusters: int, per_cluster: int, side: float, std: float, margin: float,
              seed: int, name: str = "clustered", **kw) -> Workload:
    """Isotropic Gaussian clusters; centres uniform in [margin, side - margin)^3."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(margin, side - margin, (n_clusters, 3))
    pts = centres[:, None, :] + rng.normal(0.0, std, (n_clusters, per_cluster, 3))
    pos = _clamp_cube(pts.reshape(-1, 3).T.astype(np.float32), side)
    n = n_clusters * per_cluster
    t, a, e, i = _counts(rng, n)
    return Workload(name, np.ascontiguousarray(pos), t, a, e, i,
                    default_params(side, **kw))


# -- the named workloads ----------------------------------------------------
def uniform_4k(**kw) -> Workload:
    """4,096 neurons uniform in a 10,000 um cube, p = 4, leaf capacity 32."""
    return uniform_cube(4096, 10_000.0, seed=1, name="uniform_4k", **kw)


def uniform_256k(**kw) -> Workload:
    """262,144 neurons uniform in a 40,000 um cube (same density as uniform_4k)."""
    return uniform_cube(262_144, 40_000.0, seed=2, name="uniform_256k", **kw)


def clustered_1m(**kw) -> Workload:
    """1,048,576 neurons in 64 Gaussian clusters (std 1,500 um), 100,000 um cube."""
    return clustered(64, 16_384, 100_000.0, 1500.0, 4500.0, seed=3, name="clustered_1m",
                     **kw)


def clustered_small(n_clusters: int = 2, per_cluster: int = 4096, seed: int = 7,
                    **kw) -> Workload:
    """A few clusters at the density of clustered_1m, small enough for the oracle."""
    side = 100_000.0 * (n_clusters / 64.0) ** (1.0 / 3.0)
    return clustered(n_clusters, per_cluster, side, 1500.0, min(4500.0, side / 4), seed=seed,
                     name=f"clustered_{n_clusters}x{per_cluster}", **kw)


def subset(w: Workload, idx: np.ndarray, name: str | None = None) -> Workload:
    """The neurons idx of w (same parameters)."""
    idx = np.asarray(idx)
    return Workload(name or w.name + "_sub", np.ascontiguousarray(w.pos[:, idx]),
                    w.type[idx].copy(), w.vac_axon[idx].copy(), w.vac_dend_e[idx].copy(),
                    w.vac_dend_i[idx].copy(), dict(w.params))


# -- many independent networks ------------------------------------------------
@dataclass
class Batch:
    """Independent networks, concatenated: network k holds neurons
    [offsets[k], offsets[k+1]) with kernel width sigma[k] (um)."""
    name: str
    pos: np.ndarray           # (3, N) float32, um, each network in its own frame
    type: np.ndarray
    vac_axon: np.ndarray
    vac_dend_e: np.ndarray
    vac_dend_i: np.ndarray
    offsets: np.ndarray       # (K + 1,) int64
    sigma: np.ndarray         # (K,) float64, um
    kinds: list               # "uniform" or "clustered" per network

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])

    def network_of(self) -> np.ndarray:
        return np.repeat(np.arange(len(self.sigma)), np.diff(self.offsets))

    def network(self, k: int, **kw) -> Workload:
        """Network k alone, in its own frame, with its own kernel width."""
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        pos = np.ascontiguousarray(self.pos[:, a:b])
        lo = pos.min(axis=1, keepdims=True)
        side = float((pos.max(axis=1) - lo[:, 0]).max()) * 1.001 + 1.0
        params = default_params(side, sigma=float(self.sigma[k]),
                                origin=tuple(float(v) for v in lo[:, 0]), **kw)
        return Workload(f"{self.name}_{k}", pos, self.type[a:b].copy(),
                        self.vac_axon[a:b].copy(), self.vac_dend_e[a:b].copy(),
                        self.vac_dend_i[a:b].copy(), params)

    def select(self, nets) -> "Batch":
        """The networks `nets` of this batch, in that order."""
        nets = [int(k) for k in nets]
        idx = np.concatenate([np.arange(self.offsets[k], self.offsets[k + 1]) for k in nets])
        sizes = np.diff(self.offsets)[nets]
        return Batch(f"{self.name}_part", np.ascontiguousarray(self.pos[:, idx]),
                     self.type[idx].copy(), self.vac_axon[idx].copy(),
                     self.vac_dend_e[idx].copy(), self.vac_dend_i[idx].copy(),
                     np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64),
                     self.sigma[nets].copy(), [self.kinds[k] for k in nets])

    def cell_corners(self, side: float, level: int) -> np.ndarray:
        """(3, N) low corner of every neuron's cell (sigma units): network k
        in the cell at grid coordinates 2 (k mod G, (k / G) mod G, k / G^2),
        G = 2^(level - 1)."""
        G = 2 ** (level - 1)
        k = self.network_of()
        c = np.stack([k % G, (k // G) % G, k // (G * G)]).astype(np.float64)
        return 2.0 * c * (side / 2.0 ** level)

    def framed(self, pos_local: np.ndarray, side: float, level: int, plans=None,
               **kw) -> Workload:
        """The whole batch as one problem of kernel width 1, each network in
        its own frame (positions relative to its cell, sigma units); plans:
        None, or (leaf capacities, cutoffs) per network (either may be None)."""
        frames = (self.offsets.copy(), int(level))
        if plans is not None:
            frames = frames + tuple(plans)
        return Workload(self.name + "_framed", np.ascontiguousarray(pos_local, np.float32),
                        self.type, self.vac_axon, self.vac_dend_e, self.vac_dend_i,
                        default_params(side, sigma=1.0, **kw), frames=frames)

    def placed(self, pos_local: np.ndarray, side: float, level: int, **kw) -> Workload:
        """The same problem in one common frame: every network moved to its
        cell (single precision; exact when the local positions and the cell
        corners share a fine enough dyadic grid)."""
        g = pos_local.astype(np.float64) + self.cell_corners(side, level)
        return Workload(self.name + "_placed", np.ascontiguousarray(g, np.float32),
                        self.type, self.vac_axon, self.vac_dend_e, self.vac_dend_i,
                        default_params(side, sigma=1.0, **kw))


def batch(sizes, sigmas, kinds, seed: int, name: str = "batch") -> Batch:
    """Networks of the given sizes: "uniform" ones fill a cube of side
    625 n^(1/3) um (the density of uniform_4k); "clustered" ones hold
    max(1, n / 16,384) Gaussian clusters (std 1,500 um) at the cluster spacing
    of clustered_1m."""
    rng = np.random.default_rng(seed)
    pos, offs = [], [0]
    for n, kind in zip(sizes, kinds):
        n = int(n)
        if kind == "uniform":
            side = 625.0 * n ** (1.0 / 3.0)
            p = rng.random((3, n)) * side
        else:
            nc = max(1, n // 16_384)
            side = 100_000.0 * (nc / 64.0) ** (1.0 / 3.0)
            margin = min(4500.0, side / 4)
            centres = rng.uniform(margin, side - margin, (nc, 3))
            which = rng.integers(0, nc, n)
            p = (centres[which] + rng.normal(0.0, 1500.0, (n, 3))).T
            p = np.clip(p, 0.0, side)
        pos.append(p.astype(np.float32))
        offs.append(offs[-1] + n)
    n_all = offs[-1]
    t, a, e, i = _counts(rng, n_all)
    return Batch(name, np.ascontiguousarray(np.concatenate(pos, axis=1)), t, a, e, i,
                 np.asarray(offs, np.int64), np.asarray(sigmas, np.float64), list(kinds))


def batched_256(seed: int = 5) -> Batch:
    """256 networks, n log-uniform in [1,024, 262,144] (about 12M neurons in
    all), sigma uniform in [300, 1,500] um, each uniform or clustered."""
    rng = np.random.default_rng(seed)
    k = 256
    sizes = np.exp(rng.uniform(np.log(1024), np.log(262_144), k)).astype(np.int64)
    sigmas = rng.uniform(300.0, 1500.0, k)
    kinds = ["clustered" if v else "uniform" for v in rng.random(k) < 0.5]
    return batch(sizes, sigmas, kinds, seed=seed + 1, name="batched_256")


def batched_small(seed: int = 8) -> Batch:
    """Five small networks of both kinds and different widths (oracle-sized)."""
    sizes = [700, 1500, 400, 2200, 900]
    sigmas = [300.0, 750.0, 1500.0, 500.0, 1100.0]
    kinds = ["uniform", "clustered", "uniform", "clustered", "uniform"]
    return batch(sizes, sigmas, kinds, seed=seed, name="batched_small")
