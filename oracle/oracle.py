"""ctypes wrapper of the FP64 CPU oracle (``msp_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The oracle restates the method of "Accelerating Brain Simulations with the
Fast Multipole Method" (arXiv 2301.10570) in plain double precision: the
octree of Section 3.2, the expansions of Eq. 6 / Eq. 7, the direct sum of
Eq. 8, the descent of Algorithm 1 with the choice rule of Algorithm 2 and the
request resolution of Section 4.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msp_oracle.c")
_HDR = os.path.join(_HERE, "msp_oracle.h")
_SRC_NEURON = os.path.join(_HERE, "msp_neuron.c")
_HDR_NEURON = os.path.join(_HERE, "msp_neuron.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

SPLIT, FAR, P2P, PRUNED = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    srcs = (_SRC, _HDR, _SRC_NEURON, _HDR_NEURON)
    stale = force or not os.path.exists(_LIB_PATH) or max(
        os.path.getmtime(f) for f in srcs) > os.path.getmtime(_LIB_PATH)
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, _SRC_NEURON, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(C.Structure):
    _fields_ = [("sigma", C.c_double), ("p", C.c_int), ("leaf_capacity", C.c_int),
                ("max_depth", C.c_int), ("origin", C.c_float * 3), ("side", C.c_float),
                ("seed", C.c_uint64), ("rho_max", C.c_double), ("cutoff", C.c_double),
                ("m2l_min_pairs", C.c_longlong), ("boundary_tol", C.c_double),
                ("centre_mode", C.c_int), ("mac_mode", C.c_int), ("c1", C.c_int),
                ("c2", C.c_int)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, i32, u64, d = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
            L.orc_create.restype = vp
            L.orc_create.argtypes = [C.POINTER(_Cfg)]
            L.orc_destroy.argtypes = [vp]
            L.orc_build_tree.argtypes = [vp, i64] + [vp] * 7
            L.orc_attraction.argtypes = [vp, vp]
            L.orc_select_partners.restype = i64
            L.orc_select_partners.argtypes = [vp, u64] + [vp] * 6
            L.orc_direct.argtypes = [i64] + [vp] * 7 + [d, i64, vp, vp]
            L.orc_attraction_grad.restype = C.c_int
            L.orc_attraction_grad.argtypes = [vp] * 10
            L.orc_direct_grad.argtypes = [i64] + [vp] * 7 + [d] + [vp] * 5
            L.orc_length_loss.restype = C.c_int
            L.orc_length_loss.argtypes = [vp] * 5 + [d] + [vp] * 3
            L.orc_direct_length_loss.argtypes = [i64] + [vp] * 7 + [d, d] + [vp] * 3
            L.orc_vacancy_walk.argtypes = [i64, u64, u64, vp, vp, vp]
            L.orc_expf.restype = C.c_float
            L.orc_expf.argtypes = [C.c_float]
            L.orc_growth.restype = C.c_float
            L.orc_growth.argtypes = [C.c_float] * 4
            L.orc_neuron_steps.argtypes = [i64, u64, u64, C.c_int, vp, i64] + [vp] * 9
            L.orc_update_synapses.restype = i64
            L.orc_update_synapses.argtypes = [i64, u64, u64, vp, vp, vp, i64] + [vp] * 6
            L.orc_commit_synapses.argtypes = [i64] + [vp] * 6
            for f in ("orc_num_nodes", "orc_num_pairs", "orc_num_elements"):
                getattr(L, f).restype = i64
                getattr(L, f).argtypes = [vp]
            L.orc_num_pair_depths.argtypes = [vp]
            L.orc_far_level.argtypes = [vp]
            L.orc_get_keys.argtypes = [vp, vp, vp]
            L.orc_get_nodes.argtypes = [vp] * 8
            L.orc_get_node_sums.argtypes = [vp, vp, vp]
            L.orc_get_pairs.argtypes = [vp] * 8
            L.orc_get_expansions.argtypes = [vp, i64, vp, vp, vp]
            L.orc_get_stats.argtypes = [vp, vp]
            L.orc_hermite.argtypes = [C.c_int, d, vp]
            L.orc_morton.restype = u64
            L.orc_morton.argtypes = [C.c_float, C.c_float, C.c_float, vp, C.c_float]
            L.orc_p2m.argtypes = [C.c_int, d, i64, vp, vp, vp, vp]
            L.orc_m2l.argtypes = [C.c_int, d, vp, vp, vp, vp]
            L.orc_l2p.restype = d
            L.orc_l2p.argtypes = [C.c_int, d, vp, vp, vp]
            L.orc_m2p.restype = d
            L.orc_m2p.argtypes = [C.c_int, d, vp, vp, vp]
            L.orc_philox.argtypes = [vp, vp, vp]
            L.orc_uniform.restype = d
            L.orc_uniform.argtypes = [u64, C.c_uint32, C.c_uint32, u64]
            _lib = L
    return _lib


def _cfg(params: dict) -> _Cfg:
    c = _Cfg()
    c.sigma = float(params["sigma"])
    c.p = int(params["p"])
    c.leaf_capacity = int(params["leaf_capacity"])
    c.max_depth = int(params.get("max_depth", 21))
    for d in range(3):
        c.origin[d] = float(params["origin"][d])
    c.side = float(params["side"])
    c.seed = int(params.get("seed", 0))
    c.rho_max = float(params["rho_max"])
    c.cutoff = float(params["cutoff"])
    c.m2l_min_pairs = int(params.get("m2l_min_pairs", 0))
    # draws within this relative distance of a CDF boundary are flagged: 1e-6
    # when no pair is translated (single precision sums of exact terms), 1e-5
    # with translations (their single precision coefficients move W by ~1e-5;
    # the count rule of Algorithm 2 translates whatever rho_max is)
    translates = float(params["rho_max"]) > 0.0 or int(params.get("mac_mode", 0)) == 1
    c.boundary_tol = float(params.get("boundary_tol", 1e-5 if translates else 1e-6))
    c.centre_mode = int(params.get("centre_mode", 0))
    c.mac_mode = int(params.get("mac_mode", 0))
    c.c1 = int(params.get("c1", 70))
    c.c2 = int(params.get("c2", 70))
    return c


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


class Oracle:
    """One oracle context: build_tree -> attraction -> select_partners."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self._cfg = _cfg(params)
        self._h = lib().orc_create(C.byref(self._cfg))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        self.n = 0

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- steps ------------------------------------------------------------
    def build_tree(self, pos, type_, vac_axon, vac_dend_e, vac_dend_i):
        pos = np.ascontiguousarray(pos, dtype=np.float32)
        self.n = pos.shape[1]
        self._keep = [np.ascontiguousarray(pos[d]) for d in range(3)] + [
            _u8(type_), _u8(vac_axon), _u8(vac_dend_e), _u8(vac_dend_i)]
        lib().orc_build_tree(self._h, self.n, *[_p(a) for a in self._keep])

    def attraction(self):
        u = np.zeros(max(self.n, 1), dtype=np.float64)
        lib().orc_attraction(self._h, _p(u))
        return u[: self.n]

    def attraction_grad(self, type_, vac_axon, vac_dend_e, vac_dend_i, g=None):
        """u, du/dsigma and (with g) the gradient of sum_t g_t u(t) with respect
        to w^E, w^I, over the near-field pairs of the last attraction, at the
        given counts (caller order)."""
        n = self.n
        arrs = [_u8(type_), _u8(vac_axon), _u8(vac_dend_e), _u8(vac_dend_i)]
        gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
        out = [np.zeros(max(n, 1)) for _ in range(4)]
        rc = lib().orc_attraction_grad(self._h, *[_p(a) for a in arrs],
                                       None if gg is None else _p(gg), *[_p(o) for o in out])
        if rc != 0:
            raise RuntimeError("attraction_grad needs a finished attraction without far pairs")
        u, du, gE, gI = (o[:n] for o in out)
        return dict(u=u, dudsigma=du, gE=gE if g is not None else None,
                    gI=gI if g is not None else None)

    def length_loss(self, type_, vac_axon, w_e, w_i, target, grad=True):
        """Expected mean synapse length m, loss (m - target)^2 and its
        gradient over the near-field pairs of the last attraction (w_e, w_i:
        continuous dendritic weights, caller order)."""
        n = self.n
        we = np.ascontiguousarray(w_e, dtype=np.float64)
        wi = np.ascontiguousarray(w_i, dtype=np.float64)
        ty, va = _u8(type_), _u8(vac_axon)
        out = np.zeros(4)
        gE, gI = np.zeros(max(n, 1)), np.zeros(max(n, 1))
        rc = lib().orc_length_loss(self._h, _p(ty), _p(va), _p(we), _p(wi),
                                   float(target), _p(out), _p(gE) if grad else None,
                                   _p(gI) if grad else None)
        if rc != 0:
            raise RuntimeError("length_loss needs a finished attraction without far pairs")
        return dict(loss=out[0], mean=out[1], dloss_dsigma=out[2], dmean_dsigma=out[3],
                    gE=gE[:n] if grad else None, gI=gI[:n] if grad else None)

    def select_partners(self, step: int):
        ne = int(lib().orc_num_elements(self._h))
        m = max(ne, 1)
        partner = np.full(m, -1, np.int32)
        nb = np.zeros(m, np.uint8)
        acc = np.zeros(m, np.uint8)
        pre = np.zeros(m, np.int32)
        post = np.zeros(m, np.int32)
        typ = np.zeros(m, np.uint8)
        ns = lib().orc_select_partners(self._h, int(step), _p(partner), _p(nb), _p(acc),
                                       _p(pre), _p(post), _p(typ))
        if ns < 0:
            raise RuntimeError("attraction() must run before select_partners()")
        return dict(partner=partner[:ne], near_boundary=nb[:ne].astype(bool),
                    accepted=acc[:ne].astype(bool), syn_pre=pre[:ns], syn_post=post[:ns],
                    syn_type=typ[:ns], n_syn=int(ns))

    # -- introspection ----------------------------------------------------
    def keys(self):
        k = np.zeros(max(self.n, 1), np.uint64)
        pm = np.zeros(max(self.n, 1), np.int32)
        lib().orc_get_keys(self._h, _p(k), _p(pm))
        return k[: self.n], pm[: self.n]

    def nodes(self):
        m = int(lib().orc_num_nodes(self._h))
        out = dict(level=np.zeros(m, np.uint8), prefix=np.zeros(m, np.uint64),
                   first=np.zeros(m, np.int32), count=np.zeros(m, np.int32),
                   parent=np.zeros(m, np.int32), child_first=np.zeros(m, np.int32),
                   nchild=np.zeros(m, np.uint8))
        lib().orc_get_nodes(self._h, *[_p(out[k]) for k in
                                       ("level", "prefix", "first", "count", "parent",
                                        "child_first", "nchild")])
        sums = np.zeros((m, 4), np.int32)
        cent = np.zeros((m, 6), np.float64)
        lib().orc_get_node_sums(self._h, _p(sums), _p(cent))
        out["sums"] = sums
        out["centroids"] = cent
        return out

    def pairs(self):
        m = int(lib().orc_num_pairs(self._h))
        nd = int(lib().orc_num_pair_depths(self._h))
        out = dict(X=np.zeros(m, np.int32), Y=np.zeros(m, np.int32), kind=np.zeros(m, np.uint8),
                   child_first=np.zeros(m, np.int32), wE=np.zeros(m), wI=np.zeros(m),
                   depth_start=np.zeros(nd + 1, np.int64))
        lib().orc_get_pairs(self._h, *[_p(out[k]) for k in
                                       ("X", "Y", "kind", "child_first", "wE", "wI",
                                        "depth_start")])
        return out

    def expansions(self, node: int):
        p3 = self._cfg.p ** 3
        A, M, B = (np.zeros(2 * p3) for _ in range(3))
        lib().orc_get_expansions(self._h, int(node), _p(A), _p(M), _p(B))
        return A.reshape(2, p3), M.reshape(2, p3), B.reshape(2, p3)

    def far_level(self) -> int:
        return int(lib().orc_far_level(self._h))

    def num_elements(self) -> int:
        return int(lib().orc_num_elements(self._h))

    def stats(self):
        s = np.zeros(8, np.int64)
        lib().orc_get_stats(self._h, _p(s))
        names = ("pairs", "far_pairs", "p2p_pairs", "p2p_interactions", "draws",
                 "boundary_draws", "requests", "synapses")
        return dict(zip(names, (int(v) for v in s)))


# -- free functions ---------------------------------------------------------
def direct(pos, type_, vac_axon, vac_dend_e, vac_dend_i, sigma, targets=None):
    """Eq. 8 by brute force (FP64) for the given targets (all if None)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    n = pos.shape[1]
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(
        targets, dtype=np.int64)
    arrs = [np.ascontiguousarray(pos[d]) for d in range(3)] + [
        _u8(type_), _u8(vac_axon), _u8(vac_dend_e), _u8(vac_dend_i)]
    u = np.zeros(max(len(t), 1))
    lib().orc_direct(n, *[_p(a) for a in arrs], float(sigma), len(t), _p(t), _p(u))
    return u[: len(t)]


def direct_grad(pos, type_, vac_axon, vac_dend_e, vac_dend_i, sigma, g=None):
    """u, du/dsigma and (with g) dL/dw^E, dL/dw^I for L = sum_t g_t u(t), by
    brute force over all pairs (FP64)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    n = pos.shape[1]
    arrs = [np.ascontiguousarray(pos[d]) for d in range(3)] + [
        _u8(type_), _u8(vac_axon), _u8(vac_dend_e), _u8(vac_dend_i)]
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    out = [np.zeros(max(n, 1)) for _ in range(4)]
    lib().orc_direct_grad(n, *[_p(a) for a in arrs], float(sigma),
                          None if gg is None else _p(gg), *[_p(o) for o in out])
    u, du, gE, gI = (o[:n] for o in out)
    return dict(u=u, dudsigma=du, gE=gE if g is not None else None,
                gI=gI if g is not None else None)


def direct_length_loss(pos, type_, vac_axon, w_e, w_i, sigma, target, grad=True):
    """The expected mean synapse length, its loss and gradient by brute force
    over all pairs (FP64)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    n = pos.shape[1]
    we = np.ascontiguousarray(w_e, dtype=np.float64)
    wi = np.ascontiguousarray(w_i, dtype=np.float64)
    xs = [np.ascontiguousarray(pos[d]) for d in range(3)]
    ty, va = _u8(type_), _u8(vac_axon)
    out = np.zeros(4)
    gE, gI = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    lib().orc_direct_length_loss(n, *[_p(x) for x in xs],
                                 _p(ty), _p(va), _p(we), _p(wi), float(sigma),
                                 float(target), _p(out), _p(gE) if grad else None,
                                 _p(gI) if grad else None)
    return dict(loss=out[0], mean=out[1], dloss_dsigma=out[2], dmean_dsigma=out[3],
                gE=gE[:n] if grad else None, gI=gI[:n] if grad else None)


def hermite(nmax: int, x: float):
    h = np.zeros(nmax + 1)
    lib().orc_hermite(int(nmax), float(x), _p(h))
    return h


def morton(x, y, z, origin, side):
    o = np.asarray(origin, np.float32)
    return int(lib().orc_morton(float(x), float(y), float(z), _p(o), float(side)))


def p2m(p, sigma, pts, w, c):
    pts = np.ascontiguousarray(pts, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    A = np.zeros(p ** 3)
    lib().orc_p2m(p, float(sigma), len(w), _p(pts), _p(w), _p(c), _p(A))
    return A


def m2l(p, sigma, A, cA, cD):
    A = np.ascontiguousarray(A, np.float64)
    cA = np.ascontiguousarray(cA, np.float64)
    cD = np.ascontiguousarray(cD, np.float64)
    B = np.zeros(p ** 3)
    lib().orc_m2l(p, float(sigma), _p(A), _p(cA), _p(cD), _p(B))
    return B


def l2p(p, sigma, B, cA, t):
    B, cA, t = (np.ascontiguousarray(a, np.float64) for a in (B, cA, t))
    return float(lib().orc_l2p(p, float(sigma), _p(B), _p(cA), _p(t)))


def m2p(p, sigma, A, cD, t):
    A, cD, t = (np.ascontiguousarray(a, np.float64) for a in (A, cD, t))
    return float(lib().orc_m2p(p, float(sigma), _p(A), _p(cD), _p(t)))


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(o))
    return o


def uniform(seed, c0, c1, step):
    return float(lib().orc_uniform(int(seed), int(c0), int(c1), int(step)))


def vacancy_walk(seed, step, vac_axon, vac_dend_e, vac_dend_i):
    a, e, i = (np.array(v, dtype=np.uint8, copy=True) for v in (vac_axon, vac_dend_e, vac_dend_i))
    lib().orc_vacancy_walk(len(a), int(seed), int(step), _p(a), _p(e), _p(i))
    return a, e, i


def commit_synapses(syn_pre, syn_post, syn_type, vac_axon, vac_dend_e, vac_dend_i):
    a, e, i = (np.array(v, dtype=np.uint8, copy=True) for v in (vac_axon, vac_dend_e, vac_dend_i))
    pre = np.ascontiguousarray(syn_pre, np.int32)
    post = np.ascontiguousarray(syn_post, np.int32)
    ty = np.ascontiguousarray(syn_type, np.uint8)
    lib().orc_commit_synapses(len(pre), _p(pre), _p(post), _p(ty), _p(a), _p(e), _p(i))
    return a, e, i


# -- the neuron side of the model (Section 3.1, Table 1) ---------------------
class NeuronParams(C.Structure):
    """Table 1 values (beta = 5e-4 of the table; the text says 1e-3)."""
    _fields_ = [("x0", C.c_float), ("tau_x", C.c_float), ("background", C.c_float),
                ("input_per_spike", C.c_float), ("refractory", C.c_int),
                ("beta_ca", C.c_float), ("decay_ca", C.c_float), ("eps", C.c_float),
                ("eta_axon", C.c_float), ("eta_dend", C.c_float), ("mu", C.c_float)]


TABLE1 = dict(x0=0.05, tau_x=5.0, background=0.003, input_per_spike=5e-4, refractory=4,
              beta_ca=5e-4, decay_ca=1e-5, eps=0.7, eta_axon=0.4, eta_dend=0.1, mu=1e-4)


def neuron_params(**kw):
    return NeuronParams(**dict(TABLE1, **kw))


def expf(x: float) -> float:
    return float(lib().orc_expf(float(x)))


def growth(ca: float, eta: float, eps: float, mu: float) -> float:
    return float(lib().orc_growth(float(ca), float(eta), float(eps), float(mu)))


NEURON_STATE = (("x", np.float32), ("refractory", np.uint8), ("calcium", np.float32),
                ("z_axon", np.float32), ("z_dend_e", np.float32), ("z_dend_i", np.float32),
                ("spiked", np.uint8))


def neuron_steps(seed, first_step, n_steps, params, edge_pre, edge_post, state):
    """n_steps steps of activity, spikes, calcium and elements; returns a new
    state dict (keys of NEURON_STATE)."""
    st = {k: np.array(state[k], dtype=t, copy=True) for k, t in NEURON_STATE}
    n = len(st["x"])
    pre = np.ascontiguousarray(edge_pre, np.int32)
    post = np.ascontiguousarray(edge_post, np.int32)
    lib().orc_neuron_steps(n, int(seed), int(first_step), int(n_steps), C.byref(params),
                           len(pre), _p(pre), _p(post), *[_p(st[k]) for k, _ in NEURON_STATE])
    return st


def update_synapses(seed, step, z_axon, z_dend_e, z_dend_i, edge_pre, edge_post, edge_type):
    """Deletion of excess synapses and the vacancies; returns (edges, vacancies)."""
    za, ze, zi = (np.ascontiguousarray(v, np.float32) for v in (z_axon, z_dend_e, z_dend_i))
    n = len(za)
    pre = np.array(edge_pre, np.int32, copy=True)
    post = np.array(edge_post, np.int32, copy=True)
    ty = np.array(edge_type, np.uint8, copy=True)
    va, ve, vi = (np.zeros(max(n, 1), np.uint8) for _ in range(3))
    m = lib().orc_update_synapses(n, int(seed), int(step), _p(za), _p(ze), _p(zi), len(pre),
                                  _p(pre), _p(post), _p(ty), _p(va), _p(ve), _p(vi))
    return (pre[:m], post[:m], ty[:m]), (va[:n], ve[:n], vi[:n])
