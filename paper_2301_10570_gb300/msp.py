"""Python binding of libmsp (include/msp.h): argument marshalling only.

Every step of the synapse search runs in the CUDA library; this module only
turns torch tensors into device pointers and the current torch stream into a
cudaStream_t.  There is no fallback: if the library is missing or fails to
load, constructing :class:`MSP` raises.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import threading
import weakref

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmsp.so")
_lock = threading.Lock()
_lib = None

SPLIT, FAR, P2P, PRUNED = 0, 1, 2, 3
STATUS = {0: "MSP_OK", 1: "MSP_ERR_INVALID_ARG", 2: "MSP_ERR_CUDA", 3: "MSP_ERR_OOM",
          4: "MSP_ERR_TIMEOUT", 5: "MSP_ERR_NOT_BUILT", 6: "MSP_ERR_CHECK",
          7: "MSP_ERR_CAPACITY"}

EXPORTED = ("msp_create", "msp_destroy", "msp_build_tree", "msp_attraction", "msp_direct",
            "msp_select_partners", "msp_plasticity_step_host", "msp_vacancy_walk",
            "msp_commit_synapses", "msp_get_stats", "msp_export_tree", "msp_export_pairs",
            "msp_export_expansions", "msp_last_error", "msp_direct_noalloc",
            "msp_step_graph_capture", "msp_step_graph_launch", "msp_step_graph_finish",
            "msp_set_pair_capacity", "msp_batch_layout", "msp_attraction_grad",
            "msp_set_workspace_limit", "msp_workspace_bytes", "msp_neuron_steps",
            "msp_update_synapses", "msp_append_synapses", "msp_selftest_bounded_wait",
            "msp_philox", "msp_step_graph_set_full_build", "msp_length_loss",
            "msp_set_sigma", "msp_set_frames")
MAX_VACANCY = 5         # the vacancy walk's bound on every vacant count
NOALLOC_MAX_N = 65536   # MSP_NOALLOC_MAX_N of include/msp.h


class NeuronParams(C.Structure):
    """msp_neuron_params of include/msp.h."""
    _fields_ = [("x0", C.c_float), ("tau_x", C.c_float), ("background", C.c_float),
                ("input_per_spike", C.c_float), ("refractory", C.c_int),
                ("beta_ca", C.c_float), ("decay_ca", C.c_float), ("eps", C.c_float),
                ("eta_axon", C.c_float), ("eta_dend", C.c_float), ("mu", C.c_float)]


# Table 1 (beta = 5e-4 of the table; the text says 1e-3), refractory period 4
# and 5e-4 per spiking presynaptic partner (Section 3.1)
TABLE1 = dict(x0=0.05, tau_x=5.0, background=0.003, input_per_spike=5e-4, refractory=4,
              beta_ca=5e-4, decay_ca=1e-5, eps=0.7, eta_axon=0.4, eta_dend=0.1, mu=1e-4)


def neuron_params(**kw) -> NeuronParams:
    return NeuronParams(**dict(TABLE1, **kw))


NEURON_STATE = (("x", torch.float32), ("refractory", torch.uint8), ("calcium", torch.float32),
                ("z_axon", torch.float32), ("z_dend_e", torch.float32),
                ("z_dend_i", torch.float32), ("spiked", torch.uint8))


def edge_list(capacity: int, device="cuda", pre=None, post=None, type_=None) -> dict:
    """An edge list (pre, post, type) of the given capacity, filled with the
    given edges (any array-likes) and its length in device memory."""
    e = dict(pre=torch.zeros(max(capacity, 1), dtype=torch.int32, device=device),
             post=torch.zeros(max(capacity, 1), dtype=torch.int32, device=device),
             type=torch.zeros(max(capacity, 1), dtype=torch.uint8, device=device),
             n=torch.zeros(1, dtype=torch.int64, device=device), capacity=int(capacity))
    if pre is not None:
        m = len(pre)
        if m > capacity:
            raise ValueError("more edges than the capacity")
        e["pre"][:m] = torch.as_tensor(pre, dtype=torch.int32)
        e["post"][:m] = torch.as_tensor(post, dtype=torch.int32)
        e["type"][:m] = torch.as_tensor(type_, dtype=torch.uint8)
        e["n"].fill_(m)
    return e


class MSPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("sigma", C.c_double), ("p", C.c_int), ("leaf_capacity", C.c_int),
                ("max_depth", C.c_int), ("origin", C.c_float * 3), ("side", C.c_float),
                ("seed", C.c_uint64), ("rho_max", C.c_double), ("cutoff", C.c_double),
                ("m2l_min_pairs", C.c_longlong), ("centre_mode", C.c_int),
                ("mac_mode", C.c_int), ("c1", C.c_int), ("c2", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_nodes", C.c_int64), ("n_leaves", C.c_int64),
                ("tree_depth", C.c_int32), ("far_level", C.c_int32), ("n_pairs", C.c_int64),
                ("pair_depths", C.c_int32), ("n_far", C.c_int64), ("n_p2p", C.c_int64),
                ("p2p_interactions", C.c_int64), ("n_elements", C.c_int64),
                ("n_draws", C.c_int64), ("n_requests", C.c_int64), ("n_synapses", C.c_int64),
                ("expansion_nodes", C.c_int64), ("kernel_launches", C.c_int64),
                ("near_field_ms", C.c_double)]


def load(path: str = LIB_PATH):
    """Load libmsp.so (built by paper_2301_10570_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2301_10570_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(path)
        vp, i64, u64 = C.c_void_p, C.c_int64, C.c_uint64
        L.msp_create.argtypes = [C.POINTER(vp), C.POINTER(Config), C.c_int]
        L.msp_destroy.argtypes = [vp]
        L.msp_build_tree.argtypes = [vp, i64] + [vp] * 7 + [vp]
        L.msp_attraction.argtypes = [vp, vp, vp]
        L.msp_direct.argtypes = [vp, vp, vp]
        L.msp_select_partners.argtypes = [vp, u64] + [vp] * 5 + [vp]
        L.msp_plasticity_step_host.argtypes = [vp, i64, u64] + [vp] * 13
        L.msp_vacancy_walk.argtypes = [vp, i64, u64, vp, vp, vp, vp]
        L.msp_commit_synapses.argtypes = [vp, vp, i64] + [vp] * 6 + [vp]
        L.msp_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.msp_export_tree.argtypes = [vp] * 12
        L.msp_export_pairs.argtypes = [vp] * 8
        L.msp_export_expansions.argtypes = [vp] * 5
        L.msp_last_error.restype = C.c_char_p
        L.msp_direct_noalloc.argtypes = [i64] + [vp] * 7 + [C.c_double, vp, vp]
        L.msp_direct_noalloc.restype = C.c_int
        L.msp_step_graph_capture.argtypes = [vp, i64] + [vp] * 11 + [i64, vp, vp, i64, u64, vp]
        L.msp_step_graph_launch.argtypes = [vp, i64, vp]
        L.msp_step_graph_finish.argtypes = [vp, vp, C.POINTER(u64), C.POINTER(i64)]
        L.msp_set_pair_capacity.argtypes = [vp, i64]
        L.msp_batch_layout.argtypes = [i64, vp, vp, vp, vp, vp, C.c_double, C.c_int, vp, vp, vp,
                                       C.POINTER(C.c_float), C.POINTER(C.c_int), vp]
        L.msp_batch_layout.restype = C.c_int
        L.msp_attraction_grad.argtypes = [vp] * 11
        L.msp_attraction_grad.restype = C.c_int
        L.msp_set_workspace_limit.argtypes = [i64]
        L.msp_set_workspace_limit.restype = C.c_int
        L.msp_workspace_bytes.argtypes = []
        L.msp_workspace_bytes.restype = i64
        L.msp_neuron_steps.argtypes = [vp, i64, u64, C.c_int, C.POINTER(NeuronParams), vp,
                                       i64] + [vp] * 9 + [vp]
        L.msp_update_synapses.argtypes = [vp, i64, u64] + [vp] * 7 + [i64] + [vp] * 3 + [vp]
        L.msp_append_synapses.argtypes = [vp, vp, i64] + [vp] * 7 + [i64, vp]
        L.msp_selftest_bounded_wait.argtypes = [vp, vp]
        L.msp_philox.argtypes = [i64, vp, vp, vp, vp]
        L.msp_philox.restype = C.c_int
        L.msp_step_graph_set_full_build.argtypes = [vp, C.c_int]
        L.msp_step_graph_set_full_build.restype = C.c_int
        L.msp_length_loss.argtypes = [vp] * 5 + [C.c_double] + [vp] * 4
        L.msp_length_loss.restype = C.c_int
        L.msp_set_sigma.argtypes = [vp, C.c_double]
        L.msp_set_sigma.restype = C.c_int
        L.msp_set_frames.argtypes = [vp, i64, vp, C.c_int, vp, vp]
        L.msp_set_frames.restype = C.c_int
        for name in ("msp_neuron_steps", "msp_update_synapses", "msp_append_synapses",
                     "msp_selftest_bounded_wait"):
            getattr(L, name).restype = C.c_int
        for name in ("msp_step_graph_capture", "msp_step_graph_launch", "msp_step_graph_finish",
                     "msp_set_pair_capacity", "msp_batch_layout", "msp_attraction_grad",
            "msp_set_workspace_limit", "msp_workspace_bytes", "msp_neuron_steps",
            "msp_update_synapses", "msp_append_synapses", "msp_selftest_bounded_wait"):
            getattr(L, name).restype = C.c_int
        for name in ("msp_create", "msp_destroy", "msp_build_tree", "msp_attraction",
                     "msp_direct", "msp_select_partners", "msp_plasticity_step_host",
                     "msp_vacancy_walk", "msp_commit_synapses", "msp_get_stats",
                     "msp_export_tree", "msp_export_pairs", "msp_export_expansions"):
            getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(code):
    if code != 0:
        raise MSPError(code, load().msp_last_error().decode(errors="replace"))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _np(a):
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_config(params: dict) -> Config:
    c = Config()
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
    c.centre_mode = int(params.get("centre_mode", 0))
    c.mac_mode = int(params.get("mac_mode", 0))
    c.c1 = int(params.get("c1", 70))
    c.c2 = int(params.get("c2", 70))
    return c


_live = weakref.WeakSet()


@atexit.register
def _close_all():
    """Destroy the contexts still alive at interpreter exit, while the CUDA
    runtime is still up (registered after torch, so it runs before torch's
    own exit handlers)."""
    for ctx in list(_live):
        try:
            ctx.close()
        except Exception:
            pass


class MSP:
    """One libmsp context on a CUDA device."""

    def __init__(self, params: dict, device: int = 0, frames=None):
        """frames: None, or (offsets, level) of independent networks in their
        own frames (msp_set_frames; the output of batch_layout)."""
        L = load()
        self.params = dict(params)
        self.device = device
        self._cfg = make_config(params)
        h = C.c_void_p()
        _check(L.msp_create(C.byref(h), C.byref(self._cfg), int(device)))
        self._h = h
        self.n = 0
        self._inputs = None
        _live.add(self)
        if frames is not None:
            self.set_frames(*frames)

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.synchronize(self.device)
            load().msp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the path -----------------------------------------------------------
    def build_tree(self, pos, type_, vac_axon, vac_dend_e, vac_dend_i, stream=None):
        """pos: (3, n) float32 CUDA tensor; the rest (n,) uint8 CUDA tensors."""
        pos = pos.contiguous()
        ins = [pos[0].contiguous(), pos[1].contiguous(), pos[2].contiguous(),
               type_.contiguous(), vac_axon.contiguous(), vac_dend_e.contiguous(),
               vac_dend_i.contiguous()]
        for t, dt in zip(ins, [torch.float32] * 3 + [torch.uint8] * 4):
            if not t.is_cuda or t.dtype != dt:
                raise TypeError("build_tree expects CUDA float32 positions and uint8 counts")
        self.n = int(pos.shape[1])
        self._inputs = ins
        _check(load().msp_build_tree(self._h, self.n, *[_ptr(t) for t in ins], _stream(stream)))

    def attraction(self, out=None, stream=None):
        u = out if out is not None else torch.empty(self.n, dtype=torch.float32, device="cuda")
        _check(load().msp_attraction(self._h, _ptr(u), _stream(stream)))
        return u

    def direct(self, out=None, stream=None):
        u = out if out is not None else torch.empty(self.n, dtype=torch.float32, device="cuda")
        _check(load().msp_direct(self._h, _ptr(u), _stream(stream)))
        return u

    def num_elements(self) -> int:
        return self.stats()["n_elements"]

    def select_partners(self, step: int, out=None, stream=None):
        ne = max(self.num_elements(), 1)
        if out is None:
            dev = "cuda"
            out = dict(partner=torch.empty(ne, dtype=torch.int32, device=dev),
                       syn_pre=torch.empty(ne, dtype=torch.int32, device=dev),
                       syn_post=torch.empty(ne, dtype=torch.int32, device=dev),
                       syn_type=torch.empty(ne, dtype=torch.uint8, device=dev),
                       n_syn=torch.zeros(1, dtype=torch.int64, device=dev))
        _check(load().msp_select_partners(self._h, int(step), _ptr(out["partner"]),
                                          _ptr(out["syn_pre"]), _ptr(out["syn_post"]),
                                          _ptr(out["syn_type"]), _ptr(out["n_syn"]),
                                          _stream(stream)))
        return out

    def plasticity_step_host(self, step, pos, type_, vac_axon, vac_dend_e, vac_dend_i,
                             out=None, want_u=True):
        """Whole step from host (numpy, ideally pinned) buffers; returns host results.
        Caller-given `out` buffers must hold sum(vac_axon) elements (partner,
        syn_*) and n floats (u), as msp_plasticity_step_host requires."""
        n = int(pos.shape[1])
        x, y, z = (np.ascontiguousarray(pos[d], dtype=np.float32) for d in range(3))
        t, a, e, i = (np.ascontiguousarray(v, dtype=np.uint8) for v in
                      (type_, vac_axon, vac_dend_e, vac_dend_i))
        if out is None:
            # sized by the vacant axonal elements (only when the caller gives no buffers)
            ne = max(int(a.sum(dtype=np.int64)), 1)
            out = dict(u=np.zeros(max(n, 1), np.float32), partner=np.zeros(ne, np.int32),
                       syn_pre=np.zeros(ne, np.int32), syn_post=np.zeros(ne, np.int32),
                       syn_type=np.zeros(ne, np.uint8), n_syn=np.zeros(1, np.int64))
        _check(load().msp_plasticity_step_host(
            self._h, n, int(step), _np(x), _np(y), _np(z), _np(t), _np(a), _np(e), _np(i),
            _np(out["u"]) if want_u else None, _np(out["partner"]), _np(out["syn_pre"]),
            _np(out["syn_post"]), _np(out["syn_type"]), _np(out["n_syn"])))
        return out

    def vacancy_walk(self, step, vac_axon, vac_dend_e, vac_dend_i, stream=None):
        _check(load().msp_vacancy_walk(self._h, int(vac_axon.numel()), int(step),
                                       _ptr(vac_axon), _ptr(vac_dend_e), _ptr(vac_dend_i),
                                       _stream(stream)))

    def commit_synapses(self, sel, vac_axon, vac_dend_e, vac_dend_i, stream=None):
        _check(load().msp_commit_synapses(self._h, _ptr(sel["n_syn"]), int(sel["syn_pre"].numel()),
                                          _ptr(sel["syn_pre"]), _ptr(sel["syn_post"]),
                                          _ptr(sel["syn_type"]), _ptr(vac_axon),
                                          _ptr(vac_dend_e), _ptr(vac_dend_i), _stream(stream)))

    def selftest_bounded_wait(self, stream=None):
        """Runs the device scan with a predecessor that never publishes; the
        bounded wait gives up: raises MSPError with code 4 (MSP_ERR_TIMEOUT)."""
        _check(load().msp_selftest_bounded_wait(self._h, _stream(stream)))

    # -- the neuron side of the model (Section 3.1) ------------------------------
    def neuron_steps(self, first_step, n_steps, params, edges, state, stream=None):
        """n_steps steps of activity, spikes, calcium and elements, in place on
        `state` (CUDA tensors, keys of NEURON_STATE)."""
        n = int(state["x"].numel())
        _check(load().msp_neuron_steps(
            self._h, n, int(first_step), int(n_steps), C.byref(params), _ptr(edges["n"]),
            int(edges["capacity"]), _ptr(edges["pre"]), _ptr(edges["post"]),
            *[_ptr(state[k]) for k, _ in NEURON_STATE], _stream(stream)))

    def update_synapses(self, step, state, edges, vac_axon, vac_dend_e, vac_dend_i,
                        stream=None):
        """Deletion of the synapses beyond floor(elements) and the vacancies
        (uint8 CUDA tensors, written)."""
        n = int(state["x"].numel())
        _check(load().msp_update_synapses(
            self._h, n, int(step), _ptr(state["z_axon"]), _ptr(state["z_dend_e"]),
            _ptr(state["z_dend_i"]), _ptr(edges["n"]), _ptr(edges["pre"]), _ptr(edges["post"]),
            _ptr(edges["type"]), int(edges["capacity"]), _ptr(vac_axon), _ptr(vac_dend_e),
            _ptr(vac_dend_i), _stream(stream)))

    def append_synapses(self, sel, edges, stream=None):
        """Append the synapses of a selection to the edge list."""
        _check(load().msp_append_synapses(
            self._h, _ptr(sel["n_syn"]), int(sel["syn_pre"].numel()), _ptr(sel["syn_pre"]),
            _ptr(sel["syn_post"]),
            _ptr(sel["syn_type"]), _ptr(edges["n"]), _ptr(edges["pre"]), _ptr(edges["post"]),
            _ptr(edges["type"]), int(edges["capacity"]), _stream(stream)))

    # -- derivatives ------------------------------------------------------------
    def attraction_grad(self, type_, vac_axon, vac_dend_e, vac_dend_i, g=None, want_u=True,
                        stream=None):
        """u, du/dsigma and (with g) the gradient of sum_t g_t u(t) with respect to
        w^E and w^I, over the near-field pairs of the last attraction, at the
        given counts (CUDA uint8 tensors, caller order)."""
        n = self.n
        dev = type_.device
        ins = [t.contiguous() for t in (type_, vac_axon, vac_dend_e, vac_dend_i)]
        out = dict(u=torch.empty(n, dtype=torch.float32, device=dev) if want_u else None,
                   du_dsigma=torch.empty(n, dtype=torch.float32, device=dev))
        gg = None
        if g is not None:
            gg = g.to(torch.float32).contiguous()
            out["grad_w_e"] = torch.empty(n, dtype=torch.float32, device=dev)
            out["grad_w_i"] = torch.empty(n, dtype=torch.float32, device=dev)
        _check(load().msp_attraction_grad(
            self._h, *[_ptr(t) for t in ins], _ptr(gg), _ptr(out["u"]), _ptr(out["du_dsigma"]),
            _ptr(out.get("grad_w_e")), _ptr(out.get("grad_w_i")), _stream(stream)))
        return out

    def length_loss(self, type_, vac_axon, w_e, w_i, target, grad=True, stream=None):
        """The expected mean synapse length m, the loss (m - target)^2, its
        sigma derivatives and (grad) dloss/dw^E, dloss/dw^I over the
        near-field pairs of the last attraction (msp_length_loss)."""
        n = self.n
        dev = type_.device
        ins = [type_.contiguous(), vac_axon.contiguous()]
        ws = [w_e.to(torch.float32).contiguous(), w_i.to(torch.float32).contiguous()]
        for t, dt in zip(ins + ws, [torch.uint8] * 2 + [torch.float32] * 2):
            if t.device != dev or t.dtype != dt or t.numel() != n:
                raise TypeError(f"length_loss expects {n} entries on {dev} per array")
        out = np.zeros(4, np.float64)
        gE = torch.empty(n, dtype=torch.float32, device=dev) if grad else None
        gI = torch.empty(n, dtype=torch.float32, device=dev) if grad else None
        _check(load().msp_length_loss(self._h, *[_ptr(t) for t in ins + ws], float(target),
                                      _np(out), _ptr(gE), _ptr(gI), _stream(stream)))
        return dict(loss=float(out[0]), mean=float(out[1]), dloss_dsigma=float(out[2]),
                    dmean_dsigma=float(out[3]), gE=gE, gI=gI)

    def set_sigma(self, sigma: float):
        """New kernel width; the next attraction rebuilds the pair lists."""
        _check(load().msp_set_sigma(self._h, float(sigma)))
        self.params["sigma"] = float(sigma)
        self._cfg.sigma = float(sigma)

    def set_frames(self, offsets, level: int, leaf_capacity=None, cutoff=None):
        """Independent networks in their own frames: network k holds neurons
        [offsets[k], offsets[k+1]) with positions relative to its own cell at
        `level` (msp_set_frames), optionally with its own leaf capacity and
        cutoff; offsets=None removes them."""
        if offsets is None:
            _check(load().msp_set_frames(self._h, 0, None, 0, None, None))
            return
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if off.ndim != 1 or len(off) < 2:
            raise ValueError("offsets must hold at least two entries")
        nn = len(off) - 1
        cap = cut = None
        if leaf_capacity is not None:
            cap = np.ascontiguousarray(leaf_capacity, dtype=np.int32)
            if cap.shape != (nn,):
                raise ValueError("one leaf capacity per network")
        if cutoff is not None:
            cut = np.ascontiguousarray(cutoff, dtype=np.float64)
            if cut.shape != (nn,):
                raise ValueError("one cutoff per network")
        _check(load().msp_set_frames(self._h, nn, _np(off), int(level),
                                     None if cap is None else _np(cap),
                                     None if cut is None else _np(cut)))

    # -- the whole step as a CUDA graph ---------------------------------------
    def step_graph_capture(self, pos, type_, vac_axon, vac_dend_e, vac_dend_i, first_step,
                           history_len=0, stream=None):
        """Captures walk + build + attraction + selection + commit on these CUDA
        tensors (the vacant counts are updated in place by every replay).
        build_tree and attraction must have run on the same positions.  Returns
        the output tensors the replays write."""
        pos = pos.contiguous()
        n = int(pos.shape[1])
        cap = max(MAX_VACANCY * n, 1)
        dev = pos.device
        xs = [pos[0].contiguous(), pos[1].contiguous(), pos[2].contiguous()]
        st = [type_.contiguous(), vac_axon, vac_dend_e, vac_dend_i]
        for t in st[1:]:
            if not t.is_contiguous():
                raise ValueError("vacant counts must be contiguous (updated in place)")
        out = dict(partner=torch.empty(cap, dtype=torch.int32, device=dev),
                   syn_pre=torch.empty(cap, dtype=torch.int32, device=dev),
                   syn_post=torch.empty(cap, dtype=torch.int32, device=dev),
                   syn_type=torch.empty(cap, dtype=torch.uint8, device=dev),
                   n_syn=torch.zeros(1, dtype=torch.int64, device=dev),
                   history=torch.full((max(int(history_len), 1),), -1, dtype=torch.int64,
                                      device=dev))
        self._graph_inputs = xs + st + [out]
        _check(load().msp_step_graph_capture(
            self._h, n, *[_ptr(t) for t in xs], *[_ptr(t) for t in st], _ptr(out["partner"]),
            _ptr(out["syn_pre"]), _ptr(out["syn_post"]), _ptr(out["syn_type"]), cap,
            _ptr(out["n_syn"]), _ptr(out["history"]) if history_len else None, int(history_len),
            int(first_step), _stream(stream)))
        return out

    def step_graph_set_full_build(self, full_build: bool):
        """Option of the next capture: every replay rebuilds the whole octree
        (True) or reuses the eager build's octree (False, the default)."""
        _check(load().msp_step_graph_set_full_build(self._h, 1 if full_build else 0))

    def step_graph_launch(self, n_steps, stream=None):
        _check(load().msp_step_graph_launch(self._h, int(n_steps), _stream(stream)))

    def step_graph_finish(self, stream=None):
        """Waits for the replays; returns (next step index, halt bits)."""
        nxt, halted = C.c_uint64(0), C.c_int64(0)
        _check(load().msp_step_graph_finish(self._h, _stream(stream), C.byref(nxt),
                                            C.byref(halted)))
        return int(nxt.value), int(halted.value)

    def run_steps(self, first_step, n_steps, stream=None):
        """Replays the captured step until steps first_step .. first_step+n_steps-1
        have run (a halted step is finished eagerly and the graph re-captured)."""
        step, end = int(first_step), int(first_step) + int(n_steps)
        while step < end:
            self.step_graph_launch(end - step, stream)
            step, _ = self.step_graph_finish(stream)
        return step

    def set_pair_capacity(self, pairs):
        _check(load().msp_set_pair_capacity(self._h, int(pairs)))

    # -- introspection ------------------------------------------------------
    def stats(self) -> dict:
        s = Stats()
        _check(load().msp_get_stats(self._h, C.byref(s)))
        return {name: (float if name.endswith("_ms") else int)(getattr(s, name))
                for name, _ in Stats._fields_}

    def export_tree(self):
        st = self.stats()
        n, m = st["n"], st["n_nodes"]
        out = dict(keys=np.zeros(max(n, 1), np.uint64), perm=np.zeros(max(n, 1), np.int32),
                   level=np.zeros(m, np.uint8), prefix=np.zeros(m, np.uint64),
                   first=np.zeros(m, np.int32), count=np.zeros(m, np.int32),
                   parent=np.zeros(m, np.int32), child_first=np.zeros(m, np.int32),
                   nchild=np.zeros(m, np.uint8), sums=np.zeros((m, 4), np.int32),
                   centroids=np.zeros((m, 6), np.float32))
        _check(load().msp_export_tree(self._h, *[_np(out[k]) for k in
                                                 ("keys", "perm", "level", "prefix", "first",
                                                  "count", "parent", "child_first", "nchild",
                                                  "sums", "centroids")]))
        out["keys"], out["perm"] = out["keys"][:n], out["perm"][:n]
        return out

    def export_pairs(self):
        st = self.stats()
        m, nd = st["n_pairs"], st["pair_depths"]
        out = dict(X=np.zeros(m, np.int32), Y=np.zeros(m, np.int32), kind=np.zeros(m, np.uint8),
                   child_first=np.zeros(m, np.int32), wE=np.zeros(m), wI=np.zeros(m),
                   depth_start=np.zeros(nd + 1, np.int64))
        _check(load().msp_export_pairs(self._h, *[_np(out[k]) for k in
                                                  ("X", "Y", "kind", "child_first", "wE", "wI",
                                                   "depth_start")]))
        return out

    def export_expansions(self):
        st = self.stats()
        p3 = self._cfg.p ** 3
        m = st["expansion_nodes"]
        A, M, B = (np.zeros((max(m, 1), 2, p3), np.float32) for _ in range(3))
        first = np.zeros(1, np.int64)
        _check(load().msp_export_expansions(self._h, _np(A), _np(M), _np(B), _np(first)))
        return A[:m], M[:m], B[:m], int(first[0])


class SynapseLengthLoss(torch.autograd.Function):
    """loss = (m(sigma, w^E, w^I) - target)^2 for the expected mean synapse
    length m (msp_length_loss) as a differentiable function of sigma (a 0-d
    tensor) and the dendritic weights (n-vectors): forward sets sigma, redoes
    the attraction's pair lists and computes the loss and its gradient in
    the library; backward scales that gradient by the incoming one.

        loss = SynapseLengthLoss.apply(sigma, w_e, w_i, ctx, type_, vac_axon, target)
    """

    @staticmethod
    def forward(fctx, sigma, w_e, w_i, ctx, type_, vac_axon, target):
        ctx.set_sigma(float(sigma))
        ctx.attraction()
        r = ctx.length_loss(type_, vac_axon, w_e.detach(), w_i.detach(), float(target), grad=True)
        fctx.save_for_backward(r["gE"], r["gI"])
        fctx.dsigma = r["dloss_dsigma"]
        fctx.mean = r["mean"]
        return torch.tensor(r["loss"], dtype=torch.float64, device=w_e.device)

    @staticmethod
    def backward(fctx, grad_out):
        gE, gI = fctx.saved_tensors
        go = grad_out.to(torch.float64)
        return (go * fctx.dsigma, (go * gE.double()).to(gE.dtype), (go * gI.double()).to(gI.dtype),
                None, None, None, None)


def direct_noalloc(pos, type_, vac_axon, vac_dend_e, vac_dend_i, sigma, out=None, stream=None):
    """msp_direct_noalloc: all-pairs attraction without any device allocation
    by the library, for callers that cannot allocate (n <= NOALLOC_MAX_N).
    `out` (n float32, CUDA) may be preallocated by the caller."""
    if pos.dim() != 2 or pos.shape[0] != 3:
        raise ValueError("pos must be a (3, n) tensor")
    n = int(pos.shape[1])
    dev = pos.device
    if dev.type != "cuda" or pos.dtype != torch.float32:
        raise TypeError("pos must be a float32 CUDA tensor")
    counts = [type_.contiguous(), vac_axon.contiguous(), vac_dend_e.contiguous(),
              vac_dend_i.contiguous()]
    for t in counts:
        if t.device != dev or t.dtype != torch.uint8 or t.numel() != n:
            raise TypeError(f"counts must be uint8 tensors of {n} entries on {dev}")
    if out is not None and (out.device != dev or out.dtype != torch.float32
                            or out.numel() != n or not out.is_contiguous()):
        raise TypeError(f"out must be a contiguous float32 tensor of {n} entries on {dev}")
    # the library launches on the current device: make it pos's device, and
    # take that device's current stream unless one is given
    with torch.cuda.device(dev):
        xs = [pos[d].contiguous() for d in range(3)]
        u = out if out is not None else torch.empty(n, dtype=torch.float32, device=dev)
        _check(load().msp_direct_noalloc(n, *[_ptr(t) for t in xs], *[_ptr(t) for t in counts],
                                         float(sigma), _ptr(u),
                                         _stream(stream if stream is not None else
                                                 torch.cuda.current_stream(dev))))
    return u


def philox(ctr, key, stream=None):
    """msp_philox: the library's device Philox4x32-10 on (n, 4) uint32 counters
    and (n, 2) uint32 keys (CUDA int32 tensors holding the uint32 bits);
    returns the (n, 4) output blocks (int32 tensor holding the bits)."""
    ctr = ctr.contiguous()
    key = key.contiguous()
    if ctr.dim() != 2 or ctr.shape[1] != 4 or key.shape != (ctr.shape[0], 2):
        raise ValueError("ctr must be (n, 4) and key (n, 2)")
    for t in (ctr, key):
        if not t.is_cuda or t.dtype != torch.int32 or t.device != ctr.device:
            raise TypeError("ctr and key must be int32 CUDA tensors on one device")
    out = torch.empty_like(ctr)
    with torch.cuda.device(ctr.device):
        _check(load().msp_philox(int(ctr.shape[0]), _ptr(ctr), _ptr(key), _ptr(out),
                                 _stream(stream if stream is not None else
                                         torch.cuda.current_stream(ctr.device))))
    return out


def batch_layout(pos, offsets, sigma, cutoff, leaf_capacity, stream=None):
    """Lays the networks of a batch (pos: (3, N) float32 CUDA tensor of the
    concatenated networks; offsets: N_net + 1 int64; sigma: per network) out
    as one problem of kernel width 1, each network in its own cell.  Returns
    (local (3, N) tensor: sigma units relative to the network's cell, side,
    cell level); a context then takes frames=(offsets, level)."""
    pos = pos.contiguous()
    if not pos.is_cuda or pos.dtype != torch.float32:
        raise TypeError("batch_layout expects CUDA float32 positions")
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    if len(off) != len(sig) + 1:
        raise ValueError("offsets must have one entry more than sigma")
    xs = [pos[d].contiguous() for d in range(3)]
    out = torch.empty_like(pos)
    side, level = C.c_float(0.0), C.c_int(0)
    _check(load().msp_batch_layout(len(sig), _np(off), *[_ptr(t) for t in xs], _np(sig),
                                   float(cutoff), int(leaf_capacity), _ptr(out[0]), _ptr(out[1]),
                                   _ptr(out[2]), C.byref(side), C.byref(level), _stream(stream)))
    return out, float(side.value), int(level.value)


def set_workspace_limit(nbytes: int):
    """Cap the device memory all contexts' workspaces may hold (0: no cap)."""
    _check(load().msp_set_workspace_limit(int(nbytes)))


def workspace_bytes() -> int:
    return int(load().msp_workspace_bytes())


def to_device(w, device="cuda"):
    """Move a workload's arrays to the GPU (pos (3,n) f32, counts u8)."""
    return (torch.from_numpy(np.ascontiguousarray(w.pos)).to(device),
            torch.from_numpy(w.type).to(device), torch.from_numpy(w.vac_axon).to(device),
            torch.from_numpy(w.vac_dend_e).to(device), torch.from_numpy(w.vac_dend_i).to(device))
