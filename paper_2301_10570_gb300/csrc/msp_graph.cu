// msp_graph.cu -- one whole plasticity step (vacancy walk, a1-a12, commit)
// captured as a CUDA graph and replayed once per step; and the host-buffer
// call's own graph of a1-a12 alone.
//
// Every size inside the step lives in device memory, so the captured launch
// shapes come from capacity bounds: the pair table's capacity (sized by an
// eager attraction with headroom), the element capacity (the bound kMaxVacancy
// * n that the walk keeps, or the host-buffer call's own), and the node bound
// of the tree of the same positions.  The step index of the Philox counters is
// read from device memory and advanced by the graph itself.  A step that would
// exceed a capacity sets a halt flag before its commit; from then on the walk
// and the commit of every replay do nothing, and the host finishes the halted
// step eagerly (growing what overflowed) and captures the graph again.
//
// By default a replay reuses the octree of the last eager build (neurons do
// not move: the tree depends on the positions only) and refreshes its counts
// and aggregates, checked by a checksum of the positions and the build's
// generation stamp; with the full-build option every replay runs the whole
// build (Morton keys, sort, octree, aggregates).
#include <cstring>

#include "msp_internal.cuh"

namespace msp {

void build_tree(msp_ctx& c, int64_t n, const float* x, const float* y, const float* z,
                const uint8_t* type, const uint8_t* va, const uint8_t* vde, const uint8_t* vdi,
                cudaStream_t s);
void attraction(msp_ctx& c, float* u_dev, cudaStream_t s);
void select_partners(msp_ctx& c, uint64_t step, const uint8_t* type_dev, const uint8_t* va_dev,
                     const uint8_t* vde_dev, const uint8_t* vdi_dev, int32_t* partner,
                     int32_t* syn_pre, int32_t* syn_post, uint8_t* syn_type, int64_t* n_syn,
                     cudaStream_t s);
void vacancy_walk(msp_ctx& c, int64_t n, uint64_t step, uint8_t* va, uint8_t* vde, uint8_t* vdi,
                  cudaStream_t s);
void commit_synapses(msp_ctx& c, const int64_t* n_syn, int64_t capacity, const int32_t* pre,
                     const int32_t* post, const uint8_t* styp, uint8_t* va, uint8_t* vde,
                     uint8_t* vdi, cudaStream_t s);

namespace {

// halt bits
constexpr int64_t kHaltPairs = 1, kHaltItems = 2, kHaltLevels = 4, kHaltDescent = 8,
                  kHaltElements = 16;

__global__ void k_graph_init(DevCounts* dc, uint64_t step, int64_t halt) {
    dc->step = step;
    dc->halt = halt;
    dc->steps_run = 0;
    dc->interactions_run = 0;
}

// after the build: more elements than the selection's buffers hold leave the
// step with no element (every element kernel is bounded by the count)
__global__ void k_graph_guard(DevCounts* dc, int64_t elem_cap) {
    if (dc->n_elem > elem_cap) {
        dc->halt |= kHaltElements;
        dc->n_elem = 0;
    }
}

// after the selection, before the commit
__global__ void k_graph_check(DevCounts* dc, int left_slot) {
    int64_t bad = 0;
    if (dc->overflow & 1) bad |= kHaltPairs;
    if (dc->overflow & 38) bad |= kHaltItems;
    if (dc->more_levels > 0 || (dc->overflow & 16) || dc->bad_pos) bad |= kHaltLevels;
    if (dc->items[left_slot] != 0) bad |= kHaltDescent;
    dc->halt |= bad;
}

__global__ void k_graph_step_end(DevCounts* dc, int64_t* history, int64_t len, uint64_t first) {
    dc->interactions_run += dc->interactions;   // the near field runs in every replay
    if (dc->halt) return;
    const uint64_t k = dc->step - first;
    if (history && k < (uint64_t)len) history[k] = dc->n_syn;
    dc->step += 1;
    dc->steps_run += 1;
}

// graph mode for the dry run and the capture, with the graph's options
struct GraphModeScope {
    msp_ctx& c;
    GraphModeScope(msp_ctx& cc, const msp_ctx::GraphArgs& g) : c(cc) {
        c.graph_mode = true;
        c.graph_elem_cap = g.elem_cap;
        c.graph_full_build = g.full_build;
    }
    ~GraphModeScope() {
        c.graph_mode = false;
        c.graph_full_build = false;
    }
};

// one step in graph mode on the stream (captured or, for the dry run, eager)
void record_step(msp_ctx& c, const msp_ctx::GraphArgs& g, cudaStream_t s) {
    DevCounts* dc = dcounts(c);
    if (g.walk) vacancy_walk(c, g.n, 0, g.va, g.vde, g.vdi, s);
    build_tree(c, g.n, g.x, g.y, g.z, g.type, g.va, g.vde, g.vdi, s);
    k_graph_guard<<<1, 1, 0, s>>>(dc, g.elem_cap);
    MSP_LAUNCH("graph_guard");
    attraction(c, g.u, s);
    select_partners(c, 0, g.type, g.va, g.vde, g.vdi, g.partner, g.pre, g.post, g.styp, g.n_syn,
                    s);
    k_graph_check<<<1, 1, 0, s>>>(dc, c.cap_left_slot);
    MSP_LAUNCH("graph_check");
    if (g.commit)
        commit_synapses(c, g.n_syn, g.capacity, g.pre, g.post, g.styp, g.va, g.vde, g.vdi, s);
    k_graph_step_end<<<1, 1, 0, s>>>(dc, g.history, g.history_len, g.first_step);
    MSP_LAUNCH("graph_step_end");
}

void release(msp_ctx::StepGraph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.tmpl) cudaGraphDestroy(G.tmpl);
    G.exec = nullptr;
    G.tmpl = nullptr;
    G.nf0 = G.nf1 = nullptr;
    G.kernels = 0;
}

// Sizes the workspace for the graph's capacity bounds with a dry run, then
// records one step on a stream of its own and instantiates it into G.
void capture(msp_ctx& c, msp_ctx::StepGraph& G, const msp_ctx::GraphArgs& args, cudaStream_t s) {
    if (!c.tree_built || !c.attraction_done || c.n != args.n)
        throw Error(MSP_ERR_NOT_BUILT,
                    "build the tree of these positions and run the attraction once first");
    release(G);
    DevCounts* dc = dcounts(c);
    {
        // Dry run with the halt flag set: sizes every buffer for the graph's
        // capacity bounds (the walk and the commit change nothing; the
        // selection and the attraction write into scratch of the context).
        // A pair table too small for it grows first.
        GraphModeScope gm(c, args);
        const size_t ecap = (size_t)std::max<int64_t>(args.elem_cap, 1);
        msp_ctx::GraphArgs dry = args;
        dry.partner = c.h_partner.ensure<int32_t>(ecap);
        dry.pre = c.h_pre.ensure<int32_t>(ecap);
        dry.post = c.h_post.ensure<int32_t>(ecap);
        dry.styp = c.h_type.ensure<uint8_t>(ecap);
        dry.n_syn = c.h_nsyn.ensure<int64_t>(1);
        dry.u = args.u ? c.h_u.ensure<float>((size_t)std::max<int64_t>(args.n, 1)) : nullptr;
        dry.capacity = (int64_t)ecap;
        dry.history = nullptr;
        dry.history_len = 0;
        for (int attempt = 0;; ++attempt) {
            k_graph_init<<<1, 1, 0, s>>>(dc, args.first_step, 1);
            MSP_LAUNCH("graph_init");
            record_step(c, dry, s);
            pull_counts(c, s);
            const DevCounts& hc = *c.hcount;
            if (hc.more_levels > 0)
                throw Error(MSP_ERR_NOT_BUILT, "the tree of these positions is deeper than built");
            if (!(hc.overflow & 1)) break;
            if (attempt >= 8) throw Error(MSP_ERR_CAPACITY, "pair table overflow after growth");
            c.pair_cap = std::max(2 * c.pair_cap, hc.need_pairs + hc.need_pairs / 2 + 1024);
        }
    }
    // the capture itself runs on a stream of the context (the caller's may be
    // the legacy default stream, which cannot capture)
    cudaStream_t cs = nullptr;
    MSP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    const long long k0 = g_kernel_launches.load();
    try {
        GraphModeScope gm(c, args);
        MSP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            record_step(c, args, cs);
        } catch (...) {
            cudaGraph_t dead = nullptr;
            cudaStreamEndCapture(cs, &dead);
            if (dead) cudaGraphDestroy(dead);
            throw;
        }
        MSP_CUDA(cudaStreamEndCapture(cs, &graph));
        G.left_slot = c.cap_left_slot;
        // kernels were only recorded, not run
        G.kernels = g_kernel_launches.load() - k0;
        g_kernel_launches -= G.kernels;
        size_t nn = 0;
        MSP_CUDA(cudaGraphGetNodes(graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        MSP_CUDA(cudaGraphGetNodes(graph, nodes.data(), &nn));
        cudaGraphNode_t e0 = nullptr, e1 = nullptr;
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            MSP_CUDA(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            MSP_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            if (ev == c.ev_nf0) e0 = nd;
            if (ev == c.ev_nf1) e1 = nd;
        }
        MSP_CUDA(cudaGraphInstantiate(&G.exec, graph, 0));
        // nodes of the instantiated graph are addressed through the template's
        G.nf0 = e0;
        G.nf1 = e1;
        k_graph_init<<<1, 1, 0, s>>>(dc, args.first_step, 0);
        MSP_LAUNCH("graph_init");
        MSP_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        release(G);
        throw;
    }
    // the event-record nodes are addressed through the template graph, so
    // it lives as long as the executable graph
    G.tmpl = graph;
    G.epoch = g_alloc_epoch.load();
    G.args = args;
    cudaStreamDestroy(cs);
}

}  // namespace

void graph_release(msp_ctx& c) {
    release(c.sg);
    release(c.hg);
    c.g_replays = 0;
}

void graph_capture(msp_ctx& c, const msp_ctx::GraphArgs& a, cudaStream_t s) {
    NvtxRange nv_("msp step_graph_capture");
    msp_ctx::GraphArgs args = a;
    args.elem_cap = (int64_t)kMaxVacancy * args.n;
    args.walk = true;
    args.commit = true;
    args.u = nullptr;
    args.full_build = c.sg_full_build;
    c.g_replays = 0;
    capture(c, c.sg, args, s);
}

void graph_launch(msp_ctx& c, int64_t n_steps, cudaStream_t s) {
    NvtxRange nv_("msp step_graph_launch");
    msp_ctx::StepGraph& G = c.sg;
    if (!G.exec) throw Error(MSP_ERR_NOT_BUILT, "no captured step graph");
    // a workspace buffer reallocated since the capture (by an eager call)
    // would leave the graph's kernels pointing at freed memory
    if (g_alloc_epoch.load() != G.epoch)
        throw Error(MSP_ERR_NOT_BUILT, "workspace changed since the capture: capture again");
    // replays accumulate until graph_finish; each has its own event pair
    const size_t need = (size_t)(2 * (c.g_replays + n_steps));
    while (c.g_events.size() < need) {
        cudaEvent_t e = nullptr;
        MSP_CUDA(cudaEventCreate(&e));
        c.g_events.push_back(e);
    }
    c.attraction_done = false;      // eager calls need a fresh build afterwards
    for (int64_t i = c.g_replays; i < c.g_replays + n_steps; ++i) {
        if (G.nf0 && G.nf1) {
            MSP_CUDA(cudaGraphExecEventRecordNodeSetEvent(G.exec, G.nf0, c.g_events[2 * i]));
            MSP_CUDA(cudaGraphExecEventRecordNodeSetEvent(G.exec, G.nf1, c.g_events[2 * i + 1]));
        }
        MSP_CUDA(cudaGraphLaunch(G.exec, s));
        g_kernel_launches += G.kernels;
    }
    c.g_replays += n_steps;
}

// Waits for the launched replays.  If a step halted, finishes it eagerly
// (growing what overflowed) and captures the graph again from the next step.
// Returns the index of the next step to run and whether a halt was handled.
void graph_finish(msp_ctx& c, cudaStream_t s, uint64_t* next_step, int64_t* halted) {
    NvtxRange nv_("msp step_graph_finish");
    msp_ctx::StepGraph& G = c.sg;
    if (!G.exec) throw Error(MSP_ERR_NOT_BUILT, "no captured step graph");
    pull_counts(c, s);
    const DevCounts hc = *c.hcount;
    MSP_CUDA(cudaMemsetAsync(&dcounts(c)->interactions_run, 0, sizeof(int64_t), s));
    double tot = 0.0;
    int64_t cnt = 0;
    if (G.nf0 && G.nf1)
        for (int64_t i = 0; i < c.g_replays; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c.g_events[2 * i], c.g_events[2 * i + 1]) == cudaSuccess) {
                tot += ms;
                ++cnt;
            }
        }
    c.g_nf_ms_mean = cnt ? tot / (double)cnt : 0.0;
    // statistics of the replays: the last one's sizes, the mean near-field work
    c.last_was_graph = true;
    c.n_pairs = hc.depth_start[std::min(c.tree_depth + 1, kMaxLevels + 2)];
    c.n_far = hc.n_far;
    c.n_p2p = hc.n_p2p;
    c.n_p2p_targets = hc.nseg;
    c.n_elem = hc.n_elem;
    c.n_draws = hc.draws;
    c.n_requests = hc.n_req;
    c.n_synapses = hc.n_syn;
    c.p2p_interactions = c.g_replays > 0 ? hc.interactions_run / c.g_replays : hc.interactions;
    c.g_replays = 0;
    *halted = hc.halt;
    if (hc.halt == 0) {
        *next_step = hc.step;
        return;
    }
    if (hc.halt & kHaltElements)
        throw Error(MSP_ERR_INVALID_ARG, "vacant element count above the walk's bound");
    // The halted step's walk has run; finish the step eagerly.
    msp_ctx::GraphArgs g = G.args;
    const uint64_t k = hc.step;
    build_tree(c, g.n, g.x, g.y, g.z, g.type, g.va, g.vde, g.vdi, s);
    attraction(c, nullptr, s);
    select_partners(c, k, g.type, g.va, g.vde, g.vdi, g.partner, g.pre, g.post, g.styp, g.n_syn,
                    s);
    commit_synapses(c, g.n_syn, g.capacity, g.pre, g.post, g.styp, g.va, g.vde, g.vdi, s);
    if (g.history && k - g.first_step < (uint64_t)g.history_len)
        MSP_CUDA(cudaMemcpyAsync(g.history + (k - g.first_step), g.n_syn, sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    // capture again from the next step; the history keeps its origin
    const uint64_t first = g.first_step;
    g.first_step = k + 1;
    if (g.history) {
        const uint64_t skip = k + 1 - first;
        if (skip < (uint64_t)g.history_len) {
            g.history += skip;
            g.history_len -= (int64_t)skip;
        } else {
            g.history = nullptr;
            g.history_len = 0;
        }
    }
    graph_capture(c, g, s);
    *next_step = k + 1;
}

// The host-buffer step (msp_plasticity_step_host): the inputs are copied to
// the context's staging buffers, steps a1-a12 run, and u, the partners and the
// synapses are copied back.  The first call (and any call after which the
// graph cannot serve: another size, a reallocated workspace, more vacant
// elements than its buffers, changed positions) runs the path eagerly and
// captures a graph of it on the staging buffers; later calls replay that
// graph, which reuses the octree while the positions are the same (checksum)
// and reads the step index from device memory.
void host_step(msp_ctx& c, int64_t n, uint64_t step, const float* x, const float* y,
               const float* z, const uint8_t* type, const uint8_t* va, const uint8_t* vde,
               const uint8_t* vdi, float* u, int32_t* partner, int32_t* pre, int32_t* post,
               uint8_t* styp, int64_t* n_syn, cudaStream_t s) {
    NvtxRange nv_("msp plasticity_step_host");
    size_t nn = (size_t)(n > 0 ? n : 1);
    float* dx = c.h_in[0].ensure<float>(nn);
    float* dy = c.h_in[1].ensure<float>(nn);
    float* dz = c.h_in[2].ensure<float>(nn);
    uint8_t* dt = c.h_in[3].ensure<uint8_t>(nn);
    uint8_t* da = c.h_in[4].ensure<uint8_t>(nn);
    uint8_t* de = c.h_in[5].ensure<uint8_t>(nn);
    uint8_t* di = c.h_in[6].ensure<uint8_t>(nn);
    float* du = c.hs_u.ensure<float>(nn);
    if (n > 0) {
        MSP_CUDA(cudaMemcpyAsync(dx, x, n * 4, cudaMemcpyHostToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(dy, y, n * 4, cudaMemcpyHostToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(dz, z, n * 4, cudaMemcpyHostToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(dt, type, n, cudaMemcpyHostToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(da, va, n, cudaMemcpyHostToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(de, vde, n, cudaMemcpyHostToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(di, vdi, n, cudaMemcpyHostToDevice, s));
    }
    c.in_type = dt; c.in_va = da; c.in_vde = de; c.in_vdi = di;
    msp_ctx::StepGraph& G = c.hg;
    bool replayed = false;
    int64_t ne = 0, ns = 0;
    if (G.exec && n > 0 && G.args.n == n && G.epoch == g_alloc_epoch.load()) {
        DevCounts* dc = dcounts(c);
        k_graph_init<<<1, 1, 0, s>>>(dc, step, 0);
        MSP_LAUNCH("graph_init");
        MSP_CUDA(cudaGraphLaunch(G.exec, s));
        g_kernel_launches += G.kernels;
        pull_counts(c, s);
        const DevCounts& hc = *c.hcount;
        if (hc.halt == 0) {
            replayed = true;
            ne = hc.n_elem;
            ns = hc.n_syn;
            c.n_elem = ne;
            c.n_draws = hc.draws;
            c.n_requests = hc.n_req;
            c.n_synapses = ns;
            c.n_far = hc.n_far;
            c.n_p2p = hc.n_p2p;
            c.p2p_interactions = hc.interactions;
            c.last_was_graph = false;
            c.nf_timed = false;
            c.attraction_done = false;   // eager calls need a fresh build afterwards
        }
    }
    if (!replayed) {
        // eagerly, then a graph of the same step for the next calls
        build_tree(c, n, dx, dy, dz, dt, da, de, di, s);
        attraction(c, du, s);
        ne = c.n_elem;
        const size_t ecap = (size_t)std::max<int64_t>(ne + ne / 4 + 1024, 1);
        int32_t* dp = c.hs_partner.ensure<int32_t>(ecap);
        int32_t* dpre = c.hs_pre.ensure<int32_t>(ecap);
        int32_t* dpost = c.hs_post.ensure<int32_t>(ecap);
        uint8_t* dst = c.hs_type.ensure<uint8_t>(ecap);
        int64_t* dn = c.hs_nsyn.ensure<int64_t>(1);
        select_partners(c, step, dt, da, de, di, dp, dpre, dpost, dst, dn, s);
        ns = c.n_synapses;
        const int64_t draws = c.n_draws, requests = c.n_requests;
        if (n > 0) {
            msp_ctx::GraphArgs g;
            g.x = dx; g.y = dy; g.z = dz; g.type = dt;
            g.va = da; g.vde = de; g.vdi = di;
            g.n = n;
            g.partner = dp; g.pre = dpre; g.post = dpost; g.styp = dst;
            g.capacity = (int64_t)ecap;
            g.n_syn = dn;
            g.first_step = step;
            g.u = du;
            g.elem_cap = (int64_t)ecap;
            g.walk = false;
            g.commit = false;
            g.full_build = false;
            // a capture that cannot be made leaves the eager results valid;
            // the next call runs eagerly again
            try {
                capture(c, G, g, s);
            } catch (const Error&) {
                release(G);
            }
            // the capture's dry run overwrote the counts of this step's
            // statistics; its outputs went to scratch, not to this call's
            c.n_elem = ne;
            c.n_synapses = ns;
            c.n_draws = draws;
            c.n_requests = requests;
            c.attraction_done = true;
        }
    }
    if (u && n > 0) MSP_CUDA(cudaMemcpyAsync(u, c.hs_u.get<float>(), n * 4, cudaMemcpyDeviceToHost, s));
    if (ne > 0) {
        MSP_CUDA(cudaMemcpyAsync(partner, c.hs_partner.get<int32_t>(), ne * 4,
                                 cudaMemcpyDeviceToHost, s));
        if (ns > 0) {
            MSP_CUDA(cudaMemcpyAsync(pre, c.hs_pre.get<int32_t>(), ns * 4, cudaMemcpyDeviceToHost, s));
            MSP_CUDA(cudaMemcpyAsync(post, c.hs_post.get<int32_t>(), ns * 4,
                                     cudaMemcpyDeviceToHost, s));
            MSP_CUDA(cudaMemcpyAsync(styp, c.hs_type.get<uint8_t>(), ns, cudaMemcpyDeviceToHost, s));
        }
    }
    MSP_CUDA(cudaStreamSynchronize(s));
    *n_syn = ns;
}

}  // namespace msp
