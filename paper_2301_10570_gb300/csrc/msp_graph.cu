// msp_graph.cu -- one whole plasticity step (vacancy walk, a1-a12, commit)
// captured as a CUDA graph and replayed once per step.
//
// Every size inside the step lives in device memory, so the captured launch
// shapes come from capacity bounds: the pair table's capacity (sized by an
// eager attraction with headroom), the element bound kMaxVacancy * n that the
// walk keeps, and the node bound of the tree of the same positions.  The step
// index of the Philox counters is read from device memory and advanced by the
// graph itself.  A step that would exceed a capacity sets a halt flag before
// its commit; from then on the walk and the commit of every replay do nothing,
// and the host finishes the halted step eagerly (growing what overflowed) and
// captures the graph again.
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
    if (dc->overflow & 6) bad |= kHaltItems;
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

// one step in graph mode on the stream (captured or, for the dry run, eager)
void record_step(msp_ctx& c, cudaStream_t s) {
    const msp_ctx::GraphArgs& g = c.gargs;
    DevCounts* dc = dcounts(c);
    vacancy_walk(c, g.n, 0, g.va, g.vde, g.vdi, s);
    build_tree(c, g.n, g.x, g.y, g.z, g.type, g.va, g.vde, g.vdi, s);
    k_graph_guard<<<1, 1, 0, s>>>(dc, (int64_t)kMaxVacancy * g.n);
    MSP_LAUNCH("graph_guard");
    attraction(c, nullptr, s);
    select_partners(c, 0, g.type, g.va, g.vde, g.vdi, g.partner, g.pre, g.post, g.styp, g.n_syn,
                    s);
    k_graph_check<<<1, 1, 0, s>>>(dc, c.g_left_slot);
    MSP_LAUNCH("graph_check");
    commit_synapses(c, g.n_syn, g.capacity, g.pre, g.post, g.styp, g.va, g.vde, g.vdi, s);
    k_graph_step_end<<<1, 1, 0, s>>>(dc, g.history, g.history_len, g.first_step);
    MSP_LAUNCH("graph_step_end");
}

struct GraphModeScope {
    msp_ctx& c;
    explicit GraphModeScope(msp_ctx& cc) : c(cc) { c.graph_mode = true; }
    ~GraphModeScope() { c.graph_mode = false; }
};

}  // namespace

void graph_release(msp_ctx& c) {
    if (c.gexec) cudaGraphExecDestroy(c.gexec);
    if (c.g_template) cudaGraphDestroy(c.g_template);
    c.gexec = nullptr;
    c.g_template = nullptr;
    c.g_nf0 = c.g_nf1 = nullptr;
    c.graph_kernels = 0;
    c.g_replays = 0;
}

void graph_capture(msp_ctx& c, const msp_ctx::GraphArgs& args, cudaStream_t s) {
    NvtxRange nv_("msp step_graph_capture");
    if (!c.tree_built || !c.attraction_done || c.n != args.n)
        throw Error(MSP_ERR_NOT_BUILT,
                    "build the tree of these positions and run the attraction once first");
    graph_release(c);
    DevCounts* dc = dcounts(c);
    {
        GraphModeScope gm(c);
        // Dry run with the halt flag set: sizes every buffer for the graph's
        // capacity bounds (the walk and the commit change nothing; the
        // selection writes into scratch of the context).  A pair table too
        // small for it grows first.
        const size_t ecap = (size_t)std::max<int64_t>((int64_t)kMaxVacancy * args.n, 1);
        c.gargs = args;
        c.gargs.partner = c.h_partner.ensure<int32_t>(ecap);
        c.gargs.pre = c.h_pre.ensure<int32_t>(ecap);
        c.gargs.post = c.h_post.ensure<int32_t>(ecap);
        c.gargs.styp = c.h_type.ensure<uint8_t>(ecap);
        c.gargs.n_syn = c.h_nsyn.ensure<int64_t>(1);
        c.gargs.capacity = (int64_t)ecap;
        c.gargs.history = nullptr;
        c.gargs.history_len = 0;
        for (int attempt = 0;; ++attempt) {
            k_graph_init<<<1, 1, 0, s>>>(dc, args.first_step, 1);
            MSP_LAUNCH("graph_init");
            record_step(c, s);
            pull_counts(c, s);
            const DevCounts& hc = *c.hcount;
            if (hc.more_levels > 0)
                throw Error(MSP_ERR_NOT_BUILT, "the tree of these positions is deeper than built");
            if (!(hc.overflow & 1)) break;
            if (attempt >= 8) throw Error(MSP_ERR_CAPACITY, "pair table overflow after growth");
            c.pair_cap = std::max(2 * c.pair_cap, hc.need_pairs + hc.need_pairs / 2 + 1024);
        }
    }
    c.gargs = args;
    // the capture itself runs on a stream of the context (the caller's may be
    // the legacy default stream, which cannot capture)
    cudaStream_t cs = nullptr;
    MSP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    const long long k0 = g_kernel_launches.load();
    try {
        GraphModeScope gm(c);
        MSP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            record_step(c, cs);
        } catch (...) {
            cudaGraph_t dead = nullptr;
            cudaStreamEndCapture(cs, &dead);
            if (dead) cudaGraphDestroy(dead);
            throw;
        }
        MSP_CUDA(cudaStreamEndCapture(cs, &graph));
        // kernels were only recorded, not run
        c.graph_kernels = g_kernel_launches.load() - k0;
        g_kernel_launches -= c.graph_kernels;
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
        MSP_CUDA(cudaGraphInstantiate(&c.gexec, graph, 0));
        // nodes of the instantiated graph are addressed through the template's
        c.g_nf0 = e0;
        c.g_nf1 = e1;
        k_graph_init<<<1, 1, 0, s>>>(dc, args.first_step, 0);
        MSP_LAUNCH("graph_init");
        MSP_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        graph_release(c);
        throw;
    }
    // the event-record nodes are addressed through the template graph, so
    // it lives as long as the executable graph
    c.g_template = graph;
    c.g_epoch = g_alloc_epoch.load();
    cudaStreamDestroy(cs);
}

void graph_launch(msp_ctx& c, int64_t n_steps, cudaStream_t s) {
    NvtxRange nv_("msp step_graph_launch");
    if (!c.gexec) throw Error(MSP_ERR_NOT_BUILT, "no captured step graph");
    // a workspace buffer reallocated since the capture (by an eager call)
    // would leave the graph's kernels pointing at freed memory
    if (g_alloc_epoch.load() != c.g_epoch)
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
        if (c.g_nf0 && c.g_nf1) {
            MSP_CUDA(cudaGraphExecEventRecordNodeSetEvent(c.gexec, c.g_nf0, c.g_events[2 * i]));
            MSP_CUDA(cudaGraphExecEventRecordNodeSetEvent(c.gexec, c.g_nf1, c.g_events[2 * i + 1]));
        }
        MSP_CUDA(cudaGraphLaunch(c.gexec, s));
        g_kernel_launches += c.graph_kernels;
    }
    c.g_replays += n_steps;
}

// Waits for the launched replays.  If a step halted, finishes it eagerly
// (growing what overflowed) and captures the graph again from the next step.
// Returns the index of the next step to run and whether a halt was handled.
void graph_finish(msp_ctx& c, cudaStream_t s, uint64_t* next_step, int64_t* halted) {
    NvtxRange nv_("msp step_graph_finish");
    if (!c.gexec) throw Error(MSP_ERR_NOT_BUILT, "no captured step graph");
    pull_counts(c, s);
    const DevCounts hc = *c.hcount;
    MSP_CUDA(cudaMemsetAsync(&dcounts(c)->interactions_run, 0, sizeof(int64_t), s));
    double tot = 0.0;
    int64_t cnt = 0;
    if (c.g_nf0 && c.g_nf1)
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
    msp_ctx::GraphArgs g = c.gargs;
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

}  // namespace msp
