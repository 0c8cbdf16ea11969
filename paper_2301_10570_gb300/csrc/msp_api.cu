// msp_api.cu -- the C ABI of include/msp.h: argument checks, context
// lifetime, error conversion, and the host-buffer plasticity step.
#include <cmath>
#include <cstring>

#include "msp_internal.cuh"

namespace msp {
void build_tree(msp_ctx& c, int64_t n, const float* x, const float* y, const float* z,
                const uint8_t* type, const uint8_t* va, const uint8_t* vde, const uint8_t* vdi,
                cudaStream_t s);
void attraction(msp_ctx& c, float* u_dev, cudaStream_t s);
void direct(msp_ctx& c, float* u_dev, cudaStream_t s);
void select_partners(msp_ctx& c, uint64_t step, const uint8_t* type_dev, const uint8_t* va_dev,
                     const uint8_t* vde_dev, const uint8_t* vdi_dev, int32_t* partner,
                     int32_t* syn_pre, int32_t* syn_post, uint8_t* syn_type, int64_t* n_syn,
                     cudaStream_t s);
void vacancy_walk(msp_ctx& c, int64_t n, uint64_t step, uint8_t* va, uint8_t* vde, uint8_t* vdi,
                  cudaStream_t s);
void neuron_steps(msp_ctx& c, int64_t n, uint64_t first_step, int n_steps,
                  const msp_neuron_params& mp, const int64_t* n_edges, int64_t cap,
                  const int32_t* pre,
                  const int32_t* post, float* x, uint8_t* refr, float* calcium, float* za,
                  float* ze, float* zi, uint8_t* spiked, cudaStream_t s);
void update_synapses(msp_ctx& c, int64_t n, uint64_t step, const float* za, const float* ze,
                     const float* zi, int64_t* n_edges, int32_t* pre, int32_t* post, uint8_t* typ,
                     int64_t cap, uint8_t* va, uint8_t* ve, uint8_t* vi, cudaStream_t s);
void append_synapses(msp_ctx& c, const int64_t* n_syn, int64_t syn_cap, const int32_t* sp,
                     const int32_t* sq, const uint8_t* st, int64_t* n_edges, int32_t* pre, int32_t* post,
                     uint8_t* typ, int64_t cap, cudaStream_t s);
void commit_synapses(msp_ctx& c, const int64_t* n_syn, int64_t capacity, const int32_t* pre,
                     const int32_t* post, const uint8_t* styp, uint8_t* va, uint8_t* vde,
                     uint8_t* vdi, cudaStream_t s);
void attraction_grad(msp_ctx& c, const uint8_t* type, const uint8_t* va, const uint8_t* vde,
                     const uint8_t* vdi, const float* g, float* u, float* dud, float* gE,
                     float* gI, cudaStream_t s);
void scan_wait_selftest(msp_ctx& c, cudaStream_t s);
void length_loss(msp_ctx& c, const uint8_t* type, const uint8_t* va, const float* we,
                 const float* wi, double target, double* out4, float* gE, float* gI,
                 cudaStream_t s);
void graph_release(msp_ctx& c);
void graph_capture(msp_ctx& c, const msp_ctx::GraphArgs& args, cudaStream_t s);
void graph_launch(msp_ctx& c, int64_t n_steps, cudaStream_t s);
void graph_finish(msp_ctx& c, cudaStream_t s, uint64_t* next_step, int64_t* halted);
void host_step(msp_ctx& c, int64_t n, uint64_t step, const float* x, const float* y,
               const float* z, const uint8_t* type, const uint8_t* va, const uint8_t* vde,
               const uint8_t* vdi, float* u, int32_t* partner, int32_t* pre, int32_t* post,
               uint8_t* styp, int64_t* n_syn, cudaStream_t s);
}  // namespace msp

namespace {
thread_local std::string g_last_error;
}

namespace msp {
std::atomic<long long> g_kernel_launches{0};
std::atomic<long long> g_alloc_epoch{0};
std::atomic<long long> g_ws_bytes{0};
std::atomic<long long> g_ws_limit{0};
void set_last_error(const char* msg) { g_last_error = msg; }
}

namespace {

msp_status fail(msp_status code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

template <class F>
msp_status guarded(msp_ctx* c, F&& f) {
    if (!c) return fail(MSP_ERR_INVALID_ARG, "null context");
    try {
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) return fail(MSP_ERR_CUDA, cudaGetErrorString(e));
        f();
        g_last_error.clear();
        return MSP_OK;
    } catch (const msp::Error& e) {
        return fail(e.code, e.what());
    } catch (const std::bad_alloc&) {
        return fail(MSP_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(MSP_ERR_CUDA, e.what());
    }
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void require(bool ok, const char* msg) {
    if (!ok) throw msp::Error(MSP_ERR_INVALID_ARG, msg);
}

void derive(msp_ctx& c) {
    const msp_config& cfg = c.cfg;
    c.morton_scale = (float)((double)(1u << msp::kMortonBits) / (double)cfg.side);
    // boxes whose half-width is at most rho_max * sigma may carry expansions
    // (the count rule of Algorithm 2: boxes of every level)
    c.l_far = cfg.max_depth + 1;
    for (int l = 0; l <= cfg.max_depth; ++l)
        if ((double)cfg.side / std::ldexp(1.0, l + 1) <= cfg.rho_max * cfg.sigma) {
            c.l_far = l;
            break;
        }
    if (cfg.mac_mode == 1) c.l_far = 0;
    // with frames, a box above the frame level spans several networks: it
    // carries no expansion and is never translated
    if (c.frame_level > 0) c.l_far = std::max(c.l_far, c.frame_level);
    // prune a pair when (sum of squared gaps in boxes of level l) * side_l^2
    // >= (cutoff * sigma)^2; with per-network cutoffs, the largest of them for
    // pairs above the networks' cells, and each network's own below
    auto g2_of = [&](double cutoff, int l) {
        const double bl = (double)cfg.side / std::ldexp(1.0, l);
        const double r = cutoff * cfg.sigma / bl;
        return (long long)std::ceil(r * r);
    };
    double cmax = cfg.cutoff;
    for (double v : c.frame_cut_host) cmax = std::max(cmax, v);
    for (int l = 0; l <= msp::kMortonBits; ++l) c.g2[l] = g2_of(cmax, l);
    if (c.frame_plans) {
        const size_t nf = c.frame_cut_host.size();
        std::vector<long long> g2((size_t)nf * (msp::kMortonBits + 1));
        std::vector<float> rc2(nf);
        for (size_t k = 0; k < nf; ++k) {
            for (int l = 0; l <= msp::kMortonBits; ++l)
                g2[k * (msp::kMortonBits + 1) + l] = g2_of(c.frame_cut_host[k], l);
            const double rc = c.frame_cut_host[k] * cfg.sigma;
            rc2[k] = (float)(rc * rc);
        }
        MSP_CUDA(cudaMemcpy(c.frame_g2.ensure<long long>(g2.size()), g2.data(),
                            g2.size() * sizeof(long long), cudaMemcpyHostToDevice));
        MSP_CUDA(cudaMemcpy(c.frame_rc2.ensure<float>(nf), rc2.data(), nf * sizeof(float),
                            cudaMemcpyHostToDevice));
    }
}

}  // namespace

extern "C" {

const char* msp_last_error(void) { return g_last_error.c_str(); }

msp_status msp_create(msp_ctx** out, const msp_config* cfg, int device) {
    if (!out || !cfg) return fail(MSP_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (!(cfg->sigma > 0.0) || cfg->p < 1 || cfg->p > msp::kMaxP || cfg->leaf_capacity < 1 ||
        cfg->max_depth < 0 || cfg->max_depth > msp::kMortonBits || !(cfg->side > 0.0f) ||
        !(cfg->rho_max >= 0.0) || !(cfg->cutoff > 0.0) || !(cfg->cutoff <= 5.0) ||
        cfg->m2l_min_pairs < 0 || (cfg->centre_mode != 0 && cfg->centre_mode != 1) ||
        (cfg->mac_mode != 0 && cfg->mac_mode != 1) || cfg->c1 < 0 || cfg->c2 < 0 ||
        !std::isfinite(cfg->origin[0]) || !std::isfinite(cfg->origin[1]) ||
        !std::isfinite(cfg->origin[2]) || !std::isfinite(cfg->side))
        return fail(MSP_ERR_INVALID_ARG, "configuration value out of range");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(MSP_ERR_CUDA, cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(MSP_ERR_INVALID_ARG, "no such CUDA device");
    msp_ctx* c = new (std::nothrow) msp_ctx();
    if (!c) return fail(MSP_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->device = device;
    msp_status st = guarded(c, [&] {
        MSP_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
        MSP_CUDA(cudaEventCreate(&c->ev_nf0));
        MSP_CUDA(cudaEventCreate(&c->ev_nf1));
        MSP_CUDA(cudaMallocHost(reinterpret_cast<void**>(&c->hcount), sizeof(msp::DevCounts)));
        std::memset(c->hcount, 0, sizeof(msp::DevCounts));
        MSP_CUDA(cudaMemset(c->dcount.ensure<msp::DevCounts>(1), 0, sizeof(msp::DevCounts)));
        derive(*c);
    });
    if (st != MSP_OK) {
        msp_destroy(c);
        return st;
    }
    *out = c;
    return MSP_OK;
}

msp_status msp_destroy(msp_ctx* c) {
    if (!c) return MSP_OK;
    cudaSetDevice(c->device);
    msp::DBuf* bufs[] = {&c->keys0, &c->keys1, &c->vals0, &c->vals1, &c->perm, &c->inv, &c->pts,
                         &c->wts, &c->lw, &c->elem_off, &c->leaf_of, &c->nd_level, &c->nd_prefix,
                         &c->nd_first, &c->nd_count, &c->nd_parent, &c->nd_child_first,
                         &c->nd_nchild, &c->nd_sums, &c->nd_ca, &c->nd_cd, &c->nd_arrive, &c->pr_X, &c->pr_Y,
                         &c->pr_kind, &c->pr_cf, &c->pr_nb, &c->pr_w, &c->far_q, &c->split_q, &c->m2_key0,
                         &c->m2_key1, &c->m2_val0, &c->m2_val1, &c->m2_flag, &c->m2_off,
                         &c->m2_seg, &c->p2p_key0,
                         &c->p2p_key1, &c->p2p_val0, &c->p2p_val1, &c->seg_first, &c->seg_flag,
                         &c->nf_w32, &c->nf_okey0, &c->nf_okey1, &c->nf_oval0, &c->nf_oval1, &c->nf_src,
                         &c->nr_inp, &c->nr_bout, &c->nr_bin, &c->nr_xout, &c->nr_xin,
                         &c->nr_sout, &c->nr_sin, &c->nr_cnt, &c->nr_key0, &c->nr_key1,
                         &c->nr_val0, &c->nr_val1, &c->nr_del, &c->nr_keep, &c->nr_pos,
                         &c->nr_pre2, &c->nr_post2, &c->nr_typ2, &c->nd_gc, &c->gm_key0,
                         &c->gm_key1, &c->gm_q, &c->gm_q1, &c->gm_flag, &c->gm_gid,
                         &c->gm_gstart, &c->gm_ntile, &c->gm_toff, &c->gm_tiles, &c->gm_cnt,
                         &c->frame_off, &c->frame_cap, &c->frame_g2, &c->frame_rc2,
                         &c->gr_w, &c->gr_tmp, &c->gr_key0, &c->gr_key1, &c->gr_val0,
                         &c->gr_val1, &c->gr_flag, &c->gr_off, &c->gr_seg, &c->ln_sums,
                         &c->ln_part, &c->ln_coef,
                         &c->expA, &c->expM, &c->expB, &c->u_sorted, &c->items0, &c->items1,
                         &c->leaf_items, &c->rq_key0, &c->rq_val0,
                         &c->accepted, &c->acc_off, &c->rq_gcnt, &c->rq_goff, &c->cnt, &c->off, &c->scan_tmp,
                         &c->rs_hist, &c->h_u, &c->h_partner, &c->h_pre,
                         &c->h_post, &c->h_type, &c->h_nsyn, &c->hs_u, &c->hs_partner,
                         &c->hs_pre, &c->hs_post, &c->hs_type, &c->hs_nsyn, &c->c_type,
                         &c->c_va, &c->c_vde, &c->c_vdi};
    for (msp::DBuf* b : bufs) b->release();
    for (auto& b : c->h_in) b.release();
    if (c->hcount) cudaFreeHost(c->hcount);
    c->dcount.release();
    c->sd_tmp.release();
    if (c->ev_nf0) cudaEventDestroy(c->ev_nf0);
    if (c->ev_nf1) cudaEventDestroy(c->ev_nf1);
    msp::graph_release(*c);
    for (cudaEvent_t e : c->g_events) cudaEventDestroy(e);
    delete c;
    return MSP_OK;
}

msp_status msp_build_tree(msp_ctx* c, int64_t n, const float* x, const float* y, const float* z,
                          const uint8_t* type, const uint8_t* va, const uint8_t* vde,
                          const uint8_t* vdi, void* stream) {
    return guarded(c, [&] {
        require(n >= 0 && n < 0x7ffffffell, "n out of range");
        require(n == 0 || (x && y && z && type && va && vde && vdi), "null input pointer");
        cudaStream_t s = as_stream(stream);
        size_t nn = (size_t)(n > 0 ? n : 1);
        uint8_t* ct = c->c_type.ensure<uint8_t>(nn);
        uint8_t* ca = c->c_va.ensure<uint8_t>(nn);
        uint8_t* ce = c->c_vde.ensure<uint8_t>(nn);
        uint8_t* ci = c->c_vdi.ensure<uint8_t>(nn);
        if (n > 0) {
            MSP_CUDA(cudaMemcpyAsync(ct, type, n, cudaMemcpyDeviceToDevice, s));
            MSP_CUDA(cudaMemcpyAsync(ca, va, n, cudaMemcpyDeviceToDevice, s));
            MSP_CUDA(cudaMemcpyAsync(ce, vde, n, cudaMemcpyDeviceToDevice, s));
            MSP_CUDA(cudaMemcpyAsync(ci, vdi, n, cudaMemcpyDeviceToDevice, s));
        }
        c->in_type = ct; c->in_va = ca; c->in_vde = ce; c->in_vdi = ci;
        msp::build_tree(*c, n, x, y, z, ct, ca, ce, ci, s);
    });
}

msp_status msp_attraction(msp_ctx* c, float* u, void* stream) {
    return guarded(c, [&] { msp::attraction(*c, u, as_stream(stream)); });
}

msp_status msp_direct(msp_ctx* c, float* u, void* stream) {
    return guarded(c, [&] {
        require(u || (c && c->n == 0), "null output pointer");
        msp::direct(*c, u, as_stream(stream));
    });
}

msp_status msp_select_partners(msp_ctx* c, uint64_t step, int32_t* partner, int32_t* pre,
                               int32_t* post, uint8_t* styp, int64_t* n_syn, void* stream) {
    return guarded(c, [&] {
        require(n_syn != nullptr, "null n_syn");
        require(c->n_elem == 0 || (partner && pre && post && styp), "null output pointer");
        require(c->in_type != nullptr || c->n == 0, "inputs of the build are not available");
        msp::select_partners(*c, step, c->in_type, c->in_va, c->in_vde, c->in_vdi, partner, pre,
                             post, styp, n_syn, as_stream(stream));
    });
}

msp_status msp_plasticity_step_host(msp_ctx* c, int64_t n, uint64_t step, const float* x,
                                    const float* y, const float* z, const uint8_t* type,
                                    const uint8_t* va, const uint8_t* vde, const uint8_t* vdi,
                                    float* u, int32_t* partner, int32_t* pre, int32_t* post,
                                    uint8_t* styp, int64_t* n_syn) {
    return guarded(c, [&] {
        require(n >= 0 && n < 0x7ffffffell, "n out of range");
        require(n == 0 || (x && y && z && type && va && vde && vdi), "null input pointer");
        require(n_syn != nullptr, "null n_syn");
        require(n == 0 || (partner && pre && post && styp), "null output pointer");
        msp::host_step(*c, n, step, x, y, z, type, va, vde, vdi, u, partner, pre, post, styp,
                       n_syn, 0);
    });
}

msp_status msp_vacancy_walk(msp_ctx* c, int64_t n, uint64_t step, uint8_t* va, uint8_t* vde,
                            uint8_t* vdi, void* stream) {
    return guarded(c, [&] {
        require(n >= 0, "n out of range");
        require(n == 0 || (va && vde && vdi), "null pointer");
        msp::vacancy_walk(*c, n, step, va, vde, vdi, as_stream(stream));
    });
}

msp_status msp_commit_synapses(msp_ctx* c, const int64_t* n_syn, int64_t capacity,
                               const int32_t* pre, const int32_t* post, const uint8_t* styp,
                               uint8_t* va, uint8_t* vde, uint8_t* vdi, void* stream) {
    return guarded(c, [&] {
        require(capacity >= 0, "capacity out of range");
        require(capacity == 0 || (n_syn && pre && post && styp && va && vde && vdi),
                "null pointer");
        msp::commit_synapses(*c, n_syn, capacity, pre, post, styp, va, vde, vdi,
                             as_stream(stream));
    });
}

msp_status msp_selftest_bounded_wait(msp_ctx* c, void* stream) {
    return guarded(c, [&] { msp::scan_wait_selftest(*c, as_stream(stream)); });
}

msp_status msp_neuron_steps(msp_ctx* c, int64_t n, uint64_t first_step, int n_steps,
                            const msp_neuron_params* params, const int64_t* n_edges,
                            int64_t capacity, const int32_t* pre, const int32_t* post, float* x,
                            uint8_t* refr,
                            float* calcium, float* za, float* ze, float* zi, uint8_t* spiked,
                            void* stream) {
    return guarded(c, [&] {
        require(n >= 0 && n < 0x7fffffffll, "n out of range");
        require(n_steps >= 0, "n_steps out of range");
        require(capacity >= 0 && capacity < 0x7fffffffll, "capacity out of range");
        require(params != nullptr, "null parameters");
        require(params->refractory >= 0 && params->refractory <= 255, "refractory out of range");
        require(params->tau_x != 0.f && params->eps != params->eta_axon &&
                    params->eps != params->eta_dend, "degenerate parameters");
        require(n == 0 || (n_edges && pre && post && x && refr && calcium && za && ze && zi &&
                           spiked), "null pointer");
        msp::neuron_steps(*c, n, first_step, n_steps, *params, n_edges, capacity, pre, post, x,
                          refr,
                          calcium, za, ze, zi, spiked, as_stream(stream));
    });
}

msp_status msp_update_synapses(msp_ctx* c, int64_t n, uint64_t step, const float* za,
                               const float* ze, const float* zi, int64_t* n_edges, int32_t* pre,
                               int32_t* post, uint8_t* typ, int64_t capacity, uint8_t* va,
                               uint8_t* ve, uint8_t* vi, void* stream) {
    return guarded(c, [&] {
        require(n >= 0 && n < 0x3fffffffll, "n out of range");
        require(capacity >= 0 && capacity < 0x7fffffffll, "capacity out of range");
        require(n == 0 || (za && ze && zi && n_edges && pre && post && typ && va && ve && vi),
                "null pointer");
        msp::update_synapses(*c, n, step, za, ze, zi, n_edges, pre, post, typ, capacity, va, ve,
                             vi, as_stream(stream));
    });
}

msp_status msp_append_synapses(msp_ctx* c, const int64_t* n_syn, int64_t syn_capacity,
                               const int32_t* sp, const int32_t* sq, const uint8_t* st,
                               int64_t* n_edges,
                               int32_t* pre, int32_t* post, uint8_t* typ, int64_t capacity,
                               void* stream) {
    return guarded(c, [&] {
        require(capacity >= 0 && capacity < 0x7fffffffll, "capacity out of range");
        require(syn_capacity >= 0, "synapse capacity out of range");
        require(n_syn && sp && sq && st && n_edges && pre && post && typ, "null pointer");
        msp::append_synapses(*c, n_syn, syn_capacity, sp, sq, st, n_edges, pre, post, typ,
                             capacity,
                             as_stream(stream));
    });
}

msp_status msp_step_graph_capture(msp_ctx* c, int64_t n, const float* x, const float* y,
                                  const float* z, const uint8_t* type, uint8_t* va, uint8_t* vde,
                                  uint8_t* vdi, int32_t* partner, int32_t* pre, int32_t* post,
                                  uint8_t* styp, int64_t syn_capacity, int64_t* n_syn,
                                  int64_t* history, int64_t history_len, uint64_t first_step,
                                  void* stream) {
    return guarded(c, [&] {
        require(n > 0 && n < 0x7ffffffell / msp::kMaxVacancy, "n out of range");
        require(x && y && z && type && va && vde && vdi && partner && pre && post && styp && n_syn,
                "null pointer");
        require(syn_capacity >= (int64_t)msp::kMaxVacancy * n, "synapse capacity below 5*n");
        require(history_len >= 0 && (history_len == 0 || history), "bad history buffer");
        msp_ctx::GraphArgs g;
        g.x = x; g.y = y; g.z = z; g.type = type;
        g.va = va; g.vde = vde; g.vdi = vdi;
        g.n = n;
        g.partner = partner; g.pre = pre; g.post = post; g.styp = styp;
        g.capacity = syn_capacity;
        g.n_syn = n_syn;
        g.history = history_len ? history : nullptr;
        g.history_len = history_len;
        g.first_step = first_step;
        msp::graph_capture(*c, g, as_stream(stream));
    });
}

msp_status msp_step_graph_set_full_build(msp_ctx* c, int full_build) {
    return guarded(c, [&] {
        require(full_build == 0 || full_build == 1, "full_build must be 0 or 1");
        c->sg_full_build = full_build != 0;
    });
}

msp_status msp_step_graph_launch(msp_ctx* c, int64_t n_steps, void* stream) {
    return guarded(c, [&] {
        require(n_steps >= 0, "n_steps out of range");
        msp::graph_launch(*c, n_steps, as_stream(stream));
    });
}

msp_status msp_step_graph_finish(msp_ctx* c, void* stream, uint64_t* next_step, int64_t* halted) {
    return guarded(c, [&] {
        require(next_step && halted, "null output");
        msp::graph_finish(*c, as_stream(stream), next_step, halted);
    });
}

msp_status msp_attraction_grad(msp_ctx* c, const uint8_t* type, const uint8_t* va,
                               const uint8_t* vde, const uint8_t* vdi, const float* g, float* u,
                               float* du_dsigma, float* grad_we, float* grad_wi, void* stream) {
    return guarded(c, [&] {
        require(c->n == 0 || (type && va && vde && vdi), "null input pointer");
        msp::attraction_grad(*c, type, va, vde, vdi, g, u, du_dsigma, grad_we, grad_wi,
                             as_stream(stream));
    });
}

msp_status msp_length_loss(msp_ctx* c, const uint8_t* type, const uint8_t* va, const float* we,
                           const float* wi, double target, double* out4, float* gE, float* gI,
                           void* stream) {
    return guarded(c, [&] {
        require(out4 != nullptr, "null result pointer");
        require(c->n == 0 || (type && va && we && wi), "null input pointer");
        require(std::isfinite(target), "target must be finite");
        msp::length_loss(*c, type, va, we, wi, target, out4, gE, gI, as_stream(stream));
    });
}

msp_status msp_set_sigma(msp_ctx* c, double sigma) {
    return guarded(c, [&] {
        require(sigma > 0.0 && std::isfinite(sigma), "sigma must be positive and finite");
        c->cfg.sigma = sigma;
        derive(*c);
        // the pair lists and every captured graph hold the old width
        c->attraction_done = false;
        c->lists_valid = false;
        msp::graph_release(*c);
    });
}

msp_status msp_set_frames(msp_ctx* c, int64_t n_networks, const int64_t* offsets, int level,
                          const int32_t* leaf_capacity, const double* cutoff) {
    return guarded(c, [&] {
        const msp_config& cfg = c->cfg;
        // work in flight may still read the old tables
        MSP_CUDA(cudaDeviceSynchronize());
        c->frame_plans = false;
        c->frame_cap_host.clear();
        c->frame_cut_host.clear();
        if (n_networks == 0) {
            c->frame_level = 0;
            c->frame_off_host.clear();
        } else {
            require(n_networks > 0 && offsets != nullptr, "networks and offsets required");
            require(level >= 1 && level <= 10 && level < cfg.max_depth,
                    "the frame level must lie in [1, min(10, max_depth - 1)]");
            const int64_t G = (int64_t)1 << (level - 1);
            require(n_networks <= G * G * G, "more networks than cells at that level");
            require(offsets[0] == 0, "offsets[0] must be 0");
            const double cell = (double)cfg.side / std::ldexp(1.0, level);
            for (int64_t k = 0; k < n_networks; ++k) {
                const int cap = leaf_capacity ? leaf_capacity[k] : cfg.leaf_capacity;
                const double cut = cutoff ? cutoff[k] : cfg.cutoff;
                require(cap >= 1, "leaf capacities must be positive");
                require(offsets[k + 1] > offsets[k] + cap,
                        "every network needs more neurons than its leaf capacity");
                require(cut > 0.0 && cut <= 5.0, "cutoffs must lie in (0, 5]");
                // networks one cell apart must be beyond the cutoff
                require(cell > cut * cfg.sigma, "a cell must be wider than the cutoff radius");
            }
            require(offsets[n_networks] < 0x7fffffffll, "too many neurons");
            c->frame_off_host.assign(offsets, offsets + n_networks + 1);
            if (leaf_capacity || cutoff) {
                c->frame_plans = true;
                c->frame_cap_host.resize((size_t)n_networks);
                c->frame_cut_host.resize((size_t)n_networks);
                for (int64_t k = 0; k < n_networks; ++k) {
                    c->frame_cap_host[k] = leaf_capacity ? leaf_capacity[k] : cfg.leaf_capacity;
                    c->frame_cut_host[k] = cutoff ? cutoff[k] : cfg.cutoff;
                }
                MSP_CUDA(cudaMemcpy(c->frame_cap.ensure<int32_t>((size_t)n_networks),
                                    c->frame_cap_host.data(), (size_t)n_networks * sizeof(int32_t),
                                    cudaMemcpyHostToDevice));
            }
            int64_t* d = c->frame_off.ensure<int64_t>((size_t)n_networks + 1);
            MSP_CUDA(cudaMemcpy(d, offsets, (size_t)(n_networks + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice));
            c->frame_level = level;
        }
        derive(*c);
        // the octree, the pair lists and every captured graph hold the old frames
        c->tree_built = false;
        c->attraction_done = false;
        c->lists_valid = false;
        msp::graph_release(*c);
    });
}

msp_status msp_set_workspace_limit(int64_t bytes) {
    if (bytes < 0) return fail(MSP_ERR_INVALID_ARG, "limit must not be negative");
    msp::g_ws_limit.store(bytes);
    g_last_error.clear();
    return MSP_OK;
}

int64_t msp_workspace_bytes(void) { return msp::g_ws_bytes.load(); }

msp_status msp_set_pair_capacity(msp_ctx* c, int64_t pairs) {
    return guarded(c, [&] {
        require(pairs >= 1 && pairs <= 0x7fffffffll, "capacity out of range");
        c->pair_cap = pairs;
    });
}

msp_status msp_get_stats(msp_ctx* c, msp_stats* out) {
    return guarded(c, [&] {
        require(out != nullptr, "null output");
        MSP_CUDA(cudaDeviceSynchronize());
        std::memset(out, 0, sizeof(*out));
        out->n = c->n;
        out->n_nodes = c->n_nodes;
        out->tree_depth = c->tree_depth;
        out->far_level = c->l_far;
        out->n_pairs = c->n_pairs;
        out->pair_depths = (int32_t)(c->depth_start.empty() ? 0 : c->depth_start.size() - 1);
        out->n_far = c->n_far;
        out->n_p2p = c->n_p2p;
        out->p2p_interactions = c->p2p_interactions;
        out->n_elements = c->n_elem;
        out->n_draws = c->n_draws;
        out->n_requests = c->n_requests;
        out->n_synapses = c->n_synapses;
        out->expansion_nodes = c->exp_nodes;
        out->kernel_launches = msp::g_kernel_launches.load();
        out->near_field_ms = 0.0;
        if (c->last_was_graph) {
            out->near_field_ms = c->g_nf_ms_mean;
        } else if (c->nf_timed) {
            float ms = 0.f;
            MSP_CUDA(cudaEventElapsedTime(&ms, c->ev_nf0, c->ev_nf1));
            out->near_field_ms = ms;
        }
        if (c->n_nodes > 0) {
            std::vector<int32_t> cf((size_t)c->n_nodes);
            MSP_CUDA(cudaMemcpy(cf.data(), c->nd_child_first.p, cf.size() * 4,
                                cudaMemcpyDeviceToHost));
            int64_t leaves = 0;
            for (int32_t v : cf) leaves += v < 0;
            out->n_leaves = leaves;
        }
    });
}

msp_status msp_export_tree(msp_ctx* c, uint64_t* keys, int32_t* perm, uint8_t* level,
                           uint64_t* prefix, int32_t* first, int32_t* count, int32_t* parent,
                           int32_t* child_first, uint8_t* nchild, int32_t* sums4, float* cent6) {
    return guarded(c, [&] {
        if (!c->tree_built) throw msp::Error(MSP_ERR_NOT_BUILT, "no tree");
        MSP_CUDA(cudaDeviceSynchronize());
        const size_t n = (size_t)c->n, m = (size_t)c->n_nodes;
        auto cp = [](void* dst, const void* src, size_t bytes) {
            if (dst && bytes) MSP_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        };
        cp(keys, c->keys0.p, n * 8);
        cp(perm, c->perm.p, n * 4);
        cp(level, c->nd_level.p, m);
        cp(prefix, c->nd_prefix.p, m * 8);
        cp(first, c->nd_first.p, m * 4);
        cp(count, c->nd_count.p, m * 4);
        cp(parent, c->nd_parent.p, m * 4);
        cp(child_first, c->nd_child_first.p, m * 4);
        cp(nchild, c->nd_nchild.p, m);
        cp(sums4, c->nd_sums.p, m * 16);
        if (cent6 && m) {
            std::vector<float> a(4 * m), d(4 * m);
            cp(a.data(), c->nd_ca.p, m * 16);
            cp(d.data(), c->nd_cd.p, m * 16);
            for (size_t i = 0; i < m; ++i)
                for (int k = 0; k < 3; ++k) {
                    cent6[6 * i + k] = a[4 * i + k];
                    cent6[6 * i + 3 + k] = d[4 * i + k];
                }
        }
    });
}

msp_status msp_export_pairs(msp_ctx* c, int32_t* X, int32_t* Y, uint8_t* kind,
                            int32_t* child_first, double* w_e, double* w_i,
                            int64_t* depth_start) {
    return guarded(c, [&] {
        if (!c->attraction_done) throw msp::Error(MSP_ERR_NOT_BUILT, "no attraction");
        MSP_CUDA(cudaDeviceSynchronize());
        const size_t m = (size_t)c->n_pairs;
        auto cp = [](void* dst, const void* src, size_t bytes) {
            if (dst && bytes) MSP_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        };
        cp(X, c->pr_X.p, m * 4);
        cp(Y, c->pr_Y.p, m * 4);
        cp(kind, c->pr_kind.p, m);
        cp(child_first, c->pr_cf.p, m * 4);
        if ((w_e || w_i) && m) {
            // the table's double-FP32 values (hi, lo per channel), summed in double
            std::vector<float> w(4 * m);
            cp(w.data(), c->pr_w.p, m * 16);
            for (size_t i = 0; i < m; ++i) {
                if (w_e) w_e[i] = (double)w[4 * i] + (double)w[4 * i + 1];
                if (w_i) w_i[i] = (double)w[4 * i + 2] + (double)w[4 * i + 3];
            }
        }
        if (depth_start)
            for (size_t d = 0; d < c->depth_start.size(); ++d) depth_start[d] = c->depth_start[d];
    });
}

msp_status msp_export_expansions(msp_ctx* c, float* A, float* M, float* B, int64_t* first_node) {
    return guarded(c, [&] {
        if (!c->attraction_done) throw msp::Error(MSP_ERR_NOT_BUILT, "no attraction");
        MSP_CUDA(cudaDeviceSynchronize());
        size_t m = (size_t)c->exp_nodes * 2 * c->cfg.p * c->cfg.p * c->cfg.p * sizeof(float);
        if (A && m) MSP_CUDA(cudaMemcpy(A, c->expA.p, m, cudaMemcpyDeviceToHost));
        if (M && m) MSP_CUDA(cudaMemcpy(M, c->expM.p, m, cudaMemcpyDeviceToHost));
        if (B && m) MSP_CUDA(cudaMemcpy(B, c->expB.p, m, cudaMemcpyDeviceToHost));
        if (first_node) *first_node = c->exp_first;
    });
}

}  // extern "C"
