// msp_neuron.cu -- the neuron side of the Model of Structural Plasticity
// (Section 3.1, Table 1), which produces the vacant elements the synapse
// search consumes: electrical activity with Poisson spiking, calcium,
// synaptic-element growth on the Gaussian growth curve, and the deletion of
// synapses a neuron no longer has elements for.
//
// Readings (the paper states the model in words):
//   activity   x <- x + (x0 - x)/tau_x + I + c_in * (edges s -> t whose s
//              spiked in the previous step); the neuron spikes when a uniform
//              draw U in [0,1) (24 bits of Philox) is below x, unless it
//              spiked in one of the last `refractory` steps;
//   calcium    Ca <- Ca - decay * Ca, plus beta on a spike;
//   elements   z <- max(z + g(Ca), 0), g(Ca) = mu (2 exp(-((Ca-xi)/zeta)^2) - 1),
//              xi = (eta + eps)/2, zeta = (eps - eta)/(2 sqrt(ln 2)): zero at
//              eta and eps, mu halfway (the growth curve of the cited model);
//   deletion   a side with more bound synapses than floor(z) deletes the
//              excess, uniformly at random (the excess edges with the
//              smallest Philox priorities, ties by edge position); an edge
//              chosen by either side goes; vacant = floor(z) - bound.
// The state decides integers (a spike, a floor), so every floating-point
// operation is single precision with explicit rounding intrinsics in the
// order written (no contraction into FMAs), and exp is computed here from its
// definition; the result is then reproducible bit for bit.
#include <algorithm>

#include "msp_internal.cuh"

namespace msp {

namespace {

constexpr uint32_t kTagSpike = 5u, kTagDelAxon = 6u, kTagDelDend = 7u;

__device__ __forceinline__ uint32_t nr_draw(uint64_t seed, uint32_t c0, uint32_t c1,
                                            uint64_t step) {
    uint32_t o[4];
    philox_draw(seed, c0, c1, step, o);
    return o[0];
}

// exp(x), single precision: Cody and Waite's reduction x = n ln 2 + r with
// ln 2 = 0.693359375 - 2.12194440e-4 (n times the first part is exact), the
// degree-7 Taylor polynomial of e^r (|r| <= 0.35) and the scale 2^n; 0 below
// -87.  Rounded operation by operation.
__device__ float nr_expf(float x) {
    if (x < -87.0f) return 0.0f;
    const float n = floorf(__fadd_rn(__fmul_rn(x, 1.44269504f), 0.5f));
    float r = __fadd_rn(x, -__fmul_rn(n, 0.693359375f));
    r = __fadd_rn(r, __fmul_rn(n, 2.12194440e-4f));
    float p = 1.98412698e-4f;
    p = __fadd_rn(__fmul_rn(p, r), 1.38888889e-3f);
    p = __fadd_rn(__fmul_rn(p, r), 8.33333333e-3f);
    p = __fadd_rn(__fmul_rn(p, r), 4.16666667e-2f);
    p = __fadd_rn(__fmul_rn(p, r), 1.66666667e-1f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    const float s = __uint_as_float((uint32_t)((int)n + 127) << 23);
    return __fmul_rn(p, s);
}

__device__ float nr_growth(float ca, float eta, float eps, float mu) {
    const float xi = __fmul_rn(__fadd_rn(eta, eps), 0.5f);
    const float zeta = __fdiv_rn(__fadd_rn(eps, -eta), __fmul_rn(2.0f, 0.832554611f));
    const float q = __fdiv_rn(__fadd_rn(ca, -xi), zeta);
    const float e = nr_expf(-__fmul_rn(q, q));
    return __fmul_rn(mu, __fadd_rn(__fadd_rn(e, e), -1.0f));
}

// The input of a step is event driven: the outgoing edges of each neuron, as
// a compressed list by presynaptic neuron rebuilt at the start of every
// call, and two input-count buffers; a neuron that spikes in step k adds one
// to the next buffer for each of its outgoing edges, which step k + 1 reads
// (and clears).  Edges naming a neuron outside [0, n) are skipped.
__global__ void k_out_degree(const int64_t* __restrict__ n_edges, int64_t cap, int64_t n,
                             const int32_t* __restrict__ pre, const int32_t* __restrict__ post,
                             int32_t* __restrict__ deg) {
    const int64_t m = min(*n_edges, cap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = pre[e], b = post[e];
        if (a < 0 || a >= n || b < 0 || b >= n) continue;
        atomicAdd(&deg[a], 1);
    }
}

// targets of each neuron's outgoing edges at [off[s], off[s] + deg[s]) (the
// order inside a neuron's range does not matter: only counts are formed)
__global__ void k_out_fill(const int64_t* __restrict__ n_edges, int64_t cap, int64_t n,
                           const int32_t* __restrict__ pre, const int32_t* __restrict__ post,
                           const int32_t* __restrict__ off, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ targets) {
    const int64_t m = min(*n_edges, cap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = pre[e], b = post[e];
        if (a < 0 || a >= n || b < 0 || b >= n) continue;
        targets[off[a] + atomicAdd(&cursor[a], 1)] = b;
    }
}

// the input of the first step of a call: last step's spikes
__global__ void k_seed_input(int64_t n, const uint8_t* __restrict__ spiked,
                             const int32_t* __restrict__ off, const int32_t* __restrict__ deg,
                             const int32_t* __restrict__ targets, int32_t* __restrict__ inp) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        if (spiked[t])
            for (int32_t j = off[t], j1 = off[t] + deg[t]; j < j1; ++j) atomicAdd(&inp[targets[j]], 1);
}

// edges naming a neuron outside [0, n), or a count above the capacity
__global__ void k_check_edges(const int64_t* __restrict__ n_edges, int64_t cap, int64_t n,
                              const int32_t* __restrict__ pre, const int32_t* __restrict__ post,
                              unsigned long long* __restrict__ bad) {
    const int64_t m0 = *n_edges;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (m0 < 0 || m0 > cap)) atomicAdd(bad, 1ull);
    const int64_t m = min(max(m0, (int64_t)0), cap);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = pre[e], b = post[e];
        if (a < 0 || a >= n || b < 0 || b >= n) atomicAdd(bad, 1ull);
    }
}

// The state of one neuron through one step (Section 3.1): activity with
// input `in`, the spike draw, calcium, the three element counts.  Returns the
// spike.
struct NrState {
    float x, ca, za, ze, zi;
    uint32_t rf;
};

__device__ __forceinline__ int nr_update(NrState& v, int32_t in, uint32_t t, uint64_t seed,
                                         uint64_t step, const msp_neuron_params& mp) {
    float d = __fadd_rn(mp.x0, -v.x);
    d = __fdiv_rn(d, mp.tau_x);
    float xt = __fadd_rn(v.x, d);
    xt = __fadd_rn(xt, mp.background);
    xt = __fadd_rn(xt, __fmul_rn(mp.input_per_spike, (float)in));
    v.x = xt;
    int s = 0;
    if (v.rf > 0) {
        v.rf -= 1;
    } else {
        const uint32_t o = nr_draw(seed, t, kTagSpike << 16, step);
        const float u = __fmul_rn((float)(o >> 8), 1.0f / 16777216.0f);
        s = u < xt;
        if (s) v.rf = (uint32_t)mp.refractory;
    }
    float ca = __fadd_rn(v.ca, -__fmul_rn(v.ca, mp.decay_ca));
    if (s) ca = __fadd_rn(ca, mp.beta_ca);
    v.ca = ca;
    const float a = __fadd_rn(v.za, nr_growth(ca, mp.eta_axon, mp.eps, mp.mu));
    const float gd = nr_growth(ca, mp.eta_dend, mp.eps, mp.mu);
    const float e = __fadd_rn(v.ze, gd);
    const float i = __fadd_rn(v.zi, gd);
    v.za = a > 0.0f ? a : 0.0f;
    v.ze = e > 0.0f ? e : 0.0f;
    v.zi = i > 0.0f ? i : 0.0f;
    return s;
}

// One step of every neuron: consumes (and clears) its input count in `cur`;
// a spike adds one to `next` for each outgoing edge.  With vec4 set (every
// array 16-byte aligned, the byte arrays 4-byte aligned) a thread takes four
// consecutive neurons with 16-byte loads and stores, so that more of the
// state is in flight per thread; the last n mod 4 neurons (or all, without
// vec4) go one per thread.  The step is bound by the latency of its loads:
// at most 48 registers (no spills) keep five blocks resident per SM.
__global__ void __launch_bounds__(256, 5)
k_neuron_step(int64_t n, int vec4, uint64_t seed, uint64_t step,
                              msp_neuron_params mp, int32_t* __restrict__ cur,
                              int32_t* __restrict__ next, const int32_t* __restrict__ off,
                              const int32_t* __restrict__ deg, const int32_t* __restrict__ targets,
                              float* __restrict__ x, uint8_t* __restrict__ refr,
                              float* __restrict__ calcium, float* __restrict__ za,
                              float* __restrict__ ze, float* __restrict__ zi,
                              uint8_t* __restrict__ spiked) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = vec4 ? n / 4 : 0;
    for (int64_t q = tid; q < n4; q += stride) {
        const int4 in4 = reinterpret_cast<const int4*>(cur)[q];
        const float4 x4 = reinterpret_cast<const float4*>(x)[q];
        const float4 c4 = reinterpret_cast<const float4*>(calcium)[q];
        const float4 a4 = reinterpret_cast<const float4*>(za)[q];
        const float4 e4 = reinterpret_cast<const float4*>(ze)[q];
        const float4 i4 = reinterpret_cast<const float4*>(zi)[q];
        const uint32_t r4 = reinterpret_cast<const uint32_t*>(refr)[q];
        reinterpret_cast<int4*>(cur)[q] = make_int4(0, 0, 0, 0);
        const int32_t ins[4] = {in4.x, in4.y, in4.z, in4.w};
        NrState v[4] = {{x4.x, c4.x, a4.x, e4.x, i4.x, r4 & 0xffu},
                        {x4.y, c4.y, a4.y, e4.y, i4.y, (r4 >> 8) & 0xffu},
                        {x4.z, c4.z, a4.z, e4.z, i4.z, (r4 >> 16) & 0xffu},
                        {x4.w, c4.w, a4.w, e4.w, i4.w, r4 >> 24}};
        uint32_t sp = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = nr_update(v[k], ins[k], (uint32_t)(4 * q + k), seed, step, mp);
            sp |= (uint32_t)s << (8 * k);
            if (s) {
                // the outgoing edges are read only for the neurons that spiked
                const int32_t j0 = off[4 * q + k], j1 = j0 + deg[4 * q + k];
                for (int32_t j = j0; j < j1; ++j) atomicAdd(&next[targets[j]], 1);
            }
        }
        reinterpret_cast<float4*>(x)[q] = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
        reinterpret_cast<float4*>(calcium)[q] = make_float4(v[0].ca, v[1].ca, v[2].ca, v[3].ca);
        reinterpret_cast<float4*>(za)[q] = make_float4(v[0].za, v[1].za, v[2].za, v[3].za);
        reinterpret_cast<float4*>(ze)[q] = make_float4(v[0].ze, v[1].ze, v[2].ze, v[3].ze);
        reinterpret_cast<float4*>(zi)[q] = make_float4(v[0].zi, v[1].zi, v[2].zi, v[3].zi);
        reinterpret_cast<uint32_t*>(refr)[q] = v[0].rf | (v[1].rf << 8) | (v[2].rf << 16) |
                                               (v[3].rf << 24);
        reinterpret_cast<uint32_t*>(spiked)[q] = sp;
    }
    for (int64_t t = 4 * n4 + tid; t < n; t += stride) {
        const int32_t in = cur[t];
        cur[t] = 0;
        NrState v = {x[t], calcium[t], za[t], ze[t], zi[t], refr[t]};
        const int s = nr_update(v, in, (uint32_t)t, seed, step, mp);
        x[t] = v.x;
        calcium[t] = v.ca;
        za[t] = v.za;
        ze[t] = v.ze;
        zi[t] = v.zi;
        refr[t] = (uint8_t)v.rf;
        spiked[t] = (uint8_t)s;
        if (s)
            for (int32_t j = off[t], j1 = off[t] + deg[t]; j < j1; ++j)
                atomicAdd(&next[targets[j]], 1);
    }
}

// bound synapses per neuron: outgoing, incoming per type (post*2 + type)
__global__ void k_bound(const int64_t* __restrict__ n_edges, const int32_t* __restrict__ pre,
                        const int32_t* __restrict__ post, const uint8_t* __restrict__ typ,
                        int32_t* __restrict__ bout, int32_t* __restrict__ bin) {
    const int64_t m = *n_edges;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&bout[pre[e]], 1);
        atomicAdd(&bin[2 * (int64_t)post[e] + (typ[e] ? 1 : 0)], 1);
    }
}

__device__ __forceinline__ int32_t floor_count(float z) { return (int32_t)floorf(z); }

// excess per side: bound - floor(z) when positive
__global__ void k_excess(int64_t n, const float* __restrict__ za, const float* __restrict__ ze,
                         const float* __restrict__ zi, const int32_t* __restrict__ bout,
                         const int32_t* __restrict__ bin, int32_t* __restrict__ xout,
                         int32_t* __restrict__ xin) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        xout[t] = max(bout[t] - floor_count(za[t]), 0);
        xin[2 * t] = max(bin[2 * t] - floor_count(ze[t]), 0);
        xin[2 * t + 1] = max(bin[2 * t + 1] - floor_count(zi[t]), 0);
    }
}

// sort keys (group << 32 | priority), values = edge position
__global__ void k_del_keys(const int64_t* __restrict__ n_edges, const int32_t* __restrict__ pre,
                           const int32_t* __restrict__ post, const uint8_t* __restrict__ typ,
                           int dendrite_side, uint64_t seed, uint64_t step,
                           uint64_t* __restrict__ key, int32_t* __restrict__ val) {
    const int64_t m = *n_edges;
    const uint32_t tag = (dendrite_side ? kTagDelDend : kTagDelAxon) << 16;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t g = dendrite_side ? 2 * (uint64_t)post[e] + (typ[e] ? 1 : 0)
                                         : (uint64_t)pre[e];
        key[e] = (g << 32) | nr_draw(seed, (uint32_t)e, tag, step);
        val[e] = (int32_t)e;
    }
}

// in sorted order, the first excess[group] edges of each group are deleted
__global__ void k_del_mark(const int64_t* __restrict__ n_edges, const uint64_t* __restrict__ key,
                           const int32_t* __restrict__ val, const int32_t* __restrict__ start,
                           const int32_t* __restrict__ excess, uint8_t* __restrict__ del) {
    const int64_t m = *n_edges;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = (int64_t)(key[i] >> 32);
        if (i - start[g] < excess[g]) del[val[i]] = 1;
    }
}

__global__ void k_keep_flags(const int64_t* __restrict__ n_edges, const uint8_t* __restrict__ del,
                             int32_t* __restrict__ keep) {
    const int64_t m = *n_edges;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        keep[e] = del[e] ? 0 : 1;
}

__global__ void k_compact(const int64_t* __restrict__ n_edges, const int32_t* __restrict__ keep,
                          const int32_t* __restrict__ pos, const int32_t* __restrict__ pre,
                          const int32_t* __restrict__ post, const uint8_t* __restrict__ typ,
                          int32_t* __restrict__ pre2, int32_t* __restrict__ post2,
                          uint8_t* __restrict__ typ2) {
    const int64_t m = *n_edges;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        if (keep[e]) {
            const int32_t q = pos[e];
            pre2[q] = pre[e];
            post2[q] = post[e];
            typ2[q] = typ[e];
        }
}

__global__ void k_copy_edges(const int64_t* __restrict__ n_edges, const int32_t* __restrict__ pre2,
                             const int32_t* __restrict__ post2, const uint8_t* __restrict__ typ2,
                             int32_t* __restrict__ pre, int32_t* __restrict__ post,
                             uint8_t* __restrict__ typ) {
    const int64_t m = *n_edges;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        pre[e] = pre2[e];
        post[e] = post2[e];
        typ[e] = typ2[e];
    }
}

__global__ void k_vacancies(int64_t n, const float* __restrict__ za, const float* __restrict__ ze,
                            const float* __restrict__ zi, const int32_t* __restrict__ bout,
                            const int32_t* __restrict__ bin, uint8_t* __restrict__ va,
                            uint8_t* __restrict__ ve, uint8_t* __restrict__ vi) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        va[t] = (uint8_t)min(max(floor_count(za[t]) - bout[t], 0), 255);
        ve[t] = (uint8_t)min(max(floor_count(ze[t]) - bin[2 * t], 0), 255);
        vi[t] = (uint8_t)min(max(floor_count(zi[t]) - bin[2 * t + 1], 0), 255);
    }
}

// append formed synapses at the end of the edge list (up to the capacity)
__global__ void k_append(const int64_t* __restrict__ n_syn, int64_t syn_cap,
                         const int32_t* __restrict__ sp, const int32_t* __restrict__ sq,
                         const uint8_t* __restrict__ st, const int64_t* __restrict__ n_edges,
                         int64_t cap, int32_t* __restrict__ pre, int32_t* __restrict__ post,
                         uint8_t* __restrict__ typ) {
    const int64_t m0 = *n_edges, k = min(*n_syn, syn_cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = m0 + i;
        if (e >= cap) break;
        pre[e] = sp[i];
        post[e] = sq[i];
        typ[e] = st[i];
    }
}

__global__ void k_append_count(const int64_t* __restrict__ n_syn, int64_t syn_cap, int64_t cap,
                               int64_t* __restrict__ n_edges, int64_t* __restrict__ overflow) {
    const int64_t m = *n_edges + min(*n_syn, syn_cap);
    if (m > cap) {
        *overflow |= 32;
        *n_edges = cap;
    } else {
        *n_edges = m;
    }
}

int bits_for_neuron(int64_t v) {
    int b = 1;
    while (b < 62 && ((int64_t)1 << b) <= v) ++b;
    return b;
}

}  // namespace

void neuron_steps(msp_ctx& c, int64_t n, uint64_t first_step, int n_steps,
                  const msp_neuron_params& mp, const int64_t* n_edges, int64_t cap,
                  const int32_t* pre, const int32_t* post, float* x, uint8_t* refr,
                  float* calcium, float* za, float* ze, float* zi, uint8_t* spiked,
                  cudaStream_t s) {
    NvtxRange nv_("msp neuron_steps");
    if (n <= 0 || n_steps <= 0) return;
    // two input-count buffers, the second at a 16-byte boundary
    const int64_t n_pad = (n + 3) & ~(int64_t)3;
    int32_t* inp = c.nr_inp.ensure<int32_t>((size_t)2 * n_pad);
    int32_t* deg = c.nr_bout.ensure<int32_t>((size_t)n);
    int32_t* off = c.nr_sout.ensure<int32_t>((size_t)n);
    int32_t* cursor = c.nr_xout.ensure<int32_t>((size_t)n);
    int32_t* targets = c.nr_pos.ensure<int32_t>((size_t)std::max<int64_t>(cap, 1));
    int64_t* cnt = c.nr_cnt.ensure<int64_t>(4);
    const int ge = (int)c.sm_count * 8;
    const int gn = grid_for(n, 256, (int64_t)c.sm_count * 16);
    // outgoing edges by presynaptic neuron
    MSP_CUDA(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int32_t), s));
    MSP_CUDA(cudaMemsetAsync(cursor, 0, (size_t)n * sizeof(int32_t), s));
    MSP_CUDA(cudaMemsetAsync(inp, 0, (size_t)2 * n_pad * sizeof(int32_t), s));
    k_out_degree<<<ge, 256, 0, s>>>(n_edges, cap, n, pre, post, deg);
    MSP_LAUNCH("out_degree");
    dev_set(cnt, n, s);
    scan_dev(c, deg, off, cnt, n, cnt + 2, nullptr, s);
    k_out_fill<<<ge, 256, 0, s>>>(n_edges, cap, n, pre, post, off, cursor, targets);
    MSP_LAUNCH("out_fill");
    k_seed_input<<<gn, 256, 0, s>>>(n, spiked, off, deg, targets, inp);
    MSP_LAUNCH("seed_input");
    // four neurons per thread where every array allows 16-byte (bytes: 4-byte) access
    auto al = [](const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; };
    const int32_t* inp1 = inp + n_pad;
    const int vec4 = al(inp, 16) && al(inp1, 16) && al(off, 16) && al(deg, 16) && al(x, 16) &&
                     al(calcium, 16) && al(za, 16) && al(ze, 16) && al(zi, 16) && al(refr, 4) &&
                     al(spiked, 4);
    const int gv = grid_for(vec4 ? (n + 3) / 4 : n, 256, (int64_t)c.sm_count * 16);
    for (int k = 0; k < n_steps; ++k) {
        int32_t* cur = inp + (size_t)(k & 1) * n_pad;
        int32_t* next = inp + (size_t)((k + 1) & 1) * n_pad;
        k_neuron_step<<<gv, 256, 0, s>>>(n, vec4, c.cfg.seed, first_step + (uint64_t)k, mp, cur,
                                          next, off, deg, targets, x, refr, calcium, za, ze, zi,
                                          spiked);
        MSP_LAUNCH("neuron_step");
    }
}

void update_synapses(msp_ctx& c, int64_t n, uint64_t step, const float* za, const float* ze,
                     const float* zi, int64_t* n_edges, int32_t* pre, int32_t* post, uint8_t* typ,
                     int64_t cap, uint8_t* va, uint8_t* ve, uint8_t* vi, cudaStream_t s) {
    NvtxRange nv_("msp update_synapses");
    if (n <= 0) return;
    const size_t ecap = (size_t)std::max<int64_t>(cap, 1);
    int32_t* bout = c.nr_bout.ensure<int32_t>((size_t)n);
    int32_t* bin = c.nr_bin.ensure<int32_t>((size_t)2 * n);
    int32_t* xout = c.nr_xout.ensure<int32_t>((size_t)n);
    int32_t* xin = c.nr_xin.ensure<int32_t>((size_t)2 * n);
    int32_t* sout = c.nr_sout.ensure<int32_t>((size_t)n);
    int32_t* sin = c.nr_sin.ensure<int32_t>((size_t)2 * n);
    int64_t* cnt = c.nr_cnt.ensure<int64_t>(4);   // n, 2n, scan totals
    uint64_t* k0 = c.nr_key0.ensure<uint64_t>(ecap);
    uint64_t* k1 = c.nr_key1.ensure<uint64_t>(ecap);
    int32_t* v0 = c.nr_val0.ensure<int32_t>(ecap);
    int32_t* v1 = c.nr_val1.ensure<int32_t>(ecap);
    uint8_t* del = c.nr_del.ensure<uint8_t>(ecap);
    int32_t* keep = c.nr_keep.ensure<int32_t>(ecap);
    int32_t* pos = c.nr_pos.ensure<int32_t>(ecap);
    int32_t* pre2 = c.nr_pre2.ensure<int32_t>(ecap);
    int32_t* post2 = c.nr_post2.ensure<int32_t>(ecap);
    uint8_t* typ2 = c.nr_typ2.ensure<uint8_t>(ecap);
    const int ge = (int)c.sm_count * 8;
    const int gn = grid_for(n, 256, (int64_t)c.sm_count * 16);
    // the edges must name neurons in [0, n) and fit the capacity
    dev_set(cnt + 3, 0, s);
    k_check_edges<<<ge, 256, 0, s>>>(n_edges, cap, n, pre, post,
                                     reinterpret_cast<unsigned long long*>(cnt + 3));
    MSP_LAUNCH("check_edges");
    int64_t bad = 0;
    MSP_CUDA(cudaMemcpyAsync(&bad, cnt + 3, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    if (bad) throw Error(MSP_ERR_INVALID_ARG, "an edge names a neuron outside [0, n), or the "
                                              "edge count exceeds the capacity");
    dev_set(cnt, n, s);
    dev_set(cnt + 1, 2 * n, s);
    MSP_CUDA(cudaMemsetAsync(bout, 0, (size_t)n * sizeof(int32_t), s));
    MSP_CUDA(cudaMemsetAsync(bin, 0, (size_t)2 * n * sizeof(int32_t), s));
    MSP_CUDA(cudaMemsetAsync(del, 0, ecap, s));
    k_bound<<<ge, 256, 0, s>>>(n_edges, pre, post, typ, bout, bin);
    MSP_LAUNCH("bound");
    k_excess<<<gn, 256, 0, s>>>(n, za, ze, zi, bout, bin, xout, xin);
    MSP_LAUNCH("excess");
    // group starts in (group, priority) order
    scan_dev(c, bout, sout, cnt, n, cnt + 2, nullptr, s);
    scan_dev(c, bin, sin, cnt + 1, 2 * n, cnt + 3, nullptr, s);
    const uint64_t seed = c.cfg.seed;
    // the axon side, then the dendrite side
    k_del_keys<<<ge, 256, 0, s>>>(n_edges, pre, post, typ, 0, seed, step, k0, v0);
    MSP_LAUNCH("del_keys");
    radix_sort_dev(c, k0, v0, k1, v1, n_edges, cap, 32 + bits_for_neuron(n), s);
    k_del_mark<<<ge, 256, 0, s>>>(n_edges, k0, v0, sout, xout, del);
    MSP_LAUNCH("del_mark");
    k_del_keys<<<ge, 256, 0, s>>>(n_edges, pre, post, typ, 1, seed, step, k0, v0);
    MSP_LAUNCH("del_keys");
    radix_sort_dev(c, k0, v0, k1, v1, n_edges, cap, 32 + bits_for_neuron(2 * n), s);
    k_del_mark<<<ge, 256, 0, s>>>(n_edges, k0, v0, sin, xin, del);
    MSP_LAUNCH("del_mark");
    // compaction, order kept
    k_keep_flags<<<ge, 256, 0, s>>>(n_edges, del, keep);
    MSP_LAUNCH("keep_flags");
    scan_dev(c, keep, pos, n_edges, cap, cnt + 2, nullptr, s);
    k_compact<<<ge, 256, 0, s>>>(n_edges, keep, pos, pre, post, typ, pre2, post2, typ2);
    MSP_LAUNCH("compact");
    MSP_CUDA(cudaMemcpyAsync(n_edges, cnt + 2, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    k_copy_edges<<<ge, 256, 0, s>>>(n_edges, pre2, post2, typ2, pre, post, typ);
    MSP_LAUNCH("copy_edges");
    // vacancies from the remaining synapses
    MSP_CUDA(cudaMemsetAsync(bout, 0, (size_t)n * sizeof(int32_t), s));
    MSP_CUDA(cudaMemsetAsync(bin, 0, (size_t)2 * n * sizeof(int32_t), s));
    k_bound<<<ge, 256, 0, s>>>(n_edges, pre, post, typ, bout, bin);
    MSP_LAUNCH("bound");
    k_vacancies<<<gn, 256, 0, s>>>(n, za, ze, zi, bout, bin, va, ve, vi);
    MSP_LAUNCH("vacancies");
}

void append_synapses(msp_ctx& c, const int64_t* n_syn, int64_t syn_cap, const int32_t* sp,
                     const int32_t* sq, const uint8_t* st, int64_t* n_edges, int32_t* pre,
                     int32_t* post, uint8_t* typ, int64_t cap, cudaStream_t s) {
    NvtxRange nv_("msp append_synapses");
    DevCounts* dc = dcounts(c);
    k_append<<<(int)c.sm_count * 8, 256, 0, s>>>(n_syn, syn_cap, sp, sq, st, n_edges, cap, pre,
                                                  post, typ);
    MSP_LAUNCH("append");
    k_append_count<<<1, 1, 0, s>>>(n_syn, syn_cap, cap, n_edges, &dc->overflow);
    MSP_LAUNCH("append_count");
    pull_counts(c, s);
    if (c.hcount->overflow & 32) {
        dev_set(&dc->overflow, c.hcount->overflow & ~32ll, s);
        throw Error(MSP_ERR_CAPACITY, "edge list capacity exceeded: the excess synapses were dropped");
    }
}

}  // namespace msp
