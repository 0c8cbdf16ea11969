// msp_internal.cuh -- context, device buffers and device helpers shared by the
// translation units of libmsp.  Not part of the public ABI (include/msp.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <atomic>
#include <stdexcept>
#include <string>
#include <vector>

#include "msp.h"

namespace msp {

constexpr int kMortonBits = 21;
constexpr int kMaxP = 8;
constexpr uint32_t kTagDescend = 1u, kTagLeaf = 2u, kTagAccept = 3u, kTagWalk = 4u;
enum PairKind : uint8_t { kSplit = 0, kFar = 1, kP2P = 2, kPruned = 3 };
// A draw whose total attraction is at or below this has no candidate; every
// attraction inside the cutoff radius is many orders of magnitude larger.
constexpr double kMinAttraction = 1e-30;
constexpr float kMinAttractionF = 1e-30f;

// ---------------------------------------------------------------------------
// errors: internal code throws; every C entry point converts to msp_status
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
    msp_status code;
    Error(msp_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

inline void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    msp_status c = (e == cudaErrorMemoryAllocation) ? MSP_ERR_OOM : MSP_ERR_CUDA;
    throw Error(c, std::string(what) + ": " + cudaGetErrorString(e));
}
// message of the calling thread's last error (msp_last_error)
void set_last_error(const char* msg);
// kernels launched by the library (process-wide), counted at each launch check
extern std::atomic<long long> g_kernel_launches;
#define MSP_CUDA(x) ::msp::cuda_check((x), #x)
#define MSP_LAUNCH(what) \
    (::msp::g_kernel_launches.fetch_add(1, std::memory_order_relaxed), \
     ::msp::cuda_check(cudaGetLastError(), what))

// Bumped whenever a workspace buffer is (re)allocated or freed: a captured
// step graph records it and refuses to replay once it changed (its kernels
// hold the old addresses).
extern std::atomic<long long> g_alloc_epoch;
// Device memory held by all workspace buffers, and an optional cap on it
// (0: none); an allocation beyond the cap fails with MSP_ERR_OOM.
extern std::atomic<long long> g_ws_bytes;
extern std::atomic<long long> g_ws_limit;

// a named range for profilers and tracers (NVTX; free when no tool listens)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// grow-only device buffer
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* get() const { return static_cast<T*>(p); }
    template <class T>
    T* ensure(size_t count) {
        size_t need = count * sizeof(T);
        if (need == 0) need = sizeof(T);
        if (need > bytes) {
            g_alloc_epoch.fetch_add(1, std::memory_order_relaxed);
            release();
            size_t alloc = need + need / 4 + 256;
            const long long lim = g_ws_limit.load();
            if (lim > 0 && g_ws_bytes.load() + (long long)alloc > lim)
                throw Error(MSP_ERR_OOM, "workspace limit reached");
            cuda_check(cudaMalloc(&p, alloc), "cudaMalloc");
            bytes = alloc;
            g_ws_bytes.fetch_add((long long)alloc);
        }
        return static_cast<T*>(p);
    }
    void release() {
        if (p) {
            g_alloc_epoch.fetch_add(1, std::memory_order_relaxed);
            g_ws_bytes.fetch_sub((long long)bytes);
            cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
};

// one item of the level-synchronous descent (Algorithm 1)
struct Item {
    int32_t X, Y, q, ch;   // axon box, dendrite box, traversal pair (-1 below a far pair), channel
};

constexpr int kMaxLevels = kMortonBits + 1;   // octree levels 0..21

// Sizes that the kernels produce and consume, kept in device memory so that
// a whole step runs without waiting for the host; copied to pinned host
// memory once at the end of each public call.
struct DevCounts {
    int64_t n;                               // neurons of the last build
    int64_t level_start[kMaxLevels + 2];     // level l boxes: [level_start[l], level_start[l+1])
    int64_t depth_start[kMaxLevels + 3];     // traversal depth d pairs
    int64_t n_elem;                          // vacant axonal elements
    int64_t more_levels;                     // boxes still to split below the last built level
    int64_t n_far, n_p2p, nseg;
    int64_t items[3];                        // descent items, rotating: in / out / reset
    int64_t n_leaf;                          // leaf pairs reached by the descent
    int64_t leaf_next;                       // work counter of the leaf draw
    int64_t draws;
    int64_t n_req, n_syn;
    int64_t interactions;
    int64_t overflow;                        // bit 0 pairs, 1 items, 2 leaf items, 4 tree nodes,
                                             // 5 request groups inconsistent
    int64_t need_pairs;                      // largest pair-table end asked for (before clamping)
    int64_t need_items;                      // largest descent item count asked for
    int64_t need_nodes;                      // largest octree node end asked for
    int64_t bad_pos;                         // positions outside the domain (last build)
    int64_t scan_n;                          // element count of the next scan
    // whole-step graph: the step index its kernels draw with, the halt flag
    // (nonzero: a capacity was exceeded; the state-changing kernels stop) and
    // the steps completed
    uint64_t step;
    int64_t halt;
    int64_t steps_run;
    int64_t interactions_run;                // near-field interactions over the replays
    uint64_t pos_sum;                        // checksum of the positions of the last build
    uint64_t tree_gen;                       // generation stamp of the last eager build
    int64_t m2l_n, m2l_nseg;                 // far pairs translated pair by pair, their targets
    int64_t n_split;                         // split pairs of the last traversal
    int64_t n_groups;                        // request groups (channel, dendrite): 2 n
    int64_t split_start[kMaxLevels + 3];     // depth d split pairs: split_q[split_start[d], [d+1])
};

// DevCounts::overflow bit set when a bounded wait of the single-pass scan
// gave up (its result is then wrong; the host reports MSP_ERR_TIMEOUT)
constexpr int64_t kScanTimeoutBit = 1ll << 40;

// the vacancy walk keeps every vacant count in [0, kMaxVacancy]
constexpr int kMaxVacancy = 5;

// The step index of the Philox counters: a value, or (inside the whole-step
// graph) read from device memory.
struct StepRef {
    uint64_t v;
    const uint64_t* p;
    __device__ uint64_t get() const { return p ? *p : v; }
};

}  // namespace msp

struct msp_ctx {
    msp_config cfg;
    int device = 0;
    int sm_count = 0;
    // derived constants
    float morton_scale = 0.f;
    int l_far = 0;
    long long g2[msp::kMortonBits + 1];
    // sizes
    int64_t n = 0;
    int64_t n_elem = 0;
    int64_t n_nodes = 0, n_leaves = 0;
    int tree_depth = 0;
    std::vector<int64_t> level_start;   // level l nodes: [level_start[l], level_start[l+1])
    std::vector<int64_t> depth_start;   // pair depth d: [depth_start[d], depth_start[d+1])
    int64_t n_pairs = 0, n_far = 0, n_p2p = 0, p2p_interactions = 0;
    int64_t n_draws = 0, n_requests = 0, n_synapses = 0;
    int64_t exp_first = 0, exp_nodes = 0;
    int64_t n_p2p_targets = 0;
    bool tree_built = false, attraction_done = false;
    // eager calls on fixed positions: the last build reused the octree of the
    // one before (same positions), and the interaction lists of the last
    // attraction belong to that octree (distance rule: they depend on the
    // positions and the kernel width only)
    bool tree_reused = false, lists_valid = false;
    // independent networks in local frames (msp_set_frames): network k holds
    // the caller's neurons [frame_off[k], frame_off[k+1]) with positions
    // relative to its own cell of the grid at level frame_level (0: one frame)
    int frame_level = 0;
    std::vector<int64_t> frame_off_host;
    msp::DBuf frame_off;
    // per-network plans (optional): leaf capacity, the pruning thresholds of
    // every level (as g2 below) and the leaf draw's squared truncation radius
    bool frame_plans = false;
    std::vector<int32_t> frame_cap_host;
    std::vector<double> frame_cut_host;
    msp::DBuf frame_cap, frame_g2, frame_rc2;
    // sorted points
    msp::DBuf keys0, keys1, vals0, vals1;
    msp::DBuf perm, inv, pts, wts, lw, elem_off, leaf_of;
    // octree (SoA)
    msp::DBuf nd_level, nd_prefix, nd_first, nd_count, nd_parent, nd_child_first, nd_nchild;
    msp::DBuf nd_sums, nd_ca, nd_cd;
    msp::DBuf nd_arrive;                                 // aggregation arrival counters
    // dual traversal
    msp::DBuf pr_X, pr_Y, pr_kind, pr_cf, pr_nb, pr_w;
    // lists
    msp::DBuf m2_key0, m2_key1, m2_val0, m2_val1, m2_flag, m2_off, m2_seg;   // far pairs by X
    msp::DBuf far_q, p2p_key0, p2p_key1, p2p_val0, p2p_val1, seg_first, seg_flag, nf_w32;
    msp::DBuf split_q;                                   // split pairs, by depth (int4 entries)
    msp::DBuf nf_okey0, nf_okey1, nf_oval0, nf_oval1;   // near-field segment order
    msp::DBuf nf_src;                                    // per near-field pair: (first, count) of Y
    // neuron side (msp_neuron.cu): input counts, bound synapses, excess, group
    // starts, deletion sort keys, flags and the compacted edge copy
    msp::DBuf nr_inp, nr_bout, nr_bin, nr_xout, nr_xin, nr_sout, nr_sin, nr_cnt;
    msp::DBuf nr_key0, nr_key1, nr_val0, nr_val1, nr_del, nr_keep, nr_pos;
    msp::DBuf nr_pre2, nr_post2, nr_typ2;
    // geometric expansion centres and the grouped translations (msp_m2l_gemm.cu)
    int gm_smem_set = 0;   // dynamic shared memory opted in for the grouped translations
    msp::DBuf nd_gc, gm_key0, gm_key1, gm_q, gm_q1, gm_flag, gm_gid, gm_gstart, gm_ntile,
        gm_toff, gm_tiles, gm_cnt;
    // derivatives (msp_grad.cu)
    msp::DBuf gr_w, gr_tmp, gr_key0, gr_key1, gr_val0, gr_val1, gr_flag, gr_off, gr_seg;
    // expected synapse length (msp_length.cu): per-target sums, block
    // partials and results, per-target coefficients of the transposed sums
    msp::DBuf ln_sums, ln_part, ln_coef;
    // expansions
    msp::DBuf expA, expM, expB;
    msp::DBuf u_sorted;
    // descent
    msp::DBuf items0, items1, leaf_items, rq_key0, rq_val0, accepted, acc_off;
    msp::DBuf rq_gcnt, rq_goff;                          // requests per (channel, dendrite)
    // generic scratch
    msp::DBuf cnt, off, scan_tmp, rs_hist, sd_tmp;
    // device-resident sizes and their pinned host mirror
    msp::DBuf dcount;
    msp::DevCounts* hcount = nullptr;
    int depth_hint = -1;                 // tree depth of the last build (-1: none)
    // the octree depends on the positions only: graph steps reuse the one of
    // the last eager build (levels built, checksum of its positions) and
    // refresh the counts and aggregates
    int tree_levels = 0;
    uint64_t pos_sum_ref = 0;
    int64_t pair_cap = 0;                // capacity of the pair table
    cudaEvent_t ev_nf0 = nullptr, ev_nf1 = nullptr;   // around the near-field kernel
    bool nf_timed = false;
    // per-neuron inputs of the last build in caller order (context-owned
    // copies; the selection reads them again)
    msp::DBuf c_type, c_va, c_vde, c_vdi;
    const uint8_t *in_type = nullptr, *in_va = nullptr, *in_vde = nullptr, *in_vdi = nullptr;
    // whole-step CUDA graph (msp_graph.cu).  graph_mode: sizes come from
    // capacity bounds and no call synchronises (set while capturing and for
    // the dry run that sizes the buffers before it).
    bool graph_mode = false;
    int64_t graph_elem_cap = 0;                // element capacity in graph mode
    bool graph_full_build = false;             // graph mode rebuilds the whole octree
    int cap_left_slot = 0;                     // set by the selection while recording
    // every eager build stamps a new tree generation (also in device memory);
    // a replay that reuses the octree checks the stamp it was captured with
    uint64_t tree_gen = 0;
    struct GraphArgs {
        const float *x = nullptr, *y = nullptr, *z = nullptr;
        const uint8_t* type = nullptr;
        uint8_t *va = nullptr, *vde = nullptr, *vdi = nullptr;
        int64_t n = 0;
        int32_t *partner = nullptr, *pre = nullptr, *post = nullptr;
        uint8_t* styp = nullptr;
        int64_t capacity = 0;
        int64_t* n_syn = nullptr;
        int64_t* history = nullptr;
        int64_t history_len = 0;
        uint64_t first_step = 0;
        float* u = nullptr;          // attraction out (sorted-order scatter), or none
        int64_t elem_cap = 0;        // vacant axonal elements the buffers hold
        bool walk = true;            // the step starts with the vacancy walk
        bool commit = true;          // and ends with the commit of its synapses
        bool full_build = false;     // octree rebuilt per replay (else reused)
    };
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        cudaGraph_t tmpl = nullptr;
        int64_t kernels = 0;                      // kernel launches per replay
        cudaGraphNode_t nf0 = nullptr, nf1 = nullptr;   // event records around the near field
        int left_slot = 0;                        // descent counter slot that must end empty
        long long epoch = -1;                     // allocation epoch at capture
        GraphArgs args;
    };
    StepGraph sg;            // the caller's step graph (msp_step_graph_*)
    StepGraph hg;            // the host-buffer call's own step graph
    bool sg_full_build = false;                // option of the next msp_step_graph_capture
    std::vector<cudaEvent_t> g_events;         // two per replay of the last launch
    int64_t g_replays = 0;                     // replays of the last launch
    double g_nf_ms_mean = 0.0;                 // mean near-field time over them
    bool last_was_graph = false;               // statistics come from graph replays
    // host-buffer step staging: inputs, the dry runs' scratch outputs, and
    // the outputs of the host-buffer call's graph
    msp::DBuf h_in[7];
    msp::DBuf h_u, h_partner, h_pre, h_post, h_type, h_nsyn;
    msp::DBuf hs_u, hs_partner, hs_pre, hs_post, hs_type, hs_nsyn;
};

namespace msp {

// ---------------------------------------------------------------------------
// primitives (msp_prims.cu)
// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) by the low `bits` bits of key.  The
// result ends in (keys, vals); (keys_tmp, vals_tmp) are scratch of n entries.
void radix_sort(msp_ctx& c, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp,
                int32_t* vals_tmp, int64_t n, int bits, cudaStream_t s);
// Step a9, the near field over the leaf pairs grouped by target leaf
// (msp_nearfield.cu); accumulates into u_sorted and the pair table.
// Segment and list counts live in device memory (*nseg_dev <= nseg_cap,
// *nlist_dev <= nlist_cap); no host synchronisation.
// expansions about the geometric centres (msp_m2l_gemm.cu)
void geo_centres(msp_ctx& c, cudaStream_t s);
bool m2l_gemm_fits(int p);
const int32_t* m2l_gemm(msp_ctx& c, const int32_t* far_q, const int64_t* nfar, int64_t cap,
                        const float* A, const float* M, float* B, float4* pw,
                        int64_t** first_fallback, cudaStream_t s);
void launch_near_field(msp_ctx& c, const int32_t* seg_first, const int64_t* nseg_dev,
                       int64_t nseg_cap, const int32_t* list_q, const int64_t* nlist_dev,
                       int64_t nlist_cap, float* u_sorted, unsigned long long* work,
                       bool keep_order, cudaStream_t s);
// Exclusive scan of in[0, *n_dev) (n_dev in device memory, at most n_cap)
// into out; *total_dst = total (+ *base if base).  No host synchronisation.
// With overflow given, an end above clamp_cap sets overflow_bit in *overflow,
// raises *need to it and stores *base instead.
void scan_dev(msp_ctx& c, const int32_t* in, int32_t* out, const int64_t* n_dev, int64_t n_cap,
              int64_t* total_dst, const int64_t* base, cudaStream_t s, int64_t clamp_cap = 0,
              int64_t* overflow = nullptr, int64_t* need = nullptr, int64_t overflow_bit = 1);
// Stable radix sort of the first *n_dev (<= n_cap) pairs.  No host sync.
void radix_sort_dev(msp_ctx& c, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp,
                    int32_t* vals_tmp, const int64_t* n_dev, int64_t n_cap, int bits,
                    cudaStream_t s);
// small device-side bookkeeping (msp_prims.cu)
void dev_set(int64_t* dst, int64_t v, cudaStream_t s);
void dev_store_i32(int32_t* dst, const int64_t* src, cudaStream_t s);
// device counts of a context and their host mirror (synchronous)
inline DevCounts* dcounts(msp_ctx& c) { return c.dcount.get<DevCounts>(); }
void pull_counts(msp_ctx& c, cudaStream_t s);

inline int grid_for(int64_t n, int block, int64_t cap = 1 << 20) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications, key bumped by the Weyl constants between rounds.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)p1;
        c[3] = (uint32_t)p0;
        c[0] = n0;
        c[2] = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// counter (c0, c1, step_lo, step_hi), key = seed; returns the 4 output words
__host__ __device__ inline void philox_draw(uint64_t seed, uint32_t c0, uint32_t c1,
                                            uint64_t step, uint32_t out[4]) {
    out[0] = c0;
    out[1] = c1;
    out[2] = (uint32_t)step;
    out[3] = (uint32_t)(step >> 32);
    philox4x32_10(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// U in [0,1) from the top 53 bits of the first two output words
// the 53 bits of a uniform draw U = bits 2^-53 in [0, 1)
__host__ __device__ inline uint64_t philox_bits53(uint64_t seed, uint32_t c0, uint32_t c1,
                                                  uint64_t step) {
    uint32_t o[4];
    philox_draw(seed, c0, c1, step, o);
    return (((uint64_t)o[0] << 32) | o[1]) >> 11;
}

__host__ __device__ inline double philox_uniform(uint64_t seed, uint32_t c0, uint32_t c1,
                                                 uint64_t step) {
    return (double)philox_bits53(seed, c0, c1, step) * (1.0 / 9007199254740992.0);
}

// Double-FP32 ("float-float") values hi + lo, |lo| <= ulp(hi) / 2: about 48
// significant bits on the FP32 pipe (double precision arithmetic is scarce on
// this GPU).  The pair table holds W(X,Y) of both channels as one float4
// (E hi, E lo, I hi, I lo).  Sums use Knuth's two-sum on both parts and two
// renormalisations (relative error a few units of 2^-48); the product uses
// the FMA's exact residual.
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 ff_quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float2 s = ff_two_sum(a.x, b.x);
    const float2 t = ff_two_sum(a.y, b.y);
    s = ff_quick_two_sum(s.x, __fadd_rn(s.y, t.x));
    return ff_quick_two_sum(s.x, __fadd_rn(s.y, t.y));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    const float e = __fmaf_rn(a.x, b.x, -p);
    return ff_quick_two_sum(p, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e)));
}
// a compensated running sum (Neumaier): h += x.hi, the rounding error and
// x.lo go into c; the pair (h, c) is turned into hi + lo at the end (two-sum).
// Adding one such pair to another is the same step (commutative bit for bit).
__device__ __forceinline__ void ff_acc(float& h, float& c, float xh, float xl) {
    const float2 t = ff_two_sum(h, xh);
    h = t.x;
    c = __fadd_rn(__fadd_rn(c, xl), t.y);
}
__device__ __forceinline__ bool ff_gt(float2 a, float2 b) {
    return a.x > b.x || (a.x == b.x && a.y > b.y);
}
// U = bits 2^-53 as hi + lo: the top 24 bits exactly, the other 29 rounded
__device__ __forceinline__ float2 ff_uniform(uint64_t bits53) {
    const float hi = (float)(uint32_t)(bits53 >> 29) * 0x1p-24f;
    const float lo = (float)(uint32_t)(bits53 & 0x1FFFFFFFull) * 0x1p-53f;
    return ff_quick_two_sum(hi, lo);
}

// every third bit of v (bits 0,3,6,...) packed into the low bits
__host__ __device__ inline uint32_t compact_by3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

// spread the low 21 bits of v to bits 0,3,6,...
__host__ __device__ inline uint64_t spread_by3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// A box's integer coordinate along axis d (0 = x) in units of its own side,
// counted in the frame its points are given in.  With frames (frame_level
// > 0) a box at or below the frame level is counted from the low corner of
// its frame's cell (its coordinate modulo the cell's), so its centre is
// formed in that network's own frame; a box above it spans several networks,
// is never evaluated or translated and counts from 0.
__host__ __device__ inline uint32_t box_axis(uint64_t prefix, int d, int level,
                                             int frame_level) {
    const uint32_t c = compact_by3(prefix >> (2 - d));
    if (frame_level <= 0) return c;
    return level >= frame_level ? c & ((1u << (level - frame_level)) - 1u) : 0u;
}

// The network (frame) of a box at or below the frame level: its cell's
// coordinates are the top frame_level bits of each axis of its prefix, and
// network k sits in the cell 2 (k mod G, (k / G) mod G, k / G^2), G =
// 2^(frame_level - 1).  Clamped to [0, nf).
__host__ __device__ inline int64_t box_frame(uint64_t prefix, int level, int frame_level,
                                             int64_t nf) {
    const uint64_t cell = prefix >> (3 * (level - frame_level));
    const int64_t G = 1ll << (frame_level - 1);
    const int64_t k = (int64_t)(compact_by3(cell >> 2) >> 1) +
                      G * ((int64_t)(compact_by3(cell >> 1) >> 1) +
                           G * (int64_t)(compact_by3(cell) >> 1));
    return k < 0 ? 0 : (k < nf ? k : nf - 1);
}

// packed per-point bytes: type | vac_axon << 8 | vac_dend_e << 16 | vac_dend_i << 24
__device__ inline uint32_t pk_type(uint32_t w) { return w & 0xffu; }
__device__ inline uint32_t pk_axon(uint32_t w) { return (w >> 8) & 0xffu; }
__device__ inline uint32_t pk_de(uint32_t w) { return (w >> 16) & 0xffu; }
__device__ inline uint32_t pk_di(uint32_t w) { return w >> 24; }

}  // namespace msp
