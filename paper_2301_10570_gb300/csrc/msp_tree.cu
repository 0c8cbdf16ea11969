// msp_tree.cu -- steps a1-a4: Morton keys, stable sort + gather into a
// Morton-ordered float4 array, the adaptive octree (Section 3.2) built level
// by level, and the per-box sums of vacant elements and centroids.
#include "msp_internal.cuh"

namespace msp {

namespace {

// q = floor((v - o) * scale) in single precision with round-to-nearest, then
// clamped to the 2^21 grid; NaN maps to 0.
__device__ inline uint32_t quantise(float v, float o, float scale) {
    float f = floorf(__fmul_rn(__fsub_rn(v, o), scale));
    if (!(f >= 0.0f)) return 0u;
    if (f >= 2097152.0f) return 2097151u;
    return (uint32_t)f;
}

__global__ void k_build_init(DevCounts* dc, int64_t n) {
    dc->n = n;
    dc->bad_pos = 0;
    dc->pos_sum = 0;
}

// order-independent checksum of the positions: the sum over i (modulo 2^64)
// of a mix of i and every bit of the three coordinates (the finaliser of
// SplitMix64, Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014, applied twice)
__device__ inline unsigned long long pos_mix(unsigned long long h) {
    h ^= h >> 30;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 27;
    h *= 0x94D049BB133111EBull;
    h ^= h >> 31;
    return h;
}

__global__ void k_pos_sum(const float* __restrict__ x, const float* __restrict__ y,
                          const float* __restrict__ z, int64_t n,
                          unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long xy = ((unsigned long long)__float_as_uint(x[i]) << 32) |
                                      __float_as_uint(y[i]);
        unsigned long long h = pos_mix(xy ^ ((unsigned long long)i * 0x9E3779B97F4A7C15ull));
        h = pos_mix(h ^ ((unsigned long long)__float_as_uint(z[i]) * 0xD6E8FEB86659FD93ull));
        acc += h;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// the positions of a graph step must be those its octree was built from
// a replay that reuses the octree: the positions must be those of the build
// (checksum) and the octree arrays those of that build (generation stamp)
__global__ void k_pos_check(DevCounts* dc, uint64_t ref, uint64_t gen) {
    if (dc->pos_sum != ref || dc->tree_gen != gen) dc->bad_pos = 1;
}

// a graph replay that rebuilt the octree: no capture holds this stamp, so a
// replay of another graph that reuses the octree halts instead
__global__ void k_mark_graph_tree(DevCounts* dc) { dc->tree_gen = ~0ull; }

// keys; a position outside [origin, origin + side) or not finite is counted
// (the build then fails: the tree's boxes must contain their points)
__global__ void k_morton(const float* __restrict__ x, const float* __restrict__ y,
                         const float* __restrict__ z, int64_t n, float ox, float oy, float oz,
                         float side, float scale, uint64_t* __restrict__ keys,
                         int32_t* __restrict__ vals, int64_t* __restrict__ bad) {
    bool any_bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        any_bad |= !(x[i] >= ox && x[i] < ox + side && y[i] >= oy && y[i] < oy + side &&
                     z[i] >= oz && z[i] < oz + side);
        uint32_t qx = quantise(x[i], ox, scale);
        uint32_t qy = quantise(y[i], oy, scale);
        uint32_t qz = quantise(z[i], oz, scale);
        keys[i] = (spread_by3(qx) << 2) | (spread_by3(qy) << 1) | spread_by3(qz);
        vals[i] = (int32_t)i;
    }
    if (__any_sync(0xffffffffu, any_bad) && (threadIdx.x & 31) == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(bad), 1ull);
}

// Keys of independent networks in local frames.  Neuron i belongs to the
// network k with off[k] <= i < off[k+1]; that network's cell at level L0 has
// the grid coordinates 2 (k mod G, (k / G) mod G, k / G^2), G = 2^(L0-1), and
// the neuron's position is relative to the cell's low corner, inside
// [0, cs).  Each axis of the key holds the cell's coordinate in its top L0
// bits and the local position, quantised on the same grid, below them: the
// key the point would have in one common frame, without ever forming its
// position in that frame in single precision.
__global__ void k_morton_frames(const float* __restrict__ x, const float* __restrict__ y,
                                const float* __restrict__ z, int64_t n,
                                const int64_t* __restrict__ off, int64_t nf, int L0, float cs,
                                float scale, uint64_t* __restrict__ keys,
                                int32_t* __restrict__ vals, int64_t* __restrict__ bad) {
    const int sh = kMortonBits - L0;
    const uint32_t qmax = (1u << sh) - 1u;
    const int64_t G = 1ll << (L0 - 1);
    bool any_bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nf;   // off[lo] <= i < off[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid;
        }
        const uint32_t cx = (uint32_t)(2 * (lo % G)), cy = (uint32_t)(2 * ((lo / G) % G)),
                       cz = (uint32_t)(2 * (lo / (G * G)));
        any_bad |= !(x[i] >= 0.f && x[i] < cs && y[i] >= 0.f && y[i] < cs && z[i] >= 0.f &&
                     z[i] < cs);
        const uint32_t qx = (cx << sh) | min(quantise(x[i], 0.f, scale), qmax);
        const uint32_t qy = (cy << sh) | min(quantise(y[i], 0.f, scale), qmax);
        const uint32_t qz = (cz << sh) | min(quantise(z[i], 0.f, scale), qmax);
        keys[i] = (spread_by3(qx) << 2) | (spread_by3(qy) << 1) | spread_by3(qz);
        vals[i] = (int32_t)i;
    }
    if (__any_sync(0xffffffffu, any_bad) && (threadIdx.x & 31) == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(bad), 1ull);
}

__global__ void k_gather(const int32_t* __restrict__ order, int64_t n, const float* __restrict__ x,
                         const float* __restrict__ y, const float* __restrict__ z,
                         const uint8_t* __restrict__ type, const uint8_t* __restrict__ va,
                         const uint8_t* __restrict__ vde, const uint8_t* __restrict__ vdi,
                         int32_t* __restrict__ perm, int32_t* __restrict__ inv,
                         float4* __restrict__ pts, float2* __restrict__ wts,
                         float2* __restrict__ lw) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = order[j];
        perm[j] = i;
        inv[i] = (int32_t)j;
        uint32_t packed = (uint32_t)(type[i] ? 1u : 0u) | ((uint32_t)va[i] << 8) |
                          ((uint32_t)vde[i] << 16) | ((uint32_t)vdi[i] << 24);
        pts[j] = make_float4(x[i], y[i], z[i], __uint_as_float(packed));
        wts[j] = make_float2((float)vde[i], (float)vdi[i]);
        // log2 of the dendrite weights (-inf for none), added in the exponent
        lw[j] = make_float2(vde[i] ? log2f((float)vde[i]) : -INFINITY,
                            vdi[i] ? log2f((float)vdi[i]) : -INFINITY);
    }
}

__global__ void k_u8_to_i32(const uint8_t* __restrict__ a, int64_t n, int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i];
}

__global__ void k_init_root(int64_t n, uint8_t* level, uint64_t* prefix, int32_t* first,
                            int32_t* count, int32_t* parent, int32_t* child_first,
                            uint8_t* nchild, int64_t* level_start, int64_t* overflow) {
    level_start[0] = 0;
    level_start[1] = 1;
    *overflow &= ~16ll;
    level[0] = 0;
    prefix[0] = 0;
    first[0] = 0;
    count[0] = (int32_t)n;
    parent[0] = -1;
    child_first[0] = -1;
    nchild[0] = 0;
}

// first index in [lo, hi) whose octant (at shift) is >= o; octants are
// non-decreasing inside a box because the higher bits are the box prefix
__device__ inline int32_t octant_lower_bound(const uint64_t* __restrict__ keys, int32_t lo,
                                             int32_t hi, int shift, uint32_t o) {
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (((keys[mid] >> shift) & 7u) < o)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Octant boundaries of the boxes of one level, 8 lanes per box (one binary
// search per octant): lane o of a box's group returns the end of octant o and
// the start of octant o (its neighbour's end, or the box start for o = 0).
// Whole warps take part (4 boxes per warp per round).
struct OctantSplit {
    int64_t k;         // box index within the level (valid if < nl)
    bool valid, split;
    int32_t lo, end, start;
};

// Per-network leaf capacities (Caps.cap non-null, points in frames): a box at
// or below the frame level splits above its network's capacity, a box above
// it (several networks' cells) always splits.
struct Caps {
    const int32_t* cap;        // per network, or null: leaf_capacity for every box
    const uint64_t* prefix;    // box prefixes (with cap)
    int frame_level;
    int64_t nf;
};

__device__ inline OctantSplit octant_split(int64_t base, int64_t l0, int64_t nl, int level,
                                           int leaf_capacity, int max_depth, Caps cp,
                                           const uint64_t* __restrict__ keys,
                                           const int32_t* __restrict__ first,
                                           const int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31, o = lane & 7;
    OctantSplit r;
    r.k = base + (lane >> 3);
    r.valid = r.k < nl;
    r.split = false;
    r.lo = 0;
    int32_t e = 0;
    if (r.valid) {
        const int64_t i = l0 + r.k;
        const int32_t c = count[i];
        r.lo = first[i];
        int cap = leaf_capacity;
        if (cp.cap)
            cap = level >= cp.frame_level
                      ? cp.cap[box_frame(cp.prefix[i], level, cp.frame_level, cp.nf)]
                      : -1;
        r.split = c > cap && level < max_depth;
        if (r.split)
            e = octant_lower_bound(keys, r.lo, r.lo + c, 3 * (kMortonBits - (level + 1)),
                                   (uint32_t)o + 1);
    }
    int32_t prev = __shfl_up_sync(0xffffffffu, e, 1);
    r.end = e;
    r.start = o == 0 ? r.lo : prev;
    return r;
}

// number of non-empty octants of every box at this level that is split; the
// level's boxes are [lb[0], lb[1]), their count goes to *scan_n for the scan
__global__ void k_count_children(const int64_t* __restrict__ lb, int level, int leaf_capacity,
                                 int max_depth, Caps cp, const uint64_t* __restrict__ keys,
                                 const int32_t* __restrict__ first, const int32_t* __restrict__ count,
                                 int32_t* __restrict__ cnt, int64_t* __restrict__ scan_n) {
    const int lane = threadIdx.x & 31;
    const int64_t l0 = lb[0], nl = lb[1] - lb[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) *scan_n = nl;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = wid * 4; base < nl; base += nw * 4) {
        OctantSplit r =
            octant_split(base, l0, nl, level, leaf_capacity, max_depth, cp, keys, first, count);
        const unsigned m = __ballot_sync(0xffffffffu, r.split && r.end > r.start);
        if (r.valid && (lane & 7) == 0) cnt[r.k] = __popc((m >> (lane & ~7)) & 0xffu);
    }
}

// children of the level's boxes [lb[0], lb[1]); the next level starts at lb[1]
__global__ void k_emit_children(const int64_t* __restrict__ lb, int level, int leaf_capacity,
                                int max_depth, Caps cp, const uint64_t* __restrict__ keys,
                                const int32_t* __restrict__ off, uint8_t* __restrict__ nd_level,
                                uint64_t* __restrict__ nd_prefix, int32_t* __restrict__ nd_first,
                                int32_t* __restrict__ nd_count, int32_t* __restrict__ nd_parent,
                                int32_t* __restrict__ nd_child_first,
                                uint8_t* __restrict__ nd_nchild,
                                const int64_t* __restrict__ overflow) {
    const int lane = threadIdx.x & 31, o = lane & 7;
    const int64_t l0 = lb[0], nl = lb[1] - lb[0], next0 = lb[1];
    // the node arrays could not hold the next level (a bound that cannot be
    // exceeded; guarded all the same): no children are written
    if (*overflow & 16) return;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = wid * 4; base < nl; base += nw * 4) {
        OctantSplit r = octant_split(base, l0, nl, level, leaf_capacity, max_depth, cp, keys,
                                     nd_first, nd_count);
        const bool ne = r.split && r.end > r.start;
        const unsigned m = __ballot_sync(0xffffffffu, ne);
        const unsigned grp = (m >> (lane & ~7)) & 0xffu;
        if (!r.valid || grp == 0) continue;
        const int64_t i = l0 + r.k;
        const int64_t cf = next0 + off[r.k];
        if (o == 0) {
            nd_child_first[i] = (int32_t)cf;
            nd_nchild[i] = (uint8_t)__popc(grp);
        }
        if (ne) {
            const int64_t ci = cf + __popc(grp & ((1u << o) - 1u));
            nd_level[ci] = (uint8_t)(level + 1);
            nd_prefix[ci] = (nd_prefix[i] << 3) | (uint64_t)o;
            nd_first[ci] = r.start;
            nd_count[ci] = r.end - r.start;
            nd_parent[ci] = (int32_t)i;
            nd_child_first[ci] = -1;
            nd_nchild[ci] = 0;
        }
    }
}

// Box aggregates, one launch for the whole octree.  A leaf sums its points;
// an inner box combines its children, and it is computed by the warp of its
// last child to finish: every box, once written, adds one to its parent's
// arrival counter (an acquire-release atomic: the box's results are visible
// before the arrival, the siblings' after it), and the warp that brings the
// counter to the parent's child count resets it and goes on with the parent,
// up to the root.
// Centroids are accumulated as weighted offsets from the box's geometric
// centre so that single precision keeps them accurate (with frames, the
// centre in the box's network's own frame: box_axis).  A leaf's lanes take its
// points, an inner box's lanes its children (at most 8); a fixed butterfly
// sums the lanes, then lane 0 writes the box's vacant-element sums and its
// axon / dendrite centroids (offsets summed, then divided by the weight).  The
// order of every sum is fixed whichever warp computes a box, so the results
// are those of a level-by-level pass.  The counters are zero on entry
// (cleared by the host before an eager build and whenever their buffer is new;
// every complete launch leaves them zero).
__device__ __forceinline__ void aggregate_box(int64_t i, int lane, int frame_level, float ox,
                                              float oy, float oz, float side,
                                              const float4* __restrict__ pts,
                                              const uint8_t* __restrict__ level,
                                              const uint64_t* __restrict__ prefix,
                                              const int32_t* __restrict__ first,
                                              const int32_t* __restrict__ count,
                                              const int32_t* __restrict__ child_first,
                                              const uint8_t* __restrict__ nchild,
                                              int4* __restrict__ sums, float4* __restrict__ ca,
                                              float4* __restrict__ cd,
                                              int32_t* __restrict__ leaf_of) {
    const uint64_t pre = prefix[i];
    const int lv = (int)level[i];
    const float bs = ldexpf(side, -lv);
    const float g[3] = {ox + ((float)box_axis(pre, 0, lv, frame_level) + 0.5f) * bs,
                        oy + ((float)box_axis(pre, 1, lv, frame_level) + 0.5f) * bs,
                        oz + ((float)box_axis(pre, 2, lv, frame_level) + 0.5f) * bs};
    int aE = 0, aI = 0, wE = 0, wI = 0;
    float sa[3] = {0.f, 0.f, 0.f}, sd[3] = {0.f, 0.f, 0.f};
    const int32_t cf = child_first[i];
    if (cf < 0) {
        const int32_t f = first[i], c = count[i];
        for (int32_t j = f + lane; j < f + c; j += 32) {
            const float4 p = pts[j];
            const uint32_t w = __float_as_uint(p.w);
            const int a = (int)pk_axon(w), de = (int)pk_de(w), di = (int)pk_di(w);
            if (pk_type(w)) aI += a; else aE += a;
            wE += de;
            wI += di;
            const float fa = (float)a, fd = (float)(de + di);
            const float dx = p.x - g[0], dy = p.y - g[1], dz = p.z - g[2];
            sa[0] = fmaf(fa, dx, sa[0]); sa[1] = fmaf(fa, dy, sa[1]); sa[2] = fmaf(fa, dz, sa[2]);
            sd[0] = fmaf(fd, dx, sd[0]); sd[1] = fmaf(fd, dy, sd[1]); sd[2] = fmaf(fd, dz, sd[2]);
            leaf_of[j] = (int32_t)i;
        }
    } else if (lane < nchild[i]) {
        // the children were written by other warps: read them from L2
        const int4 sm = __ldcg(&sums[cf + lane]);
        const float4 a4 = __ldcg(&ca[cf + lane]), d4 = __ldcg(&cd[cf + lane]);
        aE = sm.x; aI = sm.y; wE = sm.z; wI = sm.w;
        const float fa = (float)(sm.x + sm.y), fd = (float)(sm.z + sm.w);
        sa[0] = fa * (a4.x - g[0]); sa[1] = fa * (a4.y - g[1]); sa[2] = fa * (a4.z - g[2]);
        sd[0] = fd * (d4.x - g[0]); sd[1] = fd * (d4.y - g[1]); sd[2] = fd * (d4.z - g[2]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        aE += __shfl_xor_sync(0xffffffffu, aE, o);
        aI += __shfl_xor_sync(0xffffffffu, aI, o);
        wE += __shfl_xor_sync(0xffffffffu, wE, o);
        wI += __shfl_xor_sync(0xffffffffu, wI, o);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            sa[d] += __shfl_xor_sync(0xffffffffu, sa[d], o);
            sd[d] += __shfl_xor_sync(0xffffffffu, sd[d], o);
        }
    }
    if (lane == 0) {
        sums[i] = make_int4(aE, aI, wE, wI);
        const float ta = (float)(aE + aI), td = (float)(wE + wI);
        ca[i] = ta > 0.f ? make_float4(g[0] + sa[0] / ta, g[1] + sa[1] / ta, g[2] + sa[2] / ta, ta)
                         : make_float4(g[0], g[1], g[2], 0.f);
        cd[i] = td > 0.f ? make_float4(g[0] + sd[0] / td, g[1] + sd[1] / td, g[2] + sd[2] / td, td)
                         : make_float4(g[0], g[1], g[2], 0.f);
    }
}

// arrival at a parent: release for the box's own results, acquire for its
// siblings' (the last arrival reads them)
__device__ __forceinline__ int arrive_acq_rel(int32_t* p) {
    int old;
    asm volatile("atom.add.acq_rel.gpu.s32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

// nodes_end: the node count (device memory); one warp per leaf
__global__ void k_aggregate_tree(const int64_t* __restrict__ nodes_end, int frame_level, float ox,
                                 float oy, float oz, float side, const float4* __restrict__ pts,
                                 const uint8_t* __restrict__ level,
                                 const uint64_t* __restrict__ prefix,
                                 const int32_t* __restrict__ first,
                                 const int32_t* __restrict__ count,
                                 const int32_t* __restrict__ parent,
                                 const int32_t* __restrict__ child_first,
                                 const uint8_t* __restrict__ nchild, int4* __restrict__ sums,
                                 float4* __restrict__ ca, float4* __restrict__ cd,
                                 int32_t* __restrict__ leaf_of, int32_t* __restrict__ arrive) {
    const int64_t nn = *nodes_end;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nn; k += nw) {
        if (child_first[k] >= 0) continue;        // inner boxes: done by their last child's warp
        int64_t i = k;
        for (;;) {
            aggregate_box(i, lane, frame_level, ox, oy, oz, side, pts, level, prefix, first, count,
                          child_first, nchild, sums, ca, cd, leaf_of);
            const int32_t p = parent[i];
            if (p < 0) break;
            int last = 0;
            if (lane == 0) {
                // lane 0 wrote the box's results
                last = arrive_acq_rel(&arrive[p]) == (int)nchild[p] - 1;
                if (last) arrive[p] = 0;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (!last) break;
            __syncwarp();                         // the lanes' reads after lane 0's acquire
            i = p;
        }
    }
}

// a warp per node (the leaves all start at once), at most 16 blocks per SM
int agg_grid(int64_t nodes, int64_t sm_count) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((nodes + 3) / 4, sm_count * 16));
}

}  // namespace

void build_tree(msp_ctx& c, int64_t n, const float* x, const float* y, const float* z,
                const uint8_t* type, const uint8_t* va, const uint8_t* vde, const uint8_t* vdi,
                cudaStream_t s) {
    NvtxRange nv_("msp build_tree");
    const bool was_built = c.tree_built;
    const int64_t prev_n = c.n;
    if (!c.graph_mode) {
        c.tree_built = false;
        c.attraction_done = false;
        c.tree_reused = false;
    }
    c.n = n;
    const msp_config& cfg = c.cfg;
    DevCounts* dc = dcounts(c);
    k_build_init<<<1, 1, 0, s>>>(dc, n);
    MSP_LAUNCH("build_init");
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint64_t* k0 = c.keys0.ensure<uint64_t>(nn);
    uint64_t* k1 = c.keys1.ensure<uint64_t>(nn);
    int32_t* v0 = c.vals0.ensure<int32_t>(nn);
    int32_t* v1 = c.vals1.ensure<int32_t>(nn);
    int32_t* perm = c.perm.ensure<int32_t>(nn);
    int32_t* inv = c.inv.ensure<int32_t>(nn);
    float4* pts = c.pts.ensure<float4>(nn);
    float2* wts = c.wts.ensure<float2>(nn);
    float2* lw = c.lw.ensure<float2>(nn);
    int32_t* eoff = c.elem_off.ensure<int32_t>(nn + 1);
    int32_t* leaf_of = c.leaf_of.ensure<int32_t>(nn);
    const int B = 256;
    const int G = grid_for(n, B, (int64_t)c.sm_count * 16);
    // box centres: in the domain's frame, or (frames) in each network's own
    const bool framed = c.frame_level > 0;
    const float o3[3] = {framed ? 0.f : cfg.origin[0], framed ? 0.f : cfg.origin[1],
                         framed ? 0.f : cfg.origin[2]};
    if (framed && n != c.frame_off_host.back())
        throw Error(MSP_ERR_INVALID_ARG, "the frames (msp_set_frames) hold a different number "
                                         "of neurons");
    if (n > 0) {
        k_pos_sum<<<G, B, 0, s>>>(x, y, z, n, reinterpret_cast<unsigned long long*>(&dc->pos_sum));
        MSP_LAUNCH("pos_sum");
    }

    // An eager build on the positions of the last build (their checksum,
    // read back: one more synchronisation) keeps its sorted order and octree,
    // which depend on the positions only.
    bool eager_reuse = false;
    if (!c.graph_mode && was_built && n == prev_n && n > 0) {
        unsigned long long ps = 0;
        MSP_CUDA(cudaMemcpyAsync(&ps, &dc->pos_sum, sizeof(ps), cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        eager_reuse = ps == c.pos_sum_ref;
    }
    if (!eager_reuse && !c.graph_mode) c.lists_valid = false;

    // Inside the whole-step graph the positions are those of the last eager
    // build (checked: a different checksum halts the graph), so its sorted
    // order and octree are reused; the counts are gathered again and the
    // aggregates recomputed.  The same for an eager build on those positions.
    if ((c.graph_mode && c.tree_built && !c.graph_full_build) || eager_reuse) {
        if (c.graph_mode) {
            k_pos_check<<<1, 1, 0, s>>>(dc, c.pos_sum_ref, c.tree_gen);
            MSP_LAUNCH("pos_check");
        } else {
            // the octree arrays are those of generation tree_gen (a graph
            // replay that rebuilt them for the same positions left its mark)
            dev_set(reinterpret_cast<int64_t*>(&dc->tree_gen), (int64_t)c.tree_gen, s);
        }
        if (n > 0) {
            k_gather<<<G, B, 0, s>>>(v0, n, x, y, z, type, va, vde, vdi, perm, inv, pts, wts, lw);
            MSP_LAUNCH("gather");
            int32_t* tmp = c.cnt.ensure<int32_t>(nn);
            k_u8_to_i32<<<G, B, 0, s>>>(va, n, tmp);
            MSP_LAUNCH("u8_to_i32");
            scan_dev(c, tmp, eoff, &dc->n, n, &dc->n_elem, nullptr, s);
            dev_store_i32(eoff + n, &dc->n_elem, s);
        } else {
            dev_set(&dc->n_elem, 0, s);
        }
        const int Gt = (int)std::max<int64_t>(1, (int64_t)c.sm_count * 8);
        if (!c.graph_mode) MSP_CUDA(cudaMemsetAsync(c.nd_arrive.p, 0, c.nd_arrive.bytes, s));
        k_aggregate_tree<<<agg_grid(c.n_nodes, c.sm_count), 128, 0, s>>>(
            &dc->level_start[c.tree_levels + 1], c.frame_level, o3[0], o3[1], o3[2], cfg.side, pts,
            c.nd_level.get<uint8_t>(), c.nd_prefix.get<uint64_t>(), c.nd_first.get<int32_t>(),
            c.nd_count.get<int32_t>(), c.nd_parent.get<int32_t>(), c.nd_child_first.get<int32_t>(),
            c.nd_nchild.get<uint8_t>(), c.nd_sums.get<int4>(), c.nd_ca.get<float4>(),
            c.nd_cd.get<float4>(), leaf_of, c.nd_arrive.get<int32_t>());
        MSP_LAUNCH("aggregate");
        if (eager_reuse) {
            pull_counts(c, s);          // the one synchronisation of the build
            c.n_elem = c.hcount->n_elem;
            c.tree_built = true;
            c.tree_reused = true;
        }
        return;
    }

    // a1 + a2: keys, stable sort, gather into Morton order
    if (n > 0) {
        if (framed) {
            k_morton_frames<<<G, B, 0, s>>>(x, y, z, n, c.frame_off.get<int64_t>(),
                                            (int64_t)c.frame_off_host.size() - 1, c.frame_level,
                                            ldexpf(cfg.side, -c.frame_level), c.morton_scale, k0,
                                            v0, &dc->bad_pos);
            MSP_LAUNCH("morton_frames");
        } else {
            k_morton<<<G, B, 0, s>>>(x, y, z, n, cfg.origin[0], cfg.origin[1], cfg.origin[2],
                                     cfg.side, c.morton_scale, k0, v0, &dc->bad_pos);
            MSP_LAUNCH("morton");
        }
        radix_sort(c, k0, v0, k1, v1, n, 3 * kMortonBits, s);
        k_gather<<<G, B, 0, s>>>(v0, n, x, y, z, type, va, vde, vdi, perm, inv, pts, wts, lw);
        MSP_LAUNCH("gather");
        // element offsets: exclusive prefix of the vacant axonal counts
        int32_t* tmp = c.cnt.ensure<int32_t>(nn);
        k_u8_to_i32<<<G, B, 0, s>>>(va, n, tmp);
        MSP_LAUNCH("u8_to_i32");
        scan_dev(c, tmp, eoff, &dc->n, n, &dc->n_elem, nullptr, s);
        dev_store_i32(eoff + n, &dc->n_elem, s);
    } else {
        dev_set(&dc->n_elem, 0, s);
    }

    // a3: level-synchronous octree; the level sizes stay in device memory.
    // Levels are built down to the previous tree's depth + 1 (a first guess
    // from n and the leaf capacity otherwise); if a box of the last built level
    // would still split, the tree is rebuilt with all levels.
    int L = c.depth_hint;
    if (L < 0) {
        L = 3;
        for (int64_t m = std::max<int64_t>(n / std::max(cfg.leaf_capacity, 1), 1); m > 1; m >>= 3) ++L;
    } else {
        L += 1;
    }
    L = std::min(std::max(L, 0), cfg.max_depth);
    const int Gt = (int)std::max<int64_t>(1, (int64_t)c.sm_count * 8);
    Caps cp{nullptr, nullptr, c.frame_level, (int64_t)c.frame_off_host.size() - 1};
    int min_cap = cfg.leaf_capacity;
    if (framed && c.frame_plans)
        for (int32_t v : c.frame_cap_host) min_cap = std::min(min_cap, (int)v);
    int32_t* cnt = c.cnt.ensure<int32_t>(nn + 8);
    int32_t* off = c.off.ensure<int32_t>(nn + 8);
    // boxes at level l: at most min(8^l, n), and (l >= 1) at most 8 children
    // of each box of level l-1 that splits, i.e. holds more than C neurons
    const int64_t splitters = (int64_t)nn / ((int64_t)min_cap + 1);
    auto level_cap = [&](int l) -> int64_t {
        int64_t c = l < 8 ? std::min<int64_t>((int64_t)1 << (3 * l), (int64_t)nn) : (int64_t)nn;
        if (l >= 1) c = std::min<int64_t>(c, 8 * splitters);
        return std::max<int64_t>(c, 1);
    };
    for (;;) {
        int64_t cap = 0;
        for (int l = 0; l <= L; ++l) cap += level_cap(l);
        cap += 8;
        c.nd_level.ensure<uint8_t>((size_t)cap);
        c.nd_prefix.ensure<uint64_t>((size_t)cap);
        c.nd_first.ensure<int32_t>((size_t)cap);
        c.nd_count.ensure<int32_t>((size_t)cap);
        c.nd_parent.ensure<int32_t>((size_t)cap);
        c.nd_child_first.ensure<int32_t>((size_t)cap);
        c.nd_nchild.ensure<uint8_t>((size_t)cap);
        int4* sums = c.nd_sums.ensure<int4>((size_t)cap);
        if (framed && c.frame_plans) {
            cp.cap = c.frame_cap.get<int32_t>();
            cp.prefix = c.nd_prefix.get<uint64_t>();
        }
        float4* ca = c.nd_ca.ensure<float4>((size_t)cap);
        float4* cd = c.nd_cd.ensure<float4>((size_t)cap);
        // the arrival counters: cleared before an eager build and whenever
        // the buffer is new (a graph's dry run may build one level deeper than
        // the eager build and grow it); a replay finds them as the last
        // complete launch left them, zero
        const size_t arrive_bytes = c.nd_arrive.bytes;
        int32_t* arrive = c.nd_arrive.ensure<int32_t>((size_t)cap);
        if (!c.graph_mode || c.nd_arrive.bytes != arrive_bytes)
            MSP_CUDA(cudaMemsetAsync(arrive, 0, c.nd_arrive.bytes, s));
        k_init_root<<<1, 1, 0, s>>>(n, c.nd_level.get<uint8_t>(), c.nd_prefix.get<uint64_t>(),
                                    c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(),
                                    c.nd_parent.get<int32_t>(), c.nd_child_first.get<int32_t>(),
                                    c.nd_nchild.get<uint8_t>(), dc->level_start, &dc->overflow);
        MSP_LAUNCH("init_root");
        for (int l = 0; l < L; ++l) {
            const int64_t lcap = level_cap(l);
            k_count_children<<<Gt, B, 0, s>>>(&dc->level_start[l], l, cfg.leaf_capacity,
                                              cfg.max_depth, cp, k0, c.nd_first.get<int32_t>(),
                                              c.nd_count.get<int32_t>(), cnt, &dc->scan_n);
            MSP_LAUNCH("count_children");
            scan_dev(c, cnt, off, &dc->scan_n, lcap, &dc->level_start[l + 2],
                     &dc->level_start[l + 1], s, cap, &dc->overflow, &dc->need_nodes, 16);
            k_emit_children<<<Gt, B, 0, s>>>(
                &dc->level_start[l], l, cfg.leaf_capacity, cfg.max_depth, cp, k0, off,
                c.nd_level.get<uint8_t>(), c.nd_prefix.get<uint64_t>(), c.nd_first.get<int32_t>(),
                c.nd_count.get<int32_t>(), c.nd_parent.get<int32_t>(),
                c.nd_child_first.get<int32_t>(), c.nd_nchild.get<uint8_t>(), &dc->overflow);
            MSP_LAUNCH("emit_children");
        }
        // would a box of the last built level still split?
        if (L < cfg.max_depth) {
            k_count_children<<<Gt, B, 0, s>>>(&dc->level_start[L], L, cfg.leaf_capacity,
                                              cfg.max_depth, cp, k0, c.nd_first.get<int32_t>(),
                                              c.nd_count.get<int32_t>(), cnt, &dc->scan_n);
            MSP_LAUNCH("count_children");
            scan_dev(c, cnt, off, &dc->scan_n, (int64_t)nn, &dc->more_levels, nullptr, s);
        } else {
            dev_set(&dc->more_levels, 0, s);
        }
        // a4: aggregates, leaves up to the root in one launch
        k_aggregate_tree<<<agg_grid(cap, c.sm_count), 128, 0, s>>>(
            &dc->level_start[L + 1], c.frame_level, o3[0], o3[1], o3[2], cfg.side, pts,
            c.nd_level.get<uint8_t>(), c.nd_prefix.get<uint64_t>(), c.nd_first.get<int32_t>(),
            c.nd_count.get<int32_t>(), c.nd_parent.get<int32_t>(), c.nd_child_first.get<int32_t>(),
            c.nd_nchild.get<uint8_t>(), sums, ca, cd, leaf_of, arrive);
        MSP_LAUNCH("aggregate");
        // inside the whole-step graph the tree of the same positions has the
        // same levels; a deeper one sets more_levels, which halts the graph
        if (c.graph_mode) {
            k_mark_graph_tree<<<1, 1, 0, s>>>(dc);
            MSP_LAUNCH("mark_graph_tree");
            return;
        }
        pull_counts(c, s);          // the one synchronisation of the build
        if (c.hcount->bad_pos)
            throw Error(MSP_ERR_INVALID_ARG,
                        framed ? "a position is outside its frame's cell [0, side / 2^level) "
                                 "or not finite"
                               : "a position is outside [origin, origin + side) or not finite");
        if (c.hcount->overflow & 16) throw Error(MSP_ERR_CHECK, "octree node capacity exceeded");
        if (c.hcount->more_levels > 0 && L < cfg.max_depth) {
            L = cfg.max_depth;
            continue;
        }
        break;
    }
    const DevCounts& hc = *c.hcount;
    int depth = 0;
    for (int l = 1; l <= L; ++l)
        if (hc.level_start[l + 1] > hc.level_start[l]) depth = l;
    c.level_start.assign(hc.level_start, hc.level_start + depth + 2);
    c.n_nodes = hc.level_start[depth + 1];
    c.tree_depth = depth;
    c.depth_hint = depth;
    c.n_elem = hc.n_elem;
    c.tree_levels = L;
    c.pos_sum_ref = hc.pos_sum;
    c.tree_gen += 1;
    dev_set(reinterpret_cast<int64_t*>(&dc->tree_gen), (int64_t)c.tree_gen, s);
    c.tree_built = true;
}

}  // namespace msp
