// msp_select.cu -- steps a11-a12: the level-synchronous descent of
// Algorithm 1 with Algorithm 2's choice (candidate attractions, total, uniform
// draw, upper_bound over the inclusive prefix sums), the per-element draw of a
// dendrite neuron inside the chosen leaf, and the resolution of the requests
// at the dendrite side (Section 4).  Also the vacancy random walk and the
// consumption of formed synapses.
#include <algorithm>

#include "msp_internal.cuh"

namespace msp {

__device__ inline float ex2_approx_sel(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__constant__ float c_inv_fact_sel[kMaxP] = {1.f, 1.f, 0.5f, 1.f / 6.f, 1.f / 24.f, 1.f / 120.f,
                                            1.f / 720.f, 1.f / 5040.f};

namespace {

struct Tree {
    const uint8_t* level;
    const int32_t* first;
    const int32_t* count;
    const int32_t* child_first;
    const uint8_t* nchild;
    const int4* sums;
    const float4* ca;
    const float4* cd;
};

struct Exps {
    const float* A;
    const float* M;
    int64_t first;
    int p;
    float inv_sigma;
};

// W(X, Y) of one channel from the expansions (pairs below a translated
// pair): M2L of A(Y) about c_A(X), dotted with the axon moments M(X).  Whole
// warp; the result is returned to every lane.
__device__ float warp_far_w(const Tree& tr, const Exps& ex, int32_t X, int32_t Y, int ch,
                            float* H, float* b0, float* b1) {
    const int lane = threadIdx.x & 31;
    const int p = ex.p, p2 = p * p, p3 = p2 * p;
    if (X < ex.first || Y < ex.first) return 0.f;
    float4 a = tr.ca[X], d = tr.cd[Y];
    if (lane < 3) {
        float x = (lane == 0 ? a.x - d.x : (lane == 1 ? a.y - d.y : a.z - d.z)) * ex.inv_sigma;
        float* h = H + 16 * lane;
        float h0 = __expf(-x * x);
        h[0] = h0;
        if (2 * p - 2 >= 1) h[1] = 2.f * x * h0;
        for (int k = 1; k < 2 * p - 2; ++k) h[k + 1] = 2.f * x * h[k] - 2.f * (float)k * h[k - 1];
    }
    const float* Ag = ex.A + ((int64_t)(Y - ex.first) * 2 + ch) * p3;
    const float* Mg = ex.M + ((int64_t)(X - ex.first) * 2 + ch) * p3;
    for (int i = lane; i < p3; i += 32) b0[i] = Ag[i];
    __syncwarp();
    for (int o = lane; o < p3; o += 32) {
        int c0 = o / p2, r = o - c0 * p2;
        float s = 0.f;
        for (int k = 0; k < p; ++k) s = fmaf(H[k + c0], b0[k * p2 + r], s);
        b1[o] = s;
    }
    __syncwarp();
    for (int o = lane; o < p3; o += 32) {
        int c0 = o / p2, c1 = (o / p) % p, k2 = o % p;
        float s = 0.f;
        for (int k = 0; k < p; ++k) s = fmaf(H[16 + k + c1], b1[c0 * p2 + k * p + k2], s);
        b0[o] = s;
    }
    __syncwarp();
    float w = 0.f;
    for (int o = lane; o < p3; o += 32) {
        int c0 = o / p2, c1 = (o / p) % p, c2 = o % p;
        float s = 0.f;
        for (int k = 0; k < p; ++k) s = fmaf(H[32 + k + c2], b0[c0 * p2 + c1 * p + k], s);
        float sc = c_inv_fact_sel[c0] * c_inv_fact_sel[c1] * c_inv_fact_sel[c2];
        if ((c0 + c1 + c2) & 1) sc = -sc;
        w = fmaf(s * sc, Mg[o], w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    __syncwarp();
    return w;
}

// Algorithm 2's last steps: negative candidates (truncation) count as zero;
// -1 when the total is at most kMinAttraction; upper_bound over the inclusive
// prefix sums, and the last positive candidate when rounding puts r at the
// total.  The candidates, their prefix sums and r = U * total are double-FP32
// values (hi + lo; the sign of a value is that of hi).
__device__ inline int draw_index(const float2* w, int k, uint64_t bits53) {
    float2 pre[8];
    float2 tot = make_float2(0.f, 0.f);
    for (int i = 0; i < k; ++i) {
        tot = ff_add(tot, w[i].x > 0.f ? w[i] : make_float2(0.f, 0.f));
        pre[i] = tot;
    }
    if (!(tot.x > kMinAttractionF)) return -1;
    const float2 r = ff_mul(ff_uniform(bits53), tot);
    for (int i = 0; i < k; ++i)
        if (ff_gt(pre[i], r)) return i;
    for (int i = k - 1; i >= 0; --i)
        if (w[i].x > 0.f) return i;
    return -1;
}

constexpr int kDescWarps = 4;

// Descent counters of one level step.  The item counts rotate through three
// slots: the step reads its input count from one, appends to the next (zeroed
// by the step before) and zeroes the third for the step after.
struct DescCtr {
    const int64_t* n_in;
    unsigned long long* n_out;
    int64_t* n_reset;
    unsigned long long* n_leaf;
    unsigned long long* draws;
    unsigned long long* overflow;     // bit 1: items, bit 2: leaf items
};

// the items of both channels start at (root, root) where the root has
// vacancies and attraction in that channel
__global__ void k_init_items(const int4* __restrict__ sums, const float4* __restrict__ pw,
                             Item* __restrict__ items, DevCounts* dc) {
    const int4 rs = sums[0];
    const float4 rw = pw[0];
    int64_t k = 0;
    if (rs.x > 0 && rw.x > kMinAttractionF) items[k++] = Item{0, 0, 0, 0};
    if (rs.y > 0 && rw.z > kMinAttractionF) items[k++] = Item{0, 0, 0, 1};
    dc->items[0] = k;
    dc->items[1] = 0;
    dc->n_leaf = 0;
    dc->leaf_next = 0;
    dc->draws = 0;
    dc->overflow &= ~38ll;      // the selection's bits; bit 0 (pair table) stays
}

// One level step of the descent.  A warp takes four items, 8 lanes each
// (lane i of a group for the item's axon child i): a leaf pair goes to the
// per-element draw; a dendrite leaf is kept by every axon child with
// vacancies; otherwise each axon child draws among the children of Y from
// the pair table.  Items below a translated pair (candidates' attractions
// evaluated as translations by the whole warp) follow, one at a time.
__global__ void __launch_bounds__(kDescWarps * 32)
k_descend(const Item* __restrict__ in, Tree tr, Exps ex,
          const uint8_t* __restrict__ kind, const int32_t* __restrict__ pcf,
          const float4* __restrict__ pw, uint64_t seed, StepRef stp, Item* __restrict__ out,
          int64_t cap_out, Item* __restrict__ leaf_out, int64_t cap_leaf, DescCtr ct) {
    const uint64_t step = stp.get();
    __shared__ float sH[kDescWarps][48];
    __shared__ float sb[kDescWarps][2][kMaxP * kMaxP * kMaxP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane & 7;
    // the count may exceed the buffer (items past it were not stored and the
    // overflow bit is set)
    const int64_t n_in = min(*ct.n_in, cap_out);
    if (blockIdx.x == 0 && threadIdx.x == 0) *ct.n_reset = 0;
    const int64_t warp = (int64_t)blockIdx.x * kDescWarps + w;
    const int64_t nwarp = (int64_t)gridDim.x * kDescWarps;
    for (int64_t k0 = 4 * warp; k0 < n_in; k0 += 4 * nwarp) {
        const int64_t k = k0 + (lane >> 3);
        Item it = {0, 0, -1, 0};
        bool far_item = false, drew = false;
        if (k < n_in) {
            it = in[k];
            const int32_t X = it.X, Y = it.Y;
            const int ch = it.ch;
            const bool lx = tr.child_first[X] < 0, ly = tr.child_first[Y] < 0;
            const bool split = it.q >= 0 && kind[it.q] == kSplit;
            const int32_t cf = split ? pcf[it.q] : -1;
            // a split pair whose children did not fit in the pair table (the
            // step is halted and redone with a larger table): nothing to read
            if (split && cf < 0) {
            } else if (lx && ly) {
                // form_synapse: the leaf pair goes to the per-element draw
                if (sub == 0) {
                    const unsigned long long slot = atomicAdd(ct.n_leaf, 1ull);
                    if ((int64_t)slot < cap_leaf) leaf_out[slot] = it;
                    else atomicOr(ct.overflow, 4ull);
                }
            } else if (!lx && ly) {
                // the dendrite side is a leaf: every axon child with vacancies
                // of this channel keeps it, without a draw
                if (sub < tr.nchild[X]) {
                    const int32_t xc = tr.child_first[X] + sub;
                    const int4 sm = tr.sums[xc];
                    bool keep = (ch ? sm.y : sm.x) > 0;
                    if (keep && split)
                        keep = (ch ? pw[cf + sub].z : pw[cf + sub].x) > kMinAttractionF;
                    if (keep) {
                        const unsigned long long slot = atomicAdd(ct.n_out, 1ull);
                        const Item nx_it = {xc, Y, split ? cf + sub : -1, ch};
                        if ((int64_t)slot < cap_out) out[slot] = nx_it;
                        else atomicOr(ct.overflow, 2ull);
                    }
                }
            } else if (split) {
                // a draw among the children of Y, for X itself (X a leaf) or
                // for each axon child of X (both inner); the candidates'
                // attractions are in the pair table
                const int ny = tr.nchild[Y];
                const int32_t cy = tr.child_first[Y];
                const int nsrc = lx ? 1 : tr.nchild[X];
                if (sub < nsrc) {
                    const int32_t xc = lx ? X : tr.child_first[X] + sub;
                    const int4 sm = tr.sums[xc];
                    if (lx || (ch ? sm.y : sm.x) != 0) {
                        float2 wk[8];
                        for (int j = 0; j < ny; ++j) {
                            const float4 v = pw[cf + (int64_t)sub * ny + j];
                            wk[j] = ch ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
                        }
                        const uint32_t c1 = (uint32_t)(tr.level[Y] + 1) | ((uint32_t)ch << 8) |
                                            (kTagDescend << 16);
                        const int kk =
                            draw_index(wk, ny, philox_bits53(seed, (uint32_t)xc, c1, step));
                        drew = true;
                        if (kk >= 0) {
                            const unsigned long long slot = atomicAdd(ct.n_out, 1ull);
                            const Item nx_it = {xc, cy + kk, cf + sub * ny + kk, ch};
                            if ((int64_t)slot < cap_out) out[slot] = nx_it;
                            else atomicOr(ct.overflow, 2ull);
                        }
                    }
                }
            } else {
                far_item = true;
            }
        }
        const unsigned dm = __ballot_sync(0xffffffffu, drew);
        if (lane == 0 && dm) atomicAdd(ct.draws, (unsigned long long)__popc(dm));
        // below a translated pair: each candidate's attraction is a
        // translation the whole warp evaluates
        unsigned fm = __ballot_sync(0xffffffffu, far_item && sub == 0);
        while (fm) {
            const int src = __ffs(fm) - 1;
            fm &= fm - 1;
            const int32_t X = __shfl_sync(0xffffffffu, it.X, src);
            const int32_t Y = __shfl_sync(0xffffffffu, it.Y, src);
            const int ch = __shfl_sync(0xffffffffu, it.ch, src);
            const bool lx = tr.child_first[X] < 0;
            const int ny = tr.nchild[Y];
            const int32_t cy = tr.child_first[Y];
            const int nsrc = lx ? 1 : tr.nchild[X];
            for (int i = 0; i < nsrc; ++i) {
                const int32_t xc = lx ? X : tr.child_first[X] + i;
                if (!lx) {
                    const int4 sm = tr.sums[xc];
                    if ((ch ? sm.y : sm.x) == 0) continue;
                }
                float2 wk[8];
                for (int j = 0; j < ny; ++j)
                    wk[j] = make_float2(
                        warp_far_w(tr, ex, xc, cy + j, ch, sH[w], sb[w][0], sb[w][1]), 0.f);
                if (lane == 0) {
                    const uint32_t c1 = (uint32_t)(tr.level[Y] + 1) | ((uint32_t)ch << 8) |
                                        (kTagDescend << 16);
                    const int kk = draw_index(wk, ny, philox_bits53(seed, (uint32_t)xc, c1, step));
                    atomicAdd(ct.draws, 1ull);
                    if (kk >= 0) {
                        const unsigned long long slot = atomicAdd(ct.n_out, 1ull);
                        const Item nx_it = {xc, cy + kk, -1, ch};
                        if ((int64_t)slot < cap_out) out[slot] = nx_it;
                        else atomicOr(ct.overflow, 2ull);
                    }
                }
                __syncwarp();
            }
        }
    }
}

// Per-element draw inside the chosen dendrite leaf, one warp per leaf pair
// (X, Y, channel) taken from a device work counter: the warp stages Y's
// points with their weights of the channel in shared memory, collects X's
// neurons of that channel with vacant axons, and gives each lane one of them.
// A lane forms the weights w_s K(t,s) of the sources s != t of Y, truncated at
// the cutoff, their total and then the inclusive prefix sums in exact 64-bit
// fixed point (scale 2^shift; a weight is at most 255: integer adds are exact
// and full rate, where double precision adds are scarce on this GPU; weights
// below 2^-shift, far below exp(-cutoff^2) for the cutoffs the library
// accepts, count as zero).  The element draws r_e = floor(U_e tot) (U_e with
// 53 bits) go in groups of up to 8 sorted thresholds; one prefix walk serves
// a group: the first source whose inclusive prefix exceeds r_e.  Leaves of
// more than kLdStage points (possible only where coincident points overfill a
// leaf at the deepest level) read their points from global memory.
constexpr int kLdWarps = 4;
constexpr int kLdStage = 256;
constexpr int kLdBlocks = kLdStage / 32;   // blocks of 32 sources per lane slice

struct LdSrc {
    const float4* sp;      // staged points {x, y, z, w} or null (global memory)
    const float4* pts;
    const float2* wts;
    int32_t sf;
    int ch;
    __device__ float4 get(int j) const {
        if (sp) return sp[j];
        const float4 S = pts[sf + j];
        return make_float4(S.x, S.y, S.z, ch ? wts[sf + j].y : wts[sf + j].x);
    }
};

// floor(v * 2^shift) for a finite 0 <= v < 2^24 (shift <= 40), exact, from the
// bits of v on the integer pipe: a float to 64-bit integer conversion runs on
// the FP64 unit, which is scarce on this GPU
__device__ __forceinline__ uint64_t fixed_point(float v, int shift) {
    const uint32_t b = __float_as_uint(v);
    const int e = (int)(b >> 23);                  // biased exponent (v >= 0)
    if (e == 0) return 0ull;                       // zero or subnormal: below 2^-126
    const uint64_t m = (uint64_t)((b & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + shift;                // v * 2^shift = m * 2^sh
    if (sh >= 0) return m << sh;
    return sh > -24 ? m >> -sh : 0ull;
}

__device__ __forceinline__ uint64_t ld_weight(const float4& T, const float4& S, float k2,
                                              float rc2, int shift) {
    const float dx = T.x - S.x, dy = T.y - S.y, dz = T.z - S.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ws = r2 < rc2 ? S.w * ex2_approx_sel(-r2 * k2) : 0.f;
    return fixed_point(ws, shift);
}

// the weights of two sources at once: the distance, the exponent's argument
// and the scale in paired FP32 (each element rounded as in ld_weight, so the
// totals and the walk see the same values)
__device__ __forceinline__ void ld_weight2(const float4& T, const float4& S0, const float4& S1,
                                           float k2, float rc2, int shift, uint64_t& v0,
                                           uint64_t& v1) {
    const float2 dx = __fadd2_rn(make_float2(T.x, T.x), make_float2(-S0.x, -S1.x));
    const float2 dy = __fadd2_rn(make_float2(T.y, T.y), make_float2(-S0.y, -S1.y));
    const float2 dz = __fadd2_rn(make_float2(T.z, T.z), make_float2(-S0.z, -S1.z));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    const float2 e = __fmul2_rn(make_float2(-r2.x, -r2.y), make_float2(k2, k2));
    const float2 ws =
        __fmul2_rn(make_float2(S0.w, S1.w), make_float2(ex2_approx_sel(e.x), ex2_approx_sel(e.y)));
    v0 = fixed_point(r2.x < rc2 ? ws.x : 0.f, shift);
    v1 = fixed_point(r2.y < rc2 ? ws.y : 0.f, shift);
}

// per-network truncation radii (points in frames with per-network plans):
// the squared radius of the axon leaf's network
struct FrameRc2 {
    const float* rc2;          // per network, or null: the kernel's rc2 everywhere
    const uint64_t* prefix;
    const uint8_t* level;
    int frame_level;
    int64_t nf;
};

__global__ void __launch_bounds__(kLdWarps * 32)
k_leaf_draw_w(const Item* __restrict__ items, const int64_t* __restrict__ n_leaf, int64_t cap_leaf,
              unsigned long long* __restrict__ next, const int32_t* __restrict__ nfirst,
              const int32_t* __restrict__ ncount, const float4* __restrict__ pts,
              const float2* __restrict__ wts, const int32_t* __restrict__ perm,
              const int32_t* __restrict__ eoff, float k2, float rc2_all, FrameRc2 fr,
              uint64_t seed, StepRef stp,
              int32_t* __restrict__ partner, unsigned long long* __restrict__ draw_ctr,
              const int64_t* __restrict__ n_elem) {
    __shared__ float4 s_pts[kLdWarps][kLdStage];
    __shared__ int32_t s_tl[kLdWarps][32];
    __shared__ uint64_t s_bsum[kLdWarps][kLdBlocks][32];   // per lane: sums of 32 sources
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t step = stp.get();
    const int64_t ne = *n_elem;
    const int64_t n_items = min(*n_leaf, cap_leaf);
    unsigned long long draws = 0;
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(next, 1ull);
        k = __shfl_sync(0xffffffffu, k, 0);
        if ((int64_t)k >= n_items) break;
        const Item it = items[k];
        const int ch = it.ch;
        const float rc2 =
            fr.rc2 ? fr.rc2[box_frame(fr.prefix[it.X], fr.level[it.X], fr.frame_level, fr.nf)]
                   : rc2_all;
        const int32_t tf = nfirst[it.X], tc = ncount[it.X];
        const int32_t sf = nfirst[it.Y], sc = ncount[it.Y];
        // fixed-point scale: sc weights of at most 2^8 must stay below 2^63
        int lg = 0;
        while ((1 << lg) < sc + 1 && lg < 30) ++lg;
        const int shift = min(40, 55 - lg);
        LdSrc src{nullptr, pts, wts, sf, ch};
        if (sc <= kLdStage) {
            __syncwarp();
            for (int j = lane; j < sc; j += 32) {
                const float4 S = pts[sf + j];
                s_pts[w][j] = make_float4(S.x, S.y, S.z, ch ? wts[sf + j].y : wts[sf + j].x);
            }
            __syncwarp();
            src.sp = s_pts[w];
        }
        int32_t pos = 0;
        while (pos < tc) {
            // up to 32 of X's neurons of the channel with vacant axons, from pos on
            int nt = 0;
            while (pos < tc && nt < 32) {
                const int32_t tt = tf + pos + lane;
                uint32_t tw = 0;
                if (pos + lane < tc) tw = __float_as_uint(pts[tt].w);
                const bool mine =
                    pos + lane < tc && pk_axon(tw) > 0 && (pk_type(tw) ? 1 : 0) == ch;
                const unsigned mask = __ballot_sync(0xffffffffu, mine);
                const int room = 32 - nt, cnt = __popc(mask);
                const int take = min(cnt, room);
                const int rank = __popc(mask & ((1u << lane) - 1u));
                if (mine && rank < take) s_tl[w][nt + rank] = tt;
                nt += take;
                if (take < cnt) {
                    // continue after the lane of the last target taken
                    pos += (int32_t)__fns(mask, 0, take) + 1;
                    break;
                }
                pos += 32;
            }
            __syncwarp();
            // S lanes per target when the round has few targets (S = 32 / nt,
            // at most 8; TS = nt lanes per slice, the last 32 - S TS lanes idle):
            // lane = q * TS + ti takes target ti and slice q of the sources
            const int TS = nt <= 16 ? max(nt, 1) : 32;
            const int S = nt <= 16 ? min(8, 32 / TS) : 1;
            const int ti = lane % TS, q = lane / TS;
            const bool act = ti < nt && q < S;
            const int32_t t = act ? s_tl[w][ti] : tf;
            __syncwarp();
            const float4 T = pts[t];
            const int a = act ? (int)pk_axon(__float_as_uint(T.w)) : 0;
            const int L = (sc + S - 1) / S;
            const int j0 = min(q * L, sc), j1 = min(j0 + L, sc);
            // the slice's sum, the target's total and the slice's offset
            // (integer sums: exact, the same as one walk over all sources);
            // with at most kLdBlocks blocks of 32 sources per slice the block
            // sums are kept too, so that the walk can skip whole blocks
            const bool use_blocks = L <= 32 * kLdBlocks;
            uint64_t part = 0;
            if (nt > 0) {
                // the sum over sources [ja, jb), two at a time
                auto span = [&](int ja, int jb) {
                    uint64_t sum = 0;
                    int j = ja;
                    for (; j + 1 < jb; j += 2) {
                        uint64_t v0, v1;
                        ld_weight2(T, src.get(j), src.get(j + 1), k2, rc2, shift, v0, v1);
                        sum += (sf + j == t ? 0ull : v0) + (sf + j + 1 == t ? 0ull : v1);
                    }
                    if (j < jb) {
                        const uint64_t v = ld_weight(T, src.get(j), k2, rc2, shift);
                        sum += sf + j == t ? 0ull : v;
                    }
                    return sum;
                };
                if (use_blocks) {
                    for (int b = 0; j0 + 32 * b < j1; ++b) {
                        const uint64_t bsum = span(j0 + 32 * b, min(j1, j0 + 32 * b + 32));
                        s_bsum[w][b][lane] = bsum;
                        part += bsum;
                    }
                } else {
                    part = span(j0, j1);
                }
            }
            // inclusive scan of the slices' sums over q (offsets TS, 2 TS, ...;
            // a lane reads only from lanes of the same target below it), the
            // target's total from its last slice
            uint64_t incl = part;
            for (int o = TS; o < S * TS; o <<= 1) {
                const uint64_t up = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += up;
            }
            const uint64_t tot = __shfl_sync(0xffffffffu, incl, (S - 1) * TS + ti);
            const uint64_t off = incl - part;
            const int32_t to = perm[t];
            const bool draw = act && tot != 0 && (int64_t)eoff[to] + a <= ne;
            constexpr int kGroup = 8;
            const int groups = draw ? (a + kGroup - 1) / kGroup : 0;
            const int gmax = __reduce_max_sync(0xffffffffu, groups);
            for (int gi = 0; gi < gmax; ++gi) {
                const int e0 = gi * kGroup;
                const int ng = gi < groups ? min(kGroup, a - e0) : 0;
                uint64_t r[kGroup];
                int ord[kGroup];
                for (int e = 0; e < ng; ++e) {
                    uint32_t c1 = (uint32_t)(e0 + e) | ((uint32_t)ch << 8) | (kTagLeaf << 16);
                    uint32_t o4[4];
                    philox_draw(seed, (uint32_t)to, c1, step, o4);
                    uint64_t u53 = (((uint64_t)o4[0] << 32) | o4[1]) >> 11;
                    uint64_t v = __umul64hi(u53 << 11, tot);     // floor(u53 * tot / 2^53)
                    int jj = e;
                    while (jj > 0 && r[jj - 1] > v) {
                        r[jj] = r[jj - 1];
                        ord[jj] = ord[jj - 1];
                        --jj;
                    }
                    r[jj] = v;
                    ord[jj] = e;
                }
                // this slice owns the thresholds in [off, off + part): the
                // first source whose inclusive prefix exceeds a threshold
                // lies in the slice whose prefix range contains it
                int nx = 0;
                while (nx < ng && r[nx] < off) ++nx;
                int nend = nx;
                while (nend < ng && r[nend] < off + part) ++nend;
                uint64_t pre = off;
                if (use_blocks) {
                    // from the block holding the next threshold (the blocks
                    // before it are skipped by their sums), source by source;
                    // at most L evaluations, the warp voting in each
                    int b = 0, j = j0;
                    uint64_t cb = off;          // prefix before block b
                    bool placed = false;
                    for (int it = 0; it < L; ++it) {
                        if (!__any_sync(0xffffffffu, nx < nend)) break;
                        if (nx < nend) {
                            if (!placed) {
                                while (cb + s_bsum[w][b][lane] <= r[nx]) {
                                    cb += s_bsum[w][b][lane];
                                    ++b;
                                }
                                j = j0 + 32 * b;
                                pre = cb;
                                placed = true;
                            }
                            const uint64_t v = ld_weight(T, src.get(j), k2, rc2, shift);
                            pre += sf + j == t ? 0ull : v;
                            while (nx < nend && pre > r[nx]) {
                                partner[eoff[to] + e0 + ord[nx]] = perm[sf + j];
                                ++draws;
                                ++nx;
                            }
                            ++j;
                            // the next threshold beyond this block: skip again
                            if (nx < nend && r[nx] >= cb + s_bsum[w][b][lane]) {
                                cb += s_bsum[w][b][lane];
                                ++b;
                                placed = false;
                            }
                        }
                    }
                } else {
                    // every lane runs the same L iterations (the warp votes in each)
                    for (int jj = 0; jj < L; ++jj) {
                        const int j = j0 + jj;
                        if (!__any_sync(0xffffffffu, nx < nend && j < j1)) break;
                        if (nx < nend && j < j1) {
                            const uint64_t v = ld_weight(T, src.get(j), k2, rc2, shift);
                            pre += sf + j == t ? 0ull : v;
                            while (nx < nend && pre > r[nx]) {
                                partner[eoff[to] + e0 + ord[nx]] = perm[sf + j];
                                ++draws;
                                ++nx;
                            }
                        }
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) draws += __shfl_xor_sync(0xffffffffu, draws, o);
    if (lane == 0 && draws) atomicAdd(draw_ctr, draws);
}

// a12: the requests grouped by (channel, dendrite), group g = channel * n +
// dendrite, by a counting sort: counts per group, their exclusive scan, and a
// scatter that takes each request's slot from its group's count (counting it
// back down to zero).  The order inside a group is left to the atomics; the
// ranking below does not depend on it.
__global__ void k_req_count(int64_t n, const uint8_t* __restrict__ type,
                            const uint8_t* __restrict__ va, const int32_t* __restrict__ eoff,
                            const int32_t* __restrict__ partner, int32_t* __restrict__ gcnt,
                            const int64_t* __restrict__ n_elem, int64_t* __restrict__ n_groups) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_groups = 2 * n;
    const int64_t ne = *n_elem;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = va[t];
        const int32_t e0 = eoff[t];
        if ((int64_t)e0 + a > ne) continue;
        const int64_t base = type[t] ? n : 0;
        for (int k = 0; k < a; ++k) {
            const int32_t s = partner[e0 + k];
            if (s >= 0) atomicAdd(&gcnt[base + s], 1);
        }
    }
}

// key = priority << 32 | group, val = element; cap bounds the slots (the
// buffers' length): a slot outside it (counts that do not match) is not
// written and sets bit 5 of *overflow
__global__ void k_req_scatter(int64_t n, const uint8_t* __restrict__ type,
                              const uint8_t* __restrict__ va, const int32_t* __restrict__ eoff,
                              const int32_t* __restrict__ partner, const int32_t* __restrict__ goff,
                              int32_t* __restrict__ gcnt, uint64_t seed, StepRef stp,
                              uint64_t* __restrict__ key, int32_t* __restrict__ val,
                              const int64_t* __restrict__ n_elem, int64_t cap,
                              int64_t* __restrict__ overflow) {
    const uint64_t step = stp.get();
    const int64_t ne = *n_elem;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = va[t];
        const int32_t e0 = eoff[t];
        if ((int64_t)e0 + a > ne) continue;
        const int64_t base = type[t] ? n : 0;
        for (int k = 0; k < a; ++k) {
            const int32_t s = partner[e0 + k];
            if (s < 0) continue;
            uint32_t o[4];
            philox_draw(seed, (uint32_t)t, (uint32_t)k | (kTagAccept << 16), step, o);
            const int64_t g = base + s;
            const int64_t r = (int64_t)goff[g] + atomicSub(&gcnt[g], 1) - 1;
            if (r < 0 || r >= cap) {
                atomicOr(reinterpret_cast<unsigned long long*>(overflow), 32ull);
                continue;
            }
            key[r] = ((uint64_t)o[0] << 32) | (uint32_t)g;
            val[r] = e0 + k;
        }
    }
}

// A dendrite neuron accepts, per channel, its first `capacity` requests in
// (priority, element) order: the rank of request i is the number of requests
// of its group before it in that order.  Groups are small (the requests one
// neuron receives), so each request counts over its group directly.  A group
// whose count the scatter did not bring back to zero sets bit 5 of *overflow.
__global__ void k_accept(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                         const int32_t* __restrict__ goff, const int32_t* __restrict__ gcnt,
                         const int64_t* __restrict__ nr_dev, int64_t n,
                         const uint8_t* __restrict__ vde, const uint8_t* __restrict__ vdi,
                         uint8_t* __restrict__ accepted, int64_t* __restrict__ overflow) {
    const int64_t nr = *nr_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ki = key[i];
        const int64_t g = (int64_t)(uint32_t)ki;
        const uint32_t pr = (uint32_t)(ki >> 32);
        const int32_t ei = val[i];
        const bool inh = g >= n;
        const int64_t s = inh ? g - n : g;
        const int cap = inh ? vdi[s] : vde[s];
        if (gcnt[g] != 0) atomicOr(reinterpret_cast<unsigned long long*>(overflow), 32ull);
        const int64_t j0 = goff[g], j1 = g + 1 < 2 * n ? (int64_t)goff[g + 1] : nr;
        int rank = 0;
        for (int64_t j = j0; j < j1 && rank < cap; ++j) {
            const uint32_t pj = (uint32_t)(key[j] >> 32);
            rank += pj < pr || (pj == pr && val[j] < ei);
        }
        accepted[ei] = rank < cap ? 1 : 0;
    }
}

__global__ void k_acc_flags(const uint8_t* __restrict__ acc, const int64_t* __restrict__ n_dev,
                            int32_t* __restrict__ flag) {
    const int64_t n_elem = *n_dev;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elem;
         e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = acc[e];
}

__global__ void k_emit_synapses(int64_t n, const uint8_t* __restrict__ type,
                                const uint8_t* __restrict__ va, const int32_t* __restrict__ eoff,
                                const int32_t* __restrict__ partner,
                                const uint8_t* __restrict__ acc, const int32_t* __restrict__ soff,
                                int32_t* __restrict__ pre, int32_t* __restrict__ post,
                                uint8_t* __restrict__ styp, const int64_t* __restrict__ n_elem) {
    const int64_t ne = *n_elem;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int a = va[t];
        int32_t e0 = eoff[t];
        if ((int64_t)e0 + a > ne) continue;
        for (int k = 0; k < a; ++k) {
            if (!acc[e0 + k]) continue;
            int32_t r = soff[e0 + k];
            pre[r] = (int32_t)t;
            post[r] = partner[e0 + k];
            styp[r] = type[t] ? 1 : 0;
        }
    }
}

__global__ void k_walk(int64_t n, uint64_t seed, StepRef stp, uint8_t* __restrict__ va,
                       uint8_t* __restrict__ vde, uint8_t* __restrict__ vdi,
                       const int64_t* __restrict__ halt) {
    if (halt && *halt) return;
    const uint64_t step = stp.get();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint8_t* v[3] = {va, vde, vdi};
        for (int ch = 0; ch < 3; ++ch) {
            uint32_t o[4];
            philox_draw(seed, (uint32_t)i, (uint32_t)ch | (kTagWalk << 16), step, o);
            int nv = (int)v[ch][i] + ((o[0] & 1u) ? 1 : -1);
            nv = nv < 0 ? 0 : (nv > kMaxVacancy ? kMaxVacancy : nv);
            v[ch][i] = (uint8_t)nv;
        }
    }
}

__device__ inline void sat_dec(uint8_t* p) {
    // byte-wise saturating decrement through the containing 32-bit word
    uintptr_t addr = reinterpret_cast<uintptr_t>(p);
    unsigned int* word = reinterpret_cast<unsigned int*>(addr & ~uintptr_t(3));
    unsigned int sh = (unsigned int)(addr & 3u) * 8u;
    unsigned int old = *word, assumed;
    do {
        assumed = old;
        unsigned int b = (assumed >> sh) & 0xffu;
        if (b == 0) return;
        old = atomicCAS(word, assumed, assumed - (1u << sh));
    } while (old != assumed);
}

__global__ void k_commit(const int64_t* __restrict__ n_syn, int64_t capacity,
                         const int32_t* __restrict__ pre, const int32_t* __restrict__ post,
                         const uint8_t* __restrict__ styp, uint8_t* va, uint8_t* vde, uint8_t* vdi,
                         const int64_t* __restrict__ halt) {
    if (halt && *halt) return;
    int64_t m = *n_syn;
    if (m > capacity) m = capacity;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        sat_dec(va + pre[k]);
        sat_dec((styp[k] ? vdi : vde) + post[k]);
    }
}

__global__ void k_fill_i32(int32_t* __restrict__ p, const int64_t* __restrict__ n_dev, int32_t v) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

void select_partners(msp_ctx& c, uint64_t step, const uint8_t* type_dev, const uint8_t* va_dev,
                     const uint8_t* vde_dev, const uint8_t* vdi_dev, int32_t* partner,
                     int32_t* syn_pre, int32_t* syn_post, uint8_t* syn_type, int64_t* n_syn,
                     cudaStream_t s) {
    NvtxRange nv_("msp select_partners");
    if (!c.attraction_done) throw Error(MSP_ERR_NOT_BUILT, "msp_attraction must run first");
    const msp_config& cfg = c.cfg;
    // the element count: exact from the build, or (whole-step graph) the
    // capacity of its buffers (the vacancy walk's bound, or the host-buffer
    // call's); kernels read the exact count from device memory and never
    // index past it
    const int64_t n = c.n, ne = c.graph_mode ? c.graph_elem_cap : c.n_elem;
    const int B = 256;
    const float k2 = (float)(1.4426950408889634 / (cfg.sigma * cfg.sigma));
    // inside a leaf the kernel is truncated at the radius that prunes box pairs
    const float rc2 = (float)((cfg.cutoff * cfg.sigma) * (cfg.cutoff * cfg.sigma));
    c.n_draws = c.n_requests = c.n_synapses = 0;
    if (ne == 0) {
        MSP_CUDA(cudaMemsetAsync(n_syn, 0, sizeof(int64_t), s));
        if (!c.graph_mode) MSP_CUDA(cudaStreamSynchronize(s));
        return;
    }
    DevCounts* dc = dcounts(c);
    const StepRef stp{step, c.graph_mode ? &dc->step : nullptr};
    const int ge = grid_for(ne, B, (int64_t)c.sm_count * 16);
    k_fill_i32<<<ge, B, 0, s>>>(partner, &dc->n_elem, -1);
    MSP_LAUNCH("fill_partner");

    Tree tr;
    tr.level = c.nd_level.get<uint8_t>();
    tr.first = c.nd_first.get<int32_t>();
    tr.count = c.nd_count.get<int32_t>();
    tr.child_first = c.nd_child_first.get<int32_t>();
    tr.nchild = c.nd_nchild.get<uint8_t>();
    tr.sums = c.nd_sums.get<int4>();
    // expansion centres (the geometric ones with centre_mode 1)
    tr.ca = c.cfg.centre_mode == 1 ? c.nd_gc.get<float4>() : c.nd_ca.get<float4>();
    tr.cd = c.cfg.centre_mode == 1 ? c.nd_gc.get<float4>() : c.nd_cd.get<float4>();
    Exps ex;
    ex.A = c.expA.get<float>();
    ex.M = c.expM.get<float>();
    ex.first = c.exp_first;
    ex.p = cfg.p;
    ex.inv_sigma = (float)(1.0 / cfg.sigma);

    // a11: the level steps of the descent.  At step k every inner box of an
    // item is at level k (inner boxes always go one level down; a leaf stays),
    // and an item of two leaves goes to the per-element draw, so depth + 1
    // steps empty the item list.
    const int64_t cap_items = 2 * c.n_nodes + 64, cap_leaf = 2 * c.n_nodes + 64;
    Item* ib[2] = {c.items0.ensure<Item>((size_t)cap_items), c.items1.ensure<Item>((size_t)cap_items)};
    Item* lit = c.leaf_items.ensure<Item>((size_t)cap_leaf);
    k_init_items<<<1, 1, 0, s>>>(c.nd_sums.get<int4>(), c.pr_w.get<float4>(), ib[0], dc);
    MSP_LAUNCH("init_items");
    auto ull = [](int64_t* p) { return reinterpret_cast<unsigned long long*>(p); };
    const int n_steps = c.tree_depth + 1;
    const int gd = (int)std::max<int64_t>(1, (int64_t)c.sm_count * 16);
    for (int k = 0; k < n_steps; ++k) {
        DescCtr ct;
        ct.n_in = &dc->items[k % 3];
        ct.n_out = ull(&dc->items[(k + 1) % 3]);
        ct.n_reset = &dc->items[(k + 2) % 3];
        ct.n_leaf = ull(&dc->n_leaf);
        ct.draws = ull(&dc->draws);
        ct.overflow = ull(&dc->overflow);
        k_descend<<<gd, kDescWarps * 32, 0, s>>>(ib[k & 1], tr, ex, c.pr_kind.get<uint8_t>(),
                                                 c.pr_cf.get<int32_t>(), c.pr_w.get<float4>(),
                                                 cfg.seed, stp, ib[(k + 1) & 1], cap_items, lit,
                                                 cap_leaf, ct);
        MSP_LAUNCH("descend");
    }
    // one warp per leaf pair, from a device work counter
    FrameRc2 frc{nullptr, c.nd_prefix.get<uint64_t>(), c.nd_level.get<uint8_t>(), c.frame_level,
                 (int64_t)c.frame_off_host.size() - 1};
    if (c.frame_level > 0 && c.frame_plans) frc.rc2 = c.frame_rc2.get<float>();
    k_leaf_draw_w<<<(int)std::max<int64_t>(1, (int64_t)c.sm_count * 8), kLdWarps * 32, 0, s>>>(
        lit, &dc->n_leaf, cap_leaf, ull(&dc->leaf_next), c.nd_first.get<int32_t>(),
        c.nd_count.get<int32_t>(), c.pts.get<float4>(), c.wts.get<float2>(),
        c.perm.get<int32_t>(), c.elem_off.get<int32_t>(), k2, rc2, frc, cfg.seed, stp, partner,
        ull(&dc->draws), &dc->n_elem);
    MSP_LAUNCH("leaf_draw");

    // a12: requests grouped by (channel, dendrite), ranked by (priority, element)
    int32_t* flag = c.cnt.ensure<int32_t>((size_t)ne);
    const int gn = grid_for(n, B, (int64_t)c.sm_count * 16);
    const size_t ng = (size_t)std::max<int64_t>(2 * n, 1);
    // the group counts: cleared before an eager selection and whenever the
    // buffer is new; every complete scatter counts them back down to zero
    const size_t gcnt_bytes = c.rq_gcnt.bytes;
    int32_t* gcnt = c.rq_gcnt.ensure<int32_t>(ng);
    if (!c.graph_mode || c.rq_gcnt.bytes != gcnt_bytes)
        MSP_CUDA(cudaMemsetAsync(gcnt, 0, c.rq_gcnt.bytes, s));
    int32_t* goff = c.rq_goff.ensure<int32_t>(ng);
    uint8_t* acc = c.accepted.ensure<uint8_t>((size_t)ne);
    MSP_CUDA(cudaMemsetAsync(acc, 0, (size_t)ne, s));
    uint64_t* k0 = c.rq_key0.ensure<uint64_t>((size_t)ne);
    int32_t* v0 = c.rq_val0.ensure<int32_t>((size_t)ne);
    k_req_count<<<gn, B, 0, s>>>(n, type_dev, va_dev, c.elem_off.get<int32_t>(), partner, gcnt,
                                 &dc->n_elem, &dc->n_groups);
    MSP_LAUNCH("req_count");
    scan_dev(c, gcnt, goff, &dc->n_groups, (int64_t)ng, &dc->n_req, nullptr, s);
    k_req_scatter<<<gn, B, 0, s>>>(n, type_dev, va_dev, c.elem_off.get<int32_t>(), partner, goff,
                                   gcnt, cfg.seed, stp, k0, v0, &dc->n_elem, (int64_t)ne,
                                   &dc->overflow);
    MSP_LAUNCH("req_scatter");
    k_accept<<<ge, B, 0, s>>>(k0, v0, goff, gcnt, &dc->n_req, n, vde_dev, vdi_dev, acc,
                              &dc->overflow);
    MSP_LAUNCH("accept");
    k_acc_flags<<<ge, B, 0, s>>>(acc, &dc->n_elem, flag);
    MSP_LAUNCH("acc_flags");
    int32_t* soff = c.acc_off.ensure<int32_t>((size_t)ne);
    scan_dev(c, flag, soff, &dc->n_elem, ne, &dc->n_syn, nullptr, s);
    k_emit_synapses<<<gn, B, 0, s>>>(n, type_dev, va_dev, c.elem_off.get<int32_t>(), partner, acc,
                                     soff, syn_pre, syn_post, syn_type, &dc->n_elem);
    MSP_LAUNCH("emit_synapses");
    MSP_CUDA(cudaMemcpyAsync(n_syn, &dc->n_syn, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (c.graph_mode) {
        // checked on the device at the end of the graph's step
        c.cap_left_slot = n_steps % 3;
        return;
    }
    pull_counts(c, s);              // the one synchronisation of the selection
    const DevCounts& hc = *c.hcount;
    if (hc.overflow & 6) throw Error(MSP_ERR_CHECK, "descent item capacity exceeded");
    if (hc.overflow & 32) throw Error(MSP_ERR_CHECK, "request groups inconsistent");
    if (hc.items[n_steps % 3] != 0) throw Error(MSP_ERR_CHECK, "descent did not terminate");
    c.n_draws = hc.draws;
    c.n_requests = hc.n_req;
    c.n_synapses = hc.n_syn;
}

void vacancy_walk(msp_ctx& c, int64_t n, uint64_t step, uint8_t* va, uint8_t* vde, uint8_t* vdi,
                  cudaStream_t s) {
    if (n <= 0) return;
    DevCounts* dc = dcounts(c);
    const StepRef stp{step, c.graph_mode ? &dc->step : nullptr};
    k_walk<<<grid_for(n, 256, (int64_t)c.sm_count * 16), 256, 0, s>>>(
        n, c.cfg.seed, stp, va, vde, vdi, c.graph_mode ? &dc->halt : nullptr);
    MSP_LAUNCH("walk");
}

void commit_synapses(msp_ctx& c, const int64_t* n_syn, int64_t capacity, const int32_t* pre,
                     const int32_t* post, const uint8_t* styp, uint8_t* va, uint8_t* vde,
                     uint8_t* vdi, cudaStream_t s) {
    if (capacity <= 0) return;
    k_commit<<<grid_for(capacity, 256, (int64_t)c.sm_count * 16), 256, 0, s>>>(
        n_syn, capacity, pre, post, styp, va, vde, vdi,
        c.graph_mode ? &dcounts(c)->halt : nullptr);
    MSP_LAUNCH("commit");
}

}  // namespace msp
