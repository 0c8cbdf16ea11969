// msp_grad.cu -- derivatives of the attraction (Eq. 8), the adjoint of the
// near field: with K(t,s) = exp(-r^2/sigma^2) = 2^-q, q = r^2 log2(e)/sigma^2,
//   u(t)      = sum_{s != t} w_s^{T(t)} K                        (a_t > 0)
//   du/dsigma = sum_{s != t} w_s^{T(t)} K 2 r^2 / sigma^3
//             = (2 / (sigma log2 e)) sum_{s != t} w_s^{T(t)} q 2^-q
//   dL/dw^T_s = sum_{t != s, a_t > 0, T(t) = T} g_t K(t,s)   for L = sum_t g_t u(t)
// summed over the near-field leaf pairs of the last attraction (a plan
// without translated pairs), at counts the caller passes (the tree's own
// counts only chose the pairs).  The forward sums run one block per target
// leaf over the pair list sorted by target leaf; the transposed sums regroup
// the same pairs by source leaf (a radix sort), one block per source leaf;
// both stage the partner leaves' points in shared memory.
// Every sum has a fixed order: the results are reproducible.  The distance
// is formed as a difference (no expanded form), in single precision.
#include <algorithm>
#include <cmath>

#include "msp_internal.cuh"

namespace msp {

namespace {

__device__ inline float gr_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sorted-order weights: {w^E, w^I, g [a > 0], bit 0 type | bit 1 a > 0}
__global__ void k_grad_gather(int64_t n, const int32_t* __restrict__ perm,
                              const uint8_t* __restrict__ type, const uint8_t* __restrict__ va,
                              const uint8_t* __restrict__ vde, const uint8_t* __restrict__ vdi,
                              const float* __restrict__ g, float4* __restrict__ gw) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = perm[s];
        const bool act = va[c] > 0;
        const uint32_t flags = (type[c] ? 1u : 0u) | (act ? 2u : 0u);
        gw[s] = make_float4((float)vde[c], (float)vdi[c], (g && act) ? g[c] : 0.f,
                            __uint_as_float(flags));
    }
}

constexpr int kGrWarps = 4;
constexpr int kGrStage = 64;
constexpr int kGrList = 64;    // evaluation points per pass (two per lane)

// A staged pair of sources against one evaluation point t, whose scaled
// coordinates are broadcast into both halves of register pairs; every step is
// a paired FP32 instruction (two results, one issue slot) with the
// per-element rounding of the scalar form: dx = t - s (s is staged negated),
// q = fma(dx, dx, fma(dy, dy, dz dz)), K = 2^-q.  Staged pair j (sources
// 2j, 2j + 1): A = (-x0, -x1, -y0, -y1), B = (-z0, -z1, w0_0, w0_1),
// C = (w1_0, w1_1, index0, index1); a padding source has zero weights and
// index -1.  SELF: a source may be t itself (sorted index e); its term is zero.
template <bool FORWARD, bool SELF>
__device__ __forceinline__ void gr_term(const float4 A, const float4 B, const float4 C,
                                        float2 tx, float2 ty, float2 tz, bool inh, int32_t e,
                                        float2& a0, float2& a1) {
    const float2 dx = __fadd2_rn(tx, make_float2(A.x, A.y));
    const float2 dy = __fadd2_rn(ty, make_float2(A.z, A.w));
    const float2 dz = __fadd2_rn(tz, make_float2(B.x, B.y));
    const float2 q = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    float2 ex = make_float2(gr_ex2(-q.x), gr_ex2(-q.y));
    if (SELF) {
        ex.x = __float_as_int(C.z) == e ? 0.f : ex.x;
        ex.y = __float_as_int(C.w) == e ? 0.f : ex.y;
    }
    if (FORWARD) {
        const float2 wk = __fmul2_rn(inh ? make_float2(C.x, C.y) : make_float2(B.z, B.w), ex);
        a0 = __fadd2_rn(a0, wk);
        a1 = __ffma2_rn(wk, q, a1);
    } else {
        a0 = __ffma2_rn(make_float2(B.z, B.w), ex, a0);
        a1 = __ffma2_rn(make_float2(C.x, C.y), ex, a1);
    }
}

// The staged pairs [0, mp) against the lane's first point, and its second
// point too when NP = 2.
template <bool FORWARD, bool SELF, int NP>
__device__ __forceinline__ void gr_eval(const float4* sA, const float4* sB, const float4* sC,
                                        int mp, float2 tx0, float2 ty0, float2 tz0, float2 tx1,
                                        float2 ty1, float2 tz1, bool inh0, bool inh1, int32_t e0,
                                        int32_t e1, float2& a00, float2& a10, float2& a01,
                                        float2& a11) {
#pragma unroll 2
    for (int j = 0; j < mp; ++j) {
        const float4 A = sA[j], B = sB[j], C = sC[j];
        gr_term<FORWARD, SELF>(A, B, C, tx0, ty0, tz0, inh0, e0, a00, a10);
        if (NP == 2) gr_term<FORWARD, SELF>(A, B, C, tx1, ty1, tz1, inh1, e1, a01, a11);
    }
}

// One block per leaf L of a segment list (the evaluation leaf), its 4 warps
// taking the segment's partner leaves P round-robin.  Warp 0 lists L's
// evaluation points, up to 64 per pass (FORWARD: the targets, a_t > 0;
// ADJOINT: every point); each lane holds two of them (lane, lane + 32).  Each
// warp stages P's points in shared memory, 64 at a time in pairs, as scaled
// positions sqrt(k2) (x - o) relative to a point o of L, and two weights, and
// every lane sums over the staged pairs, q = |t^ - s^|^2 and 2^-q in single
// precision, the even and the odd sources of a point in the two halves of a
// register pair.  The 4 warps' sums are added in a fixed order, so a point's
// sum does not depend on how the points are packed into passes.
//   FORWARD: evaluation points = targets t (a_t > 0), partner weights
//            (w^E, w^I): u += w^{T(t)} 2^-q, d += w^{T(t)} q 2^-q.
//   ADJOINT: evaluation points = sources s, partner weights
//            (g_t [T(t) = E], g_t [T(t) = I]) (0 unless a_t > 0):
//            gE += w0 2^-q, gI += w1 2^-q.
// Points that are not evaluated keep the zero the caller wrote.  Six blocks
// per SM (at most 80 registers: the unrolled paired loop spills below that).
template <bool FORWARD>
__global__ void __launch_bounds__(kGrWarps * 32, 6)
k_grad_pairs(const int32_t* __restrict__ seg_first, const int64_t* __restrict__ nseg_dev,
             const int32_t* __restrict__ pairs, const int32_t* __restrict__ pEval,
             const int32_t* __restrict__ pPart, const int32_t* __restrict__ nfirst,
             const int32_t* __restrict__ ncount, const float4* __restrict__ pts,
             const float4* __restrict__ gw, const int32_t* __restrict__ perm, float sqk,
             float dscale, float* __restrict__ out0, float* __restrict__ out1) {
    __shared__ float4 sA[kGrWarps][kGrStage / 2], sB[kGrWarps][kGrStage / 2],
        sC[kGrWarps][kGrStage / 2];
    __shared__ float red[kGrWarps][2][kGrList];
    __shared__ int32_t plist[kGrList];
    __shared__ int s_np, s_pos;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nseg = *nseg_dev;
    for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const int32_t i0 = seg_first[sg], i1 = seg_first[sg + 1];
        const int32_t L = pEval[pairs[i0]];
        const int32_t lf = nfirst[L], lc = ncount[L];
        // positions relative to a point of L before scaling: small operands,
        // so the differences keep their precision
        const float4 O = pts[lf];
        int32_t pos = 0;
        for (;;) {
            if (w == 0) {
                // the next (at most) kGrList evaluation points from pos on
                int np = 0;
                int32_t p = pos;
                while (p < lc && np < kGrList) {
                    const int32_t idx = p + lane;
                    bool ok = idx < lc;
                    if (FORWARD && ok) ok = (__float_as_uint(gw[lf + idx].w) & 2u) != 0;
                    const unsigned mk = __ballot_sync(0xffffffffu, ok);
                    const int room = kGrList - np;
                    const int rank = __popc(mk & ((1u << lane) - 1u));
                    if (ok && rank < room) plist[np + rank] = lf + idx;
                    if (__popc(mk) > room) {
                        // the room-th point ends the pass: resume after it
                        unsigned keep = mk;
                        for (int k = 0; k < room; ++k) keep &= keep - 1u;
                        p += __ffs(keep) - 1;
                        np = kGrList;
                        break;
                    }
                    np += __popc(mk);
                    p += 32;
                }
                if (lane == 0) {
                    s_np = np;
                    s_pos = min(p, lc);
                }
            }
            __syncthreads();
            const int np = s_np;
            pos = s_pos;
            __syncthreads();
            if (np == 0) break;
            const bool v0 = lane < np, v1 = lane + 32 < np;
            const int32_t e0 = v0 ? plist[lane] : -1, e1 = v1 ? plist[lane + 32] : -1;
            const float4 T0 = pts[v0 ? e0 : plist[0]], T1 = pts[v1 ? e1 : plist[0]];
            const bool inh0 = __float_as_uint(gw[v0 ? e0 : plist[0]].w) & 1u;
            const bool inh1 = __float_as_uint(gw[v1 ? e1 : plist[0]].w) & 1u;
            const float x0 = (T0.x - O.x) * sqk, y0 = (T0.y - O.y) * sqk, z0 = (T0.z - O.z) * sqk;
            const float x1 = (T1.x - O.x) * sqk, y1 = (T1.y - O.y) * sqk, z1 = (T1.z - O.z) * sqk;
            const float2 tx0 = make_float2(x0, x0), ty0 = make_float2(y0, y0),
                         tz0 = make_float2(z0, z0);
            const float2 tx1 = make_float2(x1, x1), ty1 = make_float2(y1, y1),
                         tz1 = make_float2(z1, z1);
            float2 a00 = make_float2(0.f, 0.f), a10 = make_float2(0.f, 0.f);
            float2 a01 = make_float2(0.f, 0.f), a11 = make_float2(0.f, 0.f);
            for (int32_t i = i0 + w; i < i1; i += kGrWarps) {
                const int32_t P = pPart[pairs[i]];
                const int32_t pf = nfirst[P], pc = ncount[P];
                for (int32_t sb = 0; sb < pc; sb += kGrStage) {
                    const int m = min(kGrStage, pc - sb);
                    const int mp = (m + 1) >> 1;
                    __syncwarp();
                    float* fA = reinterpret_cast<float*>(sA[w]);
                    float* fB = reinterpret_cast<float*>(sB[w]);
                    float* fC = reinterpret_cast<float*>(sC[w]);
                    for (int k = lane; k < 2 * mp; k += 32) {
                        float sx = 0.f, sy = 0.f, sz = 0.f, w0 = 0.f, w1 = 0.f;
                        int32_t si = -1;
                        if (k < m) {
                            const float4 S = pts[pf + sb + k];
                            const float4 W = gw[pf + sb + k];
                            sx = (S.x - O.x) * sqk;
                            sy = (S.y - O.y) * sqk;
                            sz = (S.z - O.z) * sqk;
                            if (FORWARD) {
                                w0 = W.x;
                                w1 = W.y;
                            } else {
                                const uint32_t f2 = __float_as_uint(W.w);
                                const float gv = (f2 & 2u) ? W.z : 0.f;
                                w0 = (f2 & 1u) ? 0.f : gv;
                                w1 = (f2 & 1u) ? gv : 0.f;
                            }
                            si = pf + sb + k;
                        }
                        const int j = k >> 1, h = k & 1;
                        fA[4 * j + h] = -sx;
                        fA[4 * j + 2 + h] = -sy;
                        fB[4 * j + h] = -sz;
                        fB[4 * j + 2 + h] = w0;
                        fC[4 * j + h] = w1;
                        fC[4 * j + 2 + h] = __int_as_float(si);
                    }
                    __syncwarp();
                    if (v0) {
                        // the second point of the lanes only while the pass
                        // has more than 32 points
                        if (np > 32) {
                            if (P == L)
                                gr_eval<FORWARD, true, 2>(sA[w], sB[w], sC[w], mp, tx0, ty0, tz0,
                                                          tx1, ty1, tz1, inh0, inh1, e0, e1, a00,
                                                          a10, a01, a11);
                            else
                                gr_eval<FORWARD, false, 2>(sA[w], sB[w], sC[w], mp, tx0, ty0, tz0,
                                                           tx1, ty1, tz1, inh0, inh1, e0, e1,
                                                           a00, a10, a01, a11);
                        } else {
                            if (P == L)
                                gr_eval<FORWARD, true, 1>(sA[w], sB[w], sC[w], mp, tx0, ty0, tz0,
                                                          tx1, ty1, tz1, inh0, inh1, e0, e1, a00,
                                                          a10, a01, a11);
                            else
                                gr_eval<FORWARD, false, 1>(sA[w], sB[w], sC[w], mp, tx0, ty0, tz0,
                                                           tx1, ty1, tz1, inh0, inh1, e0, e1,
                                                           a00, a10, a01, a11);
                        }
                    }
                }
            }
            red[w][0][lane] = a00.x + a00.y;
            red[w][0][lane + 32] = a01.x + a01.y;
            red[w][1][lane] = a10.x + a10.y;
            red[w][1][lane + 32] = a11.x + a11.y;
            __syncthreads();
            if (w == 0) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int j = lane + 32 * r;
                    if (j >= np) continue;
                    float s0 = red[0][0][j], s1 = red[0][1][j];
#pragma unroll
                    for (int k = 1; k < kGrWarps; ++k) {
                        s0 += red[k][0][j];
                        s1 += red[k][1][j];
                    }
                    const int32_t c = perm[plist[j]];
                    if (FORWARD) {
                        if (out0) out0[c] = s0;
                        if (out1) out1[c] = s1 * dscale;
                    } else {
                        out0[c] = s0;
                        out1[c] = s1;
                    }
                }
            }
            __syncthreads();
            if (pos >= lc) break;
        }
    }
}

// pair list regrouped by source leaf: key = source leaf, value = pair index
__global__ void k_grad_keys(const int32_t* __restrict__ list_q, const int64_t* __restrict__ n_dev,
                            const int32_t* __restrict__ pY, uint64_t* __restrict__ key,
                            int32_t* __restrict__ val) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = list_q[i];
        key[i] = (uint64_t)pY[q];
        val[i] = q;
    }
}

__global__ void k_grad_seg_flags(const uint64_t* __restrict__ key, const int64_t* __restrict__ n_dev,
                                 int32_t* __restrict__ flag) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = i == 0 || key[i] != key[i - 1];
}

__global__ void k_grad_seg_first(const int32_t* __restrict__ flag, const int32_t* __restrict__ off,
                                 const int64_t* __restrict__ n_dev,
                                 const int64_t* __restrict__ nseg_dev,
                                 int32_t* __restrict__ seg_first) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) seg_first[off[i]] = (int32_t)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) seg_first[*nseg_dev] = (int32_t)n;
}

int bits_for_grad(int64_t v) {
    int b = 1;
    while (b < 63 && (1ll << b) <= v) ++b;
    return b;
}

}  // namespace

// The near-field pair list regrouped by source leaf (device radix sort of the
// pair indices by Y): *list receives the pair indices, *segf the first list
// entry of every source leaf's segment (segment count in dcounts(c)->scan_n).
void pairs_by_source(msp_ctx& c, cudaStream_t s, const int32_t** segf_out,
                     const int32_t** list_out) {
    DevCounts* dc = dcounts(c);
    const int B = 256;
    const int64_t nseg_cap = std::max<int64_t>(c.n_nodes, 1);
    const int64_t cap = std::max<int64_t>(c.n_p2p, 1);
    uint64_t* k0 = c.gr_key0.ensure<uint64_t>((size_t)cap);
    uint64_t* k1 = c.gr_key1.ensure<uint64_t>((size_t)cap);
    int32_t* v0 = c.gr_val0.ensure<int32_t>((size_t)cap);
    int32_t* v1 = c.gr_val1.ensure<int32_t>((size_t)cap);
    int32_t* flag = c.gr_flag.ensure<int32_t>((size_t)cap);
    int32_t* off = c.gr_off.ensure<int32_t>((size_t)cap);
    int32_t* segf = c.gr_seg.ensure<int32_t>((size_t)nseg_cap + 2);
    const int Gp = grid_for(cap, B, (int64_t)c.sm_count * 16);
    k_grad_keys<<<Gp, B, 0, s>>>(c.p2p_val0.get<int32_t>(), &dc->n_p2p, c.pr_Y.get<int32_t>(),
                                 k0, v0);
    MSP_LAUNCH("grad_keys");
    radix_sort_dev(c, k0, v0, k1, v1, &dc->n_p2p, cap, bits_for_grad(c.n_nodes), s);
    k_grad_seg_flags<<<Gp, B, 0, s>>>(k0, &dc->n_p2p, flag);
    MSP_LAUNCH("grad_seg_flags");
    scan_dev(c, flag, off, &dc->n_p2p, cap, &dc->scan_n, nullptr, s);
    k_grad_seg_first<<<Gp, B, 0, s>>>(flag, off, &dc->n_p2p, &dc->scan_n, segf);
    MSP_LAUNCH("grad_seg_first");
    *segf_out = segf;
    *list_out = v0;
}

void attraction_grad(msp_ctx& c, const uint8_t* type, const uint8_t* va, const uint8_t* vde,
                     const uint8_t* vdi, const float* g, float* u, float* dud, float* gE,
                     float* gI, cudaStream_t s) {
    NvtxRange nv_("msp attraction_grad");
    if (!c.attraction_done) throw Error(MSP_ERR_NOT_BUILT, "msp_attraction must run first");
    if (c.n_far > 0)
        throw Error(MSP_ERR_INVALID_ARG,
                    "derivatives need a plan without translated pairs (rho_max = 0)");
    if ((gE || gI) && !g) throw Error(MSP_ERR_INVALID_ARG, "weight gradients need g");
    const int64_t n = c.n;
    if (n == 0) return;
    const msp_config& cfg = c.cfg;
    const int B = 256;
    const int G = grid_for(n, B, (int64_t)c.sm_count * 16);
    DevCounts* dc = dcounts(c);
    float4* gw = c.gr_w.ensure<float4>((size_t)n);
    k_grad_gather<<<G, B, 0, s>>>(n, c.perm.get<int32_t>(), type, va, vde, vdi, g, gw);
    MSP_LAUNCH("grad_gather");
    const float sqk = (float)std::sqrt(1.4426950408889634 / (cfg.sigma * cfg.sigma));
    const float dscale = (float)(2.0 / (cfg.sigma * 1.4426950408889634));
    const int64_t nseg_cap = std::max<int64_t>(c.n_nodes, 1);
    const int32_t* list_q = c.p2p_val0.get<int32_t>();
    const int nb = (int)std::min<int64_t>(nseg_cap, 1 << 30);
    if (u || dud) {
        if (u) MSP_CUDA(cudaMemsetAsync(u, 0, (size_t)n * sizeof(float), s));
        if (dud) MSP_CUDA(cudaMemsetAsync(dud, 0, (size_t)n * sizeof(float), s));
        k_grad_pairs<true><<<nb, kGrWarps * 32, 0, s>>>(
            c.seg_first.get<int32_t>(), &dc->nseg, list_q, c.pr_X.get<int32_t>(),
            c.pr_Y.get<int32_t>(), c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(),
            c.pts.get<float4>(), gw, c.perm.get<int32_t>(), sqk, dscale, u, dud);
        MSP_LAUNCH("grad_forward");
    }
    if (gE || gI) {
        float* oE = gE ? gE : c.gr_tmp.ensure<float>((size_t)n);
        float* oI = gI ? gI : c.gr_tmp.ensure<float>((size_t)n);
        MSP_CUDA(cudaMemsetAsync(oE, 0, (size_t)n * sizeof(float), s));
        MSP_CUDA(cudaMemsetAsync(oI, 0, (size_t)n * sizeof(float), s));
        const int32_t *segf = nullptr, *v0 = nullptr;
        pairs_by_source(c, s, &segf, &v0);
        k_grad_pairs<false><<<nb, kGrWarps * 32, 0, s>>>(
            segf, &dc->scan_n, v0, c.pr_Y.get<int32_t>(), c.pr_X.get<int32_t>(),
            c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(), c.pts.get<float4>(), gw,
            c.perm.get<int32_t>(), sqk, dscale, oE, oI);
        MSP_LAUNCH("grad_adjoint");
    }
}

}  // namespace msp
