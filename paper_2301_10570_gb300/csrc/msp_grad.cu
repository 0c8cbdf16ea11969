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

// One block per leaf L of a segment list (the evaluation leaf), its 4 warps
// taking the segment's partner leaves P round-robin.  Each warp stages P's
// points in shared memory, 64 at a time, as scaled positions
// sqrt(k2) (x - o) relative to a point o of L, and two weights; each lane holds one evaluation point of
// L (several passes for leaves over 32 points) and sums over the staged
// points, q = |t^ - s^|^2 and 2^-q in single precision.  The 4 warps' sums
// are added in a fixed order.
//   FORWARD: evaluation points = targets t (a_t > 0), partner weights
//            (w^E, w^I): u += w^{T(t)} 2^-q, d += w^{T(t)} q 2^-q.
//   ADJOINT: evaluation points = sources s, partner weights
//            (g_t [T(t) = E], g_t [T(t) = I]) (0 unless a_t > 0):
//            gE += w0 2^-q, gI += w1 2^-q.
template <bool FORWARD>
__global__ void __launch_bounds__(kGrWarps * 32)
k_grad_pairs(const int32_t* __restrict__ seg_first, const int64_t* __restrict__ nseg_dev,
             const int32_t* __restrict__ pairs, const int32_t* __restrict__ pEval,
             const int32_t* __restrict__ pPart, const int32_t* __restrict__ nfirst,
             const int32_t* __restrict__ ncount, const float4* __restrict__ pts,
             const float4* __restrict__ gw, const int32_t* __restrict__ perm, float sqk,
             float dscale, float* __restrict__ out0, float* __restrict__ out1) {
    __shared__ float4 sp[kGrWarps][kGrStage];
    __shared__ float2 sw[kGrWarps][kGrStage];
    __shared__ float red[kGrWarps][2][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nseg = *nseg_dev;
    for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const int32_t i0 = seg_first[sg], i1 = seg_first[sg + 1];
        const int32_t L = pEval[pairs[i0]];
        const int32_t lf = nfirst[L], lc = ncount[L];
        // positions relative to a point of L before scaling: small operands,
        // so the differences keep their precision
        const float4 O = pts[lf];
        for (int32_t p0 = 0; p0 < lc; p0 += 32) {
            // this lane's evaluation point
            const int32_t e = lf + p0 + lane;
            const bool valid = p0 + lane < lc;
            const float4 T = pts[valid ? e : lf];
            const float4 G = gw[valid ? e : lf];
            const uint32_t fl = __float_as_uint(G.w);
            const bool act = valid && (!FORWARD || (fl & 2u));
            const bool inh = fl & 1u;
            const float tx = (T.x - O.x) * sqk, ty = (T.y - O.y) * sqk, tz = (T.z - O.z) * sqk;
            float a0 = 0.f, a1 = 0.f;
            for (int32_t i = i0 + w; i < i1; i += kGrWarps) {
                const int32_t P = pPart[pairs[i]];
                const int32_t pf = nfirst[P], pc = ncount[P];
                for (int32_t sb = 0; sb < pc; sb += kGrStage) {
                    const int m = min(kGrStage, pc - sb);
                    __syncwarp();
                    for (int k = lane; k < m; k += 32) {
                        const float4 S = pts[pf + sb + k];
                        const float4 W = gw[pf + sb + k];
                        sp[w][k] = make_float4((S.x - O.x) * sqk, (S.y - O.y) * sqk,
                                               (S.z - O.z) * sqk, __int_as_float(pf + sb + k));
                        if (FORWARD) {
                            sw[w][k] = make_float2(W.x, W.y);
                        } else {
                            const uint32_t f2 = __float_as_uint(W.w);
                            const float gv = (f2 & 2u) ? W.z : 0.f;
                            sw[w][k] = (f2 & 1u) ? make_float2(0.f, gv) : make_float2(gv, 0.f);
                        }
                    }
                    __syncwarp();
                    if (act) {
                        const bool self = P == L;
#pragma unroll 4
                        for (int k = 0; k < m; ++k) {
                            const float4 S = sp[w][k];
                            const float2 W = sw[w][k];
                            const float dx = tx - S.x, dy = ty - S.y, dz = tz - S.z;
                            const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            float ex = gr_ex2(-q);
                            if (self && __float_as_int(S.w) == e) ex = 0.f;
                            if (FORWARD) {
                                const float wk = (inh ? W.y : W.x) * ex;
                                a0 += wk;
                                a1 = fmaf(wk, q, a1);
                            } else {
                                a0 = fmaf(W.x, ex, a0);
                                a1 = fmaf(W.y, ex, a1);
                            }
                        }
                    }
                }
            }
            red[w][0][lane] = a0;
            red[w][1][lane] = a1;
            __syncthreads();
            if (w == 0 && valid) {
                float s0 = red[0][0][lane], s1 = red[0][1][lane];
#pragma unroll
                for (int k = 1; k < kGrWarps; ++k) {
                    s0 += red[k][0][lane];
                    s1 += red[k][1][lane];
                }
                const int32_t c = perm[e];
                if (FORWARD) {
                    if (out0) out0[c] = act ? s0 : 0.f;
                    if (out1) out1[c] = act ? s1 * dscale : 0.f;
                } else {
                    out0[c] = s0;
                    out1[c] = s1;
                }
            }
            __syncthreads();
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
        const int64_t cap = std::max<int64_t>(c.n_p2p, 1);
        uint64_t* k0 = c.gr_key0.ensure<uint64_t>((size_t)cap);
        uint64_t* k1 = c.gr_key1.ensure<uint64_t>((size_t)cap);
        int32_t* v0 = c.gr_val0.ensure<int32_t>((size_t)cap);
        int32_t* v1 = c.gr_val1.ensure<int32_t>((size_t)cap);
        int32_t* flag = c.gr_flag.ensure<int32_t>((size_t)cap);
        int32_t* off = c.gr_off.ensure<int32_t>((size_t)cap);
        int32_t* segf = c.gr_seg.ensure<int32_t>((size_t)nseg_cap + 2);
        const int Gp = grid_for(cap, B, (int64_t)c.sm_count * 16);
        k_grad_keys<<<Gp, B, 0, s>>>(list_q, &dc->n_p2p, c.pr_Y.get<int32_t>(), k0, v0);
        MSP_LAUNCH("grad_keys");
        radix_sort_dev(c, k0, v0, k1, v1, &dc->n_p2p, cap, bits_for_grad(c.n_nodes), s);
        k_grad_seg_flags<<<Gp, B, 0, s>>>(k0, &dc->n_p2p, flag);
        MSP_LAUNCH("grad_seg_flags");
        scan_dev(c, flag, off, &dc->n_p2p, cap, &dc->scan_n, nullptr, s);
        k_grad_seg_first<<<Gp, B, 0, s>>>(flag, off, &dc->n_p2p, &dc->scan_n, segf);
        MSP_LAUNCH("grad_seg_first");
        k_grad_pairs<false><<<nb, kGrWarps * 32, 0, s>>>(
            segf, &dc->scan_n, v0, c.pr_Y.get<int32_t>(), c.pr_X.get<int32_t>(),
            c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(), c.pts.get<float4>(), gw,
            c.perm.get<int32_t>(), sqk, dscale, oE, oI);
        MSP_LAUNCH("grad_adjoint");
    }
}

}  // namespace msp
