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
constexpr int kGrMaxR = 3;                // evaluation points per lane
constexpr int kGrList = 32 * kGrMaxR;     // evaluation points per pass

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

// The staged pairs j = ksl, ksl + slices, ... < mp against the lane's R points.
template <bool FORWARD, bool SELF, int R>
__device__ __forceinline__ void gr_eval(const float4* sA, const float4* sB, const float4* sC,
                                        int mp, int ksl, int slices, const float2 (&tx)[R],
                                        const float2 (&ty)[R], const float2 (&tz)[R],
                                        const bool (&inh)[R], const int32_t (&e)[R],
                                        float2 (&a0)[R], float2 (&a1)[R]) {
#pragma unroll 2
    for (int j = ksl; j < mp; j += slices) {
        const float4 A = sA[j], B = sB[j], C = sC[j];
#pragma unroll
        for (int r = 0; r < R; ++r)
            gr_term<FORWARD, SELF>(A, B, C, tx[r], ty[r], tz[r], inh[r], e[r], a0[r], a1[r]);
    }
}

// The transposed sums in the expanded form: with the point s^ held as 2 s^ and
// a staged partner t as (t^, -|t^|^2), E = 2 s^.t^ - |t^|^2 and
// K(t,s) = 2^E 2^-|s^|^2 (the last factor applied once per point; E <= |s^|^2,
// which the pass keeps at most kGrFastT2).  Staged pair j: A = (x0, x1, y0, y1),
// B = (z0, z1, c0, c1), C = (gE0, gE1, gI0, gI1), D = (index0, index1).
constexpr float kGrFastT2 = 20.f;

template <bool SELF>
__device__ __forceinline__ void gr_term_fast(const float4 A, const float4 B, const float4 C,
                                             const int2 D, float2 tx, float2 ty, float2 tz,
                                             int32_t e, float2& a0, float2& a1) {
    const float2 E = __ffma2_rn(tx, make_float2(A.x, A.y),
                                __ffma2_rn(ty, make_float2(A.z, A.w),
                                           __ffma2_rn(tz, make_float2(B.x, B.y),
                                                      make_float2(B.z, B.w))));
    float2 k = make_float2(gr_ex2(E.x), gr_ex2(E.y));
    if (SELF) {
        k.x = D.x == e ? 0.f : k.x;
        k.y = D.y == e ? 0.f : k.y;
    }
    a0 = __ffma2_rn(make_float2(C.x, C.y), k, a0);
    a1 = __ffma2_rn(make_float2(C.z, C.w), k, a1);
}

template <bool SELF, int R>
__device__ __forceinline__ void gr_eval_fast(const float4* sA, const float4* sB, const float4* sC,
                                             const int2* sD, int mp, int ksl, int slices,
                                             const float2 (&tx)[R], const float2 (&ty)[R],
                                             const float2 (&tz)[R], const int32_t (&e)[R],
                                             float2 (&a0)[R], float2 (&a1)[R]) {
#pragma unroll 2
    for (int j = ksl; j < mp; j += slices) {
        const float4 A = sA[j], B = sB[j], C = sC[j];
        const int2 D = SELF ? sD[j] : make_int2(0, 0);
#pragma unroll
        for (int r = 0; r < R; ++r) gr_term_fast<SELF>(A, B, C, D, tx[r], ty[r], tz[r], e[r], a0[r], a1[r]);
    }
}

// One pass over the evaluation points plist[0, np) of leaf L against the
// partner leaves of pairs [i0, i1).  A lane holds R points (slots R j .. R j
// + R - 1 of its group j); when the groups fit in fewer lanes they take
// npr = 2^k lanes and 32 / npr lanes share a group, each walking an
// interleaved slice of the staged sources.  The 4 warps take the partner
// leaves round-robin; each packs its partners' points into chunks of 64 in
// shared memory, in pairs, as scaled positions sqrt(k2) (x - o) relative to a
// point o of L, and two weights (L's own points last, in chunks of their own,
// where a point skips itself).  The slices' sums are combined by a fixed butterfly
// and the 4 warps' in a fixed order, so a point's sum does not depend on the
// timing of the warps.
template <bool FORWARD, int R, bool FAST>
__device__ __forceinline__ void gr_pass(const int32_t* plist, int np, int32_t i0, int32_t i1,
                                        int32_t L, const float4& O,
                                        const int32_t* __restrict__ pairs,
                                        const int32_t* __restrict__ pPart,
                                        const int32_t* __restrict__ nfirst,
                                        const int32_t* __restrict__ ncount,
                                        const float4* __restrict__ pts,
                                        const float4* __restrict__ gw, float sqk, float4* sAw,
                                        float4* sBw, float4* sCw, int2* sDw,
                                        float (*red)[2][kGrList]) {
    static_assert(!(FAST && FORWARD), "the expanded form serves the transposed sums only");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lg = 0;
    while ((1 << lg) < (np + R - 1) / R) ++lg;
    const int npr = 1 << lg, slices = 32 >> lg;
    const int j = lane & (npr - 1), ksl = lane >> lg;
    const bool active = R * j < np;
    float2 tx[R], ty[R], tz[R], a0[R], a1[R];
    bool inh[R];
    int32_t e[R];
    float sc[R];   // FAST: 2^-|s^|^2 of the point
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int slot = R * j + r;
        const bool v = slot < np;
        e[r] = v ? plist[slot] : -1;
        const int32_t pi = v ? e[r] : plist[0];
        const float4 T = pts[pi];
        inh[r] = (__float_as_uint(gw[pi].w) & 1u) != 0;
        const float x = (T.x - O.x) * sqk, y = (T.y - O.y) * sqk, z = (T.z - O.z) * sqk;
        const float f = FAST ? 2.f : 1.f;
        tx[r] = make_float2(f * x, f * x);
        ty[r] = make_float2(f * y, f * y);
        tz[r] = make_float2(f * z, f * z);
        sc[r] = FAST ? gr_ex2(-fmaf(x, x, fmaf(y, y, z * z))) : 1.f;
        a0[r] = make_float2(0.f, 0.f);
        a1[r] = make_float2(0.f, 0.f);
    }
    int* fD = reinterpret_cast<int*>(sDw);
    float* fA = reinterpret_cast<float*>(sAw);
    float* fB = reinterpret_cast<float*>(sBw);
    float* fC = reinterpret_cast<float*>(sCw);
    // stage sources [pf + sb, pf + sb + take) at chunk positions fill.. (two
    // per staged pair); position m of an odd chunk is padded before use
    auto stage = [&](int32_t pf, int32_t sb, int take, int fill) {
        for (int k = lane; k < take; k += 32) {
            const float4 S = pts[pf + sb + k];
            const float4 W = gw[pf + sb + k];
            float w0, w1;
            if (FORWARD) {
                w0 = W.x;
                w1 = W.y;
            } else {
                const uint32_t f2 = __float_as_uint(W.w);
                const float gv = (f2 & 2u) ? W.z : 0.f;
                w0 = (f2 & 1u) ? 0.f : gv;
                w1 = (f2 & 1u) ? gv : 0.f;
            }
            const int pos = fill + k, jj = pos >> 1, h = pos & 1;
            if (FAST) {
                const float sx = (S.x - O.x) * sqk, sy = (S.y - O.y) * sqk,
                            sz = (S.z - O.z) * sqk;
                fA[4 * jj + h] = sx;
                fA[4 * jj + 2 + h] = sy;
                fB[4 * jj + h] = sz;
                fB[4 * jj + 2 + h] = -fmaf(sx, sx, fmaf(sy, sy, sz * sz));
                fC[4 * jj + h] = w0;
                fC[4 * jj + 2 + h] = w1;
                fD[2 * jj + h] = pf + sb + k;
            } else {
                fA[4 * jj + h] = -(S.x - O.x) * sqk;
                fA[4 * jj + 2 + h] = -(S.y - O.y) * sqk;
                fB[4 * jj + h] = -(S.z - O.z) * sqk;
                fB[4 * jj + 2 + h] = w0;
                fC[4 * jj + h] = w1;
                fC[4 * jj + 2 + h] = __int_as_float(pf + sb + k);
            }
        }
    };
    auto pad = [&](int m) {
        if ((m & 1) && lane == 0) {
            const int jj = m >> 1;
            fA[4 * jj + 1] = 0.f;
            fA[4 * jj + 3] = 0.f;
            fB[4 * jj + 1] = 0.f;
            fB[4 * jj + 3] = 0.f;
            fC[4 * jj + 1] = 0.f;
            fC[4 * jj + 3] = FAST ? 0.f : __int_as_float(-1);
            if (FAST) fD[2 * jj + 1] = -1;
        }
    };
    // the staged pairs [0, mp) against the lane's points
    auto eval = [&](int mp, bool selfc) {
        if (!active) return;
        if (FAST) {
            if (selfc)
                gr_eval_fast<true, R>(sAw, sBw, sCw, sDw, mp, ksl, slices, tx, ty, tz, e, a0, a1);
            else
                gr_eval_fast<false, R>(sAw, sBw, sCw, sDw, mp, ksl, slices, tx, ty, tz, e, a0,
                                       a1);
        } else {
            if (selfc)
                gr_eval<FORWARD, true, R>(sAw, sBw, sCw, mp, ksl, slices, tx, ty, tz, inh, e, a0,
                                          a1);
            else
                gr_eval<FORWARD, false, R>(sAw, sBw, sCw, mp, ksl, slices, tx, ty, tz, inh, e,
                                           a0, a1);
        }
    };
    // the partner leaves other than L, packed into full chunks (the sums
    // need no per-pair result); then L itself, whose terms skip t = s
    int fill = 0;
    bool self = false;
    for (int32_t i = i0 + w; i < i1; i += kGrWarps) {
        const int32_t P = pPart[pairs[i]];
        if (P == L) {
            self = true;
            continue;
        }
        const int32_t pf = nfirst[P], pc = ncount[P];
        for (int32_t sb = 0; sb < pc;) {
            const int take = min(kGrStage - fill, pc - sb);
            stage(pf, sb, take, fill);
            fill += take;
            sb += take;
            if (fill == kGrStage) {
                __syncwarp();
                eval(kGrStage / 2, false);
                __syncwarp();
                fill = 0;
            }
        }
    }
    if (fill > 0) {
        pad(fill);
        __syncwarp();
        eval((fill + 1) >> 1, false);
        __syncwarp();
    }
    if (self) {
        const int32_t pf = nfirst[L], pc = ncount[L];
        for (int32_t sb = 0; sb < pc; sb += kGrStage) {
            const int m = min(kGrStage, pc - sb);
            stage(pf, sb, m, 0);
            pad(m);
            __syncwarp();
            eval((m + 1) >> 1, true);
            __syncwarp();
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float s0 = a0[r].x + a0[r].y, s1 = a1[r].x + a1[r].y;
        for (int o = npr; o < 32; o <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (FAST) {
            s0 *= sc[r];
            s1 *= sc[r];
        }
        const int slot = R * j + r;
        if (ksl == 0 && slot < np) {
            red[w][0][slot] = s0;
            red[w][1][slot] = s1;
        }
    }
}

// One block per leaf L of a segment list (the evaluation leaf; with `order`,
// the segments longest first), its 4 warps taking the segment's partner
// leaves P.  Warp 0 lists L's evaluation points, up to kGrList per pass
// (FORWARD: the targets, a_t > 0; ADJOINT: every point), and the pass holds R
// = 1..3 of them per lane, R the fewest evaluated slots per source (ties to
// the larger R: fewer shared-memory loads per evaluation).
//   FORWARD: evaluation points = targets t (a_t > 0), partner weights
//            (w^E, w^I): u += w^{T(t)} 2^-q, d += w^{T(t)} q 2^-q.
//   ADJOINT: evaluation points = sources s, partner weights
//            (g_t [T(t) = E], g_t [T(t) = I]) (0 unless a_t > 0):
//            gE += w0 2^-q, gI += w1 2^-q.
// Points that are not evaluated keep the zero the caller wrote.
template <bool FORWARD>
__global__ void __launch_bounds__(kGrWarps * 32, 7)
k_grad_pairs(const int32_t* __restrict__ seg_first, const int64_t* __restrict__ nseg_dev,
             const int32_t* __restrict__ order, const int32_t* __restrict__ pairs,
             const int32_t* __restrict__ pEval, const int32_t* __restrict__ pPart,
             const int32_t* __restrict__ nfirst, const int32_t* __restrict__ ncount,
             const float4* __restrict__ pts, const float4* __restrict__ gw,
             const int32_t* __restrict__ perm, float sqk, float dscale, float* __restrict__ out0,
             float* __restrict__ out1) {
    __shared__ float4 sA[kGrWarps][kGrStage / 2], sB[kGrWarps][kGrStage / 2],
        sC[kGrWarps][kGrStage / 2];
    __shared__ int2 sD[kGrWarps][kGrStage / 2];
    __shared__ float red[kGrWarps][2][kGrList];
    __shared__ int32_t plist[kGrList];
    __shared__ int s_np, s_pos;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nseg = *nseg_dev;
    for (int64_t b = blockIdx.x; b < nseg; b += gridDim.x) {
        const int64_t sg = order ? order[b] : b;
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
            int R = 1, best = 1 << 30;
            for (int rr = 1; rr <= kGrMaxR; ++rr) {
                const int g = (np + rr - 1) / rr;
                if (g > 32) continue;
                int npr = 1;
                while (npr < g) npr <<= 1;
                if (npr * rr <= best) {
                    best = npr * rr;
                    R = rr;
                }
            }
            // the transposed sums take the expanded form while every point of
            // the pass has |s^|^2 <= kGrFastT2 (the same value in every warp)
            bool fast = false;
            if (!FORWARD) {
                float m2 = 0.f;
                for (int k = lane; k < np; k += 32) {
                    const float4 T = pts[plist[k]];
                    const float x = (T.x - O.x) * sqk, y = (T.y - O.y) * sqk,
                                z = (T.z - O.z) * sqk;
                    m2 = fmaxf(m2, fmaf(x, x, fmaf(y, y, z * z)));
                }
                for (int o = 16; o > 0; o >>= 1) m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
                fast = m2 <= kGrFastT2;
            }
#define MSP_GR_PASS(RR, FF)                                                                   \
    gr_pass<FORWARD, RR, FF>(plist, np, i0, i1, L, O, pairs, pPart, nfirst, ncount, pts, gw, sqk, \
                             sA[w], sB[w], sC[w], sD[w], red)
            if (!FORWARD && fast) {
                if (R == 1) MSP_GR_PASS(1, !FORWARD);
                else if (R == 2) MSP_GR_PASS(2, !FORWARD);
                else MSP_GR_PASS(3, !FORWARD);
            } else {
                if (R == 1) MSP_GR_PASS(1, false);
                else if (R == 2) MSP_GR_PASS(2, false);
                else MSP_GR_PASS(3, false);
            }
#undef MSP_GR_PASS
            __syncthreads();
            if (w == 0) {
#pragma unroll
                for (int r = 0; r < kGrMaxR; ++r) {
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
        // the segments in the near field's order (longest first), kept with the lists
        k_grad_pairs<true><<<nb, kGrWarps * 32, 0, s>>>(
            c.seg_first.get<int32_t>(), &dc->nseg, c.nf_oval0.get<int32_t>(), list_q,
            c.pr_X.get<int32_t>(),
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
            segf, &dc->scan_n, nullptr, v0, c.pr_Y.get<int32_t>(), c.pr_X.get<int32_t>(),
            c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(), c.pts.get<float4>(), gw,
            c.perm.get<int32_t>(), sqk, dscale, oE, oI);
        MSP_LAUNCH("grad_adjoint");
    }
}

}  // namespace msp
