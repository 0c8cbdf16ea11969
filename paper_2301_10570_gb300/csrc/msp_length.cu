// msp_length.cu -- the expected mean synapse length and its gradient, the
// loss of the differentiation workload.
//
// An axonal element of t draws dendrite s with probability w_s K(t,s) / u(t)
// (Eq. 1 with the kernel of Eq. 8, K = exp(-r^2/sigma^2); w = the continuous
// dendritic weights of t's channel), so its synapse is l(t) = v(t)/u(t) long
// on average, with
//   u(t) = sum_s w_s K,   v(t) = sum_s w_s K r.
// Over the vacant axonal elements (a_t > 0, u(t) > 0; A = sum of their a_t):
//   m = sum_t a_t l(t) / A,   loss = (m - target)^2,
//   dm/dsigma = sum_t a_t (v' u - v u') / (A u^2),  with ' = d/dsigma:
//               u' = sum w K 2 r^2 / sigma^3,  v' = sum w K r 2 r^2 / sigma^3,
//   dm/dw^T_s = sum_{t: T(t) = T} K(t,s) (alpha_t r - beta_t),
//               alpha_t = a_t / (A u), beta_t = a_t v / (A u^2),
// and every loss derivative is 2 (m - target) times m's.  The sums run over
// the near-field leaf pairs of the last attraction (a plan without
// translations: K r has no Hermite expansion), first grouped by target leaf
// (u, v and their sigma derivatives), then by source leaf (the transposed
// sums).  One block of 4 warps per leaf, 1-2 evaluation points per lane,
// the warps taking the partner leaves; the partners' points are staged in
// shared memory, and each staged chunk's sum is added with Kahan's
// compensated summation.  Every sum has a fixed order, so
// the results are reproducible; the scalar reductions run in double.
#include <algorithm>
#include <cmath>

#include "msp_internal.cuh"

namespace msp {

void pairs_by_source(msp_ctx& c, cudaStream_t s, const int32_t** segf_out,
                     const int32_t** list_out);

namespace {

constexpr double kLog2e = 1.4426950408889634;

__device__ inline float len_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ inline float len_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ inline void kahan_add(float& acc, float& cmp, float v) {
    const float y = __fsub_rn(v, cmp);
    const float t = __fadd_rn(acc, y);
    cmp = __fsub_rn(__fsub_rn(t, acc), y);
    acc = t;
}

// sorted-order inputs: {w^E, w^I, a, type}
__global__ void k_len_gather(int64_t n, const int32_t* __restrict__ perm,
                             const uint8_t* __restrict__ type, const uint8_t* __restrict__ va,
                             const float* __restrict__ we, const float* __restrict__ wi,
                             float4* __restrict__ gw) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = perm[s];
        gw[s] = make_float4(we[c], wi[c], (float)va[c], type[c] ? 1.f : 0.f);
    }
}

constexpr int kLenWarps = 4;
constexpr int kLenStage = 32;    // staged sources per warp and chunk

// One block of 4 warps per leaf L of a segment list.  The leaf's points are
// taken 32 at a time, one per lane, and every warp holds the same points; the
// warps take the segment's partner leaves P round-robin, each packing its
// partners' points into chunks of 32 in its own shared memory, and every
// chunk's sum joins the lane's running sums by Kahan's compensated summation.
// The 4 warps' compensated sums are added in a fixed order.  Coordinates are
// scaled by sqk = sqrt(log2 e)/sigma relative to L's first point, so that
// q = |t^ - s^|^2 gives K = 2^-q and r = rs sqrt(q), rs = sigma/sqrt(log2 e);
// a point skips itself (by index).
//   FORWARD (L = the target leaf): per target t with a_t > 0, the sums
//     U = sum w K, V = sum w K r, QU = sum w K q, QV = sum w K q r
//     (w: the staged source's weight of t's channel), written in sorted order.
//   ADJOINT (L = the source leaf): per point s, for each channel T,
//     G_T = sum_{t: T(t) = T} K (alpha_t r - beta_t)
//     over the staged targets t (coefficients in cf), written in caller order.
constexpr int kLenMaxR = 2;                 // evaluation points per lane
constexpr int kLenList = 32 * kLenMaxR;     // evaluation points per pass

// The staged pairs j = ksl, ksl + slices, ... < mp of a chunk against the
// lane's R points t[r], into their compensated running sums acc/cmp (4 each).
// Staged pair j (sources 2j, 2j + 1):
//   A = (-x0, -x1, -y0, -y1), B = (-z0, -z1, index0, index1),
//   C = FORWARD: (w^E_0, w^E_1, w^I_0, w^I_1); ADJOINT: (alpha0, alpha1,
//       beta0, beta1),
//   D = ADJOINT: (I0, I1, E0, E1), the sources' channels as 0/1,
// a padding source with zero weights; every step is a paired FP32
// instruction over the two sources (two results, one issue slot) with the
// per-element rounding of the scalar form.  SELF: a source may be t itself;
// its term is zero.
template <bool FORWARD, bool SELF, int R>
__device__ __forceinline__ void len_eval(const float4* sA, const float4* sB, const float4* sC,
                                         const float4* sD, int mp, int ksl, int slices,
                                         const int32_t (&t)[R], const bool (&inh)[R],
                                         const float2 (&tx)[R], const float2 (&ty)[R],
                                         const float2 (&tz)[R], float rs, float (&acc)[R][4],
                                         float (&cmp)[R][4]) {
    const float2 rs2 = make_float2(rs, rs);
    float2 p[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[r][c] = make_float2(0.f, 0.f);
    for (int j = ksl; j < mp; j += slices) {
        const float4 A = sA[j], B = sB[j], C = sC[j];
        float4 D = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!FORWARD) D = sD[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 dx = __fadd2_rn(tx[r], make_float2(A.x, A.y));
            const float2 dy = __fadd2_rn(ty[r], make_float2(A.z, A.w));
            const float2 dz = __fadd2_rn(tz[r], make_float2(B.x, B.y));
            const float2 q = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            float2 K = make_float2(len_ex2(-q.x), len_ex2(-q.y));
            if (SELF) {
                K.x = __float_as_int(B.z) == t[r] ? 0.f : K.x;
                K.y = __float_as_int(B.w) == t[r] ? 0.f : K.y;
            }
            const float2 rr = __fmul2_rn(rs2, make_float2(len_sqrt(q.x), len_sqrt(q.y)));
            if (FORWARD) {
                const float2 wk =
                    __fmul2_rn(inh[r] ? make_float2(C.z, C.w) : make_float2(C.x, C.y), K);
                p[r][0] = __fadd2_rn(p[r][0], wk);
                p[r][1] = __ffma2_rn(wk, rr, p[r][1]);
                p[r][2] = __ffma2_rn(wk, q, p[r][2]);
                p[r][3] = __ffma2_rn(__fmul2_rn(wk, q), rr, p[r][3]);
            } else {
                const float2 v = __fmul2_rn(K, __ffma2_rn(make_float2(C.x, C.y), rr,
                                                          make_float2(-C.z, -C.w)));
                p[r][1] = __ffma2_rn(make_float2(D.x, D.y), v, p[r][1]);
                p[r][0] = __ffma2_rn(make_float2(D.z, D.w), v, p[r][0]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < (FORWARD ? 4 : 2); ++c)
            kahan_add(acc[r][c], cmp[r][c], p[r][c].x + p[r][c].y);
}

// One pass over the evaluation points plist[0, np) of leaf L (first point
// lf, O its position) against the partner leaves of pairs [i0, i1).  A lane
// holds R points (slots R j .. R j + R - 1 of its group j); when the groups
// fit in fewer lanes they take npr = 2^k lanes and 32 / npr lanes share a
// group, each walking an interleaved slice of the staged sources.  The 4
// warps take the partner leaves round-robin, packing their points into
// chunks of kLenStage in shared memory (L's own points last, in chunks of
// their own); every chunk's sums join the lane's compensated running sums.
// The slices' compensated sums are added by a fixed butterfly; the warps'
// go to red for a fixed-order sum.
template <bool FORWARD, int R>
__device__ __forceinline__ void len_pass(const int32_t* plist, int np, int32_t i0, int32_t i1,
                                         int32_t L, int32_t lf, int32_t lc, const float4& O,
                                         const int32_t* __restrict__ pairs,
                                         const int32_t* __restrict__ pPart,
                                         const int32_t* __restrict__ nfirst,
                                         const int32_t* __restrict__ ncount,
                                         const float4* __restrict__ pts,
                                         const float4* __restrict__ gw,
                                         const float2* __restrict__ cf, float sqk, float rs,
                                         float4* sA, float4* sB, float4* sC, float4* sD,
                                         float4 (*red)[kLenList]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lg = 0;
    while ((1 << lg) < (np + R - 1) / R) ++lg;
    const int npr = 1 << lg, slices = 32 >> lg;
    const int jg = lane & (npr - 1), ksl = lane >> lg;
    const bool active = R * jg < np;
    int32_t t[R];
    bool inh[R];
    float2 tx[R], ty[R], tz[R];
    float acc[R][4], cmp[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int slot = R * jg + r;
        t[r] = slot < np ? plist[slot] : -1;
        const int32_t pi = slot < np ? t[r] : plist[0];
        const float4 T = pts[pi];
        inh[r] = gw[pi].w != 0.f;
        const float x = (T.x - O.x) * sqk, y = (T.y - O.y) * sqk, z = (T.z - O.z) * sqk;
        tx[r] = make_float2(x, x);
        ty[r] = make_float2(y, y);
        tz[r] = make_float2(z, z);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cmp[r][c] = 0.f;
    }
    float* fA = reinterpret_cast<float*>(sA);
    float* fB = reinterpret_cast<float*>(sB);
    float* fC = reinterpret_cast<float*>(sC);
    float* fD = reinterpret_cast<float*>(sD);
    // stage sources [pf + sb, pf + sb + take) at chunk positions fill..;
    // position m of an odd chunk is padded before use
    auto stage = [&](int32_t pf, int32_t sb, int take, int fill) {
        if (lane < take) {
            const int32_t j = pf + sb + lane;
            const float4 S = pts[j];
            const float4 SW = gw[j];
            const int pos = fill + lane, jj = pos >> 1, h = pos & 1;
            fA[4 * jj + h] = -(S.x - O.x) * sqk;
            fA[4 * jj + 2 + h] = -(S.y - O.y) * sqk;
            fB[4 * jj + h] = -(S.z - O.z) * sqk;
            fB[4 * jj + 2 + h] = __int_as_float(j);
            if (FORWARD) {
                fC[4 * jj + h] = SW.x;
                fC[4 * jj + 2 + h] = SW.y;
            } else {
                const float2 ab = SW.z > 0.f ? cf[j] : make_float2(0.f, 0.f);
                fC[4 * jj + h] = ab.x;
                fC[4 * jj + 2 + h] = ab.y;
                fD[4 * jj + h] = SW.w != 0.f ? 1.f : 0.f;
                fD[4 * jj + 2 + h] = SW.w != 0.f ? 0.f : 1.f;
            }
        }
    };
    auto pad = [&](int m) {
        if ((m & 1) && lane == 0) {
            const int jj = m >> 1;
            fA[4 * jj + 1] = 0.f;
            fA[4 * jj + 3] = 0.f;
            fB[4 * jj + 1] = 0.f;
            fB[4 * jj + 3] = __int_as_float(-1);
            fC[4 * jj + 1] = 0.f;
            fC[4 * jj + 3] = 0.f;
            if (!FORWARD) {
                fD[4 * jj + 1] = 0.f;
                fD[4 * jj + 3] = 0.f;
            }
        }
    };
    int fill = 0;
    bool self = false;
    for (int32_t i = i0 + w; i < i1; i += kLenWarps) {
        const int32_t P = pPart[pairs[i]];
        if (P == L) {
            self = true;
            continue;
        }
        const int32_t pf = nfirst[P], pc = ncount[P];
        for (int32_t sb = 0; sb < pc;) {
            const int take = min(kLenStage - fill, pc - sb);
            stage(pf, sb, take, fill);
            fill += take;
            sb += take;
            if (fill == kLenStage) {
                __syncwarp();
                if (active)
                    len_eval<FORWARD, false, R>(sA, sB, sC, sD, kLenStage / 2, ksl, slices, t,
                                                inh, tx, ty, tz, rs, acc, cmp);
                __syncwarp();
                fill = 0;
            }
        }
    }
    if (fill > 0) {
        pad(fill);
        __syncwarp();
        if (active)
            len_eval<FORWARD, false, R>(sA, sB, sC, sD, (fill + 1) >> 1, ksl, slices, t, inh, tx,
                                        ty, tz, rs, acc, cmp);
        __syncwarp();
    }
    if (self) {
        for (int32_t sb = 0; sb < lc; sb += kLenStage) {
            const int m = min(kLenStage, lc - sb);
            stage(lf, sb, m, 0);
            pad(m);
            __syncwarp();
            if (active)
                len_eval<FORWARD, true, R>(sA, sB, sC, sD, (m + 1) >> 1, ksl, slices, t, inh, tx,
                                           ty, tz, rs, acc, cmp);
            __syncwarp();
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            v[c] = __fsub_rn(acc[r][c], cmp[r][c]);
            for (int o = npr; o < 32; o <<= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
        }
        const int slot = R * jg + r;
        if (ksl == 0 && slot < np) red[w][slot] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// One block of 4 warps per leaf L of a segment list.  Warp 0 lists L's
// evaluation points (FORWARD: the targets, a_t > 0; ADJOINT: every point), up
// to kLenList per pass, and the pass holds R = 1 or 2 of them per lane, R the
// fewest evaluated slots per source (ties to the larger R).  Coordinates are
// scaled by sqk = sqrt(log2 e)/sigma relative to L's first point, so that
// q = |t^ - s^|^2 gives K = 2^-q and r = rs sqrt(q), rs = sigma/sqrt(log2 e).
//   FORWARD (L = the target leaf): per target t with a_t > 0, the sums
//     U = sum w K, V = sum w K r, QU = sum w K q, QV = sum w K q r
//     (w: the staged source's weight of t's channel), written in sorted order.
//   ADJOINT (L = the source leaf): per point s, for each channel T,
//     G_T = sum_{t: T(t) = T} K (alpha_t r - beta_t)
//     over the staged targets t (coefficients in cf), written in caller order.
template <bool FORWARD>
__global__ void __launch_bounds__(kLenWarps * 32, 6)
k_len_pairs(const int32_t* __restrict__ seg_first, const int64_t* __restrict__ nseg_dev,
            const int32_t* __restrict__ pairs, const int32_t* __restrict__ pEval,
            const int32_t* __restrict__ pPart, const int32_t* __restrict__ nfirst,
            const int32_t* __restrict__ ncount, const float4* __restrict__ pts,
            const float4* __restrict__ gw, const float2* __restrict__ cf,
            const int32_t* __restrict__ perm, float sqk, float rs, float4* __restrict__ sums,
            float* __restrict__ gE, float* __restrict__ gI) {
    __shared__ float4 sA_all[kLenWarps][kLenStage / 2], sB_all[kLenWarps][kLenStage / 2],
        sC_all[kLenWarps][kLenStage / 2], sD_all[kLenWarps][FORWARD ? 1 : kLenStage / 2];
    __shared__ float4 red[kLenWarps][kLenList];   // the warps' compensated sums per slot
    __shared__ int32_t plist[kLenList];
    __shared__ int s_np, s_pos;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nseg = *nseg_dev;
    for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const int32_t i0 = seg_first[sg], i1 = seg_first[sg + 1];
        const int32_t L = pEval[pairs[i0]];
        const int32_t lf = nfirst[L], lc = ncount[L];
        const float4 O = pts[lf];
        int32_t pos = 0;
        for (;;) {
            if (w == 0) {
                // the next (at most) kLenList evaluation points from pos on
                int np = 0;
                int32_t p = pos;
                while (p < lc && np < kLenList) {
                    const int32_t idx = p + lane;
                    bool ok = idx < lc;
                    if (FORWARD && ok) ok = gw[lf + idx].z > 0.f;
                    const unsigned mk = __ballot_sync(0xffffffffu, ok);
                    const int room = kLenList - np;
                    const int rank = __popc(mk & ((1u << lane) - 1u));
                    if (ok && rank < room) plist[np + rank] = lf + idx;
                    if (__popc(mk) > room) {
                        // the room-th point ends the pass: resume after it
                        unsigned keep = mk;
                        for (int k = 0; k < room; ++k) keep &= keep - 1u;
                        p += __ffs(keep) - 1;
                        np = kLenList;
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
            for (int rr = 1; rr <= kLenMaxR; ++rr) {
                const int g = (np + rr - 1) / rr;
                if (g > 32) continue;
                int npr = 1;
                while (npr < g) npr <<= 1;
                if (npr * rr <= best) {
                    best = npr * rr;
                    R = rr;
                }
            }
            if (R == 1)
                len_pass<FORWARD, 1>(plist, np, i0, i1, L, lf, lc, O, pairs, pPart, nfirst,
                                     ncount, pts, gw, cf, sqk, rs, sA_all[w], sB_all[w],
                                     sC_all[w], sD_all[w], red);
            else
                len_pass<FORWARD, 2>(plist, np, i0, i1, L, lf, lc, O, pairs, pPart, nfirst,
                                     ncount, pts, gw, cf, sqk, rs, sA_all[w], sB_all[w],
                                     sC_all[w], sD_all[w], red);
            __syncthreads();
            if (w == 0) {
#pragma unroll
                for (int rr = 0; rr < kLenMaxR; ++rr) {
                    const int j = lane + 32 * rr;
                    if (j >= np) continue;
                    float4 v = red[0][j];
#pragma unroll
                    for (int k = 1; k < kLenWarps; ++k) {
                        const float4 x = red[k][j];
                        v.x += x.x;
                        v.y += x.y;
                        v.z += x.z;
                        v.w += x.w;
                    }
                    const int32_t t = plist[j];
                    if (FORWARD) {
                        sums[t] = v;
                    } else {
                        const int32_t o = perm[t];
                        if (gE) gE[o] = v.x;
                        if (gI) gI[o] = v.y;
                    }
                }
            }
            __syncthreads();
            if (pos >= lc) break;
        }
    }
}

constexpr int kLenRedThreads = 256;

// per block: the partial sums A = sum a, S = sum a V/U, D = sum a (V'U - VU')/U^2
// over the targets it takes (a > 0, U > 0), in double, reduced in a fixed
// order; V' / U' are QV / QU times dscale = 2 / (sigma log2 e)
__global__ void __launch_bounds__(kLenRedThreads)
k_len_reduce(int64_t n, const float4* __restrict__ gw, const float4* __restrict__ sums,
             double dscale, double* __restrict__ part) {
    __shared__ double red[3][kLenRedThreads];
    double A = 0.0, S = 0.0, D = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float a = gw[t].z;
        if (!(a > 0.f)) continue;
        const float4 s4 = sums[t];
        const double U = s4.x, V = s4.y;
        if (!(U > 0.0)) continue;
        const double dU = dscale * s4.z, dV = dscale * s4.w;
        A += a;
        S += a * V / U;
        D += a * (dV * U - V * dU) / (U * U);
    }
    red[0][threadIdx.x] = A;
    red[1][threadIdx.x] = S;
    red[2][threadIdx.x] = D;
    __syncthreads();
    for (int o = kLenRedThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[3 * blockIdx.x + k] = red[k][0];
}

// the blocks' partials in order; res = {loss, m, dloss/dsigma, dm/dsigma, A, f}
__global__ void k_len_final(const double* __restrict__ part, int nblocks, double target,
                            double* __restrict__ res) {
    double A = 0.0, S = 0.0, D = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        A += part[3 * b];
        S += part[3 * b + 1];
        D += part[3 * b + 2];
    }
    const double m = A > 0.0 ? S / A : 0.0;
    const double dm = A > 0.0 ? D / A : 0.0;
    const double f = 2.0 * (m - target);
    res[0] = (m - target) * (m - target);
    res[1] = m;
    res[2] = f * dm;
    res[3] = dm;
    res[4] = A;
    res[5] = f;
}

// per target: (f alpha_t, f beta_t), f = 2 (m - target), sorted order
__global__ void k_len_coef(int64_t n, const float4* __restrict__ gw,
                           const float4* __restrict__ sums, const double* __restrict__ res,
                           float2* __restrict__ cf) {
    const double A = res[4], f = res[5];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float a = gw[t].z;
        const float4 s4 = sums[t];
        const double U = s4.x, V = s4.y;
        float2 c = make_float2(0.f, 0.f);
        if (a > 0.f && U > 0.0 && A > 0.0)
            c = make_float2((float)(f * a / (A * U)), (float)(f * a * V / (A * U * U)));
        cf[t] = c;
    }
}

}  // namespace

void length_loss(msp_ctx& c, const uint8_t* type, const uint8_t* va, const float* we,
                 const float* wi, double target, double* out4, float* gE, float* gI,
                 cudaStream_t s) {
    NvtxRange nv_("msp length_loss");
    if (!c.attraction_done) throw Error(MSP_ERR_NOT_BUILT, "msp_attraction must run first");
    if (c.n_far > 0)
        throw Error(MSP_ERR_INVALID_ARG,
                    "the synapse length needs a plan without translated pairs (rho_max = 0)");
    const int64_t n = c.n;
    for (int k = 0; k < 4; ++k) out4[k] = 0.0;
    if (n == 0) return;
    const msp_config& cfg = c.cfg;
    const int B = 256;
    const int G = grid_for(n, B, (int64_t)c.sm_count * 16);
    DevCounts* dc = dcounts(c);
    float4* gw = c.gr_w.ensure<float4>((size_t)n);
    k_len_gather<<<G, B, 0, s>>>(n, c.perm.get<int32_t>(), type, va, we, wi, gw);
    MSP_LAUNCH("len_gather");
    const float sqk = (float)std::sqrt(kLog2e / (cfg.sigma * cfg.sigma));
    const float rs = (float)(cfg.sigma / std::sqrt(kLog2e));
    const double dscale = 2.0 / (cfg.sigma * kLog2e);
    const int64_t nseg_cap = std::max<int64_t>(c.n_nodes, 1);
    const int nb = (int)std::min<int64_t>(nseg_cap, 1 << 30);
    float4* sums = c.ln_sums.ensure<float4>((size_t)n);
    MSP_CUDA(cudaMemsetAsync(sums, 0, (size_t)n * sizeof(float4), s));
    k_len_pairs<true><<<nb, kLenWarps * 32, 0, s>>>(
        c.seg_first.get<int32_t>(), &dc->nseg, c.p2p_val0.get<int32_t>(), c.pr_X.get<int32_t>(),
        c.pr_Y.get<int32_t>(), c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(),
        c.pts.get<float4>(), gw, nullptr, c.perm.get<int32_t>(), sqk, rs, sums, nullptr,
        nullptr);
    MSP_LAUNCH("len_forward");
    const int Gr = (int)std::min<int64_t>(grid_for(n, kLenRedThreads), (int64_t)c.sm_count * 4);
    double* part = c.ln_part.ensure<double>((size_t)3 * Gr + 8);
    k_len_reduce<<<Gr, kLenRedThreads, 0, s>>>(n, gw, sums, dscale, part);
    MSP_LAUNCH("len_reduce");
    double* res = part + 3 * Gr;
    k_len_final<<<1, 1, 0, s>>>(part, Gr, target, res);
    MSP_LAUNCH("len_final");
    if (gE || gI) {
        float2* cf = c.ln_coef.ensure<float2>((size_t)n);
        k_len_coef<<<G, B, 0, s>>>(n, gw, sums, res, cf);
        MSP_LAUNCH("len_coef");
        if (gE) MSP_CUDA(cudaMemsetAsync(gE, 0, (size_t)n * sizeof(float), s));
        if (gI) MSP_CUDA(cudaMemsetAsync(gI, 0, (size_t)n * sizeof(float), s));
        const int32_t *segf = nullptr, *list = nullptr;
        pairs_by_source(c, s, &segf, &list);
        k_len_pairs<false><<<nb, kLenWarps * 32, 0, s>>>(
            segf, &dc->scan_n, list, c.pr_Y.get<int32_t>(), c.pr_X.get<int32_t>(),
            c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(), c.pts.get<float4>(), gw, cf,
            c.perm.get<int32_t>(), sqk, rs, nullptr, gE, gI);
        MSP_LAUNCH("len_adjoint");
    }
    MSP_CUDA(cudaMemcpyAsync(out4, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace msp
