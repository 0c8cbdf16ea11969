// msp_nearfield.cu -- step a9: the exact near field (Eq. 8) over the
// near-field leaf pairs of the dual traversal, which dominates the step.
//
// Work unit: one target leaf X (one block of 4 warps) and all its partner
// leaves Y (a contiguous segment of the pair list sorted by X).  Blocks take
// the segments longest first (the order comes from an estimate of each
// segment's work), so the last wave of blocks is short.  The block collects
// the targets of X with vacant axons, up to 125 at a time, and evaluates them
// in one pass; the warps take the partner pairs round-robin.  A lane holds R
// targets of one channel, R = 3 or 4 chosen per round (below; excitatory
// targets first, their count padded with empty slots to a multiple of R when
// inhibitory ones follow).  Each warp stages the sources of its current pair
// in its own shared memory, in pairs of sources, and every lane evaluates them
// against its targets, so one staged source pair (two shared-memory loads)
// serves 2R evaluations; when the round's target groups fit in fewer lanes
// they are padded to P = 2^k lanes and 32/P lanes share a group, walking
// interleaved slices of the sources (small leaves still fill the warp).
// The per-target sums of the 4 warps are added in a fixed order, so u is
// reproducible run to run.  Per pair, the warp reduces the box-pair
// attraction W(X,Y) = sum_t a_t sum_s w_s K(t,s) of each channel in single
// precision into a per-pair slot; a second kernel widens it into the double
// precision pair table.
//
// Arithmetic.  With k = log2(e)/sigma^2 and hats denoting sqrt(k)(position-c)
// for the geometric centre c of X,
//   w_s K(t,s) = 2^( 2 t^.s^ - |s^|^2 + log2 w_s ) * 2^(-|t^|^2),
// so a source is staged once per warp as (s^, -|s^|^2 + log2 w_s) for each
// channel and one evaluation is three FMAs, one EX2 on the SFU and one add;
// the FMAs and the add run as paired FP32 instructions over two sources.
// The first factor is at most 2^(|t^|^2 + 8), so the expanded form is used
// while |t^|^2 <= 20 for every target of X (leaves up to about 4.3 sigma
// wide; the exponent's rounding then stays near 1e-6 relative); wider leaves
// use the difference form (s^, log2 w_s) with |t^ - s^|^2.
#include <algorithm>
#include <cmath>

#include "msp_internal.cuh"

namespace msp {

namespace {

// the block's transposed per-pair W buffer (16 pairs x 32 lanes per warp, one
// padding column), set by the kernel before use
__shared__ float* s_wt;
__shared__ int32_t* s_wii;

constexpr int kNFWarps = 4;
constexpr int kNFThreads = kNFWarps * 32;
constexpr int kNFStage = 128;
constexpr int kNFMaxT = 32 * 4;    // targets per pass (3 or 4 per lane)
constexpr int kNFList = 128;       // target slots per round (one pass)
constexpr float kNFFastT2 = 20.f;  // largest |t^|^2 of the expanded form

__device__ inline float nf_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


struct NFArgs {
    const int32_t* seg_first;
    const int64_t* nseg;         // segment count (device memory)
    const int32_t* order;        // segments, longest first
    const int32_t* list_q;
    const int32_t* pX;
    const int2* src;             // per near-field pair (list order): Y's first point, count
    const uint8_t* nlevel;
    const uint64_t* nprefix;
    const int32_t* nfirst;
    const int32_t* ncount;
    const float4* pts;
    const float2* lw;
    float sqk, ox, oy, oz, side;
    int frame_level;             // > 0: box centres in each network's own frame
    float* u;
    float2* w32;                 // per near-field pair (list order): W of E and I
    unsigned long long* work;
};

// the targets of a lane (R of them, one channel), each coordinate broadcast
// into both halves of a register pair; their scale factors and axon weights
// sit in shared memory by slot (s_scale, s_fa)
template <int R>
struct Tgts {
    float2 x[R], y[R], z[R];  // 2 t^ (expanded form) or t^ (difference form)
    int ch;                   // 0 excitatory, 1 inhibitory
    int slot0;                // slot of target 0 (targets r at slot0 + r)
};

// per slot of the current pass: 2^(-|t^|^2) (or 1), a_t times it (0 for
// padding) and the target list (sorted index, -1 for padding; slots past the
// pass hold stale entries whose results are discarded), set by the kernel
// before use
__shared__ float* s_scale;
__shared__ float* s_fa;
__shared__ const int32_t* s_tl;
// per thread and target r: the compensation of the Kahan sum of the target's
// per-pair sums, targets 2i and 2i+1 as one float2 at [i * kNFThreads +
// thread] (kept in shared memory: the kernel's registers are taken by the
// evaluation loop)
__shared__ float* s_cmp;

// A warp's staged sources, in pairs: pair j (sources 2j, 2j+1) is the float4
// (x0, x1, y0, y1) at [j] and (z0, z1, c0, c1) at [kNFZE + j] for the
// excitatory and at [kNFZI + j] for the inhibitory channel (one float4 apart
// from a multiple of 128 bytes, so that the two channels' lanes read different
// banks), c = -|s^|^2 + log2 w (expanded
// form) or log2 w (difference form); an odd count is padded with c = -inf.
constexpr int kNFZE = kNFStage / 2, kNFZI = kNFStage + 1;
constexpr int kNFStageFloats = 4 * (kNFZI + kNFStage / 2);

// Evaluate the staged source pairs [0, mp) (lane slice ksl of `slices`)
// against the lane's R targets.  MODE 0: expanded form; 1: expanded, skipping
// the target itself; 2: difference form; 3: difference form, skipping the
// target.  In the expanded form one evaluation of two sources is three paired
// FMAs, two EX2 and one paired add (the paired FP32 instructions take one
// issue slot for two results); the difference form stages -s^ and takes
// t^ - s^ first.  In MODE 1 and 3 target r sits at position
// s_tl[slot0 + r] - base among the staged sources (out of range when it is not
// among them).
template <int R, int MODE>
__device__ __forceinline__ float2 nf_term(const Tgts<R>& tg, int r, const float4& A,
                                          const float4& B) {
    float2 E;
    if (MODE <= 1) {
        E = __ffma2_rn(tg.x[r], make_float2(A.x, A.y),
                       __ffma2_rn(tg.y[r], make_float2(A.z, A.w),
                                  __ffma2_rn(tg.z[r], make_float2(B.x, B.y),
                                             make_float2(B.z, B.w))));
    } else {
        const float2 dx = __fadd2_rn(tg.x[r], make_float2(A.x, A.y));
        const float2 dy = __fadd2_rn(tg.y[r], make_float2(A.z, A.w));
        const float2 dz = __fadd2_rn(tg.z[r], make_float2(B.x, B.y));
        E = __ffma2_rn(make_float2(-dx.x, -dx.y), dx,
                       __ffma2_rn(make_float2(-dy.x, -dy.y), dy,
                                  __ffma2_rn(make_float2(-dz.x, -dz.y), dz,
                                             make_float2(B.z, B.w))));
    }
    return make_float2(nf_ex2(E.x), nf_ex2(E.y));
}

template <int R, int MODE>
__device__ __forceinline__ void nf_eval(const float4* st, int mp, int ksl, int slices,
                                        const Tgts<R>& tg, int32_t base, float (&part)[R]) {
    constexpr bool kSkip = MODE == 1 || MODE == 3;
    constexpr int NA = R == 2 ? 2 : 1;   // accumulator pairs per target
    float2 P[R][NA];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NA; ++k) P[r][k] = make_float2(0.f, 0.f);
    const float4* xy = st;
    const float4* zc = st + (tg.ch ? kNFZI : kNFZE);
    int j = ksl;
    // two source pairs per iteration (one when skipping: register budget)
    for (; !kSkip && j + slices < mp; j += 2 * slices) {
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int jj = j + v * slices;
            const float4 A = xy[jj], B = zc[jj];
#pragma unroll
            for (int r = 0; r < R; ++r)
                P[r][v % NA] = __fadd2_rn(P[r][v % NA], nf_term<R, MODE>(tg, r, A, B));
        }
    }
    for (; kSkip && j < mp; j += slices) {
        const float4 A = xy[j], B = zc[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 X = nf_term<R, MODE>(tg, r, A, B);
            const int d = s_tl[tg.slot0 + r] - base - 2 * j;
            X.x = d == 0 ? 0.f : X.x;
            X.y = d == 1 ? 0.f : X.y;
            P[r][0] = __fadd2_rn(P[r][0], X);
        }
    }
    if (!kSkip && j < mp) {
        const float4 A = xy[j], B = zc[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            P[r][0] = __fadd2_rn(P[r][0], nf_term<R, MODE>(tg, r, A, B));
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float t = P[r][0].x + P[r][0].y;
        if (NA == 2) t += P[r][NA - 1].x + P[r][NA - 1].y;
        part[r] += t;
    }
}

// The expanded form when every lane walks all staged source pairs (one slice):
// unit-stride pointers, two source pairs per iteration.
template <int R>
__device__ __forceinline__ void nf_eval_unit(const float4* st, int mp, const Tgts<R>& tg,
                                             float (&part)[R]) {
    constexpr int NA = R == 2 ? 2 : 1;
    float2 P[R][NA];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NA; ++k) P[r][k] = make_float2(0.f, 0.f);
    const float4* xp = st;
    const float4* zp = st + (tg.ch ? kNFZI : kNFZE);
    const float4* const xe = st + (mp & ~1);
    for (; xp < xe; xp += 2, zp += 2) {
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const float4 A = xp[v], B = zp[v];
#pragma unroll
            for (int r = 0; r < R; ++r)
                P[r][v % NA] = __fadd2_rn(P[r][v % NA], nf_term<R, 0>(tg, r, A, B));
        }
    }
    if (mp & 1) {
        const float4 A = xp[0], B = zp[0];
#pragma unroll
        for (int r = 0; r < R; ++r) P[r][0] = __fadd2_rn(P[r][0], nf_term<R, 0>(tg, r, A, B));
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float t = P[r][0].x + P[r][0].y;
        if (NA == 2) t += P[r][NA - 1].x + P[r][NA - 1].y;
        part[r] += t;
    }
}

// the pairs of segment [i0, i1) that belong to warp w, for a lane holding R targets
template <int R>
__device__ __forceinline__ void nf_pairs(const NFArgs& a, int32_t i0, int32_t i1, int32_t tf,
                                         bool fast, float cx, float cy, float cz, int ksl,
                                         int slices, const Tgts<R>& tg, float (&acc)[R],
                                         float4* stw, unsigned long long& evals, int nreal) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float (*wt)[33] = reinterpret_cast<float (*)[33]>(s_wt + w * 16 * 33);
    int32_t* wii = s_wii + w * 16;
    const unsigned imask = __ballot_sync(0xffffffffu, tg.ch != 0);   // inhibitory lanes
    for (int32_t cb = i0 + w; cb < i1; cb += 32 * kNFWarps) {
        // metadata of the warp's next 32 pairs, one per lane
        int32_t mi = cb + kNFWarps * lane, msf = 0, msc = 0;
        if (mi < i1) {
            const int2 m = a.src[mi];
            msf = m.x;
            msc = m.y;
        }
        const int nb = min(32, (i1 - cb + kNFWarps - 1) / kNFWarps);
        for (int r = 0; r < nb; ++r) {
            const int32_t ii = __shfl_sync(0xffffffffu, mi, r);
            const int32_t sf = __shfl_sync(0xffffffffu, msf, r);
            const int32_t sc = __shfl_sync(0xffffffffu, msc, r);
            const bool self = sf == tf;
            float part[R];
#pragma unroll
            for (int k = 0; k < R; ++k) part[k] = 0.f;
            for (int32_t sb = 0; sb < sc; sb += kNFStage) {
                const int m = min(kNFStage, sc - sb);
                const int mp = (m + 1) >> 1;
                __syncwarp();
                // a lane stages source pairs (2j, 2j+1) with paired FP32 (the
                // same rounding per source as the scalar form) and three
                // 16-byte stores; an odd count's last source is padding
                // (coordinates 0, c = -inf)
                const float2 nc = make_float2(-cx, -cx), ncy = make_float2(-cy, -cy),
                             ncz = make_float2(-cz, -cz), k2 = make_float2(a.sqk, a.sqk);
                for (int j = lane; j < mp; j += 32) {
                    const int e = 2 * j;
                    const bool two = e + 1 < m;
                    const float4 S0 = a.pts[sf + sb + e];
                    const float2 L0 = a.lw[sf + sb + e];
                    const float4 S1 = two ? a.pts[sf + sb + e + 1] : S0;
                    const float2 L1 = two ? a.lw[sf + sb + e + 1] : L0;
                    float2 sx = __fmul2_rn(__fadd2_rn(make_float2(S0.x, S1.x), nc), k2);
                    float2 sy = __fmul2_rn(__fadd2_rn(make_float2(S0.y, S1.y), ncy), k2);
                    float2 sz = __fmul2_rn(__fadd2_rn(make_float2(S0.z, S1.z), ncz), k2);
                    float2 n2 = make_float2(0.f, 0.f);
                    if (fast) {
                        const float2 q = __ffma2_rn(sx, sx, __ffma2_rn(sy, sy, __fmul2_rn(sz, sz)));
                        n2 = make_float2(-q.x, -q.y);
                    }
                    float2 cE = __fadd2_rn(n2, make_float2(L0.x, L1.x));
                    float2 cI = __fadd2_rn(n2, make_float2(L0.y, L1.y));
                    if (!fast) {
                        sx = make_float2(-sx.x, -sx.y);
                        sy = make_float2(-sy.x, -sy.y);
                        sz = make_float2(-sz.x, -sz.y);
                    }
                    if (!two) {
                        sx.y = sy.y = sz.y = 0.f;
                        cE.y = cI.y = -INFINITY;
                    }
                    stw[j] = make_float4(sx.x, sx.y, sy.x, sy.y);
                    stw[kNFZE + j] = make_float4(sz.x, sz.y, cE.x, cE.y);
                    stw[kNFZI + j] = make_float4(sz.x, sz.y, cI.x, cI.y);
                }
                __syncwarp();
                if (fast) {
                    if (self)             nf_eval<R, 1>(stw, mp, ksl, slices, tg, sf + sb, part);
                    else if (slices == 1) nf_eval_unit<R>(stw, mp, tg, part);
                    else                  nf_eval<R, 0>(stw, mp, ksl, slices, tg, sf + sb, part);
                } else {
                    if (self) nf_eval<R, 3>(stw, mp, ksl, slices, tg, sf + sb, part);
                    else      nf_eval<R, 2>(stw, mp, ksl, slices, tg, sf + sb, part);
                }
            }
            // the pair's sum joins the target's total by Kahan's compensated
            // summation (the compensation holds what the running total
            // gained by rounding)
            float v = 0.f;
            // two targets at a time in paired FP32 (the same rounding per
            // target); the compensations of targets k, k+1 as one float2
#pragma unroll
            for (int k = 0; k < R; k += 2) {
                float2* cp = reinterpret_cast<float2*>(s_cmp) + (k >> 1) * kNFThreads + threadIdx.x;
                if (k + 1 < R) {
                    const float2 c2 = *cp, p2 = make_float2(part[k], part[k + 1]);
                    const float2 a2 = make_float2(acc[k], acc[k + 1]);
                    const float2 y = __fadd2_rn(p2, make_float2(-c2.x, -c2.y));
                    const float2 t2 = __fadd2_rn(a2, y);
                    const float2 d = __fadd2_rn(t2, make_float2(-a2.x, -a2.y));
                    *cp = __fadd2_rn(d, make_float2(-y.x, -y.y));
                    acc[k] = t2.x;
                    acc[k + 1] = t2.y;
                } else {
                    float* cs = reinterpret_cast<float*>(cp);
                    const float y = __fsub_rn(part[k], *cs);
                    const float t2 = __fadd_rn(acc[k], y);
                    *cs = __fsub_rn(__fsub_rn(t2, acc[k]), y);
                    acc[k] = t2;
                }
            }
#pragma unroll
            for (int k = 0; k < R; ++k) v = fmaf(s_fa[tg.slot0 + k], part[k], v);
            // W(X,Y) of each channel: every lane's term goes into a transposed
            // buffer; every 16 pairs the warp sums the rows (half a row per
            // lane, then one shuffle) and adds them to the pairs' slots
            const int slot = r & 15;
            wt[slot][lane] = v;
            if (lane == 0) wii[slot] = ii;
            if (slot == 15 || r == nb - 1) {
                __syncwarp();
                const int row = lane & 15, half = lane >> 4;
                float sE = 0.f, sI = 0.f;
#pragma unroll 4
                for (int c = 0; c < 16; ++c) {
                    const int col = half * 16 + c;
                    const float v2 = wt[row][col];
                    if ((imask >> col) & 1u) sI += v2; else sE += v2;
                }
                sE += __shfl_down_sync(0xffffffffu, sE, 16);
                sI += __shfl_down_sync(0xffffffffu, sI, 16);
                // fire-and-forget adds (a pair's slot is only touched by
                // this warp, once per round of targets, in round order)
                if (lane <= slot) atomicAdd(&a.w32[wii[lane]], make_float2(sE, sI));
                __syncwarp();
            }
            evals += (unsigned long long)sc * (unsigned long long)nreal;
        }
    }
}

// One pass over the targets tl[0, nt) (nt <= R * 32; tl[k] < 0 is padding);
// nreal of them are real.  A lane holds the R targets of slots R j .. R j + R-1
// (one channel); when they fit in fewer lanes the target groups are padded to
// a power of two P and 32/P lanes share a group, each walking an interleaved
// slice of the sources.
template <int R>
__device__ __forceinline__ void nf_targets(const NFArgs& a, const int32_t* tl, int nt, int nreal,
                                           int32_t i0, int32_t i1, int32_t tf, bool fast, float cx,
                                           float cy, float cz, float4* stw,
                                           float (*red)[kNFMaxT], unsigned long long& evals) {
    static_assert(R >= 2 && R <= 4, "two to four targets per lane (the compensation buffer holds four)");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lg = 0;
    while ((1 << lg) < (nt + R - 1) / R) ++lg;
    const int npr = 1 << lg;                // lanes per slice (target groups)
    const int slices = 32 >> lg;
    const int j = lane & (npr - 1);
    const int ksl = lane >> lg;
    Tgts<R> tg;
    tg.slot0 = R * j;
    float acc[R];
    {
        // the channel of the lane's first slot (all its slots share it)
        const int32_t t0 = tg.slot0 < nt ? tl[tg.slot0] : -1;
        tg.ch = t0 >= 0 ? (pk_type(__float_as_uint(a.pts[t0].w)) ? 1 : 0) : 0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int slot = tg.slot0 + r;
        const int32_t ts = slot < nt ? tl[slot] : -1;
        const bool valid = ts >= 0;
        const int32_t t = valid ? ts : tl[0];          // tl[0] is always a real target
        const float4 T = a.pts[t];
        const uint32_t tw = __float_as_uint(T.w);
        const float hx = (T.x - cx) * a.sqk, hy = (T.y - cy) * a.sqk, hz = (T.z - cz) * a.sqk;
        const float f2 = fast ? 2.f : 1.f;
        tg.x[r] = make_float2(f2 * hx, f2 * hx);
        tg.y[r] = make_float2(f2 * hy, f2 * hy);
        tg.z[r] = make_float2(f2 * hz, f2 * hz);
        acc[r] = 0.f;
        reinterpret_cast<float*>(reinterpret_cast<float2*>(s_cmp) + (r >> 1) * kNFThreads +
                                 threadIdx.x)[r & 1] = 0.f;
        if (w == 0 && ksl == 0) {
            const float sc = fast ? nf_ex2(-fmaf(hx, hx, fmaf(hy, hy, hz * hz))) : 1.f;
            s_scale[slot] = sc;
            s_fa[slot] = valid ? (float)pk_axon(tw) * sc : 0.f;
        }
    }
    __syncthreads();
    nf_pairs<R>(a, i0, i1, tf, fast, cx, cy, cz, ksl, slices, tg, acc, stw, evals, nreal);
    // the compensated totals, then the slices of a target group and the 4
    // warps in a fixed order
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[r] = __fsub_rn(acc[r], reinterpret_cast<float*>(reinterpret_cast<float2*>(s_cmp) +
                                                             (r >> 1) * kNFThreads +
                                                             threadIdx.x)[r & 1]);
        for (int o = npr; o < 32; o <<= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    }
    if (ksl == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) red[w][tg.slot0 + r] = acc[r];
    }
    __syncthreads();
    if (w == 0 && ksl == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int slot = tg.slot0 + r;
            const int32_t t = slot < nt ? tl[slot] : -1;
            if (t >= 0) {
                float sacc = red[0][slot];
#pragma unroll
                for (int k = 1; k < kNFWarps; ++k) sacc += red[k][slot];
                a.u[t] += sacc * s_scale[slot];
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kNFWarps * 32, 7) k_near_field(NFArgs a) {
    __shared__ float4 st[kNFWarps][kNFStageFloats / 4];
    __shared__ float red[kNFWarps][kNFMaxT];
    __shared__ int32_t tl[kNFList];
    __shared__ int s_nt, s_nreal, s_pos, s_R;
    __shared__ float wt_all[kNFWarps][16][33];
    __shared__ int32_t wii_all[kNFWarps][16];
    __shared__ float scale_all[kNFMaxT], fa_all[kNFMaxT];
    __shared__ __align__(16) float cmp_all[4 * kNFThreads];
    s_cmp = cmp_all;
    s_wt = &wt_all[0][0][0];
    s_wii = &wii_all[0][0];
    s_scale = scale_all;
    s_fa = fa_all;
    s_tl = tl;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* stw = st[w];
    const int64_t nseg = *a.nseg;
    for (int64_t b = blockIdx.x; b < nseg; b += gridDim.x) {
        const int32_t sg = a.order[b];
        const int32_t i0 = a.seg_first[sg], i1 = a.seg_first[sg + 1];
        const int32_t X = a.pX[a.list_q[i0]];
        const int32_t tf = a.nfirst[X], tc = a.ncount[X];
        const uint64_t pre = a.nprefix[X];
        const float bs = ldexpf(a.side, -(int)a.nlevel[X]);
        const int lX = (int)a.nlevel[X];
        const float cx = a.ox + ((float)box_axis(pre, 0, lX, a.frame_level) + 0.5f) * bs;
        const float cy = a.oy + ((float)box_axis(pre, 1, lX, a.frame_level) + 0.5f) * bs;
        const float cz = a.oz + ((float)box_axis(pre, 2, lX, a.frame_level) + 0.5f) * bs;
        // the expanded exponent needs |t^|^2 <= kNFFastT2 for every target of X
        const bool fast = 0.75f * a.sqk * a.sqk * bs * bs <= kNFFastT2;
        unsigned long long evals = 0;
        int32_t pos = 0;
        for (;;) {
            // warp 0 collects up to kNFList - 3 targets with vacant axons from
            // pos on: first walk counts them per channel and finds where the
            // round ends, second walk writes the excitatory ones, padding
            // entries up to a multiple of R if inhibitory ones follow, then
            // the inhibitory ones (a lane's R slots share a channel)
            if (w == 0) {
                int nt = 0, nE = 0;
                int32_t p = pos;
                while (p < tc && nt < kNFList - 3) {
                    const int32_t t = tf + p + lane;
                    const uint32_t tw = p + lane < tc ? __float_as_uint(a.pts[t].w) : 0u;
                    const bool act = pk_axon(tw) > 0;
                    const unsigned mask = __ballot_sync(0xffffffffu, act);
                    const unsigned emask = __ballot_sync(0xffffffffu, act && !pk_type(tw));
                    const int room = kNFList - 3 - nt;
                    if (__popc(mask) > room) {
                        // stop after the lane of the room-th target
                        int last = 0;
                        for (int bb = 0, c = 0; bb < 32; ++bb)
                            if ((mask >> bb) & 1u) {
                                if (c == room - 1) last = bb;
                                ++c;
                            }
                        const unsigned keep = last == 31 ? 0xffffffffu : ((1u << (last + 1)) - 1u);
                        nt += room;
                        nE += __popc(emask & keep);
                        p += last + 1;
                        break;
                    }
                    nt += __popc(mask);
                    nE += __popc(emask);
                    p += 32;
                }
                const int32_t pend = min(p, tc);
                const int nI = nt - nE;
                // R targets per lane (3 or 4), by the cost of a pass per
                // staged source pair: the iterations of a lane (npr / 32 with
                // npr lanes per slice, a power of two) times the cost of one
                // iteration, the larger of the shared-memory delivery (two
                // 16-byte loads per lane: 8 cycles) and the EX2 unit (2 R
                // results per lane at ~30 per SM per clock)
                auto pad_for = [&](int R) { return nI > 0 ? (R - nE % R) % R : 0; };
                auto cost_for = [&](int R) {
                    const int g = (nt + pad_for(R) + R - 1) / R;
                    if (g > 32) return 1 << 30;
                    int npr = 1;
                    while (npr < g) npr <<= 1;
                    return npr * max(53 * R, 200);
                };
                const int R = cost_for(3) <= cost_for(4) ? 3 : 4;
                const int pad = pad_for(R);
                int we = 0, wi = nE + pad;
                for (int32_t q = pos; q < pend; q += 32) {
                    const int32_t t = tf + q + lane;
                    const uint32_t tw = q + lane < pend ? __float_as_uint(a.pts[t].w) : 0u;
                    const bool act = pk_axon(tw) > 0;
                    const bool isE = act && !pk_type(tw);
                    const bool isI = act && pk_type(tw);
                    const unsigned me = __ballot_sync(0xffffffffu, isE);
                    const unsigned mI = __ballot_sync(0xffffffffu, isI);
                    const unsigned lt = (1u << lane) - 1u;
                    if (isE) tl[we + __popc(me & lt)] = t;
                    if (isI) tl[wi + __popc(mI & lt)] = t;
                    we += __popc(me);
                    wi += __popc(mI);
                }
                if (lane < pad) tl[nE + lane] = -1;
                if (lane == 0) {
                    s_nt = nt + pad;
                    s_nreal = nt;
                    s_R = R;
                    s_pos = pend;
                }
            }
            __syncthreads();
            const int ntl = s_nt, R = s_R, nreal = s_nreal;
            pos = s_pos;
            __syncthreads();
            if (ntl == 0) break;
            if (R == 4)
                nf_targets<4>(a, tl, ntl, nreal, i0, i1, tf, fast, cx, cy, cz, stw, red, evals);
            else
                nf_targets<3>(a, tl, ntl, nreal, i0, i1, tf, fast, cx, cy, cz, stw, red, evals);
            if (pos >= tc) break;
        }
        if (lane == 0 && evals) atomicAdd(a.work, evals);
    }
}

// Segment order, longest first: key = 16-bit complement of 1024 log2(work),
// work = targets of X times the sources of its partner leaves (an estimate:
// every neuron of X counts as a target).  Also the source range of every
// pair in list order, so the near field reads one int2 per pair.
__global__ void k_seg_order_keys(const int32_t* __restrict__ seg_first,
                                 const int64_t* __restrict__ nseg_dev,
                                 const int32_t* __restrict__ list_q,
                                 const int32_t* __restrict__ pX, const int32_t* __restrict__ pY,
                                 const int32_t* __restrict__ nfirst,
                                 const int32_t* __restrict__ ncount, uint64_t* __restrict__ key,
                                 int32_t* __restrict__ val, int2* __restrict__ src) {
    // one warp per segment, lanes over its pairs
    const int64_t nseg = *nseg_dev;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t sg = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); sg < nseg;
         sg += nw) {
        const int32_t i0 = seg_first[sg], i1 = seg_first[sg + 1];
        float srcs = 0.f;
        for (int32_t i = i0 + lane; i < i1; i += 32) {
            const int32_t Y = pY[list_q[i]];
            const int32_t cnt = ncount[Y];
            src[i] = make_int2(nfirst[Y], cnt);
            srcs += (float)cnt;
        }
        for (int o = 16; o > 0; o >>= 1) srcs += __shfl_xor_sync(0xffffffffu, srcs, o);
        if (lane == 0) {
            const float work = srcs * (float)ncount[pX[list_q[i0]]];
            const float lg = log2f(work + 1.f);
            const uint32_t q = min(0xffffu, (uint32_t)(lg * 1024.f));
            key[sg] = (uint64_t)(0xffffu - q);
            val[sg] = (int32_t)sg;
        }
    }
}

__global__ void k_zero_w(float2* __restrict__ w32, const int64_t* __restrict__ n_dev) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        w32[i] = make_float2(0.f, 0.f);
}

// the single precision per-pair attractions into the pair table (double-FP32)
__global__ void k_widen_w(const int32_t* __restrict__ list_q, const float2* __restrict__ w32,
                          const int64_t* __restrict__ n_dev, float4* __restrict__ pw) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = w32[i];
        pw[list_q[i]] = make_float4(v.x, 0.f, v.y, 0.f);
    }
}

}  // namespace

void launch_near_field(msp_ctx& c, const int32_t* seg_first, const int64_t* nseg_dev,
                       int64_t nseg_cap, const int32_t* list_q, const int64_t* nlist_dev,
                       int64_t nlist_cap, float* u_sorted, unsigned long long* work,
                       bool keep_order, cudaStream_t s) {
    if (nseg_cap <= 0 || nlist_cap <= 0) return;
    const msp_config& cfg = c.cfg;
    float2* w32 = c.nf_w32.ensure<float2>((size_t)nlist_cap);
    const int gl = (int)std::max<int64_t>(1, (int64_t)c.sm_count * 8);
    k_zero_w<<<gl, 256, 0, s>>>(w32, nlist_dev);
    MSP_LAUNCH("zero_w");
    // longest segments first
    uint64_t* ok0 = c.nf_okey0.ensure<uint64_t>((size_t)nseg_cap);
    uint64_t* ok1 = c.nf_okey1.ensure<uint64_t>((size_t)nseg_cap);
    int32_t* ov0 = c.nf_oval0.ensure<int32_t>((size_t)nseg_cap);
    int32_t* ov1 = c.nf_oval1.ensure<int32_t>((size_t)nseg_cap);
    int2* src = c.nf_src.ensure<int2>((size_t)nlist_cap);
    // the order and the source ranges depend on the lists only: kept when
    // the lists are (keep_order)
    if (!keep_order) {
        k_seg_order_keys<<<(int)std::max<int64_t>(1, (int64_t)c.sm_count * 16), 128, 0, s>>>(
            seg_first, nseg_dev, list_q, c.pr_X.get<int32_t>(), c.pr_Y.get<int32_t>(),
            c.nd_first.get<int32_t>(), c.nd_count.get<int32_t>(), ok0, ov0, src);
        MSP_LAUNCH("seg_order_keys");
        radix_sort_dev(c, ok0, ov0, ok1, ov1, nseg_dev, nseg_cap, 16, s);
    }
    NFArgs a;
    a.seg_first = seg_first;
    a.nseg = nseg_dev;
    a.order = ov0;
    a.list_q = list_q;
    a.pX = c.pr_X.get<int32_t>();
    a.src = src;
    a.nlevel = c.nd_level.get<uint8_t>();
    a.nprefix = c.nd_prefix.get<uint64_t>();
    a.nfirst = c.nd_first.get<int32_t>();
    a.ncount = c.nd_count.get<int32_t>();
    a.pts = c.pts.get<float4>();
    a.lw = c.lw.get<float2>();
    a.sqk = (float)std::sqrt(1.4426950408889634 / (cfg.sigma * cfg.sigma));
    const bool framed = c.frame_level > 0;
    a.ox = framed ? 0.f : cfg.origin[0];
    a.oy = framed ? 0.f : cfg.origin[1];
    a.oz = framed ? 0.f : cfg.origin[2];
    a.side = cfg.side;
    a.frame_level = c.frame_level;
    a.u = u_sorted;
    a.w32 = w32;
    a.work = work;
    // one block per segment; blocks past the device count return at once
    int grid = (int)std::min<int64_t>(nseg_cap, 1 << 30);
    k_near_field<<<grid, kNFWarps * 32, 0, s>>>(a);
    MSP_LAUNCH("near_field");
    k_widen_w<<<gl, 256, 0, s>>>(list_q, w32, nlist_dev, c.pr_w.get<float4>());
    MSP_LAUNCH("widen_w");
}

}  // namespace msp
