// msp_nearfield.cu -- step a9: the exact near field (Eq. 8) over the
// near-field leaf pairs of the dual traversal, which dominates the step.
//
// Work unit: one target leaf X (one block of 4 warps) and all its partner
// leaves Y (a contiguous segment of the pair list sorted by X).  The block
// first collects the targets of X with vacant axons (up to 64 per pass); the
// warps then take the partner pairs round-robin.  Each warp stages the sources
// of its current pair in its own shared memory and every lane evaluates them
// against its targets:
//   up to 32 targets: padded to T = 2^k, 32/T lanes per target walking
//                     interleaved slices of the sources (small leaves still
//                     fill the warp);
//   33..64 targets:   2 targets per lane, every lane walks all sources (each
//                     staged source is used twice).
// Capping a pass at 64 targets keeps the kernel at 64 registers (8 blocks of
// 4 warps per SM); larger leaves take several passes.
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
// channel and one evaluation is three FMAs, one EX2 on the SFU and one add.
// For leaves wider than about 2 sigma the expanded exponent could overflow,
// and the difference form (s^, log2 w_s) with |t^ - s^|^2 is used instead.
#include <algorithm>
#include <cmath>

#include "msp_internal.cuh"

namespace msp {

namespace {

// the block's transposed per-pair W buffer (16 pairs x 32 lanes per warp, one
// padding column), set by the kernel before use
__shared__ float2* s_wt;
__shared__ int32_t* s_wii;

constexpr int kNFWarps = 4;
constexpr int kNFStage = 64;
constexpr int kNFMaxT = 32 * 2;    // targets per pass (at most 2 per lane: 64 registers)

__device__ inline float nf_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct NFArgs {
    const int32_t* seg_first;
    const int64_t* nseg;         // segment count (device memory)
    const int32_t* list_q;
    const int32_t* pX;
    const int32_t* pY;
    const uint8_t* nlevel;
    const uint64_t* nprefix;
    const int32_t* nfirst;
    const int32_t* ncount;
    const float4* pts;
    const float2* lw;
    float sqk, ox, oy, oz, side;
    float* u;
    float2* w32;                 // per near-field pair (list order): W of E and I
    unsigned long long* work;
};

// one target of a lane
struct Tgt {
    float x, y, z;     // 2 t^ (expanded form) or t^ (difference form)
    float scale;       // 2^(-|t^|^2) or 1
    float fa;          // a_t * scale, 0 for padding
    int32_t t;         // sorted index, -1 for padding
    int ch;            // 0 excitatory, 1 inhibitory
};

// Evaluate the staged sources [0, m) (lane slice ksl of `slices`) against the
// lane's R targets.  MODE 0: expanded exponent; 1: expanded, skipping the
// target itself; 2: difference form, skipping the target itself.
template <int R, int MODE>
__device__ __forceinline__ void nf_eval(const float4* st, int m, int ksl, int slices,
                                        const Tgt (&tg)[R], int32_t base, float (&part)[R]) {
    constexpr int U = R == 1 ? 4 : (R == 2 ? 2 : 1);
    float p[R][U];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int v = 0; v < U; ++v) p[r][v] = 0.f;
    int e = ksl;
    if (MODE == 0) {
        for (; e + (U - 1) * slices < m; e += U * slices) {
#pragma unroll
            for (int v = 0; v < U; ++v) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float4 A = st[2 * (e + v * slices) + tg[r].ch];
                    p[r][v] += nf_ex2(fmaf(tg[r].x, A.x, fmaf(tg[r].y, A.y, fmaf(tg[r].z, A.z, A.w))));
                }
            }
        }
        for (; e < m; e += slices) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float4 A = st[2 * e + tg[r].ch];
                p[r][0] += nf_ex2(fmaf(tg[r].x, A.x, fmaf(tg[r].y, A.y, fmaf(tg[r].z, A.z, A.w))));
            }
        }
    } else {
        for (; e < m; e += slices) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float4 A = st[2 * e + tg[r].ch];
                float v;
                if (MODE == 1) {
                    v = nf_ex2(fmaf(tg[r].x, A.x, fmaf(tg[r].y, A.y, fmaf(tg[r].z, A.z, A.w))));
                } else {
                    float dx = tg[r].x - A.x, dy = tg[r].y - A.y, dz = tg[r].z - A.z;
                    v = nf_ex2(A.w - fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                }
                p[r][0] += base + e == tg[r].t ? 0.f : v;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < U; ++v) s += p[r][v];
        part[r] += s;
    }
}

// the pairs of segment [i0, i1) that belong to warp w, for a lane holding R targets
template <int R>
__device__ __forceinline__ void nf_pairs(const NFArgs& a, int32_t i0, int32_t i1, int32_t tf,
                                         bool fast, float cx, float cy, float cz, int ksl,
                                         int slices, const Tgt (&tg)[R], float (&acc)[R],
                                         float4* stw, unsigned long long& evals, int nt) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 (*wt)[33] = reinterpret_cast<float2 (*)[33]>(s_wt + w * 16 * 33);
    int32_t* wii = s_wii + w * 16;
    for (int32_t cb = i0 + w; cb < i1; cb += 32 * kNFWarps) {
        // metadata of the warp's next 32 pairs, one per lane
        int32_t mi = cb + kNFWarps * lane, msf = 0, msc = 0;
        if (mi < i1) {
            int32_t Y = a.pY[a.list_q[mi]];
            msf = a.nfirst[Y];
            msc = a.ncount[Y];
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
                __syncwarp();
                for (int e = lane; e < m; e += 32) {
                    float4 S = a.pts[sf + sb + e];
                    float2 L = a.lw[sf + sb + e];
                    float sx = (S.x - cx) * a.sqk, sy = (S.y - cy) * a.sqk, sz = (S.z - cz) * a.sqk;
                    float n2 = fast ? -fmaf(sx, sx, fmaf(sy, sy, sz * sz)) : 0.f;
                    stw[2 * e] = make_float4(sx, sy, sz, n2 + L.x);
                    stw[2 * e + 1] = make_float4(sx, sy, sz, n2 + L.y);
                }
                __syncwarp();
                if (fast && !self)
                    nf_eval<R, 0>(stw, m, ksl, slices, tg, sf + sb, part);
                else if (fast)
                    nf_eval<R, 1>(stw, m, ksl, slices, tg, sf + sb, part);
                else
                    nf_eval<R, 2>(stw, m, ksl, slices, tg, sf + sb, part);
            }
            float vE = 0.f, vI = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                acc[k] += part[k];
                float v = tg[k].fa * part[k];
                if (tg[k].ch) vI += v; else vE += v;
            }
            // W(X,Y) of each channel: every lane's term goes into a transposed
            // buffer; every 16 pairs the warp sums the rows (half a row per
            // lane, then one shuffle) and adds them to the pairs' slots
            const int slot = r & 15;
            wt[slot][lane] = make_float2(vE, vI);
            if (lane == 0) wii[slot] = ii;
            if (slot == 15 || r == nb - 1) {
                __syncwarp();
                const int row = lane & 15, half = lane >> 4;
                float2 s2 = make_float2(0.f, 0.f);
#pragma unroll 4
                for (int c = 0; c < 16; ++c) {
                    float2 v2 = wt[row][half * 16 + c];
                    s2.x += v2.x;
                    s2.y += v2.y;
                }
                s2.x += __shfl_down_sync(0xffffffffu, s2.x, 16);
                s2.y += __shfl_down_sync(0xffffffffu, s2.y, 16);
                if (lane <= slot) {
                    const int32_t pi = wii[lane];
                    float2 cur = a.w32[pi];
                    a.w32[pi] = make_float2(cur.x + s2.x, cur.y + s2.y);
                }
                __syncwarp();
            }
            evals += (unsigned long long)sc * (unsigned long long)nt;
        }
    }
}

template <int R>
__device__ __forceinline__ void nf_targets(const NFArgs& a, const int32_t* tl, int nt, int32_t i0,
                                           int32_t i1, int32_t tf, bool fast, float cx, float cy,
                                           float cz, float4* stw, float (*red)[kNFMaxT],
                                           unsigned long long& evals) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lg = 0, ntp = 32;
    if (R == 1) {
        while ((1 << lg) < nt) ++lg;
        ntp = 1 << lg;
    }
    const int slices = R == 1 ? 32 >> lg : 1;
    const int j = R == 1 ? (lane & (ntp - 1)) : lane;
    const int ksl = R == 1 ? lane >> lg : 0;
    Tgt tg[R];
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int slot = j + 32 * r;
        const bool valid = slot < nt;
        const int32_t t = valid ? tl[slot] : tl[0];
        const float4 T = a.pts[t];
        const uint32_t tw = __float_as_uint(T.w);
        const float hx = (T.x - cx) * a.sqk, hy = (T.y - cy) * a.sqk, hz = (T.z - cz) * a.sqk;
        tg[r].x = fast ? 2.f * hx : hx;
        tg[r].y = fast ? 2.f * hy : hy;
        tg[r].z = fast ? 2.f * hz : hz;
        tg[r].scale = fast ? nf_ex2(-fmaf(hx, hx, fmaf(hy, hy, hz * hz))) : 1.f;
        tg[r].fa = valid ? (float)pk_axon(tw) * tg[r].scale : 0.f;
        tg[r].t = valid ? t : -1;
        tg[r].ch = pk_type(tw) ? 1 : 0;
        acc[r] = 0.f;
    }
    nf_pairs<R>(a, i0, i1, tf, fast, cx, cy, cz, ksl, slices, tg, acc, stw, evals, nt);
    // slices of a target (R == 1), then the 4 warps in a fixed order
#pragma unroll
    for (int r = 0; r < R; ++r)
        for (int o = ntp; o < 32; o <<= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (ksl == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) red[w][j + 32 * r] = acc[r];
    }
    __syncthreads();
    if (w == 0 && ksl == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int slot = j + 32 * r;
            if (slot < nt) {
                float s = red[0][slot];
#pragma unroll
                for (int k = 1; k < kNFWarps; ++k) s += red[k][slot];
                a.u[tg[r].t] += s * tg[r].scale;
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kNFWarps * 32, 8) k_near_field(NFArgs a) {
    __shared__ float4 st[kNFWarps][2 * kNFStage];
    __shared__ float red[kNFWarps][kNFMaxT];
    __shared__ int32_t tl[kNFMaxT];
    __shared__ int s_nt, s_pos;
    __shared__ float2 wt_all[kNFWarps][16][33];
    __shared__ int32_t wii_all[kNFWarps][16];
    s_wt = &wt_all[0][0][0];
    s_wii = &wii_all[0][0];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* stw = st[w];
    const int64_t nseg = *a.nseg;
    for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const int32_t i0 = a.seg_first[sg], i1 = a.seg_first[sg + 1];
        const int32_t X = a.pX[a.list_q[i0]];
        const int32_t tf = a.nfirst[X], tc = a.ncount[X];
        const uint64_t pre = a.nprefix[X];
        const float bs = ldexpf(a.side, -(int)a.nlevel[X]);
        const float cx = a.ox + ((float)compact_by3(pre >> 2) + 0.5f) * bs;
        const float cy = a.oy + ((float)compact_by3(pre >> 1) + 0.5f) * bs;
        const float cz = a.oz + ((float)compact_by3(pre) + 0.5f) * bs;
        // the expanded exponent needs |t^|^2 <= 4 for every target of X
        const bool fast = 0.75f * a.sqk * a.sqk * bs * bs <= 4.f;
        unsigned long long evals = 0;
        int32_t pos = 0;
        for (;;) {
            // warp 0 collects up to 128 targets with vacant axons, from pos on
            if (w == 0) {
                int nt = 0;
                int32_t p = pos;
                while (p < tc && nt < kNFMaxT) {
                    const int32_t t = tf + p + lane;
                    const bool act = p + lane < tc && pk_axon(__float_as_uint(a.pts[t].w)) > 0;
                    const unsigned mask = __ballot_sync(0xffffffffu, act);
                    const int room = kNFMaxT - nt;
                    const int take = min(__popc(mask), room);
                    const int rank = __popc(mask & ((1u << lane) - 1u));
                    if (act && rank < take) tl[nt + rank] = t;
                    if (take < __popc(mask)) {
                        // stop after the lane of the last taken target
                        int last = 0;
                        for (int b = 0, c = 0; b < 32; ++b)
                            if ((mask >> b) & 1u) {
                                if (c == take - 1) last = b;
                                ++c;
                            }
                        p += last + 1;
                        nt += take;
                        break;
                    }
                    nt += take;
                    p += 32;
                }
                if (lane == 0) {
                    s_nt = nt;
                    s_pos = p;
                }
            }
            __syncthreads();
            const int nt = s_nt;
            pos = s_pos;
            __syncthreads();
            if (nt == 0) break;
            if (nt <= 32)
                nf_targets<1>(a, tl, nt, i0, i1, tf, fast, cx, cy, cz, stw, red, evals);
            else
                nf_targets<2>(a, tl, nt, i0, i1, tf, fast, cx, cy, cz, stw, red, evals);
            if (pos >= tc) break;
        }
        if (lane == 0 && evals) atomicAdd(a.work, evals);
    }
}

__global__ void k_zero_w(float2* __restrict__ w32, const int64_t* __restrict__ n_dev) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        w32[i] = make_float2(0.f, 0.f);
}

// the single precision per-pair attractions into the double precision table
__global__ void k_widen_w(const int32_t* __restrict__ list_q, const float2* __restrict__ w32,
                          const int64_t* __restrict__ n_dev, double2* __restrict__ pw) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = w32[i];
        pw[list_q[i]] = make_double2((double)v.x, (double)v.y);
    }
}

}  // namespace

void launch_near_field(msp_ctx& c, const int32_t* seg_first, const int64_t* nseg_dev,
                       int64_t nseg_cap, const int32_t* list_q, const int64_t* nlist_dev,
                       int64_t nlist_cap, float* u_sorted, unsigned long long* work,
                       cudaStream_t s) {
    if (nseg_cap <= 0 || nlist_cap <= 0) return;
    const msp_config& cfg = c.cfg;
    float2* w32 = c.nf_w32.ensure<float2>((size_t)nlist_cap);
    const int gl = (int)std::max<int64_t>(1, (int64_t)c.sm_count * 8);
    k_zero_w<<<gl, 256, 0, s>>>(w32, nlist_dev);
    MSP_LAUNCH("zero_w");
    NFArgs a;
    a.seg_first = seg_first;
    a.nseg = nseg_dev;
    a.list_q = list_q;
    a.pX = c.pr_X.get<int32_t>();
    a.pY = c.pr_Y.get<int32_t>();
    a.nlevel = c.nd_level.get<uint8_t>();
    a.nprefix = c.nd_prefix.get<uint64_t>();
    a.nfirst = c.nd_first.get<int32_t>();
    a.ncount = c.nd_count.get<int32_t>();
    a.pts = c.pts.get<float4>();
    a.lw = c.lw.get<float2>();
    a.sqk = (float)std::sqrt(1.4426950408889634 / (cfg.sigma * cfg.sigma));
    a.ox = cfg.origin[0];
    a.oy = cfg.origin[1];
    a.oz = cfg.origin[2];
    a.side = cfg.side;
    a.u = u_sorted;
    a.w32 = w32;
    a.work = work;
    // one block per segment; blocks past the device count return at once
    int grid = (int)std::min<int64_t>(nseg_cap, 1 << 30);
    k_near_field<<<grid, kNFWarps * 32, 0, s>>>(a);
    MSP_LAUNCH("near_field");
    k_widen_w<<<gl, 256, 0, s>>>(list_q, w32, nlist_dev, c.pr_w.get<double2>());
    MSP_LAUNCH("widen_w");
}

}  // namespace msp
