// msp_fmm.cu -- steps a5-a10: dual traversal with the separation / cutoff
// rule, Hermite coefficients (Eq. 7), Hermite-to-Taylor translation (Eq. 7
// composed with the Taylor expansion of Eq. 6), Taylor evaluation (Eq. 6), the
// exact near field (Eq. 8) and the box-pair attraction table; plus the
// all-pairs comparison path.
#include <cmath>

#include "msp_internal.cuh"

namespace msp {

struct Geo {
    long long g2[kMortonBits + 1];   // prune when sum of squared box gaps >= g2[level]
    int l_far;                       // boxes at level >= l_far may carry expansions
    long long m2l_min_pairs;
    int mac_mode;                    // 1: Algorithm 2's count rule
    int c1;                          // its dendrite threshold
    // per-network cutoffs (points in frames): the thresholds of the finer
    // box's network, [network][level], for levels at or below frame_level
    const long long* fg2;
    int frame_level;
    int64_t nf;
};

__device__ inline float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__constant__ float c_inv_fact[kMaxP] = {1.f, 1.f, 0.5f, 1.f / 6.f, 1.f / 24.f, 1.f / 120.f,
                                        1.f / 720.f, 1.f / 5040.f};

namespace {

struct NodeView {
    const uint8_t* level;
    const uint64_t* prefix;
    const int32_t* first;
    const int32_t* count;
    const int32_t* child_first;
    const uint8_t* nchild;
    const int4* sums;
};

// A pair is pruned by the cutoff only: a box pair without vacant axonal or
// dendritic elements contributes exactly zero (log2 0 = -inf in every term,
// or no target), so the lists depend on the positions alone and the step
// graph can keep them across steps.
__device__ inline uint8_t classify(const NodeView& nv, const Geo& geo, int32_t X, int32_t Y) {
    const int4 sy = nv.sums[Y];
    int lx = nv.level[X], ly = nv.level[Y];
    int lf = lx > ly ? lx : ly;
    uint64_t px = nv.prefix[X], py = nv.prefix[Y];
    long long gsum = 0, gmax = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        long long lox = (long long)compact_by3(px >> (2 - d)) << (lf - lx);
        long long hix = lox + (1ll << (lf - lx));
        long long loy = (long long)compact_by3(py >> (2 - d)) << (lf - ly);
        long long hiy = loy + (1ll << (lf - ly));
        long long g = 0;
        if (loy - hix > g) g = loy - hix;
        if (lox - hiy > g) g = lox - hiy;
        gsum += g * g;
        if (g > gmax) gmax = g;
    }
    long long thr = geo.g2[lf];
    if (geo.fg2 && lf >= geo.frame_level) {
        // both boxes in one network: its cutoff; in two networks: at least a
        // cell apart, beyond every network's cutoff
        const int64_t k = box_frame(lx == lf ? px : py, lf, geo.frame_level, geo.nf);
        thr = geo.fg2[k * (kMortonBits + 1) + lf];
    }
    if (gsum >= thr) return kPruned;
    const bool leafx = nv.child_first[X] < 0, leafy = nv.child_first[Y] < 0;
    const int lmin = lx < ly ? lx : ly;
    if (geo.mac_mode == 1) {
        // Algorithm 2: a leaf side is evaluated directly; an inner dendrite
        // box with more than c1 vacant dendrites is expanded; else direct
        // (boxes above l_far, which is 0 unless the points sit in frames,
        // are split)
        if (leafx && leafy) return kP2P;
        if (!leafx && !leafy && X != Y && lmin >= geo.l_far && sy.z + sy.w > geo.c1)
            return kFar;
        return kSplit;
    }
    if (lmin >= geo.l_far && gmax >= 1 &&
        (long long)nv.count[X] * (long long)nv.count[Y] >= geo.m2l_min_pairs)
        return kFar;
    if (leafx && leafy) return kP2P;
    return kSplit;
}

__device__ inline int block_size(const NodeView& nv, int32_t X, int32_t Y) {
    bool lx = nv.child_first[X] < 0, ly = nv.child_first[Y] < 0;
    return (lx ? 1 : nv.nchild[X]) * (ly ? 1 : nv.nchild[Y]);
}

// the root pair (root, root) at depth 0
__global__ void k_init_pairs(int64_t n, int32_t* pX, int32_t* pY, DevCounts* dc) {
    dc->depth_start[0] = 0;
    dc->depth_start[1] = n > 0 ? 1 : 0;
    dc->overflow &= ~1ll;       // the traversal's bit; the build's (16) stays for the step check
    dc->need_pairs = 0;
    dc->interactions = 0;
    if (n > 0) {
        pX[0] = 0;
        pY[0] = 0;
    }
}

// a replay that keeps the lists: only the near field's work counter restarts
__global__ void k_reuse_init(DevCounts* dc) {
    dc->overflow &= ~1ll;
    dc->interactions = 0;
}

// pairs of one depth: [db[0], db[1]); their count goes to *scan_n
__global__ void k_classify(const int64_t* __restrict__ db, NodeView nv, Geo geo,
                           const int32_t* __restrict__ pX, const int32_t* __restrict__ pY,
                           uint8_t* __restrict__ kind, int32_t* __restrict__ cnt,
                           int64_t* __restrict__ scan_n) {
    const int64_t q0 = db[0], nq = db[1] - db[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) *scan_n = nq;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nq;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = q0 + k;
        int32_t X = pX[q], Y = pY[q];
        uint8_t kd = classify(nv, geo, X, Y);
        kind[q] = kd;
        cnt[k] = kd == kSplit ? block_size(nv, X, Y) : 0;
    }
}

// Children of the split pairs of one depth, one contiguous block per pair,
// axon-child major, from db[1] on.  When the children do not fit in the table
// (overflow bit 0, set by the scan that also left the next depth empty) no
// child is written and the traversal ends here; the caller grows the table
// and redoes it.
__global__ void k_emit_pairs(const int64_t* __restrict__ db, NodeView nv,
                             const uint8_t* __restrict__ kind, const int32_t* __restrict__ off,
                             int32_t* __restrict__ pX, int32_t* __restrict__ pY,
                             int32_t* __restrict__ pcf, uint8_t* __restrict__ pnb,
                             float4* __restrict__ pw, int64_t cap,
                             const int64_t* __restrict__ overflow) {
    const int64_t q0 = db[0], nq = db[1] - db[0], next0 = db[1];
    const bool full = (*overflow & 1) != 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nq;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = q0 + k;
        pw[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kind[q] != kSplit) {
            pcf[q] = -1;
            continue;
        }
        int32_t X = pX[q], Y = pY[q];
        int64_t cf = next0 + off[k];
        const int nb = block_size(nv, X, Y);
        if (full || cf + nb > cap) {
            pcf[q] = -1;
            continue;
        }
        pcf[q] = (int32_t)cf;
        pnb[q] = (uint8_t)nb;
        int32_t cx = nv.child_first[X], cy = nv.child_first[Y];
        if (cx >= 0 && cy >= 0) {
            int nx = nv.nchild[X], ny = nv.nchild[Y];
            for (int i = 0; i < nx; ++i)
                for (int j = 0; j < ny; ++j) {
                    pX[cf + i * ny + j] = cx + i;
                    pY[cf + i * ny + j] = cy + j;
                }
        } else if (cx < 0) {
            int ny = nv.nchild[Y];
            for (int j = 0; j < ny; ++j) {
                pX[cf + j] = X;
                pY[cf + j] = cy + j;
            }
        } else {
            int nx = nv.nchild[X];
            for (int i = 0; i < nx; ++i) {
                pX[cf + i] = cx + i;
                pY[cf + i] = Y;
            }
        }
    }
}

__global__ void k_flag_kind(const uint8_t* __restrict__ kind, const int64_t* __restrict__ n_dev,
                            uint8_t K, int32_t* __restrict__ flag) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = kind[i] == K;
}

__global__ void k_compact_kind(const uint8_t* __restrict__ kind, const int64_t* __restrict__ n_dev,
                               uint8_t K, const int32_t* __restrict__ off,
                               const int32_t* __restrict__ pX, int32_t* __restrict__ out_q,
                               uint64_t* __restrict__ out_key) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (kind[i] == K) {
            int32_t o = off[i];
            out_q[o] = (int32_t)i;
            if (out_key) out_key[o] = (uint64_t)pX[i];
        }
}

__global__ void k_seg_flags(const uint64_t* __restrict__ key, const int64_t* __restrict__ n_dev,
                            int32_t* __restrict__ flag) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// segment starts, and seg_first[nseg] = n
__global__ void k_seg_first(const int32_t* __restrict__ flag, const int32_t* __restrict__ off,
                            const int64_t* __restrict__ n_dev, const int64_t* __restrict__ nseg_dev,
                            int32_t* __restrict__ seg_first) {
    const int64_t n = *n_dev;
    if (blockIdx.x == 0 && threadIdx.x == 0) seg_first[*nseg_dev] = (int32_t)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) seg_first[off[i]] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// a6: Hermite coefficients of the dendritic weights (Eq. 7) and axon moments
// M_beta = sum_t a_t ((t - c_A)/sigma)^beta, per channel, one block per box
// ---------------------------------------------------------------------------
constexpr int kP2MThreads = 128;
constexpr int kP2MChunk = 32;

__global__ void __launch_bounds__(kP2MThreads)
k_p2m(int64_t first_node, int p, float inv_sigma, const float4* __restrict__ pts,
      const int32_t* __restrict__ nfirst, const int32_t* __restrict__ ncount,
      const float4* __restrict__ ca, const float4* __restrict__ cd, float* __restrict__ A,
      float* __restrict__ M) {
    __shared__ float ypow[kP2MChunk][3][kMaxP];
    __shared__ float xpow[kP2MChunk][3][kMaxP];
    __shared__ float wgt[kP2MChunk][4];
    const int64_t node = first_node + blockIdx.x;
    const int p3 = p * p * p;
    const float4 cD = cd[node], cA = ca[node];
    const int32_t f = nfirst[node], c = ncount[node];
    constexpr int kMaxAcc = (4 * kMaxP * kMaxP * kMaxP + kP2MThreads - 1) / kP2MThreads;
    float acc[kMaxAcc];
#pragma unroll
    for (int r = 0; r < kMaxAcc; ++r) acc[r] = 0.f;
    for (int base = 0; base < c; base += kP2MChunk) {
        int m = min(kP2MChunk, c - base);
        __syncthreads();
        for (int t = threadIdx.x; t < m * 3; t += kP2MThreads) {
            int j = t / 3, d = t % 3;
            float4 P = pts[f + base + j];
            float pv = d == 0 ? P.x : (d == 1 ? P.y : P.z);
            float yv = (pv - (d == 0 ? cD.x : (d == 1 ? cD.y : cD.z))) * inv_sigma;
            float xv = (pv - (d == 0 ? cA.x : (d == 1 ? cA.y : cA.z))) * inv_sigma;
            float py = 1.f, px = 1.f;
            for (int k = 0; k < p; ++k) {
                ypow[j][d][k] = py;
                xpow[j][d][k] = px;
                py *= yv;
                px *= xv;
            }
            if (d == 0) {
                uint32_t w = __float_as_uint(P.w);
                float a = (float)pk_axon(w);
                bool inh = pk_type(w) != 0;
                wgt[j][0] = (float)pk_de(w);
                wgt[j][1] = (float)pk_di(w);
                wgt[j][2] = inh ? 0.f : a;
                wgt[j][3] = inh ? a : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kMaxAcc; ++r) {
            int idx = threadIdx.x + r * kP2MThreads;
            if (idx >= 4 * p3) continue;
            int which = idx / p3, a = idx - which * p3;
            int a0 = a / (p * p), a1 = (a / p) % p, a2 = a % p;
            float s = acc[r];
            if (which < 2) {
                for (int j = 0; j < m; ++j)
                    s = fmaf(wgt[j][which] * ypow[j][0][a0], ypow[j][1][a1] * ypow[j][2][a2], s);
            } else {
                for (int j = 0; j < m; ++j)
                    s = fmaf(wgt[j][which] * xpow[j][0][a0], xpow[j][1][a1] * xpow[j][2][a2], s);
            }
            acc[r] = s;
        }
    }
    const int64_t e = (int64_t)blockIdx.x;
#pragma unroll
    for (int r = 0; r < kMaxAcc; ++r) {
        int idx = threadIdx.x + r * kP2MThreads;
        if (idx >= 4 * p3) continue;
        int which = idx / p3, a = idx - which * p3;
        int a0 = a / (p * p), a1 = (a / p) % p, a2 = a % p;
        if (which < 2)
            A[(e * 2 + which) * p3 + a] = acc[r] * c_inv_fact[a0] * c_inv_fact[a1] * c_inv_fact[a2];
        else
            M[(e * 2 + which - 2) * p3 + a] = acc[r];
    }
}

// ---------------------------------------------------------------------------
// a7: translations.  With Delta = (c_A - c_D)/sigma and H_d[n] = h_n(Delta_d),
//   B_beta(X <- Y) = (-1)^|beta| / beta!  sum_alpha A_alpha(Y) H0[a0+b0] H1[a1+b1] H2[a2+b2]
// done as three passes over one dimension each (p^4 multiply-adds per pass
// and channel), and W(X,Y) = sum_beta B_beta(X <- Y) M_beta(X).  The far pairs
// are grouped by target box X (stable sort of the list by X); one warp takes
// all pairs of one X in list order, so B(X) = sum_Y B(X <- Y) is summed in
// registers in a fixed order (reproducible, no atomics) and added to B once.
// A pass is one column per lane (channel and the two indices it does not
// sum over), staged through the warp's shared memory between passes; the
// last pass's columns are the lane's own for every pair of X.
// ---------------------------------------------------------------------------
__device__ inline void hermite_row(float x, float* h, int nmax) {
    const float h0 = __expf(-x * x);
    h[0] = h0;
    if (nmax >= 1) h[1] = 2.f * x * h0;
    for (int k = 1; k < nmax; ++k) h[k + 1] = 2.f * x * h[k] - 2.f * (float)k * h[k - 1];
}

constexpr int kM2LWarps = 4;

template <int P>
__global__ void __launch_bounds__(kM2LWarps * 32)
k_m2l_seg(const int32_t* __restrict__ seg_first, const int64_t* __restrict__ nseg_dev,
          const int32_t* __restrict__ list, int64_t exp_first, float inv_sigma,
          const int32_t* __restrict__ pX, const int32_t* __restrict__ pY,
          const float4* __restrict__ ca, const float4* __restrict__ cd,
          const float* __restrict__ A, const float* __restrict__ M, float* __restrict__ B,
          float4* __restrict__ pw) {
    constexpr int P2 = P * P, P3 = P2 * P;
    constexpr int NC = 2 * P2;                 // columns of a pass (two channels)
    constexpr int NL = (NC + 31) / 32;         // columns per lane
    constexpr int NH = 2 * P - 1;              // Hermite functions h_0 .. h_{2p-2}
    __shared__ float sbuf[kM2LWarps][2][2 * P3];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* s0 = sbuf[w][0];
    float* s1 = sbuf[w][1];
    // (-1)^|beta| / beta! of the lane's last-pass columns (c, b0, b1)
    float scale[NL][P];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        const int col = lane + 32 * j;
        const int b0 = (col / P) % P, b1 = col % P;
#pragma unroll
        for (int b2 = 0; b2 < P; ++b2) {
            const float f = c_inv_fact[b0] * c_inv_fact[b1] * c_inv_fact[b2];
            scale[j][b2] = ((b0 + b1 + b2) & 1) ? -f : f;
        }
    }
    const int64_t nseg = *nseg_dev;
    for (int64_t sg = (int64_t)blockIdx.x * kM2LWarps + w; sg < nseg;
         sg += (int64_t)gridDim.x * kM2LWarps) {
        const int32_t i0 = seg_first[sg], i1 = seg_first[sg + 1];
        const int32_t X = pX[list[i0]];
        const int64_t ex = X - exp_first;
        const float4 a = ca[X];
        float acc[NL][P], mm[NL][P];
#pragma unroll
        for (int j = 0; j < NL; ++j) {
            const int col = lane + 32 * j;
            const int c = col / P2, b0 = (col / P) % P, b1 = col % P;
#pragma unroll
            for (int b2 = 0; b2 < P; ++b2) {
                acc[j][b2] = 0.f;
                mm[j][b2] = col < NC ? M[(ex * 2 + c) * P3 + b0 * P2 + b1 * P + b2] : 0.f;
            }
        }
        // the next pair's list entry, centre and coefficients are loaded
        // while the current pair is translated (a chain of dependent loads)
        constexpr int NA = (2 * P3 + 31) / 32;     // coefficients per lane
        int32_t qn = list[i0];
        int32_t yn = pY[qn];
        float4 dn = cd[yn];
        float an[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const int e = lane + 32 * k;
            an[k] = e < 2 * P3 ? A[(yn - exp_first) * 2 * P3 + e] : 0.f;
        }
        for (int32_t i = i0; i < i1; ++i) {
            const int32_t q = qn;
            const float4 d = dn;
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                const int e = lane + 32 * k;
                if (e < 2 * P3) s0[e] = an[k];
            }
            if (i + 1 < i1) {
                qn = list[i + 1];
                yn = pY[qn];
                dn = cd[yn];
#pragma unroll
                for (int k = 0; k < NA; ++k) {
                    const int e = lane + 32 * k;
                    an[k] = e < 2 * P3 ? A[(yn - exp_first) * 2 * P3 + e] : 0.f;
                }
            }
            float H[NH];
            hermite_row((a.x - d.x) * inv_sigma, H, NH - 1);
            __syncwarp();
            // pass 0 (over a0): column (c, a1, a2) -> s1[c][b0][a1][a2]
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const int col = lane + 32 * j;
                if (col >= NC) break;
                const int c = col / P2, r = col % P2;
                float v[P];
#pragma unroll
                for (int k = 0; k < P; ++k) v[k] = s0[c * P3 + k * P2 + r];
#pragma unroll
                for (int o = 0; o < P; ++o) {
                    float t = 0.f;
#pragma unroll
                    for (int k = 0; k < P; ++k) t = fmaf(H[k + o], v[k], t);
                    s1[c * P3 + o * P2 + r] = t;
                }
            }
            hermite_row((a.y - d.y) * inv_sigma, H, NH - 1);
            __syncwarp();
            // pass 1 (over a1): column (c, b0, a2) -> s0[c][b0][b1][a2]
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const int col = lane + 32 * j;
                if (col >= NC) break;
                const int c = col / P2, b0 = (col / P) % P, a2 = col % P;
                const int base = c * P3 + b0 * P2 + a2;
                float v[P];
#pragma unroll
                for (int k = 0; k < P; ++k) v[k] = s1[base + k * P];
#pragma unroll
                for (int o = 0; o < P; ++o) {
                    float t = 0.f;
#pragma unroll
                    for (int k = 0; k < P; ++k) t = fmaf(H[k + o], v[k], t);
                    s0[base + o * P] = t;
                }
            }
            hermite_row((a.z - d.z) * inv_sigma, H, NH - 1);
            __syncwarp();
            // pass 2 (over a2): the lane's own columns (c, b0, b1)
            float w0 = 0.f, w1 = 0.f;
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const int col = lane + 32 * j;
                if (col >= NC) break;
                const int base = (col / P2) * P3 + (col % P2) * P;
                float v[P];
#pragma unroll
                for (int k = 0; k < P; ++k) v[k] = s0[base + k];
                float wc = 0.f;
#pragma unroll
                for (int o = 0; o < P; ++o) {
                    float t = 0.f;
#pragma unroll
                    for (int k = 0; k < P; ++k) t = fmaf(H[k + o], v[k], t);
                    t *= scale[j][o];
                    acc[j][o] += t;
                    wc = fmaf(t, mm[j][o], wc);
                }
                if (col < P2) w0 += wc; else w1 += wc;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                w0 += __shfl_xor_sync(0xffffffffu, w0, o);
                w1 += __shfl_xor_sync(0xffffffffu, w1, o);
            }
            if (lane == 0) pw[q] = make_float4(w0, 0.f, w1, 0.f);
            __syncwarp();      // s0 is the next pair's staging
        }
        // B(X) += the sum over X's far pairs (no other warp adds to B(X) here)
#pragma unroll
        for (int j = 0; j < NL; ++j) {
            const int col = lane + 32 * j;
            if (col >= NC) break;
            const int c = col / P2, b0 = (col / P) % P, b1 = col % P;
            float* Bx = B + (ex * 2 + c) * P3 + b0 * P2 + b1 * P;
#pragma unroll
            for (int b2 = 0; b2 < P; ++b2) Bx[b2] += acc[j][b2];
        }
    }
}

// keys of the far pairs [first, nfar) of `list` for the grouping by target box
__global__ void k_m2l_keys(const int32_t* __restrict__ list, const int64_t* __restrict__ nfar,
                           const int64_t* __restrict__ first, const int32_t* __restrict__ pX,
                           uint64_t* __restrict__ key, int32_t* __restrict__ val,
                           int64_t* __restrict__ count) {
    const int64_t k0 = first ? *first : 0, n = *nfar - k0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n > 0 ? n : 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = list[k0 + i];
        key[i] = (uint64_t)pX[q];
        val[i] = q;
    }
}

// ---------------------------------------------------------------------------
// a8: Taylor evaluation (Eq. 6) at every target from each of its boxes that
// carries an expansion; initialises u_sorted.
// ---------------------------------------------------------------------------
__global__ void k_l2p(int64_t n, int64_t exp_first, int p, float inv_sigma,
                      const float4* __restrict__ pts, const int32_t* __restrict__ leaf_of,
                      const int32_t* __restrict__ parent, const float4* __restrict__ ca,
                      const float* __restrict__ B, float* __restrict__ u) {
    const int p3 = p * p * p;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        float4 P = pts[j];
        uint32_t pw = __float_as_uint(P.w);
        float acc = 0.f;
        if (pk_axon(pw) > 0) {
            int ch = pk_type(pw) ? 1 : 0;
            int32_t node = leaf_of[j];
            while (node >= exp_first) {
                float4 c = ca[node];
                float x[3] = {(P.x - c.x) * inv_sigma, (P.y - c.y) * inv_sigma,
                              (P.z - c.z) * inv_sigma};
                float px[3][kMaxP];
                for (int d = 0; d < 3; ++d) {
                    float v = 1.f;
                    for (int k = 0; k < p; ++k) {
                        px[d][k] = v;
                        v *= x[d];
                    }
                }
                const float* Bn = B + ((int64_t)(node - exp_first) * 2 + ch) * p3;
                int i = 0;
                for (int b0 = 0; b0 < p; ++b0)
                    for (int b1 = 0; b1 < p; ++b1) {
                        float s = 0.f;
                        float f01 = px[0][b0] * px[1][b1];
                        for (int b2 = 0; b2 < p; ++b2) s = fmaf(Bn[i++], px[2][b2], s);
                        acc = fmaf(f01, s, acc);
                    }
                node = parent[node];
            }
        }
        u[j] = acc;
    }
}

// a10: attraction of a split pair = sum over its child block, in double-FP32
// (compensated FP32 sums: no double precision instruction, which this GPU
// runs at 1/64 of the single precision rate).  The split pairs of each depth
// are listed once per traversal (the list keeps pair order, each entry with
// its child block); 8 lanes take one split pair, lane c summing children c,
// c + 8, ... (coalesced: 8 consecutive 16-byte entries per step, all loaded
// before the sum), then a fixed butterfly over the 8 lanes.  Both orders are
// fixed, so the table is reproducible.  sb = [first, end) of the depth's
// entries in split; an entry is (pair, first child, child count, 0).
__global__ void k_reduce_split(const int64_t* __restrict__ sb, const int4* __restrict__ split,
                               float4* __restrict__ pw) {
    const int64_t s0 = sb[0], ns = sb[1] - sb[0];
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the loop bound is uniform across the warp (its 4 groups shuffle together)
    for (int64_t k0 = 4 * warp; k0 < ns; k0 += 4 * nwarp) {
        const int64_t k = k0 + (lane >> 3);
        int4 ent = make_int4(-1, -1, 0, 0);
        if (k < ns) ent = split[s0 + k];
        const int32_t q = ent.x, cf = ent.y;
        const int nb = cf >= 0 ? ent.z : 0;     // cf < 0: children not stored (overflow)
        // a lane's children (at most 8 of a block of 64) loaded before they
        // are summed, in compensated running sums of both channels
        float4 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (sub + 8 * t < nb) v[t] = pw[cf + sub + 8 * t];
        float eh = 0.f, ec = 0.f, ih = 0.f, ic = 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (sub + 8 * t < nb) {
                ff_acc(eh, ec, v[t].x, v[t].y);
                ff_acc(ih, ic, v[t].z, v[t].w);
            }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            const float oeh = __shfl_xor_sync(0xffffffffu, eh, o);
            const float oec = __shfl_xor_sync(0xffffffffu, ec, o);
            const float oih = __shfl_xor_sync(0xffffffffu, ih, o);
            const float oic = __shfl_xor_sync(0xffffffffu, ic, o);
            ff_acc(eh, ec, oeh, oec);
            ff_acc(ih, ic, oih, oic);
        }
        if (sub == 0 && cf >= 0) {
            const float2 e = ff_two_sum(eh, ec), i = ff_two_sum(ih, ic);
            pw[q] = make_float4(e.x, e.y, i.x, i.y);
        }
    }
}

// the split pairs in pair order (off: exclusive scan of their flags), each
// with its child block
__global__ void k_compact_split(const uint8_t* __restrict__ kind, const int64_t* __restrict__ n_dev,
                                const int32_t* __restrict__ off, const int32_t* __restrict__ pcf,
                                const uint8_t* __restrict__ pnb, int4* __restrict__ split) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (kind[i] == kSplit) split[off[i]] = make_int4((int32_t)i, pcf[i], (int)pnb[i], 0);
}

// the split pairs' range of every depth d <= D in split: the exclusive scan
// of the split flags at the depth's first pair
__global__ void k_split_starts(DevCounts* dc, const int32_t* __restrict__ off, int D) {
    const int d = threadIdx.x;
    if (d > D) return;
    const int64_t q = dc->depth_start[d], n = dc->depth_start[D];
    dc->split_start[d] = q < n ? (int64_t)off[q] : dc->n_split;
}

__global__ void k_scatter_u(const float* __restrict__ us, const int32_t* __restrict__ perm,
                            int64_t n, float* __restrict__ u) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        u[perm[j]] = us[j];
}

// ---------------------------------------------------------------------------
// all-pairs comparison path: every target against every source, sources
// staged through shared memory in tiles.  Each tile's terms are summed in
// single precision and the tile sums are added with Kahan's compensated
// summation, so the error of u does not grow with the number of tiles (a
// plain running sum over a million sources erred by about 3e-5).
// ---------------------------------------------------------------------------
constexpr int kDirThreads = 256;

// first index of the sorted keys at or above v
__device__ inline int64_t lower_bound_key(const uint64_t* __restrict__ keys, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// FR: the points sit in frames (independent networks): a target takes only
// the sources of its own network, which are contiguous in Morton order (the
// key's top 3 L0 bits are the network's cell, fsh = 3 (21 - L0) bits below);
// a block walks the tiles from its first target's network to its last one's
template <bool FR>
__global__ void __launch_bounds__(kDirThreads)
k_direct(int64_t n, const float4* __restrict__ pts, const float2* __restrict__ wts, float k2,
         const uint64_t* __restrict__ keys, int fsh, float* __restrict__ u) {
    __shared__ float4 sp[kDirThreads];
    __shared__ float2 sw[kDirThreads];
    __shared__ uint32_t sc[FR ? kDirThreads : 1];
    __shared__ int64_t s_range[2];
    for (int64_t tb = (int64_t)blockIdx.x * kDirThreads; tb < n;
         tb += (int64_t)gridDim.x * kDirThreads) {
        int64_t t = tb + threadIdx.x;
        bool active = t < n;
        float4 T = active ? pts[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t tw = __float_as_uint(T.w);
        bool inh = pk_type(tw) != 0;
        uint32_t tcell = 0;
        int64_t s0 = 0, s1 = n;
        if (FR) {
            tcell = active ? (uint32_t)(keys[t] >> fsh) : 0xffffffffu;
            __syncthreads();
            if (threadIdx.x == 0) {
                const int64_t tl = tb + kDirThreads <= n ? tb + kDirThreads - 1 : n - 1;
                const uint64_t c0 = keys[tb] >> fsh, c1 = keys[tl] >> fsh;
                s_range[0] = lower_bound_key(keys, n, c0 << fsh) / kDirThreads * kDirThreads;
                s_range[1] = lower_bound_key(keys, n, (c1 + 1) << fsh);
            }
            __syncthreads();
            s0 = s_range[0];
            s1 = s_range[1];
        }
        float acc = 0.f, comp = 0.f;   // Kahan sum of the tile sums
        for (int64_t sb = s0; sb < s1; sb += kDirThreads) {
            __syncthreads();
            int64_t s = sb + threadIdx.x;
            sp[threadIdx.x] = s < n ? pts[s] : make_float4(3e30f, 3e30f, 3e30f, 0.f);
            sw[threadIdx.x] = s < n ? wts[s] : make_float2(0.f, 0.f);
            if (FR) sc[threadIdx.x] = s < n ? (uint32_t)(keys[s] >> fsh) : 0xfffffffeu;
            __syncthreads();
            float part = 0.f;
            if (sb != tb) {
#pragma unroll 8
                for (int j = 0; j < kDirThreads; ++j) {
                    float4 S = sp[j];
                    float dx = T.x - S.x, dy = T.y - S.y, dz = T.z - S.z;
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    float e = ex2_approx(-r2 * k2);
                    float wj = inh ? sw[j].y : sw[j].x;
                    if (FR && sc[j] != tcell) wj = 0.f;
                    part = fmaf(wj, e, part);
                }
            } else {
                // the tile holding the targets themselves: skip j == t
                for (int j = 0; j < kDirThreads; ++j) {
                    float4 S = sp[j];
                    float dx = T.x - S.x, dy = T.y - S.y, dz = T.z - S.z;
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    float e = ex2_approx(-r2 * k2);
                    float wj = j == (int)threadIdx.x ? 0.f : (inh ? sw[j].y : sw[j].x);
                    if (FR && sc[j] != tcell) wj = 0.f;
                    part = fmaf(wj, e, part);
                }
            }
            const float y = __fsub_rn(part, comp);
            const float t2 = __fadd_rn(acc, y);
            comp = __fsub_rn(__fsub_rn(t2, acc), y);
            acc = t2;
        }
        if (active) u[t] = pk_axon(tw) > 0 ? acc : 0.f;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static NodeView node_view(msp_ctx& c) {
    NodeView nv;
    nv.level = c.nd_level.get<uint8_t>();
    nv.prefix = c.nd_prefix.get<uint64_t>();
    nv.first = c.nd_first.get<int32_t>();
    nv.count = c.nd_count.get<int32_t>();
    nv.child_first = c.nd_child_first.get<int32_t>();
    nv.nchild = c.nd_nchild.get<uint8_t>();
    nv.sums = c.nd_sums.get<int4>();
    return nv;
}

static int bits_for(int64_t v) {
    int b = 1;
    while (b < 63 && (1ll << b) <= v) ++b;
    return b;
}

void attraction(msp_ctx& c, float* u_dev, cudaStream_t s) {
    NvtxRange nv_("msp attraction");
    if (!c.tree_built) throw Error(MSP_ERR_NOT_BUILT, "msp_build_tree must run first");
    if (!c.graph_mode) {
        c.attraction_done = false;
        c.last_was_graph = false;
    }
    const msp_config& cfg = c.cfg;
    const int64_t n = c.n;
    const int B = 256;
    // inside a stream capture the near-field events become graph nodes
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    MSP_CUDA(cudaStreamIsCapturing(s, &cst));
    const unsigned ev_flags = cst == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    NodeView nv = node_view(c);
    Geo geo;
    for (int l = 0; l <= kMortonBits; ++l) geo.g2[l] = c.g2[l];
    geo.fg2 = c.frame_level > 0 && c.frame_plans ? c.frame_g2.get<long long>() : nullptr;
    geo.frame_level = c.frame_level;
    geo.nf = (int64_t)c.frame_off_host.size() - 1;
    geo.l_far = c.l_far;
    geo.m2l_min_pairs = cfg.m2l_min_pairs;
    geo.mac_mode = cfg.mac_mode;
    geo.c1 = cfg.c1;
    const int p = cfg.p, p3 = p * p * p;
    const float inv_sigma = (float)(1.0 / cfg.sigma);
    const float k2 = (float)(1.4426950408889634 / (cfg.sigma * cfg.sigma));

    DevCounts* dc = dcounts(c);
    // traversal depth d holds the pairs whose finer box is at level d, so the
    // tree depth bounds the number of depths
    const int D = c.tree_depth + 1;
    // replays of the step graph that reuse the octree keep the traversal and
    // its lists too: the cutoff rule depends on the positions only (the count
    // rule of Algorithm 2 depends on the vacant counts and is redone)
    if (c.pair_cap <= 0) c.pair_cap = std::max<int64_t>(64 * c.n_nodes, 1 << 16);
    // an eager attraction on a reused octree keeps the lists of the last one,
    // provided no buffer that holds them is about to grow (which would lose
    // them)
    auto holds = [&](const DBuf& b, size_t elem) {
        return b.bytes >= (size_t)c.pair_cap * elem;
    };
    const bool lists_fit = holds(c.pr_X, 4) && holds(c.pr_Y, 4) && holds(c.pr_kind, 1) &&
                           holds(c.pr_cf, 4) && holds(c.pr_nb, 1) && holds(c.pr_w, 16) &&
                           holds(c.p2p_val0, 4) && holds(c.far_q, 4) && holds(c.split_q, 16) &&
                           holds(c.nf_src, 8) &&
                           holds(c.nf_w32, 8) &&
                           (c.exp_nodes == 0 || (holds(c.m2_key0, 8) && holds(c.m2_val0, 4)));
    const bool reuse_lists =
        cfg.mac_mode == 0 && ((c.graph_mode && !c.graph_full_build) ||
                              (!c.graph_mode && c.tree_reused && c.lists_valid && lists_fit));
    const int Gt = (int)std::max<int64_t>(1, (int64_t)c.sm_count * 8);
    for (int attempt = 0;; ++attempt) {
    const int64_t cap = c.pair_cap;
    if (cap > 0x7fffffffll) throw Error(MSP_ERR_CAPACITY, "pair count exceeds int32");
    c.pr_X.ensure<int32_t>((size_t)cap);
    c.pr_Y.ensure<int32_t>((size_t)cap);
    c.pr_kind.ensure<uint8_t>((size_t)cap);
    c.pr_cf.ensure<int32_t>((size_t)cap);
    c.pr_nb.ensure<uint8_t>((size_t)cap);
    c.pr_w.ensure<float4>((size_t)cap);
    int32_t* cnt = c.cnt.ensure<int32_t>((size_t)cap);
    int32_t* off = c.off.ensure<int32_t>((size_t)cap);
    uint8_t* kind = c.pr_kind.get<uint8_t>();

    int32_t* far_q = c.far_q.ensure<int32_t>((size_t)cap);
    int4* split = c.split_q.ensure<int4>((size_t)cap);
    int32_t* pv0 = c.p2p_val0.ensure<int32_t>((size_t)cap);
    int32_t* seg_first = c.seg_first.ensure<int32_t>((size_t)c.n_nodes + 2);
    const int64_t* n_pairs_dev = &dc->depth_start[D];
    if (reuse_lists) {
        // the step graph's replays keep the traversal and the lists of the
        // eager attraction of the same positions (guarded by the build's
        // checksum and generation stamp)
        k_reuse_init<<<1, 1, 0, s>>>(dc);
        MSP_LAUNCH("reuse_init");
    } else {
    // a5: breadth-first dual traversal from (root, root)
    k_init_pairs<<<1, 1, 0, s>>>(n, c.pr_X.get<int32_t>(), c.pr_Y.get<int32_t>(), dc);
    MSP_LAUNCH("init_pairs");
    for (int d = 0; d < D; ++d) {
        k_classify<<<Gt, B, 0, s>>>(&dc->depth_start[d], nv, geo, c.pr_X.get<int32_t>(),
                                    c.pr_Y.get<int32_t>(), kind, cnt, &dc->scan_n);
        MSP_LAUNCH("classify");
        scan_dev(c, cnt, off, &dc->scan_n, cap, &dc->depth_start[d + 2], &dc->depth_start[d + 1], s,
                 cap, &dc->overflow, &dc->need_pairs);
        k_emit_pairs<<<Gt, B, 0, s>>>(&dc->depth_start[d], nv, kind, off, c.pr_X.get<int32_t>(),
                                      c.pr_Y.get<int32_t>(), c.pr_cf.get<int32_t>(),
                                      c.pr_nb.get<uint8_t>(), c.pr_w.get<float4>(), cap,
                                      &dc->overflow);
        MSP_LAUNCH("emit_pairs");
    }

    // far and near-field lists
    int32_t* flag = cnt;
    k_flag_kind<<<Gt, B, 0, s>>>(kind, n_pairs_dev, kSplit, flag);
    MSP_LAUNCH("flag_split");
    scan_dev(c, flag, off, n_pairs_dev, cap, &dc->n_split, nullptr, s);
    k_compact_split<<<Gt, B, 0, s>>>(kind, n_pairs_dev, off, c.pr_cf.get<int32_t>(),
                                     c.pr_nb.get<uint8_t>(), split);
    MSP_LAUNCH("compact_split");
    k_split_starts<<<1, 32, 0, s>>>(dc, off, D);
    MSP_LAUNCH("split_starts");
    k_flag_kind<<<Gt, B, 0, s>>>(kind, n_pairs_dev, kFar, flag);
    MSP_LAUNCH("flag_far");
    scan_dev(c, flag, off, n_pairs_dev, cap, &dc->n_far, nullptr, s);
    k_compact_kind<<<Gt, B, 0, s>>>(kind, n_pairs_dev, kFar, off, c.pr_X.get<int32_t>(), far_q,
                                    nullptr);
    MSP_LAUNCH("compact_far");
    k_flag_kind<<<Gt, B, 0, s>>>(kind, n_pairs_dev, kP2P, flag);
    MSP_LAUNCH("flag_p2p");
    scan_dev(c, flag, off, n_pairs_dev, cap, &dc->n_p2p, nullptr, s);
    uint64_t* pk0 = c.p2p_key0.ensure<uint64_t>((size_t)cap);
    uint64_t* pk1 = c.p2p_key1.ensure<uint64_t>((size_t)cap);
    int32_t* pv1 = c.p2p_val1.ensure<int32_t>((size_t)cap);
    k_compact_kind<<<Gt, B, 0, s>>>(kind, n_pairs_dev, kP2P, off, c.pr_X.get<int32_t>(), pv0, pk0);
    MSP_LAUNCH("compact_p2p");
    radix_sort_dev(c, pk0, pv0, pk1, pv1, &dc->n_p2p, cap, bits_for(c.n_nodes), s);
    int32_t* sflag = c.seg_flag.ensure<int32_t>((size_t)cap);
    int32_t* soff = cnt;
    k_seg_flags<<<Gt, B, 0, s>>>(pk0, &dc->n_p2p, sflag);
    MSP_LAUNCH("seg_flags");
    scan_dev(c, sflag, soff, &dc->n_p2p, cap, &dc->nseg, nullptr, s);
    // at most one segment per box
    k_seg_first<<<Gt, B, 0, s>>>(sflag, soff, &dc->n_p2p, &dc->nseg, seg_first);
    MSP_LAUNCH("seg_first");
    }

    // a6: expansions of every box at level >= l_far
    c.exp_first = c.l_far <= c.tree_depth ? c.level_start[c.l_far] : c.n_nodes;
    c.exp_nodes = c.n_nodes - c.exp_first;
    size_t ecount = (size_t)std::max<int64_t>(c.exp_nodes, 1) * 2 * p3;
    float* eA = c.expA.ensure<float>(ecount);
    float* eM = c.expM.ensure<float>(ecount);
    float* eB = c.expB.ensure<float>(ecount);
    // expansion centres: the centroids, or the geometric centres (centre_mode 1)
    const bool geo = c.cfg.centre_mode == 1;
    const float4* eca = c.nd_ca.get<float4>();
    const float4* ecd = c.nd_cd.get<float4>();
    if (geo && c.exp_nodes > 0) {
        geo_centres(c, s);
        eca = ecd = c.nd_gc.get<float4>();
    }
    if (c.exp_nodes > 0) {
        MSP_CUDA(cudaMemsetAsync(eB, 0, ecount * sizeof(float), s));
        k_p2m<<<(unsigned)c.exp_nodes, kP2MThreads, 0, s>>>(
            c.exp_first, p, inv_sigma, c.pts.get<float4>(), c.nd_first.get<int32_t>(),
            c.nd_count.get<int32_t>(), eca, ecd, eA, eM);
        MSP_LAUNCH("p2m");
    }
    // a7: translations, accumulating B(X) and W(X,Y); with geometric centres
    // the pairs that share an offset share one operator (matrix products),
    // the rest one pair at a time
    if (c.exp_nodes > 0) {
        const int32_t* mq = far_q;
        const int64_t* first = nullptr;
        if (geo && m2l_gemm_fits(p)) {
            int64_t* fb = nullptr;
            mq = m2l_gemm(c, far_q, &dc->n_far, cap, eA, eM, eB, c.pr_w.get<float4>(), &fb, s);
            first = fb;
        }
        // the pairs [first, n_far) of mq grouped by target box
        uint64_t* mk0 = c.m2_key0.ensure<uint64_t>((size_t)cap);
        uint64_t* mk1 = c.m2_key1.ensure<uint64_t>((size_t)cap);
        int32_t* mv0 = c.m2_val0.ensure<int32_t>((size_t)cap);
        int32_t* mv1 = c.m2_val1.ensure<int32_t>((size_t)cap);
        int32_t* mflag = c.m2_flag.ensure<int32_t>((size_t)cap);
        int32_t* moff = c.m2_off.ensure<int32_t>((size_t)cap);
        int32_t* mseg = c.m2_seg.ensure<int32_t>((size_t)c.n_nodes + 2);
        if (!reuse_lists || geo) {
            k_m2l_keys<<<Gt, B, 0, s>>>(mq, &dc->n_far, first, c.pr_X.get<int32_t>(), mk0, mv0,
                                        &dc->m2l_n);
            MSP_LAUNCH("m2l_keys");
            radix_sort_dev(c, mk0, mv0, mk1, mv1, &dc->m2l_n, cap, bits_for(c.n_nodes), s);
            k_seg_flags<<<Gt, B, 0, s>>>(mk0, &dc->m2l_n, mflag);
            MSP_LAUNCH("m2l_seg_flags");
            scan_dev(c, mflag, moff, &dc->m2l_n, cap, &dc->m2l_nseg, nullptr, s);
            k_seg_first<<<Gt, B, 0, s>>>(mflag, moff, &dc->m2l_n, &dc->m2l_nseg, mseg);
            MSP_LAUNCH("m2l_seg_first");
        }
        const int gm = (int)c.sm_count * 8;
#define MSP_M2L_CASE(PP)                                                                       \
    case PP:                                                                                   \
        k_m2l_seg<PP><<<gm, kM2LWarps * 32, 0, s>>>(mseg, &dc->m2l_nseg, mv0, c.exp_first,    \
                                                    inv_sigma, c.pr_X.get<int32_t>(),         \
                                                    c.pr_Y.get<int32_t>(), eca, ecd, eA, eM,  \
                                                    eB, c.pr_w.get<float4>());                \
        break;
        switch (p) {
            MSP_M2L_CASE(1) MSP_M2L_CASE(2) MSP_M2L_CASE(3) MSP_M2L_CASE(4)
            MSP_M2L_CASE(5) MSP_M2L_CASE(6) MSP_M2L_CASE(7) MSP_M2L_CASE(8)
            default: throw Error(MSP_ERR_INVALID_ARG, "expansion order out of range");
        }
#undef MSP_M2L_CASE
        MSP_LAUNCH("m2l");
    }
    // a8: Taylor evaluation initialises u in sorted order; a9 adds the near field
    float* us = c.u_sorted.ensure<float>((size_t)std::max<int64_t>(n, 1));
    unsigned long long* work = reinterpret_cast<unsigned long long*>(&dc->interactions);
    if (n > 0) {
        k_l2p<<<grid_for(n, B, (int64_t)c.sm_count * 16), B, 0, s>>>(
            n, c.exp_first, p, inv_sigma, c.pts.get<float4>(), c.leaf_of.get<int32_t>(),
            c.nd_parent.get<int32_t>(), eca, eB, us);
        MSP_LAUNCH("l2p");
        MSP_CUDA(cudaEventRecordWithFlags(c.ev_nf0, s, ev_flags));
        launch_near_field(c, seg_first, &dc->nseg, c.n_nodes, pv0, &dc->n_p2p, cap, us, work,
                          reuse_lists, s);
        MSP_CUDA(cudaEventRecordWithFlags(c.ev_nf1, s, ev_flags));
    }
    c.nf_timed = n > 0;
    // a10: pair table, deepest pairs first
    for (int dd = D - 1; dd >= 0; --dd) {
        k_reduce_split<<<Gt, B, 0, s>>>(&dc->split_start[dd], split, c.pr_w.get<float4>());
        MSP_LAUNCH("reduce_split");
    }
    if (u_dev && n > 0) {
        k_scatter_u<<<grid_for(n, B, (int64_t)c.sm_count * 16), B, 0, s>>>(
            us, c.perm.get<int32_t>(), n, u_dev);
        MSP_LAUNCH("scatter_u");
    }
    // inside the whole-step graph the table does not grow: an overflow halts
    // the graph (checked on the device after the selection)
    if (c.graph_mode) return;
    pull_counts(c, s);              // the one synchronisation of the attraction
    const DevCounts& hc = *c.hcount;
    if (hc.overflow & 1) {
        // the pair table was too small: the traversal stopped at the first depth
        // that did not fit, so its count is a lower bound; grow and redo
        if (attempt >= 8) throw Error(MSP_ERR_CAPACITY, "pair table overflow after growth");
        c.pair_cap = std::max(2 * cap, hc.need_pairs + hc.need_pairs / 2 + 1024);
        continue;
    }
    int nd = 0;
    for (int d = 0; d < D; ++d)
        if (hc.depth_start[d + 1] > hc.depth_start[d]) nd = d + 1;
    c.depth_start.assign(hc.depth_start, hc.depth_start + nd + 1);
    c.n_pairs = hc.depth_start[D];
    c.n_far = hc.n_far;
    c.n_p2p = hc.n_p2p;
    c.n_p2p_targets = hc.nseg;
    c.p2p_interactions = hc.interactions;
    // keep a quarter of headroom for the next call
    c.pair_cap = std::max(c.pair_cap, c.n_pairs + c.n_pairs / 4 + 1024);
    break;
    }
    c.attraction_done = true;
    c.lists_valid = cfg.mac_mode == 0;
}

void direct(msp_ctx& c, float* u_dev, cudaStream_t s) {
    if (!c.tree_built) throw Error(MSP_ERR_NOT_BUILT, "msp_build_tree must run first");
    const int64_t n = c.n;
    if (n == 0) return;
    const float k2 = (float)(1.4426950408889634 / (c.cfg.sigma * c.cfg.sigma));
    float* us = c.u_sorted.ensure<float>((size_t)n);
    if (c.frame_level > 0) {
        // the sorted keys of the build are still in keys0
        k_direct<true><<<grid_for(n, kDirThreads), kDirThreads, 0, s>>>(
            n, c.pts.get<float4>(), c.wts.get<float2>(), k2, c.keys0.get<uint64_t>(),
            3 * (kMortonBits - c.frame_level), us);
    } else {
        k_direct<false><<<grid_for(n, kDirThreads), kDirThreads, 0, s>>>(
            n, c.pts.get<float4>(), c.wts.get<float2>(), k2, nullptr, 0, us);
    }
    MSP_LAUNCH("direct");
    k_scatter_u<<<grid_for(n, 256, (int64_t)c.sm_count * 16), 256, 0, s>>>(
        us, c.perm.get<int32_t>(), n, u_dev);
    MSP_LAUNCH("scatter_u");
}

}  // namespace msp
