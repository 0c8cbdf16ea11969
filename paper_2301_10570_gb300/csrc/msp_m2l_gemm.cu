// msp_m2l_gemm.cu -- step a7 with expansions about the boxes' geometric
// centres: the translations as matrix products with offset-indexed operators.
//
// The Hermite-to-Taylor translation of one channel (Eq. 6 composed with
// Eq. 7) is B(X) += T(Delta) A(Y) with
//   T[beta][alpha] = (-1)^|beta| / beta!  h_{a0+b0}(D0) h_{a1+b1}(D1) h_{a2+b2}(D2),
// Delta = (c_X - c_Y)/sigma.  With geometric centres Delta depends only on
// the two boxes' levels and integer offset, so the far pairs are sorted by
// (level of X, level of Y, offset in half-boxes of the finer level) and every
// group shares one operator: a block builds T (p^3 x p^3) in shared memory
// once per tile of 32 pairs and multiplies it with the tile's 64 coefficient
// columns (32 pairs x 2 channels).  The epilogue adds the columns to B(X) and
// forms W(X,Y) = <B(X<-Y), M(X)> per channel.  Pairs whose offset does not
// fit the key (boxes of very different levels) keep a key of all ones and
// sort last; the caller translates them one by one.
#include <algorithm>

#include "msp_internal.cuh"

namespace msp {

namespace {

constexpr int kGemmTile = 32;          // pairs per tile (64 columns)
constexpr int kGemmThreads = 256;
constexpr int kGemmMaxP = 5;           // T of p = 5 is 125 x 125 floats
constexpr int64_t kOffBias = 1 << 17;  // offsets in [-2^17, 2^17) half-boxes

__constant__ float c_inv_fact_g[kMaxP] = {1.f, 1.f, 0.5f, 1.f / 6.f, 1.f / 24.f, 1.f / 120.f,
                                          1.f / 720.f, 1.f / 5040.f};

__device__ __forceinline__ int64_t box_coord(uint64_t prefix, int d) {
    return (int64_t)compact_by3(prefix >> (2 - d));
}

// geometric centre of every box (with frames, in its network's own frame)
__global__ void k_geo_centres(int64_t n_nodes, const uint8_t* __restrict__ level,
                              const uint64_t* __restrict__ prefix, int frame_level, float ox,
                              float oy, float oz, float side, float4* __restrict__ gc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_nodes;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)level[i];
        const float bs = ldexpf(side, -l);
        const uint64_t pre = prefix[i];
        gc[i] = make_float4(ox + ((float)box_axis(pre, 0, l, frame_level) + 0.5f) * bs,
                            oy + ((float)box_axis(pre, 1, l, frame_level) + 0.5f) * bs,
                            oz + ((float)box_axis(pre, 2, l, frame_level) + 0.5f) * bs, 0.f);
    }
}

// key = level X (5 bits) | level Y (5) | three offsets of 18 bits (biased),
// the offset of centre X from centre Y in half-boxes of the finer level
__global__ void k_far_keys(const int32_t* __restrict__ far_q, const int64_t* __restrict__ nfar,
                           const int32_t* __restrict__ pX, const int32_t* __restrict__ pY,
                           const uint8_t* __restrict__ level, const uint64_t* __restrict__ prefix,
                           uint64_t* __restrict__ key, int32_t* __restrict__ val) {
    const int64_t m = *nfar;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = far_q[k];
        const int32_t X = pX[q], Y = pY[q];
        const int lx = level[X], ly = level[Y], lf = max(lx, ly);
        uint64_t kk = ((uint64_t)lx << 59) | ((uint64_t)ly << 54);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int64_t hx = (2 * box_coord(prefix[X], d) + 1) << (lf - lx);
            const int64_t hy = (2 * box_coord(prefix[Y], d) + 1) << (lf - ly);
            const int64_t o = hx - hy;
            ok = ok && o >= -kOffBias && o < kOffBias;
            kk |= (uint64_t)((o + kOffBias) & ((1 << 18) - 1)) << (36 - 18 * d);
        }
        key[k] = ok ? kk : ~0ull;
        val[k] = q;
    }
}

// group starts: flag where the key changes; ungrouped pairs (key ~0) count
// as no group and their first position is stored in *fallback
__global__ void k_group_flags(const uint64_t* __restrict__ key, const int64_t* __restrict__ nfar,
                              int32_t* __restrict__ flag, int64_t* __restrict__ fallback) {
    const int64_t m = *nfar;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool grouped = key[i] != ~0ull;
        flag[i] = grouped && (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
        if ((i == 0 || key[i - 1] != ~0ull) && !grouped) *fallback = i;
    }
}

// per group: start and number of tiles
__global__ void k_group_starts(const int32_t* __restrict__ flag, const int32_t* __restrict__ gid,
                               const int64_t* __restrict__ nfar,
                               int32_t* __restrict__ gstart) {
    const int64_t m = *nfar;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) gstart[gid[i]] = (int32_t)i;
}

__global__ void k_group_tiles(const int32_t* __restrict__ gstart, const int64_t* __restrict__ ng,
                              const int64_t* __restrict__ fallback, int32_t* __restrict__ ntile) {
    const int64_t G = *ng;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t end = g + 1 < G ? gstart[g + 1] : *fallback;
        ntile[g] = (int32_t)((end - gstart[g] + kGemmTile - 1) / kGemmTile);
    }
}

// tile -> (group, first pair)
__global__ void k_tile_list(const int32_t* __restrict__ gstart, const int32_t* __restrict__ ntile,
                            const int32_t* __restrict__ toff, const int64_t* __restrict__ ng,
                            int2* __restrict__ tiles) {
    const int64_t G = *ng;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x)
        for (int t = 0; t < ntile[g]; ++t)
            tiles[toff[g] + t] = make_int2((int32_t)g, gstart[g] + t * kGemmTile);
}

__device__ void hermite_row(float x, int nmax, float* h) {
    const float h0 = __expf(-x * x);
    h[0] = h0;
    if (nmax >= 1) h[1] = 2.f * x * h0;
    for (int k = 1; k < nmax; ++k) h[k + 1] = 2.f * x * h[k] - 2.f * (float)k * h[k - 1];
}

struct GemmArgs {
    const int2* tiles;
    const int64_t* ntiles;
    const int32_t* gstart;
    const int64_t* ng;
    const int64_t* fallback;     // first ungrouped position (= end of the groups)
    const int32_t* q;            // far pairs in key order
    const uint64_t* key;
    const int32_t* pX;
    const int32_t* pY;
    const float* A;
    const float* M;
    float* B;
    float4* pw;                // the pair table (double-FP32 W of both channels)
    int64_t exp_first;
    int p;
    float half_box_over_sigma_l0;   // side / 2 / sigma (half a level-0 box)
};

// Dynamic shared memory: the operator transposed, Tt[alpha][beta] with beta
// padded to PB = 16 RM rows (zero rows past p^3), the columns As[alpha][64],
// the product Cs[beta][64], the Hermite rows H[3][16], pair ids and W.  The
// product runs on a 16 x 16 grid of threads, each owning RM rows x 4 columns
// in registers (two 16-byte shared-memory loads per 4 RM multiply-adds).
template <int RM>
__global__ void __launch_bounds__(kGemmThreads) k_m2l_gemm(GemmArgs a) {
    extern __shared__ __align__(16) float sm[];
    constexpr int PB = 16 * RM;
    const int p = a.p, p2 = p * p, p3 = p2 * p;
    const int ncol = 2 * kGemmTile;
    float* T = sm;                                   // Tt: p3 x PB
    float* As = T + p3 * PB;
    float* Cs = As + p3 * ncol;                      // PB x ncol
    float* H = Cs + PB * ncol;                       // 3 x 16
    int32_t* sq = reinterpret_cast<int32_t*>(H + 48);  // kGemmTile pair ids
    float* sw = reinterpret_cast<float*>(sq + kGemmTile);   // ncol W values
    const int64_t nt = *a.ntiles;
    const int64_t G = *a.ng;
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int2 tg = a.tiles[tile];
        const int64_t gend = tg.x + 1 < G ? a.gstart[tg.x + 1] : *a.fallback;
        const int npair = (int)min((int64_t)kGemmTile, gend - tg.y);
        // the group's offset from its key
        const uint64_t k0 = a.key[tg.y];
        const int lx = (int)(k0 >> 59), ly = (int)((k0 >> 54) & 31), lf = max(lx, ly);
        if (threadIdx.x < 3) {
            const int d = threadIdx.x;
            const int64_t o = (int64_t)((k0 >> (36 - 18 * d)) & ((1 << 18) - 1)) - kOffBias;
            const float delta = (float)o * ldexpf(a.half_box_over_sigma_l0, -lf);
            hermite_row(delta, 2 * p - 2, H + 16 * d);
        }
        if (threadIdx.x < npair) sq[threadIdx.x] = a.q[tg.y + threadIdx.x];
        __syncthreads();
        // operator, transposed: T[al * PB + b]
        for (int i = threadIdx.x; i < p3 * PB; i += blockDim.x) {
            const int al = i / PB, b = i - al * PB;
            float v = 0.f;
            if (b < p3) {
                const int b0 = b / p2, b1 = (b / p) % p, b2 = b % p;
                const int a0 = al / p2, a1 = (al / p) % p, a2 = al % p;
                float sc = c_inv_fact_g[b0] * c_inv_fact_g[b1] * c_inv_fact_g[b2];
                if ((b0 + b1 + b2) & 1) sc = -sc;
                v = sc * H[a0 + b0] * H[16 + a1 + b1] * H[32 + a2 + b2];
            }
            T[i] = v;
        }
        // coefficient columns: column 2 i + ch = A(Y_i, ch)
        for (int i = threadIdx.x; i < p3 * ncol; i += blockDim.x) {
            const int al = i / ncol, col = i - al * ncol;
            const int pi = col >> 1, ch = col & 1;
            float v = 0.f;
            if (pi < npair) {
                const int64_t ey = a.pY[sq[pi]] - a.exp_first;
                v = a.A[(ey * 2 + ch) * p3 + al];
            }
            As[i] = v;
        }
        __syncthreads();
        // C = T As, RM x 4 outputs per thread
        {
            const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
            const int r0 = ty * RM, c0 = tx * 4;
            float acc[RM][4];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
            for (int al = 0; al < p3; ++al) {
                const float4 av = *reinterpret_cast<const float4*>(As + al * ncol + c0);
#pragma unroll
                for (int i4 = 0; i4 < RM / 4; ++i4) {
                    const float4 tv = *reinterpret_cast<const float4*>(T + al * PB + r0 + 4 * i4);
                    const float t[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        acc[4 * i4 + i][0] = fmaf(t[i], av.x, acc[4 * i4 + i][0]);
                        acc[4 * i4 + i][1] = fmaf(t[i], av.y, acc[4 * i4 + i][1]);
                        acc[4 * i4 + i][2] = fmaf(t[i], av.z, acc[4 * i4 + i][2]);
                        acc[4 * i4 + i][3] = fmaf(t[i], av.w, acc[4 * i4 + i][3]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < RM; ++i)
                *reinterpret_cast<float4*>(Cs + (r0 + i) * ncol + c0) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
        __syncthreads();
        // W per column, B(X) += column
        if (threadIdx.x < ncol) {
            const int col = threadIdx.x, pi = col >> 1, ch = col & 1;
            float w = 0.f;
            if (pi < npair) {
                const int64_t ex = a.pX[sq[pi]] - a.exp_first;
                const float* Mx = a.M + (ex * 2 + ch) * p3;
                for (int b = 0; b < p3; ++b) w = fmaf(Cs[b * ncol + col], Mx[b], w);
            }
            sw[col] = w;
        }
        for (int i = threadIdx.x; i < p3 * ncol; i += blockDim.x) {
            const int b = i / ncol, col = i - b * ncol;
            const int pi = col >> 1, ch = col & 1;
            if (pi < npair) {
                const int64_t ex = a.pX[sq[pi]] - a.exp_first;
                atomicAdd(&a.B[(ex * 2 + ch) * p3 + b], Cs[i]);
            }
        }
        __syncthreads();
        if (threadIdx.x < npair)
            a.pw[sq[threadIdx.x]] = make_float4(sw[2 * threadIdx.x], 0.f,
                                               sw[2 * threadIdx.x + 1], 0.f);
        __syncthreads();
    }
}

}  // namespace

void geo_centres(msp_ctx& c, cudaStream_t s) {
    float4* gc = c.nd_gc.ensure<float4>((size_t)std::max<int64_t>(c.n_nodes, 1));
    k_geo_centres<<<grid_for(c.n_nodes, 256, (int64_t)c.sm_count * 8), 256, 0, s>>>(
        c.n_nodes, c.nd_level.get<uint8_t>(), c.nd_prefix.get<uint64_t>(), c.frame_level,
        c.frame_level > 0 ? 0.f : c.cfg.origin[0], c.frame_level > 0 ? 0.f : c.cfg.origin[1],
        c.frame_level > 0 ? 0.f : c.cfg.origin[2], c.cfg.side, gc);
    MSP_LAUNCH("geo_centres");
}

bool m2l_gemm_fits(int p) { return p <= kGemmMaxP; }

// Translations of the far pairs far_q[0, *nfar) grouped by offset.  On return
// the far pairs are in key order in c.gm_q and *first_fallback (device)
// holds the position from which the caller translates pair by pair.
const int32_t* m2l_gemm(msp_ctx& c, const int32_t* far_q, const int64_t* nfar, int64_t cap,
                        const float* A, const float* M, float* B, float4* pw,
                        int64_t** first_fallback, cudaStream_t s) {
    const size_t ncap = (size_t)std::max<int64_t>(cap, 1);
    uint64_t* k0 = c.gm_key0.ensure<uint64_t>(ncap);
    uint64_t* k1 = c.gm_key1.ensure<uint64_t>(ncap);
    int32_t* v0 = c.gm_q.ensure<int32_t>(ncap);
    int32_t* v1 = c.gm_q1.ensure<int32_t>(ncap);
    int32_t* flag = c.gm_flag.ensure<int32_t>(ncap);
    int32_t* gid = c.gm_gid.ensure<int32_t>(ncap);
    int32_t* gstart = c.gm_gstart.ensure<int32_t>(ncap);
    int32_t* ntile = c.gm_ntile.ensure<int32_t>(ncap);
    int32_t* toff = c.gm_toff.ensure<int32_t>(ncap);
    int2* tiles = c.gm_tiles.ensure<int2>(ncap);
    int64_t* cnt = c.gm_cnt.ensure<int64_t>(4);   // groups, tiles, first ungrouped
    const int ge = (int)c.sm_count * 8;
    k_far_keys<<<ge, 256, 0, s>>>(far_q, nfar, c.pr_X.get<int32_t>(), c.pr_Y.get<int32_t>(),
                                  c.nd_level.get<uint8_t>(), c.nd_prefix.get<uint64_t>(), k0, v0);
    MSP_LAUNCH("far_keys");
    radix_sort_dev(c, k0, v0, k1, v1, nfar, cap, 64, s);
    MSP_CUDA(cudaMemcpyAsync(cnt + 2, nfar, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    k_group_flags<<<ge, 256, 0, s>>>(k0, nfar, flag, cnt + 2);
    MSP_LAUNCH("group_flags");
    scan_dev(c, flag, gid, nfar, cap, cnt, nullptr, s);
    // gid holds the exclusive count: a group's index is gid at its flag
    k_group_starts<<<ge, 256, 0, s>>>(flag, gid, nfar, gstart);
    MSP_LAUNCH("group_starts");
    k_group_tiles<<<ge, 256, 0, s>>>(gstart, cnt, cnt + 2, ntile);
    MSP_LAUNCH("group_tiles");
    scan_dev(c, ntile, toff, cnt, cap, cnt + 1, nullptr, s);
    k_tile_list<<<ge, 256, 0, s>>>(gstart, ntile, toff, cnt, tiles);
    MSP_LAUNCH("tile_list");
    const int p = c.cfg.p, p3 = p * p * p;
    const int RM = p3 <= 64 ? 4 : 8;
    const size_t PB = 16 * (size_t)RM, ncol = 2 * kGemmTile;
    const size_t smem = sizeof(float) * ((size_t)p3 * PB + (size_t)p3 * ncol + PB * ncol + 48) +
                        sizeof(int32_t) * kGemmTile + sizeof(float) * ncol;
    if (smem > 48 * 1024 && (int)smem > c.gm_smem_set) {
        MSP_CUDA(cudaFuncSetAttribute(k_m2l_gemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        MSP_CUDA(cudaFuncSetAttribute(k_m2l_gemm<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        c.gm_smem_set = (int)smem;
    }
    GemmArgs a;
    a.tiles = tiles;
    a.ntiles = cnt + 1;
    a.gstart = gstart;
    a.ng = cnt;
    a.fallback = cnt + 2;
    a.q = v0;
    a.key = k0;
    a.pX = c.pr_X.get<int32_t>();
    a.pY = c.pr_Y.get<int32_t>();
    a.A = A;
    a.M = M;
    a.B = B;
    a.pw = pw;
    a.exp_first = c.exp_first;
    a.p = p;
    a.half_box_over_sigma_l0 = (float)(0.5 * (double)c.cfg.side / c.cfg.sigma);
    const int grid = (int)c.sm_count * (smem <= 64 * 1024 ? 3 : 1);
    if (RM == 4) k_m2l_gemm<4><<<grid, kGemmThreads, smem, s>>>(a);
    else         k_m2l_gemm<8><<<grid, kGemmThreads, smem, s>>>(a);
    MSP_LAUNCH("m2l_gemm");
    *first_fallback = cnt + 2;
    return v0;
}

}  // namespace msp
