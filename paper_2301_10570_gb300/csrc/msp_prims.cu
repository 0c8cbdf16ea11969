// msp_prims.cu -- device-wide exclusive scan and stable LSD radix sort used by
// the tree build, the pair lists, the descent and the request resolution.
#include "msp_internal.cuh"

namespace msp {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline long long warp_incl_scan(long long v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan over the block of one value per thread; returns the block total
__device__ inline long long block_excl_scan(long long v, long long* total) {
    __shared__ long long warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        long long si = warp_incl_scan(s);
        if (lane < kScanThreads / 32) warp_sums[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) *total = si;
    }
    __syncthreads();
    long long r = inc - v + warp_sums[w];
    __syncthreads();
    return r;
}

// per-tile sums (int64)
template <class T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, long long* __restrict__ bsum) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
        int64_t i = base + j;
        if (i < n) s += (long long)in[i];
    }
    __shared__ long long tot;
    long long dummy = block_excl_scan(s, &tot);
    (void)dummy;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// exclusive scan of one tile, plus the tile's offset; the last tile writes the
// grand total to *total
template <class Tin, class Tout>
__global__ void k_scan_tile(const Tin* in, Tout* out, int64_t n,   // may alias
                            const long long* __restrict__ boff, long long* __restrict__ total) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j;
        v[j] = i < n ? (long long)in[i] : 0;
        s += v[j];
    }
    __shared__ long long tile_total;
    long long pre = block_excl_scan(s, &tile_total);
    long long off = boff ? boff[blockIdx.x] : 0;
    pre += off;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j;
        if (i < n) out[i] = (Tout)pre;
        pre += v[j];
    }
    if (threadIdx.x == 0 && blockIdx.x == gridDim.x - 1 && total) *total = off + tile_total;
}

// recursive scan of n int64 block sums in place (out may alias in)
void scan_i64(msp_ctx& c, long long* data, int64_t n, long long* total, long long* scratch,
              cudaStream_t s) {
    if (n <= kScanTile) {
        k_scan_tile<long long, long long><<<1, kScanThreads, 0, s>>>(data, data, n, nullptr, total);
        MSP_LAUNCH("scan_tile_i64");
        return;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    long long* bsum = scratch;
    k_scan_reduce<long long><<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, bsum);
    MSP_LAUNCH("scan_reduce_i64");
    scan_i64(c, bsum, nb, nullptr, scratch + nb, s);
    k_scan_tile<long long, long long><<<(unsigned)nb, kScanThreads, 0, s>>>(data, data, n, bsum,
                                                                          total);
    MSP_LAUNCH("scan_tile_i64");
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                             int32_t* __restrict__ hist, int nb) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int j = threadIdx.x; j < kRsTile; j += kRsThreads) {
        int64_t i = base + j;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items of a tile are ranked in index order within their
// digit.  Round r covers tile positions [r*256, r*256+256), thread order =
// index order; within a warp the rank comes from the lanes with the same digit,
// across warps from the per-warp digit counts of the round.
__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                int64_t n, int shift, const int32_t* __restrict__ offs, int nb,
                                uint64_t* __restrict__ kout, int32_t* __restrict__ vout) {
    __shared__ int32_t running[256];
    __shared__ int32_t wcnt[kRsWarps][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    running[t] = offs[(int64_t)t * nb + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kRsWarps; ++k) wcnt[k][t] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; ++r) {
        int64_t i = base + (int64_t)r * kRsThreads + t;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int32_t val = valid ? vin[i] : 0;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = running[d] + rank;
            for (int k = 0; k < w; ++k) pos += wcnt[k][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int k = 0; k < kRsWarps; ++k) {
            add += wcnt[k][t];
            wcnt[k][t] = 0;
        }
        running[t] += add;
        __syncthreads();
    }
}

__global__ void k_copy_kv(const uint64_t* __restrict__ ks, const int32_t* __restrict__ vs,
                          int64_t n, uint64_t* __restrict__ kd, int32_t* __restrict__ vd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        kd[i] = ks[i];
        vd[i] = vs[i];
    }
}

}  // namespace

void radix_sort(msp_ctx& c, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp, int32_t* vals_tmp,
                int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    int nb = (int)((n + kRsTile - 1) / kRsTile);
    int32_t* hist = c.rs_hist.ensure<int32_t>((size_t)256 * nb);
    int passes = (bits + 7) / 8;
    uint64_t *ka = keys, *kb = keys_tmp;
    int32_t *va = vals, *vb = vals_tmp;
    for (int ps = 0; ps < passes; ++ps) {
        int shift = 8 * ps;
        k_radix_hist<<<nb, kRsThreads, 0, s>>>(ka, n, shift, hist, nb);
        MSP_LAUNCH("radix_hist");
        // exclusive scan of the digit-major histogram: offsets of (digit, tile)
        {
            int64_t m = (int64_t)256 * nb;
            int64_t tb = (m + kScanTile - 1) / kScanTile;
            long long* scratch = c.scan_tmp.ensure<long long>((size_t)(2 * tb + 64));
            if (tb == 1) {
                k_scan_tile<int32_t, int32_t><<<1, kScanThreads, 0, s>>>(hist, hist, m, nullptr,
                                                                      nullptr);
            } else {
                k_scan_reduce<int32_t><<<(unsigned)tb, kScanThreads, 0, s>>>(hist, m, scratch);
                scan_i64(c, scratch, tb, nullptr, scratch + tb, s);
                k_scan_tile<int32_t, int32_t><<<(unsigned)tb, kScanThreads, 0, s>>>(
                    hist, hist, m, scratch, nullptr);
            }
            MSP_LAUNCH("radix_scan");
        }
        k_radix_scatter<<<nb, kRsThreads, 0, s>>>(ka, va, n, shift, hist, nb, kb, vb);
        MSP_LAUNCH("radix_scatter");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        k_copy_kv<<<grid_for(n, 256, 4096), 256, 0, s>>>(ka, va, n, keys, vals);
        MSP_LAUNCH("radix_copy");
    }
}

// ---------------------------------------------------------------------------
// the same primitives with the element count in device memory (no host sync;
// launch shapes come from a host-side capacity bound)
// ---------------------------------------------------------------------------
namespace {

// Single-pass exclusive scan of in[0, *n_dev) with a decoupled look-back.
// Blocks take tiles in order from a counter (status[0]), so every tile's
// predecessors have started; a tile publishes its sum (flag 1) before it
// looks back, then its inclusive prefix (flag 2), in status[1 + tile] as one
// 64-bit word (flag in the top two bits).  The look-back reads 32
// predecessors per step with a warp, waiting on each for at most kSpinLimit
// polls; a wait that gives up sets bit kScanTimeoutBit in *overflow and
// counts the tile as 0 (the result is then wrong and the host reports it).
// The last tile writes the total (+ *base) to *dst; with a clamp, an end
// beyond clamp_cap is recorded (overflow_bit, need = the largest end asked
// for) and *dst gets *base instead: the next range is empty.
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;

__global__ void __launch_bounds__(kScanThreads)
k_scan_1p(const int32_t* in, int32_t* out, const int64_t* __restrict__ n_dev,
          unsigned long long* status, int64_t* __restrict__ dst,
          const int64_t* __restrict__ base, int64_t clamp_cap, int64_t* __restrict__ overflow,
          int64_t* __restrict__ need, int64_t overflow_bit, int64_t timeout_bit, int spin_limit) {
    __shared__ int32_t s_v[kScanTile + kScanTile / 32];
    __shared__ long long s_tot, s_excl;
    __shared__ int64_t s_tile;
    const int64_t n = *n_dev;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    volatile unsigned long long* st = status;
    if (ntiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && dst) *dst = base ? *base : 0;
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(&status[0], 1ull);
        __syncthreads();
        const int64_t t = s_tile;
        __syncthreads();
        if (t >= ntiles) break;
        const int64_t t0 = t * kScanTile;
        // coalesced load into shared memory (one padding word per 32)
        for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
            const int64_t i = t0 + j;
            s_v[j + (j >> 5)] = i < n ? in[i] : 0;
        }
        __syncthreads();
        // each thread: kScanItems consecutive values
        long long v[kScanItems];
        long long sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int j = threadIdx.x * kScanItems + k;
            v[k] = s_v[j + (j >> 5)];
            sum += v[k];
        }
        const long long pre = block_excl_scan(sum, &s_tot);
        const long long agg = s_tot;
        // publish the sum, then look back
        if (threadIdx.x == 0)
            st[1 + t] = (t == 0 ? kFlagPre : kFlagAgg) | ((unsigned long long)agg & kValMask);
        if (threadIdx.x < 32) {
            long long excl = 0;
            int64_t j = t - 1;
            const int lane = threadIdx.x;
            while (j >= 0) {
                const int64_t jj = j - lane;
                unsigned long long w = kFlagPre;     // lanes past tile 0 count as a prefix of 0
                if (jj >= 0) {
                    int spin = 0;
                    w = st[1 + jj];
                    while ((w >> 62) == 0 && spin < spin_limit) {
                        ++spin;
                        w = st[1 + jj];
                    }
                    if ((w >> 62) == 0) {
                        atomicOr(reinterpret_cast<unsigned long long*>(overflow),
                                 (unsigned long long)timeout_bit);
                        w = kFlagPre;
                    }
                }
                const unsigned pmask = __ballot_sync(0xffffffffu, (w >> 62) == 2);
                const int stop = pmask ? __ffs(pmask) - 1 : 31;   // first prefix, else all 32
                long long val = lane <= stop ? (long long)(w & kValMask) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                excl += val;
                if (pmask) break;
                j -= 32;
            }
            if (lane == 0) {
                s_excl = excl;
                if (t > 0) st[1 + t] = kFlagPre | ((unsigned long long)(excl + agg) & kValMask);
            }
        }
        __syncthreads();
        const long long excl = s_excl;
        // offsets through shared memory, stored coalesced
        long long run = excl + pre;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int j = threadIdx.x * kScanItems + k;
            s_v[j + (j >> 5)] = (int32_t)run;
            run += v[k];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
            const int64_t i = t0 + j;
            if (i < n) out[i] = s_v[j + (j >> 5)];
        }
        if (t == ntiles - 1 && threadIdx.x == 0 && dst) {
            const int64_t b = base ? *base : 0;
            int64_t end = excl + agg + b;
            if (overflow && end > clamp_cap && clamp_cap > 0) {
                atomicOr(reinterpret_cast<unsigned long long*>(overflow),
                         (unsigned long long)overflow_bit);
                atomicMax(reinterpret_cast<unsigned long long*>(need), (unsigned long long)end);
                end = b;
            }
            *dst = end;
        }
        __syncthreads();
    }
}

__global__ void k_radix_hist_dev(const uint64_t* __restrict__ keys, const int64_t* __restrict__ n_dev,
                                 int shift, int32_t* __restrict__ hist, int nb) {
    __shared__ int32_t h[256];
    const int64_t n = *n_dev;
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int j = threadIdx.x; j < kRsTile; j += kRsThreads) {
        int64_t i = base + j;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter_dev(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                    const int64_t* __restrict__ n_dev, int shift,
                                    const int32_t* __restrict__ offs, int nb,
                                    uint64_t* __restrict__ kout, int32_t* __restrict__ vout) {
    const int64_t n = *n_dev;
    if ((int64_t)blockIdx.x * kRsTile >= n) return;       // whole block idle
    __shared__ int32_t running[256];
    __shared__ int32_t wcnt[kRsWarps][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    running[t] = offs[(int64_t)t * nb + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kRsWarps; ++k) wcnt[k][t] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; ++r) {
        int64_t i = base + (int64_t)r * kRsThreads + t;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int32_t val = valid ? vin[i] : 0;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = running[d] + rank;
            for (int k = 0; k < w; ++k) pos += wcnt[k][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int k = 0; k < kRsWarps; ++k) {
            add += wcnt[k][t];
            wcnt[k][t] = 0;
        }
        running[t] += add;
        __syncthreads();
    }
}

__global__ void k_copy_kv_dev(const uint64_t* __restrict__ ks, const int32_t* __restrict__ vs,
                              const int64_t* __restrict__ n_dev, uint64_t* __restrict__ kd,
                              int32_t* __restrict__ vd) {
    const int64_t n = *n_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        kd[i] = ks[i];
        vd[i] = vs[i];
    }
}

}  // namespace

namespace {
__global__ void k_dev_set(int64_t* dst, int64_t v) { *dst = v; }
__global__ void k_dev_store_i32(int32_t* dst, const int64_t* src) { *dst = (int32_t)*src; }
}  // namespace

void dev_set(int64_t* dst, int64_t v, cudaStream_t s) {
    k_dev_set<<<1, 1, 0, s>>>(dst, v);
    MSP_LAUNCH("dev_set");
}
void dev_store_i32(int32_t* dst, const int64_t* src, cudaStream_t s) {
    k_dev_store_i32<<<1, 1, 0, s>>>(dst, src);
    MSP_LAUNCH("dev_store_i32");
}
void pull_counts(msp_ctx& c, cudaStream_t s) {
    MSP_CUDA(cudaMemcpyAsync(c.hcount, c.dcount.p, sizeof(DevCounts), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    if (c.hcount->overflow & kScanTimeoutBit) {
        c.hcount->overflow &= ~kScanTimeoutBit;
        dev_set(&dcounts(c)->overflow, c.hcount->overflow, s);
        throw Error(MSP_ERR_TIMEOUT, "a bounded wait of the device scan gave up");
    }
}

void scan_dev(msp_ctx& c, const int32_t* in, int32_t* out, const int64_t* n_dev, int64_t n_cap,
              int64_t* total_dst, const int64_t* base, cudaStream_t s, int64_t clamp_cap,
              int64_t* overflow, int64_t* need, int64_t overflow_bit) {
    const int64_t tiles_cap = std::max<int64_t>((n_cap + kScanTile - 1) / kScanTile, 1);
    // single pass: a tile counter and one status word per tile, cleared first
    unsigned long long* status = c.sd_tmp.ensure<unsigned long long>((size_t)tiles_cap + 1);
    MSP_CUDA(cudaMemsetAsync(status, 0, ((size_t)tiles_cap + 1) * sizeof(unsigned long long), s));
    const int G = (int)std::min<int64_t>(tiles_cap, (int64_t)c.sm_count * 4);
    DevCounts* dc = dcounts(c);
    k_scan_1p<<<G, kScanThreads, 0, s>>>(in, out, n_dev, status, total_dst, base,
                                         overflow ? clamp_cap : 0, overflow ? overflow : &dc->overflow,
                                         need, overflow_bit, kScanTimeoutBit, kSpinLimit);
    MSP_LAUNCH("scan_dev");
}

// The scan's bounded wait, exercised: the tile counter starts at 1, so tile
// 0 is never taken and its status never published; the tiles after it wait
// on it at most `spin_limit` polls, give up, record the timeout bit and
// finish.  pull_counts then reports MSP_ERR_TIMEOUT.
void scan_wait_selftest(msp_ctx& c, cudaStream_t s) {
    const int64_t n = 3 * (int64_t)kScanTile;
    int32_t* in = c.cnt.ensure<int32_t>((size_t)n);
    int32_t* out = c.off.ensure<int32_t>((size_t)n);
    int64_t* nd = c.gm_cnt.ensure<int64_t>(4);
    unsigned long long* status = c.sd_tmp.ensure<unsigned long long>(4 + 1);
    MSP_CUDA(cudaMemsetAsync(in, 0, (size_t)n * sizeof(int32_t), s));
    MSP_CUDA(cudaMemsetAsync(status, 0, 5 * sizeof(unsigned long long), s));
    dev_set(reinterpret_cast<int64_t*>(status), 1, s);       // tile 0 is skipped
    dev_set(nd, n, s);
    k_scan_1p<<<3, kScanThreads, 0, s>>>(in, out, nd, status, nd + 1, nullptr, 0,
                                         &dcounts(c)->overflow, nullptr, 0, kScanTimeoutBit,
                                         1 << 12);
    MSP_LAUNCH("scan_wait_selftest");
    pull_counts(c, s);
}

void radix_sort_dev(msp_ctx& c, uint64_t* keys, int32_t* vals, uint64_t* keys_tmp,
                    int32_t* vals_tmp, const int64_t* n_dev, int64_t n_cap, int bits,
                    cudaStream_t s) {
    if (n_cap <= 1 || bits <= 0) return;
    const int nb = (int)((n_cap + kRsTile - 1) / kRsTile);
    int32_t* hist = c.rs_hist.ensure<int32_t>((size_t)256 * nb);
    const int passes = (bits + 7) / 8;
    uint64_t *ka = keys, *kb = keys_tmp;
    int32_t *va = vals, *vb = vals_tmp;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
        k_radix_hist_dev<<<nb, kRsThreads, 0, s>>>(ka, n_dev, shift, hist, nb);
        MSP_LAUNCH("radix_hist_dev");
        const int64_t m = (int64_t)256 * nb;
        const int64_t tb = (m + kScanTile - 1) / kScanTile;
        long long* scratch = c.scan_tmp.ensure<long long>((size_t)(2 * tb + 64));
        if (tb == 1) {
            k_scan_tile<int32_t, int32_t><<<1, kScanThreads, 0, s>>>(hist, hist, m, nullptr, nullptr);
        } else {
            k_scan_reduce<int32_t><<<(unsigned)tb, kScanThreads, 0, s>>>(hist, m, scratch);
            scan_i64(c, scratch, tb, nullptr, scratch + tb, s);
            k_scan_tile<int32_t, int32_t><<<(unsigned)tb, kScanThreads, 0, s>>>(hist, hist, m,
                                                                              scratch, nullptr);
        }
        MSP_LAUNCH("radix_scan_dev");
        k_radix_scatter_dev<<<nb, kRsThreads, 0, s>>>(ka, va, n_dev, shift, hist, nb, kb, vb);
        MSP_LAUNCH("radix_scatter_dev");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        k_copy_kv_dev<<<grid_for(n_cap, 256, (int64_t)c.sm_count * 16), 256, 0, s>>>(
            ka, va, n_dev, keys, vals);
        MSP_LAUNCH("radix_copy_dev");
    }
}

}  // namespace msp

// ---------------------------------------------------------------------------
// The counter-based generator of every draw, on caller-given counters and
// keys (msp_philox of include/msp.h)
// ---------------------------------------------------------------------------
namespace {
__global__ void k_philox_blocks(int64_t n, const uint32_t* __restrict__ ctr,
                                const uint32_t* __restrict__ key, uint32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        msp::philox4x32_10(c, key[2 * i], key[2 * i + 1]);
        out[4 * i] = c[0];
        out[4 * i + 1] = c[1];
        out[4 * i + 2] = c[2];
        out[4 * i + 3] = c[3];
    }
}
}  // namespace

extern "C" msp_status msp_philox(int64_t n, const uint32_t* ctr, const uint32_t* key,
                                 uint32_t* out, void* stream) {
    if (n < 0) {
        msp::set_last_error("msp_philox: n must not be negative");
        return MSP_ERR_INVALID_ARG;
    }
    if (n == 0) return MSP_OK;
    if (!ctr || !key || !out) {
        msp::set_last_error("msp_philox: null pointer");
        return MSP_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_philox_blocks<<<msp::grid_for(n, 256), 256, 0, s>>>(n, ctr, key, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        msp::set_last_error(cudaGetErrorString(e));
        return MSP_ERR_CUDA;
    }
    msp::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    msp::set_last_error("");
    return MSP_OK;
}
