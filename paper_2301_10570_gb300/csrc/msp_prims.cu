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

__global__ void k_sd_reduce(const int32_t* __restrict__ in, const int64_t* __restrict__ n_dev,
                            long long* __restrict__ bsum) {
    const int64_t n = *n_dev;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    __shared__ long long tot;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        long long s = 0;
        for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
            int64_t i = t * kScanTile + j;
            if (i < n) s += in[i];
        }
        long long d = block_excl_scan(s, &tot);
        (void)d;
        if (threadIdx.x == 0) bsum[t] = tot;
        __syncthreads();
    }
}

// one block: exclusive scan of the tile sums in chunks, total (+ *base) to
// *dst.  With a clamp, an end beyond clamp_cap is recorded (overflow bit 0,
// need = the largest end asked for) and *dst gets *base instead: the next
// range is empty.
__global__ void k_sd_spine(long long* __restrict__ bsum, const int64_t* __restrict__ n_dev,
                           int64_t* __restrict__ dst, const int64_t* __restrict__ base,
                           int64_t clamp_cap, int64_t* __restrict__ overflow,
                           int64_t* __restrict__ need, int64_t overflow_bit) {
    const int64_t n = *n_dev;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    __shared__ long long chunk_total;
    long long carry = 0;
    for (int64_t c0 = 0; c0 < ntiles; c0 += (int64_t)kScanThreads * kScanItems) {
        long long v[kScanItems];
        long long s = 0;
        const int64_t b = c0 + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            v[j] = b + j < ntiles ? bsum[b + j] : 0;
            s += v[j];
        }
        long long pre = block_excl_scan(s, &chunk_total) + carry;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            if (b + j < ntiles) bsum[b + j] = pre;
            pre += v[j];
        }
        carry += chunk_total;
        __syncthreads();
    }
    if (threadIdx.x == 0 && dst) {
        const int64_t b = base ? *base : 0;
        int64_t end = carry + b;
        if (overflow && end > clamp_cap) {
            atomicOr(reinterpret_cast<unsigned long long*>(overflow),
                     (unsigned long long)overflow_bit);
            atomicMax(reinterpret_cast<unsigned long long*>(need), (unsigned long long)end);
            end = b;
        }
        *dst = end;
    }
}

__global__ void k_sd_apply(const int32_t* in, int32_t* out, const int64_t* __restrict__ n_dev,
                           const long long* __restrict__ bsum) {
    const int64_t n = *n_dev;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    __shared__ long long tot;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * kScanTile + (int64_t)threadIdx.x * kScanItems;
        long long v[kScanItems];
        long long s = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            v[j] = base + j < n ? in[base + j] : 0;
            s += v[j];
        }
        long long pre = block_excl_scan(s, &tot) + bsum[t];
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            if (base + j < n) out[base + j] = (int32_t)pre;
            pre += v[j];
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
}

void scan_dev(msp_ctx& c, const int32_t* in, int32_t* out, const int64_t* n_dev, int64_t n_cap,
              int64_t* total_dst, const int64_t* base, cudaStream_t s, int64_t clamp_cap,
              int64_t* overflow, int64_t* need, int64_t overflow_bit) {
    const int64_t tiles_cap = std::max<int64_t>((n_cap + kScanTile - 1) / kScanTile, 1);
    long long* bsum = c.sd_tmp.ensure<long long>((size_t)tiles_cap);
    const int G = (int)std::min<int64_t>(tiles_cap, (int64_t)c.sm_count * 8);
    k_sd_reduce<<<G, kScanThreads, 0, s>>>(in, n_dev, bsum);
    MSP_LAUNCH("scan_dev_reduce");
    k_sd_spine<<<1, kScanThreads, 0, s>>>(bsum, n_dev, total_dst, base, clamp_cap, overflow,
                                          need, overflow_bit);
    MSP_LAUNCH("scan_dev_spine");
    k_sd_apply<<<G, kScanThreads, 0, s>>>(in, out, n_dev, bsum);
    MSP_LAUNCH("scan_dev_apply");
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
