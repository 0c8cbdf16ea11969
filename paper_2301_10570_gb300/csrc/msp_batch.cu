// msp_batch.cu -- many independent networks as one problem.
//
// The attraction depends on positions only through |t - s| / sigma, so a
// network scaled by 1/sigma has kernel width 1.  Network k (neurons
// [off_k, off_k+1) of the concatenated arrays) is scaled by 1/sigma_k and
// given its own cell of a grid of octree boxes at level L0, using every other
// cell in each dimension: any two networks are at least one empty cell (wider
// than the cutoff) apart.  Its positions are written relative to its cell's
// low corner (its own frame), and a context told of the frames
// (msp_set_frames) puts the cell in the top bits of every Morton key and
// forms each box centre in the box's network's frame, so no position is ever
// rounded to the resolution of the whole batch's domain.  Then
//   - every box pair between networks is pruned by the box-distance test at
//     the first level where the boxes are separated, so no attraction, pair
//     weight or draw ever crosses networks;
//   - every network has more than C neurons, so every box above level L0 is
//     split and every leaf, and every axon box whose choice its neurons share
//     (Algorithm 1), lies inside one network's cell;
// and the single-network path (tree, traversal, near field, descent,
// resolution) runs on the whole batch in one pass, unchanged.  The cell side
// is a power of two, so a network's key is exactly the key its points would
// have in one common frame.
#include <algorithm>
#include <cmath>
#include <vector>

#include "msp_internal.cuh"

namespace msp {

void set_last_error(const char* msg);

namespace {

// per-network bounds: one block per network, {lo x, lo y, lo z, hi x, hi y, hi z}
__global__ void k_batch_bounds(const int64_t* __restrict__ off, const float* __restrict__ x,
                               const float* __restrict__ y, const float* __restrict__ z,
                               float* __restrict__ bounds) {
    const int64_t k = blockIdx.x;
    const int64_t i0 = off[k], i1 = off[k + 1];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const float v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lo[d] = fminf(lo[d], v[d]);
            hi[d] = fmaxf(hi[d], v[d]);
        }
    }
    __shared__ float red[6][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
        if (lane == 0) {
            red[d][w] = lo[d];
            red[3 + d][w] = hi[d];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int nw = blockDim.x >> 5;
        float v = red[threadIdx.x][0];
        for (int k2 = 1; k2 < nw; ++k2)
            v = threadIdx.x < 3 ? fminf(v, red[threadIdx.x][k2]) : fmaxf(v, red[threadIdx.x][k2]);
        bounds[6 * k + threadIdx.x] = v;
    }
}

// place: one block per network; p' = (p - lo_k) / sigma_k, relative to the
// network's own cell, formed in double precision and rounded once
__global__ void k_batch_place(const int64_t* __restrict__ off, const float* __restrict__ x,
                              const float* __restrict__ y, const float* __restrict__ z,
                              const float* __restrict__ bounds, const double* __restrict__ sigma,
                              float* __restrict__ xo, float* __restrict__ yo,
                              float* __restrict__ zo) {
    const int64_t k = blockIdx.x;
    const int64_t i0 = off[k], i1 = off[k + 1];
    const double lx = bounds[6 * k], ly = bounds[6 * k + 1], lz = bounds[6 * k + 2];
    const double sg = sigma[k];
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        xo[i] = (float)(((double)x[i] - lx) / sg);
        yo[i] = (float)(((double)y[i] - ly) / sg);
        zo[i] = (float)(((double)z[i] - lz) / sg);
    }
}

}  // namespace

void batch_layout(int64_t nnet, const int64_t* off_host, const float* x, const float* y,
                  const float* z, const double* sigma, double cutoff, int leaf_capacity,
                  float* xo, float* yo, float* zo, float* side_out, int* level_out,
                  cudaStream_t s) {
    NvtxRange nv_("msp batch_layout");
    for (int64_t k = 0; k < nnet; ++k) {
        if (off_host[k + 1] <= off_host[k] + leaf_capacity)
            throw Error(MSP_ERR_INVALID_ARG, "every network needs more neurons than the leaf capacity");
        if (!(sigma[k] > 0.0)) throw Error(MSP_ERR_INVALID_ARG, "sigma must be positive");
    }
    DBuf d_off, d_bounds, d_place;
    try {
        int64_t* off = d_off.ensure<int64_t>((size_t)nnet + 1);
        float* bounds = d_bounds.ensure<float>((size_t)6 * nnet);
        double* place = d_place.ensure<double>((size_t)nnet);
        MSP_CUDA(cudaMemcpyAsync(off, off_host, (nnet + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
        k_batch_bounds<<<(unsigned)nnet, 256, 0, s>>>(off, x, y, z, bounds);
        MSP_LAUNCH("batch_bounds");
        std::vector<float> hb((size_t)6 * nnet);
        MSP_CUDA(cudaMemcpyAsync(hb.data(), bounds, hb.size() * sizeof(float),
                                 cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        // cell side: the widest scaled network plus a margin, rounded up to a
        // power of two
        double ext = 0.0;
        for (int64_t k = 0; k < nnet; ++k)
            for (int d = 0; d < 3; ++d) {
                const double e = ((double)hb[6 * k + 3 + d] - (double)hb[6 * k + d]) / sigma[k];
                if (!std::isfinite(e)) throw Error(MSP_ERR_INVALID_ARG, "non-finite position");
                ext = std::max(ext, e);
            }
        const double cell = std::exp2(std::ceil(std::log2(ext * (1.0 + 1e-3) + cutoff + 1.0)));
        if (!(cell < 1e30)) throw Error(MSP_ERR_INVALID_ARG, "networks too wide");
        // networks on the even cells of a 2G x 2G x 2G grid, G a power of two
        int lg = 0;
        while ((int64_t)1 << (3 * lg) < nnet) ++lg;
        const int64_t G = (int64_t)1 << lg;
        const int L0 = lg + 1;
        if (L0 > kMortonBits - 8) throw Error(MSP_ERR_INVALID_ARG, "too many networks");
        MSP_CUDA(cudaMemcpyAsync(place, sigma, (size_t)nnet * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
        k_batch_place<<<(unsigned)nnet, 256, 0, s>>>(off, x, y, z, bounds, place, xo, yo, zo);
        MSP_LAUNCH("batch_place");
        MSP_CUDA(cudaStreamSynchronize(s));
        *side_out = (float)(2.0 * (double)G * cell);
        *level_out = L0;
    } catch (...) {
        cudaStreamSynchronize(s);
        d_off.release();
        d_bounds.release();
        d_place.release();
        throw;
    }
    d_off.release();
    d_bounds.release();
    d_place.release();
}

}  // namespace msp

extern "C" msp_status msp_batch_layout(int64_t n_networks, const int64_t* offsets,
                                       const float* x, const float* y, const float* z,
                                       const double* sigma, double cutoff, int leaf_capacity,
                                       float* x_out, float* y_out, float* z_out,
                                       float* side_out, int* level_out, void* stream) {
    if (n_networks < 1 || n_networks > (1 << 24) || !offsets || !sigma || !side_out ||
        !level_out || !(cutoff > 0.0) || !(cutoff <= 5.0) || leaf_capacity < 1) {
        msp::set_last_error("msp_batch_layout: argument out of range or null");
        return MSP_ERR_INVALID_ARG;
    }
    if (offsets[0] != 0) {
        msp::set_last_error("msp_batch_layout: offsets[0] must be 0");
        return MSP_ERR_INVALID_ARG;
    }
    for (int64_t k = 0; k < n_networks; ++k)
        if (offsets[k + 1] < offsets[k]) {
            msp::set_last_error("msp_batch_layout: offsets must not decrease");
            return MSP_ERR_INVALID_ARG;
        }
    if (offsets[n_networks] >= 0x7fffffffll || !x || !y || !z || !x_out || !y_out || !z_out) {
        msp::set_last_error("msp_batch_layout: total size out of range or null pointer");
        return MSP_ERR_INVALID_ARG;
    }
    try {
        msp::batch_layout(n_networks, offsets, x, y, z, sigma, cutoff, leaf_capacity, x_out, y_out,
                          z_out, side_out, level_out, reinterpret_cast<cudaStream_t>(stream));
    } catch (const msp::Error& e) {
        msp::set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        msp::set_last_error(e.what());
        return MSP_ERR_CUDA;
    }
    msp::set_last_error("");
    return MSP_OK;
}
