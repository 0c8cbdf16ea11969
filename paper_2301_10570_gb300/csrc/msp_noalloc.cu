// msp_noalloc.cu -- msp_direct_noalloc: the all-pairs attraction of Eq. 8 for
// callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a simulation loop that
// must never block on the allocator (cudaMalloc/cudaFree can synchronise the
// whole device and take unbounded time), or a host framework that owns every
// device allocation through its own pool and forbids libraries to allocate
// behind its back.  This entry point needs no context (msp_create allocates)
// and no workspace: its scratch is a fixed, file-scope device array that is
// part of the loaded library image.  Every GPU that loads the library holds
// that array (MSP_NOALLOC_MAX_N * 24 bytes) until the process exits.
#include <mutex>

#include "msp_internal.cuh"

namespace msp {
void set_last_error(const char* msg);
}

namespace {

constexpr size_t kNaPtsBytes = (size_t)MSP_NOALLOC_MAX_N * sizeof(float4);
constexpr size_t kNaBytes = kNaPtsBytes + (size_t)MSP_NOALLOC_MAX_N * sizeof(float2);

// The scratch: packed positions (float4) followed by the dendrite weights
// (float2) of up to MSP_NOALLOC_MAX_N neurons.  Shared by every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch, looked up once per device and CUDA
// context.  The cache is keyed on the context's unique id (cuCtxGetId, reached
// through the runtime's driver entry points so that the library does not link
// libcuda): after a cudaDeviceReset the device's next context holds the array
// at a new address, and the next call looks it up again.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {};
unsigned long long g_na_ctx[kNaMaxDevices] = {};

typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// id of the calling thread's current context, 0 if none or not available
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

msp_status scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kNaMaxDevices) return MSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_na_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_na_ptr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return MSP_ERR_CUDA;
        g_na_ptr[dev] = p;
        g_na_ctx[dev] = current_context_id();   // the lookup made the context current
    }
    *out = g_na_ptr[dev];
    return MSP_OK;
}

// 1 when p is device (or managed) memory of device `dev`
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // a failed query leaves a (non-sticky) error: clear it
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

__device__ inline float na_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// every entry [0, n) of the scratch is rewritten before it is read, so nothing
// left by an earlier call is ever used
__global__ void k_na_pack(int64_t n, const float* __restrict__ x, const float* __restrict__ y,
                          const float* __restrict__ z, const uint8_t* __restrict__ type,
                          const uint8_t* __restrict__ va, const uint8_t* __restrict__ vde,
                          const uint8_t* __restrict__ vdi, float4* __restrict__ P,
                          float2* __restrict__ Wt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t packed = (uint32_t)(type[i] ? 1u : 0u) | ((uint32_t)va[i] << 8);
        P[i] = make_float4(x[i], y[i], z[i], __uint_as_float(packed));
        Wt[i] = make_float2((float)vde[i], (float)vdi[i]);
    }
}

constexpr int kNaThreads = 256;

// u(t) = sum_{s != t} w_s^{type t} 2^(-|t-s|^2 log2(e)/sigma^2), sources staged
// through shared memory in tiles, in the caller's order; tile sums in single
// precision, added across tiles with Kahan's compensated summation
__global__ void __launch_bounds__(kNaThreads)
k_na_direct(int64_t n, const float4* __restrict__ P, const float2* __restrict__ Wt, float k2,
            float* __restrict__ u) {
    __shared__ float4 sp[kNaThreads];
    __shared__ float2 sw[kNaThreads];
    for (int64_t tb = (int64_t)blockIdx.x * kNaThreads; tb < n; tb += (int64_t)gridDim.x * kNaThreads) {
        const int64_t t = tb + threadIdx.x;
        const bool active = t < n;
        const float4 T = active ? P[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t tw = __float_as_uint(T.w);
        const bool inh = (tw & 0xffu) != 0;
        float acc = 0.f, comp = 0.f;   // Kahan sum of the tile sums
        for (int64_t sb = 0; sb < n; sb += kNaThreads) {
            __syncthreads();
            const int64_t s = sb + threadIdx.x;
            sp[threadIdx.x] = s < n ? P[s] : make_float4(3e30f, 3e30f, 3e30f, 0.f);
            sw[threadIdx.x] = s < n ? Wt[s] : make_float2(0.f, 0.f);
            __syncthreads();
            float part = 0.f;
            for (int j = 0; j < kNaThreads; ++j) {
                const float4 S = sp[j];
                const float dx = T.x - S.x, dy = T.y - S.y, dz = T.z - S.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float wj = sb + j == t ? 0.f : (inh ? sw[j].y : sw[j].x);
                part = fmaf(wj, na_ex2(-r2 * k2), part);
            }
            const float y = __fsub_rn(part, comp);
            const float t2 = __fadd_rn(acc, y);
            comp = __fsub_rn(__fsub_rn(t2, acc), y);
            acc = t2;
        }
        if (active) u[t] = ((tw >> 8) & 0xffu) > 0 ? acc : 0.f;
    }
}

}  // namespace

extern "C" msp_status msp_direct_noalloc(int64_t n, const float* x, const float* y, const float* z,
                                         const uint8_t* type, const uint8_t* vac_axon,
                                         const uint8_t* vac_dend_e, const uint8_t* vac_dend_i,
                                         double sigma, float* u, void* stream) {
    if (n < 0 || n > MSP_NOALLOC_MAX_N) {
        msp::set_last_error("msp_direct_noalloc: n exceeds MSP_NOALLOC_MAX_N (its fixed scratch)");
        return MSP_ERR_INVALID_ARG;
    }
    if (!(sigma > 0.0)) {
        msp::set_last_error("msp_direct_noalloc: sigma must be positive");
        return MSP_ERR_INVALID_ARG;
    }
    if (n == 0) return MSP_OK;
    if (!x || !y || !z || !type || !vac_axon || !vac_dend_e || !vac_dend_i || !u) {
        msp::set_last_error("msp_direct_noalloc: null pointer");
        return MSP_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        msp::set_last_error(cudaGetErrorString(e));
        return MSP_ERR_CUDA;
    }
    void* base = nullptr;
    msp_status st = scratch_address(dev, &base);
    if (st != MSP_OK) {
        msp::set_last_error("msp_direct_noalloc: cannot resolve the scratch array on this device");
        return st;
    }
    const void* ptrs[8] = {x, y, z, type, vac_axon, vac_dend_e, vac_dend_i, u};
    for (const void* p : ptrs)
        if (!on_device(p, dev)) {
            msp::set_last_error("msp_direct_noalloc: every array must be device memory of the "
                                "current device");
            return MSP_ERR_INVALID_ARG;
        }
    float4* P = static_cast<float4*>(base);
    float2* Wt = reinterpret_cast<float2*>(static_cast<unsigned char*>(base) + kNaPtsBytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float k2 = (float)(1.4426950408889634 / (sigma * sigma));
    int g = (int)((n + kNaThreads - 1) / kNaThreads);
    k_na_pack<<<g, kNaThreads, 0, s>>>(n, x, y, z, type, vac_axon, vac_dend_e, vac_dend_i, P, Wt);
    k_na_direct<<<g, kNaThreads, 0, s>>>(n, P, Wt, k2, u);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        msp::set_last_error(cudaGetErrorString(e));
        return MSP_ERR_CUDA;
    }
    msp::g_kernel_launches.fetch_add(2, std::memory_order_relaxed);
    msp::set_last_error("");
    return MSP_OK;
}
