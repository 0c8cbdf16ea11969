// sfu_rate.cu -- measures the two rates the near-field roofline rests on:
//   1. EX2 results per SM per clock (ex2.approx.ftz.f32, eight independent
//      chains per thread, 4..16 blocks of 128 threads per SM);
//   2. the near-field evaluation w K = 2^(2 t.s + c_s) summed per target
//      (one shared-memory source, three FMAs, one EX2, one add) with two and
//      with four targets per thread.
// Build and run on the GPU:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o sfu_rate \
//        paper_2301_10570_gb300/probes/sfu_rate.cu && ./sfu_rate
// Rates are per SM per clock at the device's maximum SM clock; the program
// exits non-zero on a CUDA error.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void k_ex2(float* out, int iters) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = ex2a(-a[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// R targets per thread against 64 staged sources (two channel slots each)
template <int R>
__global__ void __launch_bounds__(128, 8) k_eval(float* out, int iters) {
    __shared__ float4 st[128];
    st[threadIdx.x] = make_float4(threadIdx.x * 1e-3f, 0.2f, -0.1f, -3.f);
    __syncthreads();
    float tx[R], ty[R], tz[R], p[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        tx[r] = threadIdx.x * 1e-4f + 0.05f * r;
        ty[r] = 0.1f - 0.07f * r;
        tz[r] = 0.2f + 0.03f * r;
        p[r][0] = p[r][1] = 0.f;
    }
    for (int i = 0; i < iters; ++i) {
        const float4* q = st + (threadIdx.x & 1);
        for (int e = 0; e < 64; e += 4, q += 8) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 A = q[2 * v];
#pragma unroll
                for (int r = 0; r < R; ++r)
                    p[r][v & 1] += ex2a(fmaf(tx[r], A.x, fmaf(ty[r], A.y, fmaf(tz[r], A.z, A.w))));
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) s += p[r][0] + p[r][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static int check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        printf("%s: %s\n", what, cudaGetErrorString(e));
        return 1;
    }
    return 0;
}

template <class L>
static double time_ms(L launch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();
    cudaDeviceSynchronize();
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

int main() {
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);      // kHz
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * sms * 16 * 128) != cudaSuccess) return check("cudaMalloc") | 1;
    const double hz = clk * 1e3;
    printf("SMs %d, maximum SM clock %d MHz\n", sms, clk / 1000);
    for (int bps : {4, 8, 16}) {
        const int grid = sms * bps, iters = 4096;
        const double ms = time_ms([&] { k_ex2<<<grid, 128>>>(out, iters); });
        const double n = (double)grid * 128 * iters * 8;
        printf("ex2            %2d blocks/SM: %8.1f G/s  %6.2f per SM per clock\n", bps,
               n / ms / 1e6, n / (ms * 1e-3) / hz / sms);
    }
    if (check("ex2")) return 1;
    {
        const int grid = sms * 8, iters = 200;
        double ms = time_ms([&] { k_eval<2><<<grid, 128>>>(out, iters); });
        double n = (double)grid * 128 * iters * 64 * 2;
        printf("evaluation R=2 8 blocks/SM: %8.1f G/s  %6.2f per SM per clock\n", n / ms / 1e6,
               n / (ms * 1e-3) / hz / sms);
        ms = time_ms([&] { k_eval<4><<<grid, 128>>>(out, iters); });
        n = (double)grid * 128 * iters * 64 * 4;
        printf("evaluation R=4 8 blocks/SM: %8.1f G/s  %6.2f per SM per clock\n", n / ms / 1e6,
               n / (ms * 1e-3) / hz / sms);
    }
    if (check("evaluation")) return 1;
    cudaFree(out);
    return 0;
}
