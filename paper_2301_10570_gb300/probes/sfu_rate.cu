// sfu_rate.cu -- measures the two rates the near-field roofline rests on:
//   1. EX2 results per SM per clock (ex2.approx.ftz.f32, eight independent
//      chains per thread, 4..16 blocks of 128 threads per SM);
//   2. the near-field evaluation w K = 2^(2 t.s + c_s) summed per target
//      (one shared-memory source, three FMAs, one EX2, one add) with two and
//      with four targets per thread, in three register layouts: scalar FMAs;
//      packed pairs of targets (the source broadcast into both halves); packed
//      pairs of sources (staged as (x0,x1,y0,y1), (z0,z1,c0,c1), the target
//      broadcast once outside the loop).
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

// R targets per thread, packed in pairs; each source broadcast into both halves
template <int R>
__global__ void __launch_bounds__(128, 8) k_eval_tp(float* out, int iters) {
    __shared__ float4 st[128];
    st[threadIdx.x] = make_float4(threadIdx.x * 1e-3f, 0.2f, -0.1f, -3.f);
    __syncthreads();
    constexpr int H = R / 2;
    float2 tx[H], ty[H], tz[H], p[H][2];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        tx[h] = make_float2(threadIdx.x * 1e-4f + 0.1f * h, threadIdx.x * 1e-4f + 0.1f * h + 0.05f);
        ty[h] = make_float2(0.1f - 0.14f * h, 0.03f - 0.14f * h);
        tz[h] = make_float2(0.2f + 0.06f * h, 0.23f + 0.06f * h);
        p[h][0] = p[h][1] = make_float2(0.f, 0.f);
    }
    for (int i = 0; i < iters; ++i) {
        const float4* q = st + (threadIdx.x & 1);
        for (int e = 0; e < 64; e += 4, q += 8) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 A = q[2 * v];
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const float2 E = __ffma2_rn(
                        tx[h], make_float2(A.x, A.x),
                        __ffma2_rn(ty[h], make_float2(A.y, A.y),
                                   __ffma2_rn(tz[h], make_float2(A.z, A.z), make_float2(A.w, A.w))));
                    p[h][v & 1] = __fadd2_rn(p[h][v & 1], make_float2(ex2a(E.x), ex2a(E.y)));
                }
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int h = 0; h < H; ++h) s += p[h][0].x + p[h][0].y + p[h][1].x + p[h][1].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// R targets per thread, sources packed in pairs: 64 sources staged as 32
// (x0,x1,y0,y1) and 2 x 32 (z0,z1,c0,c1) (one per channel slot)
template <int R>
__global__ void __launch_bounds__(128, 8) k_eval_sp(float* out, int iters) {
    __shared__ float4 sxy[32], szc[2][32];
    if (threadIdx.x < 32) {
        const float f = threadIdx.x * 2e-3f;
        sxy[threadIdx.x] = make_float4(f, f + 1e-3f, 0.2f, 0.21f);
        szc[0][threadIdx.x] = make_float4(-0.1f, -0.11f, -3.f, -3.1f);
        szc[1][threadIdx.x] = make_float4(-0.1f, -0.11f, -3.2f, -3.3f);
    }
    __syncthreads();
    float2 tx[R], ty[R], tz[R], p[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float a = threadIdx.x * 1e-4f + 0.05f * r, b = 0.1f - 0.07f * r, c = 0.2f + 0.03f * r;
        tx[r] = make_float2(a, a);
        ty[r] = make_float2(b, b);
        tz[r] = make_float2(c, c);
        p[r][0] = p[r][1] = make_float2(0.f, 0.f);
    }
    const float4* zc = szc[threadIdx.x & 1];
    for (int i = 0; i < iters; ++i) {
        for (int e = 0; e < 32; e += 2) {
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const float4 XY = sxy[e + v], ZC = zc[e + v];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 E = __ffma2_rn(
                        tx[r], make_float2(XY.x, XY.y),
                        __ffma2_rn(ty[r], make_float2(XY.z, XY.w),
                                   __ffma2_rn(tz[r], make_float2(ZC.x, ZC.y), make_float2(ZC.z, ZC.w))));
                    p[r][v] = __fadd2_rn(p[r][v], make_float2(ex2a(E.x), ex2a(E.y)));
                }
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) s += p[r][0].x + p[r][0].y + p[r][1].x + p[r][1].y;
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
    {
        const int grid = sms * 8, iters = 200;
        double ms = time_ms([&] { k_eval_tp<2><<<grid, 128>>>(out, iters); });
        double n = (double)grid * 128 * iters * 64 * 2;
        printf("target-packed R=2 8 blocks/SM: %8.1f G/s  %6.2f per SM per clock\n", n / ms / 1e6,
               n / (ms * 1e-3) / hz / sms);
        ms = time_ms([&] { k_eval_tp<4><<<grid, 128>>>(out, iters); });
        n = (double)grid * 128 * iters * 64 * 4;
        printf("target-packed R=4 8 blocks/SM: %8.1f G/s  %6.2f per SM per clock\n", n / ms / 1e6,
               n / (ms * 1e-3) / hz / sms);
        ms = time_ms([&] { k_eval_sp<2><<<grid, 128>>>(out, iters); });
        n = (double)grid * 128 * iters * 64 * 2;
        printf("source-packed R=2 8 blocks/SM: %8.1f G/s  %6.2f per SM per clock\n", n / ms / 1e6,
               n / (ms * 1e-3) / hz / sms);
        ms = time_ms([&] { k_eval_sp<4><<<grid, 128>>>(out, iters); });
        n = (double)grid * 128 * iters * 64 * 4;
        printf("source-packed R=4 8 blocks/SM: %8.1f G/s  %6.2f per SM per clock\n", n / ms / 1e6,
               n / (ms * 1e-3) / hz / sms);
    }
    if (check("packed evaluation")) return 1;
    cudaFree(out);
    return 0;
}
