// host_link.cu -- host <-> device transfer paths on GB300 (a Grace CPU on
// the NVLink-C2C link): cudaMemcpyAsync from and to pinned memory against
// kernels that read or write the pinned memory directly (mapped; the same
// pointer under unified addressing), in order (float4) or with a
// permutation on the device side -- the step that takes a caller's vector
// from node order into the format's position order, or back.  Measured with
// CUDA events, best of five.
//
// Not part of the library: it measures what the vector I/O of the library
// chooses between.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 host_link.cu -o host_link
//   ./host_link
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdint>
#include <vector>
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA %s line %d\n", cudaGetErrorString(e_), __LINE__); return 1; } } while (0)

__global__ void k_copy4(const float4 *__restrict__ src, float4 *__restrict__ dst, int64_t n4)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
// dst[perm[j]] = src[j]: sequential reads of src, scattered writes
__global__ void k_scatter_in(const float *__restrict__ src, const int *__restrict__ perm, float *__restrict__ dst, int64_t n)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dst[perm[j]] = src[j];
}
// dst[j] = src[perm[j]]: scattered reads of src, sequential writes
__global__ void k_gather_out(const float *__restrict__ src, const int *__restrict__ perm, float *__restrict__ dst, int64_t n)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = __ldg(src + perm[j]);
}

int main()
{
    const int64_t n = (int64_t)1 << 26;          // 256 MB of floats (R-MAT scale 26 vector)
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    int um = 0, pm = 0;
    CK(cudaDeviceGetAttribute(&um, cudaDevAttrUnifiedAddressing, 0));
    CK(cudaDeviceGetAttribute(&pm, cudaDevAttrCanUseHostPointerForRegisteredMem, 0));
    printf("unified addressing %d, host pointer usable %d\n", um, pm);
    float *h0 = nullptr, *h1 = nullptr, *d0 = nullptr, *d1 = nullptr;
    int *perm = nullptr;
    CK(cudaMallocHost(&h0, n * 4));
    CK(cudaMallocHost(&h1, n * 4));
    CK(cudaMalloc(&d0, n * 4));
    CK(cudaMalloc(&d1, n * 4));
    CK(cudaMalloc(&perm, n * 4));
    std::vector<int> hp((size_t)n);
    for (int64_t i = 0; i < n; ++i) hp[(size_t)i] = (int)i;
    uint64_t st = 7;
    for (int64_t i = n - 1; i > 0; --i) {       // Fisher-Yates with an LCG (Knuth MMIX constants)
        st = st * 6364136223846793005ULL + 1442695040888963407ULL;
        int64_t j = (int64_t)((st >> 33) % (uint64_t)(i + 1));
        int t = hp[(size_t)i]; hp[(size_t)i] = hp[(size_t)j]; hp[(size_t)j] = t;
    }
    CK(cudaMemcpy(perm, hp.data(), n * 4, cudaMemcpyHostToDevice));
    for (int64_t i = 0; i < n; ++i) { h0[i] = (float)i; h1[i] = 0.f; }
    CK(cudaMemset(d0, 0, n * 4));
    float *dh0 = nullptr, *dh1 = nullptr;
    CK(cudaHostGetDevicePointer((void **)&dh0, h0, 0));
    CK(cudaHostGetDevicePointer((void **)&dh1, h1, 0));
    printf("device alias equals host pointer: %d\n", dh0 == h0);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto rep = [&](const char *name, auto fn) -> int {
        float best = 1e30f;
        for (int r = 0; r < 5; ++r) {
            CK(cudaEventRecord(e0));
            fn();
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            float ms;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) best = ms;
        }
        printf("%-34s %.3f ms  %.1f GB/s\n", name, best, n * 4.0 / (best * 1e-3) / 1e9);
        return 0;
    };
    const int g = sms * 8, b = 256;
    if (rep("memcpy H2D pinned", [&] { cudaMemcpyAsync(d0, h0, n * 4, cudaMemcpyHostToDevice); })) return 1;
    if (rep("memcpy D2H pinned", [&] { cudaMemcpyAsync(h1, d0, n * 4, cudaMemcpyDeviceToHost); })) return 1;
    if (rep("kernel read host (float4)", [&] { k_copy4<<<g, b>>>((const float4 *)dh0, (float4 *)d0, n / 4); })) return 1;
    if (rep("kernel write host (float4)", [&] { k_copy4<<<g, b>>>((const float4 *)d0, (float4 *)dh1, n / 4); })) return 1;
    if (rep("kernel read host, scatter to HBM", [&] { k_scatter_in<<<g, b>>>(dh0, perm, d1, n); })) return 1;
    if (rep("kernel gather HBM, write host", [&] { k_gather_out<<<g, b>>>(d1, perm, dh1, n); })) return 1;
    if (rep("HBM gather (device only)", [&] { k_gather_out<<<g, b>>>(d1, perm, d0, n); })) return 1;
    if (rep("HBM scatter (device only)", [&] { k_scatter_in<<<g, b>>>(d0, perm, d1, n); })) return 1;
    // check: h1[j] = d1[perm[j]] = h0[j] after scatter_in + gather_out
    int bad = 0;
    for (int64_t i = 0; i < n; i += 4099) bad += h1[i] != (float)i;
    printf("round trip check: %s\n", bad ? "FAIL" : "ok");
    return bad ? 2 : 0;
}
