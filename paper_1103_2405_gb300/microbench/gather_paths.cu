// gather_paths.cu -- throughput of the ways an sm_103a kernel can fetch
// scattered 4-byte x values (the SpMV gather), measured with CUDA events:
//
//   lsu      global loads through L1/L2 (ld.global.nc), array L2-resident
//            or not: every distinct 128-byte line costs an L1 tag lookup;
//   lsu U    the same with U independent loads in flight per thread, to
//            tell a throughput ceiling from too few loads in flight;
//   tex U    1D texture fetches (tex1Dfetch over a linear buffer, the
//            paper's texture-cache path), U in flight per thread, and an
//            even mix of texture and global loads;
//   rows256  a warp-wide coalesced 256-byte row per load (the SpMM gather);
//   smem     loads from the block's own shared memory (96 KB slice);
//   dsmem    loads from a thread-block cluster's distributed shared memory
//            (the slice spread over 2-16 blocks, ld.shared::cluster);
//   gather4  TMA tile::gather4 copies of 32-byte rows into a shared-memory
//            ring (one producer warp, mbarrier completion, bounded waits).
//
// Not part of the library: it measures the hardware paths the SpMV kernel
// design chooses between (shared-memory x slice for the densest columns,
// L1/L2 for the rest).  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 gather_paths.cu -o gather_paths
//   ./gather_paths
#include <cuda.h>
#include <cuda_runtime.h>
#include <cooperative_groups.h>

#include <cstdint>
#include <cstdio>
#include <vector>

namespace cg = cooperative_groups;

#define CK(x)                                                                              \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            std::printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__); \
            return 1;                                                                      \
        }                                                                                  \
    } while (0)

constexpr int kSliceCols = 24576;   // 96 KB of floats per block

// ---------------------------------------------------------------- LSU --
__global__ void k_lsu(const float *__restrict__ x, const int *__restrict__ idx, int64_t m,
                      int span, float *out)
{
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride)
        acc += __ldg(x + (__ldg(idx + i) % span));
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// U loads in flight per thread: thread t takes the U consecutive indices
// of chunk t, t + T, ... (T threads; m a multiple of U).  PATH 0: global
// loads, 1: texture fetches, 2: even u global, odd u texture.
template <int U, int PATH>
__global__ void k_gather_u(const float *__restrict__ x, cudaTextureObject_t tex, const int *__restrict__ idx,
                           int64_t m, int span, float *out)
{
    float acc = 0.f;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * U; i0 + U <= m; i0 += nt * U) {
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = __ldg(idx + i0 + u) % span;
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            v[u] = (PATH == 0 || (PATH == 2 && (u & 1) == 0)) ? __ldg(x + c[u]) : tex1Dfetch<float>(tex, c[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u];
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// rows of 64 floats (the SpMM's X-row gather): each warp loads one random
// 256-byte row per step (float2 per lane), U rows in flight per warp
template <int U>
__global__ void k_lsu_rows(const float *__restrict__ x, const int *__restrict__ idx, int64_t m,
                           int rows, float *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t i0 = warp * U; i0 + U <= m; i0 += nwarps * U) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = __ldg(idx + i0 + u) % rows;
            v[u] = __ldg(reinterpret_cast<const float2 *>(x + (int64_t)r * 64) + lane);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) { acc.x += v[u].x; acc.y += v[u].y; }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc.x + acc.y;
}

// ------------------------------------------------ shared / distributed --
// MODE 0: own shared memory; 1: the cluster's distributed shared memory
template <int MODE>
__global__ void __launch_bounds__(1024, 1)
k_shared(const float *__restrict__ x, const int *__restrict__ idx, int64_t m, float *out)
{
    extern __shared__ float xs[];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned me = cl.block_rank(), csz = cl.num_blocks();
    for (int i = threadIdx.x; i < kSliceCols; i += blockDim.x) xs[i] = x[me * kSliceCols + i];
    cl.sync();
    const int span = (int)csz * kSliceCols;
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
        const int c = __ldg(idx + i) % span;
        if (MODE == 0) {
            acc += xs[c % kSliceCols];
        } else {
            const unsigned r = (unsigned)c / kSliceCols;
            acc += *cl.map_shared_rank(xs + (c - (int)r * kSliceCols), r);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    cl.sync();   // no block leaves while a peer may still read its slice
}

// ------------------------------------------------------------ gather4 --
constexpr int kStages = 8;
constexpr int kBatch = 256;               // 32-byte rows per stage (64 gather4)
constexpr int kStageBytes = kBatch * 32;
constexpr int kConsumerWarps = 8;
constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool wait_parity(uint64_t *bar, uint32_t phase, unsigned *err)
{
    for (uint32_t k = 0; k < kWaitLimit; ++k) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(saddr(bar)), "r"(phase) : "memory");
        if (ok) return true;
    }
    atomicOr(err, 1u);
    return false;
}

__device__ __forceinline__ void gather4(uint32_t dst, const CUtensorMap *tm, int4 r, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                 :: "r"(dst), "l"(tm), "r"(0), "r"(r.x), "r"(r.y), "r"(r.z), "r"(r.w), "r"(saddr(bar))
                 : "memory");
}

// warp 0 produces (every lane loads two index quadruples two stages ahead
// and issues two gather4), warps 1..8 consume one row each per stage
__global__ void __launch_bounds__(32 * (1 + kConsumerWarps), 1)
k_gather4(const __grid_constant__ CUtensorMap tm, const int *__restrict__ idx, int64_t m, float *out,
          unsigned *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + kStages;
    float *ring = reinterpret_cast<float *>(smem + 1024);
    const int64_t batches = m / kBatch;
    const int64_t per = (batches + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = blockIdx.x * per;
    const int64_t b1 = b0 + per < batches ? b0 + per : batches;
    const int nb = (int)(b1 > b0 ? b1 - b0 : 0);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(full + s)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(empty + s)), "r"(kConsumerWarps));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        const int4 z = make_int4(0, 0, 0, 0);
        int4 a0 = z, c0 = z, a1 = z, c1 = z;
        auto load = [&](int j, int4 &a, int4 &c) {
            const int4 *ip = reinterpret_cast<const int4 *>(idx + (b0 + j) * kBatch);
            a = __ldg(ip + lane);
            c = __ldg(ip + lane + 32);
        };
        if (nb > 0) load(0, a0, c0);
        if (nb > 1) load(1, a1, c1);
        for (int j = 0; j < nb; ++j) {
            const int s = j % kStages;
            int ok = 1;
            if (j >= kStages && lane == 0) ok = wait_parity(empty + s, ((j / kStages) - 1) & 1, err);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            const int4 ra = a0, rc = c0;
            a0 = a1;
            c0 = c1;
            if (j + 2 < nb) load(j + 2, a1, c1);
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(saddr(full + s)), "r"(kStageBytes) : "memory");
            __syncwarp();
            gather4(saddr(ring) + s * kStageBytes + lane * 128, &tm, ra, full + s);
            gather4(saddr(ring) + s * kStageBytes + (lane + 32) * 128, &tm, rc, full + s);
        }
    } else {
        const int t = threadIdx.x - 32;
        float acc = 0.f;
        for (int j = 0; j < nb; ++j) {
            const int s = j % kStages;
            if (!wait_parity(full + s, (j / kStages) & 1, err)) break;
            acc += ring[s * (kStageBytes / 4) + t * 8 + (t & 7)];
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(empty + s)) : "memory");
        }
        out[blockIdx.x * 32 * kConsumerWarps + t] = acc;
    }
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);

static float time_ms(cudaEvent_t e0, cudaEvent_t e1)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

int main()
{
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const int64_t m = (int64_t)1 << 26;
    const int64_t nx = (int64_t)1 << 27;     // 512 MB of floats
    std::vector<int> h((size_t)m);
    uint64_t st = 12345;
    for (int64_t i = 0; i < m; ++i) {         // LCG (Knuth's MMIX constants), top 31 bits
        st = st * 6364136223846793005ULL + 1442695040888963407ULL;
        h[(size_t)i] = (int)(st >> 33);
    }
    float *x = nullptr, *out = nullptr;
    int *idx = nullptr;
    unsigned *err = nullptr;
    const size_t out_len = (size_t)8 * sms * 1024;
    CK(cudaMalloc(&x, nx * sizeof(float)));
    CK(cudaMalloc(&idx, m * sizeof(int)));
    CK(cudaMalloc(&out, out_len * sizeof(float)));
    CK(cudaMalloc(&err, sizeof(unsigned)));
    CK(cudaMemset(x, 0, nx * sizeof(float)));
    CK(cudaMemset(err, 0, sizeof(unsigned)));
    CK(cudaMemcpy(idx, h.data(), m * sizeof(int), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));

    // global loads over spans from L2-resident (16 MB) to DRAM-sized (512 MB)
    for (int span : {1 << 22, 1 << 24, 1 << 27}) {
        float ms = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(e0));
            k_lsu<<<sms * 8, 256>>>(x, idx, m, span, out);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            ms = time_ms(e0, e1);
        }
        std::printf("lsu     span %9d floats: %.3e loads/s\n", span, m / (ms * 1e-3));
    }
    // loads in flight per thread, global and texture paths
    int tex_max = 0;
    CK(cudaDeviceGetAttribute(&tex_max, cudaDevAttrMaxTexture1DLinearWidth, 0));
    for (int span : {1 << 22, 1 << 24, 1 << 27}) {
        cudaTextureObject_t tex = 0;
        const bool have_tex = span <= tex_max;
        if (have_tex) {
            cudaResourceDesc rd = {};
            rd.resType = cudaResourceTypeLinear;
            rd.res.linear.devPtr = x;
            rd.res.linear.desc = cudaCreateChannelDesc<float>();
            rd.res.linear.sizeInBytes = (size_t)span * sizeof(float);
            cudaTextureDesc td = {};
            td.readMode = cudaReadModeElementType;
            CK(cudaCreateTextureObject(&tex, &rd, &td, nullptr));
        }
        for (int path = 0; path < (have_tex ? 3 : 1); ++path) {
            for (int u : {1, 4, 8}) {
                float ms = 0.f;
                for (int rep = 0; rep < 3; ++rep) {
                    CK(cudaEventRecord(e0));
                    const dim3 g(sms * 8), b(256);
                    if (path == 0 && u == 1) k_gather_u<1, 0><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 0 && u == 4) k_gather_u<4, 0><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 0 && u == 8) k_gather_u<8, 0><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 1 && u == 1) k_gather_u<1, 1><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 1 && u == 4) k_gather_u<4, 1><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 1 && u == 8) k_gather_u<8, 1><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 2 && u == 1) k_gather_u<2, 2><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 2 && u == 4) k_gather_u<4, 2><<<g, b>>>(x, tex, idx, m, span, out);
                    if (path == 2 && u == 8) k_gather_u<8, 2><<<g, b>>>(x, tex, idx, m, span, out);
                    CK(cudaEventRecord(e1));
                    CK(cudaEventSynchronize(e1));
                    CK(cudaGetLastError());
                    ms = time_ms(e0, e1);
                }
                static const char *name[3] = {"lsu", "tex", "lsu+tex"};
                std::printf("%-7s span %9d floats, %d in flight per thread: %.3e loads/s\n", name[path], span,
                            path == 2 && u == 1 ? 2 : u, m / (ms * 1e-3));
            }
        }
        if (have_tex) CK(cudaDestroyTextureObject(tex));
    }
    // 256-byte rows (an n x 64 FP32 block): 2^18 rows (64 MB, fits L2) and
    // 2^21 rows (512 MB), 8 or 16 rows in flight per warp
    for (int rows : {1 << 18, 1 << 21}) {
        for (int u : {8, 16}) {
            float ms = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                CK(cudaEventRecord(e0));
                if (u == 8) k_lsu_rows<8><<<sms * 8, 256>>>(x, idx, m, rows, out);
                else k_lsu_rows<16><<<sms * 8, 256>>>(x, idx, m, rows, out);
                CK(cudaEventRecord(e1));
                CK(cudaEventSynchronize(e1));
                CK(cudaGetLastError());
                ms = time_ms(e0, e1);
            }
            std::printf("rows256 %9d rows, %2d in flight per warp: %.3e rows/s = %.2f TB/s\n", rows, u,
                        m / (ms * 1e-3), m * 256.0 / (ms * 1e-3) / 1e12);
        }
    }
    // own and distributed shared memory, one 1024-thread block per SM
    for (int csz : {1, 2, 4, 8, 16}) {
        for (int mode = 0; mode < (csz > 1 ? 2 : 1); ++mode) {
            auto kern = mode == 0 ? k_shared<0> : k_shared<1>;
            CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSliceCols * 4));
            if (csz > 8) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = csz;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = kSliceCols * 4;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cfg.gridDim = dim3(csz);
            int nclu = 0;
            CK(cudaOccupancyMaxActiveClusters(&nclu, kern, &cfg));
            if ((size_t)nclu * csz * 1024 > out_len) nclu = (int)(out_len / 1024 / csz);
            cfg.gridDim = dim3(nclu * csz);
            float ms = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                CK(cudaEventRecord(e0));
                CK(cudaLaunchKernelEx(&cfg, kern, (const float *)x, (const int *)idx, m, out));
                CK(cudaEventRecord(e1));
                CK(cudaEventSynchronize(e1));
                CK(cudaGetLastError());
                ms = time_ms(e0, e1);
            }
            std::printf("%s cluster %2d (%3d blocks): %.3e loads/s\n", mode == 0 ? "smem   " : "dsmem  ", csz,
                        nclu * csz, m / (ms * 1e-3));
        }
    }
    // TMA gather4 of 32-byte rows (x as a [rows, 8] FP32 tensor)
    EncodeTiled enc = nullptr;
    cudaDriverEntryPointQueryResult q;
    CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&enc, 12000, cudaEnableDefault, &q));
    if (!enc || q != cudaDriverEntryPointSuccess) {
        std::printf("gather4: no tensor-map encoder\n");
        return 1;
    }
    std::vector<int> rowidx((size_t)m);
    for (int64_t rows : {(int64_t)1 << 19, (int64_t)1 << 24}) {
        for (int64_t i = 0; i < m; ++i) rowidx[(size_t)i] = (int)((uint32_t)h[(size_t)i] % (uint64_t)rows);
        CK(cudaMemcpy(idx, rowidx.data(), m * sizeof(int), cudaMemcpyHostToDevice));
        CUtensorMap tm;
        cuuint64_t dims[2] = {8, (cuuint64_t)rows};
        cuuint64_t strides[1] = {32};
        cuuint32_t box[2] = {8, 1};
        cuuint32_t es[2] = {1, 1};
        if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, x, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            std::printf("gather4: tensor map refused\n");
            return 1;
        }
        const int smem = 1024 + kStages * kStageBytes;
        CK(cudaFuncSetAttribute(k_gather4, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        float ms = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(e0));
            k_gather4<<<sms, 32 * (1 + kConsumerWarps), smem>>>(tm, idx, m, out, err);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            ms = time_ms(e0, e1);
            unsigned he = 0;
            CK(cudaMemcpy(&he, err, sizeof he, cudaMemcpyDeviceToHost));
            if (he) {
                std::printf("gather4: a bounded wait ran out\n");
                return 2;
            }
        }
        std::printf("gather4 %9lld rows of 32 B: %.3e rows/s\n", (long long)rows, m / (ms * 1e-3));
    }
    return 0;
}
