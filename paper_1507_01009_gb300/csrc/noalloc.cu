// noalloc.cu -- a perturber search that allocates nothing.
//
// Some callers cannot call cudaMalloc: a chain integrator that looks for
// perturbers from inside its own step (for example from a host callback, or
// from code that runs while another library owns the allocator), or a host
// application that forbids device allocation after start-up. For them
// rv_select_radius_static finds the stars inside a sphere without a context
// or workspace: its only scratch -- one count per block of 2048 stars plus a
// total -- lives in the file-scope device array below, which every GPU that
// loads librv holds until the process exits.
//
// The host obtains the array's device address once per device with
// cudaGetSymbolAddress (the array's name in host code is only a host-side
// stand-in, not a device address) and passes that address to the kernels.
#include <mutex>

#include "rv_internal.cuh"

namespace rv {

constexpr int kStaticSelChunk = 2048;                      // stars per block
constexpr int kStaticSelMaxBlocks = 8192;                  // 32 KiB of counts
constexpr int64_t kStaticSelMaxN = (int64_t)kStaticSelChunk * kStaticSelMaxBlocks;  // 16,777,216 stars

// Per-block counts, scanned in place, then the total at [kStaticSelMaxBlocks].
// Every call overwrites the entries it uses before reading them.
static __device__ __align__(256) int g_sel_scratch[kStaticSelMaxBlocks + 1];

constexpr int kMaxDevices = 64;
static int *g_sel_addr[kMaxDevices];
static std::mutex g_sel_mutex;

__device__ __forceinline__ bool inside(const float *x, const float *y, const float *z, int64_t i, float3 c, float r2) {
    float dx = __fsub_rn(x[i], c.x), dy = __fsub_rn(y[i], c.y), dz = __fsub_rn(z[i], c.z);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return d2 < r2;
}

__device__ int block_exclusive_scan_256(int v, int *sw, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < 8) ? sw[lane] : 0;
        for (int o = 1; o < 8; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < 8) sw[lane] = w;
    }
    __syncthreads();
    int base = (wid > 0) ? sw[wid - 1] : 0;
    total = sw[7];
    __syncthreads();
    return base + x - v;
}

// Pass 1: stars inside the sphere per block of 2048 (thread t: stars 8t..8t+7).
__global__ void __launch_bounds__(256) static_sel_count_k(int64_t n, const float *x, const float *y, const float *z,
                                                           float3 c, float r2, int *scratch) {
    __shared__ int sw[8];
    int64_t base = (int64_t)blockIdx.x * kStaticSelChunk + threadIdx.x * 8;
    int cnt = 0;
    for (int k = 0; k < 8; k++) {
        int64_t i = base + k;
        if (i < n && inside(x, y, z, i, c, r2)) cnt++;
    }
    int total;
    block_exclusive_scan_256(cnt, sw, total);
    if (threadIdx.x == 0) scratch[blockIdx.x] = total;
}

// Pass 2: exclusive scan of the block counts; the total goes to scratch and to
// *count (untruncated: a total above cap tells the caller that only the first
// cap indices were written).
__global__ void __launch_bounds__(1024) static_sel_scan_k(int nb, int *scratch, int *count) {
    __shared__ int sw[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int b = b0 + threadIdx.x;
        int v = (b < nb) ? scratch[b] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sw[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = sw[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            sw[lane] = w;
        }
        __syncthreads();
        int ex = ((wid > 0) ? sw[wid - 1] : 0) + x - v;
        int tot = sw[31];
        __syncthreads();
        if (b < nb) scratch[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        scratch[kStaticSelMaxBlocks] = carry;
        *count = carry;
    }
}

// Pass 3: write the indices in ascending order, the first `cap` only.
__global__ void __launch_bounds__(256) static_sel_write_k(int64_t n, const float *x, const float *y, const float *z,
                                                           float3 c, float r2, int cap, const int *scratch,
                                                           int *idx) {
    __shared__ int sw[8];
    int64_t base = (int64_t)blockIdx.x * kStaticSelChunk + threadIdx.x * 8;
    unsigned flags = 0;
    int cnt = 0;
    for (int k = 0; k < 8; k++) {
        int64_t i = base + k;
        if (i < n && inside(x, y, z, i, c, r2)) { flags |= 1u << k; cnt++; }
    }
    int total;
    int pos = block_exclusive_scan_256(cnt, sw, total) + scratch[blockIdx.x];
    for (int k = 0; k < 8; k++)
        if (flags & (1u << k)) {
            if (pos < cap) idx[pos] = (int)(base + k);
            pos++;
        }
}

// Device address of g_sel_scratch on the current device; looked up on the
// first call on each device and cached.
static rv_status scratch_address(int **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RV_E_CUDA;
    std::lock_guard<std::mutex> lock(g_sel_mutex);
    if (!g_sel_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sel_scratch) != cudaSuccess || !p) return RV_E_CUDA;
        g_sel_addr[dev] = (int *)p;
    }
    *out = g_sel_addr[dev];
    return RV_OK;
}

}  // namespace rv

using namespace rv;

extern "C" rv_status rv_select_radius_static(int64_t n, const float *x, const float *y, const float *z,
                                             const float centre[3], float radius, int32_t cap, int32_t *idx,
                                             int32_t *count, void *stream) {
    if (n < 0 || !centre || !count || cap < 0 || !(radius >= 0.f)) return RV_E_INVAL;
    if (n > kStaticSelMaxN) return RV_E_TOO_LARGE;
    if (n > 0 && (!x || !y || !z)) return RV_E_INVAL;
    if (cap > 0 && !idx) return RV_E_INVAL;
    int *scratch = nullptr;
    rv_status st = scratch_address(&scratch);
    if (st != RV_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float3 c = make_float3(centre[0], centre[1], centre[2]);
    float r2 = radius * radius;  // one FP32 product
    int nb = (int)((n + kStaticSelChunk - 1) / kStaticSelChunk);
    // each launch's own status (cudaLaunchKernel returns it), so that an error
    // left by unrelated earlier work is neither reported nor cleared here
    cudaError_t e = cudaSuccess;
    if (nb > 0) {
        void *a[] = {&n, &x, &y, &z, &c, &r2, &scratch};
        e = cudaLaunchKernel((const void *)static_sel_count_k, dim3(nb), dim3(256), a, 0, s);
    }
    if (e == cudaSuccess) {
        void *a[] = {&nb, &scratch, &count};
        e = cudaLaunchKernel((const void *)static_sel_scan_k, dim3(1), dim3(1024), a, 0, s);
    }
    if (e == cudaSuccess && nb > 0) {
        void *a[] = {&n, &x, &y, &z, &c, &r2, &cap, &scratch, &idx};
        e = cudaLaunchKernel((const void *)static_sel_write_k, dim3(nb), dim3(256), a, 0, s);
    }
    return e == cudaSuccess ? RV_OK : RV_E_CUDA;
}
