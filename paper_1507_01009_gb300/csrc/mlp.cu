// mlp.cu -- learned correction of cell forces (not in the paper).
//
// A small network (11 features -> 64 -> 64 -> 3, SiLU, bfloat16 weights and
// activations, FP32 accumulation on the tensor cores)
// predicts, for a star (or a walk group's centre) at r from an accepted
// cell, the difference between the cell's exact softened force and its
// monopole + quadrupole force, scaled by |r|^2 / M. Features: r/|r| (3),
// s/|r|, eps/|r|, Q/(M s^2) (6), s the cell side.
//
// Inference (rv_mlp_forward and the correction in the walk) runs on tcgen05:
// operands in shared memory, accumulators in tensor memory, 128 rows per tile.
// Training (per minibatch): warp-level mma.sync forward, FP32 backward (exact
// gradients of the same rounded forward), per-block gradient partials summed
// in a fixed order, Adam on FP32 master weights, bfloat16 copies refreshed.
// Samples: random stars, a random cell among those each star's walk accepts
// at a given angle (reservoir choice), features and exact residual target.
// Inference in the tree force: the walk records the (group, cell) pairs
// accepted at theta that a walk at theta_rec < theta would open; the network
// evaluates each pair at the group's centre and the correction is added to
// every star of the group.
#include <cuda_bf16.h>

#include <algorithm>
#include <string.h>

#include "rv_internal.cuh"

namespace rv {

constexpr int kIn = 14, kInPad = 16, kHid = 64, kOut = 3, kOutPad = 8;
// FP32 parameter vector (master weights, Adam moments and gradients share it):
constexpr int oW1 = 0;                  // W1[k][n], 16 x 64 (rows 11..15 zero)
constexpr int ob1 = oW1 + kInPad * kHid;
constexpr int oW2 = ob1 + kHid;         // W2[k][n], 64 x 64
constexpr int ob2 = oW2 + kHid * kHid;
constexpr int oW3 = ob2 + kHid;         // W3[k][n], 64 x 8 (columns 3..7 zero)
constexpr int ob3 = oW3 + kHid * kOutPad;
constexpr int kParams = ob3 + kOutPad;  // 5768
// bfloat16 copies, n-major (B operand of mma: element (k, n) at [n][k])
constexpr int oW1t = 0;                 // [64][16]
constexpr int oW2t = oW1t + kHid * kInPad;   // [64][64]
constexpr int oW3t = oW2t + kHid * kHid;     // [8][64]
constexpr int kBf16 = oW3t + kOutPad * kHid;  // 5632
// then the feature box: lo[16], hi[16] (FP32)
constexpr size_t kBlockBytes = sizeof(float) * 3 * kParams + sizeof(__nv_bfloat16) * kBf16 + sizeof(float) * 2 * kInPad;

struct MlpBlock {
    float *w, *m, *v;      // master weights, Adam moments
    __nv_bfloat16 *wb;     // bfloat16 copies
    float *box;            // features the network was trained on: lo[16], hi[16]
};

__host__ __device__ inline MlpBlock mlp_block(void *p) {
    MlpBlock b;
    b.w = reinterpret_cast<float *>(p);
    b.m = b.w + kParams;
    b.v = b.m + kParams;
    b.wb = reinterpret_cast<__nv_bfloat16 *>(b.v + kParams);
    b.box = reinterpret_cast<float *>(b.wb + kBf16);
    return b;
}

// ---------------------------------------------------------------------------
// counter-based random numbers: SplitMix64 (Steele, Lea & Flood 2014)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    float s = 1.f / (1.f + expf(-z));
    return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weights and biases staged in shared memory by a block.
struct MlpSmem {
    __nv_bfloat16 wb[kBf16];
    float b1[kHid], b2[kHid], b3[kOutPad];
};

__device__ void load_mlp_smem(const MlpBlock &P, MlpSmem &S) {
    for (int i = threadIdx.x; i < kBf16; i += blockDim.x) S.wb[i] = P.wb[i];
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        S.b1[i] = P.w[ob1 + i];
        S.b2[i] = P.w[ob2 + i];
    }
    if (threadIdx.x < kOutPad) S.b3[threadIdx.x] = P.w[ob3 + threadIdx.x];
}

__device__ __forceinline__ unsigned ldb(const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned *>(p); }

// Forward pass of one warp over 16 rows. Input fragment a (rows g, g+8 of the
// warp's 16, columns 2t.. / 2t+8..) in bfloat16; outputs y[4] (rows g, g+8,
// columns 2t, 2t+1). If z1/z2 are given, the pre-activations are kept
// ([8][4] fragments: tile j holds columns 8j + 2t, +1).
__device__ __forceinline__ void mlp_warp_forward(const MlpSmem &S, const unsigned a[4], float y[4],
                                                 float (*z1)[4], float (*z2)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float h[8][4];
    // layer 1: 16 -> 64
#pragma unroll
    for (int j = 0; j < 8; j++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const __nv_bfloat16 *bn = S.wb + oW1t + (8 * j + g) * kInPad;
        mma_bf16(c, a, ldb(bn + 2 * t), ldb(bn + 2 * t + 8));
        const float bb0 = S.b1[8 * j + 2 * t], bb1 = S.b1[8 * j + 2 * t + 1];
        c[0] += bb0; c[1] += bb1; c[2] += bb0; c[3] += bb1;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (z1) z1[j][q] = c[q];
            h[j][q] = silu(c[q]);
        }
    }
    unsigned A2[4][4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        A2[k][0] = pack_bf16(h[2 * k][0], h[2 * k][1]);
        A2[k][1] = pack_bf16(h[2 * k][2], h[2 * k][3]);
        A2[k][2] = pack_bf16(h[2 * k + 1][0], h[2 * k + 1][1]);
        A2[k][3] = pack_bf16(h[2 * k + 1][2], h[2 * k + 1][3]);
    }
    // layer 2: 64 -> 64
#pragma unroll
    for (int j = 0; j < 8; j++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const __nv_bfloat16 *bn = S.wb + oW2t + (8 * j + g) * kHid;
#pragma unroll
        for (int k = 0; k < 4; k++) mma_bf16(c, A2[k], ldb(bn + 16 * k + 2 * t), ldb(bn + 16 * k + 8 + 2 * t));
        const float bb0 = S.b2[8 * j + 2 * t], bb1 = S.b2[8 * j + 2 * t + 1];
        c[0] += bb0; c[1] += bb1; c[2] += bb0; c[3] += bb1;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (z2) z2[j][q] = c[q];
            h[j][q] = silu(c[q]);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        A2[k][0] = pack_bf16(h[2 * k][0], h[2 * k][1]);
        A2[k][1] = pack_bf16(h[2 * k][2], h[2 * k][3]);
        A2[k][2] = pack_bf16(h[2 * k + 1][0], h[2 * k + 1][1]);
        A2[k][3] = pack_bf16(h[2 * k + 1][2], h[2 * k + 1][3]);
    }
    // layer 3: 64 -> 8 (3 used)
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16 *bn = S.wb + oW3t + g * kHid;
#pragma unroll
    for (int k = 0; k < 4; k++) mma_bf16(c, A2[k], ldb(bn + 16 * k + 2 * t), ldb(bn + 16 * k + 8 + 2 * t));
    y[0] = c[0] + S.b3[2 * t];
    y[1] = c[1] + S.b3[2 * t + 1];
    y[2] = c[2] + S.b3[2 * t];
    y[3] = c[3] + S.b3[2 * t + 1];
}

// A fragment of 16 rows of FP32 features x[row][16] (rows >= n are zero).
__device__ __forceinline__ void load_a(const float *x, int64_t r0, int64_t n, unsigned a[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t ra = r0 + g, rb = r0 + g + 8;
    float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (ra < n) {
        v[0] = x[ra * kInPad + 2 * t]; v[1] = x[ra * kInPad + 2 * t + 1];
        v[4] = x[ra * kInPad + 2 * t + 8]; v[5] = x[ra * kInPad + 2 * t + 9];
    }
    if (rb < n) {
        v[2] = x[rb * kInPad + 2 * t]; v[3] = x[rb * kInPad + 2 * t + 1];
        v[6] = x[rb * kInPad + 2 * t + 8]; v[7] = x[rb * kInPad + 2 * t + 9];
    }
    a[0] = pack_bf16(v[0], v[1]);
    a[1] = pack_bf16(v[2], v[3]);
    a[2] = pack_bf16(v[4], v[5]);
    a[3] = pack_bf16(v[6], v[7]);
}

// ---------------------------------------------------------------------------
// init, bfloat16 refresh, forward
// ---------------------------------------------------------------------------
// Glorot-uniform weights from SplitMix64(seed, index), zero biases, zero padding.
__global__ void mlp_init_k(MlpBlock P, unsigned long long seed) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
        float a = 0.f;
        bool use = false;
        if (i < ob1) { int k = (i - oW1) / kHid; use = k < kIn; a = sqrtf(6.f / (kIn + kHid)); }
        else if (i >= oW2 && i < ob2) { use = true; a = sqrtf(6.f / (2 * kHid)); }
        else if (i >= oW3 && i < ob3) { int n = (i - oW3) % kOutPad; use = n < kOut; a = sqrtf(6.f / (kHid + kOut)); }
        float u = (float)((splitmix64(seed ^ (0xA5A5A5A5ull + (unsigned long long)i)) >> 40) * (1.0 / 16777216.0));
        P.w[i] = use ? a * (2.f * u - 1.f) : 0.f;
        P.m[i] = 0.f;
        P.v[i] = 0.f;
    }
    // no feature box yet: every feature is inside
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * kInPad) P.box[i] = __int_as_float(i < kInPad ? 0xff800000 : 0x7f800000);
}

// The box of the features x[n][16] (n >= 1): per feature the smallest and the
// largest value. One block of 512 threads: thread t takes feature t % 16 of
// rows t / 16, t / 16 + 32, ...
__global__ void __launch_bounds__(512) mlp_box_k(MlpBlock P, int64_t n, const float *x) {
    __shared__ float lo[512], hi[512];
    const int t = threadIdx.x, k = t & (kInPad - 1);
    float a = __int_as_float(0x7f800000), b = __int_as_float(0xff800000);
    for (int64_t r = t >> 4; r < n; r += 512 / kInPad) {
        const float v = x[r * kInPad + k];
        a = fminf(a, v);
        b = fmaxf(b, v);
    }
    lo[t] = a;
    hi[t] = b;
    __syncthreads();
    for (int h = 256; h >= kInPad; h >>= 1) {
        if (t < h) {
            lo[t] = fminf(lo[t], lo[t + h]);
            hi[t] = fmaxf(hi[t], hi[t + h]);
        }
        __syncthreads();
    }
    if (t < kInPad) {
        P.box[t] = lo[t];
        P.box[kInPad + t] = hi[t];
    }
}

__global__ void mlp_sync_k(MlpBlock P) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kBf16; i += gridDim.x * blockDim.x) {
        float v;
        if (i < oW2t) { int n = i / kInPad, k = i % kInPad; v = P.w[oW1 + k * kHid + n]; }
        else if (i < oW3t) { int j = i - oW2t, n = j / kHid, k = j % kHid; v = P.w[oW2 + k * kHid + n]; }
        else { int j = i - oW3t, n = j / kHid, k = j % kHid; v = P.w[oW3 + k * kOutPad + n]; }
        P.wb[i] = __float2bfloat16_rn(v);
    }
}

// ---------------------------------------------------------------------------
// gradients: one block = 64 rows; FP32 backward through the rounded forward
// ---------------------------------------------------------------------------
struct GradSmem {
    MlpSmem W;
    float x0[64][kInPad];
    float z1[64][kHid], h1[64][kHid], z2[64][kHid], h2[64][kHid];
    float dy[64][kOutPad];
    float red[128];
};

__global__ void __launch_bounds__(128) mlp_grad_k(MlpBlock P, int64_t n, const float *x, const float *tgt,
                                                  float *partial, float *loss_partial) {
    extern __shared__ __align__(16) char smem_raw[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(smem_raw);
    load_mlp_smem(P, S.W);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int64_t r0 = (int64_t)blockIdx.x * 64 + wid * 16;
    const float inv = 2.f / (float)(n * kOut);
    // forward of this warp's 16 rows, keeping what the backward needs
    {
        unsigned a[4];
        load_a(x, r0, n, a);
        float z1[8][4], z2[8][4], y[4];
        mlp_warp_forward(S.W, a, y, z1, z2);
        const int ra = wid * 16 + g, rb = ra + 8;
#pragma unroll
        for (int j = 0; j < 8; j++)
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int col = 8 * j + 2 * t + q;
                S.z1[ra][col] = z1[j][q];
                S.z1[rb][col] = z1[j][2 + q];
                S.z2[ra][col] = z2[j][q];
                S.z2[rb][col] = z2[j][2 + q];
                S.h1[ra][col] = __bfloat162float(__float2bfloat16_rn(silu(z1[j][q])));
                S.h1[rb][col] = __bfloat162float(__float2bfloat16_rn(silu(z1[j][2 + q])));
                S.h2[ra][col] = __bfloat162float(__float2bfloat16_rn(silu(z2[j][q])));
                S.h2[rb][col] = __bfloat162float(__float2bfloat16_rn(silu(z2[j][2 + q])));
            }
        float lsum = 0.f;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int col = 2 * t + q;
            const int64_t gra = r0 + g, grb = r0 + g + 8;
            float da = 0.f, db = 0.f;
            if (col < kOut && gra < n) { float e = y[q] - tgt[gra * kOut + col]; da = inv * e; lsum += e * e; }
            if (col < kOut && grb < n) { float e = y[2 + q] - tgt[grb * kOut + col]; db = inv * e; lsum += e * e; }
            S.dy[ra][col] = da;
            S.dy[rb][col] = db;
        }
        for (int c = 0; c < kInPad; c++) {
            // rounded inputs, row by row (two rows per lane group)
            if (lane < 16) {
                const int64_t r = r0 + lane;
                S.x0[wid * 16 + lane][c] = (r < n) ? __bfloat162float(__float2bfloat16_rn(x[r * kInPad + c])) : 0.f;
            }
        }
        S.red[threadIdx.x] = lsum;
    }
    __syncthreads();
    // dZ2 = (dY W3b^T) . silu'(Z2), in place of z2
    for (int e = threadIdx.x; e < 64 * kHid; e += 128) {
        const int r = e / kHid, i = e % kHid;
        float s = 0.f;
        for (int o = 0; o < kOut; o++) s += S.dy[r][o] * __bfloat162float(S.W.wb[oW3t + o * kHid + i]);
        S.z2[r][i] = s * silu_grad(S.z2[r][i]);
    }
    __syncthreads();
    // dZ1 = (dZ2 W2b^T) . silu'(Z1), in place of z1
    for (int e = threadIdx.x; e < 64 * kHid; e += 128) {
        const int r = e / kHid, i = e % kHid;
        float s = 0.f;
        for (int j = 0; j < kHid; j++) s += S.z2[r][j] * __bfloat162float(S.W.wb[oW2t + j * kHid + i]);
        S.z1[r][i] = s * silu_grad(S.z1[r][i]);
    }
    __syncthreads();
    // this block's share of every gradient entry (sums over its 64 rows)
    float *out = partial + (int64_t)blockIdx.x * kParams;
    for (int p = threadIdx.x; p < kParams; p += 128) {
        float s = 0.f;
        if (p < ob1) { int k = p / kHid, j = p % kHid; for (int r = 0; r < 64; r++) s += S.x0[r][k] * S.z1[r][j]; }
        else if (p < oW2) { int j = p - ob1; for (int r = 0; r < 64; r++) s += S.z1[r][j]; }
        else if (p < ob2) { int k = (p - oW2) / kHid, j = (p - oW2) % kHid; for (int r = 0; r < 64; r++) s += S.h1[r][k] * S.z2[r][j]; }
        else if (p < oW3) { int j = p - ob2; for (int r = 0; r < 64; r++) s += S.z2[r][j]; }
        else if (p < ob3) { int k = (p - oW3) / kOutPad, o = (p - oW3) % kOutPad; for (int r = 0; r < 64; r++) s += S.h2[r][k] * S.dy[r][o]; }
        else { int o = p - ob3; for (int r = 0; r < 64; r++) s += S.dy[r][o]; }
        out[p] = s;
    }
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < 128; i++) s += S.red[i];
        loss_partial[blockIdx.x] = s;
    }
}

// grad[p] = sum over blocks in block order; loss = mean squared error
__global__ void mlp_reduce_k(int nblk, const float *partial, const float *loss_partial, float *grad, float *loss,
                             int64_t n) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kParams; p += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblk; b++) s += partial[(int64_t)b * kParams + p];
        grad[p] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        float s = 0.f;
        for (int b = 0; b < nblk; b++) s += loss_partial[b];
        *loss = s / (float)(n * kOut);
    }
}

// Adam (Kingma & Ba 2015), step t >= 1, on the FP32 master weights
__global__ void mlp_adam_k(MlpBlock P, const float *grad, int t, float lr, float b1, float b2, float eps) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float m = b1 * P.m[i] + (1.f - b1) * gr;
        const float v = b2 * P.v[i] + (1.f - b2) * gr * gr;
        P.m[i] = m;
        P.v[i] = v;
        P.w[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// Minibatch of training: row i of step k is row idx = floor(h n / 2^64) of
// (x, t) with h = SplitMix64(seed + k batch + i) (64-bit wrap-around), copied
// to (bx, bt).
__global__ void mlp_draw_k(int64_t n, const float *x, const float *t, int batch, unsigned long long seed, long long k,
                           float *bx, float *bt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        const unsigned long long h = splitmix64(seed + (unsigned long long)k * (unsigned long long)batch + i);
        const int64_t r = (int64_t)__umul64hi(h, (unsigned long long)n);
        const float4 *src = reinterpret_cast<const float4 *>(x + r * kInPad);
        float4 *dst = reinterpret_cast<float4 *>(bx + (int64_t)i * kInPad);
#pragma unroll
        for (int c = 0; c < kInPad / 4; c++) dst[c] = src[c];
#pragma unroll
        for (int q = 0; q < kOut; q++) bt[(int64_t)i * kOut + q] = t[r * kOut + q];
    }
}

// ---------------------------------------------------------------------------
// features of a (point, cell) pair; residual of the cell's multipole force
// ---------------------------------------------------------------------------
struct CellGeo {
    const float4 *pos;
    const int4 *cbox;
    const int4 *clink;
    const float4 *cmom;
    const float4 *coct;   // each cell's traceless octupole (octupole_k), 3 float4
    const int64_t *moff;
    int M;
    const double *mbounds;
    const int *mroot;
    int ncell;
};

__device__ __forceinline__ void member_geo(const CellGeo &T, int m, float lo[3], float &unit) {
    const double *b = T.mbounds + 5 * m;
    lo[0] = (float)b[0]; lo[1] = (float)b[1]; lo[2] = (float)b[2];
    unit = (float)(b[3] / 2097152.0);
}

// Traceless third moment of every cell about its centre of mass (the term the
// quadrupole expansion leaves out): a leaf from its stars, O_abc = sum_j m_j
// d_a d_b d_c (d = x_j - com); an internal cell from its children k (offset
// D_k of the child's centre of mass, mass M_k, traceless quadrupole Q_k):
// O_abc = sum_k [M_k D_a D_b D_c + (D_a Q_k,bc + D_b Q_k,ac + D_c Q_k,ab) / 3]
// (the children's own third moments left out); then O^T = O - (delta t + ..)/5,
// t_a = O_akk. Stored as (xxx, xxy, xxz, xyy), (xyz, xzz, yyy, yyz), (yzz, zzz, 0, 0).
__device__ __forceinline__ void oct_add(float O[10], float w, float dx, float dy, float dz) {
    const float wx = w * dx, wy = w * dy, wz = w * dz;
    O[0] += wx * dx * dx; O[1] += wx * dx * dy; O[2] += wx * dx * dz; O[3] += wx * dy * dy; O[4] += wx * dy * dz;
    O[5] += wx * dz * dz; O[6] += wy * dy * dy; O[7] += wy * dy * dz; O[8] += wy * dz * dz; O[9] += wz * dz * dz;
}
__global__ void octupole_k(CellGeo T, float4 *coct) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < T.ncell; c += gridDim.x * blockDim.x) {
        const int4 lk = T.clink[c];
        const float4 r0 = T.cmom[3 * c];
        float O[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (r0.x > 0.f && lk.z >= 0 && lk.w >= lk.z) {
            const int m = member_of(T.moff, T.M, lk.z);
            float lo[3], unit;
            const double *b = T.mbounds + 5 * m;
            lo[0] = (float)b[0]; lo[1] = (float)b[1]; lo[2] = (float)b[2];
            unit = (float)(b[3] / 2097152.0);
            float c0[3];
            geo_centre(T.cbox[c], lo, unit, c0);
            if (lk.x == lk.y) {   // a leaf: its stars
                for (int j = lk.z; j < lk.w; j++) {
                    const float4 p = T.pos[j];
                    oct_add(O, p.w, (p.x - c0[0]) - r0.y, (p.y - c0[1]) - r0.z, (p.z - c0[2]) - r0.w);
                }
            } else {              // its children
                for (int k = lk.x; k < lk.y && k < T.ncell; k++) {
                    const float4 a = T.cmom[3 * k], qa = T.cmom[3 * k + 1], qb = T.cmom[3 * k + 2];
                    float ck[3];
                    geo_centre(T.cbox[k], lo, unit, ck);
                    const float D[3] = {(ck[0] - c0[0]) + (a.y - r0.y), (ck[1] - c0[1]) + (a.z - r0.z),
                                        (ck[2] - c0[2]) + (a.w - r0.w)};
                    oct_add(O, a.x, D[0], D[1], D[2]);
                    // (D_a Q_bc + D_b Q_ac + D_c Q_ab) / 3, Q = (xx, yy, zz, xy, xz, yz) = (qa.x, qa.y, qa.z, qa.w, qb.x, qb.y)
                    const float Qxx = qa.x, Qyy = qa.y, Qzz = qa.z, Qxy = qa.w, Qxz = qb.x, Qyz = qb.y;
                    const float t3 = 1.f / 3.f;
                    O[0] += t3 * 3.f * D[0] * Qxx;                               // xxx
                    O[1] += t3 * (2.f * D[0] * Qxy + D[1] * Qxx);                // xxy
                    O[2] += t3 * (2.f * D[0] * Qxz + D[2] * Qxx);                // xxz
                    O[3] += t3 * (D[0] * Qyy + 2.f * D[1] * Qxy);                // xyy
                    O[4] += t3 * (D[0] * Qyz + D[1] * Qxz + D[2] * Qxy);         // xyz
                    O[5] += t3 * (D[0] * Qzz + 2.f * D[2] * Qxz);                // xzz
                    O[6] += t3 * 3.f * D[1] * Qyy;                               // yyy
                    O[7] += t3 * (2.f * D[1] * Qyz + D[2] * Qyy);                // yyz
                    O[8] += t3 * (D[1] * Qzz + 2.f * D[2] * Qyz);                // yzz
                    O[9] += t3 * 3.f * D[2] * Qzz;                               // zzz
                }
            }
            // traceless part: t = (xxx + xyy + xzz, xxy + yyy + yzz, xxz + yyz + zzz)
            const float tx = O[0] + O[3] + O[5], ty = O[1] + O[6] + O[8], tz = O[2] + O[7] + O[9];
            const float f5 = 0.2f;
            O[0] -= f5 * 3.f * tx; O[1] -= f5 * ty; O[2] -= f5 * tz; O[3] -= f5 * tx; O[4] -= 0.f;
            O[5] -= f5 * tx; O[6] -= f5 * 3.f * ty; O[7] -= f5 * tz; O[8] -= f5 * ty; O[9] -= f5 * 3.f * tz;
        }
        coct[3 * c] = make_float4(O[0], O[1], O[2], O[3]);
        coct[3 * c + 1] = make_float4(O[4], O[5], O[6], O[7]);
        coct[3 * c + 2] = make_float4(O[8], O[9], 0.f, 0.f);
    }
}

// O^T(., rh, rh) of a cell's stored traceless octupole
__device__ __forceinline__ void oct_dir(const float4 o0, const float4 o1, const float4 o2, const float rh[3], float v[3]) {
    const float x = rh[0], y = rh[1], z = rh[2];
    const float xxx = o0.x, xxy = o0.y, xxz = o0.z, xyy = o0.w, xyz = o1.x, xzz = o1.y, yyy = o1.z, yyz = o1.w,
                yzz = o2.x, zzz = o2.y;
    v[0] = xxx * x * x + xyy * y * y + xzz * z * z + 2.f * (xxy * x * y + xxz * x * z + xyz * y * z);
    v[1] = xxy * x * x + yyy * y * y + yzz * z * z + 2.f * (xyy * x * y + xyz * x * z + yyz * y * z);
    v[2] = xxz * x * x + yyz * y * y + zzz * z * z + 2.f * (xyz * x * y + xzz * x * z + yzz * y * z);
}

// r = x - com with x given relative to the point g (xr = x - g), gc = cell
// centre - g: com - g = gc + (com - c0). Writes 16 features (14 used: the
// direction, s / |r|, eps / |r|, Q / (M s^2), and the octupole term of the
// cell's acceleration in the output's units, (5/2) [3 v - 7 r^ (r^ . v)] /
// (M |r|^3) with v = O^T(., r^, r^), from the potential -(5/2) O^T(r^, r^, r^)
// / |r|^4) and returns M / |r|^2.
__device__ float pair_features(const float4 r0, const float4 q0, const float4 q1, const float4 *oct, float side,
                               float eps, const float r[3], float f[kInPad]) {
    const float d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    if (!(r0.x > 0.f) || !(d2 > 0.f)) {  // massless (ghost) cell: no correction
        for (int k = 0; k < kInPad; k++) f[k] = 0.f;
        return 0.f;
    }
    const float d = sqrtf(d2), id = 1.f / d;
    f[0] = r[0] * id; f[1] = r[1] * id; f[2] = r[2] * id;
    f[3] = side * id;
    f[4] = eps * id;
    const float qs = 1.f / (r0.x * side * side);
    f[5] = q0.x * qs; f[6] = q0.y * qs; f[7] = q0.z * qs; f[8] = q0.w * qs; f[9] = q1.x * qs; f[10] = q1.y * qs;
    const float rh[3] = {f[0], f[1], f[2]};
    float v[3];
    oct_dir(oct[0], oct[1], oct[2], rh, v);
    const float rv = rh[0] * v[0] + rh[1] * v[1] + rh[2] * v[2];
    const float os = 2.5f * id * id * id / r0.x;
    f[11] = os * (3.f * v[0] - 7.f * rh[0] * rv);
    f[12] = os * (3.f * v[1] - 7.f * rh[1] * rv);
    f[13] = os * (3.f * v[2] - 7.f * rh[2] * rv);
    for (int k = kIn; k < kInPad; k++) f[k] = 0.f;
    return r0.x / d2;
}

// Sample s: star i = SplitMix64 pick; walk of that star alone at theta
// (box: its grid cell) choosing uniformly among accepted cells (reservoir);
// features, residual target and the pair (i, cell).
__global__ void mlp_samples_k(CellGeo T, MacTable mac, int64_t n, float eps, unsigned long long seed, int64_t ns,
                              float *xo, float *to, int2 *pairs, DevState *st) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long h = splitmix64(seed + 2 * (unsigned long long)s);
        const int i = (int)(h % (unsigned long long)n);
        const float4 p = T.pos[i];
        const int m = member_of(T.moff, T.M, i);
        const double *mb = T.mbounds + 5 * m;
        int blo[3], bhi[3];
        const float pv[3] = {p.x, p.y, p.z};
        for (int a = 0; a < 3; a++) {
            double q = floor(__dmul_rn(__dsub_rn((double)pv[a], mb[a]), mb[4]));
            q = fmin(fmax(q, -8388608.0), 8388608.0);
            blo[a] = (int)q;
            bhi[a] = (int)q + 1;
        }
        int stack[192];
        int top = 0, chosen = -1;
        long long nacc = 0;
        stack[top++] = T.mroot[m];
        int guard = T.ncell + 1;
        while (top > 0) {
            if (--guard < 0) { latch_err(st, kErrStack); break; }
            const int c = stack[--top];
            if (c < 0 || c >= T.ncell) { latch_err(st, kErrCells); break; }
            const int4 b = T.cbox[c];
            const int side = 1 << (kMaxLevel - b.w);
            long long gx = (b.x >= bhi[0]) ? b.x - bhi[0] : ((blo[0] >= b.x + side) ? blo[0] - (b.x + side) : 0);
            long long gy = (b.y >= bhi[1]) ? b.y - bhi[1] : ((blo[1] >= b.y + side) ? blo[1] - (b.y + side) : 0);
            long long gz = (b.z >= bhi[2]) ? b.z - bhi[2] : ((blo[2] >= b.z + side) ? blo[2] - (b.z + side) : 0);
            const unsigned long long d2 = (unsigned long long)(gx * gx + gy * gy + gz * gz);
            if (d2 >= mac.thr[b.w]) {
                nacc++;
                const unsigned long long u = splitmix64(seed + 2 * (unsigned long long)s + 1 + 0x51ED27ull * nacc);
                if (u % (unsigned long long)nacc == 0) chosen = c;
                continue;
            }
            const int4 lk = T.clink[c];
            if (lk.x == lk.y) continue;
            if (top + (lk.y - lk.x) > 192) { latch_err(st, kErrStack); break; }
            for (int ch = lk.y - 1; ch >= lk.x; ch--) stack[top++] = ch;
        }
        float f[kInPad], tr[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < kInPad; k++) f[k] = 0.f;
        if (chosen >= 0) {
            float lo[3], unit;
            member_geo(T, m, lo, unit);
            const int4 b = T.cbox[chosen];
            float c0[3];
            geo_centre(b, lo, unit, c0);
            const float4 r0 = T.cmom[3 * chosen], q0 = T.cmom[3 * chosen + 1], q1 = T.cmom[3 * chosen + 2];
            // r = x - com = (x - c0) - (com - c0)
            const float r[3] = {(p.x - c0[0]) - r0.y, (p.y - c0[1]) - r0.z, (p.z - c0[2]) - r0.w};
            const float side = unit * (float)(1 << (kMaxLevel - b.w));
            const float norm = pair_features(r0, q0, q1, T.coct + 3 * chosen, side, eps, r, f);
            // exact softened force of the cell's stars
            const int4 lk = T.clink[chosen];
            float ex[3] = {0.f, 0.f, 0.f};
            for (int j = lk.z; j < lk.w; j++) {
                const float4 sj = T.pos[j];
                const float dx = sj.x - p.x, dy = sj.y - p.y, dz = sj.z - p.z;
                const float q2 = dx * dx + dy * dy + dz * dz + eps * eps;
                const float ri = rsqrtf(q2);
                const float w = sj.w * ri * ri * ri;
                ex[0] += w * dx; ex[1] += w * dy; ex[2] += w * dz;
            }
            // its monopole + quadrupole force
            const float rho2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps * eps;
            const float ri = rsqrtf(rho2), ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
            const float qx = q0.x * r[0] + q0.w * r[1] + q1.x * r[2];
            const float qy = q0.w * r[0] + q0.y * r[1] + q1.y * r[2];
            const float qz = q1.x * r[0] + q1.y * r[1] + q0.z * r[2];
            const float rqr = r[0] * qx + r[1] * qy + r[2] * qz;
            const float qd[3] = {qx, qy, qz};
            for (int a = 0; a < 3; a++) {
                const float quad = -r0.x * r[a] * ri3 + qd[a] * ri5 - 2.5f * rqr * r[a] * ri7;
                tr[a] = (norm > 0.f) ? (ex[a] - quad) / norm : 0.f;
            }
        }
        for (int k = 0; k < kInPad; k++) xo[s * kInPad + k] = f[k];
        for (int a = 0; a < 3; a++) to[s * kOut + a] = tr[a];
        if (pairs) pairs[s] = make_int2(i, chosen);
    }
}

// ---------------------------------------------------------------------------
// inference on the 5th-generation tensor cores (tcgen05)
// ---------------------------------------------------------------------------
// One CTA of 128 threads evaluates the network on tiles of 128 rows; thread i
// owns row i of a tile, which is lane i of the accumulator in tensor memory
// (warp w reads lanes 32w .. 32w + 31). Per tile: the features (bfloat16) go
// to shared memory, one thread issues the MMAs of a layer (M = 128, FP32
// accumulator in TMEM columns 0 .. 63) and commits them to an mbarrier; every
// thread then reads its row back, adds the bias, applies SiLU and writes the
// next layer's A operand straight into its own TMEM lane (columns 64 .. 95, two
// bfloat16 per column, even k in the low half), so the hidden activations
// never pass through shared memory. The weights (B) and layer 1's features
// (A) sit in shared memory in the no-swizzle K-major layout of the tcgen05
// matrix descriptors: 8 rows x 16 bytes per core matrix (rows 16 bytes apart),
// core matrices adjacent in K 128 bytes apart (leading byte offset), 8-row
// groups K x 16 bytes apart (stride byte offset).
constexpr int kTcRows = 128;   // rows per tile (the MMA's M)
// TMEM columns of a CTA: the three layers' FP32 accumulators (0 .. 63) and the
// bfloat16 hidden activations as the next layer's A operand (64 .. 95, two per
// column)
constexpr int kTcCols = 128;
constexpr int kTcACol = 64;
constexpr int kTcOutN = 16;    // layer 3's N (3 outputs, padded)
constexpr int kTcCtas = 4;     // resident CTAs per SM (4 x 128 of 512 TMEM columns)

struct TcSmem {
    alignas(128) __nv_bfloat16 a1[kTcRows * kInPad];   // features: K = 16
    alignas(128) __nv_bfloat16 w1[kHid * kInPad];      // W1^T: N = 64 rows, K = 16
    alignas(128) __nv_bfloat16 w2[kHid * kHid];        // W2^T: 64 x 64
    alignas(128) __nv_bfloat16 w3[kTcOutN * kHid];     // W3^T: 16 x 64 (rows 8 .. 15 zero)
    float b1[kHid], b2[kHid], b3[kOutPad];             // b1, b2 hold half the biases (silu_pair)
    float blo[kInPad], bhi[kInPad];                    // the feature box of the training data
    float red[4][32][3];                               // pair rows: per-warp terms for the group sums
    unsigned long long bar;                            // MMA completion
    unsigned tmem;                                     // TMEM base address from tcgen05.alloc
};

// element offset of (row r, column k) in a K-wide operand tile
__device__ __forceinline__ int tc_off(int r, int k, int K) {
    return (r >> 3) * (8 * K) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of a K-wide tile (no swizzle, K-major)
__device__ __forceinline__ unsigned long long tc_desc(const void *tile, int K) {
    const unsigned a = smem_u32(tile);
    return (unsigned long long)((a & 0x3FFFFu) >> 4) | ((unsigned long long)(128 >> 4) << 16) |
           ((unsigned long long)((16 * K) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, bfloat16 A and B,
// both K-major, M x N
__host__ __device__ constexpr unsigned tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the same with the A operand in tensor memory at column address a
__device__ __forceinline__ void tc_mma_ta(unsigned d, unsigned a, unsigned long long b, unsigned idesc,
                                          unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
        :
        : "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory writes of this thread become visible to the tensor cores' reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the phase of parity `ph` of the barrier; false after `limit`
// clock cycles (default 2^31, ~1 s) without completion.
__device__ __forceinline__ bool bar_wait(unsigned long long *bar, unsigned ph, long long limit = 1ll << 31) {
    const unsigned a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(ph)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// 16 consecutive FP32 columns of this thread's TMEM lane, starting at taddr
__device__ __forceinline__ void tc_ld16(unsigned taddr, float v[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    // the registers are read only after the load completed
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// Weights (bfloat16, n-major as stored: element (k, n) at [n][k]) and biases
// into the operand layout.
__device__ void tc_load_weights(const MlpBlock &P, TcSmem &S) {
    for (int i = threadIdx.x; i < kHid * kInPad; i += blockDim.x)
        S.w1[tc_off(i / kInPad, i % kInPad, kInPad)] = P.wb[oW1t + i];
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x)
        S.w2[tc_off(i / kHid, i % kHid, kHid)] = P.wb[oW2t + i];
    for (int i = threadIdx.x; i < kTcOutN * kHid; i += blockDim.x) {
        const int nn = i / kHid, k = i % kHid;
        S.w3[tc_off(nn, k, kHid)] = nn < kOutPad ? P.wb[oW3t + i] : __float2bfloat16_rn(0.f);
    }
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        S.b1[i] = 0.5f * P.w[ob1 + i];   // exact: a power-of-two scaling
        S.b2[i] = 0.5f * P.w[ob2 + i];
    }
    if (threadIdx.x < kOutPad) S.b3[threadIdx.x] = P.w[ob3 + threadIdx.x];
    if (threadIdx.x < kInPad) {
        S.blo[threadIdx.x] = P.box[threadIdx.x];
        S.bhi[threadIdx.x] = P.box[kInPad + threadIdx.x];
    }
}

// This thread's 16 features into row r of the layer-1 operand.
__device__ __forceinline__ void tc_put_features(TcSmem &S, int r, const float f[kInPad]) {
#pragma unroll
    for (int c = 0; c < 2; c++) {
        uint4 u;
        u.x = pack_bf16(f[8 * c + 0], f[8 * c + 1]);
        u.y = pack_bf16(f[8 * c + 2], f[8 * c + 3]);
        u.z = pack_bf16(f[8 * c + 4], f[8 * c + 5]);
        u.w = pack_bf16(f[8 * c + 6], f[8 * c + 7]);
        *reinterpret_cast<uint4 *>(S.a1 + tc_off(r, 8 * c, kInPad)) = u;
    }
}

// Two SiLUs at once. SiLU of z = v + b (v the accumulator, b the bias) is
// h + h tanh(h) with h = z / 2 = v / 2 + b / 2 (z sigma(z) = z (1 + tanh(z / 2))
// / 2): h and h + h t are packed FP32 FMAs (fma.rn.f32x2, one instruction for
// both elements) and t = tanh(h) is the special-function unit's approximation
// (tanh.approx.f32), per element -- a third of the instructions of an
// exponential and a division, which bounded the epilogue. The approximation's
// measured error on GB300 is below 1.1e-5 relative (2^-16.5; PTX documents
// 2^-11 at most), far below the bfloat16 rounding of the result (2^-9).
__device__ __forceinline__ void silu_pair(float v0, float v1, float hb0, float hb1, float &s0, float &s1) {
    unsigned long long v, hb, h, t, o;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(v0), "f"(v1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(hb) : "f"(hb0), "f"(hb1));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(h) : "l"(v), "l"(0x3F0000003F000000ull), "l"(hb));   // 0.5f, 0.5f
    float h0, h1, t0, t1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(h0), "=f"(h1) : "l"(h));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(h0));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(h1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(t) : "f"(t0), "f"(t1));
    asm("fma.rn.f32x2 %0, %1, %2, %1;" : "=l"(o) : "l"(h), "l"(t));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(s0), "=f"(s1) : "l"(o));
}

// 32 FP32 columns of this thread's TMEM lane into r, without waiting
__device__ __forceinline__ void tc_ld32_issue(unsigned taddr, unsigned r[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}
// waits for every TMEM load this thread issued; r is read only after it
__device__ __forceinline__ void tc_ld_wait32(unsigned r[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]) : : "memory");
}

// 32 columns c0 .. c0 + 31 (in u) + half bias -> SiLU -> 16 bfloat16 pairs into this row's TMEM lane
__device__ __forceinline__ void tc_hidden32(const unsigned u[32], int c0, const float *hbias, unsigned a_taddr) {
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; j += 2)
        silu_pair(__uint_as_float(u[j]), __uint_as_float(u[j + 1]), hbias[c0 + j], hbias[c0 + j + 1], v[j], v[j + 1]);
    unsigned w[16];
#pragma unroll
    for (int c = 0; c < 16; c++) w[c] = pack_bf16(v[2 * c], v[2 * c + 1]);
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(a_taddr + (unsigned)(c0 / 2)), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]),
                   "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]),
                   "r"(w[13]), "r"(w[14]), "r"(w[15])
                 : "memory");
}

// All 64 accumulator columns of the row in flight at once (two 32-column
// loads), then 32 SiLU pairs with no load between them.
__device__ __forceinline__ void tc_hidden_wide(unsigned tlane, const float *hbias) {
    const unsigned at = tlane + kTcACol;
    unsigned a[32], b[32];
    tc_ld32_issue(tlane, a);
    tc_ld32_issue(tlane + 32, b);
    tc_ld_wait32(a);
    tc_ld_wait32(b);
    tc_hidden32(a, 0, hbias, at);
    tc_hidden32(b, 32, hbias, at);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Issues layer `layer` (1, 2, 3) of the tile by one thread and waits for it
// with every thread. The operands were written by all threads before.
__device__ __forceinline__ bool tc_layer(TcSmem &S, int layer, unsigned tmem, unsigned &phase) {
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_after_sync();
        if (layer == 1) {
            tc_mma(tmem, tc_desc(S.a1, kInPad), tc_desc(S.w1, kInPad), tc_idesc(kTcRows, kHid), 0u);
        } else {
            const unsigned long long db = layer == 2 ? tc_desc(S.w2, kHid) : tc_desc(S.w3, kHid);
            const unsigned id = layer == 2 ? tc_idesc(kTcRows, kHid) : tc_idesc(kTcRows, kTcOutN);
            // K = 64 in four steps of 16: A 8 TMEM columns further, B 2 core matrices (256 bytes) further each
#pragma unroll
            for (int s = 0; s < kHid / 16; s++)
                tc_mma_ta(tmem, tmem + kTcACol + 8u * s, db + 16ull * s, id, s > 0 ? 1u : 0u);
        }
        tc_commit(&S.bar);
    }
    const bool ok = bar_wait(&S.bar, phase);
    phase ^= 1u;
    tc_after_sync();
    return !__syncthreads_or(!ok);   // the same answer in every thread
}

__device__ __forceinline__ void tc_setup(TcSmem &S, const MlpBlock &P) {
    tc_load_weights(P, S);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&S.tmem)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
}

// A wait that timed out: wait once more (bounded) for the MMAs in flight, then
// free the tensor memory. Every thread calls it.
__device__ __forceinline__ void tc_teardown(TcSmem &S, bool ok, unsigned phase) {
    if (!ok) bar_wait(&S.bar, phase ^ 1u);
    tc_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(kTcCols) : "memory");
    }
}

// One tile after its features are in a1: the three layers; returns the three
// outputs of this thread's row (false, in every thread: a wait timed out).
__device__ __forceinline__ bool tc_tile(TcSmem &S, unsigned tmem, unsigned tlane, int r, unsigned &phase,
                                        float out[kOut]) {
    if (!tc_layer(S, 1, tmem, phase)) return false;
    tc_hidden_wide(tlane, S.b1);
    if (!tc_layer(S, 2, tmem, phase)) return false;
    tc_hidden_wide(tlane, S.b2);
    if (!tc_layer(S, 3, tmem, phase)) return false;
    float v[16];
    tc_ld16(tlane, v);
#pragma unroll
    for (int q = 0; q < kOut; q++) out[q] = v[q] + S.b3[q];
    return true;
}

// The bounded completion wait on its own: TMEM allocated as the inference
// kernels do, then a wait of `limit` cycles on an mbarrier that receives its
// one arrival (arrive = 1) or none (arrive = 0: the wait must give up), then
// TMEM freed. gave_up[0] = 1 if the wait gave up in any thread.
__global__ void __launch_bounds__(kTcRows) wait_selftest_k(long long limit, int arrive, int *gave_up) {
    __shared__ unsigned long long bar;
    __shared__ unsigned tmem;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem)), "r"(32) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (arrive && threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    }
    const bool ok = bar_wait(&bar, 0u, limit);
    const bool all_ok = !__syncthreads_or(!ok);
    tc_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
    }
    if (threadIdx.x == 0) gave_up[0] = all_ok ? 0 : 1;
}

// rows of x (n x 16 FP32) -> y (n x 3); a timed-out wait leaves NaN in the tile's rows
__global__ void __launch_bounds__(kTcRows) mlp_forward_tc_k(MlpBlock P, int64_t n, const float *x, float *y) {
    __shared__ TcSmem S;
    tc_setup(S, P);
    const int r = threadIdx.x;
    const unsigned tmem = S.tmem, tlane = tmem + ((unsigned)(32 * (r >> 5)) << 16);
    unsigned phase = 0;
    bool ok = true;
    const int64_t ntile = (n + kTcRows - 1) / kTcRows;
    const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    // this thread's row of tile t (zero past the end)
    auto load_row = [&](int64_t t, float f[kInPad]) {
        const int64_t row = t * kTcRows + r;
        if (row < n && vec) {
            const float4 *s = reinterpret_cast<const float4 *>(x + row * kInPad);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float4 u = __ldg(s + c);
                f[4 * c] = u.x; f[4 * c + 1] = u.y; f[4 * c + 2] = u.z; f[4 * c + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kInPad; k++) f[k] = row < n ? x[row * kInPad + k] : 0.f;
        }
    };
    float f[kInPad];
    load_row(blockIdx.x, f);
    for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        const int64_t row = t * kTcRows + r;
        tc_put_features(S, r, f);
        // the next tile's row is loaded while this tile runs
        load_row(t + gridDim.x, f);
        float o[kOut];
        ok = tc_tile(S, tmem, tlane, r, phase, o);
        if (row < n)
            for (int q = 0; q < kOut; q++) y[row * kOut + q] = ok ? o[q] : __int_as_float(0x7fc00000);
    }
    tc_teardown(S, ok, phase);
}


// ---------------------------------------------------------------------------
// correction of recorded (group, cell) pairs, evaluated at the group centre
// ---------------------------------------------------------------------------
// One row per recorded pair: features of the cell seen from the group's
// centre, the network on the tensor cores, and the output scaled by M / |r|^2
// summed into the group's correction (rows of one group within a warp are
// summed first: one atomic per group, warp and component).
__global__ void __launch_bounds__(kTcRows) mlp_pairs_tc_k(MlpBlock P, CellGeo T, const int4 *groups,
                                                          const int2 *pairs, const int *npairs, int cap, float eps,
                                                          float *gcorr, DevState *st) {
    __shared__ TcSmem S;
    tc_setup(S, P);
    const int r = threadIdx.x, lane = r & 31, wid = r >> 5;
    const unsigned tmem = S.tmem, tlane = tmem + ((unsigned)(32 * wid) << 16);
    unsigned phase = 0;
    bool ok = true;
    const int np = min(*npairs, cap);
    const int ntile = (np + kTcRows - 1) / kTcRows;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int p = t * kTcRows + r;
        float f[kInPad];
        float norm = 0.f;
        int gg = -1;
        if (p < np) {
            const int2 pr = pairs[p];
            gg = pr.x;
            const GroupRec grp = load_group(groups, pr.x);
            const int m = member_of(T.moff, T.M, grp.first);
            float lo[3], unit;
            member_geo(T, m, lo, unit);
            float gcen[3], c0[3];
            box_centre(grp.lo, grp.hi, lo, unit, gcen);
            const int4 b = T.cbox[pr.y];
            geo_centre(b, lo, unit, c0);
            const float4 q = T.cmom[3 * pr.y], q0 = T.cmom[3 * pr.y + 1], q1 = T.cmom[3 * pr.y + 2];
            // r = g - com = -((c0 - g) + (com - c0))
            const float rr[3] = {-((c0[0] - gcen[0]) + q.y), -((c0[1] - gcen[1]) + q.z),
                                 -((c0[2] - gcen[2]) + q.w)};
            const float side = unit * (float)(1 << (kMaxLevel - b.w));
            norm = pair_features(q, q0, q1, T.coct + 3 * pr.y, side, eps, rr, f);
            // outside the features the network was trained on: no correction (the plain tree)
            bool inside = true;
#pragma unroll
            for (int k = 0; k < kIn; k++) inside &= (f[k] >= S.blo[k]) && (f[k] <= S.bhi[k]);
            if (!inside) {
                norm = 0.f;
#pragma unroll
                for (int k = 0; k < kInPad; k++) f[k] = 0.f;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kInPad; k++) f[k] = 0.f;
        }
        tc_put_features(S, r, f);
        float o[kOut];
        ok = tc_tile(S, tmem, tlane, r, phase, o);
        if (!ok) {
            if (r == 0) latch_err(st, kErrTimeout);
            break;
        }
#pragma unroll
        for (int q = 0; q < kOut; q++) S.red[wid][lane][q] = o[q] * norm;
        const unsigned peers = __match_any_sync(0xffffffffu, gg);
        __syncwarp();
        if (gg >= 0 && lane == __ffs(peers) - 1) {
            float sum[kOut] = {0.f, 0.f, 0.f};
            for (unsigned mm = peers; mm; mm &= mm - 1) {
                const int l = __ffs(mm) - 1;
#pragma unroll
                for (int q = 0; q < kOut; q++) sum[q] += S.red[wid][l][q];
            }
#pragma unroll
            for (int q = 0; q < kOut; q++) atomicAdd(&gcorr[3 * gg + q], sum[q]);
        }
        __syncwarp();
    }
    tc_teardown(S, ok, phase);
}

// every star of group k gets the group's correction
__global__ void mlp_apply_k(const int4 *groups, const int *ngroup, const int *perm, const float *gcorr, float *ax,
                            float *ay, float *az) {
    const int ng = *ngroup;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += gridDim.x * blockDim.x) {
        const int4 grp = groups[2 * k];   // (first, count, ...)
        const float cx = gcorr[3 * k], cy = gcorr[3 * k + 1], cz = gcorr[3 * k + 2];
        for (int i = grp.x; i < grp.x + grp.y; i++) {
            const int o = perm[i];
            ax[o] += cx; ay[o] += cy; az[o] += cz;
        }
    }
}

// Dynamic shared memory that keeps at most CTAS CTAs of `kern` on an SM.
// Each CTA allocates kTcCols of the SM's 512 TMEM columns; a further CTA
// that registers and shared memory would still admit would wait in
// tcgen05.alloc until another CTA on its SM finishes, stretching the kernel's
// tail. Padding the CTA's shared memory just past the (CTAS + 1)-CTA share
// makes the scheduler place at most CTAS. Returns -1 on a CUDA error.
template <int CTAS, typename K>
static int tc_pad_smem(K kern) {
    static int cached = -2;
    if (cached != -2) return cached;
    int dev = 0, per_sm = 0, reserved = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
        return -1;
    int pad = std::max(0, per_sm / (CTAS + 1) - reserved - (int)fa.sharedSizeBytes + 128);
    pad = (pad + 127) & ~127;
    for (int k = 0; k < 64; k++, pad += 128) {
        if (pad > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pad) != cudaSuccess)
            return -1;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kTcRows, pad) != cudaSuccess) return -1;
        if (blocks <= CTAS) break;
    }
    cached = pad;
    return pad;
}

static CellGeo cell_geo(rv_ctx *c, int ncell_host) {
    CellGeo T;
    T.pos = c->w.pos;
    T.cbox = c->w.cbox;
    T.clink = reinterpret_cast<const int4 *>(c->w.clink);
    T.cmom = c->w.cmom;
    T.coct = c->w.coct;
    T.moff = c->w.moff;
    T.M = c->n_members;
    T.mbounds = c->w.mbounds;
    T.mroot = c->w.mroot;
    T.ncell = ncell_host;
    return T;
}

static rv_status read_ncell(rv_ctx *c, cudaStream_t s, int *ncell, int *ngroup) {
    int v[2];
    cudaError_t e = cudaMemcpyAsync(v, &c->w.st->ncell, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(c, e, "tree size");
    *ncell = (int)std::min<int64_t>(v[0], c->cell_cap);
    *ngroup = v[1];
    return RV_OK;
}

}  // namespace rv

using namespace rv;

extern "C" {

size_t rv_mlp_param_bytes(void) { return kBlockBytes; }

size_t rv_mlp_scratch_bytes(int64_t batch) {
    if (batch < 0) return 0;
    const int64_t nblk = (batch + 63) / 64;
    return sizeof(float) * (size_t)((nblk + 1) * kParams + nblk + 1);
}

rv_status rv_mlp_init(void *params, uint64_t seed, void *stream) {
    if (!params) return RV_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MlpBlock P = mlp_block(params);
    mlp_init_k<<<ceil_div(kParams, 256), 256, 0, s>>>(P, seed);
    mlp_sync_k<<<ceil_div(kBf16, 256), 256, 0, s>>>(P);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_mlp_forward(const void *params, int64_t n, const float *x, float *y, void *stream) {
    NvtxRange nvtx_range("rv_mlp_forward");
    if (!params || n < 0 || (n > 0 && (!x || !y))) return RV_E_INVAL;
    if (n == 0) return RV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    MlpBlock P = mlp_block(const_cast<void *>(params));
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return RV_E_CUDA;
    const int64_t ntile = (n + kTcRows - 1) / kTcRows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntile, (int64_t)sms * kTcCtas));
    const int pad = tc_pad_smem<kTcCtas>(mlp_forward_tc_k);
    if (pad < 0) return RV_E_CUDA;
    mlp_forward_tc_k<<<grid, kTcRows, pad, s>>>(P, n, x, y);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_mlp_fit_feature_box(void *params, int64_t n, const float *x, void *stream) {
    if (!params || n < 1 || !x) return RV_E_INVAL;
    mlp_box_k<<<1, 512, 0, (cudaStream_t)stream>>>(mlp_block(params), n, x);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_mlp_set_feature_box(void *params, const float *lo, const float *hi, void *stream) {
    if (!params || !lo || !hi) return RV_E_INVAL;
    for (int k = 0; k < kInPad; k++)
        if (!(lo[k] <= hi[k])) return RV_E_INVAL;
    MlpBlock P = mlp_block(params);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(P.box, lo, sizeof(float) * kInPad, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.box + kInPad, hi, sizeof(float) * kInPad, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host arrays may go out of scope after return
    return e == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_wait_selftest(int64_t limit_cycles, int32_t arrive, int32_t *gave_up, void *stream) {
    if (!gave_up || limit_cycles < 0 || limit_cycles > (1ll << 32) || (arrive != 0 && arrive != 1)) return RV_E_INVAL;
    wait_selftest_k<<<1, kTcRows, 0, (cudaStream_t)stream>>>((long long)limit_cycles, arrive, gave_up);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_mlp_gradient(const void *params, int64_t n, const float *x, const float *t, float *grad, float *loss,
                          void *scratch, size_t scratch_bytes, void *stream) {
    NvtxRange nvtx_range("rv_mlp_gradient");
    if (!params || n <= 0 || !x || !t || !grad || !scratch) return RV_E_INVAL;
    if (scratch_bytes < rv_mlp_scratch_bytes(n)) return RV_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpBlock P = mlp_block(const_cast<void *>(params));
    const int nblk = (int)((n + 63) / 64);
    float *partial = reinterpret_cast<float *>(scratch);
    float *lpart = partial + (int64_t)nblk * kParams;
    const size_t smem = sizeof(GradSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return RV_E_CUDA;
    mlp_grad_k<<<nblk, 128, smem, s>>>(P, n, x, t, partial, lpart);
    mlp_reduce_k<<<ceil_div(kParams, 256), 256, 0, s>>>(nblk, partial, lpart, grad, loss, n);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_mlp_adam(void *params, const float *grad, int32_t step, float lr, float beta1, float beta2,
                      float adam_eps, void *stream) {
    if (!params || !grad || step < 1) return RV_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MlpBlock P = mlp_block(params);
    mlp_adam_k<<<ceil_div(kParams, 256), 256, 0, s>>>(P, grad, step, lr, beta1, beta2, adam_eps);
    mlp_sync_k<<<ceil_div(kBf16, 256), 256, 0, s>>>(P);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

size_t rv_mlp_train_scratch_bytes(int32_t batch) {
    if (batch < 1) return 0;
    const size_t rows = sizeof(float) * (size_t)batch * (kInPad + kOut);
    return ((rows + 255) & ~(size_t)255) + ((sizeof(float) * kParams + 255) & ~(size_t)255) +
           rv_mlp_scratch_bytes(batch);
}

rv_status rv_mlp_train(void *params, const rv_mlp_train_cfg *cfg, float *losses, void *scratch,
                       size_t scratch_bytes, void *stream) {
    NvtxRange nvtx_range("rv_mlp_train");
    if (!params || !cfg || !scratch) return RV_E_INVAL;
    const rv_mlp_train_cfg &C = *cfg;
    if (C.n < 1 || !C.x || !C.t || C.steps < 0 || C.batch < 1 || C.step0 < 1 || !(C.lr >= 0.f) ||
        !(C.beta1 >= 0.f && C.beta1 < 1.f) || !(C.beta2 >= 0.f && C.beta2 < 1.f) || !(C.adam_eps > 0.f) ||
        (C.fit_box != 0 && C.fit_box != 1) || (reinterpret_cast<uintptr_t>(C.x) & 15) != 0 ||
        (int64_t)C.step0 + C.steps > (1ll << 31) - 1)
        return RV_E_INVAL;
    if (scratch_bytes < rv_mlp_train_scratch_bytes(C.batch)) return RV_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpBlock P = mlp_block(params);
    char *base = reinterpret_cast<char *>(scratch);
    const size_t rows = sizeof(float) * (size_t)C.batch * (kInPad + kOut);
    float *bx = reinterpret_cast<float *>(base);
    float *bt = bx + (size_t)C.batch * kInPad;
    float *grad = reinterpret_cast<float *>(base + ((rows + 255) & ~(size_t)255));
    char *gscr = base + ((rows + 255) & ~(size_t)255) + ((sizeof(float) * kParams + 255) & ~(size_t)255);
    const int nblk = (int)((C.batch + 63) / 64);
    float *partial = reinterpret_cast<float *>(gscr);
    float *lpart = partial + (int64_t)nblk * kParams;
    const size_t smem = sizeof(GradSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return RV_E_CUDA;
    for (int k = 0; k < C.steps; k++) {
        mlp_draw_k<<<ceil_div(C.batch, 256), 256, 0, s>>>(C.n, C.x, C.t, C.batch, C.seed, k, bx, bt);
        mlp_grad_k<<<nblk, 128, smem, s>>>(P, C.batch, bx, bt, partial, lpart);
        mlp_reduce_k<<<ceil_div(kParams, 256), 256, 0, s>>>(nblk, partial, lpart, grad, losses ? losses + k : nullptr,
                                                           C.batch);
        mlp_adam_k<<<ceil_div(kParams, 256), 256, 0, s>>>(P, grad, C.step0 + k, C.lr, C.beta1, C.beta2, C.adam_eps);
        mlp_sync_k<<<ceil_div(kBf16, 256), 256, 0, s>>>(P);
    }
    if (C.fit_box) mlp_box_k<<<1, 512, 0, s>>>(P, C.n, C.x);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

// Saved network state: a 64-byte header (magic, version, the layout's sizes,
// the block's byte count), then the parameter block as it is on the device.
struct MlpStateHeader {
    char magic[8];
    uint32_t version, in, in_pad, hid, out, out_pad, params, bf16;
    uint64_t block_bytes;
    uint32_t pad[4];
};
static_assert(sizeof(MlpStateHeader) == 64, "state header is 64 bytes");
static MlpStateHeader mlp_header() {
    MlpStateHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "rvmlp\0\0\0", 8);
    h.version = 1;
    h.in = kIn; h.in_pad = kInPad; h.hid = kHid; h.out = kOut; h.out_pad = kOutPad;
    h.params = kParams; h.bf16 = kBf16; h.block_bytes = kBlockBytes;
    return h;
}

size_t rv_mlp_state_bytes(void) { return sizeof(MlpStateHeader) + kBlockBytes; }

rv_status rv_mlp_save(const void *params, void *host, size_t bytes, void *stream) {
    if (!params || !host || bytes < rv_mlp_state_bytes()) return RV_E_INVAL;
    const MlpStateHeader h = mlp_header();
    memcpy(host, &h, sizeof h);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(reinterpret_cast<char *>(host) + sizeof h, params, kBlockBytes,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_mlp_load(void *params, const void *host, size_t bytes, void *stream) {
    if (!params || !host || bytes < rv_mlp_state_bytes()) return RV_E_INVAL;
    const MlpStateHeader want = mlp_header();
    if (memcmp(host, &want, sizeof want) != 0) return RV_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(params, reinterpret_cast<const char *>(host) + sizeof want, kBlockBytes,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host buffer may be freed after return
    return e == cudaSuccess ? RV_OK : RV_E_CUDA;
}

rv_status rv_mlp_samples(rv_ctx *c, float theta, float eps_star, int64_t n_samples, uint64_t seed, float *x,
                         float *t, int32_t *pairs, void *stream) {
    NvtxRange nvtx_range("rv_mlp_samples");
    if (!c) return RV_E_INVAL;
    if (!c->ws) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (!c->built || c->n == 0) return set_err(c, RV_E_NOTBUILT, "samples need a built, non-empty tree");
    if (n_samples < 0 || (n_samples > 0 && (!x || !t)) || !(theta > 0.f && theta < 2.f))
        return set_err(c, RV_E_INVAL, "bad sample arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int ncell, ngroup;
    rv_status r = read_ncell(c, s, &ncell, &ngroup);
    if (r != RV_OK || n_samples == 0) return r;
    const int grid = (int)std::min<int64_t>((n_samples + 127) / 128, (int64_t)c->num_sms * 16);
    octupole_k<<<std::max(1, std::min(ceil_div(ncell, 256), c->num_sms * 8)), 256, 0, s>>>(cell_geo(c, ncell),
                                                                                           c->w.coct);
    count_launch(c);
    mlp_samples_k<<<grid, 128, 0, s>>>(cell_geo(c, ncell), mac_table(theta), c->n, eps_star, seed, n_samples, x, t,
                                        reinterpret_cast<int2 *>(pairs), c->w.st);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "mlp samples");
}

rv_status rv_tree_forces_mlp(rv_ctx *c, const void *params, float theta, float theta_rec, float eps_star, float *ax,
                             float *ay, float *az, float *pot, int32_t *pairs, int32_t pair_cap, int32_t *npairs,
                             float *gcorr, void *stream) {
    NvtxRange nvtx_range("rv_tree_forces_mlp");
    if (!c) return RV_E_INVAL;
    if (!c->ws) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (!c->built) return set_err(c, RV_E_NOTBUILT, "rv_tree_forces_mlp before a build");
    if (!params || !pairs || !npairs || !gcorr || pair_cap < 0 || !(theta_rec > 0.f && theta_rec <= theta) ||
        !(theta < 2.f) || !(eps_star > 0.f) || (c->n > 0 && (!ax || !ay || !az || !pot)))
        return set_err(c, RV_E_INVAL, "bad arguments");
    if (c->cfg.quadrupole == 0) return set_err(c, RV_E_INVAL, "the correction is learned on quadrupole cells");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(npairs, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gcorr, 0, sizeof(float) * 3 * std::max<int64_t>(c->n, 1), s);
    if (e != cudaSuccess) return cuda_check(c, e, "mlp reset");
    PairRecord rec{theta_rec, reinterpret_cast<int2 *>(pairs), npairs, pair_cap};
    rv_status r = tree_walk(c, theta, eps_star, 0, nullptr, nullptr, nullptr, 0, ax, ay, az, pot, nullptr, s, &rec);
    if (r != RV_OK || c->n == 0) return r;
    int ncell, ngroup;
    if ((r = read_ncell(c, s, &ncell, &ngroup)) != RV_OK) return r;
    MlpBlock P = mlp_block(const_cast<void *>(params));
    octupole_k<<<std::max(1, std::min(ceil_div(ncell, 256), c->num_sms * 8)), 256, 0, s>>>(cell_geo(c, ncell),
                                                                                           c->w.coct);
    count_launch(c);
    const int grid = std::max(1, std::min(ceil_div(pair_cap, kTcRows), c->num_sms * kTcCtas));
    const int pad = tc_pad_smem<kTcCtas>(mlp_pairs_tc_k);
    if (pad < 0) return set_err(c, RV_E_CUDA, "network kernel attributes");
    mlp_pairs_tc_k<<<grid, kTcRows, pad, s>>>(P, cell_geo(c, ncell), c->w.groups, reinterpret_cast<const int2 *>(pairs),
                                            npairs, pair_cap, eps_star, gcorr, c->w.st);
    count_launch(c);
    mlp_apply_k<<<std::max(1, ceil_div(ngroup, 256)), 256, 0, s>>>(c->w.groups, &c->w.st->ngroup, c->w.perm, gcorr, ax,
                                                                 ay, az);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "mlp forces");
}

}  // extern "C"
