// build.cu -- octree construction on the GPU: bounding cube, Morton keys,
// stable LSD radix sort, gather into key order, topology, walk groups and
// cell multipoles (monopole + traceless quadrupole about the centre of mass,
// the expansion a tree code uses for distant groups, Sect. 1).
//
// Topology without per-level launches: for sorted keys, let D(j) be the first
// level at which key[j-1] and key[j] differ (D(0) = D(n) = 0, 22 for equal
// keys). At level l the key prefixes cut the sorted array at the positions
// with D(j) <= l. A star i lies in a cell at level l iff every coarser cell
// holding it has more than n_leaf stars, i.e. iff l <= lambda_i, the first
// level whose segment around i holds at most n_leaf stars (capped at 21).
// lambda_i only depends on D within n_leaf positions of i, so one pass over
// a window finds it; cells starting at i are levels D(i)..lambda_i, and their
// breadth-first index (level, first star) comes from per-level ballots and
// one flat scan.
#include <algorithm>

#include "rv_internal.cuh"

namespace rv {

// ---------------------------------------------------------------------------
// block helpers
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int *smem_warp, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < NT / 32) ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) smem_warp[lane] = w;
    }
    __syncthreads();
    int warp_base = (wid > 0) ? smem_warp[wid - 1] : 0;
    total = smem_warp[NT / 32 - 1];
    __syncthreads();
    return warp_base + x - v;
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (in place), length *d_len (<= nmax) or nmax
// ---------------------------------------------------------------------------
__global__ void scan_reduce_k(const int *data, int64_t nmax, const int *d_len, int *partials) {
    __shared__ int sw[8];
    int64_t len = d_len ? min((int64_t)*d_len, nmax) : nmax;
    int64_t base = (int64_t)blockIdx.x * kScanChunk;
    int sum = 0;
    for (int i = threadIdx.x; i < kScanChunk; i += 256) {
        int64_t j = base + i;
        if (j < len) sum += data[j];
    }
    int total;
    block_exclusive_scan<256>(sum, sw, total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void scan_partials_k(int *partials, int nb, int *d_total) {
    __shared__ int sw[32];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int b = b0 + threadIdx.x;
        int v = (b < nb) ? partials[b] : 0;
        int total;
        int ex = block_exclusive_scan<1024>(v, sw, total);
        if (b < nb) partials[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void scan_down_k(int *data, int64_t nmax, const int *d_len, const int *partials) {
    __shared__ int sw[8];
    int64_t len = d_len ? min((int64_t)*d_len, nmax) : nmax;
    int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * 8;
    int v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        int64_t j = base + k;
        v[k] = (j < len) ? data[j] : 0;
        s += v[k];
    }
    int total;
    int ex = block_exclusive_scan<256>(s, sw, total) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        int64_t j = base + k;
        if (j < len) data[j] = ex;
        ex += v[k];
    }
}

rv_status exclusive_scan(rv_ctx *c, int *data, int64_t nmax, const int *d_len, int *d_total, cudaStream_t s) {
    if (nmax <= 0) {
        if (d_total) return cuda_check(c, cudaMemsetAsync(d_total, 0, sizeof(int), s), "scan memset");
        return RV_OK;
    }
    int nb = ceil_div(nmax, kScanChunk);
    scan_reduce_k<<<nb, 256, 0, s>>>(data, nmax, d_len, c->w.partials);
    count_launch(c);
    scan_partials_k<<<1, 1024, 0, s>>>(c->w.partials, nb, d_total);
    count_launch(c);
    scan_down_k<<<nb, 256, 0, s>>>(data, nmax, d_len, c->w.partials);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "scan");
}

// ---------------------------------------------------------------------------
// bounding cube
// ---------------------------------------------------------------------------
// Blocks (bx, m): member m's stars, strided by bpm blocks.
__global__ void bounds_partial_k(const int64_t *moff, int bpm, const float *x, const float *y, const float *z,
                                 float *part) {
    const int m = blockIdx.y;
    const int64_t s = moff[m], e = moff[m + 1];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = s + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < e; i += (int64_t)bpm * blockDim.x) {
        float v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            lo[a] = fminf(lo[a], v[a]);
            hi[a] = fmaxf(hi[a], v[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    __shared__ float sh[8][6];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; a++) { sh[wid][a] = lo[a]; sh[wid][3 + a] = hi[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        float r = sh[0][threadIdx.x];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++)
            r = (threadIdx.x < 3) ? fminf(r, sh[w][threadIdx.x]) : fmaxf(r, sh[w][threadIdx.x]);
        part[6 * ((int64_t)m * bpm + blockIdx.x) + threadIdx.x] = r;
    }
}

// One warp per member: min per axis; L = max_a (max_a - min_a) with FP64
// differences; scale = 2^21 / L (min and max are exact, so order is free).
__global__ void bounds_final_k(int bpm, const float *part, double *mbounds, DevState *st) {
    const int m = blockIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < bpm; b += 32)
        for (int a = 0; a < 3; a++) {
            lo[a] = fminf(lo[a], part[6 * ((int64_t)m * bpm + b) + a]);
            hi[a] = fmaxf(hi[a], part[6 * ((int64_t)m * bpm + b) + 3 + a]);
        }
    for (int a = 0; a < 3; a++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if (threadIdx.x != 0) return;
    double out[5];
    double L = 0.0;
    for (int a = 0; a < 3; a++) {
        bool empty = !(lo[a] <= hi[a]);
        double e = empty ? 0.0 : __dsub_rn((double)hi[a], (double)lo[a]);
        if (e > L) L = e;
        out[a] = empty ? 0.0 : (double)lo[a];
    }
    out[3] = L;
    out[4] = (L > 0.0) ? __ddiv_rn(2097152.0, L) : 0.0;
    for (int k = 0; k < 5; k++) {
        mbounds[5 * m + k] = out[k];
        if (m == 0) st->bounds[k] = out[k];
    }
}

// ---------------------------------------------------------------------------
// Morton keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x | (x >> 4)) & 0x100f00f00f00f00full;
    x = (x | (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x | (x >> 16)) & 0x1f00000000ffffull;
    x = (x | (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

// q = min(floor((x - min) * scale), 2^21 - 1): one FP64 subtraction, one FP64
// product; for 0 <= t < 2^21 - 1 the floor is the conversion toward zero.
__device__ __forceinline__ uint32_t grid_coord(float v, double lo, double scale) {
    const double t = __dmul_rn(__dsub_rn((double)v, lo), scale);
    if (!(t >= 0.0)) return 0u;
    if (t >= 2097151.0) return 2097151u;
    return (uint32_t)__double2uint_rz(t);
}

// The same q decided in FP32 where FP32 can decide it (GB300's FP64 rate is
// a small fraction of its FP32 rate, and the FP64 rule bound the key kernel).
// d = x - min is formed exactly as an unevaluated pair of floats dh + dl
// (Knuth's two-sum), scale as the pair sh + sl (sl the FP32 rounding of the
// FP64 difference scale - sh, itself exact), and d * scale as ph + c: ph =
// dh sh rounded, its rounding error recovered exactly by an FMA, the cross
// terms dh sl and dl sh added by FMAs, dl sl left out. Then
// |ph + c - d scale| < 2^-45 d scale < 2^-23 while d scale < 2^22, the FP64
// rule's two roundings move its t by at most 2^-52 t < 2^-30 from d scale, and
// r = (ph - floor(ph)) + c carries one more rounding (< 2^-23). So when r lies
// farther than 2^-20 from every integer, floor(t) = floor(ph) + floor(r); next
// to an integer (t at or near a grid boundary, d = 0), or out of range or not
// finite, the FP64 rule is evaluated as written. Integers below 2^22 are exact
// in FP32.
struct GridAxis {
    double lo, scale;
    float lo32, sh, sl;
    bool fast;   // lo is an FP32 value (the minimum of FP32 coordinates) and the split is finite
};

__device__ __forceinline__ GridAxis grid_axis(double lo, double scale) {
    GridAxis g;
    g.lo = lo;
    g.scale = scale;
    g.lo32 = __double2float_rn(lo);
    g.sh = __double2float_rn(scale);
    g.sl = __double2float_rn(__dsub_rn(scale, (double)g.sh));
    g.fast = (double)g.lo32 == lo && isfinite(g.sh) && isfinite(g.sl);
    return g;
}

__device__ __forceinline__ uint32_t grid_coord_fast(float v, const GridAxis &g) {
    if (g.fast) {
        const float b = -g.lo32;
        const float dh = __fadd_rn(v, b);
        const float bb = __fsub_rn(dh, v);
        const float dl = __fadd_rn(__fsub_rn(v, __fsub_rn(dh, bb)), __fsub_rn(b, bb));
        const float ph = __fmul_rn(dh, g.sh);
        const float pl = __fmaf_rn(dh, g.sh, -ph);
        const float c = __fmaf_rn(dh, g.sl, __fmaf_rn(dl, g.sh, pl));
        if (ph >= 0.f && ph < 4194304.f) {
            const float f = floorf(ph);
            const float r = __fadd_rn(__fsub_rn(ph, f), c);
            constexpr float M = 9.5367431640625e-07f;   // 2^-20
            float q = -2.f;
            if (r > M && r < 1.f - M) q = f;
            else if (r > 1.f + M && r < 2.f - M) q = f + 1.f;
            else if (r > M - 1.f && r < -M) q = f - 1.f;
            if (q >= 0.f) return q >= 2097151.f ? 2097151u : (uint32_t)q;
        }
    }
    return grid_coord(v, g.lo, g.scale);
}

// Blocks (bx, m): member m's stars with member m's bounding cube. Each star's
// (x, y, z, m) is also packed into one float4 (caller order), so that the
// gather into key order reads one 16-byte record per star instead of four
// scattered 4-byte values (each costing a 32-byte sector).
__global__ void keys_k(const int64_t *moff, int bpm, const float *x, const float *y, const float *z,
                       const float *mass, const double *mbounds, uint64_t *key, float4 *xyzm) {
    const int m = blockIdx.y;
    const double sc = mbounds[5 * m + 4];
    const GridAxis gx = grid_axis(mbounds[5 * m], sc), gy = grid_axis(mbounds[5 * m + 1], sc),
                   gz = grid_axis(mbounds[5 * m + 2], sc);
    const int64_t s = moff[m], e = moff[m + 1];
    for (int64_t i = s + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < e; i += (int64_t)bpm * blockDim.x) {
        const float xi = x[i], yi = y[i], zi = z[i];
        uint64_t k = spread3(grid_coord_fast(xi, gx)) | (spread3(grid_coord_fast(yi, gy)) << 1) |
                     (spread3(grid_coord_fast(zi, gz)) << 2);
        key[i] = k;
        xyzm[i] = make_float4(xi, yi, zi, mass[i]);
    }
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, index), 9-bit digits
// ---------------------------------------------------------------------------
// Digit of element j: 9 key bits from `shift`, or (member pass) the member of
// its caller index, which groups the members while keeping each one's order.
__device__ __forceinline__ int sort_digit(const uint64_t *key, const int *idx, int64_t j, int shift,
                                          const int64_t *moff, int M) {
    if (moff) return member_of(moff, M, (int64_t)idx[j]);
    return (int)((key[j] >> shift) & (kSortBins - 1));
}

__global__ void __launch_bounds__(kSortThreads) sort_upsweep_k(int64_t n, const uint64_t *key, const int *idx,
                                                               int shift, const int64_t *moff, int M, int ntiles,
                                                               int *hist) {
    __shared__ int h[kSortBins];
    for (int b = threadIdx.x; b < kSortBins; b += kSortThreads) h[b] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    int d[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {   // the tile's loads first
        const int64_t j = base + k * kSortThreads + threadIdx.x;
        d[k] = j < n ? sort_digit(key, idx, j, shift, moff, M) : -1;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; k++)
        if (d[k] >= 0) atomicAdd(&h[d[k]], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < kSortBins; b += kSortThreads) hist[(int64_t)b * ntiles + blockIdx.x] = h[b];
}

// Each warp ranks 256 consecutive keys in 8 rounds of 32 (warp-private digit
// counters), so the in-tile order is (warp, round, lane) = input order and the
// sort is stable. The ranked tile is then staged in shared memory in digit
// order and written out from there: consecutive threads write consecutive
// slots of a digit's output run (coalesced), instead of each thread writing
// its own element straight to a scattered destination.
__global__ void __launch_bounds__(kSortThreads) sort_downsweep_k(int64_t n, const uint64_t *key_in,
                                                                 const int *idx_in, int shift, const int64_t *moff,
                                                                 int M, int ntiles, const int *hist,
                                                                 uint64_t *key_out, int *idx_out) {
    constexpr int NW = kSortThreads / 32;
    __shared__ unsigned short cnt[NW][kSortBins];
    __shared__ int gbase[kSortBins];
    __shared__ int lstart[kSortBins];            // first staged slot of each digit
    __shared__ uint64_t skey[kSortTile];
    __shared__ int sidx[kSortTile];
    __shared__ unsigned short sdig[kSortTile];
    __shared__ int sw[NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b = lane; b < kSortBins; b += 32) cnt[wid][b] = 0;
    for (int b = threadIdx.x; b < kSortBins; b += kSortThreads)
        gbase[b] = hist[(int64_t)b * ntiles + blockIdx.x];
    __syncwarp();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + wid * (32 * kSortItems);
    uint64_t kk[kSortItems];
    int ix[kSortItems], digit[kSortItems], rank[kSortItems];
    // every load of the tile first, so that their latencies overlap (the
    // ranking rounds below synchronise the warp)
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t j = base + r * 32 + lane;
        const bool ok = j < n;
        kk[r] = ok ? key_in[j] : 0ull;
        ix[r] = ok ? (idx_in ? idx_in[j] : (int)j) : 0;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t j = base + r * 32 + lane;
        int d = kSortBins;
        if (j < n) d = moff ? member_of(moff, M, (int64_t)ix[r]) : (int)((kk[r] >> shift) & (kSortBins - 1));
        digit[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int before = (d < kSortBins) ? cnt[wid][d] : 0;
        rank[r] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (d < kSortBins && lane == __ffs(peers) - 1) cnt[wid][d] = (unsigned short)(before + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    // per digit: the warps' counts become offsets within the digit's run of this tile
    static_assert(kSortBins % kSortThreads == 0, "each thread owns whole digits");
    int tot[kSortBins / kSortThreads];
#pragma unroll
    for (int q = 0; q < kSortBins / kSortThreads; q++) {
        const int b = threadIdx.x * (kSortBins / kSortThreads) + q;
        int run = 0;
        for (int w = 0; w < NW; w++) {
            int t = cnt[w][b];
            cnt[w][b] = (unsigned short)run;
            run += t;
        }
        tot[q] = run;
    }
    // digit runs in digit order: exclusive scan of the tile's digit totals
    {
        int mine = 0;
#pragma unroll
        for (int q = 0; q < kSortBins / kSortThreads; q++) mine += tot[q];
        int total;
        int ex = block_exclusive_scan<kSortThreads>(mine, sw, total);
#pragma unroll
        for (int q = 0; q < kSortBins / kSortThreads; q++) {
            lstart[threadIdx.x * (kSortBins / kSortThreads) + q] = ex;
            ex += tot[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        int64_t j = base + r * 32 + lane;
        if (j < n) {
            const int d = digit[r];
            const int slot = lstart[d] + cnt[wid][d] + rank[r];
            skey[slot] = kk[r];
            sidx[slot] = ix[r];
            sdig[slot] = (unsigned short)d;
        }
    }
    __syncthreads();
    const int tn = (int)min((int64_t)kSortTile, n - tile0);
    for (int t = threadIdx.x; t < tn; t += kSortThreads) {
        const int d = sdig[t];
        const int64_t dst = (int64_t)gbase[d] + (t - lstart[d]);
        key_out[dst] = skey[t];
        idx_out[dst] = sidx[t];
    }
}

rv_status radix_sort(rv_ctx *c, int64_t n, int passes, uint64_t **keys, int **idx, bool identity_idx,
                     cudaStream_t s, bool member_pass) {
    if (n <= 0) return RV_OK;
    int ntiles = ceil_div(n, kSortTile);
    uint64_t *kin = c->w.key_a, *kout = c->w.key_b;
    int *iin = identity_idx ? nullptr : c->w.idx_a, *iout = c->w.idx_b;
    const int M = c->n_members;
    const int total = passes + ((member_pass && M > 1) ? 1 : 0);
    for (int p = 0; p < total; p++) {
        int shift = p * kSortBits;
        const int64_t *moff = (p == passes) ? c->w.moff : nullptr;  // last pass: members
        sort_upsweep_k<<<ntiles, kSortThreads, 0, s>>>(n, kin, iin, shift, moff, M, ntiles, c->w.hist);
        count_launch(c);
        rv_status st = exclusive_scan(c, c->w.hist, (int64_t)kSortBins * ntiles, nullptr, nullptr, s);
        if (st != RV_OK) return st;
        sort_downsweep_k<<<ntiles, kSortThreads, 0, s>>>(n, kin, iin, shift, moff, M, ntiles, c->w.hist, kout,
                                                          iout);
        count_launch(c);
        // next pass reads what this one wrote
        uint64_t *tk = kin; kin = kout; kout = tk;
        int *ti = (iin == nullptr) ? c->w.idx_a : iin;
        iin = iout; iout = ti;
    }
    *keys = kin;
    *idx = iin;
    return cuda_check(c, cudaGetLastError(), "radix sort");
}

// ---------------------------------------------------------------------------
// gather (x, y, z, m) into key order
// ---------------------------------------------------------------------------
__global__ void gather_k(int64_t n, const int *perm, const float4 *xyzm, float4 *pos) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pos[i] = xyzm[perm[i]];
}

// ---------------------------------------------------------------------------
// topology
// ---------------------------------------------------------------------------
__device__ __forceinline__ int diff_level(uint64_t a, uint64_t b) {
    uint64_t d = a ^ b;
    if (d == 0) return kLevels;  // equal keys never separate
    int h = 63 - __clzll((long long)d);
    return (65 - h) / 3;
}

// Window of D values for one block: D(j) for j in [b0 - n_leaf + 1, b0 + NT + n_leaf].
// Out-of-range positions are not boundaries (99); D(0) = D(n) = 0.
// A member's first star is a cut at every level, like position 0.
__device__ void load_window(int64_t n, const uint64_t *key, int64_t b0, int n_leaf, const int64_t *moff, int M,
                            unsigned char *win) {
    int wlen = kTopoBlock + 2 * n_leaf;
    for (int t = threadIdx.x; t < wlen; t += blockDim.x) {
        int64_t j = b0 - n_leaf + 1 + t;
        int d;
        if (j < 0 || j > n) d = 99;
        else if (j == 0 || j == n) d = 0;
        else if (M > 1 && moff[member_of(moff, M, j)] == j) d = 0;
        else d = diff_level(key[j - 1], key[j]);
        win[t] = (unsigned char)d;
    }
}

// lambda_i from the window (i = b0 + threadIdx.x): the smallest level l such
// that positions b1 <= i < b2, b2 - b1 <= n_leaf, are both cuts at l.
__device__ __forceinline__ int leaf_level(const unsigned char *win, int t, int n_leaf) {
    // win index of position j is j - (b0 - n_leaf + 1); i sits at t + n_leaf - 1
    const int wi = t + n_leaf - 1;
    int pm = 99, L = 99;
    for (int s = n_leaf - 1; s >= 0; s--) {
        int u = n_leaf - s;
        pm = min(pm, (int)win[wi + u]);
        L = min(L, max((int)win[wi - s], pm));
    }
    return min(L, kMaxLevel);
}

// Per-level ballots of "a cell starts at star i at level l" (D_i <= l <= lambda_i)
// and their warp prefix counts (shared, [kLevels][NW]).
struct TopoBallots {
    unsigned mask[kLevels];
};

__device__ __forceinline__ void topo_ballots(bool valid, int Di, int lam, TopoBallots &b) {
#pragma unroll
    for (int l = 0; l < kLevels; l++) b.mask[l] = __ballot_sync(0xffffffffu, valid && Di <= l && l <= lam);
}

__global__ void __launch_bounds__(kTopoBlock) topo_count_k(int64_t n, const uint64_t *key, int n_leaf,
                                                           const int64_t *moff, int M, uint8_t *dlev,
                                                           uint8_t *lam_out, int *lvcnt, int nblk) {
    extern __shared__ unsigned char win[];
    __shared__ int wc[kLevels][kTopoBlock / 32];
    int64_t b0 = (int64_t)blockIdx.x * kTopoBlock;
    load_window(n, key, b0, n_leaf, moff, M, win);
    __syncthreads();
    int64_t i = b0 + threadIdx.x;
    bool valid = i < n;
    int Di = 0, lam = -1;
    if (valid) {
        Di = win[threadIdx.x + n_leaf - 1];
        lam = leaf_level(win, threadIdx.x, n_leaf);
        dlev[i] = (uint8_t)Di;
        lam_out[i] = (uint8_t)lam;
    }
    TopoBallots b;
    topo_ballots(valid, Di, lam, b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int l = 0; l < kLevels; l++) wc[l][wid] = __popc(b.mask[l]);
    __syncthreads();
    if (threadIdx.x < kLevels) {
        int s = 0;
        for (int w = 0; w < kTopoBlock / 32; w++) s += wc[threadIdx.x][w];
        lvcnt[(int64_t)threadIdx.x * nblk + blockIdx.x] = s;
    }
}

__device__ __forceinline__ int4 cell_box(uint64_t key, int l) {
    int sh = 3 * (kMaxLevel - l);
    uint64_t pre = (sh >= 64) ? 0ull : ((key >> sh) << sh);
    return make_int4((int)compact3(pre), (int)compact3(pre >> 1), (int)compact3(pre >> 2), l);
}

// Writes every cell's box, first star, child first, parent; and, as the star
// that ends a cell, its end star and child end.
__global__ void __launch_bounds__(kTopoBlock) topo_write_k(int64_t n, const uint64_t *key, const uint8_t *dlev,
                                                           const uint8_t *lamv, const int *lvscan, int nblk,
                                                           int64_t cap, const int64_t *moff, int M, int4 *cbox,
                                                           int *clink, int *cparent, int *carrive, int *mroot,
                                                           DevState *st) {
    __shared__ int wp[kLevels][kTopoBlock / 32];
    __shared__ int lvoff[kLevels + 1];
    __shared__ int bbase[kLevels + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t i = (int64_t)blockIdx.x * kTopoBlock + threadIdx.x;
    bool valid = i < n;
    int Di = valid ? dlev[i] : 0, lam = valid ? lamv[i] : -1;
    TopoBallots b;
    topo_ballots(valid, Di, lam, b);
    if (lane == 0)
        for (int l = 0; l < kLevels; l++) wp[l][wid] = __popc(b.mask[l]);
    if (threadIdx.x <= kLevels) {
        int l = threadIdx.x;
        // level offsets: scanned value at the first block of each level; total at the end
        int tot = st->ncell;
        lvoff[l] = (l < kLevels) ? lvscan[(int64_t)l * nblk] : tot;
        bbase[l] = (l < kLevels) ? lvscan[(int64_t)l * nblk + blockIdx.x] : tot;
    }
    __syncthreads();
    if (threadIdx.x < kLevels) {
        int run = 0;
        for (int w = 0; w < kTopoBlock / 32; w++) {
            int t = wp[threadIdx.x][w];
            wp[threadIdx.x][w] = run;
            run += t;
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x <= kLevels) st->lvoff[threadIdx.x] = lvoff[threadIdx.x];
    if (!valid) return;
    const unsigned lt = lanemask_lt();
    // exclusive global rank of star i among cells of level l
    auto rank = [&](int l) -> int { return bbase[l] + wp[l][wid] + __popc(b.mask[l] & lt); };
    uint64_t k = key[i];
    for (int l = Di; l <= lam; l++) {
        int c = rank(l);
        if (c >= cap) { latch_err(st, kErrCells); return; }
        cbox[c] = cell_box(k, l);
        clink[4 * c + 0] = (l < lam) ? rank(l + 1) : 0;  // first child: cell (l + 1, i)
        if (l == lam) clink[4 * c + 1] = 0;
        clink[4 * c + 2] = (int)i;
        cparent[c] = (l == 0) ? -1 : rank(l - 1) - ((Di == l) ? 1 : 0);
        carrive[c] = 0;
        if (l == 0) mroot[member_of(moff, M, i)] = c;
    }
    // cells containing star i-1 that end at i: levels D(i)..lambda_{i-1}
    if (i > 0) {
        int lp = lamv[i - 1];
        for (int l = Di; l <= lp; l++) {
            int c = rank(l) - 1;
            if (c >= cap) { latch_err(st, kErrCells); return; }
            clink[4 * c + 3] = (int)i;
            if (l < lp) clink[4 * c + 1] = rank(l + 1);
        }
    }
    // the last cell of every level that holds star n-1 ends at n
    if (i == n - 1) {
        for (int l = 0; l <= lam; l++) {
            int c = lvoff[l + 1] - 1;
            if (c >= cap) { latch_err(st, kErrCells); return; }
            clink[4 * c + 3] = (int)n;
            if (l < lam) clink[4 * c + 1] = lvoff[l + 2];
        }
    }
}

// ---------------------------------------------------------------------------
// walk groups
// ---------------------------------------------------------------------------
// A unit is a maximal cell with at most U = 16 G stars (one with <= U stars
// whose parent has more, or a member's root) or a leaf with more than U stars.
// Each unit is cut into runs of G consecutive stars in key order, the last run
// possibly shorter; each run is a group. A group's box is the tightest box on
// the member's integer grid that holds its stars' grid cells: per axis
// [min q, max q + 1), q the star's de-interleaved key. Every star lies in its
// group's box, so a cell the box-box test accepts passes the opening test for
// each star of the group.
// gcnt[c] = groups of cell c (0 unless c is a unit).
__global__ void groups_count_k(const int4 *cbox, const int4 *clink, const int *cparent, int G, int U, int64_t cap,
                               const DevState *st, int *gcnt) {
    const int ncell = (int)min((int64_t)st->ncell, cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const int4 lk = clink[c];
        const int cnt = lk.w - lk.z;
        bool unit;
        if (cnt > U) {
            unit = (lk.x == lk.y);   // an overfull leaf
        } else if (cbox[c].w == 0) {
            unit = true;             // a member's root
        } else {
            const int p = cparent[c];
            unit = false;
            if (p >= 0 && p < ncell) {
                const int4 pl = clink[p];
                unit = (pl.w - pl.z) > U;
            }
        }
        gcnt[c] = unit ? (cnt + G - 1) / G : 0;
    }
}

// One warp per unit cell: writes its runs with their boxes from the scanned
// offsets gofs (exclusive prefix of gcnt).
__global__ void groups_write_k(const uint64_t *skey, const int4 *clink, const int *gofs, const int *gcnt_total,
                               int G, int64_t cap, const DevState *st, int4 *groups) {
    const int lane = threadIdx.x & 31;
    const int ncell = (int)min((int64_t)st->ncell, cap);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < ncell; c += nw) {
        const int g0 = gofs[c];
        const int g1 = (c + 1 < ncell) ? gofs[c + 1] : *gcnt_total;
        if (g1 <= g0) continue;
        const int4 lk = clink[c];
        for (int r = 0; r < g1 - g0; r++) {
            const int first = lk.z + r * G;
            const int cnt = min(G, lk.w - first);
            unsigned qlo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, qhi[3] = {0u, 0u, 0u};
            for (int i = lane; i < cnt; i += 32) {   // a run may hold up to 64 stars
                const uint64_t key = skey[first + i];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const unsigned q = compact3(key >> a);
                    qlo[a] = min(qlo[a], q);
                    qhi[a] = max(qhi[a], q + 1);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; a++)
                for (int o = 16; o > 0; o >>= 1) {
                    qlo[a] = min(qlo[a], __shfl_xor_sync(0xffffffffu, qlo[a], o));
                    qhi[a] = max(qhi[a], __shfl_xor_sync(0xffffffffu, qhi[a], o));
                }
            if (lane == 0) {
                const int g = g0 + r;
                groups[2 * g] = make_int4(first, cnt, (int)qlo[0], (int)qlo[1]);
                groups[2 * g + 1] = make_int4((int)qlo[2], (int)qhi[0], (int)qhi[1], (int)qhi[2]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// multipoles, bottom-up: each leaf computes its moments from its stars; the
// last child to finish a parent (atomic arrival count) computes the parent
// from its children in child order, so the result does not depend on timing.
// FP32, accumulated relative to the cell's geometric centre.
// ---------------------------------------------------------------------------
// Moments are stored relative to the cell's geometric centre c0 (geo_centre):
// (M, com - c0), (Qxx, Qyy, Qzz, Qxy), (Qxz, Qyz, 0, 0).
struct Mom {
    float M, cx, cy, cz, q[6];  // cx..cz: centre of mass minus c0; q: xx, yy, zz, xy, xz, yz
};

__device__ __forceinline__ void store_mom(float4 *cmom, int c, const Mom &m) {
    cmom[3 * c + 0] = make_float4(m.M, m.cx, m.cy, m.cz);
    cmom[3 * c + 1] = make_float4(m.q[0], m.q[1], m.q[2], m.q[3]);
    cmom[3 * c + 2] = make_float4(m.q[4], m.q[5], 0.f, 0.f);
}



__device__ __forceinline__ void add_q(float q[6], float m, float dx, float dy, float dz) {
    float d2 = dx * dx + dy * dy + dz * dz;
    q[0] += m * (3.f * dx * dx - d2);
    q[1] += m * (3.f * dy * dy - d2);
    q[2] += m * (3.f * dz * dz - d2);
    q[3] += m * 3.f * dx * dy;
    q[4] += m * 3.f * dx * dz;
    q[5] += m * 3.f * dy * dz;
}

__global__ void moments_k(int64_t n, const float4 *pos, const int4 *cbox, const int *clink, const int *cparent,
                          int *carrive, float4 *cmom, int64_t cap, const int64_t *moff, int M,
                          const double *mbounds, DevState *st) {
    int ncell = (int)min((int64_t)st->ncell, cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        int4 lk = reinterpret_cast<const int4 *>(clink)[c];
        if (lk.y != lk.x) continue;  // not a leaf
        if (lk.z < 0 || lk.w > n || lk.z >= lk.w) { latch_err(st, kErrCells); continue; }
        const int mb = member_of(moff, M, lk.z);
        const float lo[3] = {(float)mbounds[5 * mb], (float)mbounds[5 * mb + 1], (float)mbounds[5 * mb + 2]};
        const float unit = (float)(mbounds[5 * mb + 3] / 2097152.0);
        float g[3];
        geo_centre(cbox[c], lo, unit, g);
        Mom m = {};
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int j = lk.z; j < lk.w; j++) {
            float4 p = pos[j];
            m.M += p.w;
            sx += p.w * (p.x - g[0]);
            sy += p.w * (p.y - g[1]);
            sz += p.w * (p.z - g[2]);
        }
        if (m.M > 0.f) {
            m.cx = sx / m.M; m.cy = sy / m.M; m.cz = sz / m.M;
            for (int j = lk.z; j < lk.w; j++) {
                float4 p = pos[j];
                add_q(m.q, p.w, (p.x - g[0]) - m.cx, (p.y - g[1]) - m.cy, (p.z - g[2]) - m.cz);
            }
        }
        store_mom(cmom, c, m);
        // climb while this thread is the last child to arrive (at most 21 levels)
        int cur = c;
        for (int guard = 0; guard <= kMaxLevel; guard++) {
            int p = cparent[cur];
            if (p < 0) break;
            if (p >= cur) { latch_err(st, kErrCells); break; }  // parents precede children
            __threadfence();
            int4 pl = reinterpret_cast<const int4 *>(clink)[p];
            int nch = pl.y - pl.x;
            if (pl.x <= p || pl.y > ncell || nch < 1 || nch > 8) { latch_err(st, kErrCells); break; }
            if (atomicAdd(&carrive[p], 1) != nch - 1) break;
            __threadfence();
            float pg[3];
            geo_centre(cbox[p], lo, unit, pg);
            Mom P = {};
            float px = 0.f, py = 0.f, pz = 0.f;
            for (int ch = pl.x; ch < pl.y; ch++) {
                float4 a = __ldcg(&cmom[3 * ch]);
                float cg[3];
                geo_centre(cbox[ch], lo, unit, cg);
                P.M += a.x;
                px += a.x * ((cg[0] - pg[0]) + a.y);
                py += a.x * ((cg[1] - pg[1]) + a.z);
                pz += a.x * ((cg[2] - pg[2]) + a.w);
            }
            if (P.M > 0.f) {
                P.cx = px / P.M; P.cy = py / P.M; P.cz = pz / P.M;
                for (int ch = pl.x; ch < pl.y; ch++) {
                    float4 a = __ldcg(&cmom[3 * ch]);
                    float4 b = __ldcg(&cmom[3 * ch + 1]);
                    float4 e = __ldcg(&cmom[3 * ch + 2]);
                    float cg[3];
                    geo_centre(cbox[ch], lo, unit, cg);
                    P.q[0] += b.x; P.q[1] += b.y; P.q[2] += b.z; P.q[3] += b.w; P.q[4] += e.x; P.q[5] += e.y;
                    add_q(P.q, a.x, ((cg[0] - pg[0]) + a.y) - P.cx, ((cg[1] - pg[1]) + a.z) - P.cy,
                          ((cg[2] - pg[2]) + a.w) - P.cz);
                }
            }
            store_mom(cmom, p, P);
            cur = p;
        }
    }
}

// ---------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------
static int grid_for(rv_ctx *c, int64_t n, int per_block) {
    int64_t b = (n + per_block - 1) / per_block;
    int64_t cap = (int64_t)c->num_sms * 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

// Copies the member offsets to the device only when they differ from the
// last ones sent (a captured step must not copy from host memory).
rv_status upload_offsets(rv_ctx *c, int M, const int64_t *offsets, cudaStream_t s) {
    bool same = c->moff_on_device && c->n_members == M;
    for (int k = 0; k <= M && same; k++) same = (c->moff_host[k] == offsets[k]);
    if (same) return RV_OK;
    for (int k = 0; k <= M; k++) c->moff_host[k] = offsets[k];
    c->n_members = M;
    rv_status r = cuda_check(c, cudaMemcpyAsync(c->w.moff, c->moff_host, sizeof(int64_t) * (M + 1),
                                                cudaMemcpyHostToDevice, s), "member offsets");
    if (r == RV_OK) r = cuda_check(c, cudaStreamSynchronize(s), "member offsets");
    if (r == RV_OK) c->moff_on_device = true;
    return r;
}

// Members are independent systems stored one after another (offsets on the
// host, M >= 1). Each gets its own bounding cube, keys, tree and groups; all
// of them share these launches, and the walk serves them together.
rv_status build_tree(rv_ctx *c, int n_members, const int64_t *offsets, const float *x, const float *y,
                     const float *z, const float *m, cudaStream_t s) {
    Workspace &w = c->w;
    const int M = n_members;
    const int64_t n = offsets[M];
    c->n = n;
    c->built = false;
    int64_t big = 0;
    for (int k = 0; k < M; k++) big = std::max<int64_t>(big, offsets[k + 1] - offsets[k]);
    c->max_member = big;
    rv_status r = upload_offsets(c, M, offsets, s);
    if (r != RV_OK) return r;
    if (n == 0) {
        r = cuda_check(c, cudaMemsetAsync(w.st, 0, sizeof(DevState), s), "state reset");
        if (r == RV_OK) c->built = true;
        return r;
    }
    if ((r = cuda_check(c, cudaMemsetAsync(w.mroot, 0xff, sizeof(int) * M, s), "roots")) != RV_OK) return r;
    // bounds and keys: blocks per member sized by the largest member
    const int bpm = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(big, kBoundsChunk), 512 / M + 1));
    bounds_partial_k<<<dim3(bpm, M), 256, 0, s>>>(w.moff, bpm, x, y, z, w.bpart);
    count_launch(c);
    bounds_final_k<<<M, 32, 0, s>>>(bpm, w.bpart, w.mbounds, w.st);
    count_launch(c);
    const int kpm = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(big, 256), (int64_t)c->num_sms * 8 / M + 1));
    // the packed stars live in the group records' space until the gather: the
    // groups are written after it (32 B per star of room there, 16 needed)
    float4 *xyzm = reinterpret_cast<float4 *>(w.groups);
    keys_k<<<dim3(kpm, M), 256, 0, s>>>(w.moff, kpm, x, y, z, m, w.mbounds, w.key_a, xyzm);
    count_launch(c);
    uint64_t *skey;
    int *perm;
    if ((r = radix_sort(c, n, 7, &skey, &perm, true, s, true)) != RV_OK) return r;
    w.skey = skey;
    w.perm = perm;
    gather_k<<<grid_for(c, n, 256), 256, 0, s>>>(n, perm, xyzm, w.pos);
    count_launch(c);
    // topology
    int nblk = ceil_div(n, kTopoBlock);
    size_t win = kTopoBlock + 2 * c->cfg.n_leaf;
    topo_count_k<<<nblk, kTopoBlock, win, s>>>(n, skey, c->cfg.n_leaf, w.moff, M, w.dlev, w.lam, w.lvcnt, nblk);
    count_launch(c);
    if ((r = exclusive_scan(c, w.lvcnt, (int64_t)kLevels * nblk, nullptr, &w.st->ncell, s)) != RV_OK) return r;
    topo_write_k<<<nblk, kTopoBlock, 0, s>>>(n, skey, w.dlev, w.lam, w.lvcnt, nblk, c->cell_cap, w.moff, M, w.cbox,
                                             w.clink, w.cparent, w.carrive, w.mroot, w.st);
    count_launch(c);
    // groups
    const int G = c->cfg.group, U = 16 * c->cfg.group;
    const int4 *clink4 = reinterpret_cast<const int4 *>(w.clink);
    int gb = grid_for(c, c->cell_cap, 256);
    groups_count_k<<<gb, 256, 0, s>>>(w.cbox, clink4, w.cparent, G, U, c->cell_cap, w.st, w.gcnt);
    count_launch(c);
    if ((r = exclusive_scan(c, w.gcnt, c->cell_cap, &w.st->ncell, &w.st->ngroup, s)) != RV_OK) return r;
    groups_write_k<<<grid_for(c, c->cell_cap, 8), 256, 0, s>>>(skey, clink4, w.gcnt, &w.st->ngroup, G, c->cell_cap,
                                                                w.st, w.groups);
    count_launch(c);
    // multipoles
    moments_k<<<gb, 128, 0, s>>>(n, w.pos, w.cbox, w.clink, w.cparent, w.carrive, w.cmom, c->cell_cap, w.moff, M,
                                 w.mbounds, w.st);
    count_launch(c);
    r = cuda_check(c, cudaGetLastError(), "build_tree");
    if (r == RV_OK) c->built = true;
    return r;
}

}  // namespace rv
