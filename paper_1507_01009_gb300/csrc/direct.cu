// direct.cu -- FP64 direct summation on the GPU for a sample of targets: the
// reference the tree's force error is measured against (the accuracy criterion
// of Sect. 3/4 compares tree forces with direct summation).
//
//   a_i   =  sum_{j != i} m_j d / (d.d + e_ij^2)^{3/2}
//   phi_i = -sum_{j != i} m_j / (d.d + e_ij^2)^{1/2},   d = x_j - x_i,  G = 1,
//
// Plummer softening (Sect. 3) with the pair length e_ij = max(e_i, e_j), none
// if either is 0 (an unsoftened body such as an SMBH); a pair with
// d.d + e_ij^2 = 0 (coincident unsoftened bodies) adds nothing.
//
// Targets are spread over blocks of 128 threads (one target a thread) and the
// sources over up to 128 chunks (grid y), each staged through shared memory in
// tiles of 128; a second kernel adds the chunks' partial sums in chunk order,
// so the result does not depend on scheduling. Sums are plain FP64.
#include <algorithm>

#include "rv_internal.cuh"

namespace rv {

constexpr int kDirTile = 128;         // targets per block, sources per shared-memory tile
constexpr int kDirMaxChunks = 128;    // source chunks, i.e. partial sums per target

__global__ void __launch_bounds__(kDirTile) direct_fp64_k(int64_t n, const double *x, const double *y,
                                                          const double *z, const double *m, const double *eps,
                                                          int64_t nt, const int64_t *tidx, int64_t chunk,
                                                          double *part) {
    __shared__ double sx[kDirTile], sy[kDirTile], sz[kDirTile], sm[kDirTile], se[kDirTile];
    const int64_t t = (int64_t)blockIdx.x * kDirTile + threadIdx.x;
    const int c = blockIdx.y;
    const int64_t j0 = (int64_t)c * chunk, j1 = (j0 + chunk < n) ? j0 + chunk : n;
    int64_t i = -1;
    bool bad = false;
    double xi = 0.0, yi = 0.0, zi = 0.0, ei = 0.0;
    if (t < nt) {
        i = tidx[t];
        bad = i < 0 || i >= n;   // an index outside the bodies: NaN results, no read
        if (!bad) {
            xi = x[i]; yi = y[i]; zi = z[i]; ei = eps[i];
        }
    }
    double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
    for (int64_t b = j0; b < j1; b += kDirTile) {
        const int64_t j = b + threadIdx.x;
        __syncthreads();
        if (j < j1) {
            sx[threadIdx.x] = x[j]; sy[threadIdx.x] = y[j]; sz[threadIdx.x] = z[j];
            sm[threadIdx.x] = m[j]; se[threadIdx.x] = eps[j];
        }
        __syncthreads();
        const int cnt = (j1 - b < kDirTile) ? (int)(j1 - b) : kDirTile;
        if (t < nt && !bad) {
            for (int k = 0; k < cnt; k++) {
                if (b + k == i) continue;
                const double ej = se[k];
                const double e = (ei == 0.0 || ej == 0.0) ? 0.0 : fmax(ei, ej);
                const double dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
                const double r2 = dx * dx + dy * dy + dz * dz + e * e;
                if (!(r2 > 0.0)) continue;
                const double rinv = rsqrt(r2);
                const double mr = sm[k] * rinv;
                const double mr3 = mr * rinv * rinv;
                ax += mr3 * dx;
                ay += mr3 * dy;
                az += mr3 * dz;
                ph -= mr;
            }
        }
    }
    if (t < nt) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        double *p = part + (size_t)c * 4 * nt;
        p[t] = bad ? nan : ax;
        p[nt + t] = bad ? nan : ay;
        p[2 * nt + t] = bad ? nan : az;
        p[3 * nt + t] = bad ? nan : ph;
    }
}

__global__ void direct_reduce_k(int64_t nt, int nchunk, const double *part, double *ax, double *ay, double *az,
                                double *pot) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < nchunk; c++)
            for (int q = 0; q < 4; q++) s[q] += part[((size_t)c * 4 + q) * nt + t];
        ax[t] = s[0];
        ay[t] = s[1];
        az[t] = s[2];
        pot[t] = s[3];
    }
}

}  // namespace rv

using namespace rv;

extern "C" {

size_t rv_direct_fp64_scratch_bytes(int64_t nt) {
    return nt <= 0 ? 0 : sizeof(double) * 4 * (size_t)kDirMaxChunks * (size_t)nt;
}

rv_status rv_direct_fp64(int64_t n, const double *x, const double *y, const double *z, const double *m,
                         const double *eps, int64_t nt, const int64_t *targets, double *ax, double *ay, double *az,
                         double *pot, void *scratch, size_t scratch_bytes, void *stream) {
    NvtxRange nvtx_range("rv_direct_fp64");
    if (n < 1 || nt < 0 || !x || !y || !z || !m || !eps) return RV_E_INVAL;
    if (nt == 0) return RV_OK;
    if (!targets || !ax || !ay || !az || !pot || !scratch) return RV_E_INVAL;
    if (scratch_bytes < rv_direct_fp64_scratch_bytes(nt)) return RV_E_WORKSPACE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RV_E_CUDA;
    const int64_t tblk = (nt + kDirTile - 1) / kDirTile;
    if (tblk > 0x7fffffffll) return RV_E_INVAL;
    // enough blocks to fill the GPU (about 8 per SM), chunks of at least one tile
    int64_t nchunk = std::max<int64_t>(1, ((int64_t)sms * 8 + tblk - 1) / tblk);
    nchunk = std::min<int64_t>({nchunk, (int64_t)kDirMaxChunks, (n + kDirTile - 1) / kDirTile});
    const int64_t chunk = (n + nchunk - 1) / nchunk;
    cudaStream_t s = (cudaStream_t)stream;
    double *part = reinterpret_cast<double *>(scratch);
    direct_fp64_k<<<dim3((unsigned)tblk, (unsigned)nchunk), kDirTile, 0, s>>>(n, x, y, z, m, eps, nt, targets, chunk,
                                                                              part);
    const int rgrid = (int)std::max<int64_t>(1, std::min<int64_t>((nt + 255) / 256, (int64_t)sms * 4));
    direct_reduce_k<<<rgrid, 256, 0, s>>>(nt, (int)nchunk, part, ax, ay, az, pot);
    return cudaGetLastError() == cudaSuccess ? RV_OK : RV_E_CUDA;
}

}  // extern "C"
