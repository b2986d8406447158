// chain.cu -- the regularised chain's coupling to the tree (Sect. 2), the
// kick-drift-kick step and the FP64 energy/momentum totals.
//
// The chain (an SMBH, or an SMBH pair with the stars absorbed into it) is
// seen by the tree as one unsoftened particle at its centre of mass. Stars
// near it ("perturbers") get the pull of the resolved members instead of the
// centre-of-mass point mass; each member feels the perturbers directly; the
// centre-of-mass force is corrected by Eq. 3. All of this is unsoftened FP64;
// sums run in a fixed order so results do not depend on scheduling.
#include <algorithm>

#include "rv_internal.cuh"

namespace rv {

// ---------------------------------------------------------------------------
// perturber selection
// ---------------------------------------------------------------------------
// FP32 squared distance, every operation rounded separately in this order.
__device__ __forceinline__ float dist2_f32(float x, float y, float z, float cx, float cy, float cz) {
    float dx = __fsub_rn(x, cx), dy = __fsub_rn(y, cy), dz = __fsub_rn(z, cz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ float3 centre_of(const float *cdev, float3 chost) {
    return cdev ? make_float3(cdev[0], cdev[1], cdev[2]) : chost;
}

// Membership test of a sphere-like selection around a chain centre:
//   mode 1 (radius): d2 < r2 (FP32);
//   mode 3 (tidal criterion of Eq. 2): r < (2 m_j / (gamma M))^(1/3) r_crit,
//   taken without a cube root in FP64, one rounding per operation:
//   (d2 d2) d2 < (q q) rc6, q = (2 m_j) / (gamma M), rc6 = (rc2 rc2) rc2.
// M is the chain's FP32 total mass (the 4th value of its centre record).
struct SelRule {
    int mode;
    float r2;         // mode 1
    const float *m;   // mode 3: star masses
    float gamma;      // mode 3
    double rc6;       // mode 3
};

__device__ __forceinline__ bool sel_inside(const SelRule &R, float d2, int64_t i, float mchain) {
    if (R.mode != 3) return d2 < R.r2;
    const double dd = (double)d2;
    const double q = __ddiv_rn(__dmul_rn(2.0, (double)R.m[i]), __dmul_rn((double)R.gamma, (double)mchain));
    return __dmul_rn(__dmul_rn(dd, dd), dd) < __dmul_rn(__dmul_rn(q, q), R.rc6);
}

static SelRule sel_rule(int mode, float radius, const float *m, float gamma) {
    SelRule R;
    R.mode = mode;
    R.r2 = radius * radius;   // one FP32 product
    R.m = m;
    R.gamma = gamma;
    const double rc2 = (double)radius * (double)radius;
    R.rc6 = (rc2 * rc2) * rc2;
    return R;
}

__global__ void sel_radius_flag_k(int64_t n, const float *x, const float *y, const float *z, const float *cdev,
                                  float4 chost, SelRule R, int *flag) {
    const float3 c = centre_of(cdev, make_float3(chost.x, chost.y, chost.z));
    const float mc = cdev ? cdev[3] : chost.w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = sel_inside(R, dist2_f32(x[i], y[i], z[i], c.x, c.y, c.z), i, mc) ? 1 : 0;
}

__global__ void sel_radius_write_k(int64_t n, const float *x, const float *y, const float *z, const float *cdev,
                                   float4 chost, SelRule R, const int *ofs, const int *total, int cap, int *idx,
                                   int *count, DevState *st) {
    const float3 c = centre_of(cdev, make_float3(chost.x, chost.y, chost.z));
    const float mc = cdev ? cdev[3] : chost.w;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (sel_inside(R, dist2_f32(x[i], y[i], z[i], c.x, c.y, c.z), i, mc)) {
            int p = ofs[i];
            if (p < cap) idx[p] = (int)i;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int t = *total;
        *count = min(t, cap);
        st->n_pert = min(t, cap);
        if (t > cap) latch_err(st, kErrPert);
    }
}

// key = bits of the (non-negative) FP32 squared distance: integer order = float order
__global__ void sel_knn_keys_k(int64_t n, const float *x, const float *y, const float *z, const float *cdev,
                               float3 chost, uint64_t *key) {
    float3 c = centre_of(cdev, chost);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = (uint64_t)__float_as_uint(dist2_f32(x[i], y[i], z[i], c.x, c.y, c.z));
}

__global__ void sel_knn_write_k(const int *sorted_idx, int64_t n, int k, int *idx, int *count, DevState *st) {
    int kk = (int)min((int64_t)k, n);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kk; p += gridDim.x * blockDim.x) idx[p] = sorted_idx[p];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *count = kk;
        st->n_pert = kk;
    }
}

// Eq. 1 ingredients from the stars sorted by FP32 squared distance (keys =
// the d2 bits, ties by index): r(<2 M_bh), sigma of the k nearest, M_bh / sigma^2.
// One thread, sums in distance order in FP64, exactly as the rule reads.
__global__ void influence_k(int64_t n, const uint64_t *skey, const int *sidx, const float *vx, const float *vy,
                            const float *vz, const float *m, double m_bh, int64_t k, double *out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double cum = 0.0, r2m = __longlong_as_double(0x7ff0000000000000ll);
    for (int64_t i = 0; i < n; i++) {
        cum = __dadd_rn(cum, (double)m[sidx[i]]);
        if (cum >= 2.0 * m_bh) {
            r2m = __dsqrt_rn((double)__uint_as_float((unsigned)skey[i]));
            break;
        }
    }
    double mx = 0.0, my = 0.0, mz = 0.0;
    for (int64_t i = 0; i < k; i++) {
        const int j = sidx[i];
        mx = __dadd_rn(mx, (double)vx[j]); my = __dadd_rn(my, (double)vy[j]); mz = __dadd_rn(mz, (double)vz[j]);
    }
    mx = __ddiv_rn(mx, (double)k); my = __ddiv_rn(my, (double)k); mz = __ddiv_rn(mz, (double)k);
    double s = 0.0;
    for (int64_t i = 0; i < k; i++) {
        const int j = sidx[i];
        const double dx = __dsub_rn((double)vx[j], mx), dy = __dsub_rn((double)vy[j], my),
                     dz = __dsub_rn((double)vz[j], mz);
        s = __dadd_rn(s, __dmul_rn(dx, dx));
        s = __dadd_rn(s, __dmul_rn(dy, dy));
        s = __dadd_rn(s, __dmul_rn(dz, dz));
    }
    const double s2 = __ddiv_rn(s, __dmul_rn(3.0, (double)k));
    out[0] = r2m;
    out[1] = __dsqrt_rn(s2);
    out[2] = __ddiv_rn(m_bh, s2);
}

static int grid_n(rv_ctx *c, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8));
}

rv_status select_perturbers(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z,
                            const float *centre_dev, const float *centre_host, int mode, float radius, int k,
                            int cap, int *idx, int *count, cudaStream_t s, const float *m, float gamma) {
    // centre_host: (x, y, z, chain mass) -- the mass is read by the tidal rule only
    float4 ch = centre_host ? make_float4(centre_host[0], centre_host[1], centre_host[2], centre_host[3])
                            : make_float4(0, 0, 0, 0);
    Workspace &w = c->w;
    if (mode == 1 || mode == 3) {
        const SelRule R = sel_rule(mode, radius, m, gamma);
        if (n == 0) return cuda_check(c, cudaMemsetAsync(count, 0, sizeof(int), s), "select");
        sel_radius_flag_k<<<grid_n(c, n), 256, 0, s>>>(n, x, y, z, centre_dev, ch, R, w.sel_flag);
        count_launch(c);
        int *total = &w.st->n_pert;  // scratch for the total; overwritten by the clamped count
        rv_status r = exclusive_scan(c, w.sel_flag, n, nullptr, total, s);
        if (r != RV_OK) return r;
        sel_radius_write_k<<<grid_n(c, n), 256, 0, s>>>(n, x, y, z, centre_dev, ch, R, w.sel_flag, total, cap, idx,
                                                        count, w.st);
        count_launch(c);
    } else {
        if (n == 0 || k <= 0) {
            cudaMemsetAsync(&w.st->n_pert, 0, sizeof(int), s);
            return cuda_check(c, cudaMemsetAsync(count, 0, sizeof(int), s), "select");
        }
        // the sort buffers are shared with the tree build: the tree is invalid afterwards
        c->built = false;
        sel_knn_keys_k<<<grid_n(c, n), 256, 0, s>>>(n, x, y, z, centre_dev, make_float3(ch.x, ch.y, ch.z), w.key_a);
        count_launch(c);
        uint64_t *sk;
        int *si;
        rv_status r = radix_sort(c, n, 4, &sk, &si, true, s);
        if (r != RV_OK) return r;
        sel_knn_write_k<<<ceil_div(std::min<int64_t>(k, n), 256), 256, 0, s>>>(si, n, std::min(k, cap), idx, count, w.st);
        count_launch(c);
    }
    return cuda_check(c, cudaGetLastError(), "select perturbers");
}

rv_status influence_radius(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z, const float *vx,
                           const float *vy, const float *vz, const float *m, const float centre[3], double m_bh,
                           int64_t n_sigma, double out[3], cudaStream_t s) {
    Workspace &w = c->w;
    c->built = false;   // the sort buffers are shared with the tree build
    sel_knn_keys_k<<<grid_n(c, n), 256, 0, s>>>(n, x, y, z, nullptr, make_float3(centre[0], centre[1], centre[2]),
                                                w.key_a);
    count_launch(c);
    uint64_t *sk;
    int *si;
    rv_status r = radix_sort(c, n, 4, &sk, &si, true, s);
    if (r != RV_OK) return r;
    influence_k<<<1, 32, 0, s>>>(n, sk, si, vx, vy, vz, m, m_bh, std::min<int64_t>(n_sigma, n), w.out8);
    count_launch(c);
    r = cuda_check(c, cudaMemcpyAsync(out, w.out8, 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "influence");
    if (r == RV_OK) r = cuda_check(c, cudaStreamSynchronize(s), "influence");
    return r;
}

// ---------------------------------------------------------------------------
// perturber selection per member (systems of several members): one stable
// sort of (member, key) over all stars; member m's stars occupy the same
// slots [moff[m], moff[m+1]) in sorted order, best first.
//   k nearest: key = FP32 squared distance bits to the member's centre
//   radius:    key = 0 inside, 1 outside (inside stars first, ascending index)
// ---------------------------------------------------------------------------
__global__ void sel_member_keys_k(const int64_t *moff, int bpm, const float *x, const float *y, const float *z,
                                  const float *xyzm, int C, int j, SelRule R, uint64_t *key) {
    const int m = blockIdx.y;
    const float *q = xyzm + 4 * ((int64_t)m * C + j);   // chain j of member m
    const float cx = q[0], cy = q[1], cz = q[2], mc = q[3];
    for (int64_t i = moff[m] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < moff[m + 1];
         i += (int64_t)bpm * blockDim.x) {
        float d2 = dist2_f32(x[i], y[i], z[i], cx, cy, cz);
        key[i] = (R.mode == 2) ? (uint64_t)__float_as_uint(d2) : (sel_inside(R, d2, i, mc) ? 0ull : 1ull);
    }
}

// member m: its first min(k, n_m) sorted slots (k nearest), or its leading
// "inside" slots (radius), written to idx[m cap ..], count to npert[m]
__global__ void sel_member_write_k(const int64_t *moff, const uint64_t *skey, const int *sidx, int mode, int k,
                                   int cap, int C, int j, int *idx, int *npert, DevState *st) {
    const int m = blockIdx.x;
    const int64_t s = moff[m], e = moff[m + 1];
    int cnt;
    if (mode == 2) {
        cnt = (int)min((int64_t)k, e - s);
    } else {
        // first "outside" key in the member's slots
        int64_t lo = s, hi = e;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (skey[mid] == 0ull) lo = mid + 1; else hi = mid;
        }
        cnt = (int)(lo - s);
    }
    if (cnt > cap && threadIdx.x == 0) latch_err(st, kErrPert);
    cnt = min(cnt, cap);
    const int64_t ch = (int64_t)m * C + j;   // chain j of member m
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) idx[ch * cap + p] = sidx[s + p];
    if (threadIdx.x == 0) npert[ch] = cnt;
}

static int member_cap(int M) { return std::min(kMaxPert, kPertTotal / std::max(1, M)); }

// ---------------------------------------------------------------------------
// FP64 chain / perturber coupling, one chain per member
// ---------------------------------------------------------------------------
// f = m r / |r|^3 and -m/|r| for r = to - from (zero separation: nothing).
__device__ __forceinline__ void kep(double rx, double ry, double rz, double m, double &ax, double &ay, double &az,
                                    double &p) {
    double r2 = rx * rx + ry * ry + rz * rz;
    if (r2 <= 0.0) return;
    double rinv = 1.0 / sqrt(r2);
    double s = m * rinv * rinv * rinv;
    ax += s * rx; ay += s * ry; az += s * rz;
    p -= m * rinv;
}

// Per member m (out8 + 16 m): [0..3) corr (Eq. 3), [3..6) sub, [6] sum_k m_k
// pot_chain[k] / M, [7] sub potential, [8..11) centre of mass, [11] M.
// With xyzm, the centre of mass also becomes member m's extra particle m
// (FP32, unsoftened). With xq, the chain's traceless quadrupole about its
// centre of mass, Q_ab = sum_k m_k (3 d_a d_b - |d|^2 delta_ab), d = x_k - c
// (the expansion of Sect. 1 applied to the chain), computed in FP64, goes
// rounded to FP32 to xq[2 m] = (xx, yy, zz, xy), xq[2 m + 1] = (xz, yz, 0, 0)
// for the walk.
__global__ void chain_com_k(int M, int n_ch, const double *cm, const double *cx, double *out8, float *xyzm,
                            float *xeps, float4 *xq = nullptr) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const double *mm = cm + (int64_t)m * n_ch, *xx = cx + 3 * (int64_t)m * n_ch;
        double Mt = 0, c[3] = {0, 0, 0};
        for (int k = 0; k < n_ch; k++) {
            Mt += mm[k];
            for (int a = 0; a < 3; a++) c[a] += mm[k] * xx[3 * k + a];
        }
        for (int a = 0; a < 3; a++) c[a] = (Mt > 0) ? c[a] / Mt : 0.0;
        double *o = out8 + 16 * (int64_t)m;
        o[8] = c[0]; o[9] = c[1]; o[10] = c[2]; o[11] = Mt;
        if (xyzm) {
            xyzm[4 * m] = (float)c[0]; xyzm[4 * m + 1] = (float)c[1]; xyzm[4 * m + 2] = (float)c[2];
            xyzm[4 * m + 3] = (float)Mt;
            xeps[m] = 0.f;
        }
        if (xq) {
            double q[6] = {0, 0, 0, 0, 0, 0};
            for (int k = 0; k < n_ch; k++) {
                const double d0 = xx[3 * k] - c[0], d1 = xx[3 * k + 1] - c[1], d2 = xx[3 * k + 2] - c[2];
                const double dd = d0 * d0 + d1 * d1 + d2 * d2;
                q[0] += mm[k] * (3.0 * d0 * d0 - dd);
                q[1] += mm[k] * (3.0 * d1 * d1 - dd);
                q[2] += mm[k] * (3.0 * d2 * d2 - dd);
                q[3] += mm[k] * 3.0 * d0 * d1;
                q[4] += mm[k] * 3.0 * d0 * d2;
                q[5] += mm[k] * 3.0 * d1 * d2;
            }
            xq[2 * m] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
            xq[2 * m + 1] = make_float4((float)q[4], (float)q[5], 0.f, 0.f);
        }
    }
}

// Member addressing shared by the coupling kernels (blockIdx.y = member).
struct ChainView {
    int n_ch;            // members of each chain
    int cap;             // perturber slots per member
    const double *cm, *cx;
    const int *npert;    // perturbers per member (nullptr: cap)
    const double *pm, *px;
};

__device__ __forceinline__ int npert_of(const ChainView &V, int m) { return V.npert ? min(V.npert[m], V.cap) : V.cap; }

// perturbers: resolved members minus the centre-of-mass point mass (the walk
// gives perturbers the point mass only, never the chain's quadrupole)
__global__ void pert_on_stars_k(ChainView V, const double *out8, double *a_pert, double *pot_pert) {
    const int m = blockIdx.y;
    const int np = npert_of(V, m);
    const double *cm = V.cm + (int64_t)m * V.n_ch, *cx = V.cx + 3 * (int64_t)m * V.n_ch;
    const double *o = out8 + 16 * (int64_t)m;
    const double M = o[11];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)m * V.cap + p;
        double x = V.px[3 * q], y = V.px[3 * q + 1], z = V.px[3 * q + 2];
        double ax = 0, ay = 0, az = 0, ph = 0;
        for (int k = 0; k < V.n_ch; k++) kep(cx[3 * k] - x, cx[3 * k + 1] - y, cx[3 * k + 2] - z, cm[k], ax, ay, az, ph);
        double bx = 0, by = 0, bz = 0, bp = 0;
        kep(o[8] - x, o[9] - y, o[10] - z, M, bx, by, bz, bp);
        a_pert[3 * q] = ax - bx; a_pert[3 * q + 1] = ay - by; a_pert[3 * q + 2] = az - bz;
        pot_pert[q] = ph - bp;
    }
}

template <int NT>
__device__ void block_sum4(double v[4], double (*sm)[NT]) {
    for (int a = 0; a < 4; a++) sm[a][threadIdx.x] = v[a];
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int a = 0; a < 4; a++) sm[a][threadIdx.x] += sm[a][threadIdx.x + o];
        __syncthreads();
    }
    for (int a = 0; a < 4; a++) v[a] = sm[a][0];
    __syncthreads();
}

// block (k, m): perturbers of member m on its chain member k (fixed order)
__global__ void __launch_bounds__(256) pert_on_members_k(ChainView V, double *a_chain, double *pot_chain) {
    __shared__ double sm[4][256];
    const int k = blockIdx.x, m = blockIdx.y;
    const int np = npert_of(V, m);
    const int64_t kk = (int64_t)m * V.n_ch + k;
    double x = V.cx[3 * kk], y = V.cx[3 * kk + 1], z = V.cx[3 * kk + 2];
    double v[4] = {0, 0, 0, 0};
    for (int p = threadIdx.x; p < np; p += 256) {
        const int64_t q = (int64_t)m * V.cap + p;
        kep(V.px[3 * q] - x, V.px[3 * q + 1] - y, V.px[3 * q + 2] - z, V.pm[q], v[0], v[1], v[2], v[3]);
    }
    block_sum4<256>(v, sm);
    if (threadIdx.x == 0) {
        a_chain[3 * kk] = v[0]; a_chain[3 * kk + 1] = v[1]; a_chain[3 * kk + 2] = v[2];
        pot_chain[kk] = v[3];
    }
}

// block m: Eq. 3 correction, and the perturbers' direct terms on the centre of mass
__global__ void __launch_bounds__(256) pert_totals_k(ChainView V, const double *a_chain, const double *pot_chain,
                                                     double *out8) {
    __shared__ double sm[4][256];
    const int m = blockIdx.x;
    const int np = npert_of(V, m);
    double *o = out8 + 16 * (int64_t)m;
    const double M = o[11];
    double v[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < V.n_ch; k += 256) {
        const int64_t kk = (int64_t)m * V.n_ch + k;
        const double mk = V.cm[kk];
        v[0] += mk * a_chain[3 * kk]; v[1] += mk * a_chain[3 * kk + 1]; v[2] += mk * a_chain[3 * kk + 2];
        v[3] += mk * pot_chain[kk];
    }
    block_sum4<256>(v, sm);
    double u[4] = {0, 0, 0, 0};
    for (int p = threadIdx.x; p < np; p += 256) {
        const int64_t q = (int64_t)m * V.cap + p;
        kep(V.px[3 * q] - o[8], V.px[3 * q + 1] - o[9], V.px[3 * q + 2] - o[10], V.pm[q], u[0], u[1], u[2], u[3]);
    }
    block_sum4<256>(u, sm);
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; a++) o[a] = (M > 0) ? v[a] / M : 0.0;
        for (int a = 0; a < 3; a++) o[3 + a] = u[a];
        o[6] = (M > 0) ? v[3] / M : 0.0;
        o[7] = u[3];
    }
}

static rv_status coupling(rv_ctx *c, int M, const ChainView &V, double *a_pert, double *pot_pert, double *a_chain,
                          double *pot_chain, double *out8, cudaStream_t s) {
    chain_com_k<<<ceil_div(M, 128), 128, 0, s>>>(M, V.n_ch, V.cm, V.cx, out8, nullptr, nullptr);
    count_launch(c);
    if (V.cap > 0) {
        pert_on_stars_k<<<dim3(ceil_div(V.cap, 128), M), 128, 0, s>>>(V, out8, a_pert, pot_pert);
        count_launch(c);
    }
    if (V.n_ch > 0) {
        pert_on_members_k<<<dim3(V.n_ch, M), 256, 0, s>>>(V, a_chain, pot_chain);
        count_launch(c);
    }
    pert_totals_k<<<M, 256, 0, s>>>(V, a_chain, pot_chain, out8);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "perturber forces");
}

rv_status perturber_forces(rv_ctx *c, int n_ch, const double *cm, const double *cx, int n_pert_max,
                           const int *d_npert, const double *pm, const double *px, double *a_pert,
                           double *pot_pert, double *a_chain, double *pot_chain, double *out8, cudaStream_t s) {
    ChainView V{n_ch, n_pert_max, cm, cx, d_npert, pm, px};
    return coupling(c, 1, V, a_pert, pot_pert, a_chain, pot_chain, out8, s);
}

// ---------------------------------------------------------------------------
// system force evaluation
// ---------------------------------------------------------------------------
__global__ void gather_pert_k(int cap, const int *idx, const int *npert, const float *x, const float *y,
                              const float *z, const float *m, double *pm, double *px) {
    const int mb = blockIdx.y;
    const int np = min(npert[mb], cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)mb * cap + p;
        const int i = idx[q];
        pm[q] = (double)m[i];
        px[3 * q] = (double)x[i]; px[3 * q + 1] = (double)y[i]; px[3 * q + 2] = (double)z[i];
    }
}

// flag[i] = 1 for every star that is a perturber of some chain (the walk gives
// those no chain quadrupole: they feel the resolved members instead)
__global__ void mark_pert_k(int cap, const int *idx, const int *npert, uint8_t *flag) {
    const int mb = blockIdx.y;
    const int np = min(npert[mb], cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
        flag[idx[(int64_t)mb * cap + p]] = 1;
}

// perturbers of the last selection predicted to first order, dt after the force pass
// (Sect. 2: the chain integrator predicts them at each of its force evaluations):
// x_p(dt) = x_p + v_p dt in FP64, one rounding per operation
__global__ void predict_pert_k(int cap, const int *idx, const int *npert, const float *x, const float *y,
                               const float *z, const float *vx, const float *vy, const float *vz, const float *m,
                               double dt, double *pm, double *px) {
    const int mb = blockIdx.y;
    const int np = min(npert[mb], cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)mb * cap + p;
        const int i = idx[q];
        pm[q] = (double)m[i];
        px[3 * q] = __dadd_rn((double)x[i], __dmul_rn((double)vx[i], dt));
        px[3 * q + 1] = __dadd_rn((double)y[i], __dmul_rn((double)vy[i], dt));
        px[3 * q + 2] = __dadd_rn((double)z[i], __dmul_rn((double)vz[i], dt));
    }
}

// stars that are perturbers: add the FP64 correction (resolved chain - centre-of-mass point mass)
// (block time steps: only the stars active now, whose forces this pass wrote)
__global__ void apply_pert_k(int cap, const int *idx, const int *npert, const double *a_pert, const double *pot_pert,
                             float *ax, float *ay, float *az, float *pot, const int8_t *level, long long n, int L) {
    const int mb = blockIdx.y;
    const int np = min(npert[mb], cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)mb * cap + p;
        const int i = idx[q];
        if (level && (n & ((1ll << (L - min(max((int)level[i], 0), L))) - 1)) != 0) continue;
        ax[i] = (float)((double)ax[i] + a_pert[3 * q]);
        ay[i] = (float)((double)ay[i] + a_pert[3 * q + 1]);
        az[i] = (float)((double)az[i] + a_pert[3 * q + 2]);
        pot[i] = (float)((double)pot[i] + pot_pert[q]);
    }
}

// Chain member k of member m: mutual unsoftened FP64 pull of the other chain
// members, plus the perturbers on k, plus the tree's force on the centre of
// mass without the perturbers' direct terms (those are resolved per member).
__global__ void chain_accel_k(int M, int n_ch, const double *cm, const double *cx, const double *a_ext,
                              const double *pot_ext, const float *xout, const double *out8, double *ca, double *cpot) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M * n_ch; t += gridDim.x * blockDim.x) {
        const int m = t / n_ch, k = t % n_ch;
        const double *o = out8 + 16 * (int64_t)m;
        const double *mm = cm + (int64_t)m * n_ch, *xx = cx + 3 * (int64_t)m * n_ch;
        double tx = (double)xout[4 * m] - o[3], ty = (double)xout[4 * m + 1] - o[4], tz = (double)xout[4 * m + 2] - o[5];
        double tp = (double)xout[4 * m + 3] - o[7];
        double ax = 0, ay = 0, az = 0, ph = 0;
        for (int j = 0; j < n_ch; j++) {
            if (j == k) continue;
            kep(xx[3 * j] - xx[3 * k], xx[3 * j + 1] - xx[3 * k + 1], xx[3 * j + 2] - xx[3 * k + 2], mm[j], ax, ay, az,
                ph);
        }
        ca[3 * (int64_t)t] = ax + a_ext[3 * (int64_t)t] + tx;
        ca[3 * (int64_t)t + 1] = ay + a_ext[3 * (int64_t)t + 1] + ty;
        ca[3 * (int64_t)t + 2] = az + a_ext[3 * (int64_t)t + 2] + tz;
        cpot[t] = ph + pot_ext[t] + tp;
    }
}

static const int64_t *system_offsets(const rv_system *sys, int64_t tmp[2]);

// Perturber pull on the chain members at chain positions chain_x (member-major
// FP64), the perturbers of the last force pass predicted dt ahead.
rv_status chain_perturber_forces(rv_ctx *c, const rv_system *sys, double dt, const double *chain_x, double *a_chain,
                                 double *pot_chain, cudaStream_t s) {
    Workspace &w = c->w;
    const int M = system_chains(sys);   // the coupling kernels treat each chain as a unit
    const int cap = member_cap(M);
    predict_pert_k<<<dim3(ceil_div(cap, 128), M), 128, 0, s>>>(cap, w.pert_idx, w.npert, sys->x, sys->y, sys->z,
                                                               sys->vx, sys->vy, sys->vz, sys->m, dt, w.pert_m,
                                                               w.pert_x);
    count_launch(c);
    ChainView V{sys->n_chain, cap, sys->chain_m, chain_x, w.npert, w.pert_m, w.pert_x};
    pert_on_members_k<<<dim3(sys->n_chain, M), 256, 0, s>>>(V, a_chain, pot_chain ? pot_chain : w.chain_ext_pot);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "chain perturber forces");
}

static const int64_t *system_offsets(const rv_system *sys, int64_t tmp[2]) {
    if (sys->n_members > 1 || sys->member_offsets) return sys->member_offsets;
    tmp[0] = 0;
    tmp[1] = sys->n;
    return tmp;
}

int system_members(const rv_system *sys) { return std::max(1, (int)sys->n_members); }
int chains_per_member(const rv_system *sys) { return std::max(1, (int)sys->n_chains); }
int system_chains(const rv_system *sys) {
    return sys->n_chain > 0 ? system_members(sys) * chains_per_member(sys) : 0;
}

rv_status system_forces(rv_ctx *c, rv_system *sys, cudaStream_t s, const BlockSel *blk) {
    Workspace &w = c->w;
    rv_status r;
    const bool chain = sys->n_chain > 0;
    const int M = system_members(sys);
    const int C = chains_per_member(sys);
    const int NC = system_chains(sys);   // chains: the unit of every chain kernel below
    int64_t tmp[2];
    const int64_t *off = system_offsets(sys, tmp);
    const int cap = member_cap(std::max(1, NC));
    // the chain's quadrupole acts on the stars beyond its perturbers (rv_system.chain_quad)
    const bool quad = chain && sys->chain_quad != 0 && sys->n_chain > 1;
    if (chain) {
        chain_com_k<<<ceil_div(NC, 128), 128, 0, s>>>(NC, sys->n_chain, sys->chain_m, sys->chain_x, w.out8,
                                                      w.extra_xyzm, w.extra_eps, quad ? w.extra_quad : nullptr);
        count_launch(c);
    }
    if ((r = upload_offsets(c, M, off, s)) != RV_OK) return r;
    if (chain && (sys->pert_mode == 1 || sys->pert_mode == 2 || sys->pert_mode == 3)) {
        // one selection per chain j of every member (perturber slots of chain m C + j)
        for (int j = 0; j < C; j++) {
            if (M == 1) {
                r = select_perturbers(c, sys->n, sys->x, sys->y, sys->z, w.extra_xyzm + 4 * j, nullptr,
                                      sys->pert_mode, sys->pert_radius, sys->pert_k, cap, w.pert_idx + (int64_t)j * cap,
                                      w.npert + j, s, sys->m, sys->pert_gamma);
                if (r != RV_OK) return r;
            } else {
                // the sort buffers are shared with the tree build, which comes next
                const int bpm = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(c->max_member, 256), 64));
                const SelRule R = sel_rule(sys->pert_mode, sys->pert_radius, sys->m, sys->pert_gamma);
                sel_member_keys_k<<<dim3(bpm, M), 256, 0, s>>>(w.moff, bpm, sys->x, sys->y, sys->z, w.extra_xyzm, C,
                                                               j, R, w.key_a);
                count_launch(c);
                uint64_t *sk;
                int *si;
                if ((r = radix_sort(c, sys->n, sys->pert_mode == 2 ? 4 : 1, &sk, &si, true, s, true)) != RV_OK)
                    return r;
                sel_member_write_k<<<M, 256, 0, s>>>(w.moff, sk, si, sys->pert_mode, sys->pert_k, cap, C, j,
                                                     w.pert_idx, w.npert, w.st);
                count_launch(c);
            }
        }
    } else if (chain) {
        cudaMemsetAsync(w.npert, 0, sizeof(int) * NC, s);
    }
    if (quad) {
        cudaMemsetAsync(w.pflag, 0, (size_t)std::max<int64_t>(sys->n, 1), s);
        mark_pert_k<<<dim3(ceil_div(cap, 128), NC), 128, 0, s>>>(cap, w.pert_idx, w.npert, w.pflag);
        count_launch(c);
    }
    if ((r = build_tree(c, M, off, sys->x, sys->y, sys->z, sys->m, s)) != RV_OK) return r;
    const uint8_t *gact = nullptr;
    if (blk) {
        launch_block_groups(c, *blk, s);
        gact = w.gact;
    }
    // relative criterion (cfg.mac = 1): the accelerations in the system arrays (the previous
    // pass's, zero before the first one) are the references, read before they are overwritten
    const RelMac rel{c->cfg.alpha, sys->ax, sys->ay, sys->az};
    if ((r = tree_walk(c, c->cfg.theta, c->cfg.eps_star, NC, w.extra_xyzm, w.extra_eps, nullptr, C,
                       sys->ax, sys->ay, sys->az, sys->pot, w.extra_out, s, nullptr,
                       c->cfg.mac == 1 ? &rel : nullptr, gact, quad ? w.extra_quad : nullptr,
                       quad ? w.pflag : nullptr)) != RV_OK)
        return r;
    c->pert_members = NC;
    if (chain) {
        gather_pert_k<<<dim3(ceil_div(cap, 128), NC), 128, 0, s>>>(cap, w.pert_idx, w.npert, sys->x, sys->y, sys->z,
                                                                  sys->m, w.pert_m, w.pert_x);
        count_launch(c);
        ChainView V{sys->n_chain, cap, sys->chain_m, sys->chain_x, w.npert, w.pert_m, w.pert_x};
        r = coupling(c, NC, V, w.pert_a, w.pert_pot, w.chain_ext_a, w.chain_ext_pot, w.out8, s);
        if (r != RV_OK) return r;
        apply_pert_k<<<dim3(ceil_div(cap, 128), NC), 128, 0, s>>>(cap, w.pert_idx, w.npert, w.pert_a, w.pert_pot,
                                                                 sys->ax, sys->ay, sys->az, sys->pot,
                                                                 blk ? blk->level : nullptr, blk ? blk->n : 0,
                                                                 blk ? blk->L : 0);
        count_launch(c);
        chain_accel_k<<<ceil_div(NC * sys->n_chain, 128), 128, 0, s>>>(NC, sys->n_chain, sys->chain_m, sys->chain_x,
                                                                      w.chain_ext_a, w.chain_ext_pot, w.extra_out,
                                                                      w.out8, sys->chain_a, sys->chain_pot);
        count_launch(c);
    }
    return cuda_check(c, cudaGetLastError(), "system forces");
}

// ---------------------------------------------------------------------------
// kick-drift-kick
// ---------------------------------------------------------------------------
__global__ void kick_drift_k(int64_t n, float *x, float *y, float *z, float *vx, float *vy, float *vz,
                             const float *ax, const float *ay, const float *az, float hdt, float dt, int drift) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float u = fmaf(ax[i], hdt, vx[i]), v = fmaf(ay[i], hdt, vy[i]), w = fmaf(az[i], hdt, vz[i]);
        vx[i] = u; vy[i] = v; vz[i] = w;
        if (drift) {
            x[i] = fmaf(u, dt, x[i]); y[i] = fmaf(v, dt, y[i]); z[i] = fmaf(w, dt, z[i]);
        }
    }
}

__global__ void chain_kick_drift_k(int n, double *cx, double *cv, const double *ca, double hdt, double dt, int drift) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        for (int a = 0; a < 3; a++) {
            cv[3 * k + a] += ca[3 * k + a] * hdt;
            if (drift) cx[3 * k + a] += cv[3 * k + a] * dt;
        }
}

void kick(rv_ctx *c, rv_system *sys, double dt, int drift, cudaStream_t s) {
    if (sys->n > 0) {
        kick_drift_k<<<grid_n(c, sys->n), 256, 0, s>>>(sys->n, sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz,
                                                      sys->ax, sys->ay, sys->az, (float)(0.5 * dt), (float)dt, drift);
        count_launch(c);
    }
    if (sys->n_chain > 0) {
        const int nc = system_chains(sys) * sys->n_chain;
        chain_kick_drift_k<<<ceil_div(nc, 128), 128, 0, s>>>(nc, sys->chain_x, sys->chain_v, sys->chain_a, 0.5 * dt, dt,
                                                             drift);
        count_launch(c);
    }
}

rv_status kdk(rv_ctx *c, rv_system *sys, double dt, int nsteps, cudaStream_t s) {
    for (int step = 0; step < nsteps; step++) {
        kick(c, sys, dt, 1, s);
        rv_status r = system_forces(c, sys, s);
        if (r != RV_OK) return r;
        kick(c, sys, dt, 0, s);
    }
    return cuda_check(c, cudaGetLastError(), "kdk");
}

// ---------------------------------------------------------------------------
// FP64 totals per member: fixed grid, fixed per-thread striding, fixed tree
// reductions, so the result does not depend on scheduling
// ---------------------------------------------------------------------------
constexpr int kRedQ = 9;  // ekin, epot, P(3), L(3), mass

static int energy_bpm(int M) { return std::max(1, std::min(256, kRedSlots / M)); }

__global__ void __launch_bounds__(256) energy_partial_k(const int64_t *moff, int bpm, const float *x, const float *y,
                                                        const float *z, const float *vx, const float *vy,
                                                        const float *vz, const float *m, const float *pot,
                                                        double *part) {
    __shared__ double sm[kRedQ][256];
    const int mb = blockIdx.y;
    double q[kRedQ] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = moff[mb] + (int64_t)blockIdx.x * 256 + threadIdx.x; i < moff[mb + 1]; i += (int64_t)bpm * 256) {
        double mi = m[i], X = x[i], Y = y[i], Z = z[i], U = vx[i], V = vy[i], W = vz[i];
        q[0] += 0.5 * mi * (U * U + V * V + W * W);
        q[1] += 0.5 * mi * (double)pot[i];
        q[2] += mi * U; q[3] += mi * V; q[4] += mi * W;
        q[5] += mi * (Y * W - Z * V); q[6] += mi * (Z * U - X * W); q[7] += mi * (X * V - Y * U);
        q[8] += mi;
    }
    for (int a = 0; a < kRedQ; a++) sm[a][threadIdx.x] = q[a];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int a = 0; a < kRedQ; a++) sm[a][threadIdx.x] += sm[a][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < kRedQ) part[kRedQ * ((int64_t)mb * bpm + blockIdx.x) + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) energy_final_k(const double *part, int bpm, int n_ch, const double *cm,
                                                      const double *cx, const double *cv, const double *cpot,
                                                      double *out) {
    __shared__ double sm[kRedQ][256];
    const int mb = blockIdx.x;
    for (int a = 0; a < kRedQ; a++)
        sm[a][threadIdx.x] = ((int)threadIdx.x < bpm) ? part[kRedQ * ((int64_t)mb * bpm + threadIdx.x) + a] : 0.0;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int a = 0; a < kRedQ; a++) sm[a][threadIdx.x] += sm[a][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double q[kRedQ];
        for (int a = 0; a < kRedQ; a++) q[a] = sm[a][0];
        for (int k = 0; k < n_ch; k++) {
            const int64_t kk = (int64_t)mb * n_ch + k;
            double mk = cm[kk];
            const double *X = cx + 3 * kk, *V = cv + 3 * kk;
            q[0] += 0.5 * mk * (V[0] * V[0] + V[1] * V[1] + V[2] * V[2]);
            q[1] += 0.5 * mk * cpot[kk];
            q[2] += mk * V[0]; q[3] += mk * V[1]; q[4] += mk * V[2];
            q[5] += mk * (X[1] * V[2] - X[2] * V[1]);
            q[6] += mk * (X[2] * V[0] - X[0] * V[2]);
            q[7] += mk * (X[0] * V[1] - X[1] * V[0]);
            q[8] += mk;
        }
        double *o = out + 10 * (int64_t)mb;
        o[0] = q[0]; o[1] = q[1]; o[2] = q[0] + q[1];
        for (int a = 0; a < 6; a++) o[3 + a] = q[2 + a];
        o[9] = q[8];
    }
}

rv_status energy(rv_ctx *c, const rv_system *sys, double *out, cudaStream_t s) {
    const int M = system_members(sys);
    int64_t tmp[2];
    rv_status r = upload_offsets(c, M, system_offsets(sys, tmp), s);
    if (r != RV_OK) return r;
    const int bpm = energy_bpm(M);
    energy_partial_k<<<dim3(bpm, M), 256, 0, s>>>(c->w.moff, bpm, sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz,
                                                  sys->m, sys->pot, c->w.red);
    count_launch(c);
    // chain members of member m: the n_chains chains of that member, one after another
    energy_final_k<<<M, 256, 0, s>>>(c->w.red, bpm, sys->n_chain > 0 ? chains_per_member(sys) * sys->n_chain : 0,
                                     sys->chain_m, sys->chain_x, sys->chain_v, sys->chain_pot, out);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "energy");
}

// ---------------------------------------------------------------------------
// CUDA graph of one step (kick-drift-kick [+ energy]), captured once per
// (system, dt, energy output) and replayed
// ---------------------------------------------------------------------------
static unsigned long long graph_key(const rv_system *sys, double dt, const double *eout) {
    unsigned long long h = 1469598103934665603ull;
    const unsigned char *p = reinterpret_cast<const unsigned char *>(sys);
    for (size_t i = 0; i < sizeof(rv_system); i++) h = (h ^ p[i]) * 1099511628211ull;
    const int M = system_members(sys);
    if (sys->member_offsets)
        for (int k = 0; k <= M; k++) h = (h ^ (unsigned long long)sys->member_offsets[k]) * 1099511628211ull;
    unsigned long long d;
    memcpy(&d, &dt, sizeof d);
    h = (h ^ d) * 1099511628211ull;
    h = (h ^ (unsigned long long)(uintptr_t)eout) * 1099511628211ull;
    return h;
}

rv_status kdk_graph(rv_ctx *c, rv_system *sys, double dt, int nsteps, double *eout, cudaStream_t s) {
    const unsigned long long key = graph_key(sys, dt, eout);
    if (!c->graph || c->graph_key != key) {
        if (c->graph) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
        // settle everything a capture must not do (offset upload, kernel attributes) with an uncaptured
        // force evaluation at the current positions, which the step's first kick already expects
        rv_status r = system_forces(c, sys, s);
        if (r != RV_OK) return r;
        if ((r = cuda_check(c, cudaStreamSynchronize(s), "graph prepare")) != RV_OK) return r;
        cudaGraph_t g = nullptr;
        if ((r = cuda_check(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture")) != RV_OK)
            return r;
        const long long l0 = c->launches;
        r = kdk(c, sys, dt, 1, s);
        if (r == RV_OK && eout) r = energy(c, sys, eout, s);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (r != RV_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return cuda_check(c, e, "end capture");
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_check(c, e, "graph instantiate");
        c->graph = ge;
        c->graph_key = key;
        c->graph_launches = c->launches - l0;
        c->launches = l0;
    }
    for (int k = 0; k < nsteps; k++) {
        cudaError_t e = cudaGraphLaunch(c->graph, s);
        if (e != cudaSuccess) return cuda_check(c, e, "graph launch");
        c->launches += c->graph_launches;
    }
    return RV_OK;
}

}  // namespace rv
