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

__global__ void sel_radius_flag_k(int64_t n, const float *x, const float *y, const float *z, const float *cdev,
                                  float3 chost, float r2, int *flag) {
    float3 c = centre_of(cdev, chost);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = dist2_f32(x[i], y[i], z[i], c.x, c.y, c.z) < r2 ? 1 : 0;
}

__global__ void sel_radius_write_k(int64_t n, const float *x, const float *y, const float *z, const float *cdev,
                                   float3 chost, float r2, const int *ofs, const int *total, int cap, int *idx,
                                   int *count, DevState *st) {
    float3 c = centre_of(cdev, chost);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (dist2_f32(x[i], y[i], z[i], c.x, c.y, c.z) < r2) {
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

static int grid_n(rv_ctx *c, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8));
}

rv_status select_perturbers(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z,
                            const float *centre_dev, const float *centre_host, int mode, float radius, int k,
                            int cap, int *idx, int *count, cudaStream_t s) {
    float3 ch = centre_host ? make_float3(centre_host[0], centre_host[1], centre_host[2]) : make_float3(0, 0, 0);
    Workspace &w = c->w;
    if (mode == 1) {
        float r2 = radius * radius;  // one FP32 product
        if (n == 0) return cuda_check(c, cudaMemsetAsync(count, 0, sizeof(int), s), "select");
        sel_radius_flag_k<<<grid_n(c, n), 256, 0, s>>>(n, x, y, z, centre_dev, ch, r2, w.sel_flag);
        count_launch(c);
        int *total = &w.st->n_pert;  // scratch for the total; overwritten by the clamped count
        rv_status r = exclusive_scan(c, w.sel_flag, n, nullptr, total, s);
        if (r != RV_OK) return r;
        sel_radius_write_k<<<grid_n(c, n), 256, 0, s>>>(n, x, y, z, centre_dev, ch, r2, w.sel_flag, total, cap, idx,
                                                        count, w.st);
        count_launch(c);
    } else {
        if (n == 0 || k <= 0) {
            cudaMemsetAsync(&w.st->n_pert, 0, sizeof(int), s);
            return cuda_check(c, cudaMemsetAsync(count, 0, sizeof(int), s), "select");
        }
        // the sort buffers are shared with the tree build: the tree is invalid afterwards
        c->built = false;
        sel_knn_keys_k<<<grid_n(c, n), 256, 0, s>>>(n, x, y, z, centre_dev, ch, w.key_a);
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

// ---------------------------------------------------------------------------
// FP64 chain / perturber coupling
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

// out8 layout: [0..3) corr (Eq. 3), [3..6) sub, [6] sum_k m_k pot_chain[k] / M, [7] sub potential,
// [8..11) centre of mass, [11] M.
__global__ void chain_com_k(int n_ch, const double *cm, const double *cx, double *out8, float *xyzm, float *xeps) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double M = 0, c[3] = {0, 0, 0};
    for (int k = 0; k < n_ch; k++) {
        M += cm[k];
        for (int a = 0; a < 3; a++) c[a] += cm[k] * cx[3 * k + a];
    }
    for (int a = 0; a < 3; a++) c[a] = (M > 0) ? c[a] / M : 0.0;
    out8[8] = c[0]; out8[9] = c[1]; out8[10] = c[2]; out8[11] = M;
    if (xyzm) {
        xyzm[0] = (float)c[0]; xyzm[1] = (float)c[1]; xyzm[2] = (float)c[2]; xyzm[3] = (float)M;
        xeps[0] = 0.f;
    }
}

// perturbers: resolved members minus the centre-of-mass point mass
__global__ void pert_on_stars_k(int n_ch, const double *cm, const double *cx, int n_max, const int *d_np,
                                const double *px, const double *out8, double *a_pert, double *pot_pert) {
    int np = d_np ? min(*d_np, n_max) : n_max;
    double M = out8[11];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        double x = px[3 * p], y = px[3 * p + 1], z = px[3 * p + 2];
        double ax = 0, ay = 0, az = 0, ph = 0;
        for (int k = 0; k < n_ch; k++) kep(cx[3 * k] - x, cx[3 * k + 1] - y, cx[3 * k + 2] - z, cm[k], ax, ay, az, ph);
        double bx = 0, by = 0, bz = 0, bp = 0;
        kep(out8[8] - x, out8[9] - y, out8[10] - z, M, bx, by, bz, bp);
        a_pert[3 * p] = ax - bx; a_pert[3 * p + 1] = ay - by; a_pert[3 * p + 2] = az - bz;
        pot_pert[p] = ph - bp;
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

// one block per member: perturbers on member k (fixed order: strided partials + tree)
__global__ void __launch_bounds__(256) pert_on_members_k(int n_ch, const double *cx, int n_max, const int *d_np,
                                                         const double *pm, const double *px, double *a_chain,
                                                         double *pot_chain) {
    __shared__ double sm[4][256];
    int np = d_np ? min(*d_np, n_max) : n_max;
    int k = blockIdx.x;
    double x = cx[3 * k], y = cx[3 * k + 1], z = cx[3 * k + 2];
    double v[4] = {0, 0, 0, 0};
    for (int p = threadIdx.x; p < np; p += 256)
        kep(px[3 * p] - x, px[3 * p + 1] - y, px[3 * p + 2] - z, pm[p], v[0], v[1], v[2], v[3]);
    block_sum4<256>(v, sm);
    if (threadIdx.x == 0) {
        a_chain[3 * k] = v[0]; a_chain[3 * k + 1] = v[1]; a_chain[3 * k + 2] = v[2];
        pot_chain[k] = v[3];
    }
}

// Eq. 3 correction, and the perturbers' direct terms on the centre of mass
__global__ void __launch_bounds__(256) pert_totals_k(int n_ch, const double *cm, const double *a_chain,
                                                     const double *pot_chain, int n_max, const int *d_np,
                                                     const double *pm, const double *px, double *out8) {
    __shared__ double sm[4][256];
    int np = d_np ? min(*d_np, n_max) : n_max;
    double M = out8[11];
    double v[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < n_ch; k += 256) {
        v[0] += cm[k] * a_chain[3 * k]; v[1] += cm[k] * a_chain[3 * k + 1]; v[2] += cm[k] * a_chain[3 * k + 2];
        v[3] += cm[k] * pot_chain[k];
    }
    block_sum4<256>(v, sm);
    double u[4] = {0, 0, 0, 0};
    for (int p = threadIdx.x; p < np; p += 256)
        kep(px[3 * p] - out8[8], px[3 * p + 1] - out8[9], px[3 * p + 2] - out8[10], pm[p], u[0], u[1], u[2], u[3]);
    block_sum4<256>(u, sm);
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; a++) out8[a] = (M > 0) ? v[a] / M : 0.0;
        for (int a = 0; a < 3; a++) out8[3 + a] = u[a];
        out8[6] = (M > 0) ? v[3] / M : 0.0;
        out8[7] = u[3];
    }
}

rv_status perturber_forces(rv_ctx *c, int n_ch, const double *cm, const double *cx, int n_pert_max,
                           const int *d_npert, const double *pm, const double *px, double *a_pert,
                           double *pot_pert, double *a_chain, double *pot_chain, double *out8, cudaStream_t s) {
    chain_com_k<<<1, 32, 0, s>>>(n_ch, cm, cx, out8, nullptr, nullptr);
    count_launch(c);
    if (n_pert_max > 0) {
        pert_on_stars_k<<<ceil_div(n_pert_max, 128), 128, 0, s>>>(n_ch, cm, cx, n_pert_max, d_npert, px, out8, a_pert,
                                                                  pot_pert);
        count_launch(c);
    }
    if (n_ch > 0) {
        pert_on_members_k<<<n_ch, 256, 0, s>>>(n_ch, cx, n_pert_max, d_npert, pm, px, a_chain, pot_chain);
        count_launch(c);
    }
    pert_totals_k<<<1, 256, 0, s>>>(n_ch, cm, a_chain, pot_chain, n_pert_max, d_npert, pm, px, out8);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "perturber forces");
}

// ---------------------------------------------------------------------------
// system force evaluation
// ---------------------------------------------------------------------------
__global__ void gather_pert_k(const int *idx, const int *d_np, const float *x, const float *y, const float *z,
                              const float *m, double *pm, double *px) {
    int np = min(*d_np, kMaxPert);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        int i = idx[p];
        pm[p] = (double)m[i];
        px[3 * p] = (double)x[i]; px[3 * p + 1] = (double)y[i]; px[3 * p + 2] = (double)z[i];
    }
}

// stars that are perturbers: add the FP64 correction (resolved chain - centre-of-mass point mass)
__global__ void apply_pert_k(const int *idx, const int *d_np, const double *a_pert, const double *pot_pert, float *ax,
                             float *ay, float *az, float *pot) {
    int np = min(*d_np, kMaxPert);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        int i = idx[p];
        ax[i] = (float)((double)ax[i] + a_pert[3 * p]);
        ay[i] = (float)((double)ay[i] + a_pert[3 * p + 1]);
        az[i] = (float)((double)az[i] + a_pert[3 * p + 2]);
        pot[i] = (float)((double)pot[i] + pot_pert[p]);
    }
}

// Member k: mutual unsoftened FP64 pull of the other members, plus the
// perturbers on k, plus the tree's force on the centre of mass without the
// perturbers' direct terms (those are now resolved per member).
__global__ void chain_accel_k(int n_ch, const double *cm, const double *cx, const double *a_ext,
                              const double *pot_ext, const float *xout, const double *out8, double *ca,
                              double *cpot) {
    double tx = (double)xout[0] - out8[3], ty = (double)xout[1] - out8[4], tz = (double)xout[2] - out8[5];
    double tp = (double)xout[3] - out8[7];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_ch; k += gridDim.x * blockDim.x) {
        double ax = 0, ay = 0, az = 0, ph = 0;
        for (int j = 0; j < n_ch; j++) {
            if (j == k) continue;
            kep(cx[3 * j] - cx[3 * k], cx[3 * j + 1] - cx[3 * k + 1], cx[3 * j + 2] - cx[3 * k + 2], cm[j], ax, ay, az,
                ph);
        }
        ca[3 * k] = ax + a_ext[3 * k] + tx;
        ca[3 * k + 1] = ay + a_ext[3 * k + 1] + ty;
        ca[3 * k + 2] = az + a_ext[3 * k + 2] + tz;
        cpot[k] = ph + pot_ext[k] + tp;
    }
}

rv_status system_forces(rv_ctx *c, rv_system *sys, cudaStream_t s) {
    Workspace &w = c->w;
    rv_status r;
    const bool chain = sys->n_chain > 0;
    if (chain) {
        chain_com_k<<<1, 32, 0, s>>>(sys->n_chain, sys->chain_m, sys->chain_x, w.out8, w.extra_xyzm, w.extra_eps);
        count_launch(c);
        if (sys->pert_mode == 1 || sys->pert_mode == 2) {
            r = select_perturbers(c, sys->n, sys->x, sys->y, sys->z, w.extra_xyzm, nullptr, sys->pert_mode,
                                  sys->pert_radius, sys->pert_k, kMaxPert, w.pert_idx, &w.st->n_pert, s);
            if (r != RV_OK) return r;
        } else {
            cudaMemsetAsync(&w.st->n_pert, 0, sizeof(int), s);
        }
    }
    if ((r = build_tree(c, sys->n, sys->x, sys->y, sys->z, sys->m, s)) != RV_OK) return r;
    if ((r = tree_walk(c, c->cfg.theta, c->cfg.eps_star, chain ? 1 : 0, w.extra_xyzm, w.extra_eps, sys->ax, sys->ay,
                       sys->az, sys->pot, w.extra_out, s)) != RV_OK)
        return r;
    if (chain) {
        gather_pert_k<<<ceil_div(kMaxPert, 128), 128, 0, s>>>(w.pert_idx, &w.st->n_pert, sys->x, sys->y, sys->z,
                                                              sys->m, w.pert_m, w.pert_x);
        count_launch(c);
        r = perturber_forces(c, sys->n_chain, sys->chain_m, sys->chain_x, kMaxPert, &w.st->n_pert, w.pert_m, w.pert_x,
                             w.pert_a, w.pert_pot, w.chain_ext_a, w.chain_ext_pot, w.out8, s);
        if (r != RV_OK) return r;
        apply_pert_k<<<ceil_div(kMaxPert, 128), 128, 0, s>>>(w.pert_idx, &w.st->n_pert, w.pert_a, w.pert_pot, sys->ax,
                                                             sys->ay, sys->az, sys->pot);
        count_launch(c);
        chain_accel_k<<<1, 256, 0, s>>>(sys->n_chain, sys->chain_m, sys->chain_x, w.chain_ext_a, w.chain_ext_pot,
                                        w.extra_out, w.out8, sys->chain_a, sys->chain_pot);
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

__global__ void chain_kick_drift_k(int n_ch, double *cx, double *cv, const double *ca, double hdt, double dt,
                                   int drift) {
    for (int k = threadIdx.x; k < n_ch; k += blockDim.x)
        for (int a = 0; a < 3; a++) {
            cv[3 * k + a] += ca[3 * k + a] * hdt;
            if (drift) cx[3 * k + a] += cv[3 * k + a] * dt;
        }
}

rv_status kdk(rv_ctx *c, rv_system *sys, double dt, int nsteps, cudaStream_t s) {
    const float hdt = (float)(0.5 * dt), fdt = (float)dt;
    const int g = grid_n(c, sys->n);
    for (int step = 0; step < nsteps; step++) {
        if (sys->n > 0) {
            kick_drift_k<<<g, 256, 0, s>>>(sys->n, sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz, sys->ax, sys->ay,
                                          sys->az, hdt, fdt, 1);
            count_launch(c);
        }
        if (sys->n_chain > 0) {
            chain_kick_drift_k<<<1, 256, 0, s>>>(sys->n_chain, sys->chain_x, sys->chain_v, sys->chain_a, 0.5 * dt, dt,
                                                 1);
            count_launch(c);
        }
        rv_status r = system_forces(c, sys, s);
        if (r != RV_OK) return r;
        if (sys->n > 0) {
            kick_drift_k<<<g, 256, 0, s>>>(sys->n, sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz, sys->ax, sys->ay,
                                          sys->az, hdt, fdt, 0);
            count_launch(c);
        }
        if (sys->n_chain > 0) {
            chain_kick_drift_k<<<1, 256, 0, s>>>(sys->n_chain, sys->chain_x, sys->chain_v, sys->chain_a, 0.5 * dt, dt,
                                                 0);
            count_launch(c);
        }
    }
    return cuda_check(c, cudaGetLastError(), "kdk");
}

// ---------------------------------------------------------------------------
// FP64 totals: fixed grid, fixed per-thread striding, fixed tree reductions
// ---------------------------------------------------------------------------
constexpr int kRedBlocks = 256;
constexpr int kRedQ = 9;  // ekin, epot, P(3), L(3), mass

__global__ void __launch_bounds__(256) energy_partial_k(int64_t n, const float *x, const float *y, const float *z,
                                                        const float *vx, const float *vy, const float *vz,
                                                        const float *m, const float *pot, double *part) {
    __shared__ double sm[kRedQ][256];
    double q[kRedQ] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)kRedBlocks * 256) {
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
    if (threadIdx.x < kRedQ) part[kRedQ * blockIdx.x + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void __launch_bounds__(256) energy_final_k(const double *part, int64_t n, const float *m, int n_ch,
                                                      const double *cm, const double *cx, const double *cv,
                                                      const double *cpot, double *out) {
    __shared__ double sm[kRedQ][256];
    for (int a = 0; a < kRedQ; a++) sm[a][threadIdx.x] = part[kRedQ * threadIdx.x + a];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int a = 0; a < kRedQ; a++) sm[a][threadIdx.x] += sm[a][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double q[kRedQ];
        for (int a = 0; a < kRedQ; a++) q[a] = sm[a][0];
        double M = q[8];
        for (int k = 0; k < n_ch; k++) {
            double mk = cm[k];
            const double *X = cx + 3 * k, *V = cv + 3 * k;
            q[0] += 0.5 * mk * (V[0] * V[0] + V[1] * V[1] + V[2] * V[2]);
            q[1] += 0.5 * mk * cpot[k];
            q[2] += mk * V[0]; q[3] += mk * V[1]; q[4] += mk * V[2];
            q[5] += mk * (X[1] * V[2] - X[2] * V[1]);
            q[6] += mk * (X[2] * V[0] - X[0] * V[2]);
            q[7] += mk * (X[0] * V[1] - X[1] * V[0]);
            M += mk;
        }
        out[0] = q[0]; out[1] = q[1]; out[2] = q[0] + q[1];
        for (int a = 0; a < 6; a++) out[3 + a] = q[2 + a];
        out[9] = M;
    }
}

rv_status energy(rv_ctx *c, const rv_system *sys, double *out, cudaStream_t s) {
    energy_partial_k<<<kRedBlocks, 256, 0, s>>>(sys->n, sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz, sys->m,
                                                sys->pot, c->w.red);
    count_launch(c);
    energy_final_k<<<1, 256, 0, s>>>(c->w.red, sys->n, sys->m, sys->n_chain, sys->chain_m, sys->chain_x, sys->chain_v,
                                     sys->chain_pot, out);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "energy");
}

}  // namespace rv
