// membership.cu -- who belongs to a regularised chain (Sect. 2).
//
// Absorption (Eq. 4): a star joins the chain when it comes closer to the
// chain's centre of mass than the chain radius, the largest distance of any
// member from the centre of mass. This runs over all stars on the GPU.
//
// Escape (Eq. 5): a member leaves when it is farther than gamma r_chain,0 from
// the centre of mass and moving away from it; with the rules around it
// (absorption first, termination, a new designated SMBH). It looks at the at
// most 250 members of one chain and runs on the host.
//
// Both decide in FP64 with one rounding per operation in a fixed order (the
// host routine is compiled without floating-point contraction), so the same
// inputs give the same membership everywhere.
#include <math.h>

#include <algorithm>

#include "rv_internal.cuh"

namespace rv {

// centre of mass (members in index order) and the largest squared member
// distance from it, into st->absorb
__global__ void absorb_setup_k(int n_ch, const double *cm, const double *cx, DevState *st) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double M = 0.0, c[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < n_ch; k++) {
        M = __dadd_rn(M, cm[k]);
        for (int a = 0; a < 3; a++) c[a] = __dadd_rn(c[a], __dmul_rn(cm[k], cx[3 * k + a]));
    }
    for (int a = 0; a < 3; a++) c[a] = (M > 0.0) ? __ddiv_rn(c[a], M) : 0.0;
    double rc2 = 0.0;
    for (int k = 0; k < n_ch; k++) {
        const double dx = __dsub_rn(cx[3 * k], c[0]), dy = __dsub_rn(cx[3 * k + 1], c[1]),
                     dz = __dsub_rn(cx[3 * k + 2], c[2]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (d2 > rc2) rc2 = d2;
    }
    st->absorb[0] = c[0];
    st->absorb[1] = c[1];
    st->absorb[2] = c[2];
    st->absorb[3] = rc2;
}

__device__ __forceinline__ bool absorbed(const DevState *st, float x, float y, float z) {
    const double dx = __dsub_rn((double)x, st->absorb[0]), dy = __dsub_rn((double)y, st->absorb[1]),
                 dz = __dsub_rn((double)z, st->absorb[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 < st->absorb[3];
}

__global__ void absorb_flag_k(int64_t n, const float *x, const float *y, const float *z, const DevState *st,
                              int *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = absorbed(st, x[i], y[i], z[i]) ? 1 : 0;
}

__global__ void absorb_write_k(int64_t n, const float *x, const float *y, const float *z, const DevState *st,
                               const int *ofs, const int *total, int cap, int *idx, int *count, double *r_chain) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (absorbed(st, x[i], y[i], z[i])) {
            const int p = ofs[i];
            if (p < cap) idx[p] = (int)i;
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *count = n > 0 ? *total : 0;
        if (r_chain) *r_chain = __dsqrt_rn(st->absorb[3]);
    }
}

}  // namespace rv

using namespace rv;

extern "C" {

rv_status rv_chain_absorb(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z, int32_t n_ch,
                          const double *chain_m, const double *chain_x, int32_t cap, int32_t *idx, int32_t *count,
                          double *r_chain, void *stream) {
    NvtxRange nvtx_range("rv_chain_absorb");
    if (!c) return RV_E_INVAL;
    if (!c->ws) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (n < 0 || n > c->n_max || n_ch < 1 || n_ch > kMaxChain || !chain_m || !chain_x || cap < 0 ||
        (cap > 0 && !idx) || !count)
        return set_err(c, RV_E_INVAL, "bad absorption arguments");
    if (n > 0 && (!x || !y || !z)) return set_err(c, RV_E_INVAL, "null star array");
    cudaStream_t s = (cudaStream_t)stream;
    Workspace &w = c->w;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8));
    absorb_setup_k<<<1, 32, 0, s>>>(n_ch, chain_m, chain_x, w.st);
    count_launch(c);
    int *total = &w.st->n_pert;   // scratch for the scan's total
    if (n > 0) {
        absorb_flag_k<<<grid, 256, 0, s>>>(n, x, y, z, w.st, w.sel_flag);
        count_launch(c);
        rv_status r = exclusive_scan(c, w.sel_flag, n, nullptr, total, s);
        if (r != RV_OK) return r;
    }
    absorb_write_k<<<grid, 256, 0, s>>>(n, x, y, z, w.st, w.sel_flag, total, cap, idx, count, r_chain);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "chain absorption");
}

rv_status rv_chain_escape(int32_t n_ch, const double *m, const double *x, const double *v, const int32_t *massive,
                          int32_t designated, double r_chain0, double gamma, int32_t n_absorbing, int32_t *escape,
                          rv_chain_escape_result *res) {
    if (n_ch < 1 || n_ch > kMaxChain || !m || !x || !v || !massive || !escape || !res || designated < 0 ||
        designated >= n_ch || !(r_chain0 >= 0.0) || !(gamma >= 0.0))
        return RV_E_INVAL;
    double M = 0.0, c[3] = {0.0, 0.0, 0.0}, vc[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < n_ch; k++) {
        M += m[k];
        for (int a = 0; a < 3; a++) {
            c[a] += m[k] * x[3 * k + a];
            vc[a] += m[k] * v[3 * k + a];
        }
    }
    for (int a = 0; a < 3; a++) {
        c[a] = M > 0.0 ? c[a] / M : 0.0;
        vc[a] = M > 0.0 ? vc[a] / M : 0.0;
    }
    const double r_esc = gamma * r_chain0;
    const double re2 = r_esc * r_esc;
    double rc2 = 0.0;
    for (int k = 0; k < n_ch; k++) {
        const double d[3] = {x[3 * k] - c[0], x[3 * k + 1] - c[1], x[3 * k + 2] - c[2]};
        const double u[3] = {v[3 * k] - vc[0], v[3 * k + 1] - vc[1], v[3 * k + 2] - vc[2]};
        const double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        const double du = (d[0] * u[0] + d[1] * u[1]) + d[2] * u[2];
        rc2 = std::max(rc2, d2);
        escape[k] = (d2 > re2 && du > 0.0) ? 1 : 0;
    }
    // absorption goes first: escapes wait while perturbers are being absorbed,
    // unless the chain radius is more than 5 % over the escape radius
    const double grown = 1.05 * r_esc;
    if (n_absorbing > 0 && !(rc2 > grown * grown))
        for (int k = 0; k < n_ch; k++) escape[k] = 0;
    int left = 0;
    for (int k = 0; k < n_ch; k++) left += escape[k] ? 0 : 1;
    int terminate = left < 2 ? 1 : 0;
    int des = designated;
    if (escape[des]) {
        int best = -1;
        for (int k = 0; k < n_ch; k++)
            if (massive[k] && !escape[k] && (best < 0 || m[k] > m[best])) best = k;
        if (best >= 0) des = best;
        else terminate = 1;
    }
    res->escape_count = n_ch - left;
    res->terminate = terminate;
    res->designated = des;
    res->r_chain = sqrt(rc2);
    res->r_escape = r_esc;
    return RV_OK;
}

}  // extern "C"
