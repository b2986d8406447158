// blocks.cu -- individual hierarchical block time steps (Sect. 2: the tree
// code advances particles on a hierarchy of time-step levels) in
// kick-drift-kick form, with walks restricted to the groups that hold an
// active star.
//
// Star i sits on level l_i: its step is dt_max / 2^l_i; the finest level L
// sets the substep dt_min = dt_max / 2^L. Substep n -> n + 1 drifts every star
// and the chain by dt_min; the stars whose step ends at n + 1 (n + 1 a
// multiple of 2^(L - l_i)) are active: the tree is rebuilt from all stars,
// only the groups holding an active star are walked, active stars get their
// closing half kick, a new level (criteria below; a coarser level only where
// it is synchronised), and the opening half kick of their next step. The
// chain members move on the finest level.
//
// Level criteria (reading of the paper's tau_acc, tau_vel accuracy
// parameters, Sect. 3): dt_i = min(tau_acc sqrt(eps / |a|), tau_vel eps / |v|),
// level = smallest l in [0, L] with dt_max 2^-l <= dt_i (L if none), all in
// FP64 with one rounding per operation on the FP32 a and v.
#include <algorithm>

#include "rv_internal.cuh"

namespace rv {

// (a level outside [0, L] is read as the nearest bound)
__device__ __forceinline__ bool is_active(int lvl, long long n, int L) {
    lvl = min(max(lvl, 0), L);
    const long long mask = (1ll << (L - lvl)) - 1;
    return (n & mask) == 0;
}

// gact[g] = 1 if group g holds a star whose step ends at substep n; counts active stars
__global__ void block_groups_k(const int4 *groups, const int *ngroup, const int *perm, const int8_t *level,
                               long long n, int L, uint8_t *gact, unsigned long long *count) {
    const int ng = *ngroup;
    unsigned long long act = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int4 r = groups[2 * g];   // (first, count, ...)
        int a = 0;
        for (int i = r.x; i < r.x + r.y; i++) a += is_active(level[perm[i]], n, L) ? 1 : 0;
        gact[g] = a > 0;
        act += (unsigned long long)a;
    }
    for (int o = 16; o > 0; o >>= 1) act += __shfl_xor_sync(0xffffffffu, act, o);
    if ((threadIdx.x & 31) == 0 && act) atomicAdd(count, act);
}

__global__ void drift_all_k(int64_t n, float *x, float *y, float *z, const float *vx, const float *vy,
                            const float *vz, float dt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fmaf(vx[i], dt, x[i]);
        y[i] = fmaf(vy[i], dt, y[i]);
        z[i] = fmaf(vz[i], dt, z[i]);
    }
}

// Level from the criteria (FP64, fixed operation order).
__device__ __forceinline__ int level_of(float ax, float ay, float az, float vx, float vy, float vz, double dt_max,
                                        int L, double tau_acc, double tau_vel, double eps) {
    const double a2 = __dadd_rn(__dadd_rn(__dmul_rn((double)ax, (double)ax), __dmul_rn((double)ay, (double)ay)),
                                __dmul_rn((double)az, (double)az));
    const double v2 = __dadd_rn(__dadd_rn(__dmul_rn((double)vx, (double)vx), __dmul_rn((double)vy, (double)vy)),
                                __dmul_rn((double)vz, (double)vz));
    double dt = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    if (a2 > 0.0) dt = __dmul_rn(tau_acc, __dsqrt_rn(__ddiv_rn(eps, __dsqrt_rn(a2))));
    if (v2 > 0.0) dt = fmin(dt, __ddiv_rn(__dmul_rn(tau_vel, eps), __dsqrt_rn(v2)));
    int l = 0;
    double step = dt_max;
    while (l < L && step > dt) {
        step *= 0.5;   // exact
        l++;
    }
    return l;
}

// Active stars (their step ends at substep n): closing half kick with the old
// level, a new level (adapt), opening half kick with it. start = 1: every star
// is at the start of a step (no closing kick, any level allowed).
__global__ void block_kick_k(int64_t n_st, float *vx, float *vy, float *vz, const float *ax, const float *ay,
                             const float *az, int8_t *level, long long n, int L, double dt_max, double tau_acc,
                             double tau_vel, double eps, int adapt, int start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_st;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lvl = min(max((int)level[i], 0), L);
        if (!start && !is_active(lvl, n, L)) continue;
        float u = vx[i], v = vy[i], w = vz[i];
        if (!start) {
            const float h = (float)(0.5 * ldexp(dt_max, -lvl));
            u = fmaf(ax[i], h, u); v = fmaf(ay[i], h, v); w = fmaf(az[i], h, w);
        }
        if (adapt) {
            int nl = level_of(ax[i], ay[i], az[i], u, v, w, dt_max, L, tau_acc, tau_vel, eps);
            // a finer level may start now; a coarser one only where its step boundary is now
            if (!start)
                while (nl < lvl && !is_active(nl, n, L)) nl++;
            lvl = nl;
            level[i] = (int8_t)lvl;
        }
        const float h = (float)(0.5 * ldexp(dt_max, -lvl));
        vx[i] = fmaf(ax[i], h, u); vy[i] = fmaf(ay[i], h, v); vz[i] = fmaf(az[i], h, w);
    }
}

// The level rule alone, for stars active at substep n (start: all, unconstrained).
__global__ void block_levels_k(int64_t n_st, const float *ax, const float *ay, const float *az, const float *vx,
                               const float *vy, const float *vz, int8_t *level, long long n, int L, double dt_max,
                               double tau_acc, double tau_vel, double eps, int start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_st;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int lvl = min(max((int)level[i], 0), L);
        if (!start && !is_active(lvl, n, L)) continue;
        int nl = level_of(ax[i], ay[i], az[i], vx[i], vy[i], vz[i], dt_max, L, tau_acc, tau_vel, eps);
        if (!start)
            while (nl < lvl && !is_active(nl, n, L)) nl++;
        level[i] = (int8_t)nl;
    }
}

rv_status block_levels(rv_ctx *c, int64_t n_st, const float *ax, const float *ay, const float *az, const float *vx,
                       const float *vy, const float *vz, const rv_blocks *b, int start, cudaStream_t s) {
    if (n_st > 0) {
        block_levels_k<<<(int)std::max<int64_t>(1, std::min<int64_t>((n_st + 255) / 256, (int64_t)c->num_sms * 8)), 256,
                         0, s>>>(n_st, ax, ay, az, vx, vy, vz, b->level, b->substep, b->max_level, b->dt_max,
                                 b->tau_acc, b->tau_vel, b->eps, start);
        count_launch(c);
    }
    return cuda_check(c, cudaGetLastError(), "block levels");
}

__global__ void chain_kick_k(int n, double *cv, const double *ca, double hdt) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * n; k += gridDim.x * blockDim.x) cv[k] += ca[k] * hdt;
}

__global__ void chain_drift_k(int n, double *cx, const double *cv, double dt) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * n; k += gridDim.x * blockDim.x) cx[k] += cv[k] * dt;
}

void launch_block_groups(rv_ctx *c, const BlockSel &b, cudaStream_t s) {
    Workspace &w = c->w;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((c->n + 255) / 256, (int64_t)c->num_sms * 4));
    block_groups_k<<<grid, 256, 0, s>>>(w.groups, &w.st->ngroup, w.perm, b.level, b.n, b.L, w.gact, w.block_count);
    count_launch(c);
}

static int grid_of(rv_ctx *c, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8));
}

static void chain_kick(rv_ctx *c, rv_system *sys, double hdt, cudaStream_t s) {
    if (sys->n_chain <= 0) return;
    const int nc = system_chains(sys) * sys->n_chain;
    chain_kick_k<<<ceil_div(3 * nc, 128), 128, 0, s>>>(nc, sys->chain_v, sys->chain_a, hdt);
    count_launch(c);
}

rv_status block_start(rv_ctx *c, rv_system *sys, rv_blocks *b, cudaStream_t s) {
    rv_status r = system_forces(c, sys, s);
    if (r != RV_OK) return r;
    const double dt_min = ldexp(b->dt_max, -b->max_level);
    if (sys->n > 0) {
        block_kick_k<<<grid_of(c, sys->n), 256, 0, s>>>(sys->n, sys->vx, sys->vy, sys->vz, sys->ax, sys->ay, sys->az,
                                                        b->level, 0, b->max_level, b->dt_max, b->tau_acc, b->tau_vel,
                                                        b->eps, b->adapt, 1);
        count_launch(c);
    }
    chain_kick(c, sys, 0.5 * dt_min, s);
    b->substep = 0;
    r = cuda_check(c, cudaMemsetAsync(c->w.block_count, 0, 16, s), "block counters");
    if (r != RV_OK) return r;
    return cuda_check(c, cudaGetLastError(), "block start");
}

rv_status block_steps(rv_ctx *c, rv_system *sys, rv_blocks *b, int nsub, cudaStream_t s) {
    const int L = b->max_level;
    const double dt_min = ldexp(b->dt_max, -L);
    for (int k = 0; k < nsub; k++) {
        if (sys->n > 0) {
            drift_all_k<<<grid_of(c, sys->n), 256, 0, s>>>(sys->n, sys->x, sys->y, sys->z, sys->vx, sys->vy, sys->vz,
                                                           (float)dt_min);
            count_launch(c);
        }
        if (sys->n_chain > 0) {
            const int nc = system_chains(sys) * sys->n_chain;
            chain_drift_k<<<ceil_div(3 * nc, 128), 128, 0, s>>>(nc, sys->chain_x, sys->chain_v, dt_min);
            count_launch(c);
        }
        const long long n = b->substep + 1;
        // the tree of all stars, then only the groups holding an active star
        const BlockSel sel{b->level, n, L};
        rv_status r = system_forces(c, sys, s, &sel);
        if (r != RV_OK) return r;
        if (sys->n > 0) {
            block_kick_k<<<grid_of(c, sys->n), 256, 0, s>>>(sys->n, sys->vx, sys->vy, sys->vz, sys->ax, sys->ay,
                                                            sys->az, b->level, n, L, b->dt_max, b->tau_acc,
                                                            b->tau_vel, b->eps, b->adapt, 0);
            count_launch(c);
        }
        chain_kick(c, sys, 0.5 * dt_min, s);   // closing and opening half kicks of the finest level
        chain_kick(c, sys, 0.5 * dt_min, s);
        b->substep = n;
    }
    return cuda_check(c, cudaGetLastError(), "block steps");
}

}  // namespace rv
