// rv_api.cu -- the extern "C" entry points of librv: argument checks,
// workspace layout, and dispatch to the kernels in build.cu, walk.cu and
// chain.cu.
#include <stdarg.h>

#include <algorithm>
#include <stdlib.h>
#include <string.h>

#include "rv_internal.cuh"

namespace rv {

rv_status set_err(rv_ctx *c, rv_status s, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

rv_status cuda_check(rv_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return RV_OK;
    return set_err(c, RV_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int64_t cell_capacity(int64_t n, int n_leaf) {
    int64_t nn = n > 0 ? n : 1;
    int64_t per_level = std::min<int64_t>(nn, 8 * nn / (n_leaf + 1) + 8);
    int64_t worst = 2 + (int64_t)kMaxLevel * per_level;
    int64_t typical = 96 + 3 * (8 * nn / (n_leaf + 1));
    return std::min(worst, typical);
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

size_t layout(int64_t n_max, const rv_config &cfg, char *base, Workspace *w, int64_t *cell_cap) {
    int64_t n = n_max > 0 ? n_max : 1;
    int64_t cap = cell_capacity(n, cfg.n_leaf);
    if (cell_cap) *cell_cap = cap;
    int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    int64_t nblk = (n + kTopoBlock - 1) / kTopoBlock;
    int64_t scan_max = std::max<int64_t>(std::max<int64_t>((int64_t)kSortBins * ntiles, (int64_t)kLevels * nblk),
                                         std::max<int64_t>(cap, n));
    int64_t nparts = std::max<int64_t>(6 * 1024, scan_max / kScanChunk + 2);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    Workspace t;
    t.key_a = (uint64_t *)take(8 * n);
    t.key_b = (uint64_t *)take(8 * n);
    t.idx_a = (int *)take(4 * n);
    t.idx_b = (int *)take(4 * n);
    t.hist = (int *)take(4 * (size_t)kSortBins * ntiles);
    t.skey = nullptr;
    t.perm = nullptr;
    t.pos = (float4 *)take(16 * n);
    t.dlev = (uint8_t *)take(n);
    t.lam = (uint8_t *)take(n);
    t.lvcnt = (int *)take(4 * (size_t)kLevels * nblk);
    t.cbox = (int4 *)take(16 * cap);
    t.clink = (int *)take(16 * cap);
    t.cmom = (float4 *)take(48 * cap);
    t.coct = (float4 *)take(48 * cap);
    t.cparent = (int *)take(4 * cap);
    t.carrive = (int *)take(4 * cap);
    t.gcnt = (int *)take(4 * cap);
    t.groups = (int4 *)take(32 * (n + 1));   // every group holds a star
    t.gact = (uint8_t *)take(n + 1);
    t.scost = (float *)take(4 * n);
    t.gorder = (int *)take(4 * (n + 1));
    t.gbin = (int *)take(4 * (n + 1));
    t.obins = (int *)take(4 * 1024);
    t.block_count = (unsigned long long *)take(16);
    t.partials = (int *)take(4 * nparts);
    t.pert_idx = (int *)take(4 * kPertTotal);
    t.pert_m = (double *)take(8 * kPertTotal);
    t.pert_x = (double *)take(24 * kPertTotal);
    t.pert_a = (double *)take(24 * kPertTotal);
    t.pert_pot = (double *)take(8 * kPertTotal);
    t.chain_ext_a = (double *)take(24 * kChainTotal);
    t.chain_ext_pot = (double *)take(8 * kChainTotal);
    t.out8 = (double *)take(8 * 16 * kMaxMembers);
    t.extra_xyzm = (float *)take(16 * kExtraTotal);
    t.extra_eps = (float *)take(4 * kExtraTotal);
    t.extra_out = (float *)take(16 * kExtraTotal);
    t.extra_quad = (float4 *)take(32 * kExtraTotal);
    t.pflag = (uint8_t *)take(n);
    t.red = (double *)take(8 * 9 * kRedSlots);
    t.sel_flag = (int *)take(4 * n);
    t.moff = (int64_t *)take(8 * (kMaxMembers + 1));
    t.mbounds = (double *)take(8 * 5 * kMaxMembers);
    t.mroot = (int *)take(4 * kMaxMembers);
    t.bpart = (float *)take(4 * 6 * 2048);
    t.xmem = (int *)take(4 * kExtraTotal);
    t.npert = (int *)take(4 * kMaxMembers);
    t.gstack = (int *)take(4 * (size_t)kStackSpillWarps * kStackSpill);
    t.st = (DevState *)take(sizeof(DevState));
    if (w) *w = t;
    return off;
}

static bool config_ok(const rv_config *cfg) {
    return cfg && cfg->theta >= 0.f && cfg->theta < 2.f && cfg->eps_star >= 0.f && cfg->n_leaf >= 1 &&
           cfg->n_leaf <= 64 && cfg->group >= 1 && cfg->group <= kMaxGroup && (cfg->quadrupole == 0 || cfg->quadrupole == 1) &&
           cfg->tile >= 32 && cfg->tile <= 256 && cfg->tile % 32 == 0 && (cfg->mac == 0 || cfg->mac == 1) &&
           cfg->alpha >= 0.f && cfg->alpha < 3e38f && (cfg->softening == 0 || cfg->softening == 1);
}

static bool ready(rv_ctx *c) { return c && c->ws; }

}  // namespace rv

using namespace rv;

extern "C" {

void rv_default_config(rv_config *cfg) {
    if (!cfg) return;
    cfg->theta = 0.5f;
    cfg->eps_star = 0.01f;
    cfg->n_leaf = 16;
    cfg->group = 32;
    cfg->quadrupole = 1;
    cfg->tile = 64;
    cfg->mac = 0;
    cfg->alpha = 1e-3f;
    cfg->softening = 0;
}

size_t rv_workspace_size(int64_t n_max, const rv_config *cfg) {
    if (!config_ok(cfg) || n_max < 0) return 0;
    return layout(n_max, *cfg, nullptr, nullptr, nullptr);
}

rv_status rv_create(rv_ctx **out, int64_t n_max, const rv_config *cfg) {
    if (!out) return RV_E_INVAL;
    *out = nullptr;
    if (!config_ok(cfg) || n_max < 0 || n_max > (int64_t)1 << 30) return RV_E_INVAL;
    int64_t cap = cell_capacity(n_max, cfg->n_leaf);
    if (cap >= ((int64_t)1 << 27)) return RV_E_INVAL;  // child ranges are packed as (first << 4 | count)
    rv_ctx *c = (rv_ctx *)calloc(1, sizeof(rv_ctx));
    if (!c) return RV_E_INVAL;
    c->cfg = *cfg;
    c->n_members = 1;
    c->n_max = n_max;
    c->cell_cap = cap;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        free(c);
        return RV_E_CUDA;
    }
    *out = c;
    return RV_OK;
}

void rv_destroy(rv_ctx *c) {
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (int k = 0; k < 2 * c->cap_walk_events; k++)
        if (c->walk_events[k]) cudaEventDestroy(c->walk_events[k]);
    free(c->walk_events);
    free(c);
}

rv_status rv_profile_walk(rv_ctx *c, int32_t enable) {
    if (!c) return RV_E_INVAL;
    c->profile_walk = enable != 0;
    c->n_walk_events = 0;
    return RV_OK;
}

rv_status rv_walk_time(rv_ctx *c, double *total_ms, int64_t *launches) {
    if (!c || !total_ms || !launches) return RV_E_INVAL;
    double t = 0.0;
    for (int k = 0; k < c->n_walk_events; k++) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(c->walk_events[2 * k + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->walk_events[2 * k], c->walk_events[2 * k + 1]);
        if (e != cudaSuccess) return cuda_check(c, e, "walk time");
        t += ms;
    }
    *total_ms = t;
    *launches = c->n_walk_events;
    return RV_OK;
}

rv_status rv_set_workspace(rv_ctx *c, void *dev, size_t bytes) {
    if (!c || !dev) return RV_E_INVAL;
    size_t need = layout(c->n_max, c->cfg, nullptr, nullptr, nullptr);
    if (bytes < need || ((uintptr_t)dev & 255))
        return set_err(c, RV_E_WORKSPACE, "workspace: need %zu bytes, 256-aligned; got %zu", need, bytes);
    c->ws = (char *)dev;
    c->ws_bytes = bytes;
    layout(c->n_max, c->cfg, c->ws, &c->w, &c->cell_cap);
    c->built = false;
    c->moff_on_device = false;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    cudaError_t e = cudaMemset(c->w.st, 0, sizeof(DevState));
    return cuda_check(c, e, "workspace init");
}

rv_status rv_build_tree(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z, const float *m,
                        void *stream) {
    NvtxRange nvtx_range("rv_build_tree");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (n < 0 || n > c->n_max) return set_err(c, RV_E_INVAL, "n = %lld outside [0, %lld]", (long long)n, (long long)c->n_max);
    if (n > 0 && (!x || !y || !z || !m)) return set_err(c, RV_E_INVAL, "null star array");
    const int64_t off[2] = {0, n};
    return build_tree(c, 1, off, x, y, z, m, (cudaStream_t)stream);
}

static rv_status check_offsets(rv_ctx *c, int M, const int64_t *off, int64_t n) {
    if (M < 1 || M > kMaxMembers || !off) return set_err(c, RV_E_INVAL, "need 1 <= n_members <= %d and offsets", kMaxMembers);
    if (off[0] != 0 || off[M] != n) return set_err(c, RV_E_INVAL, "offsets must run from 0 to n");
    for (int k = 0; k < M; k++)
        if (off[k + 1] < off[k]) return set_err(c, RV_E_INVAL, "offsets must not decrease");
    return RV_OK;
}

rv_status rv_build_tree_members(rv_ctx *c, int32_t n_members, const int64_t *offsets, const float *x,
                                const float *y, const float *z, const float *m, void *stream) {
    NvtxRange nvtx_range("rv_build_tree_members");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (!offsets || n_members < 1) return set_err(c, RV_E_INVAL, "bad members");
    const int64_t n = offsets[n_members > kMaxMembers ? 0 : n_members];
    rv_status r = check_offsets(c, n_members, offsets, n);
    if (r != RV_OK) return r;
    if (n > c->n_max) return set_err(c, RV_E_INVAL, "n = %lld above n_max %lld", (long long)n, (long long)c->n_max);
    if (n > 0 && (!x || !y || !z || !m)) return set_err(c, RV_E_INVAL, "null star array");
    return build_tree(c, n_members, offsets, x, y, z, m, (cudaStream_t)stream);
}

rv_status rv_tree_forces(rv_ctx *c, float theta, float eps_star, int32_t n_extra, const float *extra_xyzm,
                         const float *extra_eps, float *ax, float *ay, float *az, float *pot, float *extra_out,
                         void *stream) {
    NvtxRange nvtx_range("rv_tree_forces");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (!c->built) return set_err(c, RV_E_NOTBUILT, "rv_tree_forces before rv_build_tree");
    if (!(theta >= 0.f && theta < 2.f) || !(eps_star >= 0.f)) return set_err(c, RV_E_INVAL, "bad theta/eps");
    if (n_extra < 0 || n_extra > kMaxExtra) return set_err(c, RV_E_INVAL, "n_extra must be in [0, %d]", kMaxExtra);
    if (n_extra > 0 && (!extra_xyzm || !extra_eps || !extra_out)) return set_err(c, RV_E_INVAL, "null extra array");
    if (c->n > 0 && (!ax || !ay || !az || !pot)) return set_err(c, RV_E_INVAL, "null output array");
    return tree_walk(c, theta, eps_star, n_extra, extra_xyzm, extra_eps, nullptr, 0, ax, ay, az, pot, extra_out,
                     (cudaStream_t)stream);
}

rv_status rv_tree_forces_rel(rv_ctx *c, float alpha, float eps_star, const float *ref_ax, const float *ref_ay,
                             const float *ref_az, float *ax, float *ay, float *az, float *pot, void *stream) {
    NvtxRange nvtx_range("rv_tree_forces_rel");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (!c->built) return set_err(c, RV_E_NOTBUILT, "rv_tree_forces_rel before rv_build_tree");
    if (!(alpha >= 0.f) || !(alpha < 3e38f) || !(eps_star >= 0.f)) return set_err(c, RV_E_INVAL, "bad alpha/eps");
    if (c->n > 0 && (!ax || !ay || !az || !pot || !ref_ax || !ref_ay || !ref_az))
        return set_err(c, RV_E_INVAL, "null array");
    RelMac rel{alpha, ref_ax, ref_ay, ref_az};
    // groups without a reference yet use the context's opening angle
    return tree_walk(c, c->cfg.theta, eps_star, 0, nullptr, nullptr, nullptr, 0, ax, ay, az, pot, nullptr,
                     (cudaStream_t)stream, nullptr, &rel);
}

rv_status rv_tree_forces_members(rv_ctx *c, float theta, float eps_star, int32_t n_extra, const float *extra_xyzm,
                                 const float *extra_eps, const int32_t *extra_member, float *ax, float *ay, float *az,
                                 float *pot, float *extra_out, void *stream) {
    NvtxRange nvtx_range("rv_tree_forces_members");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (!c->built) return set_err(c, RV_E_NOTBUILT, "rv_tree_forces_members before a build");
    if (!(theta >= 0.f && theta < 2.f) || !(eps_star >= 0.f)) return set_err(c, RV_E_INVAL, "bad theta/eps");
    if (n_extra < 0 || n_extra > kMaxExtra) return set_err(c, RV_E_INVAL, "n_extra must be in [0, %d]", kMaxExtra);
    if (n_extra > 0 && (!extra_xyzm || !extra_eps || !extra_out)) return set_err(c, RV_E_INVAL, "null extra array");
    if (c->n > 0 && (!ax || !ay || !az || !pot)) return set_err(c, RV_E_INVAL, "null output array");
    return tree_walk(c, theta, eps_star, n_extra, extra_xyzm, extra_eps, extra_member, 0, ax, ay, az, pot,
                     extra_out, (cudaStream_t)stream);
}

rv_status rv_perturber_forces(rv_ctx *c, int32_t n_ch, const double *chain_m, const double *chain_x,
                              int32_t n_pert, const double *pert_m, const double *pert_x, double *a_pert,
                              double *pot_pert, double *a_chain, double *pot_chain, double *out8, void *stream) {
    NvtxRange nvtx_range("rv_perturber_forces");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (n_ch < 1 || n_ch > kMaxChain || n_pert < 0 || n_pert > kMaxPert)
        return set_err(c, RV_E_INVAL, "need 1 <= n_ch <= %d and 0 <= n_pert <= %d", kMaxChain, kMaxPert);
    if (!chain_m || !chain_x || !a_chain || !pot_chain || !out8) return set_err(c, RV_E_INVAL, "null chain array");
    if (n_pert > 0 && (!pert_m || !pert_x || !a_pert || !pot_pert)) return set_err(c, RV_E_INVAL, "null perturber array");
    return perturber_forces(c, n_ch, chain_m, chain_x, n_pert, nullptr, pert_m, pert_x, a_pert, pot_pert, a_chain,
                            pot_chain, out8, (cudaStream_t)stream);
}

static rv_status check_system(rv_ctx *c, const rv_system *s) {
    if (!s) return set_err(c, RV_E_INVAL, "null system");
    if (s->n < 0 || s->n > c->n_max) return set_err(c, RV_E_INVAL, "system n outside [0, n_max]");
    const int M = std::max(1, (int)s->n_members);
    if (s->n_members > 1 || s->member_offsets) {
        rv_status r = check_offsets(c, M, s->member_offsets, s->n);
        if (r != RV_OK) return r;
    }
    if (s->n_chains < 0 || (int64_t)M * std::max(1, (int)s->n_chains) > kExtraTotal)
        return set_err(c, RV_E_INVAL, "more than %d chains", kExtraTotal);
    if ((int64_t)M * std::max(1, (int)s->n_chains) * s->n_chain > kChainTotal)
        return set_err(c, RV_E_INVAL, "more than %d chain members", kChainTotal);
    if (s->n > 0 && (!s->x || !s->y || !s->z || !s->vx || !s->vy || !s->vz || !s->m || !s->ax || !s->ay || !s->az ||
                     !s->pot))
        return set_err(c, RV_E_INVAL, "null star array in system");
    if (s->n_chain < 0 || s->n_chain > kMaxChain) return set_err(c, RV_E_INVAL, "n_chain outside [0, %d]", kMaxChain);
    if (s->n_chain > 0 && (!s->chain_m || !s->chain_x || !s->chain_v || !s->chain_a || !s->chain_pot))
        return set_err(c, RV_E_INVAL, "null chain array in system");
    if (s->n_chain > 0 && (s->pert_mode < 0 || s->pert_mode > 3)) return set_err(c, RV_E_INVAL, "bad pert_mode");
    if (s->n_chain > 0 && s->pert_mode == 3 && (!(s->pert_gamma > 0.f) || !(s->pert_radius >= 0.f)))
        return set_err(c, RV_E_INVAL, "tidal selection needs pert_gamma > 0 and pert_radius >= 0");
    if (s->pert_mode == 2 && (s->pert_k < 0 || s->pert_k > kMaxPert)) return set_err(c, RV_E_INVAL, "bad pert_k");
    return RV_OK;
}

rv_status rv_system_forces(rv_ctx *c, rv_system *sys, void *stream) {
    NvtxRange nvtx_range("rv_system_forces");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    rv_status r = check_system(c, sys);
    if (r != RV_OK) return r;
    return system_forces(c, sys, (cudaStream_t)stream);
}

rv_status rv_kdk_step(rv_ctx *c, rv_system *sys, double dt, int32_t nsteps, void *stream) {
    NvtxRange nvtx_range("rv_kdk_step");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    rv_status r = check_system(c, sys);
    if (r != RV_OK) return r;
    if (nsteps < 0 || !(dt == dt)) return set_err(c, RV_E_INVAL, "bad dt/nsteps");
    return kdk(c, sys, dt, nsteps, (cudaStream_t)stream);
}

rv_status rv_kdk_step_graph(rv_ctx *c, rv_system *sys, double dt, int32_t nsteps, double *energy_out,
                            void *stream) {
    NvtxRange nvtx_range("rv_kdk_step_graph");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    rv_status r = check_system(c, sys);
    if (r != RV_OK) return r;
    if (nsteps < 0 || !(dt == dt)) return set_err(c, RV_E_INVAL, "bad dt/nsteps");
    cudaStream_t s = (cudaStream_t)stream;
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return set_err(c, RV_E_INVAL, "graph capture needs a created stream");
    return kdk_graph(c, sys, dt, nsteps, energy_out, s);
}

rv_status rv_energy(rv_ctx *c, const rv_system *sys, double *out, void *stream) {
    NvtxRange nvtx_range("rv_energy");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    rv_status r = check_system(c, sys);
    if (r != RV_OK) return r;
    if (!out) return set_err(c, RV_E_INVAL, "null out");
    return energy(c, sys, out, (cudaStream_t)stream);
}

rv_status rv_select_perturbers(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z,
                               const float centre[3], int32_t mode, float radius, int32_t k, int32_t cap,
                               int32_t *idx, int32_t *count, void *stream) {
    NvtxRange nvtx_range("rv_select_perturbers");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (n < 0 || n > c->n_max || !centre || !idx || !count || cap < 0 || (mode != 1 && mode != 2))
        return set_err(c, RV_E_INVAL, "bad selection arguments");
    if (n > 0 && (!x || !y || !z)) return set_err(c, RV_E_INVAL, "null star array");
    if (mode == 1 && !(radius >= 0.f)) return set_err(c, RV_E_INVAL, "bad radius");
    const float c4[4] = {centre[0], centre[1], centre[2], 0.f};
    return select_perturbers(c, n, x, y, z, nullptr, c4, mode, radius, k, cap, idx, count, (cudaStream_t)stream);
}

rv_status rv_chain_perturber_forces(rv_ctx *c, const rv_system *sys, double dt, const double *chain_x,
                                    double *a_chain, double *pot_chain, void *stream) {
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    rv_status r = check_system(c, sys);
    if (r != RV_OK) return r;
    if (sys->n_chain <= 0 || !chain_x || !a_chain) return set_err(c, RV_E_INVAL, "needs a chain and its arrays");
    if (c->pert_members != system_chains(sys))
        return set_err(c, RV_E_NOTBUILT, "rv_chain_perturber_forces before rv_system_forces of this system");
    if (!(dt == dt)) return set_err(c, RV_E_INVAL, "bad dt");
    return chain_perturber_forces(c, sys, dt, chain_x, a_chain, pot_chain, (cudaStream_t)stream);
}

static rv_status check_blocks(rv_ctx *c, const rv_system *sys, const rv_blocks *b) {
    if (!b) return set_err(c, RV_E_INVAL, "null block parameters");
    if (!(b->dt_max > 0.0) || b->max_level < 0 || b->max_level > 20 || (sys->n > 0 && !b->level))
        return set_err(c, RV_E_INVAL, "bad block parameters (dt_max > 0, max_level 0..20, level array)");
    if (b->adapt && !(b->tau_acc > 0.f && b->tau_vel > 0.f && b->eps > 0.f))
        return set_err(c, RV_E_INVAL, "adaptive levels need tau_acc, tau_vel, eps > 0");
    return RV_OK;
}

rv_status rv_block_start(rv_ctx *c, rv_system *sys, rv_blocks *b, void *stream) {
    NvtxRange nvtx_range("rv_block_start");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    rv_status r = check_system(c, sys);
    if (r == RV_OK) r = check_blocks(c, sys, b);
    if (r != RV_OK) return r;
    return block_start(c, sys, b, (cudaStream_t)stream);
}

rv_status rv_block_steps(rv_ctx *c, rv_system *sys, rv_blocks *b, int32_t nsub, void *stream) {
    NvtxRange nvtx_range("rv_block_steps");
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    rv_status r = check_system(c, sys);
    if (r == RV_OK) r = check_blocks(c, sys, b);
    if (r != RV_OK) return r;
    if (nsub < 0) return set_err(c, RV_E_INVAL, "nsub < 0");
    return block_steps(c, sys, b, nsub, (cudaStream_t)stream);
}

rv_status rv_block_levels(rv_ctx *c, int64_t n, const float *ax, const float *ay, const float *az, const float *vx,
                          const float *vy, const float *vz, rv_blocks *b, int32_t start, void *stream) {
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (n < 0 || (n > 0 && (!ax || !ay || !az || !vx || !vy || !vz))) return set_err(c, RV_E_INVAL, "bad arrays");
    if (!b || !(b->dt_max > 0.0) || b->max_level < 0 || b->max_level > 20 || (n > 0 && !b->level) ||
        !(b->tau_acc > 0.f && b->tau_vel > 0.f && b->eps > 0.f))
        return set_err(c, RV_E_INVAL, "bad block parameters");
    return block_levels(c, n, ax, ay, az, vx, vy, vz, b, start ? 1 : 0, (cudaStream_t)stream);
}

rv_status rv_block_count(rv_ctx *c, int64_t *active_updates, void *stream) {
    if (!c || !active_updates) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    unsigned long long v = 0;
    rv_status r = cuda_check(c, cudaMemcpyAsync(&v, c->w.block_count, sizeof v, cudaMemcpyDeviceToHost,
                                                (cudaStream_t)stream), "block count");
    if (r == RV_OK) r = cuda_check(c, cudaStreamSynchronize((cudaStream_t)stream), "block count");
    *active_updates = (int64_t)v;
    return r;
}

rv_status rv_chain_start_radius(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z, const float *vx,
                                const float *vy, const float *vz, const float *m, const float centre[3], double m_bh,
                                int32_t n_sigma, double alpha, double beta, double eps, double out[5], void *stream) {
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (n < 1 || n > c->n_max || !x || !y || !z || !vx || !vy || !vz || !m || !centre || !out || n_sigma < 1 ||
        !(m_bh > 0.0))
        return set_err(c, RV_E_INVAL, "bad chain start radius arguments");
    double o3[3];
    rv_status r = influence_radius(c, n, x, y, z, vx, vy, vz, m, centre, m_bh, n_sigma, o3, (cudaStream_t)stream);
    if (r != RV_OK) return r;
    const double r_infl = std::min(o3[0], o3[2]);
    out[0] = o3[0];
    out[1] = o3[1];
    out[2] = o3[2];
    out[3] = r_infl;
    out[4] = std::max(alpha * r_infl, beta * eps);
    return RV_OK;
}

rv_status rv_select_perturbers_tidal(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z,
                                     const float *m, const float centre[3], float m_chain, float gamma_crit,
                                     float r_crit, int32_t cap, int32_t *idx, int32_t *count, void *stream) {
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (n < 0 || n > c->n_max || !centre || !idx || !count || cap < 0) return set_err(c, RV_E_INVAL, "bad selection arguments");
    if (n > 0 && (!x || !y || !z || !m)) return set_err(c, RV_E_INVAL, "null star array");
    if (!(m_chain > 0.f) || !(gamma_crit > 0.f) || !(r_crit >= 0.f)) return set_err(c, RV_E_INVAL, "bad tidal parameters");
    const float c4[4] = {centre[0], centre[1], centre[2], m_chain};
    return select_perturbers(c, n, x, y, z, nullptr, c4, 3, r_crit, 0, cap, idx, count, (cudaStream_t)stream, m,
                             gamma_crit);
}

rv_status rv_get_tree(rv_ctx *c, rv_tree_view *out, void *stream) {
    if (!c || !out) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    if (!c->built) return set_err(c, RV_E_NOTBUILT, "no tree");
    cudaStream_t s = (cudaStream_t)stream;
    int sz[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(sz, &c->w.st->ncell, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(c, e, "get tree");
    out->n = c->n;
    out->ncell = std::min<int64_t>(sz[0], c->cell_cap);
    out->ngroup = sz[1];
    out->keys = c->w.skey;
    out->perm = c->w.perm;
    out->pos = reinterpret_cast<const float *>(c->w.pos);
    out->cbox = reinterpret_cast<const int32_t *>(c->w.cbox);
    out->clink = c->w.clink;
    out->cmom = reinterpret_cast<const float *>(c->w.cmom);
    out->cparent = c->w.cparent;
    out->groups = reinterpret_cast<const int32_t *>(c->w.groups);
    out->bounds = c->w.st->bounds;
    return RV_OK;
}

rv_status rv_walk_stats(rv_ctx *c, int64_t out[3], void *stream) {
    if (!c || !out) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long v[2];
    int hwm = 0;
    cudaError_t e = cudaMemcpyAsync(v, &c->w.st->n_p2p, sizeof(v), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hwm, &c->w.st->stack_hwm, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(c, e, "walk stats");
    out[0] = (int64_t)v[0];
    out[1] = (int64_t)v[1];
    out[2] = hwm;
    return RV_OK;
}

rv_status rv_sync_status(rv_ctx *c, void *stream) {
    if (!c) return RV_E_INVAL;
    if (!ready(c)) return set_err(c, RV_E_WORKSPACE, "no workspace");
    cudaStream_t s = (cudaStream_t)stream;
    int err = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&err, &c->w.st->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(&c->w.st->err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_check(c, e, "sync status");
    switch (err) {
        case kErrNone: return RV_OK;
        case kErrStack: return set_err(c, RV_E_STACK, "walk stack overflow (more than %d pending child ranges)", kStackCap);
        case kErrCells: return set_err(c, RV_E_WORKSPACE, "tree has more cells than the workspace holds (%lld)", (long long)c->cell_cap);
        case kErrPert: return set_err(c, RV_E_WORKSPACE, "more perturbers inside the radius than the output holds");
        case kErrPairs: return set_err(c, RV_E_WORKSPACE, "more recorded (group, cell) pairs than the buffer holds");
        case kErrTimeout: return set_err(c, RV_E_TIMEOUT, "a tensor-core completion wait timed out");
        default: return set_err(c, RV_E_CUDA, "unknown device error %d", err);
    }
}

int64_t rv_launch_count(const rv_ctx *c) { return c ? (int64_t)c->launches : 0; }

const char *rv_last_error(const rv_ctx *c) { return c ? c->err : "null context"; }

}  // extern "C"
