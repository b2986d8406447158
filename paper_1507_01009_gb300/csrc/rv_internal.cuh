// rv_internal.cuh -- context, workspace layout and small device helpers of librv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "rv.h"

#include <nvtx3/nvToolsExt.h>

namespace rv {

constexpr int kMaxLevel = 21;           // 21 bits per axis, levels 0..21
constexpr int kLevels = kMaxLevel + 1;  // 22
constexpr int kSortBits = 9;            // radix digit width
constexpr int kSortBins = 1 << kSortBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per tile
constexpr int kTopoBlock = 256;
constexpr int kScanChunk = 2048;        // elements per scan block
#ifndef RV_WALK_WARPS
#define RV_WALK_WARPS 1
#endif
constexpr int kWalkWarps = RV_WALK_WARPS;  // warps per walk block (each warp walks its own groups)
constexpr int kMaxGroup = 64;           // stars per walk group (two per lane)
constexpr int kStackCap = 1408;         // walk traversal stack entries per warp (64 a level, 22 levels)
constexpr int kStackSm = 256;           // of them in shared memory; the deeper ones in the spill area
constexpr int kStackSpill = kStackCap - kStackSm;
constexpr int kStackSpillWarps = 4096;  // walk warps the spill area serves (the walk's grid is capped to it)
constexpr int kMaxExtra = 8;            // extra particles through rv_tree_forces
constexpr int kMaxMembers = 512;        // independent systems built and walked together (9-bit sort digit)
constexpr int kBoundsChunk = 2048;      // stars per bounds/keys block within a member
constexpr int kPertTotal = 65536;       // perturber slots over all members
constexpr int kChainTotal = 2048;       // chain members over all members
constexpr int kExtraTotal = kMaxMembers;  // extra particles (chain centres) over all members
constexpr int kRedSlots = 1024;         // energy partial-sum blocks over all members
constexpr int kMaxChain = 250;
constexpr int kMaxPert = 5000;

// Error codes latched by kernels (first one wins).
enum DevErr : int { kErrNone = 0, kErrStack = 1, kErrCells = 2, kErrPert = 3, kErrPairs = 4, kErrTimeout = 5 };

// Device-resident scalars (one small block in the workspace).
struct DevState {
    int ncell;        // cells of the last build
    int ngroup;       // walk groups of the last build
    int next_group;   // walk work counter
    int err;          // latched DevErr
    int n_pert;       // perturbers selected by the last selection
    int stack_hwm;    // deepest walk stack seen
    int cost_n;       // stars whose walk costs scost holds (0: none)
    int pad;
    unsigned long long n_p2p, n_m2p;  // interaction counts of the last walk
    double bounds[5];                 // min x, y, z, L, 2^21 / L
    double absorb[4];                 // chain absorption: centre of mass x, y, z and the squared chain radius
    int lvoff[kLevels + 1];           // first cell of each level, then ncell
};

struct Workspace {
    // tree build
    uint64_t *key_a, *key_b;
    int *idx_a, *idx_b;
    int *hist;            // radix histograms [bins x tiles]
    uint64_t *skey;       // sorted keys of the last build (key_a or key_b)
    int *perm;            // sorted slot -> caller index of the last build (idx_a or idx_b)
    float4 *pos;          // sorted (x, y, z, m)
    uint8_t *dlev, *lam;  // per sorted star: first differing level with its predecessor, leaf level
    int *lvcnt;           // per (level, topo block) counts, scanned in place
    int4 *cbox;           // (ox, oy, oz, level)
    int *clink;           // [4 ncell] child first, child end, first star, end star
    float4 *cmom;         // [3 ncell]
    float4 *coct;         // [3 ncell] traceless octupoles (the learned correction's features only)
    int *cparent, *carrive;
    int *gcnt;            // groups of each cell, scanned in place to each cell's first group
    int4 *groups;         // 2 int4 per group: (first, count, lo x, lo y), (lo z, hi x, hi y, hi z)
    uint8_t *gact;        // block time steps: groups holding an active star
    float *scost;         // per caller star: list cost of its group in the last walk (scheduling only)
    int *gorder;          // the walk's queue order of the groups
    int *gbin;            // each group's cost bin (queue order scratch)
    int *obins;           // bin counts, then next free slots (queue order scratch, 1024)
    unsigned long long *block_count;  // block time steps: active star updates so far
    int *partials;        // scan block sums
    // perturbers and chain hand-off
    int *pert_idx;        // [kMaxPert]
    double *pert_m, *pert_x;           // [kMaxPert], [3 kMaxPert]
    double *pert_a, *pert_pot;         // [3 kMaxPert], [kMaxPert]
    double *chain_ext_a, *chain_ext_pot;  // [3 kMaxChain], [kMaxChain]
    double *out8;         // Eq. 3 correction, sub, potentials
    float *extra_xyzm, *extra_eps, *extra_out;  // [4 kMaxExtra], [kMaxExtra], [4 kMaxExtra]
    float4 *extra_quad;   // [2 kExtraTotal]: each chain's traceless quadrupole (xx, yy, zz, xy), (xz, yz, 0, 0)
    uint8_t *pflag;       // [n]: 1 for the stars that are perturbers of a chain (caller order)
    double *red;          // energy partial sums
    int *sel_flag;        // perturber selection flags (n)
    // members (independent systems sharing one build and one walk)
    int64_t *moff;        // member star offsets [kMaxMembers + 1]
    double *mbounds;      // per member: min x, y, z, L, 2^21 / L
    int *mroot;           // root cell of each member (-1 if empty)
    float *bpart;         // bounds partials
    int *xmem;            // member of each extra particle
    int *npert;           // perturbers selected per member
    int *gstack;          // walk stack entries beyond kStackSm, kStackSpill per warp [kStackSpillWarps]
    DevState *st;
};

}  // namespace rv

struct rv_ctx {
    rv_config cfg;
    int64_t n_max;
    int64_t n;            // stars in the last build
    int64_t cell_cap;
    int device;
    int num_sms;
    bool built;
    long long launches;   // kernels launched through this context
    char *ws;
    size_t ws_bytes;
    rv::Workspace w;
    int n_members;                          // members of the last build (>= 1)
    int64_t moff_host[rv::kMaxMembers + 1]; // their star offsets
    int64_t max_member;                     // largest member
    bool moff_on_device;                    // moff_host[0..n_members] already uploaded
    int pert_members;                       // members whose perturber sets the last force pass chose (0: none)
    // walk timing (rv_profile_walk): event pairs recorded around each walk launch
    bool profile_walk;
    int n_walk_events;
    int cap_walk_events;
    cudaEvent_t *walk_events;               // [2 cap_walk_events]
    // captured kick-drift-kick step (rv_kdk_step_graph)
    cudaGraphExec_t graph;
    long long graph_launches;
    unsigned long long graph_key;
    char err[512];
};

namespace rv {

// Workspace layout: one pass computes sizes (base == nullptr) or assigns pointers.
size_t layout(int64_t n_max, const rv_config &cfg, char *base, Workspace *w, int64_t *cell_cap);
int64_t cell_capacity(int64_t n_max, int n_leaf);

rv_status set_err(rv_ctx *c, rv_status s, const char *fmt, ...);
rv_status cuda_check(rv_ctx *c, cudaError_t e, const char *what);

// build.cu
rv_status build_tree(rv_ctx *c, int n_members, const int64_t *offsets, const float *x, const float *y,
                     const float *z, const float *m, cudaStream_t s);
rv_status upload_offsets(rv_ctx *c, int M, const int64_t *offsets, cudaStream_t s);
rv_status radix_sort(rv_ctx *c, int64_t n, int passes, uint64_t **keys, int **idx, bool identity_idx,
                     cudaStream_t s, bool member_pass = false);
rv_status exclusive_scan(rv_ctx *c, int *data, int64_t nmax, const int *d_len, int *d_total, cudaStream_t s);

// Opening test on integer grid distances: accept iff d^2 >= thr[level].
struct MacTable {
    unsigned long long thr[kLevels];
};
MacTable mac_table(float theta);

// walk.cu
// Record of (group, cell) pairs accepted at theta but opened at theta_rec.
struct PairRecord {
    float theta_rec;
    int2 *pairs;
    int *npairs;
    int cap;
};

// Relative opening criterion of a walk (see walk.cu): tolerance alpha and the
// stars' reference accelerations (device FP32 [n] each, caller order).
struct RelMac {
    float alpha;
    const float *rx, *ry, *rz;
};

// extra particles: xmem[k] = member of extra k (device), or nullptr when
// extra k belongs to member k (one chain per member) -- see walk.cu.
rv_status tree_walk(rv_ctx *c, float theta, float eps_star, int n_extra, const float *xyzm, const float *xeps,
                    const int *xmem, int extras_per_member, float *ax, float *ay, float *az, float *pot,
                    float *xout, cudaStream_t s, const PairRecord *rec = nullptr, const RelMac *rel = nullptr,
                    const uint8_t *gact = nullptr, const float4 *xquad = nullptr,
                    const uint8_t *xq_skip = nullptr);

// chain.cu
// mode 1 radius, 2 k nearest, 3 tidal (Eq. 2: radius = r_crit, star masses m, gamma);
// centre_dev / centre_host hold (x, y, z, chain mass)
rv_status select_perturbers(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z,
                            const float *centre_dev, const float *centre_host, int mode, float radius, int k,
                            int cap, int *idx, int *count, cudaStream_t s, const float *m = nullptr,
                            float gamma = 0.f);
rv_status influence_radius(rv_ctx *c, int64_t n, const float *x, const float *y, const float *z, const float *vx,
                           const float *vy, const float *vz, const float *m, const float centre[3], double m_bh,
                           int64_t n_sigma, double out[3], cudaStream_t s);
rv_status chain_perturber_forces(rv_ctx *c, const rv_system *sys, double dt, const double *chain_x, double *a_chain,
                                 double *pot_chain, cudaStream_t s);
rv_status perturber_forces(rv_ctx *c, int n_ch, const double *cm, const double *cx, int n_pert_max,
                           const int *d_npert, const double *pm, const double *px, double *a_pert,
                           double *pot_pert, double *a_chain, double *pot_chain, double *out8, cudaStream_t s);
// Block time steps: the stars' levels, the substep n that ends now, the finest level L.
struct BlockSel {
    const int8_t *level;
    long long n;
    int L;
};
// blk (optional): after the build, walk only the groups holding a star active at blk->n
rv_status system_forces(rv_ctx *c, rv_system *sys, cudaStream_t s, const BlockSel *blk = nullptr);
// blocks.cu
void launch_block_groups(rv_ctx *c, const BlockSel &b, cudaStream_t s);
rv_status block_start(rv_ctx *c, rv_system *sys, rv_blocks *b, cudaStream_t s);
rv_status block_steps(rv_ctx *c, rv_system *sys, rv_blocks *b, int nsub, cudaStream_t s);
rv_status block_levels(rv_ctx *c, int64_t n_st, const float *ax, const float *ay, const float *az, const float *vx,
                       const float *vy, const float *vz, const rv_blocks *b, int start, cudaStream_t s);
rv_status kdk(rv_ctx *c, rv_system *sys, double dt, int nsteps, cudaStream_t s);
void kick(rv_ctx *c, rv_system *sys, double dt, int drift, cudaStream_t s);
int system_members(const rv_system *sys);
int system_chains(const rv_system *sys);   // chains over all members (0 without a chain)
int chains_per_member(const rv_system *sys);
rv_status energy(rv_ctx *c, const rv_system *sys, double *out, cudaStream_t s);
rv_status kdk_graph(rv_ctx *c, rv_system *sys, double dt, int nsteps, double *eout, cudaStream_t s);

inline void count_launch(rv_ctx *c) { c->launches++; }

// A named NVTX range for the lifetime of the object: the library's entry points
// show up as ranges in a timeline profiler (a few nanoseconds without one).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Member holding star i: the largest m < M with moff[m] <= i (empty members
// are skipped because their successor has the same offset).
__device__ __forceinline__ int member_of(const int64_t *moff, int M, int64_t i) {
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (moff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- device helpers ----
__device__ __forceinline__ void latch_err(DevState *st, int code) { atomicCAS(&st->err, 0, code); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Neumaier compensated accumulation of a tile sum x into (s, c).
__device__ __forceinline__ void nadd(float &s, float &c, float x) {
    float t = __fadd_rn(s, x);
    if (fabsf(s) >= fabsf(x))
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), x));
    else
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), s));
    s = t;
}

__host__ __device__ __forceinline__ int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Geometric centre of the grid box b = (ox, oy, oz, level) in FP32:
// lo + (o + side/2) * unit, every operation rounded once, so that the tree
// build and the walk get the same value. (o + side/2 is exact in FP32.)
__device__ __forceinline__ void geo_centre(const int4 b, const float lo[3], float unit, float g[3]) {
    float half = __int_as_float((127 + kMaxLevel - 1 - b.w) << 23);  // 2^(20 - level)
    g[0] = __fadd_rn(lo[0], __fmul_rn(__fadd_rn((float)b.x, half), unit));
    g[1] = __fadd_rn(lo[1], __fmul_rn(__fadd_rn((float)b.y, half), unit));
    g[2] = __fadd_rn(lo[2], __fmul_rn(__fadd_rn((float)b.z, half), unit));
}

// Centre of the grid box [blo, bhi) in FP32: lo + (blo + bhi) * (unit / 2),
// each operation rounded once (blo + bhi is exact in FP32 for boxes inside
// the grid, unit / 2 is exact).
__device__ __forceinline__ void box_centre(const int blo[3], const int bhi[3], const float lo[3], float unit,
                                           float g[3]) {
    const float hu = 0.5f * unit;
#pragma unroll
    for (int a = 0; a < 3; a++) g[a] = __fadd_rn(lo[a], __fmul_rn((float)(blo[a] + bhi[a]), hu));
}

// A walk group: stars [first, first + count) in key order and its box [lo, hi)
// on the member's integer grid.
struct GroupRec {
    int first, count, lo[3], hi[3];
};
__device__ __forceinline__ GroupRec load_group(const int4 *groups, int g) {
    const int4 a = groups[2 * g], b = groups[2 * g + 1];
    GroupRec r;
    r.first = a.x; r.count = a.y;
    r.lo[0] = a.z; r.lo[1] = a.w; r.lo[2] = b.x;
    r.hi[0] = b.y; r.hi[1] = b.z; r.hi[2] = b.w;
    return r;
}

}  // namespace rv
