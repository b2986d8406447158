// walk.cu -- Barnes-Hut tree walk and interaction evaluation (FP32).
//
// One warp walks the tree for one group of up to 64 consecutive stars. Cells
// are tested up to 64 a pass, two per lane, under the box-box opening test;
// accepted cells are staged in shared memory as multipole records, opened
// leaves stage their stars, opened internal cells push their child range on
// a per-warp stack. Whenever a staged list holds a full tile, the warp
// evaluates it: a lane holds two stars of the group (a target pair), each of
// the p = ceil(s / 2) pairs is served by k = floor(32 / p) lanes, lane t + i p
// taking list pairs i, i + k, ... with broadcast shared-memory reads and
// evaluating every loaded source pair on both its stars; tile sums are added
// to running totals with Neumaier compensation, and the k partial totals of a
// star are combined in lane order at the end. Particles outside the tree (a chain's
// centre of mass) are walked by the same kernel as one-star groups before the
// tree's own groups.
//
// Staged lists hold list entries in pairs, each field of the two entries
// side by side, so that one lane evaluates two interactions with the packed
// two-wide FP32 instructions (add/mul/fma .f32x2): the walk is bound by
// instruction issue, and a packed instruction does two lanes' worth of FP32
// work in one issue slot. Each interaction is still computed element by
// element in FP32 round-to-nearest; only the order of the running sums
// differs from one entry per instruction.
//
// Interactions (G = 1, Sect. 3 Plummer softening; multipoles about the cell's
// centre of mass, Sect. 1):
//   star j on star i:  a += m_j r / (r^2 + e^2)^{3/2},  phi -= m_j (r^2 + e^2)^{-1/2},  r = x_j - x_i
//   cell on star i:    r = x_i - com, rho^2 = r.r + e^2,
//                      a += -M r / rho^3 + Q r / rho^5 - 5 (r.Q.r) r / (2 rho^7),
//                      phi -= M / rho + (r.Q.r) / (2 rho^5).
// Flops per interaction in this source (add/mul 1, FMA 2, rsqrt 1):
//   star-star 20, cell (monopole + quadrupole) 54, cell (monopole) 18.
#include <algorithm>

#include "rv_internal.cuh"

// Unrolling of the evaluation loops (list pairs in flight per lane, each on
// two targets; measured on GB300: star pairs 1, cell pairs 3) and the
// register budget of the walk kernel. The kernel runs one warp per block, so
// the register budget alone sets the resident warps: 104 registers a thread
// (the running sums live in shared memory) give 18-19 warps per SM, against
// 16 at 128 registers; 96 registers spill, 112 and 128 were slower
// (2^24 stars at theta 0.8 and tile 96: 80.9 ms at 104 registers, 84.8 at
// 112, 84.8 at 128, 88.6 at 96).
#ifndef RV_P2P_UNROLL
#define RV_P2P_UNROLL 1
#endif
#ifndef RV_M2P_UNROLL
#define RV_M2P_UNROLL 3
#endif
#ifndef RV_WALK_MAXNREG
#define RV_WALK_MAXNREG 104
#endif
#ifdef RV_WALK_MIN_BLOCKS
#define RV_WALK_BOUNDS __launch_bounds__(kWalkWarps * 32, RV_WALK_MIN_BLOCKS)
#else
#define RV_WALK_BOUNDS __maxnreg__(RV_WALK_MAXNREG)
#endif

namespace rv {

// spline softening lengths (h = 2.8 eps): h^2, 1/h, 1/h^3
struct Spline {
    float h2, hinv, hinv3;
};

struct WalkArgs {
    const float4 *pos;   // sorted (x, y, z, m)
    const int4 *cbox;
    const int4 *clink;   // (child first, child end, first star, end star)
    const float4 *cmom;  // relative to the cell's geometric centre
    const int4 *groups;
    const int *perm;
    DevState *st;
    int cell_cap;
    int n;               // stars of the tree
    const int64_t *moff; // member star offsets [M + 1]
    int M;               // members (independent systems)
    const double *mbounds;  // per member: min x, y, z, L, 2^21 / L
    const int *mroot;    // root cell of each member
    const int *xmem;     // member of each extra particle (nullptr: member 0)
    int extra_per_member;  // > 0: extras [m e, (m + 1) e) belong to member m (e chains per member)
    MacTable mac;
    float eps2;          // star-star and star-cell softening^2
    float eps_star;
    int tile;
    int n_extra;
    const float *xyzm;   // extra particles (x, y, z, m)
    const float *xeps;
    const float4 *xquad; // optional: each extra particle's traceless quadrupole, 2 float4 (see extra_terms)
    const uint8_t *xq_skip;  // optional, per star (caller order): 1 = no quadrupole terms (a chain's perturber)
    float *ax, *ay, *az, *pot;
    float *xout;
    // optional record of accepted (group, cell) pairs that a walk at the
    // smaller angle theta_rec would have opened (the learned correction's input)
    MacTable rec;
    int2 *pairs;
    int *npairs;
    int pair_cap;
    // relative opening criterion: tolerance and reference acceleration per star (caller order)
    float rel_alpha;
    const float *arx, *ary, *arz;
    // optional group mask (block time steps): only groups with gact[g] != 0 are walked
    const uint8_t *gact;
    // queue order of the groups (null: build order), and the per-star list cost
    // written for the next walk's order
    const int *order;
    float *scost;
    // spline softening of the stars (h = 2.8 eps)
    Spline spl;
    // the walk stack's entries beyond kStackSm: kStackSpill per warp of the launch
    int *gstack;
};

// Per-warp shared memory: stack | lane_cell[32] | cell staging | star staging |
// running sums. Cell staging: (tile + 32) / 2 pairs of multipole records, 5
// float4 per pair holding (M, cx), (cy, cz), (-Qxx, -Qyy), (-Qzz, -Qxy),
// (-Qxz, -Qyz) of both entries side by side (cx.. = centre of mass relative
// to the group centre). Star staging: (tile + 32) / 2 pairs, 2 float4 per
// pair: (x, y), (z, m). Running sums: 16 floats per lane (AccSm).
constexpr int kCellPairF4 = 5, kStarPairF4 = 2;
constexpr int kAccWords = 16 * 32;
constexpr int kP2PUnroll = RV_P2P_UNROLL, kM2PUnroll = RV_M2P_UNROLL;
__host__ __device__ inline size_t warp_staging_bytes(int tile) {
    return (size_t)kStackSm * 4 + 192 * 4 + (size_t)(tile + 64) / 2 * 16 * kCellPairF4 +
           (size_t)(tile + 32) / 2 * 16 * kStarPairF4;
}
__host__ __device__ inline size_t warp_smem_bytes(int tile) { return warp_staging_bytes(tile) + 4 * kAccWords; }

// The tree of one member as the walk sees it.
struct TreeGeo {
    int ncell;           // cells of all trees (at most the workspace capacity)
    int root;            // the member's root cell (-1: empty member)
    float lo[3], unit;   // the member's bounding-cube corner and grid unit in FP32
};

__device__ __forceinline__ TreeGeo tree_geo(const WalkArgs &A, int member) {
    TreeGeo t;
    t.ncell = min(A.st->ncell, A.cell_cap);
    t.root = A.mroot[member];
    const double *b = A.mbounds + 5 * member;
    t.lo[0] = (float)b[0];
    t.lo[1] = (float)b[1];
    t.lo[2] = (float)b[2];
    t.unit = (float)(b[3] / 2097152.0);
    return t;
}

struct Acc {
    float ax, ay, az, ph;      // running sums
    float cx, cy, cz, cp;      // Neumaier compensation
};

// Two FP32 values in one 64-bit register (low half: the even list entry).
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float f2_sum(f2 v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo + hi;
}
__device__ __forceinline__ f2 f2_rsqrt(f2 v, bool guard_zero) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    float a = rsqrtf(lo), b = rsqrtf(hi);
    if (guard_zero) {
        a = (lo > 0.f) ? a : 0.f;
        b = (hi > 0.f) ? b : 0.f;
    }
    return f2_pack(a, b);
}
constexpr f2 kF2MinusHalf = 0xBF000000BF000000ull;     // (-0.5f, -0.5f)
constexpr f2 kF2MinusFiveHalf = 0xC0200000C0200000ull; // (-2.5f, -2.5f)

// A lane's two targets (minus their positions relative to the group's
// centre, each in both halves) and its share of a staged list: pairs j0,
// j0 + k, ... (j0 >= 2^20: the lane takes no share). Both targets use every
// source pair the lane loads.
struct Tgt {
    f2 nx[2], ny[2], nz[2];
    int j0, k;
};

// A lane's running sums for its two targets, kept in the warp's shared
// memory (not registers, which the evaluation loops need): for target q,
// field k = ax, ay, az, ph, then their Neumaier compensations (k + 4), at
// word (q * 8 + k) * 32 + lane, so the 32 lanes touch 32 consecutive words.
struct AccSm {
    float *p;   // the warp's region + lane
    __device__ __forceinline__ float &f(int q, int k) const { return p[(q * 8 + k) * 32]; }
};

__device__ __forceinline__ void add_tile(const AccSm &A, int q, f2 tx, f2 ty, f2 tz, f2 tp) {
    const float v[4] = {f2_sum(tx), f2_sum(ty), f2_sum(tz), -f2_sum(tp)};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float sum = A.f(q, k), comp = A.f(q, k + 4);
        nadd(sum, comp, v[k]);
        A.f(q, k) = sum;
        A.f(q, k + 4) = comp;
    }
}

// Spline softening (the "spline" option of Sect. 2): the point mass smoothed
// by the cubic spline kernel of support h = 2.8 eps, so that phi(0) = -m/eps
// as for Plummer softening of length eps. From the kernel's enclosed mass,
// a = m d f(u) / h^3 and phi = (m/h) P(u) with u = |d| / h:
//   u < 1/2:  f = 32/3 - 192/5 u^2 + 32 u^3,  P = -14/5 + 16/3 u^2 - 48/5 u^4 + 32/5 u^5
//   u < 1:    f = 64/3 - 48 u + 192/5 u^2 - 32/3 u^3 - 1/(15 u^3),
//             P = -16/5 + 1/(15 u) + 32/3 u^2 - 16 u^3 + 48/5 u^4 - 32/15 u^5
//   u >= 1:   Newton.


// m f / h^3 and -m P / h (the walk sums -phi) for one pair at squared distance r2 < h^2
__device__ __forceinline__ void spline_terms(float r2, float m, const Spline &S, float &mr3, float &mr) {
    const float u = sqrtf(r2) * S.hinv;
    const float u2 = u * u;
    float f, P;
    if (u < 0.5f) {
        f = fmaf(u2, fmaf(32.f, u, -192.f / 5.f), 32.f / 3.f);
        P = fmaf(u2, fmaf(u2, fmaf(32.f / 5.f, u, -48.f / 5.f), 16.f / 3.f), -14.f / 5.f);
    } else {
        const float iu = 1.f / u;
        f = fmaf(u2, fmaf(-32.f / 3.f, u, 192.f / 5.f), fmaf(-48.f, u, 64.f / 3.f)) - (1.f / 15.f) * (iu * iu * iu);
        P = fmaf(u2, fmaf(u, fmaf(u, fmaf(-32.f / 15.f, u, 48.f / 5.f), -16.f), 32.f / 3.f),
                 fmaf(1.f / 15.f, iu, -16.f / 5.f));
    }
    mr3 = m * f * S.hinv3;
    mr = -m * P * S.hinv;
}

// One packed pair of star-star terms under spline softening: Newton beyond h,
// the kernel's field inside (per element).
__device__ __forceinline__ void spline_pair(f2 r2, f2 m2, const Spline &S, f2 &mr, f2 &mr3) {
    float ra, rb, ma, mb;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(ra), "=f"(rb) : "l"(r2));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(ma), "=f"(mb) : "l"(m2));
    float o3[2], o1[2];
    const float rr[2] = {ra, rb}, mm[2] = {ma, mb};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (rr[h] >= S.h2) {
            const float ri = rsqrtf(rr[h]);
            o1[h] = mm[h] * ri;
            o3[h] = o1[h] * (ri * ri);
        } else {
            spline_terms(rr[h], mm[h], S, o3[h], o1[h]);
        }
    }
    mr = f2_pack(o1[0], o1[1]);
    mr3 = f2_pack(o3[0], o3[1]);
}

// Star pairs 0 .. npair-1 of a staged star list on this lane's targets:
//   d = x_j - x_i, a += m_j d / (d.d + e^2)^{3/2}, phi -= m_j / (d.d + e^2)^{1/2}
// (SPL: the spline field instead).
template <bool SOFT, bool SPL>
__device__ __forceinline__ void eval_p2p(const float4 *src, int npair, const Tgt &t, f2 eps2, const Spline &S,
                                         const AccSm &A) {
    f2 tx[2] = {0, 0}, ty[2] = {0, 0}, tz[2] = {0, 0}, tp[2] = {0, 0};   // tp sums +m/r
#pragma unroll kP2PUnroll
    for (int j = t.j0; j < npair; j += t.k) {
        const ulonglong2 a = reinterpret_cast<const ulonglong2 *>(src)[2 * j];      // x, y
        const ulonglong2 b = reinterpret_cast<const ulonglong2 *>(src)[2 * j + 1];  // z, m
#pragma unroll
        for (int q = 0; q < 2; q++) {
            f2 dx = f2_add(a.x, t.nx[q]), dy = f2_add(a.y, t.ny[q]), dz = f2_add(b.x, t.nz[q]);
            f2 mr, mr3;
            if (SPL) {
                f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                spline_pair(r2, b.y, S, mr, mr3);
            } else {
                f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_fma(dz, dz, eps2)));
                f2 rinv = f2_rsqrt(r2, !SOFT);
                mr = f2_mul(b.y, rinv);
                mr3 = f2_mul(mr, f2_mul(rinv, rinv));
            }
            tx[q] = f2_fma(mr3, dx, tx[q]);
            ty[q] = f2_fma(mr3, dy, ty[q]);
            tz[q] = f2_fma(mr3, dz, tz[q]);
            tp[q] = f2_add(tp[q], mr);
        }
    }
    add_tile(A, 0, tx[0], ty[0], tz[0], tp[0]);
    add_tile(A, 1, tx[1], ty[1], tz[1], tp[1]);
}

// Cell pairs 0 .. npair-1 of a staged cell list on this lane's targets. With
// d = com - x_i = -r, rho^2 = d.d + e^2, the staged -Q gives q = -Q d = Q r
// and s = d.q / rho^4 = -(r.Q.r) / rho^4, so that
//   a += (M - 5/2 s) d / rho^3 + q / rho^5,  phi -= (M - s/2) / rho,
// which is the monopole + quadrupole expansion of the file header. SPL: the
// unsoftened expansion (e = 0), and a cell closer than h acts as the spline
// monopole.
template <bool QUAD, bool SPL>
__device__ __forceinline__ void eval_m2p(const float4 *src, int npair, const Tgt &t, f2 eps2, const Spline &S,
                                         const AccSm &A) {
    f2 tx[2] = {0, 0}, ty[2] = {0, 0}, tz[2] = {0, 0}, tp[2] = {0, 0};   // tp sums +(M - s/2)/rho
    if (SPL) eps2 = 0;
#pragma unroll kM2PUnroll
    for (int j = t.j0; j < npair; j += t.k) {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(src) + kCellPairF4 * j;
        const ulonglong2 a = p[0];   // M, cx
        const ulonglong2 b = p[1];   // cy, cz
        ulonglong2 c = make_ulonglong2(0, 0), e = c, f = c;
        if (QUAD) {
            c = p[2];   // -Qxx, -Qyy
            e = p[3];   // -Qzz, -Qxy
            f = p[4];   // -Qxz, -Qyz
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            f2 dx = f2_add(a.y, t.nx[q]), dy = f2_add(b.x, t.ny[q]), dz = f2_add(b.y, t.nz[q]);
            f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_fma(dz, dz, eps2)));
            // r > 0: an accepted cell's box is separated from the group's box
            f2 rinv = f2_rsqrt(r2, false);
            f2 u = f2_mul(rinv, rinv);
            f2 rinv3 = f2_mul(rinv, u);
            f2 ix, iy, iz, ip;   // this pair's terms
            if (QUAD) {
                f2 qx = f2_fma(c.x, dx, f2_fma(e.y, dy, f2_mul(f.x, dz)));
                f2 qy = f2_fma(e.y, dx, f2_fma(c.y, dy, f2_mul(f.y, dz)));
                f2 qz = f2_fma(f.x, dx, f2_fma(f.y, dy, f2_mul(e.x, dz)));
                f2 dq = f2_fma(dx, qx, f2_fma(dy, qy, f2_mul(dz, qz)));
                f2 sw = f2_mul(dq, f2_mul(u, u));
                f2 rinv5 = f2_mul(rinv3, u);
                f2 B = f2_mul(rinv3, f2_fma(kF2MinusFiveHalf, sw, a.x));
                if (!SPL) {
                    tx[q] = f2_fma(B, dx, f2_fma(rinv5, qx, tx[q]));
                    ty[q] = f2_fma(B, dy, f2_fma(rinv5, qy, ty[q]));
                    tz[q] = f2_fma(B, dz, f2_fma(rinv5, qz, tz[q]));
                    tp[q] = f2_fma(rinv, f2_fma(kF2MinusHalf, sw, a.x), tp[q]);
                    continue;
                }
                ix = f2_fma(B, dx, f2_mul(rinv5, qx));
                iy = f2_fma(B, dy, f2_mul(rinv5, qy));
                iz = f2_fma(B, dz, f2_mul(rinv5, qz));
                ip = f2_mul(rinv, f2_fma(kF2MinusHalf, sw, a.x));
            } else {
                f2 mr3 = f2_mul(a.x, rinv3);
                if (!SPL) {
                    tx[q] = f2_fma(mr3, dx, tx[q]);
                    ty[q] = f2_fma(mr3, dy, ty[q]);
                    tz[q] = f2_fma(mr3, dz, tz[q]);
                    tp[q] = f2_fma(a.x, rinv, tp[q]);
                    continue;
                }
                ix = f2_mul(mr3, dx);
                iy = f2_mul(mr3, dy);
                iz = f2_mul(mr3, dz);
                ip = f2_mul(a.x, rinv);
            }
            if (SPL) {
                float ra, rb;
                asm("mov.b64 {%0, %1}, %2;" : "=f"(ra), "=f"(rb) : "l"(r2));
                if (ra < S.h2 || rb < S.h2) {   // a cell closer than h: the spline monopole
                    float m0, m1, o3, o1;
                    asm("mov.b64 {%0, %1}, %2;" : "=f"(m0), "=f"(m1) : "l"(a.x));
                    float v[4][2];
                    const f2 in4[4] = {ix, iy, iz, ip};
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(v[k][0]), "=f"(v[k][1]) : "l"(in4[k]));
                    float dd[3][2];
                    const f2 d3[3] = {dx, dy, dz};
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(dd[k][0]), "=f"(dd[k][1]) : "l"(d3[k]));
                    const float rr[2] = {ra, rb}, mm[2] = {m0, m1};
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
                        if (rr[hh] < S.h2) {
                            spline_terms(rr[hh], mm[hh], S, o3, o1);
                            v[0][hh] = o3 * dd[0][hh];
                            v[1][hh] = o3 * dd[1][hh];
                            v[2][hh] = o3 * dd[2][hh];
                            v[3][hh] = o1;
                        }
                    }
                    ix = f2_pack(v[0][0], v[0][1]);
                    iy = f2_pack(v[1][0], v[1][1]);
                    iz = f2_pack(v[2][0], v[2][1]);
                    ip = f2_pack(v[3][0], v[3][1]);
                }
                tx[q] = f2_add(tx[q], ix);
                ty[q] = f2_add(ty[q], iy);
                tz[q] = f2_add(tz[q], iz);
                tp[q] = f2_add(tp[q], ip);
            }
        }
    }
    add_tile(A, 0, tx[0], ty[0], tz[0], tp[0]);
    add_tile(A, 1, tx[1], ty[1], tz[1], tp[1]);
}

// Field f of staged entry e in a pair-interleaved list whose pairs are
// `pair_f4` float4 long.
__device__ __forceinline__ float *staged(float4 *base, int pair_f4, int e, int f) {
    return reinterpret_cast<float *>(base + pair_f4 * (e >> 1)) + 2 * f + (e & 1);
}

// An odd list gets a massless partner in its last pair at the position of
// the entry beside it (finite, nonzero distance; contributes exactly 0).
__device__ __forceinline__ void pad_cells(float4 *m2p, int cnt) {
    if ((cnt & 1) && (threadIdx.x & 31) == 0) {
        float *d = reinterpret_cast<float *>(m2p + kCellPairF4 * (cnt >> 1));
        d[1] = 0.f;
        d[3] = d[2]; d[5] = d[4]; d[7] = d[6];
        for (int f = 4; f < 10; f++) d[2 * f + 1] = 0.f;
    }
}
__device__ __forceinline__ void pad_stars(float4 *p2p, int cnt) {
    if ((cnt & 1) && (threadIdx.x & 31) == 0) {
        float *d = reinterpret_cast<float *>(p2p + kStarPairF4 * (cnt >> 1));
        d[1] = d[0]; d[3] = d[2]; d[5] = d[4];
        d[7] = 0.f;
    }
}

__device__ __forceinline__ int gap1(int blo, int bhi, int clo, int chi) {
    return (clo >= bhi) ? clo - bhi : ((blo >= chi) ? blo - chi : 0);
}

// Walks the tree for one group; returns false if a bound was violated.
// Positions in the walk are relative to g, the geometric centre of the
// group's box: targets and staged sources are shifted once, cell centres of
// mass are (cell centre - g) + (centre of mass - cell centre). Differences of
// nearby FP32 coordinates are exact, so FP32 keeps its relative precision at
// any distance from the origin.
template <bool SOFT, bool QUAD, bool REC, bool REL, bool SPL>
__device__ __forceinline__ bool walk_group(const WalkArgs &A, const TreeGeo &G, const unsigned long long *thr,
                                           const unsigned long long *thr_rec, int gid, char *wsm, const int blo[3],
                                           const int bhi[3], const float g[3], const Tgt &tg, f2 eps2, const AccSm &acc,
                                           unsigned long long &np2p, unsigned long long &nm2p, float K) {
    const int lane = threadIdx.x & 31;
    const int T = A.tile;
    // the range stack: entries below kStackSm in shared memory, the deeper ones
    // (rare: a pass pushes at most 32, and the walk is depth-first) in this
    // warp's spill area in global memory; __syncwarp orders both for the warp
    int *stack = reinterpret_cast<int *>(wsm);
    int *spill = A.gstack + (size_t)(blockIdx.x * kWalkWarps + (threadIdx.x >> 5)) * kStackSpill;
    auto st_get = [&](int i) -> int { return i < kStackSm ? stack[i] : spill[i - kStackSm]; };
    int *lane_cell = stack + kStackSm;                             // a pass's 64 cells
    int *lf_first = lane_cell + 64, *lf_start = lane_cell + 128;   // a pass's opened leaves
    float4 *m2p = reinterpret_cast<float4 *>(lane_cell + 192);
    float4 *p2p = m2p + kCellPairF4 * ((T + 64) / 2);
    const unsigned lt = lanemask_lt();
    const int ncell = G.ncell;

    if (lane == 0) stack[0] = (G.root << 4) | 1;  // the member's root: a range of one cell
    int top = 1, nm = 0, np = 0, hwm = 1;
    bool ok = true;
    // every pass tests at least one new cell, so a walk ends within ncell passes
    int guard = ncell + 1;
    __syncwarp();
    // a cell's records, opening test and link check (one of a pass's two slots per lane)
    struct Slot {
        int c;
        bool accept, leaf, open, band;
        int4 lk, b;
        float4 r0, q1, q2;
    };
    auto load_slot = [&](Slot &x) {
        x.accept = x.leaf = x.open = x.band = false;
        x.lk = make_int4(0, 0, 0, 0);
        x.b = make_int4(0, 0, 0, 0);
        x.r0 = make_float4(0.f, 0.f, 0.f, 0.f);
        x.q1 = x.r0;
        x.q2 = x.r0;
        if (x.c >= 0) {
            // every record of the cell at once: one L2 round trip per pass
            x.b = __ldg(&A.cbox[x.c]);
            x.lk = __ldg(&A.clink[x.c]);
            x.r0 = __ldg(&A.cmom[3 * x.c + 0]);
            if (QUAD) {
                x.q1 = __ldg(&A.cmom[3 * x.c + 1]);
                x.q2 = __ldg(&A.cmom[3 * x.c + 2]);
            }
        }
    };
    auto test_slot = [&](Slot &x) -> bool {   // returns "bad link"
        if (x.c >= 0) {
            const int4 b = x.b;
            const int side = 1 << (kMaxLevel - b.w);
            const long long gx = gap1(blo[0], bhi[0], b.x, b.x + side);
            const long long gy = gap1(blo[1], bhi[1], b.y, b.y + side);
            const long long gz = gap1(blo[2], bhi[2], b.z, b.z + side);
            const unsigned long long d2 = (unsigned long long)(gx * gx + gy * gy + gz * gz);
            if (REL && K >= 0.f) {
                // relative criterion: the group's box outside the cell's box grown by
                // side/10 per side (integers x 10), and M s^2 <= (K d^2) d^2 in FP32
                const int bo[3] = {b.x, b.y, b.z};
                bool outside = false;
#pragma unroll
                for (int a = 0; a < 3; a++)
                    outside |= (10 * bhi[a] <= 10 * bo[a] - side) || (10 * blo[a] >= 10 * (bo[a] + side) + side);
                const float d2f = __ull2float_rn(d2);
                const float s2 = __fmul_rn((float)side, (float)side);
                x.accept = outside && (__fmul_rn(x.r0.x, s2) <= __fmul_rn(__fmul_rn(K, d2f), d2f));
            } else {
                x.accept = d2 >= thr[b.w];
            }
            if (REC) x.band = x.accept && d2 < thr_rec[b.w];
            if (!x.accept) {
                x.leaf = (x.lk.x == x.lk.y);
                x.open = !x.leaf;
            }
        }
        // links must stay inside the tree (a violated bound ends the walk with an error)
        return (x.open && (x.lk.x <= x.c || x.lk.y > ncell || x.lk.y - x.lk.x > 8)) ||
               (x.leaf && (x.lk.z < 0 || x.lk.w > A.n || x.lk.z > x.lk.w));
    };
    auto stage_cell = [&](const Slot &x, int p) {
        float c0[3];
        geo_centre(x.b, G.lo, G.unit, c0);
        *staged(m2p, kCellPairF4, p, 0) = x.r0.x;
        *staged(m2p, kCellPairF4, p, 1) = (c0[0] - g[0]) + x.r0.y;
        *staged(m2p, kCellPairF4, p, 2) = (c0[1] - g[1]) + x.r0.z;
        *staged(m2p, kCellPairF4, p, 3) = (c0[2] - g[2]) + x.r0.w;
        if (QUAD) {   // q1 = (Qxx, Qyy, Qzz, Qxy), q2 = (Qxz, Qyz, 0, 0)
            *staged(m2p, kCellPairF4, p, 4) = -x.q1.x;
            *staged(m2p, kCellPairF4, p, 5) = -x.q1.y;
            *staged(m2p, kCellPairF4, p, 6) = -x.q1.z;
            *staged(m2p, kCellPairF4, p, 7) = -x.q1.w;
            *staged(m2p, kCellPairF4, p, 8) = -x.q2.x;
            *staged(m2p, kCellPairF4, p, 9) = -x.q2.y;
        }
    };
    auto push = [&](int p, const int4 lk) {
        if (p < kStackSm) stack[p] = (lk.x << 4) | (lk.y - lk.x);
        else if (p < kStackCap) spill[p - kStackSm] = (lk.x << 4) | (lk.y - lk.x);
    };
    while (top > 0) {
        if (--guard < 0) { ok = false; break; }
        // pop whole child ranges from the top while they fit in the pass's 64
        // slots (slot s: lane s % 32, its first or second cell)
        const int avail = min(top, 64);
        const int e0 = (lane < avail) ? st_get(top - 1 - lane) : 0;
        const int e1 = (lane + 32 < avail) ? st_get(top - 33 - lane) : 0;
        const int n0 = e0 & 15, n1 = e1 & 15;
        int in0 = n0, in1 = n1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y0 = __shfl_up_sync(0xffffffffu, in0, o);
            const int y1 = __shfl_up_sync(0xffffffffu, in1, o);
            if (lane >= o) {
                in0 += y0;
                in1 += y1;
            }
        }
        in1 += __shfl_sync(0xffffffffu, in0, 31);
        const unsigned fit0 = __ballot_sync(0xffffffffu, lane < avail && in0 <= 64);
        const unsigned fit1 = __ballot_sync(0xffffffffu, lane + 32 < avail && in1 <= 64);
        const int kk = __popc(fit0) + __popc(fit1);
        const int tA = __shfl_sync(0xffffffffu, in0, min(kk, 32) - 1);
        const int tB = __shfl_sync(0xffffffffu, in1, max(kk - 33, 0));
        const int total = kk <= 32 ? tA : tB;
        __syncwarp();
        if (lane < kk) {
            const int b0 = in0 - n0, c0 = e0 >> 4;
            for (int t = 0; t < n0; t++) lane_cell[b0 + t] = c0 + t;
        }
        if (lane + 32 < kk) {
            const int b1 = in1 - n1, c1 = e1 >> 4;
            for (int t = 0; t < n1; t++) lane_cell[b1 + t] = c1 + t;
        }
        top -= kk;
        __syncwarp();
        Slot xa, xb;
        xa.c = (lane < total) ? lane_cell[lane] : -1;
        xb.c = (lane + 32 < total) ? lane_cell[lane + 32] : -1;
        __syncwarp();
        if (__any_sync(0xffffffffu, xa.c >= ncell || xb.c >= ncell)) { ok = false; break; }
        load_slot(xa);
        load_slot(xb);
        const bool bad_a = test_slot(xa), bad_b = test_slot(xb);
        if (__any_sync(0xffffffffu, bad_a || bad_b)) { ok = false; break; }
        // opened internal cells: push their child ranges (slot order)
        const unsigned oma = __ballot_sync(0xffffffffu, xa.open), omb = __ballot_sync(0xffffffffu, xb.open);
        if (xa.open) push(top + __popc(oma & lt), xa.lk);
        if (xb.open) push(top + __popc(oma) + __popc(omb & lt), xb.lk);
        top += __popc(oma) + __popc(omb);
        hwm = max(hwm, top);
        if (top > kStackCap) { ok = false; break; }
        // accepted cells: stage their multipole records, centre of mass relative to g, -Q
        const unsigned ama = __ballot_sync(0xffffffffu, xa.accept), amb = __ballot_sync(0xffffffffu, xb.accept);
        if (xa.accept) stage_cell(xa, nm + __popc(ama & lt));
        if (xb.accept) stage_cell(xb, nm + __popc(ama) + __popc(amb & lt));
        nm += __popc(ama) + __popc(amb);
        nm2p += __popc(ama) + __popc(amb);
        if (REC) {
            const unsigned bma = __ballot_sync(0xffffffffu, xa.band), bmb = __ballot_sync(0xffffffffu, xb.band);
            if (bma | bmb) {
                int base = 0;
                if (lane == 0) base = atomicAdd(A.npairs, __popc(bma) + __popc(bmb));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (xa.band) {
                    const int p = base + __popc(bma & lt);
                    if (p < A.pair_cap) A.pairs[p] = make_int2(gid, xa.c);
                    else latch_err(A.st, kErrPairs);
                }
                if (xb.band) {
                    const int p = base + __popc(bma) + __popc(bmb & lt);
                    if (p < A.pair_cap) A.pairs[p] = make_int2(gid, xb.c);
                    else latch_err(A.st, kErrPairs);
                }
            }
        }
        // opened leaves: stage their stars relative to g, leaves in slot order
        // and stars in order within each (the order the tiles take them), 32
        // stars a round whichever leaves they come from, so that the loads of
        // a pass's leaves overlap instead of following one another
        const unsigned lma = __ballot_sync(0xffffffffu, xa.leaf), lmb = __ballot_sync(0xffffffffu, xb.leaf);
        if (lma | lmb) {
            const int ca = xa.leaf ? xa.lk.w - xa.lk.z : 0, cb = xb.leaf ? xb.lk.w - xb.lk.z : 0;
            int ia = ca, ib = cb;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int ya = __shfl_up_sync(0xffffffffu, ia, o);
                const int yb = __shfl_up_sync(0xffffffffu, ib, o);
                if (lane >= o) {
                    ia += ya;
                    ib += yb;
                }
            }
            ib += __shfl_sync(0xffffffffu, ia, 31);
            const int total_stars = __shfl_sync(0xffffffffu, ib, 31);
            const int nla = __popc(lma), nl = nla + __popc(lmb);
            if (xa.leaf) {
                const int k = __popc(lma & lt);
                lf_first[k] = xa.lk.z;
                lf_start[k] = ia - ca;
            }
            if (xb.leaf) {
                const int k = nla + __popc(lmb & lt);
                lf_first[k] = xb.lk.z;
                lf_start[k] = ib - cb;
            }
            __syncwarp();
            for (int base = 0; base < total_stars; base += 32) {
                const int idx = base + lane, cc = min(32, total_stars - base);
                if (lane < cc) {
                    // the leaf holding star idx of the pass: the last one starting at or before idx
                    int lo = 0, hi = nl - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (lf_start[mid] <= idx) lo = mid; else hi = mid - 1;
                    }
                    const float4 s = __ldg(&A.pos[lf_first[lo] + (idx - lf_start[lo])]);
                    const int e = np + lane;
                    *staged(p2p, kStarPairF4, e, 0) = s.x - g[0];
                    *staged(p2p, kStarPairF4, e, 1) = s.y - g[1];
                    *staged(p2p, kStarPairF4, e, 2) = s.z - g[2];
                    *staged(p2p, kStarPairF4, e, 3) = s.w;
                }
                np += cc;
                np2p += cc;
                if (np >= T) {
                    __syncwarp();
                    eval_p2p<SOFT, SPL>(p2p, T / 2, tg, eps2, A.spl, acc);
                    __syncwarp();
                    // T is even: the leftover entries move pair by pair
                    if (lane < (np - T + 1) / 2) {
                        p2p[kStarPairF4 * lane] = p2p[kStarPairF4 * (T / 2 + lane)];
                        p2p[kStarPairF4 * lane + 1] = p2p[kStarPairF4 * (T / 2 + lane) + 1];
                    }
                    np -= T;
                    __syncwarp();
                }
            }
        }
        // a pass adds up to 64 cells: flush while a full tile is staged (nm < T
        // before every pass, so at most T + 63 entries are ever staged)
        while (nm >= T) {
            __syncwarp();
            eval_m2p<QUAD, SPL>(m2p, T / 2, tg, eps2, A.spl, acc);
            __syncwarp();
            // the leftover (up to 32 pairs) to the front; read all before writing any,
            // as source and destination overlap when T < 64
            const int mv = (nm - T + 1) / 2;
            for (int f = 0; f < kCellPairF4; f++) {   // field by field: every read of a field before its writes
                const float4 v = lane < mv ? m2p[kCellPairF4 * (T / 2 + lane) + f] : make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                if (lane < mv) m2p[kCellPairF4 * lane + f] = v;
                __syncwarp();
            }
            nm -= T;
        }
        __syncwarp();
    }
    __syncwarp();
    if (ok) {
        pad_stars(p2p, np);
        pad_cells(m2p, nm);
        __syncwarp();
        if (np > 0) eval_p2p<SOFT, SPL>(p2p, (np + 1) / 2, tg, eps2, A.spl, acc);
        if (nm > 0) eval_m2p<QUAD, SPL>(m2p, (nm + 1) / 2, tg, eps2, A.spl, acc);
    }
    __syncwarp();
    if (lane == 0) atomicMax(&A.st->stack_hwm, hwm);
    return ok;
}

// Lane l serves target pair t = l % p (stars 2t and 2t + 1) with share
// l / p; the k lanes t, t + p, ..., t + (k - 1) p of a pair add their partial
// totals in that order, read from the warp's running sums (AccSm). Returns the
// totals of stars `lane` and `lane + 32`.
__device__ __forceinline__ void combine_shares(const float *accw, int s, int p, int k, Acc out[2]) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int i = lane + 32 * h;   // star of the group
        Acc o = {};
        if (i < s)
            for (int m = 0; m < k; m++) {
                const float *e = accw + (i & 1) * 8 * 32 + (i >> 1) + m * p;
                nadd(o.ax, o.cx, e[0]); nadd(o.ay, o.cy, e[32]);
                nadd(o.az, o.cz, e[64]); nadd(o.ph, o.cp, e[96]);
                o.cx += e[128]; o.cy += e[160]; o.cz += e[192]; o.cp += e[224];
            }
        out[h] = o;
    }
    __syncwarp();
}

// Direct terms of the extra particles of `member` on one target (pair
// softening rule of Sect. 3: max(eps_i, eps_j), none if either is
// unsoftened), absolute FP32. With A.xquad, an extra particle (a chain seen
// from outside) also carries a traceless quadrupole Q about its position,
// (xx, yy, zz, xy), (xz, yz, 0, 0), whose field is added as for a cell: with
// d = x_extra - x_i = -r and rho^2 = d.d + e^2,
//   a += -Q d / rho^5 + 5/2 (d.Q.d) d / rho^7,  phi -= (d.Q.d) / (2 rho^5),
// unless use_quad is false (a target that is a chain's perturber).
__device__ __forceinline__ void extra_terms(const WalkArgs &A, float xi, float yi, float zi, float ei, int skip,
                                            int member, Acc &acc, bool use_quad = true) {
    float tx = 0.f, ty = 0.f, tz = 0.f, tp = 0.f;
    const int k0 = A.extra_per_member ? member * A.extra_per_member : 0;
    const int k1 = A.extra_per_member ? min(k0 + A.extra_per_member, A.n_extra) : A.n_extra;
    for (int k = k0; k < k1; k++) {
        if (k == skip) continue;
        if (!A.extra_per_member && (A.xmem ? A.xmem[k] : 0) != member) continue;
        float ek = A.xeps[k];
        float e = (ei == 0.f || ek == 0.f) ? 0.f : fmaxf(ei, ek);
        float dx = A.xyzm[4 * k] - xi, dy = A.xyzm[4 * k + 1] - yi, dz = A.xyzm[4 * k + 2] - zi;
        float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e * e)));
        if (r2 <= 0.f) continue;
        float rinv = rsqrtf(r2);
        float mr = A.xyzm[4 * k + 3] * rinv;
        float mr3 = mr * rinv * rinv;
        tx = fmaf(mr3, dx, tx); ty = fmaf(mr3, dy, ty); tz = fmaf(mr3, dz, tz);
        tp -= mr;
        if (A.xquad && use_quad) {
            const float4 q1 = A.xquad[2 * k], q2 = A.xquad[2 * k + 1];
            const float qx = fmaf(q1.x, dx, fmaf(q1.w, dy, q2.x * dz));
            const float qy = fmaf(q1.w, dx, fmaf(q1.y, dy, q2.y * dz));
            const float qz = fmaf(q2.x, dx, fmaf(q2.y, dy, q1.z * dz));
            const float dqd = fmaf(dx, qx, fmaf(dy, qy, dz * qz));
            const float u = rinv * rinv;
            const float r5 = rinv * u * u;
            const float b = 2.5f * dqd * r5 * u;
            tx = fmaf(b, dx, fmaf(-r5, qx, tx));
            ty = fmaf(b, dy, fmaf(-r5, qy, ty));
            tz = fmaf(b, dz, fmaf(-r5, qz, tz));
            tp = fmaf(-0.5f * dqd, r5, tp);
        }
    }
    nadd(acc.ax, acc.cx, tx); nadd(acc.ay, acc.cy, ty); nadd(acc.az, acc.cz, tz); nadd(acc.ph, acc.cp, tp);
}

// Work items 0 .. n_extra-1 are the extra particles (one-star groups whose box
// is their own grid cell [q, q+1)^3, q = floor((x - min) 2^21 / L) limited
// to +-2^23); the tree's groups follow.
template <bool SOFT, bool QUAD, bool REC, bool REL, bool SPL>
__global__ void RV_WALK_BOUNDS walk_tree_k(WalkArgs A) {
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // per-level opening thresholds in shared memory: lanes of a warp test cells
    // of different levels, which a constant-bank read would serialise
    __shared__ unsigned long long mac_thr[kLevels];
    __shared__ unsigned long long rec_thr[REC ? kLevels : 1];
    if (threadIdx.x < kLevels) mac_thr[threadIdx.x] = A.mac.thr[threadIdx.x];
    if (REC && threadIdx.x < kLevels) rec_thr[threadIdx.x] = A.rec.thr[threadIdx.x];
    __syncthreads();
    char *wsm = smem + wib * warp_smem_bytes(A.tile);
    const int nitem = A.n_extra + A.st->ngroup;
    unsigned long long np2p = 0, nm2p = 0;
    while (true) {
        int gi = 0;
        if (lane == 0) gi = atomicAdd(&A.st->next_group, 1);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= nitem) break;
        float *accw = reinterpret_cast<float *>(wsm + warp_staging_bytes(A.tile));
        const AccSm acc{accw + lane};
#pragma unroll
        for (int k = 0; k < 16; k++) accw[32 * k + lane] = 0.f;
        __syncwarp();
        unsigned long long a2 = 0, a3 = 0;
        if (gi < A.n_extra) {
            // ---- a particle outside the tree: all 32 lanes share its interaction list
            // (both target slots hold it; the second slot's sums are not used)
            const int kx = gi;
            const int mk = A.extra_per_member ? kx / A.extra_per_member : (A.xmem ? A.xmem[kx] : 0);
            const TreeGeo G = tree_geo(A, mk);
            const double *mb = A.mbounds + 5 * mk;
            float xi = A.xyzm[4 * kx], yi = A.xyzm[4 * kx + 1], zi = A.xyzm[4 * kx + 2];
            float ek = A.xeps[kx];
            float e = (ek == 0.f || A.eps_star == 0.f) ? 0.f : fmaxf(ek, A.eps_star);
            int blo[3], bhi[3];
            const float pv[3] = {xi, yi, zi};
            for (int a = 0; a < 3; a++) {
                double q = floor(__dmul_rn(__dsub_rn((double)pv[a], mb[a]), mb[4]));
                q = fmin(fmax(q, -8388608.0), 8388608.0);
                blo[a] = (int)q;
                bhi[a] = (int)q + 1;
            }
            float g[3];
            geo_centre(make_int4(blo[0], blo[1], blo[2], kMaxLevel), G.lo, G.unit, g);
            Tgt tg;
            tg.nx[0] = tg.nx[1] = f2_pack(g[0] - xi, g[0] - xi);
            tg.ny[0] = tg.ny[1] = f2_pack(g[1] - yi, g[1] - yi);
            tg.nz[0] = tg.nz[1] = f2_pack(g[2] - zi, g[2] - zi);
            tg.j0 = lane;
            tg.k = 32;
            bool ok = true;
            if (G.ncell > 0 && G.root >= 0)
                ok = walk_group<false, QUAD, false, false, false>(A, G, mac_thr, rec_thr, -1, wsm, blo, bhi, g, tg,
                                                           f2_pack(e * e, e * e), acc, a2, a3, -1.f);
            if (!ok) {
                if (lane == 0) latch_err(A.st, kErrStack);
                continue;
            }
            Acc tots[2];
            combine_shares(accw, 1, 1, 32, tots);
            Acc &tot = tots[0];
            if (lane == 0) {
                extra_terms(A, xi, yi, zi, ek, kx, mk, tot);
                A.xout[4 * kx] = tot.ax + tot.cx;
                A.xout[4 * kx + 1] = tot.ay + tot.cy;
                A.xout[4 * kx + 2] = tot.az + tot.cz;
                A.xout[4 * kx + 3] = tot.ph + tot.cp;
            }
            continue;
        }
        // ---- a group of the tree, in queue order (skipped when the mask says none of its stars is active)
        const int gk = A.order ? A.order[gi - A.n_extra] : gi - A.n_extra;
        if (A.gact && !A.gact[gk]) continue;
        const GroupRec grp = load_group(A.groups, gk);
        if (grp.first < 0 || grp.count < 1 || grp.count > kMaxGroup || grp.first + grp.count > A.n) {
            if (lane == 0) latch_err(A.st, kErrStack);
            continue;
        }
        const int mg = member_of(A.moff, A.M, grp.first);
        const TreeGeo G = tree_geo(A, mg);
        if (G.root < 0) {
            if (lane == 0) latch_err(A.st, kErrStack);
            continue;
        }
        const int *blo = grp.lo, *bhi = grp.hi;
        float g[3];
        box_centre(blo, bhi, G.lo, G.unit, g);
        // p target pairs (stars 2t, 2t + 1), k lanes per pair
        const int s = grp.count, p = (s + 1) >> 1, k = 32 / p;
        Tgt tg;
        {
            const int t = lane % p, sub = lane / p;
#pragma unroll
            for (int q = 0; q < 2; q++) {
                // an odd group's last pair repeats its star; those sums are not used
                const float4 pq = __ldg(&A.pos[grp.first + min(2 * t + q, s - 1)]);
                // minus the star's position relative to g (exact: FP32 negation)
                const float nx = -(pq.x - g[0]), ny = -(pq.y - g[1]), nz = -(pq.z - g[2]);
                tg.nx[q] = f2_pack(nx, nx);
                tg.ny[q] = f2_pack(ny, ny);
                tg.nz[q] = f2_pack(nz, nz);
            }
            tg.j0 = (sub < k) ? sub : (1 << 20);  // lanes beyond k p take no list pairs
            tg.k = k;
        }
        // relative criterion: K = (alpha |a|min) u^2 of the group, as in the oracle;
        // a group without a reference (|a|min = 0, no force pass yet) walks at theta (K < 0)
        float K = -1.f;
        if (REL) {
            float am = __int_as_float(0x7f800000);
            for (int i = lane; i < s; i += 32) {
                // |a| = sqrt((x x + y y) + z z) in FP32, one rounding per operation, as the oracle takes it
                const int j = A.perm[grp.first + i];
                const float x = A.arx[j], y = A.ary[j], z = A.arz[j];
                am = fminf(am, sqrtf(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z))));
            }
            for (int o = 16; o > 0; o >>= 1) am = fminf(am, __shfl_xor_sync(0xffffffffu, am, o));
            if (am > 0.f) K = __fmul_rn(__fmul_rn(A.rel_alpha, am), __fmul_rn(G.unit, G.unit));
        }
        bool ok = walk_group<SOFT, QUAD, REC, REL, SPL>(A, G, mac_thr, rec_thr, gk, wsm, blo, bhi, g, tg,
                                                   f2_pack(A.eps2, A.eps2), acc, a2, a3, K);
        if (!ok) {
            if (lane == 0) latch_err(A.st, kErrStack);
            continue;
        }
        np2p += a2 * (unsigned long long)s;
        nm2p += a3 * (unsigned long long)s;
        Acc tots[2];
        combine_shares(accw, s, p, k, tots);
        const float cost = (float)a2 + 2.5f * (float)a3;   // list pairs, a cell costing ~2.5 stars
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int i = lane + 32 * h;
            if (i >= s) continue;
            Acc &tot = tots[h];
            const float4 ps = __ldg(&A.pos[grp.first + i]);
            // the star's own pair was evaluated at r = 0: remove its -m/eps (the product
            // rounded on its own, as in the pair, so that the two cancel exactly)
            if (SOFT) tot.ph += __fmul_rn(ps.w, rsqrtf(A.eps2));
            int o = A.perm[grp.first + i];
            if (A.n_extra > 0) extra_terms(A, ps.x, ps.y, ps.z, A.eps_star, -1, mg, tot, !(A.xq_skip && A.xq_skip[o]));
            A.ax[o] = tot.ax + tot.cx;
            A.ay[o] = tot.ay + tot.cy;
            A.az[o] = tot.az + tot.cz;
            A.pot[o] = tot.ph + tot.cp;
            A.scost[o] = cost;
        }
    }
    if (lane == 0) {
        atomicAdd(&A.st->n_p2p, np2p);
        atomicAdd(&A.st->n_m2p, nm2p);
    }
}

// ---------------------------------------------------------------------------
// Queue order of the groups: most expensive first (longest-processing-time
// first: the walk's tail then holds the cheapest groups). The estimate is the
// list cost the last walk recorded for the group's first star, if that walk
// covered the same number of stars (st->cost_n); otherwise the volume of the
// group's box, smallest first (small boxes sit in dense regions with long
// lists). Groups are bucketed by log2 of the estimate (1/16 steps); the
// order within a bucket is unspecified. The forces do not depend on it.
constexpr int kOrderBins = 1024;   // the workspace's obins holds this many
constexpr int kOrderMinStars = 1 << 17;   // smaller systems walk their groups in build order

__device__ __forceinline__ int order_bin(const int4 *groups, const int *perm, const float *scost, int n, bool hist,
                                         int g) {
    const GroupRec r = load_group(groups, g);
    float lv;
    if (hist) {
        const int first = min(max(r.first, 0), n - 1);
        // any stored value is a finite estimate >= 1 here (NaN -> 1)
        const float c = fminf(fmaxf(scost[perm[first]], 1.f), 1e30f);
        lv = 64.f - log2f(c);   // descending cost (a cost above 2^64 shares the first bin)
    } else {
        lv = log2f((float)max(r.hi[0] - r.lo[0], 1)) + log2f((float)max(r.hi[1] - r.lo[1], 1)) +
             log2f((float)max(r.hi[2] - r.lo[2], 1));
    }
    return min(max((int)(16.f * lv), 0), kOrderBins - 1);
}

// (A) each group's bin, and the bin counts (bins zeroed before)
__global__ void group_bins_k(const int4 *groups, DevState *st, const int *perm, const float *scost, int n, int *gbin,
                             int *bins) {
    const int ng = st->ngroup;
    const bool hist = st->cost_n == n;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int b = order_bin(groups, perm, scost, n, hist, g);
        gbin[g] = b;
        atomicAdd(&bins[b], 1);
    }
}

// (B) exclusive scan of the bin counts, one bin per thread; the walk that
// follows records the costs of its stars
__global__ void __launch_bounds__(kOrderBins) group_bins_scan_k(DevState *st, int n, int *bins) {
    __shared__ int wsum[kOrderBins / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int v = bins[t];
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int x = wsum[lane];
        int sx = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, sx, o);
            if (lane >= o) sx += y;
        }
        wsum[lane] = sx - x;
    }
    __syncthreads();
    bins[t] = incl - v + wsum[w];
    if (t == 0) st->cost_n = n;
}

// (C) each group to its place: order[next free slot of its bin] = g
__global__ void group_scatter_k(const DevState *st, const int *gbin, int *bins, int *order) {
    const int ng = st->ngroup;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        order[atomicAdd(&bins[gbin[g]], 1)] = g;
}

// MAC thresholds: the smallest integer D with fl(theta^2 * D) > s^2 (FP64,
// theta^2 = theta * theta rounded once), so that "d^2 >= thr" is exactly the
// FP64 test s^2 < theta^2 d^2 on integer grid distances.
MacTable mac_table(float theta) {
    MacTable t;
    double th2 = (double)theta * (double)theta;
    for (int l = 0; l < kLevels; l++) {
        double s2 = ldexp(1.0, 2 * (kMaxLevel - l));
        if (!(th2 > 0.0)) { t.thr[l] = ~0ull; continue; }
        unsigned long long lo = 0, hi = 1ull << 53;
        if (!(th2 * (double)hi > s2)) { t.thr[l] = ~0ull; continue; }  // no grid distance can pass
        while (lo < hi) {
            unsigned long long mid = lo + (hi - lo) / 2;
            if (th2 * (double)mid > s2) hi = mid; else lo = mid + 1;
        }
        t.thr[l] = lo;
    }
    return t;
}

template <bool SOFT, bool QUAD, bool REC, bool REL = false, bool SPL = false>
static cudaError_t launch_walk(rv_ctx *c, const WalkArgs &A, cudaStream_t s) {
    size_t smem = warp_smem_bytes(A.tile) * kWalkWarps;
    auto kern = walk_tree_k<SOFT, QUAD, REC, REL, SPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalkWarps * 32, smem);
    if (e != cudaSuccess) return e;
    // every warp of the launch has its stack spill area
    int grid = std::min(std::max(1, per_sm) * c->num_sms, kStackSpillWarps / kWalkWarps);
    kern<<<grid, kWalkWarps * 32, smem, s>>>(A);
    count_launch(c);
    return cudaGetLastError();
}

rv_status tree_walk(rv_ctx *c, float theta, float eps_star, int n_extra, const float *xyzm, const float *xeps,
                    const int *xmem, int extras_per_member, float *ax, float *ay, float *az, float *pot,
                    float *xout, cudaStream_t s, const PairRecord *rec, const RelMac *rel, const uint8_t *gact,
                    const float4 *xquad, const uint8_t *xq_skip) {
    Workspace &w = c->w;
    WalkArgs A;
    A.pos = w.pos;
    A.cbox = w.cbox;
    A.clink = reinterpret_cast<const int4 *>(w.clink);
    A.cmom = w.cmom;
    A.groups = w.groups;
    A.perm = w.perm;
    A.st = w.st;
    A.cell_cap = (int)c->cell_cap;
    A.n = (int)c->n;
    A.moff = w.moff;
    A.M = c->n_members;
    A.mbounds = w.mbounds;
    A.mroot = w.mroot;
    A.xmem = xmem;
    A.extra_per_member = extras_per_member;
    A.mac = mac_table(theta);
    A.eps2 = eps_star * eps_star;
    A.eps_star = eps_star;
    A.tile = c->cfg.tile;
    A.n_extra = n_extra;
    A.xyzm = xyzm;
    A.xeps = xeps;
    A.xquad = n_extra > 0 ? xquad : nullptr;
    A.xq_skip = xq_skip;
    A.ax = ax; A.ay = ay; A.az = az; A.pot = pot;
    A.xout = xout;
    A.pairs = rec ? rec->pairs : nullptr;
    A.npairs = rec ? rec->npairs : nullptr;
    A.pair_cap = rec ? rec->cap : 0;
    if (rec) A.rec = mac_table(rec->theta_rec);
    A.gact = gact;
    A.gstack = w.gstack;
    // systems with fewer groups than resident walk warps gain nothing from an order
    A.order = c->n >= kOrderMinStars ? w.gorder : nullptr;
    A.scost = w.scost;
    const bool spline = c->cfg.softening == 1 && eps_star > 0.f;
    {
        const float h = 2.8f * eps_star;
        A.spl.h2 = h * h;
        A.spl.hinv = spline ? 1.f / h : 0.f;
        A.spl.hinv3 = A.spl.hinv * A.spl.hinv * A.spl.hinv;
    }
    A.rel_alpha = rel ? rel->alpha : 0.f;
    A.arx = rel ? rel->rx : nullptr;
    A.ary = rel ? rel->ry : nullptr;
    A.arz = rel ? rel->rz : nullptr;
    if (rel && rec) return set_err(c, RV_E_INVAL, "no pair record under the relative criterion");
    // reset the work counter and statistics (next_group, n_p2p, n_m2p)
    cudaError_t e = cudaMemsetAsync(&w.st->next_group, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&w.st->n_p2p, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_check(c, e, "walk reset");
    if (c->n == 0 && n_extra == 0) return RV_OK;
    const bool quad = c->cfg.quadrupole != 0;
    // optional timing of this launch on its own stream (not while a graph is being captured)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (c->profile_walk) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (cs == cudaStreamCaptureStatusNone) {
            if (c->n_walk_events == c->cap_walk_events) {
                int cap = c->cap_walk_events ? 2 * c->cap_walk_events : 64;
                cudaEvent_t *ev = (cudaEvent_t *)realloc(c->walk_events, sizeof(cudaEvent_t) * 2 * cap);
                if (!ev) return set_err(c, RV_E_CUDA, "walk timing events");
                for (int k = 2 * c->cap_walk_events; k < 2 * cap; k++) ev[k] = nullptr;
                c->walk_events = ev;
                c->cap_walk_events = cap;
            }
            cudaEvent_t *pair = c->walk_events + 2 * c->n_walk_events;
            if (!pair[0]) cudaEventCreate(&pair[0]);
            if (!pair[1]) cudaEventCreate(&pair[1]);
            ev0 = pair[0];
            ev1 = pair[1];
            c->n_walk_events++;
        }
    }
    if (ev0) cudaEventRecord(ev0, s);
    if (A.order) {
        int *bins = w.obins, *gbin = w.gbin;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((c->n + 255) / 256, (int64_t)c->num_sms * 4));
        e = cudaMemsetAsync(bins, 0, sizeof(int) * kOrderBins, s);
        if (e != cudaSuccess) return cuda_check(c, e, "walk order");
        group_bins_k<<<grid, 256, 0, s>>>(w.groups, w.st, w.perm, w.scost, (int)c->n, gbin, bins);
        group_bins_scan_k<<<1, kOrderBins, 0, s>>>(w.st, (int)c->n, bins);
        group_scatter_k<<<grid, 256, 0, s>>>(w.st, gbin, bins, w.gorder);
        c->launches += 3;
    }
    if (spline) {
        if (rec) return set_err(c, RV_E_INVAL, "no pair record with spline softening");
        if (rel)
            e = quad ? launch_walk<true, true, false, true, true>(c, A, s)
                     : launch_walk<true, false, false, true, true>(c, A, s);
        else
            e = quad ? launch_walk<true, true, false, false, true>(c, A, s)
                     : launch_walk<true, false, false, false, true>(c, A, s);
    } else if (rel) {
        if (eps_star > 0.f)
            e = quad ? launch_walk<true, true, false, true>(c, A, s) : launch_walk<true, false, false, true>(c, A, s);
        else
            e = quad ? launch_walk<false, true, false, true>(c, A, s) : launch_walk<false, false, false, true>(c, A, s);
    } else if (rec) {
        if (!(eps_star > 0.f) || !quad) return set_err(c, RV_E_INVAL, "pair record needs softening and quadrupoles");
        e = launch_walk<true, true, true>(c, A, s);
    } else if (eps_star > 0.f) {
        e = quad ? launch_walk<true, true, false>(c, A, s) : launch_walk<true, false, false>(c, A, s);
    } else {
        e = quad ? launch_walk<false, true, false>(c, A, s) : launch_walk<false, false, false>(c, A, s);
    }
    if (ev1) cudaEventRecord(ev1, s);
    if (e != cudaSuccess) return cuda_check(c, e, "walk launch");
    return RV_OK;
}

}  // namespace rv
